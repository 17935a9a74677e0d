// Forward pass along x: real-to-complex transform of V_x, V_y, V_z rows.
//
// Sec. III-B transforms each component of V with a 3D FFT.  This first pass
// reads the splatted field straight from the brick pool (bricks no stencil
// touched are zero and are never read), transforms 16 rows (y0..y0+15, z) of
// the three components per CTA and writes the half spectra k_x = 0..n_x/2 in
// the layout [c][k_x][z][y] (y fastest), so that the next pass reads
// contiguous y lines.  Two real rows share one complex transform
// (z = a + i b, A = (Z[k] + conj Z[N-k]) / 2, B = (Z[k] - conj Z[N-k]) / 2i):
// 16 (V_x, V_y) pairs and 8 (V_z, V_z) pairs, 24 lines per CTA.  The x
// component is multiplied here by j w_x (numerator w_x = 0 at the Nyquist
// bin), which is all the filter needs from this axis.
#include "fft_common.cuh"
#include "ftr_internal.h"

namespace ftr {
namespace {

constexpr int kRows = 16;
constexpr int kLines = 24;

template <int N>
__global__ void __launch_bounds__(kLines * Xchg<N, kLines>::NT)
    k_fx(GridDev g, const int* __restrict__ slot_tab, const float* __restrict__ vpool, float2* __restrict__ s0,
         int64_t Mh, const float2* __restrict__ tw, float wx_scale, const int* __restrict__ meta) {
    pdl_wait();
    using X = Xchg<N, kLines>;
    constexpr int NB = N / kBrick;
    constexpr int NKX = N / 2 + 1;
    constexpr int ZS = kLines + 1;      // stride of the parked spectra
    extern __shared__ float2 smem[];
    __shared__ int s_slot[2][NB];
    __shared__ int s_any;
    const int ny = g.n[1], nz = g.n[2];
    const int y0 = blockIdx.x * kRows;
    const int z = blockIdx.y;
    const int tid = threadIdx.x;
    // z-planes outside the 16-aligned slab of touched bricks are never read
    // by the later passes: nothing to write there
    int zl, zh;
    live_z_range(meta, zl, zh);
    if (z < zl || z >= zh) return;
    if (tid == 0) s_any = 0;
    __syncthreads();
    const int bz = z >> 3;
    for (int k = tid; k < 2 * NB; k += blockDim.x) {
        const int r = k / NB, bx = k % NB;
        const int s = slot_tab[bx + g.nb[0] * ((y0 >> 3) + r + g.nb[1] * bz)];
        s_slot[r][bx] = s;
        if (s >= 0) s_any = 1;
    }
    __syncthreads();
    if (!s_any) {
        const float2 zero = make_float2(0.f, 0.f);
        for (int k = tid; k < kRows * NKX; k += blockDim.x) {
            const int r = k & (kRows - 1), kx = k >> 4;
            const size_t o = (size_t)(y0 + r) + (size_t)ny * (z + (size_t)nz * kx);
            s0[o] = zero;
            s0[Mh + o] = zero;
            s0[2 * Mh + o] = zero;
        }
        return;
    }
    const int f = tid / X::NT, r = tid % X::NT;
    const int lz = z & 7;
    if (r < X::N2) {
        const int ra = f < 16 ? f : f - 16;
        const int rb = f < 16 ? f : f - 8;
        const int ca = f < 16 ? 0 : 2;
        const int cb = f < 16 ? 1 : 2;
        float2 v[X::N1];
#pragma unroll
        for (int n1 = 0; n1 < X::N1; ++n1) {
            const int x = X::N2 * n1 + r;
            const int sa = s_slot[ra >> 3][x >> 3];
            const int sb = s_slot[rb >> 3][x >> 3];
            const int la = (x & 7) + 8 * ((ra & 7) + 8 * lz);
            const int lb = (x & 7) + 8 * ((rb & 7) + 8 * lz);
            const float a = sa >= 0 ? vpool[(size_t)sa * 3 * kBrickVox + ca * kBrickVox + la] : 0.f;
            const float b = sb >= 0 ? vpool[(size_t)sb * 3 * kBrickVox + cb * kBrickVox + lb] : 0.f;
            v[n1] = make_float2(a, b);
        }
        fft_step1<N, kLines, -1>(v, f, r, smem, tw);
    }
    __syncthreads();
    float2 o[X::N2];
    if (r < X::N1) fft_step2<N, kLines, -1>(o, f, r, smem);
    __syncthreads();
    if (r < X::N1) {
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) smem[f + ZS * (r + X::N1 * k2)] = o[k2];
    }
    __syncthreads();
    for (int k = tid; k < kRows * NKX; k += blockDim.x) {
        const int row = k & (kRows - 1), kx = k >> 4;
        const int km = kx == 0 ? 0 : N - kx;
        const float2 za = smem[row + ZS * kx];
        const float2 zb = cconj(smem[row + ZS * km]);
        float2 vx = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y + zb.y));
        const float2 dy = csub(za, zb);
        const float2 vy = make_float2(0.5f * dy.y, -0.5f * dy.x);
        const int fz = 16 + (row & 7);
        const float2 zc = smem[fz + ZS * kx];
        const float2 zd = cconj(smem[fz + ZS * km]);
        float2 vz;
        if (row < 8) {
            vz = make_float2(0.5f * (zc.x + zd.x), 0.5f * (zc.y + zd.y));
        } else {
            const float2 dz = csub(zc, zd);
            vz = make_float2(0.5f * dz.y, -0.5f * dz.x);
        }
        const float wx = (kx == N / 2) ? 0.f : wx_scale * (float)kx;   // j w_x, Nyquist numerator 0
        vx = make_float2(-wx * vx.y, wx * vx.x);
        const size_t oi = (size_t)(y0 + row) + (size_t)ny * (z + (size_t)nz * kx);
        s0[oi] = vx;
        s0[Mh + oi] = vy;
        s0[2 * Mh + oi] = vz;
    }
}

template <int N>
cudaError_t run_fx(ftr_ctx* c) {
    using X = Xchg<N, kLines>;
    const size_t smem = sizeof(float2) * X::SIZE;
    static bool attr_done[64] = {};
    if (!attr_done[c->device & 63]) {
        cudaError_t e = cudaFuncSetAttribute(k_fx<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done[c->device & 63] = true;
    }
    dim3 grid(c->g.n[1] / kRows, c->g.n[2]);
    const float wx_scale = (float)(2.0 * 3.14159265358979323846 / (c->g.n[0] * c->g.h[0]));
    launch_pdl(k_fx<N>, grid, kLines * X::NT, smem, c->stream, c->g, c->d_brick_slot, c->d_vpool, c->d_s0, c->Mh,
                                                       c->d_tw[0], wx_scale, c->d_meta);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace

cudaError_t fft_fx_init(const float2* w96) { return upload_w96_table(w96); }

cudaError_t launch_fx(ftr_ctx* c) {
    if (c->p.precision != FTR_PREC_FP32) return launch_tc_pass(c, 0);
    switch (c->g.n[0]) {
        case 32: return run_fx<32>(c);
        case 48: return run_fx<48>(c);
        case 64: return run_fx<64>(c);
        case 96: return run_fx<96>(c);
        case 128: return run_fx<128>(c);
        case 192: return run_fx<192>(c);
        case 256: return run_fx<256>(c);
        case 384: return run_fx<384>(c);
        case 512: return run_fx<512>(c);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ftr
