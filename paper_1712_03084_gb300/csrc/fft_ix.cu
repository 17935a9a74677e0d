// Inverse pass along x: complex-to-real transform into the indicator A.
//
// Last axis of the inverse 3D FFT of Sec. III-B.  Input [k_x][z][y] half
// spectra (k_x = 0..n_x/2); a CTA stages 16 rows (y0..y0+15, z) in shared
// memory and runs two real rows per complex inverse transform: with the
// Hermitian extension X[n-k] = conj X[k], Z = X_a + i X_b gives
// IDFT(Z) = x_a + i x_b.  The imaginary parts of the k_x = 0 and k_x = n_x/2
// bins are dropped (they are zero for an exactly Hermitian spectrum).  The
// 1/M normalisation was applied in the z pass.  Output: A[z][y][x], and per
// grid row (y + n_y z) the minimum and maximum of the values written (NaN
// for both if the row holds a NaN), from which the marching cubes fill rows
// that lie wholly on one side of the level without reading them.
#include "fft_common.cuh"
#include "ftr_internal.h"

namespace ftr {
namespace {

constexpr int kRows = 16;
constexpr int kLines = 8;     // complex transforms per CTA (row pairs r, r + 8)
constexpr int kHs = kRows + 1;

template <int N>
__global__ void __launch_bounds__(kLines * Xchg<N, kLines>::NT)
    k_ix(GridDev g, const float2* __restrict__ src, float* __restrict__ A, const float2* __restrict__ tw,
         float2* __restrict__ rowmm) {
    pdl_wait();
    __shared__ float2 s_mm[kRows][Xchg<N, kLines>::NT];
    using X = Xchg<N, kLines>;
    constexpr int NKX = N / 2 + 1;
    extern __shared__ float2 smem[];
    float2* hs = smem + X::SIZE;            // staged half spectra, [k_x][row]
    const int ny = g.n[1], nz = g.n[2];
    const int y0 = blockIdx.x * kRows;
    const int z = blockIdx.y;
    const int tid = threadIdx.x;
    const uint64_t pin = l2_evict_first(), pout = l2_evict_last();
    // every load of the staging is issued before the first shared-memory store
    constexpr int kPer = (kRows * NKX + kLines * Xchg<N, kLines>::NT - 1) / (kLines * Xchg<N, kLines>::NT);
    {
        float2 st[kPer];
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int k = tid + i * (int)blockDim.x;
            const int row = k & (kRows - 1), kx = k >> 4;
            st[i] = k < kRows * NKX ? ld_l2hint(src + (size_t)(y0 + row) + (size_t)ny * (z + (size_t)nz * kx), pin)
                                    : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < kPer; ++i) {
            const int k = tid + i * (int)blockDim.x;
            if (k < kRows * NKX) hs[(k >> 4) * kHs + (k & (kRows - 1))] = st[i];
        }
    }
    __syncthreads();
    const int f1 = tid % kLines, j1 = tid / kLines;
    if (j1 < X::N2) {
        const int ra = f1, rb = f1 + kLines;
        float2 v[X::N1];
#pragma unroll
        for (int n1 = 0; n1 < X::N1; ++n1) {
            const int k = X::N2 * n1 + j1;
            float2 xa, xb;
            if (k <= N / 2) {
                xa = hs[k * kHs + ra];
                xb = hs[k * kHs + rb];
                if (k == 0 || k == N / 2) {
                    xa.y = 0.f;
                    xb.y = 0.f;
                }
            } else {
                xa = cconj(hs[(N - k) * kHs + ra]);
                xb = cconj(hs[(N - k) * kHs + rb]);
            }
            v[n1] = make_float2(xa.x - xb.y, xa.y + xb.x);
        }
        fft_step1<N, kLines, +1>(v, f1, j1, smem, tw);
    }
    __syncthreads();
    const int f2 = tid / X::NT, i2 = tid % X::NT;
    if (i2 < X::N1) {
        float2 o[X::N2];
        fft_step2<N, kLines, +1>(o, f2, i2, smem);
        float* ra = A + (size_t)N * ((size_t)(y0 + f2) + (size_t)ny * z);
        float* rb = A + (size_t)N * ((size_t)(y0 + f2 + kLines) + (size_t)ny * z);
        float mna = INFINITY, mxa = -INFINITY, mnb = INFINITY, mxb = -INFINITY;
        bool nan = false;
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) {
            st_l2hint(ra + i2 + X::N1 * k2, o[k2].x, pout);
            st_l2hint(rb + i2 + X::N1 * k2, o[k2].y, pout);
            mna = fminf(mna, o[k2].x);
            mxa = fmaxf(mxa, o[k2].x);
            mnb = fminf(mnb, o[k2].y);
            mxb = fmaxf(mxb, o[k2].y);
            nan |= (o[k2].x != o[k2].x) | (o[k2].y != o[k2].y);
        }
        if (nan) mna = mxa = mnb = mxb = NAN;     // NaN bounds: the row is read in full
        s_mm[f2][i2] = make_float2(mna, mxa);
        s_mm[f2 + kLines][i2] = make_float2(mnb, mxb);
    }
    __syncthreads();
    if (tid < kRows) {
        float mn = INFINITY, mx = -INFINITY;
        bool nan = false;
#pragma unroll
        for (int i = 0; i < X::N1; ++i) {
            const float2 m = s_mm[tid][i];
            nan |= m.x != m.x;
            mn = fminf(mn, m.x);
            mx = fmaxf(mx, m.y);
        }
        rowmm[(size_t)(y0 + tid) + (size_t)ny * z] = nan ? make_float2(NAN, NAN) : make_float2(mn, mx);
    }
}

template <int N>
cudaError_t run_ix(ftr_ctx* c) {
    using X = Xchg<N, kLines>;
    const size_t smem = sizeof(float2) * (X::SIZE + kHs * (N / 2 + 1));
    static bool attr_done[64] = {};
    if (!attr_done[c->device & 63]) {
        cudaError_t e = cudaFuncSetAttribute(k_ix<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done[c->device & 63] = true;
    }
    dim3 grid(c->g.n[1] / kRows, c->g.n[2]);
    launch_pdl(k_ix<N>, grid, kLines * X::NT, smem, c->stream, c->g, c->d_s0, c->d_A, c->d_tw[0], c->d_rowmm);
    c->launches++;
    c->rowmm_valid = true;
    return cudaGetLastError();
}

}  // namespace

cudaError_t fft_ix_init(const float2* w96) { return upload_w96_table(w96); }

cudaError_t launch_ix(ftr_ctx* c) {
    if (c->p.precision != FTR_PREC_FP32) {
        c->rowmm_valid = false;   // the tensor-core x inverse writes no row bounds
        return launch_tc_pass(c, 4);
    }
    switch (c->g.n[0]) {
        case 32: return run_ix<32>(c);
        case 48: return run_ix<48>(c);
        case 64: return run_ix<64>(c);
        case 96: return run_ix<96>(c);
        case 128: return run_ix<128>(c);
        case 192: return run_ix<192>(c);
        case 256: return run_ix<256>(c);
        case 384: return run_ix<384>(c);
        case 512: return run_ix<512>(c);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ftr
