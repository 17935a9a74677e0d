// Forward pass along y, with the x and y terms of the filter combined.
//
// Input: the x-pass half spectra [c][k_x][z][y] (j w_x already applied to
// c = x).  Each CTA transforms 16 contiguous y lines (z0..z0+15 at one k_x)
// of the three components.  Because the integration filter of Sec. III-B is
// j (w . V^) / |w|^2 and w_y depends only on k_y, the x and y components can
// be summed as soon as both are transformed along y:
//   W(k_x, k_y, z) = Y[j w_x X V_x] + j w_y Y[X V_y]      (numerator w_y = 0 at Nyquist)
// so only two fields leave this pass: W and Y[X V_z], both in the layout
// [k_x][k_y][z] (z fastest) for the z pass.
#include "fft_common.cuh"
#include "ftr_internal.h"
#include "tc_sm100.cuh"

namespace ftr {
namespace {

// Load line f's elements y = N2 n1 + r (contiguous) and run step 1.
template <int N, int F>
__device__ __forceinline__ void load_step1(const float2* __restrict__ src, int r, int f, float2* smem,
                                           const float2* __restrict__ tw, uint64_t pol) {
    using X = Xchg<N, F>;
    float2 v[X::N1];
#pragma unroll
    for (int n1 = 0; n1 < X::N1; ++n1) v[n1] = ld_l2hint(src + X::N2 * n1 + r, pol);
    fft_step1<N, F, -1>(v, f, r, smem, tw);
}

// F lines per CTA (the tile plan; 8, 16 or 32).
template <int N, int F>
__global__ void __launch_bounds__(F * Xchg<N, F>::NT, MinCtasF<N, F>::value)
    k_fy(GridDev g, const float2* __restrict__ s0, float2* __restrict__ s1, int64_t Mh,
         const float2* __restrict__ tw, float wy_scale, const int* __restrict__ meta) {
    pdl_wait();
    using X = Xchg<N, F>;
    extern __shared__ float2 smem[];
    const int nz = g.n[2];
    const int z0 = blockIdx.x * F;
    const int kx = blockIdx.y;
    const int tid = threadIdx.x;
    // tiles outside the slab of touched bricks are zero; the z pass treats
    // them as zero without reading, so nothing is read or written here (a
    // tile that straddles the slab edge is transformed whole: its lines
    // outside the slab are never read by the z pass)
    int zl, zh;
    live_z_range(meta, zl, zh);
    if (z0 + F <= zl || z0 >= zh) return;
    // step-1 mapping: element index fastest (contiguous y lines)
    const int f1 = tid / X::NT, r1 = tid % X::NT;
    // step-2 mapping: line index fastest (contiguous z in the output)
    const int f2 = tid % F, i2 = tid / F;
    const size_t out_base = (size_t)(z0 + f2) + (size_t)nz * ((size_t)N * kx);
    // the transformed x component waits in shared memory (line index fastest)
    float2* stash = smem + X::SIZE;
    const float2* line = s0 + (size_t)N * (z0 + f1 + (size_t)nz * kx);
    // the y and z components' lines go to L2 while the x component is
    // transformed (one prefetch per 128-byte line per thread)
    if (r1 < X::N2 && (r1 & 15) == 0) {
#pragma unroll
        for (int n1 = 0; n1 < X::N1; ++n1) {
            prefetch_l2(line + Mh + X::N2 * n1 + r1);
            prefetch_l2(line + 2 * Mh + X::N2 * n1 + r1);
        }
    }
    const uint64_t pin = l2_evict_first(), pout = l2_evict_last();
    // x component: transform along y and park it (line index fastest)
    if (r1 < X::N2) load_step1<N, F>(line, r1, f1, smem, tw, pin);
    __syncthreads();
    float2 o[X::N2];
    if (i2 < X::N1) fft_step2<N, F, -1>(o, f2, i2, smem);
    __syncthreads();
    if (i2 < X::N1) {
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) stash[f2 + (F + 1) * (i2 + X::N1 * k2)] = o[k2];
    }
    // y component: transform, then W = x + j w_y y goes out as field 0
    if (r1 < X::N2) load_step1<N, F>(line + Mh, r1, f1, smem, tw, pin);
    __syncthreads();
    if (i2 < X::N1) fft_step2<N, F, -1>(o, f2, i2, smem);
    __syncthreads();
    if (i2 < X::N1) {
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) {
            const int ky = i2 + X::N1 * k2;
            const float wy = (ky == N / 2) ? 0.f : wy_scale * (float)signed_bin(ky, N);
            const float2 w = stash[f2 + (F + 1) * ky];
            st_l2hint(s1 + out_base + (size_t)nz * ky, make_float2(w.x - wy * o[k2].y, w.y + wy * o[k2].x), pout);
        }
    }
    // z component: transform and write as field 1
    if (r1 < X::N2) load_step1<N, F>(line + 2 * Mh, r1, f1, smem, tw, pin);
    __syncthreads();
    if (i2 < X::N1) {
        fft_step2<N, F, -1>(o, f2, i2, smem);
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) st_l2hint(s1 + Mh + out_base + (size_t)nz * (i2 + X::N1 * k2), o[k2], pout);
    }
}

// The same pass with the CTA's three component tiles (16 lines each, one
// contiguous block per component) fetched by bulk asynchronous copies at
// the start, so that all of its input is in flight at once; each tile's
// buffer then serves as that component's exchange buffer, and the x
// component's as the stash.  Waits are bounded (a timeout sets *err).
template <int N>
__global__ void __launch_bounds__(16 * Xchg<N, 16>::NT, 2)
    k_fy_bulk(GridDev g, const float2* __restrict__ s0, float2* __restrict__ s1, int64_t Mh,
              const float2* __restrict__ tw, float wy_scale, const int* __restrict__ meta, int* err) {
    pdl_wait();
    constexpr int F = 16;
    using X = Xchg<N, F>;
    constexpr int BUF = cmax(X::SIZE, (F + 1) * N);
    constexpr uint32_t kBytes = F * N * sizeof(float2);
    extern __shared__ __align__(16) float2 smem[];
    __shared__ uint64_t mbar[3];
    const int nz = g.n[2];
    const int z0 = blockIdx.x * F;
    const int kx = blockIdx.y;
    const int tid = threadIdx.x;
    int zl, zh;
    live_z_range(meta, zl, zh);
    if (z0 + F <= zl || z0 >= zh) return;
    const size_t tile = (size_t)N * ((size_t)z0 + (size_t)nz * kx);
    if (tid == 0) {
        for (int c = 0; c < 3; ++c) tc::mbar_init(&mbar[c], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int c = 0; c < 3; ++c) {
            tc::mbar_expect_tx(&mbar[c], kBytes);
            tc::bulk_g2s(smem + c * BUF, s0 + (size_t)c * Mh + tile, kBytes, &mbar[c]);
        }
    }
    __syncthreads();
    const int f1 = tid / X::NT, r1 = tid % X::NT;
    const int f2 = tid % F, i2 = tid / F;
    const size_t out_base = (size_t)(z0 + f2) + (size_t)nz * ((size_t)N * kx);
    float2* stash = smem;                      // the x component's buffer, once its exchange is done
    float2 o[X::N2];
    for (int c = 0; c < 3; ++c) {
        float2* B = smem + c * BUF;
        if (!tc::mbar_wait(&mbar[c], 0, 1u << 22)) atomicExch(err, 1);
        float2 v[X::N1];
        if (r1 < X::N2) {
#pragma unroll
            for (int n1 = 0; n1 < X::N1; ++n1) v[n1] = B[f1 * N + X::N2 * n1 + r1];
        }
        __syncthreads();                       // the staged lines are in registers: B becomes the exchange
        if (r1 < X::N2) fft_step1<N, F, -1>(v, f1, r1, B, tw);
        __syncthreads();
        if (i2 < X::N1) fft_step2<N, F, -1>(o, f2, i2, B);
        if (c == 0) {
            __syncthreads();                   // every exchange read done: B becomes the stash
            if (i2 < X::N1) {
#pragma unroll
                for (int k2 = 0; k2 < X::N2; ++k2) stash[f2 + (F + 1) * (i2 + X::N1 * k2)] = o[k2];
            }
        } else if (c == 1) {
            if (i2 < X::N1) {
#pragma unroll
                for (int k2 = 0; k2 < X::N2; ++k2) {
                    const int ky = i2 + X::N1 * k2;
                    const float wy = (ky == N / 2) ? 0.f : wy_scale * (float)signed_bin(ky, N);
                    const float2 w = stash[f2 + (F + 1) * ky];
                    s1[out_base + (size_t)nz * ky] = make_float2(w.x - wy * o[k2].y, w.y + wy * o[k2].x);
                }
            }
        } else {
            if (i2 < X::N1) {
#pragma unroll
                for (int k2 = 0; k2 < X::N2; ++k2) s1[Mh + out_base + (size_t)nz * (i2 + X::N1 * k2)] = o[k2];
            }
        }
    }
}

template <int N>
cudaError_t run_fy_bulk(ftr_ctx* c) {
    using X = Xchg<N, 16>;
    const size_t smem = sizeof(float2) * 3 * cmax(X::SIZE, 17 * N);
    cudaError_t e = ensure_smem(k_fy_bulk<N>, smem, c->device);
    if (e != cudaSuccess) return e;
    if (c->occ_query) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(c->occ_query, k_fy_bulk<N>, 16 * X::NT, smem);
    dim3 grid(c->g.n[2] / 16, c->g.n[0] / 2 + 1);
    const float wy_scale = (float)(2.0 * 3.14159265358979323846 / (c->g.n[1] * c->g.h[1]));
    launch_pdl(k_fy_bulk<N>, grid, 16 * X::NT, smem, c->stream, c->g, c->d_s0, c->d_s1, c->Mh, c->d_tw[1], wy_scale,
               c->d_meta, c->d_kerr);
    c->launches++;
    return cudaGetLastError();
}

template <int N, int F>
cudaError_t run_fy_f(ftr_ctx* c) {
    using X = Xchg<N, F>;
    const size_t smem = sizeof(float2) * (X::SIZE + (F + 1) * N);
    cudaError_t e = ensure_smem(k_fy<N, F>, smem, c->device);
    if (e != cudaSuccess) return e;
    if (c->occ_query)   // the autotuner asks how many CTAs of this plan fit on an SM
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(c->occ_query, k_fy<N, F>, F * X::NT, smem);
    dim3 grid(c->g.n[2] / F, c->g.n[0] / 2 + 1);
    const float wy_scale = (float)(2.0 * 3.14159265358979323846 / (c->g.n[1] * c->g.h[1]));
    launch_pdl(k_fy<N, F>, grid, F * X::NT, smem, c->stream, c->g, c->d_s0, c->d_s1, c->Mh, c->d_tw[1], wy_scale,
                                                       c->d_meta);
    c->launches++;
    return cudaGetLastError();
}

template <int N>
cudaError_t run_fy(ftr_ctx* c) {
    switch (c->plan_lines[0]) {
        case 8: return run_fy_f<N, 8>(c);
        case 32: return run_fy_f<N, 32>(c);
        case -16:
            if (N <= 256) return run_fy_bulk<N>(c);
            return run_fy_f<N, 16>(c);
        default: return run_fy_f<N, 16>(c);
    }
}

}  // namespace

cudaError_t fft_fy_init(const float2* w96) { return upload_w96_table(w96); }

cudaError_t launch_fy(ftr_ctx* c) {
    if (c->p.precision != FTR_PREC_FP32) return launch_tc_pass(c, 1);
    switch (c->g.n[1]) {
        case 32: return run_fy<32>(c);
        case 48: return run_fy<48>(c);
        case 64: return run_fy<64>(c);
        case 96: return run_fy<96>(c);
        case 128: return run_fy<128>(c);
        case 192: return run_fy<192>(c);
        case 256: return run_fy<256>(c);
        case 384: return run_fy<384>(c);
        case 512: return run_fy<512>(c);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ftr
