// Inverse pass along y (Sec. III-B inverse 3D FFT, second axis).
//
// Input: A^ transformed back along z, layout [k_x][k_y][z] (z fastest).  A CTA
// takes 16 consecutive z at one k_x (contiguous 128-byte rows for every k_y),
// transforms them along y and writes [k_x][z][y] (y fastest) for the final
// complex-to-real x pass.
#include "fft_common.cuh"
#include "ftr_internal.h"

namespace ftr {
namespace {

// F lines per CTA (the tile plan; 8, 16 or 32).
template <int N, int F>
__global__ void __launch_bounds__(F * Xchg<N, F>::NT)
    k_iy(GridDev g, const float2* __restrict__ src, float2* __restrict__ dst, const float2* __restrict__ tw) {
    pdl_wait();
    using X = Xchg<N, F>;
    extern __shared__ float2 smem[];
    const int nz = g.n[2];
    const int z0 = blockIdx.x * F;
    const int kx = blockIdx.y;
    const int tid = threadIdx.x;
    const uint64_t pin = l2_evict_first(), pout = l2_evict_last();
    // step 1: line index fastest (the input is contiguous along z)
    const int f1 = tid % F, j1 = tid / F;
    if (j1 < X::N2) {
        float2 v[X::N1];
#pragma unroll
        for (int n1 = 0; n1 < X::N1; ++n1) {
            const int ky = X::N2 * n1 + j1;
            v[n1] = ld_l2hint(src + (size_t)(z0 + f1) + (size_t)nz * ((size_t)ky + (size_t)N * kx), pin);
        }
        fft_step1<N, F, +1>(v, f1, j1, smem, tw);
    }
    __syncthreads();
    // step 2: element index fastest (the output is contiguous along y)
    const int f2 = tid / X::NT, i2 = tid % X::NT;
    if (i2 < X::N1) {
        float2 o[X::N2];
        fft_step2<N, F, +1>(o, f2, i2, smem);
        float2* out = dst + (size_t)N * ((size_t)(z0 + f2) + (size_t)nz * kx);
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) st_l2hint(out + i2 + X::N1 * k2, o[k2], pout);
    }
}

template <int N, int F>
cudaError_t run_iy_f(ftr_ctx* c) {
    using X = Xchg<N, F>;
    const size_t smem = sizeof(float2) * X::SIZE;
    cudaError_t e = ensure_smem(k_iy<N, F>, smem, c->device);
    if (e != cudaSuccess) return e;
    if (c->occ_query)   // the autotuner asks how many CTAs of this plan fit on an SM
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(c->occ_query, k_iy<N, F>, F * X::NT, smem);
    dim3 grid(c->g.n[2] / F, c->g.n[0] / 2 + 1);
    launch_pdl(k_iy<N, F>, grid, F * X::NT, smem, c->stream, c->g, c->d_s1, c->d_s0, c->d_tw[1]);
    c->launches++;
    return cudaGetLastError();
}

template <int N>
cudaError_t run_iy(ftr_ctx* c) {
    switch (c->plan_lines[2]) {
        case 8: return run_iy_f<N, 8>(c);
        case 32: return run_iy_f<N, 32>(c);
        default: return run_iy_f<N, 16>(c);
    }
}

}  // namespace

cudaError_t fft_iy_init(const float2* w96) { return upload_w96_table(w96); }

cudaError_t launch_iy(ftr_ctx* c) {
    if (c->p.precision != FTR_PREC_FP32) return launch_tc_pass(c, 3);
    switch (c->g.n[1]) {
        case 32: return run_iy<32>(c);
        case 48: return run_iy<48>(c);
        case 64: return run_iy<64>(c);
        case 96: return run_iy<96>(c);
        case 128: return run_iy<128>(c);
        case 192: return run_iy<192>(c);
        case 256: return run_iy<256>(c);
        case 384: return run_iy<384>(c);
        case 512: return run_iy<512>(c);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ftr
