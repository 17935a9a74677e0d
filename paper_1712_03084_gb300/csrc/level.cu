// Iso-level L (Sec. III-B): the mean of A at the input sample positions.
//
// Every accepted point contributes the trilinear interpolation of A between
// its 8 surrounding cell-centred nodes (floor(t) .. floor(t) + 1, weights from
// t - floor(t)); accepted points are interior, so no clamping is needed.  The
// interpolation runs in float32 (A itself is float32); the sum over points
// runs in float64 with a fixed grid, a fixed per-thread order and a fixed
// reduction tree, so L is bit-reproducible run to run.
#include <cuda_runtime.h>

#include "ftr_internal.h"

namespace ftr {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kThreads / 32; ++w) s += sh[w];
    __syncthreads();
    return s;
}

__global__ void __launch_bounds__(kThreads) k_level_partial(GridDev g, const int4* __restrict__ pbase,
                                                            const float4* __restrict__ pfrac, int64_t n,
                                                            const float* __restrict__ A, double* part) {
    __shared__ double sh[kThreads / 32];
    const int nx = g.n[0];
    const int64_t nxy = (int64_t)nx * g.n[1];
    double sum = 0.0, cnt = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
        const int4 b = pbase[i];
        if (!(b.w & 1)) continue;
        const float4 fr = pfrac[i];
        const float fx = fr.x, fy = fr.y, fz = fr.z;
        const float* a0 = A + b.x + (int64_t)nx * b.y + nxy * b.z;
        // trilinear interpolation in float32; the sum over points in float64
        const float c00 = fmaf(fx, a0[1] - a0[0], a0[0]);
        const float c10 = fmaf(fx, a0[nx + 1] - a0[nx], a0[nx]);
        const float c01 = fmaf(fx, a0[nxy + 1] - a0[nxy], a0[nxy]);
        const float c11 = fmaf(fx, a0[nxy + nx + 1] - a0[nxy + nx], a0[nxy + nx]);
        const float c0 = fmaf(fy, c10 - c00, c00);
        const float c1 = fmaf(fy, c11 - c01, c01);
        sum += (double)fmaf(fz, c1 - c0, c0);
        cnt += 1.0;
    }
    const double s = block_sum(sum, sh);
    const double c = block_sum(cnt, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s;
        part[2 * blockIdx.x + 1] = c;
    }
}

// One warp: lane l sums partials l, l + 32, ... in order, then a fixed
// shuffle tree combines the lanes.
__global__ void k_level_final(const double* __restrict__ part, int nblocks, double* level, float* levelf) {
    const int lane = threadIdx.x;
    double s = 0.0, c = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
        s += part[2 * b];
        c += part[2 * b + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        const double L = c > 0.0 ? s / c : 0.0;
        level[0] = L;
        level[1] = c;
        levelf[0] = __double2float_ru(L);   // A >= L (float64) <=> A >= levelf[0] for float32 A
        levelf[1] = __double2float_rn(L);
    }
}

}  // namespace

cudaError_t launch_level(ftr_ctx* c) {
    k_level_partial<<<c->level_blocks, kThreads, 0, c->stream>>>(c->g, c->pts.base, c->pts.frac, c->n_pts, c->d_A,
                                                                 c->d_level_part);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_level_final<<<1, 32, 0, c->stream>>>(c->d_level_part, c->level_blocks, c->d_level, c->d_levelf);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace ftr
