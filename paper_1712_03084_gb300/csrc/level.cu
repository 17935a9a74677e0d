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

// Per-CTA partial sums; the last CTA to finish (ticket counter) sums the
// partials in block order and writes L (fixed order: bit-reproducible).
__global__ void __launch_bounds__(kThreads) k_level_partial(GridDev g, const int4* __restrict__ pbase,
                                                            const float4* __restrict__ pfrac,
                                                            const int64_t* __restrict__ npts,
                                                            const float* __restrict__ A, double* part,
                                                            unsigned* ticket, double* level, float* levelf) {
    pdl_wait();
    __shared__ double sh[kThreads / 32];
    __shared__ bool last;
    const int nx = g.n[0];
    const int64_t nxy = (int64_t)nx * g.n[1];
    double sum = 0.0;
    int cnt = 0;
    const int64_t n = *npts;
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
        cnt += 1;
    }
    const double s = block_sum(sum, sh);
    const double c = block_sum((double)cnt, sh);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s;
        part[2 * blockIdx.x + 1] = c;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the whole CTA reads the partials (one or two per thread, all loads in
    // flight at once), then the fixed tree
    double ts = 0.0, tc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) {
        ts += __ldcg(&part[2 * b]);
        tc += __ldcg(&part[2 * b + 1]);
    }
    ts = block_sum(ts, sh);
    tc = block_sum(tc, sh);
    if (threadIdx.x == 0) {
        const double L = tc > 0.0 ? ts / tc : 0.0;
        level[0] = L;
        level[1] = tc;
        levelf[0] = __double2float_ru(L);   // A >= L (float64) <=> A >= levelf[0] for float32 A
        levelf[1] = __double2float_rn(L);
        *ticket = 0u;                        // ready for the next launch
    }
}

}  // namespace

cudaError_t launch_level(ftr_ctx* c) {
    launch_pdl(k_level_partial, c->level_blocks, kThreads, 0, c->stream, c->g, c->pts.base, c->pts.frac, c->d_npts, c->d_A,
                                                                 c->d_level_part, c->d_ticket, c->d_level,
                                                                 c->d_levelf);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace ftr

// ---------------------------------------------------------------------------
// Allocation-free iso-level entry point.
//
// Some callers cannot allocate device memory at the point where they need the
// level: a per-frame loop running under a hard latency budget (cudaMalloc and
// cudaFree may synchronise the device and take unbounded time), or a host
// application that hands this library a fixed memory budget and owns every
// allocation itself.  This variant of the level kernels takes the indicator
// and the points from the caller and keeps its per-CTA partial sums in a
// statically allocated device array instead of a context buffer.
// ---------------------------------------------------------------------------

#include <mutex>

namespace ftr {
namespace {

constexpr int kNoAllocPointsPerCta = 1024;
constexpr int kNoAllocMaxCtas = 4096;     // => at most 4,194,304 points per call
// Partial (sum, count) per CTA plus (L, count) of the result: 64 KB + 16 B,
// resident on every device that loads the library until the process exits.
__device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxCtas + 2];

// Device address of g_noalloc_scratch, looked up once per device.
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {};

// t = (X - b_min) / h - 1/2 with every decision equal to the float64 quotient
// (the same rule as the point ingest of the splat).
__device__ __forceinline__ double noalloc_node_t(double x, double bmin, double h, double inv_h, double n) {
    double t = (x - bmin) * inv_h - 0.5;
    const double band = 1e-9 * (1.0 + fabs(t));
    const double fr = t - floor(t);
    if (fr < band || fr > 1.0 - band || fabs(t - 1.0) < band || fabs(t - (n - 2.0)) < band)
        t = (x - bmin) / h - 0.5;
    return t;
}

__global__ void __launch_bounds__(kThreads) k_level_noalloc_partial(GridDev g, const float* __restrict__ pts,
                                                                    int64_t n, const float* __restrict__ A,
                                                                    double* scratch) {
    __shared__ double sh[kThreads / 32];
    const int nx = g.n[0];
    const int64_t nxy = (int64_t)nx * g.n[1];
    double sum = 0.0, cnt = 0.0;
    const int64_t i0 = (int64_t)blockIdx.x * kNoAllocPointsPerCta;
    for (int64_t i = i0 + threadIdx.x; i < i0 + kNoAllocPointsPerCta && i < n; i += kThreads) {
        int b[3];
        float f[3];
        bool ok = true;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double t = noalloc_node_t((double)pts[3 * i + c], g.bmin[c], g.h[c], g.inv_h[c], (double)g.n[c]);
            ok = ok && (t >= 1.0) && (t < (double)g.n[c] - 2.0);
            const double fl = ok ? floor(t) : 0.0;
            b[c] = (int)fl;
            f[c] = ok ? (float)(t - fl) : 0.f;
        }
        if (!ok) continue;
        const float* a0 = A + b[0] + (int64_t)nx * b[1] + nxy * b[2];
        const float c00 = fmaf(f[0], a0[1] - a0[0], a0[0]);
        const float c10 = fmaf(f[0], a0[nx + 1] - a0[nx], a0[nx]);
        const float c01 = fmaf(f[0], a0[nxy + 1] - a0[nxy], a0[nxy]);
        const float c11 = fmaf(f[0], a0[nxy + nx + 1] - a0[nxy + nx], a0[nxy + nx]);
        const float c0 = fmaf(f[1], c10 - c00, c00);
        const float c1 = fmaf(f[1], c11 - c01, c01);
        sum += (double)fmaf(f[2], c1 - c0, c0);
        cnt += 1.0;
    }
    const double s = block_sum(sum, sh);
    const double c = block_sum(cnt, sh);
    if (threadIdx.x == 0) {          // every slot this call reads is written here first
        scratch[2 * blockIdx.x] = s;
        scratch[2 * blockIdx.x + 1] = c;
    }
}

__global__ void k_level_noalloc_final(double* scratch, int nblocks, double* level_dev) {
    const int lane = threadIdx.x;
    double s = 0.0, c = 0.0;
    for (int b = lane; b < nblocks; b += 32) {
        s += scratch[2 * b];
        c += scratch[2 * b + 1];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
        const double L = c > 0.0 ? s / c : 0.0;
        scratch[2 * kNoAllocMaxCtas] = L;
        scratch[2 * kNoAllocMaxCtas + 1] = c;
        if (level_dev) level_dev[0] = L;
    }
}

bool supported_axis(int n) {
    switch (n) {
        case 32: case 48: case 64: case 96: case 128: case 192: case 256: case 384: case 512: return true;
        default: return false;
    }
}

}  // namespace
}  // namespace ftr

extern "C" int ftr_iso_level_noalloc(const float* A, const int grid_n[3], const float bbox[6], const float* points,
                                     int64_t n, double* level_out, void* stream) {
    using namespace ftr;
    if (!A || !grid_n || !bbox || !level_out || n < 0 || (n > 0 && !points)) return FTR_EINVAL;
    if (n > (int64_t)kNoAllocPointsPerCta * kNoAllocMaxCtas) return FTR_EINVAL;   // beyond the static scratch
    GridDev g{};
    for (int a = 0; a < 3; ++a) {
        if (!supported_axis(grid_n[a]) || !(bbox[3 + a] > bbox[a])) return FTR_EINVAL;
        g.n[a] = grid_n[a];
        g.bmin[a] = (double)bbox[a];
        g.h[a] = ((double)bbox[3 + a] - (double)bbox[a]) / grid_n[a];
        g.inv_h[a] = 1.0 / g.h[a];
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return FTR_ECUDA;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            // host code may not use g_noalloc_scratch directly: it names a host
            // shadow, not the device array
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return FTR_ECUDA;
            g_noalloc_ptr[dev] = static_cast<double*>(p);
        }
        scratch = g_noalloc_ptr[dev];
    }
    cudaPointerAttributes pa;
    bool out_on_device = false;
    if (cudaPointerGetAttributes(&pa, level_out) == cudaSuccess)
        out_on_device = pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged;
    else
        cudaGetLastError();
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!out_on_device) {
        // a host level_out needs a wait for the stream, which a stream under
        // capture cannot do: refuse before anything is enqueued
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FTR_ECUDA;
        if (cs != cudaStreamCaptureStatusNone) return FTR_EINVAL;
    }
    const int nblocks = n > 0 ? (int)((n + kNoAllocPointsPerCta - 1) / kNoAllocPointsPerCta) : 1;
    k_level_noalloc_partial<<<nblocks, kThreads, 0, st>>>(g, points, n, A, scratch);
    if (cudaGetLastError() != cudaSuccess) return FTR_ECUDA;
    k_level_noalloc_final<<<1, 32, 0, st>>>(scratch, nblocks, out_on_device ? level_out : nullptr);
    if (cudaGetLastError() != cudaSuccess) return FTR_ECUDA;
    if (!out_on_device) {
        if (cudaMemcpyAsync(level_out, scratch + 2 * kNoAllocMaxCtas, sizeof(double), cudaMemcpyDeviceToHost, st) !=
            cudaSuccess)
            return FTR_ECUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return FTR_ECUDA;
    }
    return FTR_OK;
}
