// Splat of oriented points into the gradient field V (Sec. III-B, eq. 1-2).
//
//   U(q) = sum_i g(|X_i - p(q)|; sigma1) W_i N_i,  d(q) = sum_i g(|X_i - p(q)|; sigma2) W_i
//   g(x; s) = s^-1 exp(-x^2 / s^2),                V(q) = U(q) / d(q)
//
// over the 4^3 nodes floor(t)-1 .. floor(t)+2 around each point.  The grid is
// cut into 8^3-node bricks; only bricks touched by some stencil get storage.
// Per frame:
//   ingest  point -> (floor t, t - floor t, W, N), acceptance test in FP64
//   count   per point, +1 on every brick its stencil overlaps
//   scan    one CTA: brick offsets, dense slot per touched brick
//   fill    per point, append its index to each overlapped brick's list
//   accum   one CTA per touched brick: 64 lanes per point evaluate the stencil
//           nodes inside the brick and add the contributions to shared-memory
//           int64 fixed-point accumulators (value * 2^40, exact and
//           order-independent, so the result is bit-reproducible); then
//           V = (sigma2 / sigma1) U / d is written to the brick's slot.
// The simple variant (nearest node floor(t + 1/2), V = mean N) uses the same
// bricks with one node per point and d counting points.
#include <cuda_runtime.h>
#include <math.h>

#include "ftr_internal.h"

namespace ftr {

namespace {

__global__ void k_ingest(const float* __restrict__ pts, const float* __restrict__ nrm,
                         const float* __restrict__ w, int64_t n, int64_t base, GridDev g, int4* pbase,
                         float4* pfrac, float4* pnrm, unsigned long long* dropped) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool ok = true;
    int fl[3] = {0, 0, 0};
    float fr[3] = {0.f, 0.f, 0.f};
    int up = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double t = ((double)pts[3 * i + c] - g.bmin[c]) / g.h[c] - 0.5;
        bool in = (t >= 1.0) && (t < (double)g.n[c] - 2.0);   // false for NaN
        ok = ok && in;
        if (in) {
            double f = floor(t);
            fl[c] = (int)f;
            fr[c] = (float)(t - f);
            if (floor(t + 0.5) > f) up |= 1 << c;
        }
    }
    if (!ok) {
        atomicAdd(dropped, 1ull);
        fl[0] = fl[1] = fl[2] = 0;
    }
    pbase[base + i] = make_int4(fl[0], fl[1], fl[2], ok ? (1 | (up << 1)) : 0);
    pfrac[base + i] = make_float4(fr[0], fr[1], fr[2], w ? w[i] : 1.0f);
    pnrm[base + i] = make_float4(nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2], 0.f);
}

// Brick range [lo, hi] per axis that the point's stencil overlaps.
__device__ __forceinline__ bool stencil_bricks(const int4 b, int mode, int lo[3], int hi[3]) {
    if (!(b.w & 1)) return false;
    const int bb[3] = {b.x, b.y, b.z};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (mode == FTR_SPLAT_WEIGHTED) {
            lo[c] = (bb[c] - 1) >> 3;
            hi[c] = (bb[c] + 2) >> 3;
        } else {
            int node = bb[c] + ((b.w >> (1 + c)) & 1);
            lo[c] = hi[c] = node >> 3;
        }
    }
    return true;
}

__global__ void k_brick_count(const int4* __restrict__ pbase, int64_t n, GridDev g, int* cnt) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo[3], hi[3];
    if (!stencil_bricks(pbase[i], g.mode, lo, hi)) return;
    for (int bz = lo[2]; bz <= hi[2]; ++bz)
        for (int by = lo[1]; by <= hi[1]; ++by)
            for (int bx = lo[0]; bx <= hi[0]; ++bx) atomicAdd(&cnt[bx + g.nb[0] * (by + g.nb[1] * bz)], 1);
}

__global__ void k_brick_fill(const int4* __restrict__ pbase, int64_t n, GridDev g, int* cursor, int* entries) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo[3], hi[3];
    if (!stencil_bricks(pbase[i], g.mode, lo, hi)) return;
    for (int bz = lo[2]; bz <= hi[2]; ++bz)
        for (int by = lo[1]; by <= hi[1]; ++by)
            for (int bx = lo[0]; bx <= hi[0]; ++bx) {
                int pos = atomicAdd(&cursor[bx + g.nb[0] * (by + g.nb[1] * bz)], 1);
                entries[pos] = (int)i;
            }
}

// One CTA of 1024 threads: exclusive scan of the brick counts, dense slots
// for the touched bricks, and the z-range of touched bricks.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_brick_scan(const int* __restrict__ cnt, int nb, int nbxy,
                                                             int* off, int* cursor, int* slot, int* active,
                                                             int* meta) {
    __shared__ int s_sum[kScanThreads / 32], s_act[kScanThreads / 32];
    __shared__ int s_zmin, s_zmax;
    const int t = threadIdx.x;
    const int per = (nb + kScanThreads - 1) / kScanThreads;
    const int b0 = min(nb, t * per), b1 = min(nb, b0 + per);
    if (t == 0) {
        s_zmin = 0x7fffffff;
        s_zmax = -1;
    }
    int sum = 0, act = 0;
    for (int b = b0; b < b1; ++b) {
        int c = cnt[b];
        sum += c;
        act += (c > 0);
    }
    // block exclusive scan of (sum, act)
    const int lane = t & 31, wid = t >> 5;
    int is = sum, ia = act;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int vs = __shfl_up_sync(0xffffffffu, is, o);
        int va = __shfl_up_sync(0xffffffffu, ia, o);
        if (lane >= o) {
            is += vs;
            ia += va;
        }
    }
    if (lane == 31) {
        s_sum[wid] = is;
        s_act[wid] = ia;
    }
    __syncthreads();
    if (wid == 0) {
        int ws = s_sum[lane], wa = s_act[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int vs = __shfl_up_sync(0xffffffffu, ws, o);
            int va = __shfl_up_sync(0xffffffffu, wa, o);
            if (lane >= o) {
                ws += vs;
                wa += va;
            }
        }
        s_sum[lane] = ws;
        s_act[lane] = wa;
    }
    __syncthreads();
    int es = is - sum + (wid ? s_sum[wid - 1] : 0);
    int ea = ia - act + (wid ? s_act[wid - 1] : 0);
    int zmin = 0x7fffffff, zmax = -1;
    for (int b = b0; b < b1; ++b) {
        int c = cnt[b];
        off[b] = es;
        cursor[b] = es;
        if (c > 0) {
            slot[b] = ea;
            active[ea] = b;
            ++ea;
            int bz = b / nbxy;
            zmin = min(zmin, bz);
            zmax = max(zmax, bz);
        } else {
            slot[b] = -1;
        }
        es += c;
    }
    if (zmax >= 0) {
        atomicMin(&s_zmin, zmin);
        atomicMax(&s_zmax, zmax);
    }
    __syncthreads();
    if (t == kScanThreads - 1) {
        off[nb] = es;
        meta[0] = ea;
        meta[1] = es;
        meta[2] = s_zmax >= 0 ? s_zmin : 0;
        meta[3] = s_zmax;
    }
}

constexpr int kAccThreads = 256;
constexpr float kFix = 1099511627776.0f;    // 2^40

__global__ void __launch_bounds__(kAccThreads) k_splat_accum(GridDev g, const int* __restrict__ active,
                                                             const int* __restrict__ meta,
                                                             const int* __restrict__ off,
                                                             const int* __restrict__ entries,
                                                             const int4* __restrict__ pbase,
                                                             const float4* __restrict__ pfrac,
                                                             const float4* __restrict__ pnrm,
                                                             float* __restrict__ vpool) {
    __shared__ unsigned long long acc[4][kBrickVox];
    const int nact = meta[0];
    const int tid = threadIdx.x;
    const int o = tid & 63;
    const int ox = o & 3, oy = (o >> 2) & 3, oz = o >> 4;
    const int pl = tid >> 6;
    for (int s = blockIdx.x; s < nact; s += gridDim.x) {
        const int b = active[s];
        const int bx = b % g.nb[0], by = (b / g.nb[0]) % g.nb[1], bz = b / (g.nb[0] * g.nb[1]);
        const int org[3] = {bx * kBrick, by * kBrick, bz * kBrick};
        for (int k = tid; k < 4 * kBrickVox; k += kAccThreads) (&acc[0][0])[k] = 0ull;
        __syncthreads();
        const int e0 = off[b], e1 = off[b + 1];
        if (g.mode == FTR_SPLAT_WEIGHTED) {
            for (int e = e0 + pl; e < e1; e += kAccThreads / 64) {
                const int i = entries[e];
                const int4 pb = pbase[i];
                const int lx = pb.x - 1 + ox - org[0];
                const int ly = pb.y - 1 + oy - org[1];
                const int lz = pb.z - 1 + oz - org[2];
                if ((unsigned)lx >= kBrick || (unsigned)ly >= kBrick || (unsigned)lz >= kBrick) continue;
                const float4 fr = pfrac[i];
                const float4 nr = pnrm[i];
                // X - p(q) = (t - q) h with t - q = frac + 1 - offset
                const float dx = (fr.x + 1.0f - (float)ox) * g.hf[0];
                const float dy = (fr.y + 1.0f - (float)oy) * g.hf[1];
                const float dz = (fr.z + 1.0f - (float)oz) * g.hf[2];
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float e1v = expf(-r2 * g.inv_s1sq) * fr.w;   // sigma1 * g1 * W
                const float e2v = expf(-r2 * g.inv_s2sq) * fr.w;   // sigma2 * g2 * W
                const int li = lx + kBrick * (ly + kBrick * lz);
                atomicAdd(&acc[0][li], (unsigned long long)__float2ll_rn(e1v * nr.x * kFix));
                atomicAdd(&acc[1][li], (unsigned long long)__float2ll_rn(e1v * nr.y * kFix));
                atomicAdd(&acc[2][li], (unsigned long long)__float2ll_rn(e1v * nr.z * kFix));
                atomicAdd(&acc[3][li], (unsigned long long)__float2ll_rn(e2v * kFix));
            }
        } else {
            for (int e = e0 + tid; e < e1; e += kAccThreads) {
                const int i = entries[e];
                const int4 pb = pbase[i];
                const int lx = pb.x + ((pb.w >> 1) & 1) - org[0];
                const int ly = pb.y + ((pb.w >> 2) & 1) - org[1];
                const int lz = pb.z + ((pb.w >> 3) & 1) - org[2];
                const float4 nr = pnrm[i];
                const int li = lx + kBrick * (ly + kBrick * lz);
                atomicAdd(&acc[0][li], (unsigned long long)__float2ll_rn(nr.x * kFix));
                atomicAdd(&acc[1][li], (unsigned long long)__float2ll_rn(nr.y * kFix));
                atomicAdd(&acc[2][li], (unsigned long long)__float2ll_rn(nr.z * kFix));
                atomicAdd(&acc[3][li], (unsigned long long)(1ll << 40));
            }
        }
        __syncthreads();
        float* out = vpool + (size_t)s * 3 * kBrickVox;
        for (int li = tid; li < kBrickVox; li += kAccThreads) {
            const long long d = (long long)acc[3][li];
            if (d > 0) {
                const double sc = g.v_scale / (double)d;
                out[li] = (float)((double)(long long)acc[0][li] * sc);
                out[kBrickVox + li] = (float)((double)(long long)acc[1][li] * sc);
                out[2 * kBrickVox + li] = (float)((double)(long long)acc[2][li] * sc);
            } else {
                out[li] = 0.f;
                out[kBrickVox + li] = 0.f;
                out[2 * kBrickVox + li] = 0.f;
            }
        }
        __syncthreads();
    }
}

__global__ void k_dense_V(GridDev g, const int* __restrict__ slot, const float* __restrict__ vpool, int64_t M,
                          float* out) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M) return;
    const int x = (int)(q % g.n[0]);
    const int y = (int)((q / g.n[0]) % g.n[1]);
    const int z = (int)(q / ((int64_t)g.n[0] * g.n[1]));
    const int s = slot[(x >> 3) + g.nb[0] * ((y >> 3) + g.nb[1] * (z >> 3))];
    const int li = (x & 7) + 8 * ((y & 7) + 8 * (z & 7));
#pragma unroll
    for (int c = 0; c < 3; ++c)
        out[c * M + q] = s >= 0 ? vpool[(size_t)s * 3 * kBrickVox + c * kBrickVox + li] : 0.f;
}

__global__ void k_load_dense_V(GridDev g, const float* __restrict__ V, int64_t M, int* slot, int* active,
                               float* vpool) {
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= M) return;
    const int x = (int)(q % g.n[0]);
    const int y = (int)((q / g.n[0]) % g.n[1]);
    const int z = (int)(q / ((int64_t)g.n[0] * g.n[1]));
    const int b = (x >> 3) + g.nb[0] * ((y >> 3) + g.nb[1] * (z >> 3));
    const int li = (x & 7) + 8 * ((y & 7) + 8 * (z & 7));
    if (li == 0) {
        slot[b] = b;
        active[b] = b;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) vpool[(size_t)b * 3 * kBrickVox + c * kBrickVox + li] = V[c * M + q];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_ingest(ftr_ctx* c, const float* pts, const float* nrm, const float* w, int64_t n) {
    if (n == 0) return cudaSuccess;
    k_ingest<<<blocks_for(n, 256), 256, 0, c->stream>>>(pts, nrm, w, n, c->n_pts, c->g, c->pts.base, c->pts.frac,
                                                       c->pts.nrm, c->d_dropped);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_splat(ftr_ctx* c) {
    cudaError_t e;
    const int64_t n = c->n_pts;
    prof_begin(c, ST_SPLAT_BIN);
    if ((e = cudaMemsetAsync(c->d_brick_cnt, 0, sizeof(int) * c->n_bricks, c->stream)) != cudaSuccess) return e;
    if (n > 0) {
        k_brick_count<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->pts.base, n, c->g, c->d_brick_cnt);
        c->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_brick_scan<<<1, kScanThreads, 0, c->stream>>>(c->d_brick_cnt, c->n_bricks, c->g.nb[0] * c->g.nb[1],
                                                   c->d_brick_off, c->d_brick_cursor, c->d_brick_slot,
                                                   c->d_active, c->d_meta);
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (n > 0) {
        k_brick_fill<<<blocks_for(n, 256), 256, 0, c->stream>>>(c->pts.base, n, c->g, c->d_brick_cursor,
                                                               c->d_entries);
        c->launches++;
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    prof_end(c, ST_SPLAT_BIN);
    prof_begin(c, ST_SPLAT_ACC);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    const int grid = (sms > 0 ? sms : 152) * 8;
    k_splat_accum<<<grid, kAccThreads, 0, c->stream>>>(c->g, c->d_active, c->d_meta, c->d_brick_off, c->d_entries,
                                                       c->pts.base, c->pts.frac, c->pts.nrm, c->d_vpool);
    c->launches++;
    prof_end(c, ST_SPLAT_ACC);
    return cudaGetLastError();
}

cudaError_t launch_load_dense_V(ftr_ctx* c, const float* V_dev) {
    k_load_dense_V<<<blocks_for(c->M, 256), 256, 0, c->stream>>>(c->g, V_dev, c->M, c->d_brick_slot, c->d_active,
                                                                 c->d_vpool);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int meta[4] = {c->n_bricks, 0, 0, c->g.nb[2] - 1};
    return cudaMemcpyAsync(c->d_meta, meta, sizeof(meta), cudaMemcpyHostToDevice, c->stream);
}

cudaError_t launch_dense_V(ftr_ctx* c, float* out_dev) {
    k_dense_V<<<blocks_for(c->M, 256), 256, 0, c->stream>>>(c->g, c->d_brick_slot, c->d_vpool, c->M, out_dev);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace ftr
