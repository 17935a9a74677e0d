// Splat of oriented points into the gradient field V (Sec. III-B, eq. 1-2).
//
//   U(q) = sum_i g(|X_i - p(q)|; sigma1) W_i N_i,  d(q) = sum_i g(|X_i - p(q)|; sigma2) W_i
//   g(x; s) = s^-1 exp(-x^2 / s^2),                V(q) = U(q) / d(q)
//
// over the 4^3 nodes floor(t)-1 .. floor(t)+2 around each point.  The grid is
// cut into 8^3-node bricks; only bricks touched by some stencil get storage.
// Per frame:
//   ingest  point -> (floor t, t - floor t, W, N); t as a float pair, the
//           float64 path only within 1e-5 of a decision; an accepted point
//           adds 1 to every brick its stencil overlaps (counts zeroed when
//           the frame is reset)
//   scan    256-brick tiles: per-tile sums, then each tile adds the sums
//           before it and writes brick offsets, a dense slot per touched
//           brick and the accumulation chunks (no single-CTA scan)
//   fill    per point, append its index to each overlapped brick's list
//   accum   persistent CTAs take work units (up to 1024 (point, brick) pairs
//           of one touched brick) from a per-frame ticket: 64 lanes per point
//           evaluate the stencil nodes inside the brick and add the
//           contributions to shared-memory fixed-point accumulators (value *
//           2^40 as 32-bit hi/lo halves, exact and order-independent, so the
//           result is bit-reproducible); a brick of several units adds each
//           unit's exact sums into an int64 global accumulator and its last
//           unit writes V = (sigma2 / sigma1) U / d to the brick's slot.
// The simple variant (nearest node floor(t + 1/2), V = mean N) uses the same
// bricks with one node per point and d counting points.
#include <cuda_runtime.h>
#include <math.h>

#include "ftr_internal.h"

namespace ftr {

namespace {

// t = (X - b_min) / h - 1/2 per axis.  The float64 product with 1/h is exact
// enough for the stencil offsets; wherever it could round to the other side
// of a decision (the acceptance bounds, floor(t), floor(t + 1/2)) the
// quotient is recomputed with a true division, so every decision equals that
// of (X - b_min) / h in float64.
__device__ __forceinline__ double node_t(double x, double bmin, double h, double inv_h, double n) {
    double t = (x - bmin) * inv_h - 0.5;
    const double band = 1e-9 * (1.0 + fabs(t));
    const double fr = t - floor(t);
    const double fh = (t + 0.5) - floor(t + 0.5);
    if (fr < band || fr > 1.0 - band || fh < band || fh > 1.0 - band || fabs(t - 1.0) < band ||
        fabs(t - (n - 2.0)) < band)
        t = (x - bmin) / h - 0.5;
    return t;
}

// The same t without float64 arithmetic: x - b_min exactly as a sum of two
// floats (two-sum), times 1/h held as a float pair, gives t = th + tl with an
// error below 1e-11 for t < 2^9 (|tl| stays below ~5e-5).  The fraction
// r = (th - floor th) + tl is rounded once (error < 6e-8); floor(t), the
// nearest-node round-up and acceptance (floor(t) in [1, n - 3]) follow from
// it.  Returns false when r lies within 1e-6 of 0, 1/2 or 1, where node_t
// decides instead.
__device__ __forceinline__ bool node_t_pair(float x, float bmin, float ih, float ih_lo, int& fl, float& fr,
                                            bool& up) {
    const float s = x - bmin;
    const float bb = s - x;
    const float e = (x - (s - bb)) + (-bmin - bb);
    const float p = s * ih;
    const float tl = fmaf(s, ih, -p) + fmaf(s, ih_lo, e * ih);
    const float th = p - 0.5f;
    if (!(fabsf(th) < 8388608.0f)) return false;   // NaN, inf or huge: float64 path
    const float f = floorf(th);
    float r = (th - f) + tl;                       // th - f is exact
    int fi = (int)f;
    const float band = 1e-6f;
    if (fabsf(r) < band || fabsf(r - 1.0f) < band || fabsf(r - 0.5f) < band) return false;
    if (r < 0.f) {
        r += 1.0f;
        fi -= 1;
    } else if (r > 1.0f) {
        r -= 1.0f;
        fi += 1;
    }
    fl = fi;
    fr = r;
    up = r > 0.5f;
    return true;
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

// n_dev (nullable): the point count on the device; n then only bounds it.
// One point: t per axis with every decision equal to the float64 one, the
// acceptance test, and the point record at slot `dst`.
// An accepted point also counts itself into every brick its stencil overlaps
// (cnt: per-brick point counts of the frame, zeroed when the frame starts).
__device__ __forceinline__ void ingest_one(const float* p, const float* q, const float* wp, int64_t dst, const GridDev& g,
                                           int4* pbase, float4* pfrac, float4* pnrm, unsigned long long* dropped,
                                           int* wild_weights, int* cnt) {
    bool ok = true;
    int fl[3] = {0, 0, 0};
    float fr[3] = {0.f, 0.f, 0.f};
    int up = 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float x = p[c];
        int fli;
        float r;
        bool u;
        if (node_t_pair(x, g.bminf[c], g.inv_hf[c], g.inv_h_lo[c], fli, r, u)) {
            const bool in = fli >= 1 && fli <= g.n[c] - 3;   // 1 <= t < n - 2
            ok = ok && in;
            if (in) {
                fl[c] = fli;
                fr[c] = r;
                if (u) up |= 1 << c;
            }
        } else {
            const double t = node_t((double)x, g.bmin[c], g.h[c], g.inv_h[c], (double)g.n[c]);
            const bool in = (t >= 1.0) && (t < (double)g.n[c] - 2.0);   // false for NaN
            ok = ok && in;
            if (in) {
                const double f = floor(t);
                fl[c] = (int)f;
                fr[c] = (float)(t - f);
                if (floor(t + 0.5) > f) up |= 1 << c;
            }
        }
    }
    if (!ok) {
        atomicAdd(dropped, 1ull);
        fl[0] = fl[1] = fl[2] = 0;
    }
    const int4 rec = make_int4(fl[0], fl[1], fl[2], ok ? (1 | (up << 1)) : 0);
    pbase[dst] = rec;
    // per brick slot k of the at most 2 x 2 x 2 bricks the stencil overlaps,
    // the lanes counting into the same brick add their number with one atomic
    const unsigned act = __activemask();
    int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
    const bool any = stencil_bricks(rec, g.mode, lo, hi);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int bx = lo[0] + (k & 1), by = lo[1] + ((k >> 1) & 1), bz = lo[2] + (k >> 2);
        const bool valid = any && bx <= hi[0] && by <= hi[1] && bz <= hi[2];
        const int b = valid ? bx + g.nb[0] * (by + g.nb[1] * bz) : -1;
        const unsigned peers = __match_any_sync(act, b);
        if (valid && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(&cnt[b], __popc(peers));
    }
    const float wi = wp ? *wp : 1.0f;
    if (ok && !(wi >= 0.f && wi <= 1.f)) atomicOr(wild_weights, 1);   // outside the fast path's range
    pfrac[dst] = make_float4(fr[0], fr[1], fr[2], wi);
    pnrm[dst] = make_float4(q[0], q[1], q[2], 0.f);
}

__global__ void k_ingest(const float* __restrict__ pts, const float* __restrict__ nrm,
                         const float* __restrict__ w, int64_t n, int64_t base, GridDev g, int4* pbase,
                         float4* pfrac, float4* pnrm, unsigned long long* dropped, int* wild_weights,
                         int64_t* npts_dev, const int* __restrict__ n_dev, int* cnt) {
    pdl_wait();
    if (n_dev) n = min(n, (int64_t)*n_dev);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *npts_dev = base + n;   // points stored so far: later kernels read the count here
    if (i >= n) return;
    ingest_one(pts + 3 * i, nrm + 3 * i, w ? w + i : nullptr, base + i, g, pbase, pfrac, pnrm, dropped, wild_weights,
               cnt);
}

// Several point sets in one launch: thread i ingests point i of the
// concatenation of the sets (set order, as separate launches would store them).
__global__ void k_ingest_sets(IngestSets S, GridDev g, int4* pbase, float4* pfrac, float4* pnrm,
                              unsigned long long* dropped, int* wild_weights, int64_t* npts_dev, int* cnt) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *npts_dev = S.base + S.off[S.k];
    if (i >= S.off[S.k]) return;
    int s = 0;
    while (s + 1 < S.k && i >= S.off[s + 1]) ++s;
    const int64_t j = i - S.off[s];
    ingest_one(S.pts[s] + 3 * j, S.nrm[s] + 3 * j, S.w[s] ? S.w[s] + j : nullptr, S.base + i, g, pbase, pfrac, pnrm,
               dropped, wild_weights, cnt);
}

// Grid-stride over the stored points; the count is read on the device, so the
// launch does not depend on it.
// A warp takes 32 consecutive points (neighbouring pixels of one camera,
// mostly the same bricks): per brick slot k of the at most 2 x 2 x 2 bricks
// a stencil overlaps, the lanes that append to the same brick reserve their
// places with one atomic (the lowest lane's) and write at their rank.
__global__ void k_brick_fill(const int4* __restrict__ pbase, const int64_t* __restrict__ npts, GridDev g,
                             int* cursor, int* entries) {
    pdl_wait();
    const int64_t n = *npts;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform loop: every lane reaches each match below
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); i0 < n; i0 += stride) {
        const int64_t i = i0 + lane;
        int lo[3] = {0, 0, 0}, hi[3] = {-1, -1, -1};
        const bool ok = i < n && stencil_bricks(pbase[i], g.mode, lo, hi);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int bx = lo[0] + (k & 1), by = lo[1] + ((k >> 1) & 1), bz = lo[2] + (k >> 2);
            const bool valid = ok && bx <= hi[0] && by <= hi[1] && bz <= hi[2];
            const int b = valid ? bx + g.nb[0] * (by + g.nb[1] * bz) : -1;
            const unsigned peers = __match_any_sync(0xffffffffu, b);
            if (valid) {
                const int leader = __ffs(peers) - 1;
                int pos = 0;
                if (lane == leader) pos = atomicAdd(&cursor[b], __popc(peers));
                pos = __shfl_sync(peers, pos, leader) + __popc(peers & ((1u << lane) - 1u));
                entries[pos] = (int)i;
            }
        }
    }
}

// Exclusive scan of the brick counts in three coalesced launches over tiles
// of kTile bricks: (1) per-tile sums of the counts and of the touched
// bricks, (2) each tile adds up the sums before it, rescans itself with
// that offset and writes the brick offsets, the dense slot of every
// touched brick (-1 otherwise), the list of touched bricks and the z-range.
constexpr int kScanT = 256;
constexpr int kTile = kBrickScanTile;
static_assert(kTile % kScanT == 0, "a tile is a whole number of block scans");
// A brick's pairs are accumulated in chunks of at most kChunk (point, brick)
// pairs, one chunk per CTA at a time; the 32-bit hi/lo accumulators stay exact
// for up to 2047 contributions per voxel.
constexpr int kChunk = kSplatChunk;

// Block-wide exclusive scan of four ints per thread (kScanT threads).
__device__ __forceinline__ int4 block_scan4(int4 v, int4& total, int4* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int4 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, inc.x, o);
        const int b = __shfl_up_sync(0xffffffffu, inc.y, o);
        const int c = __shfl_up_sync(0xffffffffu, inc.z, o);
        const int d = __shfl_up_sync(0xffffffffu, inc.w, o);
        if (lane >= o) {
            inc.x += a;
            inc.y += b;
            inc.z += c;
            inc.w += d;
        }
    }
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int4 w = lane < kScanT / 32 ? sh[lane] : make_int4(0, 0, 0, 0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, w.x, o);
            const int b = __shfl_up_sync(0xffffffffu, w.y, o);
            const int c = __shfl_up_sync(0xffffffffu, w.z, o);
            const int d = __shfl_up_sync(0xffffffffu, w.w, o);
            if (lane >= o) {
                w.x += a;
                w.y += b;
                w.z += c;
                w.w += d;
            }
        }
        if (lane < kScanT / 32) sh[lane] = w;
    }
    __syncthreads();
    const int4 before = wid ? sh[wid - 1] : make_int4(0, 0, 0, 0);
    total = sh[kScanT / 32 - 1];
    __syncthreads();
    return make_int4(before.x + inc.x - v.x, before.y + inc.y - v.y, before.z + inc.z - v.z,
                     before.w + inc.w - v.w);
}

// Per brick of c (point, brick) pairs: (pairs, touched, accumulation chunks,
// heavy = more than one chunk).
__device__ __forceinline__ int4 brick_counts(int c) {
    const int ch = (c + kChunk - 1) / kChunk;
    return make_int4(c, c > 0, ch, ch > 1);
}

__global__ void __launch_bounds__(kScanT) k_brick_tile_sums(const int* __restrict__ cnt, int nb, int4* tile_sum,
                                                            int* meta) {
    pdl_wait();
    __shared__ int4 sh[kScanT / 32];
    int4 v = make_int4(0, 0, 0, 0);
    for (int k = 0; k < kTile / kScanT; ++k) {
        const int b = blockIdx.x * kTile + k * kScanT + threadIdx.x;
        if (b < nb) {
            const int4 q = brick_counts(cnt[b]);
            v.x += q.x;
            v.y += q.y;
            v.z += q.z;
            v.w += q.w;
        }
    }
    int4 tot;
    block_scan4(v, tot, sh);
    if (threadIdx.x == 0) {
        tile_sum[blockIdx.x] = tot;
        if (blockIdx.x == 0) {       // the z range is min/max-reduced by the write kernel
            meta[2] = 0x7fffffff;
            meta[3] = -1;
        }
    }
}

// Per tile: its exclusive offset is the sum of the (few) tile sums before it,
// summed by every CTA itself (no separate scan launch); CTA 0 also writes the
// totals.  Then the tile's bricks get their offsets, slots and chunk ranges.
__global__ void __launch_bounds__(kScanT) k_brick_tile_write(const int* __restrict__ cnt, int nb, int nbxy,
                                                             const int4* __restrict__ tile_sum, int ntiles, int* off,
                                                             int* cursor, int* slot, int* active, int* meta,
                                                             int* unit_off, int* heavy_idx, int* unit_slot) {
    pdl_wait();
    __shared__ int4 sh[kScanT / 32];
    int4 pre = make_int4(0, 0, 0, 0), all = make_int4(0, 0, 0, 0);
    for (int i = threadIdx.x; i < ntiles; i += kScanT) {
        const int4 v = tile_sum[i];
        if (i < (int)blockIdx.x) {
            pre.x += v.x;
            pre.y += v.y;
            pre.z += v.z;
            pre.w += v.w;
        }
        all.x += v.x;
        all.y += v.y;
        all.z += v.z;
        all.w += v.w;
    }
    int4 run, total;
    block_scan4(pre, run, sh);
    block_scan4(all, total, sh);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        off[nb] = total.x;
        unit_off[total.y] = total.z;   // end of the last touched brick's chunks
        meta[0] = total.y;
        meta[1] = total.x;
        meta[4] = 0;                   // chunk ticket of the accumulation
        meta[5] = total.z;             // chunks in all
        meta[6] = total.w;             // heavy bricks
    }
    int zmin = 0x7fffffff, zmax = -1;
    for (int k = 0; k < kTile / kScanT; ++k) {
        const int b = blockIdx.x * kTile + k * kScanT + threadIdx.x;
        const int c = b < nb ? cnt[b] : 0;
        const int4 q = brick_counts(c);
        int4 tot;
        const int4 ex = block_scan4(q, tot, sh);
        if (b < nb) {
            off[b] = run.x + ex.x;
            cursor[b] = run.x + ex.x;
            if (c > 0) {
                const int s = run.y + ex.y;
                slot[b] = s;
                active[s] = b;
                unit_off[s] = run.z + ex.z;
                for (int j = 0; j < q.z; ++j) unit_slot[run.z + ex.z + j] = s;
                heavy_idx[s] = q.w ? run.w + ex.w : -1;
                const int bz = b / nbxy;
                zmin = min(zmin, bz);
                zmax = max(zmax, bz);
            } else {
                slot[b] = -1;
            }
        }
        run.x += tot.x;
        run.y += tot.y;
        run.z += tot.z;
        run.w += tot.w;
    }
    if (zmax >= 0) {
        atomicMin(&meta[2], zmin);
        atomicMax(&meta[3], zmax);
    }
}

constexpr int kAccThreads = 512;

// round(v * 2^40) as int64 without a 64-bit conversion (those run on the slow
// double-precision pipe): with x = v 2^9, hi = trunc(x) and r = x - hi (exact:
// Sterbenz, or r = x when |x| < 1), v 2^40 = hi 2^31 + r 2^31 where r 2^31 is
// an exact float in (-2^31, 2^31) rounded to the nearest integer (ties to
// even, like the direct conversion, since hi 2^31 is even).
__device__ __forceinline__ long long fix40(float v) {
    const float x = v * 512.0f;
    const float hf = truncf(x);
    const int lo = __float2int_rn((x - hf) * 2147483648.0f);
    return (long long)(int)hf * 2147483648ll + (long long)lo;
}

// int64 -> float32 of its magnitude's two 32-bit halves, sign restored after
// (no cancellation for small negative values; no 64-bit conversion)
__device__ __forceinline__ float fix_to_float(long long v) {
    const bool neg = v < 0;
    const unsigned long long m = neg ? (unsigned long long)(-v) : (unsigned long long)v;
    const float f = fmaf((float)(unsigned)(m >> 32), 4294967296.0f, (float)(unsigned)(m & 0xffffffffull));
    return neg ? -f : f;
}

constexpr int kStage = kAccThreads;   // point records staged in shared memory per batch (one per thread)

// Fixed-point contribution round(v * 2^40) = hi 2^20 + lo with two float to
// int conversions: hi = round(v 2^20); r = v - hi 2^-20 is exact (Sterbenz,
// or r = v when hi = 0) with |r| <= 2^-21, and lo = round(r 2^40) in
// [-2^19, 2^19].  Ties go to even as in a direct conversion (hi 2^20 is even).
__device__ __forceinline__ void fix40_split(float v, int& hi, int& lo) {
    const float hf = rintf(v * 1048576.0f);
    hi = (int)hf;
    lo = __float2int_rn(fmaf(hf, -9.5367431640625e-07f, v) * 1099511627776.0f);
}

// Persistent CTAs take work units from a per-frame ticket: a unit is one
// chunk of at most kChunk (point, brick) pairs of one touched brick.  64
// lanes per point evaluate the stencil nodes that fall inside the brick and
// add the fixed-point contributions to shared-memory accumulators.  Integer
// sums are exact and order-independent, so V is bit-reproducible.  32-bit
// atomics on the (hi, lo) parts, exact while a voxel receives fewer than 2^11
// contributions of magnitude <= 1 (a chunk has at most kChunk points; weights
// in [0, 1]: |sum hi| < 2^31, |sum lo| < 2^30); weights outside [0, 1] take
// 64-bit shared atomics.  A brick of one chunk writes V directly; the chunks
// of a heavier brick add their exact sums into its int64 accumulator in
// global memory, and the chunk that completes last (a per-brick counter)
// writes V and clears the accumulator for the next frame.
__global__ void __launch_bounds__(kAccThreads) k_splat_accum(GridDev g, const int* __restrict__ active,
                                                             const int* __restrict__ meta,
                                                             const int* __restrict__ off,
                                                             const int* __restrict__ entries,
                                                             const int4* __restrict__ pbase,
                                                             const float4* __restrict__ pfrac,
                                                             const float4* __restrict__ pnrm,
                                                             const int* __restrict__ wild_weights,
                                                             float* __restrict__ vpool, int* __restrict__ ticket,
                                                             const int* __restrict__ unit_off,
                                                             const int* __restrict__ unit_slot,
                                                             const int* __restrict__ heavy_idx,
                                                             unsigned long long* __restrict__ heavy_acc,
                                                             int* __restrict__ heavy_done) {
    pdl_wait();
    __shared__ __align__(16) unsigned acc[8][kBrickVox];   // fast: [c] hi, [4 + c] lo; slow: 4 x int64
    __shared__ int4 s_base[kStage];
    __shared__ float4 s_frac[kStage];
    __shared__ float4 s_nrm[kStage];
    unsigned long long* acc64 = reinterpret_cast<unsigned long long*>(&acc[0][0]);
    const int tid = threadIdx.x;
    const int o = tid & 63;
    const int ox = o & 3, oy = (o >> 2) & 3, oz = o >> 4;
    const int pl = tid >> 6;
    const bool weights_ok = wild_weights[0] == 0;
    const int nunits = meta[5];
    __shared__ int s_unit, s_slot;
    __shared__ bool s_last;
    for (;;) {
        if (tid == 0) {
            const int u = atomicAdd(ticket, 1);
            s_unit = u;
            s_slot = u < nunits ? unit_slot[u] : 0;   // the touched brick whose chunks hold unit u
        }
        __syncthreads();
        const int unit = s_unit, s = s_slot;
        if (unit >= nunits) break;                                      // block-uniform
        const int b = active[s];
        const int bx = b % g.nb[0], by = (b / g.nb[0]) % g.nb[1], bz = b / (g.nb[0] * g.nb[1]);
        const int orgx = bx * kBrick, orgy = by * kBrick, orgz = bz * kBrick;
        const int nchunks = unit_off[s + 1] - unit_off[s];
        const int e0 = off[b] + (unit - unit_off[s]) * kChunk;
        const int e1 = min(off[b + 1], e0 + kChunk);
        const bool fast = weights_ok;                                   // block-uniform
        for (int k = tid; k < 8 * kBrickVox; k += kAccThreads) (&acc[0][0])[k] = 0u;
        for (int eb = e0; eb < e1; eb += kStage) {
            const int nbatch = min(kStage, e1 - eb);
            __syncthreads();
            if (tid < nbatch) {
                const int i = entries[eb + tid];
                s_base[tid] = pbase[i];
                s_frac[tid] = pfrac[i];
                s_nrm[tid] = pnrm[i];
            }
            __syncthreads();
            if (g.mode == FTR_SPLAT_WEIGHTED) {
                for (int p = pl; p < nbatch; p += kAccThreads / 64) {
                    const int4 pb = s_base[p];
                    const int lx = pb.x - 1 + ox - orgx;
                    const int ly = pb.y - 1 + oy - orgy;
                    const int lz = pb.z - 1 + oz - orgz;
                    if ((unsigned)lx >= kBrick || (unsigned)ly >= kBrick || (unsigned)lz >= kBrick) continue;
                    const float4 fr = s_frac[p];
                    const float4 nr = s_nrm[p];
                    // X - p(q) = (t - q) h with t - q = frac + 1 - offset
                    const float dx = (fr.x + 1.0f - (float)ox) * g.hf[0];
                    const float dy = (fr.y + 1.0f - (float)oy) * g.hf[1];
                    const float dz = (fr.z + 1.0f - (float)oz) * g.hf[2];
                    const float r2 = dx * dx + dy * dy + dz * dz;
                    const float e1v = expf(-r2 * g.inv_s1sq) * fr.w;   // sigma1 * g1 * W
                    const float e2v = expf(-r2 * g.inv_s2sq) * fr.w;   // sigma2 * g2 * W
                    const int li = lx + kBrick * (ly + kBrick * lz);
                    const float val[4] = {e1v * nr.x, e1v * nr.y, e1v * nr.z, e2v};
                    if (fast) {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            int hi, lo;
                            fix40_split(val[c], hi, lo);
                            atomicAdd(reinterpret_cast<int*>(&acc[c][li]), hi);
                            atomicAdd(reinterpret_cast<int*>(&acc[4 + c][li]), lo);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            atomicAdd(&acc64[c * kBrickVox + li], (unsigned long long)fix40(val[c]));
                    }
                }
            } else {
                for (int p = tid; p < nbatch; p += kAccThreads) {
                    const int4 pb = s_base[p];
                    const int lx = pb.x + ((pb.w >> 1) & 1) - orgx;
                    const int ly = pb.y + ((pb.w >> 2) & 1) - orgy;
                    const int lz = pb.z + ((pb.w >> 3) & 1) - orgz;
                    const float4 nr = s_nrm[p];
                    const int li = lx + kBrick * (ly + kBrick * lz);
                    const float val[3] = {nr.x, nr.y, nr.z};
                    if (fast) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            int hi, lo;
                            fix40_split(val[c], hi, lo);
                            atomicAdd(reinterpret_cast<int*>(&acc[c][li]), hi);
                            atomicAdd(reinterpret_cast<int*>(&acc[4 + c][li]), lo);
                        }
                        atomicAdd(reinterpret_cast<int*>(&acc[3][li]), 1 << 20);   // count: 2^40 = 2^20 * 2^20
                    } else {
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            atomicAdd(&acc64[c * kBrickVox + li], (unsigned long long)fix40(val[c]));
                        atomicAdd(&acc64[3 * kBrickVox + li], 1ull << 40);
                    }
                }
            }
        }
        __syncthreads();
        float* out = vpool + (size_t)s * 3 * kBrickVox;
        unsigned long long* gacc = nullptr;
        if (nchunks > 1) {
            // add this chunk's exact sums to the brick's global accumulator
            gacc = heavy_acc + (size_t)heavy_idx[s] * 4 * kBrickVox;
            for (int li = tid; li < kBrickVox; li += kAccThreads) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const long long v = fast ? (long long)(int)acc[c][li] * (1ll << 20) + (long long)(int)acc[4 + c][li]
                                             : (long long)acc64[c * kBrickVox + li];
                    if (v != 0) atomicAdd(&gacc[c * kBrickVox + li], (unsigned long long)v);
                }
            }
            __threadfence();
            __syncthreads();
            if (tid == 0) s_last = atomicAdd(&heavy_done[heavy_idx[s]], 1) == nchunks - 1;
            __syncthreads();
            if (!s_last) continue;                                      // block-uniform; next unit
            __threadfence();
        }
        for (int li = tid; li < kBrickVox; li += kAccThreads) {
            long long u[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if (gacc) {
                    u[c] = (long long)__ldcg(&gacc[c * kBrickVox + li]);
                    gacc[c * kBrickVox + li] = 0ull;                    // cleared for the next frame
                } else {
                    u[c] = fast ? (long long)(int)acc[c][li] * (1ll << 20) + (long long)(int)acc[4 + c][li]
                                : (long long)acc64[c * kBrickVox + li];
                }
            }
            if (u[3] > 0) {
                // exact integer sums, one float32 quotient per voxel
                const float sc = g.v_scale_f / fix_to_float(u[3]);
                out[li] = fix_to_float(u[0]) * sc;
                out[kBrickVox + li] = fix_to_float(u[1]) * sc;
                out[2 * kBrickVox + li] = fix_to_float(u[2]) * sc;
            } else {
                out[li] = 0.f;
                out[kBrickVox + li] = 0.f;
                out[2 * kBrickVox + li] = 0.f;
            }
        }
        if (gacc && tid == 0) heavy_done[heavy_idx[s]] = 0;
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

cudaError_t launch_ingest(ftr_ctx* c, const float* pts, const float* nrm, const float* w, int64_t n,
                          const int* n_dev) {
    if (n == 0) return cudaSuccess;
    // small CTAs spread the few float64 operations per point over every SM
    launch_pdl(k_ingest, blocks_for(n, 32), 32, 0, c->stream, pts, nrm, w, n, c->n_pts, c->g, c->pts.base, c->pts.frac,
                                                       c->pts.nrm, c->d_dropped, c->d_wild, c->d_npts, n_dev,
                                                       c->d_brick_cnt);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_ingest_sets(ftr_ctx* c, const IngestSets& S) {
    const int64_t n = S.off[S.k];
    if (n == 0) return cudaSuccess;
    launch_pdl(k_ingest_sets, blocks_for(n, 32), 32, 0, c->stream, S, c->g, c->pts.base, c->pts.frac, c->pts.nrm,
               c->d_dropped, c->d_wild, c->d_npts, c->d_brick_cnt);
    c->launches++;
    return cudaGetLastError();
}

cudaError_t launch_splat(ftr_ctx* c) {
    cudaError_t e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    if (sms <= 0) sms = 152;
    prof_begin(c, ST_SPLAT_BIN);
    // the per-brick point counts were taken by the ingest
    const int ntiles = (c->n_bricks + kTile - 1) / kTile;
    launch_pdl(k_brick_tile_sums, ntiles, kScanT, 0, c->stream, c->d_brick_cnt, c->n_bricks, c->d_tile, c->d_meta);
    launch_pdl(k_brick_tile_write, ntiles, kScanT, 0, c->stream, c->d_brick_cnt, c->n_bricks, c->g.nb[0] * c->g.nb[1],
               c->d_tile, ntiles, c->d_brick_off, c->d_brick_cursor, c->d_brick_slot, c->d_active, c->d_meta,
               c->d_unit_off, c->d_heavy_idx, c->d_unit_slot);
    c->launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    launch_pdl(k_brick_fill, sms * 2, 256, 0, c->stream, c->pts.base, c->d_npts, c->g, c->d_brick_cursor, c->d_entries);
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    prof_end(c, ST_SPLAT_BIN);
    prof_begin(c, ST_SPLAT_ACC);
    const int grid = sms * 4;
    launch_pdl(k_splat_accum, grid, kAccThreads, 0, c->stream, c->g, c->d_active, c->d_meta, c->d_brick_off, c->d_entries,
               c->pts.base, c->pts.frac, c->pts.nrm, c->d_wild, c->d_vpool, c->d_meta + 4, c->d_unit_off,
               c->d_unit_slot, c->d_heavy_idx, c->d_heavy_acc, c->d_heavy_done);
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
