// Marching cubes on A at level L (Sec. III-B, [35]), scan-compacted.
//
// Corner bit = 1 iff A >= L with A promoted to float64.  Because A is float32,
// that is the same as A >= Lf with Lf = L rounded up to float32, so the
// kernels compare in float32 and still take the float64 decision.  A node owns
// the grid edges toward +x, +y, +z; an edge carries a vertex when its two bits
// differ.  Vertex ids are the rank of (node, axis) in linear node order and
// triangles follow cell order then table order, so the mesh does not depend
// on scheduling.
//
// One warp walks one grid row (y, z) in 32-node segments.  Per segment it
// loads the rows (y, z), (y+1, z), (y, z+1), (y+1, z+1) once, turns them into
// four 32-bit ballots, and reads every node's edge bits and cube class from
// those masks (the +x neighbour is the next bit; lane 31 fetches the first
// node of the next segment).  Launches:
//   count  per row: active nodes (owning a vertex or lower corner of a cell
//          with triangles), vertices, triangles
//   scan   three coalesced launches: exclusive offsets of the row counts
//   emit   rows with surface only: one 16-byte record per active node (node,
//          edge bits | class << 8, first vertex, first triangle), vertex
//          positions t = (L - A0)/(A1 - A0) in float64 and normals -grad A
//          (central differences, one-sided at the border, lerped); in-row
//          offsets come from ballot popcounts
//   tris   one thread per active node: triangle corners from the case table;
//          an edge owned by another node is found by binary search in the
//          sorted node records.
#include <cuda_runtime.h>

#include "ftr_internal.h"

namespace ftr {
namespace {

__constant__ int c_ntri[256];
__constant__ signed char c_tri[256][kMaxTrisPerCase][3];


struct NodeInfo {
    int flags;     // bit a: edge toward +a crosses
    int cls;       // cube class, 0 if the node is not a cell's lower corner
};

__device__ __forceinline__ NodeInfo classify_node(const float* __restrict__ A, int64_t n, int x, int y, int z,
                                                  const GridDev& g, float L) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const bool hx = x < nx - 1, hy = y < ny - 1, hz = z < nz - 1;
    const int b0 = A[n] >= L;
    NodeInfo r;
    r.flags = 0;
    r.cls = 0;
    const int bx = hx ? (A[n + 1] >= L) : b0;
    const int by = hy ? (A[n + sy] >= L) : b0;
    const int bz = hz ? (A[n + sz] >= L) : b0;
    r.flags = (bx != b0) | ((by != b0) << 1) | ((bz != b0) << 2);
    if (hx && hy && hz) {
        const int bxy = A[n + 1 + sy] >= L;
        const int bxz = A[n + 1 + sz] >= L;
        const int byz = A[n + sy + sz] >= L;
        const int bxyz = A[n + 1 + sy + sz] >= L;
        r.cls = b0 | (bx << 1) | (by << 2) | (bxy << 3) | (bz << 4) | (bxz << 5) | (byz << 6) | (bxyz << 7);
    }
    return r;
}

constexpr int kRowsPerCta = kMcThreads / 32;

// One 128-node segment of row (y, z) starting at x0: lane l holds nodes
// x0 + 4l .. x0 + 4l + 3.  bits[r] packs, for the rows r = (y,z), (y+1,z),
// (y,z+1), (y+1,z+1), bit j = (A >= L) at node j of the lane and bit 4 = the
// same at the lane's +x neighbour of node 3.
struct Seg4 {
    int bits[4];
};

__device__ __forceinline__ int nib(float4 v, float L) {
    return (v.x >= L) | ((v.y >= L) << 1) | ((v.z >= L) << 2) | ((v.w >= L) << 3);
}

__device__ __forceinline__ Seg4 seg_load(const float* __restrict__ A, int64_t rowbase, int x0, int nx,
                                         int64_t sy, int64_t sz, bool hy, bool hz, float L) {
    const int lane = threadIdx.x & 31;
    const int x = x0 + 4 * lane;
    const bool valid = x < nx;
    const float4* p = reinterpret_cast<const float4*>(A + rowbase + x);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 r00 = valid ? p[0] : z4;
    const float4 r10 = (valid && hy) ? *reinterpret_cast<const float4*>(A + rowbase + x + sy) : z4;
    const float4 r01 = (valid && hz) ? *reinterpret_cast<const float4*>(A + rowbase + x + sz) : z4;
    const float4 r11 = (valid && hy && hz) ? *reinterpret_cast<const float4*>(A + rowbase + x + sy + sz) : z4;
    Seg4 s;
    s.bits[0] = valid ? nib(r00, L) : 0;
    s.bits[1] = (valid && hy) ? nib(r10, L) : 0;
    s.bits[2] = (valid && hz) ? nib(r01, L) : 0;
    s.bits[3] = (valid && hy && hz) ? nib(r11, L) : 0;
    // +x neighbour of node 3: the next lane's node 0, or the next segment's
    // first node for lane 31
    int nb[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) nb[r] = __shfl_down_sync(0xffffffffu, s.bits[r], 1) & 1;
    if (lane == 31) {
        const int64_t n = rowbase + x + 4;
        const bool more = x + 4 < nx;
        nb[0] = more && A[n] >= L;
        nb[1] = more && hy && A[n + sy] >= L;
        nb[2] = more && hz && A[n + sz] >= L;
        nb[3] = more && hy && hz && A[n + sy + sz] >= L;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) s.bits[r] |= nb[r] << 4;
    return s;
}

// Edge bits and cube class of node j (0..3) of this lane.
__device__ __forceinline__ NodeInfo seg_node(const Seg4& s, int j, int x, int nx, bool hy, bool hz) {
    const bool hx = x < nx - 1;
    const int b0 = (s.bits[0] >> j) & 1, bx = (s.bits[0] >> (j + 1)) & 1;
    const int by = (s.bits[1] >> j) & 1, bxy = (s.bits[1] >> (j + 1)) & 1;
    const int bz = (s.bits[2] >> j) & 1, bxz = (s.bits[2] >> (j + 1)) & 1;
    const int byz = (s.bits[3] >> j) & 1, bxyz = (s.bits[3] >> (j + 1)) & 1;
    NodeInfo r;
    r.flags = (hx && bx != b0) | ((hy && by != b0) << 1) | ((hz && bz != b0) << 2);
    r.cls = (hx && hy && hz)
                ? (b0 | (bx << 1) | (by << 2) | (bxy << 3) | (bz << 4) | (bxz << 5) | (byz << 6) | (bxyz << 7))
                : 0;
    return r;
}

__device__ __forceinline__ int ntri_of(int cls) { return (cls == 0 || cls == 255) ? 0 : c_ntri[cls]; }

// Loads of one segment (issued before any of them is used).
struct SegLoads {
    float4 r00, r10, r01, r11;
    float e[4];
};

__device__ __forceinline__ SegLoads seg_issue(const float* __restrict__ A, int64_t rowbase, int x0, int nx,
                                              int64_t sy, int64_t sz, bool hy, bool hz) {
    const int lane = threadIdx.x & 31;
    const int x = x0 + 4 * lane;
    const bool valid = x < nx;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    SegLoads l;
    l.r00 = valid ? *reinterpret_cast<const float4*>(A + rowbase + x) : z4;
    l.r10 = (valid && hy) ? *reinterpret_cast<const float4*>(A + rowbase + x + sy) : z4;
    l.r01 = (valid && hz) ? *reinterpret_cast<const float4*>(A + rowbase + x + sz) : z4;
    l.r11 = (valid && hy && hz) ? *reinterpret_cast<const float4*>(A + rowbase + x + sy + sz) : z4;
    const bool more = lane == 31 && x + 4 < nx;
    const int64_t n = rowbase + x + 4;
    l.e[0] = more ? A[n] : 0.f;
    l.e[1] = (more && hy) ? A[n + sy] : 0.f;
    l.e[2] = (more && hz) ? A[n + sz] : 0.f;
    l.e[3] = (more && hy && hz) ? A[n + sy + sz] : 0.f;
    return l;
}

__device__ __forceinline__ Seg4 seg_bits_of(const SegLoads& l, int x0, int nx, bool hy, bool hz, float L) {
    const int lane = threadIdx.x & 31;
    const int x = x0 + 4 * lane;
    const bool valid = x < nx;
    Seg4 s;
    s.bits[0] = valid ? nib(l.r00, L) : 0;
    s.bits[1] = (valid && hy) ? nib(l.r10, L) : 0;
    s.bits[2] = (valid && hz) ? nib(l.r01, L) : 0;
    s.bits[3] = (valid && hy && hz) ? nib(l.r11, L) : 0;
    int nb[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) nb[r] = __shfl_down_sync(0xffffffffu, s.bits[r], 1) & 1;
    if (lane == 31) {
        const bool more = x + 4 < nx;
        nb[0] = more && l.e[0] >= L;
        nb[1] = more && hy && l.e[1] >= L;
        nb[2] = more && hz && l.e[2] >= L;
        nb[3] = more && hy && hz && l.e[3] >= L;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) s.bits[r] |= nb[r] << 4;
    return s;
}

template <int SEGS>
__global__ void __launch_bounds__(kMcThreads) k_mc_count(GridDev g, const float* __restrict__ A,
                                                         const float* __restrict__ levelf, int* __restrict__ cnt,
                                                         int nrows) {
    const float L = levelf[0];
    const int row = blockIdx.x * kRowsPerCta + (threadIdx.x >> 5);
    if (row >= nrows) return;                    // warp-uniform
    const int lane = threadIdx.x & 31;
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int y = row % ny, z = row / ny;
    const bool hy = y < ny - 1, hz = z < nz - 1;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const int64_t rowbase = (int64_t)row * nx;
    SegLoads ld[SEGS];
#pragma unroll
    for (int k = 0; k < SEGS; ++k) ld[k] = seg_issue(A, rowbase, 128 * k, nx, sy, sz, hy, hz);
    int na = 0, nv = 0, nt = 0;
#pragma unroll
    for (int k = 0; k < SEGS; ++k) {
        const int x0 = 128 * k;
        const Seg4 sb = seg_bits_of(ld[k], x0, nx, hy, hz, L);
        const int xl = x0 + 4 * lane;
        // all four rows agree on all five bits: no edge or cell changes here
        const int all = sb.bits[0] & sb.bits[1] & sb.bits[2] & sb.bits[3];
        const int any = sb.bits[0] | sb.bits[1] | sb.bits[2] | sb.bits[3];
        if (xl < nx && !(all == 0x1f || any == 0)) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const NodeInfo ni = seg_node(sb, j, xl + j, nx, hy, hz);
                const int t = ntri_of(ni.cls);
                na += (ni.flags != 0 || t > 0);
                nv += __popc(ni.flags);
                nt += t;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        na += __shfl_down_sync(0xffffffffu, na, o);
        nv += __shfl_down_sync(0xffffffffu, nv, o);
        nt += __shfl_down_sync(0xffffffffu, nt, o);
    }
    if (lane == 0) {
        cnt[row] = na;
        cnt[nrows + row] = nv;
        cnt[2 * nrows + row] = nt;
    }
}

// Block-wide exclusive scan of 3 ints (kMcThreads threads); returns totals.
__device__ __forceinline__ int3 block_scan3(int3 v, int3& total, int3* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int3 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int a = __shfl_up_sync(0xffffffffu, inc.x, o);
        const int b = __shfl_up_sync(0xffffffffu, inc.y, o);
        const int c = __shfl_up_sync(0xffffffffu, inc.z, o);
        if (lane >= o) {
            inc.x += a;
            inc.y += b;
            inc.z += c;
        }
    }
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int3 w = lane < kMcThreads / 32 ? sh[lane] : make_int3(0, 0, 0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, w.x, o);
            const int b = __shfl_up_sync(0xffffffffu, w.y, o);
            const int c = __shfl_up_sync(0xffffffffu, w.z, o);
            if (lane >= o) {
                w.x += a;
                w.y += b;
                w.z += c;
            }
        }
        if (lane < kMcThreads / 32) sh[lane] = w;
    }
    __syncthreads();
    const int3 before = wid ? sh[wid - 1] : make_int3(0, 0, 0);
    total = sh[kMcThreads / 32 - 1];
    __syncthreads();
    return make_int3(before.x + inc.x - v.x, before.y + inc.y - v.y, before.z + inc.z - v.z);
}

// Exclusive scan of the three row-count arrays (length nb) in tiles of
// kScanTile: tile sums, one CTA over the tile sums, then each tile writes
// off[a * (nb + 1) + i]; totals go to off[a * (nb + 1) + nb].
constexpr int kScanTile = 2048;

__global__ void __launch_bounds__(kMcThreads) k_mc_tile_sums(const int* __restrict__ blk, int nb, int3* tile) {
    __shared__ int3 sh[kMcThreads / 32];
    int3 v = make_int3(0, 0, 0);
    for (int k = 0; k < kScanTile / kMcThreads; ++k) {
        const int i = blockIdx.x * kScanTile + k * kMcThreads + threadIdx.x;
        if (i < nb) {
            v.x += blk[i];
            v.y += blk[nb + i];
            v.z += blk[2 * nb + i];
        }
    }
    int3 tot;
    block_scan3(v, tot, sh);
    if (threadIdx.x == 0) tile[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kMcThreads) k_mc_tile_scan(int3* tile, int ntiles, int nb, int* off) {
    __shared__ int3 sh[kMcThreads / 32];
    int3 carry = make_int3(0, 0, 0);
    for (int base = 0; base < ntiles; base += kMcThreads) {
        const int i = base + threadIdx.x;
        const int3 v = i < ntiles ? tile[i] : make_int3(0, 0, 0);
        int3 tot;
        const int3 ex = block_scan3(v, tot, sh);
        if (i < ntiles) tile[i] = make_int3(carry.x + ex.x, carry.y + ex.y, carry.z + ex.z);
        carry.x += tot.x;
        carry.y += tot.y;
        carry.z += tot.z;
    }
    if (threadIdx.x == 0) {
        off[nb] = carry.x;
        off[(nb + 1) + nb] = carry.y;
        off[2 * (nb + 1) + nb] = carry.z;
        off[3 * (nb + 1) + 0] = carry.x;     // totals for the host
        off[3 * (nb + 1) + 1] = carry.y;
        off[3 * (nb + 1) + 2] = carry.z;
    }
}

__global__ void __launch_bounds__(kMcThreads) k_mc_tile_write(const int* __restrict__ blk, int nb,
                                                              const int3* __restrict__ tile, int* off) {
    __shared__ int3 sh[kMcThreads / 32];
    int3 run = tile[blockIdx.x];
    for (int k = 0; k < kScanTile / kMcThreads; ++k) {
        const int i = blockIdx.x * kScanTile + k * kMcThreads + threadIdx.x;
        const int3 v = i < nb ? make_int3(blk[i], blk[nb + i], blk[2 * nb + i]) : make_int3(0, 0, 0);
        int3 tot;
        const int3 ex = block_scan3(v, tot, sh);
        if (i < nb) {
            off[i] = run.x + ex.x;
            off[(nb + 1) + i] = run.y + ex.y;
            off[2 * (nb + 1) + i] = run.z + ex.z;
        }
        run.x += tot.x;
        run.y += tot.y;
        run.z += tot.z;
    }
}

__device__ __forceinline__ float grad_axis(const float* __restrict__ A, int64_t n, int q, int nq, int64_t stride,
                                           float inv_h) {
    if (q == 0) return (A[n + stride] - A[n]) * inv_h;
    if (q == nq - 1) return (A[n] - A[n - stride]) * inv_h;
    return (A[n + stride] - A[n - stride]) * (0.5f * inv_h);
}

// Vertices on the crossing edges of node n: t = (L - A0) / (A1 - A0) and the
// position p(q) + t h_a e_a, in float32 (no decision depends on them; the
// error is a few float32 ulps of the coordinates), normal = -grad A lerped.
__device__ __forceinline__ void emit_vertices(const GridDev& g, const float* __restrict__ A, float Ln,
                                              int64_t n, const int q[3], int flags, int vi, int cap_v,
                                              float* __restrict__ verts, float* __restrict__ vnrm) {
    const int nn[3] = {g.n[0], g.n[1], g.n[2]};
    const int64_t st[3] = {1, (int64_t)g.n[0], (int64_t)g.n[0] * g.n[1]};
    float g0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) g0[c] = grad_axis(A, n, q[c], nn[c], st[c], g.inv_hf[c]);
    for (int a = 0; a < 3; ++a) {
        if (!((flags >> a) & 1)) continue;
        const int64_t n1 = n + st[a];
        const float a0 = A[n], a1 = A[n1];
        const float tt = (Ln - a0) / (a1 - a0);
        int q1[3] = {q[0], q[1], q[2]};
        q1[a] += 1;
        float g1[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) g1[c] = grad_axis(A, n1, q1[c], nn[c], st[c], g.inv_hf[c]);
        float p[3], nv[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float qc = (float)q[c] + 0.5f + (c == a ? tt : 0.0f);
            p[c] = fmaf(qc, g.hf[c], g.bminf[c]);
            nv[c] = -((1.0f - tt) * g0[c] + tt * g1[c]);
        }
        const float len2 = nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2];
        const float inv = len2 > 0.f ? rsqrtf(len2) : 0.f;
        if (vi >= cap_v) return;   // buffers too small: the host grows them and runs again
        verts[3 * (int64_t)vi + 0] = p[0];
        verts[3 * (int64_t)vi + 1] = p[1];
        verts[3 * (int64_t)vi + 2] = p[2];
        vnrm[3 * (int64_t)vi + 0] = nv[0] * inv;
        vnrm[3 * (int64_t)vi + 1] = nv[1] * inv;
        vnrm[3 * (int64_t)vi + 2] = nv[2] * inv;
        ++vi;
    }
}

__global__ void __launch_bounds__(kMcThreads) k_mc_emit(GridDev g, const float* __restrict__ A,
                                                        const float* __restrict__ levelf,
                                                        const int* __restrict__ cnt, const int* __restrict__ off,
                                                        int nrows, int4* __restrict__ nodes, int cap_nodes,
                                                        float* __restrict__ verts, float* __restrict__ vnrm,
                                                        int cap_v) {
    const int row = blockIdx.x * kRowsPerCta + (threadIdx.x >> 5);
    if (row >= nrows || cnt[row] == 0) return;   // warp-uniform: no surface on this row
    const int lane = threadIdx.x & 31;
    const float L = levelf[0];
    const float Ln = levelf[1];
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int y = row % ny, z = row / ny;
    const bool hy = y < ny - 1, hz = z < nz - 1;
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    const int64_t rowbase = (int64_t)row * nx;
    int ia = off[row];
    int iv = off[(nrows + 1) + row];
    int it = off[2 * (nrows + 1) + row];
    for (int x0 = 0; x0 < nx; x0 += 128) {
        const Seg4 sb = seg_load(A, rowbase, x0, nx, sy, sz, hy, hz, L);
        const int xl = x0 + 4 * lane;
        NodeInfo ni[4];
        int ca = 0, cv = 0, ct = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            ni[j].flags = 0;
            ni[j].cls = 0;
            if (xl < nx) ni[j] = seg_node(sb, j, xl + j, nx, hy, hz);
            const int t = ntri_of(ni[j].cls);
            ca += (ni[j].flags != 0 || t > 0);
            cv += __popc(ni[j].flags);
            ct += t;
        }
        // exclusive prefix over lanes (x order), then in-lane order j
        int pa = ca, pv = cv, pt = ct;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int a = __shfl_up_sync(0xffffffffu, pa, o);
            const int b = __shfl_up_sync(0xffffffffu, pv, o);
            const int c = __shfl_up_sync(0xffffffffu, pt, o);
            if (lane >= o) {
                pa += a;
                pv += b;
                pt += c;
            }
        }
        const int ta = __shfl_sync(0xffffffffu, pa, 31);
        const int tv = __shfl_sync(0xffffffffu, pv, 31);
        const int tt = __shfl_sync(0xffffffffu, pt, 31);
        int ja = ia + pa - ca, jv = iv + pv - cv, jt = it + pt - ct;
        if (ca > 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int t = ntri_of(ni[j].cls);
                if (ni[j].flags == 0 && t == 0) continue;
                const int64_t n = rowbase + xl + j;
                if (ja < cap_nodes) nodes[ja] = make_int4((int)n, ni[j].flags | (ni[j].cls << 8), jv, jt);
                ++ja;
                if (ni[j].flags) {
                    const int q[3] = {xl + j, y, z};
                    emit_vertices(g, A, Ln, n, q, ni[j].flags, jv, cap_v, verts, vnrm);
                }
                jv += __popc(ni[j].flags);
                jt += t;
            }
        }
        ia += ta;
        iv += tv;
        it += tt;
    }
}

// The owner of a triangle corner is this node or a node of the same row
// (+x), of the next row (+y) or of the next plane (+z): its record is found
// by a short scan of that row's records, whose range comes from the row
// offsets of the scan (off_rows[row] .. off_rows[row + 1]).
__device__ __forceinline__ void tris_of_node(const GridDev& g, const int4* __restrict__ nodes, int r,
                                                  const int* __restrict__ off_rows, int32_t* __restrict__ tris) {
    const int4 rec = nodes[r];
    const int cls = rec.y >> 8;
    const int nt = ntri_of(cls);
    if (nt == 0) return;
    const int nx = g.n[0], ny = g.n[1];
    const int row = rec.x / nx;
    const int x = rec.x - row * nx;
    for (int t = 0; t < nt; ++t) {
        for (int j = 0; j < 3; ++j) {
            const int e = c_tri[cls][t][j];
            const int axis = e >> 2;
            const int cu = e & 1, cv = (e >> 1) & 1;
            // owner offset: the edge's fixed coordinates on the two other axes
            const int ox = axis == 0 ? 0 : cu;
            const int oy = axis == 1 ? 0 : (axis == 0 ? cu : cv);
            const int oz = axis == 2 ? 0 : cv;
            int4 orec = rec;
            if (ox | oy | oz) {
                const int orow = row + oy + ny * oz;
                const int ox_node = x + ox;
                int k = off_rows[orow];
                const int kend = off_rows[orow + 1];
                while (k < kend - 1 && nodes[k].x - orow * nx < ox_node) ++k;
                orec = nodes[k];
            }
            const int below = (orec.y & 7) & ((1 << axis) - 1);
            tris[3 * (int64_t)(rec.w + t) + j] = orec.z + __popc(below);
        }
    }
}

__global__ void __launch_bounds__(256) k_mc_tris(GridDev g, const int4* __restrict__ nodes,
                                                 const int* __restrict__ totals, int cap_nodes, int cap_tris,
                                                 const int* __restrict__ off_rows, int32_t* __restrict__ tris) {
    const int n_nodes = totals[0];
    if (n_nodes > cap_nodes || totals[2] > cap_tris) return;   // the host grows the buffers and runs again
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_nodes; r += gridDim.x * blockDim.x)
        tris_of_node(g, nodes, r, off_rows, tris);
}

__global__ void k_mc_classes(GridDev g, const float* __restrict__ A, const float* __restrict__ levelf,
                             uint8_t* out) {
    const int cx = g.n[0] - 1, cy = g.n[1] - 1, cz = g.n[2] - 1;
    const int64_t ncell = (int64_t)cx * cy * cz;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ncell) return;
    const int z = (int)(i / ((int64_t)cx * cy));
    const int rem = (int)(i - (int64_t)z * cx * cy);
    const int y = rem / cx;
    const int x = rem - y * cx;
    const int64_t n = x + (int64_t)g.n[0] * (y + (int64_t)g.n[1] * z);
    out[i] = (uint8_t)classify_node(A, n, x, y, z, g, levelf[0]).cls;
}

}  // namespace

cudaError_t mc_init() {
    int32_t ntri[256];
    int32_t tris[256 * kMaxTrisPerCase * 3];
    mc_generate_table(ntri, tris);
    signed char t8[256][kMaxTrisPerCase][3];
    for (int c = 0; c < 256; ++c)
        for (int t = 0; t < kMaxTrisPerCase; ++t)
            for (int j = 0; j < 3; ++j) t8[c][t][j] = (signed char)tris[(c * kMaxTrisPerCase + t) * 3 + j];
    cudaError_t e = cudaMemcpyToSymbol(c_ntri, ntri, sizeof(ntri));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(c_tri, t8, sizeof(t8));
}

cudaError_t launch_mc_count(ftr_ctx* c) {
    const int nr = c->mc_blocks;              // grid rows n_y n_z
    const int ctas = (nr + kRowsPerCta - 1) / kRowsPerCta;
    prof_begin(c, ST_MC_COUNT);
    switch ((c->g.n[0] + 127) / 128) {
        case 1: k_mc_count<1><<<ctas, kMcThreads, 0, c->stream>>>(c->g, c->d_A, c->d_levelf, c->d_mc_blk, nr); break;
        case 2: k_mc_count<2><<<ctas, kMcThreads, 0, c->stream>>>(c->g, c->d_A, c->d_levelf, c->d_mc_blk, nr); break;
        case 3: k_mc_count<3><<<ctas, kMcThreads, 0, c->stream>>>(c->g, c->d_A, c->d_levelf, c->d_mc_blk, nr); break;
        default: k_mc_count<4><<<ctas, kMcThreads, 0, c->stream>>>(c->g, c->d_A, c->d_levelf, c->d_mc_blk, nr); break;
    }
    c->launches++;
    cudaError_t e = cudaGetLastError();
    prof_end(c, ST_MC_COUNT);
    if (e != cudaSuccess) return e;
    prof_begin(c, ST_MC_SCAN);
    const int ntiles = (nr + kScanTile - 1) / kScanTile;
    k_mc_tile_sums<<<ntiles, kMcThreads, 0, c->stream>>>(c->d_mc_blk, nr, c->d_mc_tile);
    k_mc_tile_scan<<<1, kMcThreads, 0, c->stream>>>(c->d_mc_tile, ntiles, nr, c->d_mc_off);
    k_mc_tile_write<<<ntiles, kMcThreads, 0, c->stream>>>(c->d_mc_blk, nr, c->d_mc_tile, c->d_mc_off);
    c->launches += 3;
    e = cudaGetLastError();
    prof_end(c, ST_MC_SCAN);
    if (e != cudaSuccess) return e;
    return cudaMemcpyAsync(c->h_mc_tot, c->d_mc_off + 3 * (nr + 1), 3 * sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream);
}

cudaError_t launch_mc_emit(ftr_ctx* c) {
    const int nr = c->mc_blocks;
    const int ctas = (nr + kRowsPerCta - 1) / kRowsPerCta;
    prof_begin(c, ST_MC_EMIT);
    k_mc_emit<<<ctas, kMcThreads, 0, c->stream>>>(c->g, c->d_A, c->d_levelf, c->d_mc_blk, c->d_mc_off, nr,
                                                  c->d_mc_nodes, (int)c->cap_mc_nodes, c->d_verts, c->d_vnrm,
                                                  (int)c->cap_verts);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    prof_end(c, ST_MC_EMIT);
    if (e != cudaSuccess) return e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    prof_begin(c, ST_MC_TRIS);
    k_mc_tris<<<(sms > 0 ? sms : 152) * 4, 256, 0, c->stream>>>(c->g, c->d_mc_nodes, c->d_mc_off + 3 * (nr + 1),
                                                                 (int)c->cap_mc_nodes, (int)c->cap_tris,
                                                                 c->d_mc_off, c->d_tris);
    c->launches++;
    e = cudaGetLastError();
    prof_end(c, ST_MC_TRIS);
    return e;
}

cudaError_t launch_mc_classes(ftr_ctx* c, uint8_t* out_dev) {
    const int64_t ncell = (int64_t)(c->g.n[0] - 1) * (c->g.n[1] - 1) * (c->g.n[2] - 1);
    k_mc_classes<<<(unsigned)((ncell + 255) / 256), 256, 0, c->stream>>>(c->g, c->d_A, c->d_levelf, out_dev);
    c->launches++;
    return cudaGetLastError();
}

}  // namespace ftr
