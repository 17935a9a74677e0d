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
// The inside bits are computed once (one warp per grid row, one ballot per
// 32 nodes: 1 bit per node, 2 MB at 256^3) and both passes below work on
// 32-node words: a thread takes word w of row (y, z) and the same word of
// the rows (y+1, z), (y, z+1), (y+1, z+1); XORs give the crossing edges
// toward +x, +y, +z and AND/OR of the eight corner masks the cells whose
// corners differ (exactly the cells with triangles).  Launches:
//   bits   the inside bits of every node
//   count  per tile of (row, word) threads: active nodes (owning a vertex
//          or lower corner of a cell with triangles), vertices, triangles;
//          also summed per group of 256 tiles
//   emit   per tile: its offset from the group and tile sums before it, a
//          CTA scan of its counts, the rows' offsets, per active node in x
//          order one 16-byte record (node, edge bits | class << 8, first
//          vertex, first triangle), and per word with active nodes its first
//          record index and active mask (a tile with no active node writes
//          only its rows' offsets)
//   tris   one thread per active node: the vertices of its crossing edges
//          (t = (L - A0)/(A1 - A0), normal -grad A by central differences,
//          one-sided at the border, lerped), then its triangles' corners
//          from the case table; the record of an edge's owner node is its
//          word's first record plus the active nodes before it in the word.
#include <cuda_runtime.h>
#include <math.h>

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

__device__ __forceinline__ int ntri_of(int cls) { return (cls == 0 || cls == 255) ? 0 : c_ntri[cls]; }

// ---------------------------------------------------------------- bit masks
// The inside bits (A >= L) of every node, 32 per word: word w of grid row r
// (y + n_y z) holds x = 32 w .. 32 w + 31 (bit i = node 32 w + i; zero past
// n_x); rows are `wp` words apart (wp = the words per row rounded up to a
// power of two).  One warp per row, one ballot per word.
// It also zeroes `zero[0 .. nzero)` (the group sums of k_mc_count_tiles).
// rowmm (nullable): per row the minimum and maximum of A; a row whose maximum
// is below the level, or whose minimum is at or above it, gets its words
// without reading A (the same bits: every node of the row decides alike).
__global__ void __launch_bounds__(kMcThreads) k_mc_bits(GridDev g, const float* __restrict__ A,
                                                        const float* __restrict__ levelf, unsigned* __restrict__ bits,
                                                        int nrows, int wp, int* __restrict__ zero, int nzero,
                                                        const float2* __restrict__ rowmm) {
    pdl_wait();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nzero; i += gridDim.x * blockDim.x) zero[i] = 0;
    const int lane = threadIdx.x & 31;
    const float L = levelf[0];
    const int nx = g.n[0];
    const int nw = (nx + 31) >> 5;
    // one warp per row (warp-uniform); the stride covers any grid size
    for (int row = blockIdx.x * kRowsPerCta + (threadIdx.x >> 5); row < nrows; row += gridDim.x * kRowsPerCta) {
        const float* a = A + (int64_t)row * nx;
        if (rowmm) {
            const float2 mm = rowmm[row];
            if (mm.y < L || mm.x >= L) {            // false for NaN bounds
                if (lane < wp) {
                    unsigned word = 0u;
                    if (lane < nw && mm.x >= L) word = (32 * (lane + 1) <= nx) ? 0xffffffffu : ((1u << (nx - 32 * lane)) - 1u);
                    bits[(int64_t)row * wp + lane] = word;
                }
                continue;
            }
        }
        unsigned mine = 0u;
        // up to 8 words per batch: all loads are issued before the first ballot
        for (int w0 = 0; w0 < nw; w0 += 8) {
            float v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int x = 32 * (w0 + k) + lane;
                v[k] = (w0 + k < nw && x < nx) ? a[x] : -INFINITY;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const unsigned b = __ballot_sync(0xffffffffu, v[k] >= L);
                if (lane == w0 + k) mine = b;
            }
        }
        if (lane < wp) bits[(int64_t)row * wp + lane] = lane < nw ? mine : 0u;
    }
}

// Per (row, word): the masks of the nodes of word w that own a crossing
// edge toward +x, +y, +z, and that are the lower corner of a cell whose
// corners are not all on one side ("mixed": exactly the cells with
// triangles).  Nodes with any of the four are the row's active nodes.
struct WordMasks {
    unsigned ex, ey, ez, mixed;
    unsigned c[8];   // corner bits of the cells whose lower corner is in the word
};

__device__ __forceinline__ WordMasks word_masks(const unsigned* __restrict__ bits, int row, int w, int nw, int wp,
                                                int x_count, bool hy, bool hz, int ny) {
    const int64_t r00 = (int64_t)row * wp, r10 = r00 + wp, r01 = r00 + (int64_t)ny * wp, r11 = r01 + wp;
    const bool more = w + 1 < nw;
    const unsigned b00 = bits[r00 + w], n00 = more ? bits[r00 + w + 1] : 0u;
    const unsigned b10 = hy ? bits[r10 + w] : 0u, n10 = (hy && more) ? bits[r10 + w + 1] : 0u;
    const unsigned b01 = hz ? bits[r01 + w] : 0u, n01 = (hz && more) ? bits[r01 + w + 1] : 0u;
    const unsigned b11 = (hy && hz) ? bits[r11 + w] : 0u, n11 = (hy && hz && more) ? bits[r11 + w + 1] : 0u;
    // nodes of the word that exist, and those with a +x neighbour
    const int base = 32 * w;
    const unsigned valid = x_count - base >= 32 ? 0xffffffffu : ((1u << (x_count - base)) - 1u);
    const unsigned vx = x_count - 1 - base >= 32 ? 0xffffffffu
                        : (x_count - 1 - base <= 0 ? 0u : ((1u << (x_count - 1 - base)) - 1u));
    WordMasks m;
    m.c[0] = b00;
    m.c[1] = (b00 >> 1) | (n00 << 31);
    m.c[2] = b10;
    m.c[3] = (b10 >> 1) | (n10 << 31);
    m.c[4] = b01;
    m.c[5] = (b01 >> 1) | (n01 << 31);
    m.c[6] = b11;
    m.c[7] = (b11 >> 1) | (n11 << 31);
    m.ex = (m.c[0] ^ m.c[1]) & vx;
    m.ey = hy ? ((b00 ^ b10) & valid) : 0u;
    m.ez = hz ? ((b00 ^ b01) & valid) : 0u;
    unsigned all = 0xffffffffu, any = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        all &= m.c[k];
        any |= m.c[k];
    }
    m.mixed = (hy && hz) ? ((any & ~all) & vx) : 0u;
    return m;
}

__device__ __forceinline__ int cell_class(const WordMasks& m, int i) {
    int cls = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) cls |= (int)((m.c[k] >> i) & 1u) << k;
    return cls;
}

// Block-wide exclusive scan of 3 ints (T threads); returns totals.
template <int T>
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
        int3 w = lane < T / 32 ? sh[lane] : make_int3(0, 0, 0);
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
        if (lane < T / 32) sh[lane] = w;
    }
    __syncthreads();
    const int3 before = wid ? sh[wid - 1] : make_int3(0, 0, 0);
    total = sh[T / 32 - 1];
    __syncthreads();
    return make_int3(before.x + inc.x - v.x, before.y + inc.y - v.y, before.z + inc.z - v.z);
}

// ------------------------------------------------- tiles: count, then emit
// Both kernels run over the (row, word) threads in node order in the same
// tiles of T threads (the context's marching-cubes tile size: 128, 256 or
// 512; the mesh does not depend on it).  The count kernel writes each tile's sums (active
// nodes, vertices, triangles) and adds them into its group's sums (256 tiles
// per group; integer atomics, so the order does not matter).  The emit
// kernel's tile gets its offset from the groups before it and the tiles
// before it in its group (at most 255 + a few loads, spread over the CTA),
// scans its own counts, and writes its rows' offsets and its node records.
//
// Tile state (agg) and group sums (sup, zeroed by k_mc_bits) as int4: active
// nodes, vertices, triangles, unused.
struct WordCounts {
    WordMasks m;
    unsigned act;
    int3 c;
};

__device__ __forceinline__ WordCounts word_counts(const GridDev& g, const unsigned* __restrict__ bits, int64_t t,
                                                  int nrows, int wp, const unsigned char* s_ntri) {
    WordCounts r;
    r.act = 0u;
    r.c = make_int3(0, 0, 0);
    const int row = (int)(t / wp), w = (int)(t % wp);
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int nw = (nx + 31) >> 5;
    if (row < nrows && w < nw) {
        const int y = row % ny, z = row / ny;
        r.m = word_masks(bits, row, w, nw, wp, nx, y < ny - 1, z < nz - 1, ny);
        r.act = r.m.ex | r.m.ey | r.m.ez | r.m.mixed;
        r.c.x = __popc(r.act);
        r.c.y = __popc(r.m.ex) + __popc(r.m.ey) + __popc(r.m.ez);
        unsigned mm = r.m.mixed;
        while (mm) {
            const int i = __ffs(mm) - 1;
            mm &= mm - 1;
            r.c.z += s_ntri[cell_class(r.m, i)];
        }
    }
    return r;
}

constexpr int kMcGroup = 256;     // tiles per group sum

template <int T>
__global__ void __launch_bounds__(T) k_mc_count_tiles(GridDev g, const unsigned* __restrict__ bits,
                                                               int nrows, int wp, int4* __restrict__ agg,
                                                               int* __restrict__ sup) {
    pdl_wait();
    __shared__ unsigned char s_ntri[256];
    __shared__ int3 sh[T / 32];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) s_ntri[k] = (unsigned char)c_ntri[k];
    __syncthreads();
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const WordCounts wc = word_counts(g, bits, t, nrows, wp, s_ntri);
    int3 tot;
    block_scan3<T>(wc.c, tot, sh);
    if (threadIdx.x == 0) {
        agg[blockIdx.x] = make_int4(tot.x, tot.y, tot.z, 0);
        int* s = sup + 4 * (blockIdx.x / kMcGroup);
        if (tot.x) atomicAdd(&s[0], tot.x);
        if (tot.y) atomicAdd(&s[1], tot.y);
        if (tot.z) atomicAdd(&s[2], tot.z);
    }
}

template <int T>
__global__ void __launch_bounds__(T) k_mc_emit_tiles(GridDev g, const unsigned* __restrict__ bits,
                                                              int nrows, int wp, int ntiles,
                                                              const int4* __restrict__ agg,
                                                              const int4* __restrict__ sup, int* __restrict__ off,
                                                              int4* __restrict__ nodes, int cap_nodes,
                                                              int2* __restrict__ wordinfo) {
    pdl_wait();
    __shared__ unsigned char s_ntri[256];
    __shared__ int3 sh[T / 32];
    for (int k = threadIdx.x; k < 256; k += blockDim.x) s_ntri[k] = (unsigned char)c_ntri[k];
    // the sums of every tile before this one: whole groups, then this group's tiles
    const int tile = blockIdx.x, grp = tile / kMcGroup;
    int3 pre = make_int3(0, 0, 0);
    for (int k = threadIdx.x; k < grp; k += blockDim.x) {
        const int4 v = sup[k];
        pre.x += v.x;
        pre.y += v.y;
        pre.z += v.z;
    }
    for (int k = grp * kMcGroup + threadIdx.x; k < tile; k += blockDim.x) {
        const int4 v = agg[k];
        pre.x += v.x;
        pre.y += v.y;
        pre.z += v.z;
    }
    __syncthreads();
    int3 base;
    block_scan3<T>(pre, base, sh);
    const int64_t t = (int64_t)tile * blockDim.x + threadIdx.x;
    // a tile the count found empty (most of the grid) has only its rows'
    // offsets to write
    const int4 mine = agg[tile];
    WordCounts wc;
    int3 tot = make_int3(0, 0, 0), ex = make_int3(0, 0, 0);
    if ((mine.x | mine.y | mine.z) != 0) {
        wc = word_counts(g, bits, t, nrows, wp, s_ntri);
        ex = block_scan3<T>(wc.c, tot, sh);
    } else {
        wc.act = 0u;
    }
    const int row = (int)(t / wp), w = (int)(t % wp);
    int ja = base.x + ex.x, jv = base.y + ex.y, jt = base.z + ex.z;
    if (w == 0 && row < nrows) {
        off[row] = ja;
        off[(nrows + 1) + row] = jv;
        off[2 * (nrows + 1) + row] = jt;
    }
    if (tile == ntiles - 1 && threadIdx.x == 0) {
        const int3 all = make_int3(base.x + tot.x, base.y + tot.y, base.z + tot.z);
        off[nrows] = all.x;
        off[(nrows + 1) + nrows] = all.y;
        off[2 * (nrows + 1) + nrows] = all.z;
        off[3 * (nrows + 1) + 0] = all.x;     // totals for the host
        off[3 * (nrows + 1) + 1] = all.y;
        off[3 * (nrows + 1) + 2] = all.z;
    }
    // the word's first record and its active nodes: the triangle pass finds
    // a corner's owner record from these without scanning the row
    if (wc.act) wordinfo[t] = make_int2(ja, (int)wc.act);
    const int64_t rowbase = (int64_t)row * g.n[0];
    unsigned rem = wc.act;
    while (rem) {
        const int i = __ffs(rem) - 1;
        rem &= rem - 1;
        const int flags = (int)((wc.m.ex >> i) & 1u) | ((int)((wc.m.ey >> i) & 1u) << 1) |
                          ((int)((wc.m.ez >> i) & 1u) << 2);
        const int cls = ((wc.m.mixed >> i) & 1u) ? cell_class(wc.m, i) : 0;
        if (ja < cap_nodes) nodes[ja] = make_int4((int)(rowbase + 32 * w + i), flags | (cls << 8), jv, jt);
        ++ja;
        jv += __popc(flags);
        jt += cls ? s_ntri[cls] : 0;
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

// The owner of a triangle corner is this node or a node of the same row
// (+x), of the next row (+y) or of the next plane (+z).  The owner is active
// (it owns the crossing edge), so its word was written by the emit pass:
// its record index is the word's first record plus the active nodes before
// it in the word.
__device__ __forceinline__ void tris_of_node(const GridDev& g, const int4* __restrict__ nodes, int r,
                                             const int2* __restrict__ wordinfo, int wp, int n_nodes,
                                             int32_t* __restrict__ tris) {
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
                const int2 wi = wordinfo[(int64_t)orow * wp + (ox_node >> 5)];
                const unsigned before = (unsigned)wi.y & ((1u << (ox_node & 31)) - 1u);
                // clamped: an inconsistent lookup gives a wrong index, never an access outside the records
                orec = nodes[min(max(wi.x + __popc(before), 0), n_nodes - 1)];
            }
            const int below = (orec.y & 7) & ((1 << axis) - 1);
            tris[3 * (int64_t)(rec.w + t) + j] = orec.z + __popc(below);
        }
    }
}

// One thread per node record: the vertices on its crossing edges, then its
// triangles.
__global__ void __launch_bounds__(256) k_mc_tris(GridDev g, const float* __restrict__ A,
                                                 const float* __restrict__ levelf, const int4* __restrict__ nodes,
                                                 const int* __restrict__ totals, int cap_nodes, int cap_tris,
                                                 const int2* __restrict__ wordinfo, int wp,
                                                 int32_t* __restrict__ tris, float* __restrict__ verts,
                                                 float* __restrict__ vnrm, int cap_v) {
    pdl_wait();
    const int n_nodes = totals[0];
    if (n_nodes > cap_nodes || totals[2] > cap_tris) return;   // the host grows the buffers and runs again
    const float Ln = levelf[1];
    const int nx = g.n[0], ny = g.n[1];
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_nodes; r += gridDim.x * blockDim.x) {
        const int4 rec = nodes[r];
        const int flags = rec.y & 7;
        if (flags) {
            const int row = rec.x / nx;
            const int q[3] = {rec.x - row * nx, row % ny, row / ny};
            emit_vertices(g, A, Ln, (int64_t)rec.x, q, flags, rec.z, cap_v, verts, vnrm);
        }
        tris_of_node(g, nodes, r, wordinfo, wp, n_nodes, tris);
    }
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

// Words per grid row of the inside bits, rounded up to a power of two.
static int mc_words(int nx) {
    const int nw = (nx + 31) / 32;
    int wp = 1;
    while (wp < nw) wp <<= 1;
    return wp;
}

// Tiles of T (row, word) threads (T = the context's marching-cubes tile size),
// and where the tile sums and the
// group sums sit in the per-row count buffer (3 x n_rows ints: room for both
// with up to 16 words per row, every supported grid).
static int mc_tiles(int nrows, int wp, int t) { return (int)(((int64_t)nrows * wp + t - 1) / t); }
static int mc_groups(int ntiles) { return (ntiles + kMcGroup - 1) / kMcGroup; }

// CTAs of the inside-bit pass: one warp per row.  (A grid of one resident
// wave taking rows in a stride was as fast for one frame and 4-7 % slower
// when frames of several contexts overlap: short CTAs fill in around other
// kernels' CTAs.)
static unsigned mc_bits_grid(int nrows) { return (unsigned)((nrows + kRowsPerCta - 1) / kRowsPerCta); }

cudaError_t launch_mc_bits(ftr_ctx* c) {
    const int nr = c->mc_blocks;
    launch_pdl(k_mc_bits, mc_bits_grid(nr), kMcThreads, 0, c->stream, c->g, c->d_A, c->d_levelf,
               c->d_mc_bits, nr, mc_words(c->g.n[0]), (int*)nullptr, 0,
               (const float2*)(c->rowmm_valid ? c->d_rowmm : nullptr));
    c->launches++;
    return cudaGetLastError();
}

int mc_words_per_row(int nx) { return mc_words(nx); }

// A launch of the count or emit kernel instantiated for the tile size T.
template <template <int> class K, class... Args>
void launch_tiles(int t, int ntiles, cudaStream_t st, Args... args) {
    switch (t) {
        case 128: launch_pdl(K<128>::fn, ntiles, 128, 0, st, args...); break;
        case 512: launch_pdl(K<512>::fn, ntiles, 512, 0, st, args...); break;
        default: launch_pdl(K<256>::fn, ntiles, 256, 0, st, args...); break;
    }
}
template <int T> struct CountK { static constexpr auto fn = k_mc_count_tiles<T>; };
template <int T> struct EmitK { static constexpr auto fn = k_mc_emit_tiles<T>; };

bool mc_plan_valid(int tile, int tris_per_sm) {
    return (tile == 128 || tile == 256 || tile == 512) && tris_per_sm >= 1 && tris_per_sm <= 16;
}

cudaError_t launch_mc_count(ftr_ctx* c) {
    const int nr = c->mc_blocks;              // grid rows n_y n_z
    const int wp = mc_words(c->g.n[0]);
    const int ntiles = mc_tiles(nr, wp, c->mc_tile);
    if (4 * (ntiles + mc_groups(ntiles)) > 3 * nr) return cudaErrorInvalidValue;
    int4* agg = reinterpret_cast<int4*>(c->d_mc_blk);
    int* sup = c->d_mc_blk + 4 * ntiles;
    prof_begin(c, ST_MC_COUNT);
    launch_pdl(k_mc_bits, mc_bits_grid(nr), kMcThreads, 0, c->stream, c->g, c->d_A, c->d_levelf,
               c->d_mc_bits, nr, wp, sup, 4 * mc_groups(ntiles),
               (const float2*)(c->rowmm_valid ? c->d_rowmm : nullptr));
    launch_tiles<CountK>(c->mc_tile, ntiles, c->stream, c->g, (const unsigned*)c->d_mc_bits, nr, wp, agg, sup);
    c->launches += 2;
    cudaError_t e = cudaGetLastError();
    prof_end(c, ST_MC_COUNT);
    return e;
}

// The three totals (active nodes, vertices, triangles) into pinned host
// memory; enqueued after the frame's last kernel so that no copy sits between
// two kernels of the frame.
cudaError_t launch_mc_totals(ftr_ctx* c) {
    const int nr = c->mc_blocks;
    return cudaMemcpyAsync(c->h_mc_tot, c->d_mc_off + 3 * (nr + 1), 3 * sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream);
}

// The rows' offsets and the node records, then the vertices and triangles.
cudaError_t launch_mc_emit(ftr_ctx* c) {
    const int nr = c->mc_blocks;
    const int wp = mc_words(c->g.n[0]);
    const int ntiles = mc_tiles(nr, wp, c->mc_tile);
    const int4* agg = reinterpret_cast<const int4*>(c->d_mc_blk);
    const int4* sup = reinterpret_cast<const int4*>(c->d_mc_blk + 4 * ntiles);
    prof_begin(c, ST_MC_EMIT);
    launch_tiles<EmitK>(c->mc_tile, ntiles, c->stream, c->g, (const unsigned*)c->d_mc_bits, nr, wp, ntiles, agg, sup,
                        c->d_mc_off, c->d_mc_nodes, (int)c->cap_mc_nodes, c->d_mc_word);
    c->launches++;
    cudaError_t e = cudaGetLastError();
    prof_end(c, ST_MC_EMIT);
    if (e != cudaSuccess) return e;
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    prof_begin(c, ST_MC_TRIS);
    launch_pdl(k_mc_tris, (sms > 0 ? sms : 152) * c->mc_tris_per_sm, 256, 0, c->stream, c->g, c->d_A, c->d_levelf, c->d_mc_nodes,
               c->d_mc_off + 3 * (nr + 1), (int)c->cap_mc_nodes, (int)c->cap_tris, (const int2*)c->d_mc_word, wp,
               c->d_tris, c->d_verts, c->d_vnrm, (int)c->cap_verts);
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
