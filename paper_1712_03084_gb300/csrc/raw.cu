// Raw reconstruction of oriented, weighted points from depth maps (Sec. III-A).
//
// Per depth view and foreground pixel u (D(u) > 0): the camera point
// x_c = ((u_x - c_x) / f_x D, (u_y - c_y) / f_y D, D); its world point
// X = R^T (x_c - t); its normal from the organised triangulation of the pixel
// grid (two triangles per 2 x 2 quad, (p00, p01, p10) and (p01, p11, p10); a
// triangle is kept iff its pixels are foreground, its largest corner depth
// difference is <= step + 3 noise z_max^2 and its area is not zero; its unit
// normal faces the camera; the pixel's normal is the normalised sum of the
// kept triangles that contain it); its confidence W = W1 W2 with
// W1 = max(<-x_c / |x_c|, N>, 0) and W2 the mean of the silhouette over a
// (2r+1)^2 window, zero outside the image.  A pixel gives a point iff it is
// foreground and lies on a kept triangle.  Points come out in row-major pixel
// order per view.
//
// A CTA takes 256 consecutive pixels of one row.  Triangle edges are formed
// from exact depth differences (x_b - x_a = ((u_b - u_a) D_b + (u_a - c_x)
// (D_b - D_a)) / f_x), so the float32 normals keep ~1e-7 relative accuracy.
// Every discrete decision (the depth-step test, the orientation flip, a zero
// normal sum) is taken in float32 and redone in float64 with the float64
// formula, operation by operation, whenever it falls within a guard band of
// its threshold.
//
// Launches per call: count (points per tile), one-CTA scan of the tile
// counts, emit (recomputes each pixel, writes the compacted points, normals,
// weights and the per-pixel confidence map).
#include <cuda_runtime.h>
#include <math.h>

#include "ftr_internal.h"

namespace ftr {

namespace {

constexpr int kRawT = 256;          // pixels per CTA (one row segment)
constexpr int kRawMaxR = 16;        // largest W2 radius

struct RawView {
    int w, h;
    float fx, fy, cx, cy;
    double fxd, fyd, cxd, cyd;
    float R[9], t[3];
    const float* depth;
    float* conf;                    // nullable: per-pixel W
    int tile_base;                  // first tile of this view in the tile arrays
    int tiles_x;
};
struct RawSet {
    int k;
    RawView v[kMaxViews];
};

// Triangle (a, b, c) given by pixel offsets; returns false when a decision is
// too close to call in float32 (the caller redoes the pixel in float64).
struct Corner {
    int du, dv;
};

// Float64 restatement of one triangle, operation by operation as the plain
// definition (no fused multiply-add): keep flag and unit camera-facing normal.
__device__ bool tri_f64(const RawView& V, int u0, int v0, const Corner (&cn)[3], double step, double noise,
                        double n_out[3]) {
    double P[3][3], Z[3];
    for (int k = 0; k < 3; ++k) {
        const int u = u0 + cn[k].du, v = v0 + cn[k].dv;
        const double D = (double)V.depth[(int64_t)v * V.w + u];
        Z[k] = D;
        P[k][0] = __dmul_rn(__ddiv_rn(__dsub_rn((double)u, V.cxd), V.fxd), D);
        P[k][1] = __dmul_rn(__ddiv_rn(__dsub_rn((double)v, V.cyd), V.fyd), D);
        P[k][2] = D;
    }
    if (!(Z[0] > 0.0 && Z[1] > 0.0 && Z[2] > 0.0)) return false;
    const double zmax = fmax(fmax(Z[0], Z[1]), Z[2]);
    const double dz = fmax(fmax(fabs(Z[0] - Z[1]), fabs(Z[1] - Z[2])), fabs(Z[0] - Z[2]));
    const double thr = __dadd_rn(step, __dmul_rn(__dmul_rn(__dmul_rn(3.0, noise), zmax), zmax));
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = __dsub_rn(P[1][c], P[0][c]);
        e2[c] = __dsub_rn(P[2][c], P[0][c]);
    }
    double n[3] = {__dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1])),
                   __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2])),
                   __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]))};
    const double ln = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(n[0], n[0]), __dmul_rn(n[1], n[1])),
                                           __dmul_rn(n[2], n[2])));
    if (!(dz <= thr) || !(ln > 0.0)) return false;
    double dot = 0.0;
    for (int c = 0; c < 3; ++c) {
        n[c] = __ddiv_rn(n[c], ln);
        const double cen = __ddiv_rn(__dadd_rn(__dadd_rn(P[0][c], P[1][c]), P[2][c]), 3.0);
        dot = __dadd_rn(dot, __dmul_rn(n[c], cen));
    }
    const double s = dot > 0.0 ? -1.0 : 1.0;
    for (int c = 0; c < 3; ++c) n_out[c] = s * n[c];
    return true;
}

// Float32 triangle: 1 kept (n_out set), 0 dropped, -1 undecided.
__device__ __forceinline__ int tri_f32(const RawView& V, int u0, int v0, const Corner (&cn)[3], float step,
                                       float noise, float n_out[3]) {
    float Z[3];
    for (int k = 0; k < 3; ++k) Z[k] = V.depth[(int64_t)(v0 + cn[k].dv) * V.w + (u0 + cn[k].du)];
    if (!(Z[0] > 0.f && Z[1] > 0.f && Z[2] > 0.f)) return 0;
    const float zmax = fmaxf(fmaxf(Z[0], Z[1]), Z[2]);
    const float dz = fmaxf(fmaxf(fabsf(Z[0] - Z[1]), fabsf(Z[1] - Z[2])), fabsf(Z[0] - Z[2]));
    const float thr = step + 3.f * noise * zmax * zmax;
    if (fabsf(dz - thr) <= 1e-5f * thr) return -1;
    if (dz > thr) return 0;
    // edges from exact depth differences
    float e[2][3];
    for (int k = 1; k < 3; ++k) {
        const float u_a = (float)(u0 + cn[0].du), v_a = (float)(v0 + cn[0].dv);
        const float du = (float)(cn[k].du - cn[0].du), dv = (float)(cn[k].dv - cn[0].dv);
        const float dd = Z[k] - Z[0];
        e[k - 1][0] = (du * Z[k] + (u_a - V.cx) * dd) / V.fx;
        e[k - 1][1] = (dv * Z[k] + (v_a - V.cy) * dd) / V.fy;
        e[k - 1][2] = dd;
    }
    float n[3] = {e[0][1] * e[1][2] - e[0][2] * e[1][1], e[0][2] * e[1][0] - e[0][0] * e[1][2],
                  e[0][0] * e[1][1] - e[0][1] * e[1][0]};
    const float ln = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    const float el = sqrtf(e[0][0] * e[0][0] + e[0][1] * e[0][1] + e[0][2] * e[0][2]) *
                     sqrtf(e[1][0] * e[1][0] + e[1][1] * e[1][1] + e[1][2] * e[1][2]);
    if (!(ln > 1e-5f * el)) return -1;            // (nearly) degenerate: float64 decides
    // orientation: n . centroid
    float cen[3];
    for (int c = 0; c < 3; ++c) cen[c] = 0.f;
    for (int k = 0; k < 3; ++k) {
        const float D = Z[k];
        cen[0] += ((float)(u0 + cn[k].du) - V.cx) / V.fx * D;
        cen[1] += ((float)(v0 + cn[k].dv) - V.cy) / V.fy * D;
        cen[2] += D;
    }
    const float dot = n[0] * cen[0] + n[1] * cen[1] + n[2] * cen[2];
    const float cl = sqrtf(cen[0] * cen[0] + cen[1] * cen[1] + cen[2] * cen[2]);
    if (fabsf(dot) <= 1e-4f * ln * cl) return -1;
    const float s = (dot > 0.f ? -1.f : 1.f) / ln;
    for (int c = 0; c < 3; ++c) n_out[c] = s * n[c];
    return 1;
}

// The six triangles containing pixel (u, v): (quad offset, family).
__device__ __forceinline__ void tri_of(int t, int& qu, int& qv, Corner (&cn)[3]) {
    // family A: (0,0) (1,0) (0,1) in (du, dv); family B: (1,0) (1,1) (0,1)
    const int fam = t < 3 ? 0 : 1;
    if (fam == 0) {
        cn[0] = {0, 0};
        cn[1] = {1, 0};
        cn[2] = {0, 1};
    } else {
        cn[0] = {1, 0};
        cn[1] = {1, 1};
        cn[2] = {0, 1};
    }
    // quads whose family-A triangle contains the pixel: (0,0) (-1,0) (0,-1);
    // family B: (-1,0) (-1,-1) (0,-1)
    const int qa[3][2] = {{0, 0}, {-1, 0}, {0, -1}};
    const int qb[3][2] = {{-1, 0}, {-1, -1}, {0, -1}};
    qu = fam == 0 ? qa[t][0] : qb[t - 3][0];
    qv = fam == 0 ? qa[t][1] : qb[t - 3][1];
}

// Camera-space unit normal of pixel (u, v); 1 = a point, 0 = none.
__device__ int pixel_normal(const RawView& V, int u, int v, float step, float noise, double stepd, double noised,
                            float n[3]) {
    if (!(V.depth[(int64_t)v * V.w + u] > 0.f)) return 0;
    float acc[3] = {0.f, 0.f, 0.f};
    bool f64 = false;
    int kept = 0;
    for (int t = 0; t < 6 && !f64; ++t) {
        int qu, qv;
        Corner cn[3];
        tri_of(t, qu, qv, cn);
        const int u0 = u + qu, v0 = v + qv;
        if (u0 < 0 || v0 < 0 || u0 >= V.w - 1 || v0 >= V.h - 1) continue;
        float tn[3];
        const int r = tri_f32(V, u0, v0, cn, step, noise, tn);
        if (r < 0) {
            f64 = true;
        } else if (r > 0) {
            ++kept;
            for (int c = 0; c < 3; ++c) acc[c] += tn[c];
        }
    }
    if (!f64) {
        if (kept == 0) return 0;
        const float l2 = acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2];
        if (l2 > 1e-6f) {          // else the unit normals (nearly) cancel: float64 decides
            const float inv = rsqrtf(l2);
            for (int c = 0; c < 3; ++c) n[c] = acc[c] * inv;
            return 1;
        }
    }
    // float64: the whole pixel
    double a[3] = {0.0, 0.0, 0.0};
    for (int t = 0; t < 6; ++t) {
        int qu, qv;
        Corner cn[3];
        tri_of(t, qu, qv, cn);
        const int u0 = u + qu, v0 = v + qv;
        if (u0 < 0 || v0 < 0 || u0 >= V.w - 1 || v0 >= V.h - 1) continue;
        double tn[3];
        if (tri_f64(V, u0, v0, cn, stepd, noised, tn))
            for (int c = 0; c < 3; ++c) a[c] = __dadd_rn(a[c], tn[c]);
    }
    const double ln = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if (!(ln > 0.0)) return 0;
    for (int c = 0; c < 3; ++c) n[c] = (float)(a[c] / ln);
    return 1;
}

__device__ __forceinline__ int block_excl_scan(int v, int& total, int* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int x = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += x;
    }
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int w = lane < kRawT / 32 ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += x;
        }
        if (lane < kRawT / 32) sh[lane] = w;
    }
    __syncthreads();
    const int before = wid ? sh[wid - 1] : 0;
    total = sh[kRawT / 32 - 1];
    __syncthreads();
    return before + inc - v;
}

__global__ void __launch_bounds__(kRawT) k_raw_count(RawSet S, float step, float noise, double stepd,
                                                     double noised, int* __restrict__ tile_cnt) {
    pdl_wait();
    __shared__ int sh[kRawT / 32];
    const RawView& V = S.v[blockIdx.z];
    const int tx = blockIdx.x, v = blockIdx.y;
    if (tx >= V.tiles_x || v >= V.h) return;       // block-uniform
    const int u = tx * kRawT + threadIdx.x;
    float n[3];
    const int p = u < V.w ? pixel_normal(V, u, v, step, noise, stepd, noised, n) : 0;
    int total;
    block_excl_scan(p, total, sh);
    if (threadIdx.x == 0) tile_cnt[V.tile_base + v * V.tiles_x + tx] = total;
}

// One CTA: exclusive scan of the tile counts in place; the total into *total.
__global__ void __launch_bounds__(1024) k_raw_scan(int* tile_cnt, int ntiles, int* total) {
    pdl_wait();
    __shared__ int sh[32];
    __shared__ int s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int base = 0; base < ntiles; base += 1024) {
        const int i = base + threadIdx.x;
        const int v = i < ntiles ? tile_cnt[i] : 0;
        int inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += x;
        }
        if (lane == 31) sh[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int w = sh[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int x = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += x;
            }
            sh[lane] = w;
        }
        __syncthreads();
        const int carry = s_carry;
        if (i < ntiles) tile_cnt[i] = carry + (wid ? sh[wid - 1] : 0) + inc - v;
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + sh[31];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = s_carry;
}

__global__ void __launch_bounds__(kRawT) k_raw_emit(RawSet S, float step, float noise, double stepd, double noised,
                                                    int radius, const int* __restrict__ tile_off,
                                                    float* __restrict__ P, float* __restrict__ N,
                                                    float* __restrict__ W) {
    pdl_wait();
    __shared__ int sh[kRawT / 32];
    __shared__ unsigned short colsum[kRawT + 2 * kRawMaxR];
    const RawView& V = S.v[blockIdx.z];
    const int tx = blockIdx.x, v = blockIdx.y;
    if (tx >= V.tiles_x || v >= V.h) return;       // block-uniform
    const int u = tx * kRawT + threadIdx.x;
    // W2: silhouette counts of the window columns, then the horizontal window
    const int x0 = tx * kRawT - radius;
    for (int k = threadIdx.x; k < kRawT + 2 * radius; k += kRawT) {
        const int x = x0 + k;
        int s = 0;
        if (x >= 0 && x < V.w)
            for (int dy = -radius; dy <= radius; ++dy) {
                const int y = v + dy;
                if (y >= 0 && y < V.h) s += V.depth[(int64_t)y * V.w + x] > 0.f;
            }
        colsum[k] = (unsigned short)s;
    }
    __syncthreads();
    float n[3];
    const int p = u < V.w ? pixel_normal(V, u, v, step, noise, stepd, noised, n) : 0;
    int total;
    const int slot = tile_off[V.tile_base + v * V.tiles_x + tx] + block_excl_scan(p, total, sh);
    if (u >= V.w) return;
    float wk = 0.f;
    if (p) {
        int cnt = 0;
        for (int dx = 0; dx <= 2 * radius; ++dx) cnt += colsum[threadIdx.x + dx];
        const float k2 = (float)((2 * radius + 1) * (2 * radius + 1));
        const float D = V.depth[(int64_t)v * V.w + u];
        const float xc[3] = {((float)u - V.cx) / V.fx * D, ((float)v - V.cy) / V.fy * D, D};
        const float l = sqrtf(xc[0] * xc[0] + xc[1] * xc[1] + xc[2] * xc[2]);
        const float w1 = fmaxf(-(xc[0] * n[0] + xc[1] * n[1] + xc[2] * n[2]) / l, 0.f);
        wk = w1 * ((float)cnt / k2);
        // world: R^T (x_c - t), R^T n
        const float d[3] = {xc[0] - V.t[0], xc[1] - V.t[1], xc[2] - V.t[2]};
        for (int c = 0; c < 3; ++c) {
            P[3 * (int64_t)slot + c] = V.R[c] * d[0] + V.R[3 + c] * d[1] + V.R[6 + c] * d[2];
            N[3 * (int64_t)slot + c] = V.R[c] * n[0] + V.R[3 + c] * n[1] + V.R[6 + c] * n[2];
        }
        W[slot] = wk;
    }
    if (V.conf) V.conf[(int64_t)v * V.w + u] = wk;
}

}  // namespace

cudaError_t launch_raw(ftr_ctx* c, const RawParams& rp, const ftr_view* views, int k, float* const* conf_maps,
                       float* P, float* N, float* W, int* d_tile_cnt, int* d_total) {
    RawSet S{};
    S.k = k;
    int tiles = 0, max_tx = 0, max_h = 0;
    for (int i = 0; i < k; ++i) {
        RawView& V = S.v[i];
        const ftr_view& src = views[i];
        V.w = src.w;
        V.h = src.h;
        V.fx = src.K[0];
        V.fy = src.K[4];
        V.cx = src.K[2];
        V.cy = src.K[5];
        V.fxd = src.K[0];
        V.fyd = src.K[4];
        V.cxd = src.K[2];
        V.cyd = src.K[5];
        for (int r = 0; r < 3; ++r) {
            for (int q = 0; q < 3; ++q) V.R[3 * r + q] = src.world_to_cam[4 * r + q];
            V.t[r] = src.world_to_cam[4 * r + 3];
        }
        V.depth = src.depth;
        V.conf = conf_maps ? conf_maps[i] : nullptr;
        V.tiles_x = (src.w + kRawT - 1) / kRawT;
        V.tile_base = tiles;
        tiles += V.tiles_x * src.h;
        max_tx = max_tx > V.tiles_x ? max_tx : V.tiles_x;
        max_h = max_h > src.h ? max_h : src.h;
    }
    const dim3 grid(max_tx, max_h, k);
    launch_pdl(k_raw_count, grid, kRawT, 0, c->stream, S, rp.step_f, rp.noise_f, rp.step, rp.noise, d_tile_cnt);
    launch_pdl(k_raw_scan, 1, 1024, 0, c->stream, d_tile_cnt, tiles, d_total);
    launch_pdl(k_raw_emit, grid, kRawT, 0, c->stream, S, rp.step_f, rp.noise_f, rp.step, rp.noise, rp.radius,
               (const int*)d_tile_cnt, P, N, W);
    c->launches += 3;
    return cudaGetLastError();
}

int raw_tiles(const ftr_view* views, int k) {
    int tiles = 0;
    for (int i = 0; i < k; ++i) tiles += ((views[i].w + kRawT - 1) / kRawT) * views[i].h;
    return tiles;
}

int raw_max_radius() { return kRawMaxR; }

}  // namespace ftr
