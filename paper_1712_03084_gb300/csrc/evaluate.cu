// Objective evaluation of a reconstruction against sensor views (Sec. III-E).
//
// Geometry (eq. (3)-(5)), for one view with the rendered depth D_r and the
// sensor depth D_g (0 = background; silhouettes S_r = D_r > 0, S_g = D_g > 0):
//   k_ev_cols    one thread per column: the vertical distance of every pixel
//                to the nearest pixel of S_g and of S_r in its column (two
//                sweeps), and the counts |S_r|, |S_g|, |xor|, |or|;
//   k_ev_rows    one CTA per row: for each pixel of S_r the exact squared
//                distance to S_g, min over columns x' of (x - x')^2 + col(x')^2
//                (searched outwards, stopped once (x - x')^2 exceeds the best),
//                and the same from S_g to S_r; the maxima (eq. (4)) by
//                atomicMax -- integers throughout, so exact;
//   k_ev_points  one thread per pixel: back-projects the foreground pixels,
//                X = z (dx, dy, 1), into two compacted lists (warp-aggregated
//                appends; the order does not matter, see below);
//   k_ev_cp      (sensor tile of 256) x (chunk of rendered points): the
//                squared distance to the closest rendered point, float32,
//                merged per sensor pixel with atomicMin on the float bits (a
//                minimum does not depend on the order it is taken in);
//   k_sum / k_sum_final  the float64 sum of those distances in pixel order,
//                fixed blocks and a fixed tree (deterministic).
//
// Appearance (eq. (6)(7)), per scale j = 1..3:
//   k_ap_luma / k_ap_down   luma planes and silhouette, then 2 x 2 block
//                mean (silhouette: block AND) for the next scale;
//   k_ap_ssim    16 x 16 pixels per CTA with an 11 x 11-window halo in shared
//                memory: per silhouette pixel the window means, then the
//                second moments about those means (centred, so flat regions
//                give exactly zero variance up to rounding of the mean),
//                l, c, s and w(u); block partial sums in float64;
//   k_sum_final  the partials in a fixed order.
// The host side combines the per-scale means into WMS3IM.
#include <cuda_runtime.h>
#include <math.h>

#include <limits>

#include "ftr_internal.h"

namespace ftr {

namespace {

constexpr int kNone = 1 << 28;      // column distance when the column holds no pixel of the set
constexpr long long kFar = 0x7fffffffffffffffLL;   // no pixel of the set in the whole image
constexpr int kTile = 16;           // appearance: output pixels per CTA side
constexpr int kR = 5;               // SSIM window radius (11 x 11)
constexpr int kHalo = kTile + 2 * kR;
constexpr int kSumBlocks = 256;
// Sec. III-E3: exponents of the three scales (luminance, contrast, structure)
constexpr double kAlpha[3] = {0.0, 0.0, 0.1333};
constexpr double kBeta[3] = {0.0448, 0.3001, 0.1333};
constexpr double kGamma[3] = {0.0448, 0.3001, 0.1333};

struct Taps {
    float g[2 * kR + 1];
};

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(128) k_ev_cols(const float* __restrict__ rd, const float* __restrict__ gd, int w,
                                                 int h, int* __restrict__ colG, int* __restrict__ colR,
                                                 unsigned long long* __restrict__ cnt) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nr = 0, ng = 0, nx = 0, no = 0;
    if (x < w) {
        int lastG = -1, lastR = -1;
        for (int y = 0; y < h; ++y) {
            const int64_t i = (int64_t)y * w + x;
            const bool g = gd[i] > 0.f, r = rd[i] > 0.f;
            if (g) lastG = y;
            if (r) lastR = y;
            colG[i] = lastG >= 0 ? y - lastG : kNone;
            colR[i] = lastR >= 0 ? y - lastR : kNone;
            nr += r;
            ng += g;
            nx += (r != g);
            no += (r || g);
        }
        int nextG = -1, nextR = -1;
        for (int y = h - 1; y >= 0; --y) {
            const int64_t i = (int64_t)y * w + x;
            if (gd[i] > 0.f) nextG = y;
            if (rd[i] > 0.f) nextR = y;
            if (nextG >= 0) colG[i] = min(colG[i], nextG - y);
            if (nextR >= 0) colR[i] = min(colR[i], nextR - y);
        }
    }
    nr = warp_sum_u64(nr);
    ng = warp_sum_u64(ng);
    nx = warp_sum_u64(nx);
    no = warp_sum_u64(no);
    if ((threadIdx.x & 31) == 0 && (nr | ng | no)) {
        atomicAdd(cnt + 0, nr);
        atomicAdd(cnt + 1, ng);
        atomicAdd(cnt + 2, nx);
        atomicAdd(cnt + 3, no);
    }
}

// Smallest (x - x')^2 + col(x')^2 over the row; kNone columns hold no pixel.
__device__ __forceinline__ long long row_min(const int* __restrict__ col, int w, int x) {
    long long best = kFar;
    for (int d = 0; d < w; ++d) {
        const long long dd = (long long)d * d;
        if (dd >= best) break;
        if (x - d >= 0) {
            const int c = col[x - d];
            if (c != kNone) best = min(best, dd + (long long)c * c);
        }
        if (d > 0 && x + d < w) {
            const int c = col[x + d];
            if (c != kNone) best = min(best, dd + (long long)c * c);
        }
    }
    return best;
}

__global__ void __launch_bounds__(256) k_ev_rows(const float* __restrict__ rd, const float* __restrict__ gd, int w,
                                                 const int* __restrict__ colG, const int* __restrict__ colR,
                                                 unsigned long long* __restrict__ cnt) {
    const int y = blockIdx.x;
    const int64_t row = (int64_t)y * w;
    unsigned long long mrg = 0, mgr = 0;
    for (int x = threadIdx.x; x < w; x += blockDim.x) {
        if (rd[row + x] > 0.f) {
            const long long b = row_min(colG + row, w, x);
            if (b != kFar) mrg = max(mrg, (unsigned long long)b);
        }
        if (gd[row + x] > 0.f) {
            const long long b = row_min(colR + row, w, x);
            if (b != kFar) mgr = max(mgr, (unsigned long long)b);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mrg = max(mrg, __shfl_xor_sync(0xffffffffu, mrg, o));
        mgr = max(mgr, __shfl_xor_sync(0xffffffffu, mgr, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (mrg) atomicMax(cnt + 4, mrg);
        if (mgr) atomicMax(cnt + 5, mgr);
    }
}

struct Intr {
    double K[9];
};

__global__ void __launch_bounds__(256) k_ev_points(const float* __restrict__ rd, const float* __restrict__ gd,
                                                   int w, int64_t npx, Intr in, float4* __restrict__ ptsG,
                                                   float4* __restrict__ ptsR, float* __restrict__ d2,
                                                   unsigned long long* __restrict__ cnt) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = p < npx;
    const float zg = live ? gd[p] : 0.f, zr = live ? rd[p] : 0.f;
    const bool g = zg > 0.f, r = zr > 0.f;
    double dx = 0.0, dy = 0.0;
    if (g || r) {
        const double py = (double)(p / w), px = (double)(p % w);
        dy = __ddiv_rn(__dsub_rn(py, in.K[5]), in.K[4]);
        dx = __ddiv_rn(__dsub_rn(__dsub_rn(px, in.K[2]), __dmul_rn(in.K[1], dy)), in.K[0]);
    }
    if (live) d2[p] = g ? __uint_as_float(0x7f800000u) : 0.f;
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned bg = __ballot_sync(0xffffffffu, g), br = __ballot_sync(0xffffffffu, r);
    unsigned long long baseG = 0, baseR = 0;
    if (lane == 0) {
        if (bg) baseG = atomicAdd(cnt + 6, (unsigned long long)__popc(bg));
        if (br) baseR = atomicAdd(cnt + 7, (unsigned long long)__popc(br));
    }
    baseG = __shfl_sync(0xffffffffu, baseG, 0);
    baseR = __shfl_sync(0xffffffffu, baseR, 0);
    const float tag = __int_as_float((int)p);
    if (g) {
        const double z = zg;
        ptsG[baseG + __popc(bg & lt)] = make_float4((float)(z * dx), (float)(z * dy), zg, tag);
    }
    if (r) {
        const double z = zr;
        ptsR[baseR + __popc(br & lt)] = make_float4((float)(z * dx), (float)(z * dy), zr, tag);
    }
}

__global__ void __launch_bounds__(256) k_ev_cp(const float4* __restrict__ G, const float4* __restrict__ R, int64_t I,
                                               int64_t J, int64_t chunk, float* __restrict__ d2) {
    __shared__ float4 s[256];
    const int64_t gi = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * chunk;
    const int64_t r1 = min(r0 + chunk, J);
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gi < I) q = G[gi];
    float best = __uint_as_float(0x7f800000u);
    for (int64_t rb = r0; rb < r1; rb += 256) {
        __syncthreads();
        if (rb + threadIdx.x < r1) s[threadIdx.x] = R[rb + threadIdx.x];
        __syncthreads();
        const int n = (int)min((int64_t)256, r1 - rb);
#pragma unroll 8
        for (int j = 0; j < n; ++j) {
            const float4 t = s[j];
            const float ex = q.x - t.x, ey = q.y - t.y, ez = q.z - t.z;
            best = fminf(best, ex * ex + ey * ey + ez * ez);
        }
    }
    if (gi < I) atomicMin(reinterpret_cast<unsigned*>(d2) + __float_as_int(q.w), __float_as_uint(best));
}

// float64 sums of n values in a fixed order: block b takes the indices
// b*256 + t + k*gridDim*256, then a fixed tree.
template <class T>
__global__ void __launch_bounds__(256) k_sum(const T* __restrict__ v, int64_t n, double* __restrict__ part) {
    __shared__ double s[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) acc += (double)v[i];
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

// out[c] = sum over blocks b of part[b * stride + c], c < comps, fixed order.
__global__ void __launch_bounds__(256) k_sum_final(const double* __restrict__ part, int64_t nblocks, int comps,
                                                   int stride, double* __restrict__ out) {
    __shared__ double s[256];
    for (int c = 0; c < comps; ++c) {
        double acc = 0.0;
        for (int64_t b = threadIdx.x; b < nblocks; b += 256) acc += part[b * stride + c];
        s[threadIdx.x] = acc;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[c] = s[0];
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_ap_luma(const uint8_t* __restrict__ rr, const uint8_t* __restrict__ rg,
                                                 const float* __restrict__ rd, int64_t npx, float* __restrict__ X,
                                                 float* __restrict__ Y, uint8_t* __restrict__ S) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npx) return;
    X[p] = 0.299f * rr[3 * p] + 0.587f * rr[3 * p + 1] + 0.114f * rr[3 * p + 2];
    Y[p] = 0.299f * rg[3 * p] + 0.587f * rg[3 * p + 1] + 0.114f * rg[3 * p + 2];
    S[p] = rd[p] > 0.f;
}

__global__ void __launch_bounds__(256) k_ap_down(const float* __restrict__ X, const float* __restrict__ Y,
                                                 const uint8_t* __restrict__ S, int w, int w2, int h2,
                                                 float* __restrict__ X2, float* __restrict__ Y2,
                                                 uint8_t* __restrict__ S2) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)w2 * h2) return;
    const int64_t y = p / w2, x = p % w2;
    const int64_t a = 2 * y * w + 2 * x, b = a + w;
    X2[p] = 0.25f * (((X[a] + X[a + 1]) + X[b]) + X[b + 1]);
    Y2[p] = 0.25f * (((Y[a] + Y[a + 1]) + Y[b]) + Y[b + 1]);
    S2[p] = S[a] & S[a + 1] & S[b] & S[b + 1];
}

__global__ void __launch_bounds__(256) k_ap_ssim(const float* __restrict__ X, const float* __restrict__ Y,
                                                 const uint8_t* __restrict__ S, int w, int h, Taps tp,
                                                 double* __restrict__ part) {
    __shared__ float sx[kHalo][kHalo + 1];
    __shared__ float sy[kHalo][kHalo + 1];
    __shared__ uint8_t ss[kHalo][kHalo + 1];
    __shared__ double red[4][256];
    const int bx = blockIdx.x * kTile - kR, by = blockIdx.y * kTile - kR;
    for (int i = threadIdx.x; i < kHalo * kHalo; i += 256) {
        const int ty = i / kHalo, tx = i % kHalo;
        const int gx = bx + tx, gy = by + ty;
        const bool in = gx >= 0 && gx < w && gy >= 0 && gy < h;
        const int64_t gi = (int64_t)gy * w + gx;
        sx[ty][tx] = in ? X[gi] : 0.f;
        sy[ty][tx] = in ? Y[gi] : 0.f;
        ss[ty][tx] = in ? S[gi] : 0;
    }
    __syncthreads();
    const int tx = threadIdx.x % kTile, ty = threadIdx.x / kTile;
    const int x = blockIdx.x * kTile + tx, y = blockIdx.y * kTile + ty;
    double cl = 0.0, cc = 0.0, cs = 0.0, cw = 0.0;
    if (x < w && y < h && ss[ty + kR][tx + kR]) {
        const float C1 = (0.01f * 255.f) * (0.01f * 255.f);
        const float C2 = (0.03f * 255.f) * (0.03f * 255.f);
        const float C3 = 0.5f * C2;
        // taps inside the image: i in [i0, i1], j in [j0, j1]
        const int i0 = max(-kR, -x), i1 = min(kR, w - 1 - x);
        const int j0 = max(-kR, -y), j1 = min(kR, h - 1 - y);
        float gsx = 0.f, gsy = 0.f;
        for (int i = i0; i <= i1; ++i) gsx += tp.g[i + kR];
        for (int j = j0; j <= j1; ++j) gsy += tp.g[j + kR];
        const float inv = 1.f / (gsx * gsy);
        float mx = 0.f, my = 0.f;
        int count = 0;
        for (int j = j0; j <= j1; ++j) {
            float rx = 0.f, ry = 0.f;
            for (int i = i0; i <= i1; ++i) {
                const float g = tp.g[i + kR];
                rx += g * sx[ty + kR + j][tx + kR + i];
                ry += g * sy[ty + kR + j][tx + kR + i];
                count += ss[ty + kR + j][tx + kR + i];
            }
            mx += tp.g[j + kR] * rx;
            my += tp.g[j + kR] * ry;
        }
        mx *= inv;
        my *= inv;
        float vx = 0.f, vy = 0.f, cxy = 0.f;
        for (int j = j0; j <= j1; ++j) {
            float ax = 0.f, ay = 0.f, axy = 0.f;
            for (int i = i0; i <= i1; ++i) {
                const float g = tp.g[i + kR];
                const float ex = sx[ty + kR + j][tx + kR + i] - mx;
                const float ey = sy[ty + kR + j][tx + kR + i] - my;
                ax += g * ex * ex;
                ay += g * ey * ey;
                axy += g * ex * ey;
            }
            vx += tp.g[j + kR] * ax;
            vy += tp.g[j + kR] * ay;
            cxy += tp.g[j + kR] * axy;
        }
        vx *= inv;
        vy *= inv;
        cxy *= inv;
        const float sgx = sqrtf(vx), sgy = sqrtf(vy);
        const float l = (2.f * mx * my + C1) / (mx * mx + my * my + C1);
        const float c = (2.f * sgx * sgy + C2) / (vx + vy + C2);
        const float s = (cxy + C3) / (sgx * sgy + C3);
        cw = (double)count;
        cl = cw * l;
        cc = cw * c;
        cs = cw * s;
    }
    red[0][threadIdx.x] = cl;
    red[1][threadIdx.x] = cc;
    red[2][threadIdx.x] = cs;
    red[3][threadIdx.x] = cw;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
#pragma unroll
            for (int m = 0; m < 4; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) part[4 * ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) + threadIdx.x] = red[threadIdx.x][0];
}

bool dev_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t grow(T** p, int64_t* cap, int64_t need) {
    if (*cap >= need) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc((void**)p, (size_t)need * sizeof(T));
    if (e == cudaSuccess) *cap = need;
    return e;
}

cudaError_t grow_pixels(ftr_ctx* c, EvalScratch* ev, int64_t npx) {
    if (ev->pix_cap >= npx) return cudaSuccess;
    cudaStreamSynchronize(c->stream);
    if (ev->col) cudaFree(ev->col);
    if (ev->pts) cudaFree(ev->pts);
    if (ev->d2) cudaFree(ev->d2);
    ev->col = nullptr;
    ev->pts = nullptr;
    ev->d2 = nullptr;
    ev->pix_cap = 0;
    cudaError_t e;
    if ((e = cudaMalloc((void**)&ev->col, (size_t)npx * 2 * sizeof(int))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&ev->pts, (size_t)npx * 2 * sizeof(float4))) != cudaSuccess) return e;
    if ((e = cudaMalloc((void**)&ev->d2, (size_t)npx * sizeof(float))) != cudaSuccess) return e;
    ev->pix_cap = npx;
    return cudaSuccess;
}

cudaError_t grow_part(ftr_ctx* c, EvalScratch* ev, int64_t n) {
    if (ev->part_cap >= n) return cudaSuccess;
    cudaStreamSynchronize(c->stream);
    return grow(&ev->part, &ev->part_cap, n);
}

}  // namespace

EvalScratch* eval_scratch(ftr_ctx* c) {
    if (c->ev) return c->ev;
    EvalScratch* ev = new EvalScratch();
    if (cudaMalloc((void**)&ev->cnt, 8 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost((void**)&ev->h_res, 32 * sizeof(double)) != cudaSuccess) {
        if (ev->cnt) cudaFree(ev->cnt);
        delete ev;
        return nullptr;
    }
    c->ev = ev;
    return ev;
}

void eval_free(ftr_ctx* c) {
    EvalScratch* ev = c->ev;
    if (!ev) return;
    if (ev->zkey) cudaFree(ev->zkey);
    if (ev->big) cudaFree(ev->big);
    if (ev->col) cudaFree(ev->col);
    if (ev->pts) cudaFree(ev->pts);
    if (ev->d2) cudaFree(ev->d2);
    if (ev->cnt) cudaFree(ev->cnt);
    if (ev->part) cudaFree(ev->part);
    if (ev->h_res) cudaFreeHost(ev->h_res);
    if (ev->img) cudaFree(ev->img);
    if (ev->mask) cudaFree(ev->mask);
    delete ev;
    c->ev = nullptr;
}

}  // namespace ftr

using namespace ftr;

int ftr_eval_geometry(ftr_ctx* c, const ftr_camera* cam, const float* rendered_depth, const float* sensor_depth,
                      float* cp_d2_out, ftr_geometry_eval* out) {
    if (!c) return FTR_EINVAL;
    if (!camera_ok(cam) || !out)
        return set_err(c, FTR_EINVAL, "ftr_eval_geometry: a camera (w, h in 1..16384, focal != 0) and out");
    if (!dev_ptr(rendered_depth) || !dev_ptr(sensor_depth) || (cp_d2_out && !dev_ptr(cp_d2_out)))
        return set_err(c, FTR_EINVAL, "ftr_eval_geometry: depth images must be device memory");
    EvalScratch* ev = eval_scratch(c);
    if (!ev) return set_err(c, FTR_ENOMEM, "ftr_eval_geometry: scratch");
    const int w = cam->w, h = cam->h;
    const int64_t npx = (int64_t)w * h;
    cudaError_t e;
    if ((e = grow_pixels(c, ev, npx)) != cudaSuccess) return cuda_fail(c, e, "ftr_eval_geometry: scratch");
    if ((e = grow_part(c, ev, 4 * kSumBlocks)) != cudaSuccess) return cuda_fail(c, e, "ftr_eval_geometry: scratch");
    cudaStream_t st = c->stream;
    float* d2 = cp_d2_out ? cp_d2_out : ev->d2;
    int* colG = ev->col;
    int* colR = ev->col + npx;
    float4* ptsG = ev->pts;
    float4* ptsR = ev->pts + npx;
    if ((e = cudaMemsetAsync(ev->cnt, 0, 8 * sizeof(unsigned long long), st)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_eval_geometry");
    k_ev_cols<<<(w + 127) / 128, 128, 0, st>>>(rendered_depth, sensor_depth, w, h, colG, colR, ev->cnt);
    k_ev_rows<<<h, 256, 0, st>>>(rendered_depth, sensor_depth, w, colG, colR, ev->cnt);
    Intr in;
    for (int j = 0; j < 9; ++j) in.K[j] = cam->K[j];
    k_ev_points<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(rendered_depth, sensor_depth, w, npx, in, ptsG, ptsR,
                                                                d2, ev->cnt);
    c->launches += 3;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ftr_eval_geometry: silhouettes");
    // the list sizes shape the closest-point launch
    unsigned long long* hc = reinterpret_cast<unsigned long long*>(ev->h_res);
    if ((e = cudaMemcpyAsync(hc, ev->cnt, 8 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_eval_geometry: counts");
    const int64_t I = (int64_t)hc[6], J = (int64_t)hc[7];
    out->rendered_px = (int64_t)hc[0];
    out->sensor_px = (int64_t)hc[1];
    out->xor_px = (int64_t)hc[2];
    out->or_px = (int64_t)hc[3];
    out->vre = out->or_px ? (double)out->xor_px / (double)out->or_px : 0.0;
    const double inf = std::numeric_limits<double>::infinity();
    if (out->rendered_px == 0 && out->sensor_px == 0)
        out->hausdorff_px = 0.0;
    else if (out->rendered_px == 0 || out->sensor_px == 0)
        out->hausdorff_px = inf;
    else
        out->hausdorff_px = sqrt((double)(hc[4] > hc[5] ? hc[4] : hc[5]));
    out->sensor_points = I;
    out->rendered_points = J;
    if (I > 0 && J > 0) {
        // about four CTAs per SM: split the rendered points into chunks
        const int64_t gx = (I + 255) / 256;
        int64_t gy = (4 * 152 + gx - 1) / gx;
        if (gy < 1) gy = 1;
        int64_t chunk = (J + gy - 1) / gy;
        chunk = ((chunk + 255) / 256) * 256;
        gy = (J + chunk - 1) / chunk;
        k_ev_cp<<<dim3((unsigned)gx, (unsigned)gy), 256, 0, st>>>(ptsG, ptsR, I, J, chunk, d2);
        c->launches++;
    }
    k_sum<float><<<kSumBlocks, 256, 0, st>>>(d2, npx, ev->part);
    k_sum_final<<<1, 256, 0, st>>>(ev->part, kSumBlocks, 1, 1, ev->part + kSumBlocks);
    c->launches += 2;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ftr_eval_geometry: closest points");
    if ((e = cudaMemcpyAsync(ev->h_res + 8, ev->part + kSumBlocks, sizeof(double), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_eval_geometry: sum");
    if (I == 0)
        out->cp_rmse = std::numeric_limits<double>::quiet_NaN();
    else if (J == 0)
        out->cp_rmse = inf;
    else
        out->cp_rmse = sqrt(ev->h_res[8] / (double)I);
    return FTR_OK;
}

int ftr_eval_appearance(ftr_ctx* c, int w, int h, const float* rendered_depth, const uint8_t* rendered_rgb,
                        const uint8_t* sensor_rgb, ftr_appearance_eval* out) {
    if (!c) return FTR_EINVAL;
    if (w < 1 || h < 1 || w > 16384 || h > 16384 || !out)
        return set_err(c, FTR_EINVAL, "ftr_eval_appearance: 1 <= w, h <= 16384 and out");
    if (!dev_ptr(rendered_depth) || !dev_ptr(rendered_rgb) || !dev_ptr(sensor_rgb))
        return set_err(c, FTR_EINVAL, "ftr_eval_appearance: images must be device memory");
    EvalScratch* ev = eval_scratch(c);
    if (!ev) return set_err(c, FTR_ENOMEM, "ftr_eval_appearance: scratch");
    int ws[3], hs[3];
    int64_t off[4] = {0, 0, 0, 0}, boff[4] = {0, 0, 0, 0};
    unsigned gx[3], gy[3];
    for (int j = 0; j < 3; ++j) {
        ws[j] = j ? ws[j - 1] / 2 : w;
        hs[j] = j ? hs[j - 1] / 2 : h;
        off[j + 1] = off[j] + (int64_t)ws[j] * hs[j];
        gx[j] = (unsigned)((ws[j] + kTile - 1) / kTile);
        gy[j] = (unsigned)((hs[j] + kTile - 1) / kTile);
        boff[j + 1] = boff[j] + (int64_t)gx[j] * gy[j];
    }
    const double nan = std::numeric_limits<double>::quiet_NaN();
    cudaError_t e;
    const int64_t planes = off[3];
    if (planes > ev->img_cap) {
        cudaStreamSynchronize(c->stream);
        if (ev->img) cudaFree(ev->img);
        if (ev->mask) cudaFree(ev->mask);
        ev->img = nullptr;
        ev->mask = nullptr;
        ev->img_cap = 0;
        if ((e = cudaMalloc((void**)&ev->img, (size_t)planes * 2 * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc((void**)&ev->mask, (size_t)planes)) != cudaSuccess)
            return cuda_fail(c, e, "ftr_eval_appearance: scratch");
        ev->img_cap = planes;
    }
    if ((e = grow_part(c, ev, 4 * boff[3] + 16)) != cudaSuccess) return cuda_fail(c, e, "ftr_eval_appearance");
    cudaStream_t st = c->stream;
    float* X = ev->img;
    float* Y = ev->img + planes;
    uint8_t* S = ev->mask;
    k_ap_luma<<<(unsigned)((off[1] + 255) / 256), 256, 0, st>>>(rendered_rgb, sensor_rgb, rendered_depth, off[1], X,
                                                                 Y, S);
    c->launches++;
    Taps tp;
    for (int i = -kR; i <= kR; ++i) tp.g[i + kR] = (float)exp(-(double)(i * i) / (2.0 * 1.5 * 1.5));
    for (int j = 0; j < 3; ++j) {
        if (j) {
            const int64_t n = (int64_t)ws[j] * hs[j];
            if (n > 0) {
                k_ap_down<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X + off[j - 1], Y + off[j - 1], S + off[j - 1],
                                                                       ws[j - 1], ws[j], hs[j], X + off[j], Y + off[j],
                                                                       S + off[j]);
                c->launches++;
            }
        }
        if ((int64_t)gx[j] * gy[j] > 0) {
            k_ap_ssim<<<dim3(gx[j], gy[j]), 256, 0, st>>>(X + off[j], Y + off[j], S + off[j], ws[j], hs[j], tp,
                                                         ev->part + 4 * boff[j]);
            k_sum_final<<<1, 256, 0, st>>>(ev->part + 4 * boff[j], boff[j + 1] - boff[j], 4, 4,
                                           ev->part + 4 * boff[3] + 4 * j);
            c->launches += 2;
        }
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ftr_eval_appearance: kernels");
    if ((e = cudaMemcpyAsync(ev->h_res, ev->part + 4 * boff[3], 12 * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_eval_appearance: sums");
    double prod = 1.0;
    for (int j = 0; j < 3; ++j) {
        const double* r = ev->h_res + 4 * j;
        const bool empty = (int64_t)gx[j] * gy[j] == 0 || !(r[3] > 0.0);
        if (empty) {
            for (int m = 0; m < 3; ++m) out->l[m] = out->c[m] = out->s[m] = nan;
            out->wms3im = nan;
            return FTR_OK;
        }
        out->l[j] = r[0] / r[3];
        out->c[j] = r[1] / r[3];
        out->s[j] = r[2] / r[3];
        const double vals[3] = {out->l[j], out->c[j], out->s[j]};
        const double ex[3] = {kAlpha[j], kBeta[j], kGamma[j]};
        for (int m = 0; m < 3; ++m)
            if (ex[m] != 0.0) prod *= pow(vals[m] > 0.0 ? vals[m] : 0.0, ex[m]);
    }
    out->wms3im = prod;
    return FTR_OK;
}
