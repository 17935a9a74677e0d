// Rendering a triangle mesh into a pinhole camera (Sec. III-C, III-E).
//
// Sec. III-E projects the reconstructed mesh into every sensor view and reads
// back the depth and colour buffers; Sec. III-C draws each triangle with the
// per-vertex weights and UVs (multitexture blend).  No graphics API is used:
//
//   k_raster   one thread per triangle: project the three vertices, walk the
//              pixel centres of the screen bounding box, test coverage with
//              the three edge functions, intersect the pixel's ray with the
//              triangle's plane and keep the nearest surface with a 64-bit
//              atomicMin on (float32 z bits << 32 | triangle index); a
//              triangle with more than 1024 pixel centres in its box is
//              listed instead and k_raster_big shares its pixels among the
//              threads of a CTA (the same per-pixel code);
//   k_resolve  one thread per pixel: depth from the key, colour from the
//              winning triangle (perspective-correct barycentrics of the hit
//              point; vertex colours or the weighted blend of the views).
//
// Coverage and depth decide which triangle a pixel shows, so they are
// evaluated in float64 with every product, sum and quotient rounded on its
// own (no contraction) in one fixed order:
//   x_c = ((r0 X + r1 Y) + r2 Z) + t per row, a = x_c/z_c, b = y_c/z_c,
//   u = (K00 a + K01 b) + K02, v = K11 b + K12,
//   e_ab = (ub - ua)(py - va) - (vb - va)(px - ua) (and cyclic),
//   dy = (py - K12)/K11, dx = ((px - K02) - K01 dy)/K00,
//   n = (B - A) x (C - A), z = ((nx Ax + ny Ay) + nz Az) / ((nx dx + ny dy) + nz).
// The colours are float32 (they only feed the final rounding to u8).
#include <cuda_runtime.h>
#include <math.h>

#include "ftr_internal.h"

namespace ftr {

namespace {

constexpr double kZNear = 0.01;     // metres: a triangle with a vertex nearer the camera plane is not drawn
constexpr int kBigPx = 1024;        // bounding-box pixels above which a triangle is shared by a CTA

struct CamDev {
    int w, h;
    double K[9], RT[12];
    float Kf[9], RTf[12];
};

struct TexDev {
    int k;
    int rgb_w[kMaxViews], rgb_h[kMaxViews];
    const uint8_t* rgb[kMaxViews];
};

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ds(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dd(double a, double b) { return __ddiv_rn(a, b); }

__device__ __forceinline__ void cam_point(const CamDev& c, const float* X, double xc[3]) {
    const double x = X[0], y = X[1], z = X[2];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        xc[r] = da(da(da(dm(c.RT[4 * r], x), dm(c.RT[4 * r + 1], y)), dm(c.RT[4 * r + 2], z)), c.RT[4 * r + 3]);
}

__device__ __forceinline__ double edge(double ua, double va, double ub, double vb, double px, double py) {
    return ds(dm(ds(ub, ua), ds(py, va)), dm(ds(vb, va), ds(px, ua)));
}

// Everything a pixel test needs, set up once per triangle.
struct TriSetup {
    double u[3], v[3];
    double nx, ny, nz, num;
    double x0, x1, y0, y1;
};

// Projects the triangle and its plane; false if it is not drawn (an index
// out of range, a vertex nearer than kZNear, zero area, or no pixel centre
// in its clipped bounding box).
__device__ __forceinline__ bool tri_setup(const CamDev& cam, const float* __restrict__ verts,
                                          const int32_t* __restrict__ tris, int64_t t, int64_t nv, TriSetup& s) {
    const int i3[3] = {tris[3 * t], tris[3 * t + 1], tris[3 * t + 2]};
    double xc[3][3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        if (i3[m] < 0 || i3[m] >= nv) return false;
        cam_point(cam, verts + 3 * (int64_t)i3[m], xc[m]);
        if (!(xc[m][2] >= kZNear)) return false;
        const double a = dd(xc[m][0], xc[m][2]);
        const double b = dd(xc[m][1], xc[m][2]);
        s.u[m] = da(da(dm(cam.K[0], a), dm(cam.K[1], b)), cam.K[2]);
        s.v[m] = da(dm(cam.K[4], b), cam.K[5]);
    }
    const double area = ds(dm(ds(s.u[1], s.u[0]), ds(s.v[2], s.v[0])), dm(ds(s.v[1], s.v[0]), ds(s.u[2], s.u[0])));
    if (!isfinite(area) || area == 0.0) return false;
    s.x0 = fmax(ceil(fmin(fmin(s.u[0], s.u[1]), s.u[2])), 0.0);
    s.x1 = fmin(floor(fmax(fmax(s.u[0], s.u[1]), s.u[2])), (double)(cam.w - 1));
    s.y0 = fmax(ceil(fmin(fmin(s.v[0], s.v[1]), s.v[2])), 0.0);
    s.y1 = fmin(floor(fmax(fmax(s.v[0], s.v[1]), s.v[2])), (double)(cam.h - 1));
    if (s.x1 < s.x0 || s.y1 < s.y0) return false;
    double e1v[3], e2v[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        e1v[r] = ds(xc[1][r], xc[0][r]);
        e2v[r] = ds(xc[2][r], xc[0][r]);
    }
    s.nx = ds(dm(e1v[1], e2v[2]), dm(e1v[2], e2v[1]));
    s.ny = ds(dm(e1v[2], e2v[0]), dm(e1v[0], e2v[2]));
    s.nz = ds(dm(e1v[0], e2v[1]), dm(e1v[1], e2v[0]));
    s.num = da(da(dm(s.nx, xc[0][0]), dm(s.ny, xc[0][1])), dm(s.nz, xc[0][2]));
    return true;
}

// Coverage and depth of pixel (px, py) (dy = its ray's y slope); the key
// goes to the z-buffer when the pixel is covered.
__device__ __forceinline__ void tri_pixel(const CamDev& cam, const TriSetup& s, double px, double py, double dy,
                                          unsigned long long tid, unsigned long long* __restrict__ zkey) {
    const double e0 = edge(s.u[0], s.v[0], s.u[1], s.v[1], px, py);
    const double e1 = edge(s.u[1], s.v[1], s.u[2], s.v[2], px, py);
    const double e2 = edge(s.u[2], s.v[2], s.u[0], s.v[0], px, py);
    const bool in = (e0 >= 0.0 && e1 >= 0.0 && e2 >= 0.0) || (e0 <= 0.0 && e1 <= 0.0 && e2 <= 0.0);
    if (!in) return;
    const double dx = dd(ds(ds(px, cam.K[2]), dm(cam.K[1], dy)), cam.K[0]);
    const double den = da(da(dm(s.nx, dx), dm(s.ny, dy)), s.nz);
    if (den == 0.0) return;
    const double z = dd(s.num, den);
    if (!(z > 0.0) || !isfinite(z)) return;
    const unsigned long long key = ((unsigned long long)__float_as_uint(__double2float_rn(z)) << 32) | tid;
    atomicMin(zkey + (int64_t)py * cam.w + (int64_t)px, key);
}

// One thread per triangle; a triangle whose bounding box holds more than
// kBigPx pixel centres is listed for k_raster_big instead.
__global__ void __launch_bounds__(128) k_raster(CamDev cam, const float* __restrict__ verts,
                                                const int32_t* __restrict__ tris, int64_t nt, int64_t nv,
                                                unsigned long long* __restrict__ zkey, int* __restrict__ big,
                                                int* __restrict__ nbig) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    TriSetup s;
    if (!tri_setup(cam, verts, tris, t, nv, s)) return;
    if ((s.x1 - s.x0 + 1.0) * (s.y1 - s.y0 + 1.0) > (double)kBigPx) {
        big[atomicAdd(nbig, 1)] = (int)t;          // at most nt entries
        return;
    }
    for (double py = s.y0; py <= s.y1; py += 1.0) {
        const double dy = dd(ds(py, cam.K[5]), cam.K[4]);
        for (double px = s.x0; px <= s.x1; px += 1.0) tri_pixel(cam, s, px, py, dy, (unsigned long long)t, zkey);
    }
}

// The listed large triangles, one CTA each (grid-stride over the list): the
// CTA's threads share the triangle's pixel centres.
__global__ void __launch_bounds__(256) k_raster_big(CamDev cam, const float* __restrict__ verts,
                                                    const int32_t* __restrict__ tris, int64_t nv,
                                                    unsigned long long* __restrict__ zkey,
                                                    const int* __restrict__ big, const int* __restrict__ nbig) {
    const int n = *nbig;
    for (int j = blockIdx.x; j < n; j += gridDim.x) {
        const int64_t t = big[j];
        TriSetup s;
        if (!tri_setup(cam, verts, tris, t, nv, s)) continue;    // always drawn: listed by k_raster
        const int64_t wx = (int64_t)(s.x1 - s.x0) + 1, hy = (int64_t)(s.y1 - s.y0) + 1;
        for (int64_t k = threadIdx.x; k < wx * hy; k += blockDim.x) {
            const double py = s.y0 + (double)(k / wx), px = s.x0 + (double)(k % wx);
            const double dy = dd(ds(py, cam.K[5]), cam.K[4]);
            tri_pixel(cam, s, px, py, dy, (unsigned long long)t, zkey);
        }
    }
}

__device__ __forceinline__ void cam_point_f(const CamDev& c, const float* X, float xc[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        xc[r] = c.RTf[4 * r] * X[0] + c.RTf[4 * r + 1] * X[1] + c.RTf[4 * r + 2] * X[2] + c.RTf[4 * r + 3];
}

__device__ __forceinline__ float dot_cross(const float n[3], const float a[3], const float b[3]) {
    // n . (a x b)
    return n[0] * (a[1] * b[2] - a[2] * b[1]) + n[1] * (a[2] * b[0] - a[0] * b[2]) +
           n[2] * (a[0] * b[1] - a[1] * b[0]);
}

__device__ __forceinline__ void bilinear(const uint8_t* img, int w, int h, float u, float v, float out[3]) {
    const float fu = floorf(u), fv = floorf(v);
    const int x0 = (int)fu, y0 = (int)fv;
    const float fx = u - fu, fy = v - fv;
    const int xa = min(max(x0, 0), w - 1), xb = min(max(x0 + 1, 0), w - 1);
    const int ya = min(max(y0, 0), h - 1), yb = min(max(y0 + 1, 0), h - 1);
    const uint8_t* p00 = img + 3 * ((int64_t)ya * w + xa);
    const uint8_t* p10 = img + 3 * ((int64_t)ya * w + xb);
    const uint8_t* p01 = img + 3 * ((int64_t)yb * w + xa);
    const uint8_t* p11 = img + 3 * ((int64_t)yb * w + xb);
#pragma unroll
    for (int c = 0; c < 3; ++c)
        out[c] = (1.f - fx) * (1.f - fy) * p00[c] + fx * (1.f - fy) * p10[c] + (1.f - fx) * fy * p01[c] +
                 fx * fy * p11[c];
}

__global__ void __launch_bounds__(256) k_resolve(CamDev cam, const float* __restrict__ verts,
                                                 const int32_t* __restrict__ tris,
                                                 const unsigned long long* __restrict__ zkey,
                                                 float* __restrict__ depth, uint8_t* __restrict__ rgb,
                                                 const uint8_t* __restrict__ vrgb, const float* __restrict__ tw,
                                                 const float* __restrict__ tuv, TexDev tex) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t npx = (int64_t)cam.w * cam.h;
    if (p >= npx) return;
    const unsigned long long key = zkey[p];
    if (key == ~0ull) {
        depth[p] = 0.f;
        if (rgb) rgb[3 * p] = rgb[3 * p + 1] = rgb[3 * p + 2] = 0;
        return;
    }
    const float z = __uint_as_float((unsigned)(key >> 32));
    depth[p] = z;
    if (!rgb) return;
    const int64_t t = (int64_t)(key & 0xffffffffull);
    const int ia = tris[3 * t], ib = tris[3 * t + 1], ic = tris[3 * t + 2];
    float A[3], B[3], C[3];
    cam_point_f(cam, verts + 3 * (int64_t)ia, A);
    cam_point_f(cam, verts + 3 * (int64_t)ib, B);
    cam_point_f(cam, verts + 3 * (int64_t)ic, C);
    const float py = (float)(p / cam.w), px = (float)(p % cam.w);
    const float dy = (py - cam.Kf[5]) / cam.Kf[4];
    const float dx = ((px - cam.Kf[2]) - cam.Kf[1] * dy) / cam.Kf[0];
    const float P[3] = {z * dx, z * dy, z};
    float e1[3], e2[3], n[3], pa[3], pb[3], pc[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        e1[r] = B[r] - A[r];
        e2[r] = C[r] - A[r];
        pa[r] = A[r] - P[r];
        pb[r] = B[r] - P[r];
        pc[r] = C[r] - P[r];
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    const float nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
    const float la = dot_cross(n, pb, pc) / nn;
    const float lb = dot_cross(n, pc, pa) / nn;
    const float lc = dot_cross(n, pa, pb) / nn;
    float col[3] = {0.f, 0.f, 0.f};
    if (vrgb) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            col[c] = la * vrgb[3 * ia + c] + lb * vrgb[3 * ib + c] + lc * vrgb[3 * ic + c];
    } else if (tw) {
        const int K = tex.k;
        float acc[3] = {0.f, 0.f, 0.f}, wsum = 0.f;
        for (int k = 0; k < K; ++k) {
            const float wa = tw[(int64_t)ia * K + k], wb = tw[(int64_t)ib * K + k], wc = tw[(int64_t)ic * K + k];
            if (!(wa > 0.f && wb > 0.f && wc > 0.f)) continue;
            const float wk = la * wa + lb * wb + lc * wc;
            const float uk = la * tuv[2 * ((int64_t)ia * K + k)] + lb * tuv[2 * ((int64_t)ib * K + k)] +
                             lc * tuv[2 * ((int64_t)ic * K + k)];
            const float vk = la * tuv[2 * ((int64_t)ia * K + k) + 1] + lb * tuv[2 * ((int64_t)ib * K + k) + 1] +
                             lc * tuv[2 * ((int64_t)ic * K + k) + 1];
            float s[3];
            bilinear(tex.rgb[k], tex.rgb_w[k], tex.rgb_h[k], uk, vk, s);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] += wk * s[c];
            wsum += wk;
        }
        if (wsum > 0.f) {
#pragma unroll
            for (int c = 0; c < 3; ++c) col[c] = acc[c] / wsum;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) rgb[3 * p + c] = (uint8_t)fminf(fmaxf(floorf(col[c] + 0.5f), 0.f), 255.f);
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

CamDev make_cam(const ftr_camera& c) {
    CamDev d{};
    d.w = c.w;
    d.h = c.h;
    for (int j = 0; j < 9; ++j) d.K[j] = d.Kf[j] = c.K[j];
    for (int j = 0; j < 12; ++j) d.RT[j] = d.RTf[j] = c.world_to_cam[j];
    return d;
}

}  // namespace

bool camera_ok(const ftr_camera* cam) {
    return cam && cam->w >= 1 && cam->h >= 1 && cam->w <= 16384 && cam->h <= 16384 && cam->K[0] != 0.f &&
           cam->K[4] != 0.f;
}

}  // namespace ftr

using namespace ftr;

int ftr_render(ftr_ctx* c, const ftr_render_src* src, const ftr_camera* cam, float* depth_out, uint8_t* rgb_out) {
    if (!c) return FTR_EINVAL;
    if (!src || !camera_ok(cam) || !depth_out)
        return set_err(c, FTR_EINVAL, "ftr_render: a source, a camera (w, h in 1..16384, focal != 0) and depth_out");
    if (src->n_tris < 0 || src->n_tris >= (int64_t)1 << 31 || src->n_vertices < 0)
        return set_err(c, FTR_EINVAL, "ftr_render: 0 <= n_tris < 2^31");
    if (src->vertex_rgb && src->tex_weights)
        return set_err(c, FTR_EINVAL, "ftr_render: one colour source at most");
    if ((src->vertex_rgb || src->tex_weights) && !rgb_out)
        return set_err(c, FTR_EINVAL, "ftr_render: a colour source needs rgb_out");
    if (!dev_ptr(depth_out) || (rgb_out && !dev_ptr(rgb_out)))
        return set_err(c, FTR_EINVAL, "ftr_render: outputs must be device memory");
    if (src->n_tris > 0 && (!dev_ptr(src->vertices) || !dev_ptr(src->tris)))
        return set_err(c, FTR_EINVAL, "ftr_render: vertices and tris must be device memory");
    if (src->vertex_rgb && !dev_ptr(src->vertex_rgb))
        return set_err(c, FTR_EINVAL, "ftr_render: vertex_rgb must be device memory");
    TexDev tex{};
    if (src->tex_weights) {
        if (src->tex_k < 1 || src->tex_k > kMaxViews || !src->tex_views || !dev_ptr(src->tex_weights) ||
            !dev_ptr(src->tex_uv))
            return set_err(c, FTR_EINVAL, "ftr_render: 1 <= tex_k <= 8 views, device weights and uv");
        tex.k = src->tex_k;
        for (int k = 0; k < tex.k; ++k) {
            const ftr_view& v = src->tex_views[k];
            if (v.rgb_w < 1 || v.rgb_h < 1 || !dev_ptr(v.rgb))
                return set_err(c, FTR_EINVAL, "ftr_render: view %d needs a device RGB image", k);
            tex.rgb_w[k] = v.rgb_w;
            tex.rgb_h[k] = v.rgb_h;
            tex.rgb[k] = v.rgb;
        }
    }
    EvalScratch* ev = eval_scratch(c);
    if (!ev) return set_err(c, FTR_ENOMEM, "ftr_render: scratch");
    const int64_t npx = (int64_t)cam->w * cam->h;
    cudaError_t e;
    if (npx > ev->zkey_cap) {
        cudaStreamSynchronize(c->stream);
        if (ev->zkey) cudaFree(ev->zkey);
        ev->zkey = nullptr;
        ev->zkey_cap = 0;
        if ((e = cudaMalloc((void**)&ev->zkey, (size_t)npx * sizeof(unsigned long long))) != cudaSuccess)
            return cuda_fail(c, e, "ftr_render: z-buffer");
        ev->zkey_cap = npx;
    }
    if (src->n_tris + 1 > ev->big_cap) {
        cudaStreamSynchronize(c->stream);
        if (ev->big) cudaFree(ev->big);
        ev->big = nullptr;
        ev->big_cap = 0;
        if ((e = cudaMalloc((void**)&ev->big, (size_t)(src->n_tris + 1) * sizeof(int))) != cudaSuccess)
            return cuda_fail(c, e, "ftr_render: triangle list");
        ev->big_cap = src->n_tris + 1;
    }
    const CamDev cd = make_cam(*cam);
    if ((e = cudaMemsetAsync(ev->zkey, 0xff, (size_t)npx * sizeof(unsigned long long), c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_render: clear");
    if (src->n_tris > 0) {
        int* nbig = ev->big + src->n_tris;
        if ((e = cudaMemsetAsync(nbig, 0, sizeof(int), c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "ftr_render: clear");
        k_raster<<<(unsigned)((src->n_tris + 127) / 128), 128, 0, c->stream>>>(
            cd, src->vertices, src->tris, src->n_tris, src->n_vertices, ev->zkey, ev->big, nbig);
        k_raster_big<<<2 * 152, 256, 0, c->stream>>>(cd, src->vertices, src->tris, src->n_vertices, ev->zkey, ev->big,
                                                     nbig);
        c->launches += 2;
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ftr_render: raster");
    }
    k_resolve<<<(unsigned)((npx + 255) / 256), 256, 0, c->stream>>>(
        cd, src->vertices, src->tris, ev->zkey, depth_out, rgb_out, src->vertex_rgb, src->tex_weights,
        src->tex_uv, tex);
    c->launches++;
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ftr_render: resolve");
    return FTR_OK;
}
