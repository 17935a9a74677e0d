// Per-vertex texture data (Sec. III-C).
//
// For each mesh vertex X and view k: x_c = R_k X + t_k, (u, v) = K x_c /
// (K x_c).z; X is visible in camera k iff x_c.z > 0, its nearest depth pixel
// (floor(u + 1/2), floor(v + 1/2)) lies inside the image and is foreground
// (D > 0), and |D - x_c.z| <= tau.  Visibility in the RGB camera is taken
// equal to that of its depth camera, as in the paper.  The weight is W_k at
// that depth pixel (0 when invisible, or when the RGB projection leaves the
// RGB image); the UV is the RGB projection in pixels.  The headless stand-in
// for the paper's OpenGL multitexture blend is the weighted mean of bilinear
// RGB samples, stored as floor(c + 1/2).  Every discrete decision (pixel
// choice, z > 0, the depth test, the RGB bounds) must match a float64
// evaluation of the same formulas: each camera is evaluated in float32, and a
// decision whose quantity falls within a guard band (2e-3 px, 1e-4 m) of its
// threshold -- far wider than the float32 error -- is re-decided from that
// quantity recomputed in float64 (float64 is slow on this GPU, so nothing
// else is redone); a vertex within 1e-4 m of a camera plane is evaluated
// entirely in float64.
#include <cuda_runtime.h>
#include <math.h>

#include "ftr_internal.h"

namespace ftr {
namespace {

template <class T>
__device__ __forceinline__ void project(const T* K, const T* RT, const T X[3], T& u, T& v, T& z) {
    const T xc = RT[0] * X[0] + RT[1] * X[1] + RT[2] * X[2] + RT[3];
    const T yc = RT[4] * X[0] + RT[5] * X[1] + RT[6] * X[2] + RT[7];
    const T zc = RT[8] * X[0] + RT[9] * X[1] + RT[10] * X[2] + RT[11];
    const T uu = K[0] * xc + K[1] * yc + K[2] * zc;
    const T vv = K[3] * xc + K[4] * yc + K[5] * zc;
    const T ww = K[6] * xc + K[7] * yc + K[8] * zc;
    u = uu / ww;
    v = vv / ww;
    z = zc;
}

template <class T> struct Cams;
template <> struct Cams<double> {
    __device__ static const double* K(const ViewDev& v) { return v.K; }
    __device__ static const double* RT(const ViewDev& v) { return v.RT; }
    __device__ static const double* Krgb(const ViewDev& v) { return v.Krgb; }
    __device__ static const double* RTrgb(const ViewDev& v) { return v.RTrgb; }
};

template <class T>
__device__ __forceinline__ bool near_half_int(T u, T band) {
    const T s = u + (T)0.5;
    const T d = s - floor(s);
    return d < band || d > (T)1 - band;
}

// One camera for one vertex, entirely in precision T.
template <class T>
__device__ __forceinline__ void eval_camera(const ViewDev& vw, const T X[3], T tau, T& wk, T& ur, T& vr, T rgb[3]) {
    T u, v, z;
    project<T>(Cams<T>::K(vw), Cams<T>::RT(vw), X, u, v, z);
    wk = 0;
    ur = -1;
    vr = -1;
    if (z > (T)0) {
        const T px = floor(u + (T)0.5), py = floor(v + (T)0.5);
        if (px >= (T)0 && px < (T)vw.w && py >= (T)0 && py < (T)vw.h) {
            const int64_t pi = (int64_t)py * vw.w + (int64_t)px;
            const T D = (T)vw.depth[pi];
            if (D > (T)0) {
                const T dz = fabs(D - z);
                if (dz <= tau) wk = (T)vw.conf[pi];
            }
        }
    }
    if (wk > (T)0) {
        T zr;
        project<T>(Cams<T>::Krgb(vw), Cams<T>::RTrgb(vw), X, ur, vr, zr);
        const T xmax = (T)(vw.rgb_w - 1), ymax = (T)(vw.rgb_h - 1);
        if (!(zr > (T)0 && ur >= (T)0 && ur <= xmax && vr >= (T)0 && vr <= ymax)) wk = 0;
    }
    if (wk > (T)0) {
        const T fx0 = floor(ur), fy0 = floor(vr);
        const T fx = ur - fx0, fy = vr - fy0;
        const int x0 = (int)fx0, y0 = (int)fy0;
        const int xa = min(max(x0, 0), vw.rgb_w - 1), xb = min(max(x0 + 1, 0), vw.rgb_w - 1);
        const int ya = min(max(y0, 0), vw.rgb_h - 1), yb = min(max(y0 + 1, 0), vw.rgb_h - 1);
        const uint8_t* p00 = vw.rgb + 3 * ((int64_t)ya * vw.rgb_w + xa);
        const uint8_t* p10 = vw.rgb + 3 * ((int64_t)ya * vw.rgb_w + xb);
        const uint8_t* p01 = vw.rgb + 3 * ((int64_t)yb * vw.rgb_w + xa);
        const uint8_t* p11 = vw.rgb + 3 * ((int64_t)yb * vw.rgb_w + xb);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            rgb[c] = ((T)1 - fx) * ((T)1 - fy) * (T)p00[c] + fx * ((T)1 - fy) * (T)p10[c] +
                     ((T)1 - fx) * fy * (T)p01[c] + fx * fy * (T)p11[c];
    } else {
        ur = -1;
        vr = -1;
    }
}

// One camera for one vertex: everything in float32, except that a decision
// whose float32 quantity lies inside the guard band is re-decided from that
// quantity alone in float64 (the depth camera's u, v for the pixel choice,
// its z for the depth test, the RGB projection for the RGB bounds).  The
// values that are not decisions (W, the UV, the colour) stay float32.
// Returns false only for a vertex within band_m of a camera plane; the
// caller then evaluates the whole camera in float64.
__device__ __forceinline__ bool eval_camera_mixed(const ViewDev& vw, const float X[3], float tau, double taud,
                                                  float& wk, float& ur, float& vr, float rgb[3]) {
    const float band_px = 2e-3f, band_m = 1e-4f;
    const double Xd[3] = {X[0], X[1], X[2]};
    float u, v, z;
    project<float>(vw.Kf, vw.RTf, X, u, v, z);
    wk = 0.f;
    ur = -1.f;
    vr = -1.f;
    if (fabsf(z) < band_m) return false;
    if (z > 0.f) {
        int64_t px, py;
        if (near_half_int(u, band_px) || near_half_int(v, band_px)) {
            double ud, vd, zd;
            project<double>(vw.K, vw.RT, Xd, ud, vd, zd);
            px = (int64_t)floor(ud + 0.5);
            py = (int64_t)floor(vd + 0.5);
        } else {
            px = (int64_t)floorf(u + 0.5f);
            py = (int64_t)floorf(v + 0.5f);
        }
        if (px >= 0 && px < vw.w && py >= 0 && py < vw.h) {
            const int64_t pi = py * vw.w + px;
            const float D = vw.depth[pi];
            if (D > 0.f) {
                const float dz = fabsf(D - z);
                bool vis;
                if (fabsf(dz - tau) < band_m) {
                    const double* RT = vw.RT;
                    const double zd = RT[8] * Xd[0] + RT[9] * Xd[1] + RT[10] * Xd[2] + RT[11];
                    vis = fabs((double)D - zd) <= taud;
                } else {
                    vis = dz <= tau;
                }
                if (vis) wk = vw.conf[pi];
            }
        }
    }
    if (wk > 0.f) {
        float zr;
        project<float>(vw.Krgbf, vw.RTrgbf, X, ur, vr, zr);
        const float xmax = (float)(vw.rgb_w - 1), ymax = (float)(vw.rgb_h - 1);
        bool in;
        if (fabsf(zr) < band_m || fabsf(ur) < band_px || fabsf(ur - xmax) < band_px || fabsf(vr) < band_px ||
            fabsf(vr - ymax) < band_px) {
            double ud, vd, zd;
            project<double>(vw.Krgb, vw.RTrgb, Xd, ud, vd, zd);
            in = zd > 0.0 && ud >= 0.0 && ud <= (double)xmax && vd >= 0.0 && vd <= (double)ymax;
        } else {
            in = zr > 0.f && ur >= 0.f && ur <= xmax && vr >= 0.f && vr <= ymax;
        }
        if (!in) wk = 0.f;
    }
    if (wk > 0.f) {
        const float fx0 = floorf(ur), fy0 = floorf(vr);
        const float fx = ur - fx0, fy = vr - fy0;
        const int x0 = (int)fx0, y0 = (int)fy0;
        const int xa = min(max(x0, 0), vw.rgb_w - 1), xb = min(max(x0 + 1, 0), vw.rgb_w - 1);
        const int ya = min(max(y0, 0), vw.rgb_h - 1), yb = min(max(y0 + 1, 0), vw.rgb_h - 1);
        const uint8_t* p00 = vw.rgb + 3 * ((int64_t)ya * vw.rgb_w + xa);
        const uint8_t* p10 = vw.rgb + 3 * ((int64_t)ya * vw.rgb_w + xb);
        const uint8_t* p01 = vw.rgb + 3 * ((int64_t)yb * vw.rgb_w + xa);
        const uint8_t* p11 = vw.rgb + 3 * ((int64_t)yb * vw.rgb_w + xb);
#pragma unroll
        for (int c = 0; c < 3; ++c)
            rgb[c] = (1.f - fx) * (1.f - fy) * (float)p00[c] + fx * (1.f - fy) * (float)p10[c] +
                     (1.f - fx) * fy * (float)p01[c] + fx * fy * (float)p11[c];
    } else {
        ur = -1.f;
        vr = -1.f;
    }
    return true;
}

// One thread per (vertex, camera): G = next power of two >= k lanes per
// vertex, the blend sums combined across the group with shuffles.
// nv_dev (optional): the vertex count on the device; nv then bounds it.
template <int G>
__global__ void __launch_bounds__(256) k_texture(ViewSet vs, const float* __restrict__ verts, int64_t nv,
                                                 const int* __restrict__ nv_dev, double tau,
                                                 float* __restrict__ wout, float* __restrict__ uvout,
                                                 uint8_t* __restrict__ rgbout, uint8_t* __restrict__ texout) {
    pdl_wait();
    if (nv_dev) nv = min(nv, (int64_t)nv_dev[0]);
    // (vertex, camera) threads; the count is read here, the stride covers any
    // grid size
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x; t0 < nv * G; t0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = t0 + threadIdx.x;
        const int64_t i = t / G;
        const int k = (int)(t % G);
        const bool live = i < nv && k < vs.k;
        float wk = 0.f, ur = -1.f, vr = -1.f, rgb[3] = {0.f, 0.f, 0.f};
        if (live) {
            const ViewDev& vw = vs.v[k];
            const float Xf[3] = {verts[3 * i], verts[3 * i + 1], verts[3 * i + 2]};
            if (!eval_camera_mixed(vw, Xf, (float)tau, tau, wk, ur, vr, rgb)) {
                const double Xd[3] = {Xf[0], Xf[1], Xf[2]};
                double wd, ud, vd, cd[3];
                eval_camera<double>(vw, Xd, tau, wd, ud, vd, cd);
                wk = (float)wd;
                ur = (float)ud;
                vr = (float)vd;
                rgb[0] = (float)cd[0];
                rgb[1] = (float)cd[1];
                rgb[2] = (float)cd[2];
            }
            if (wout) wout[i * vs.k + k] = wk;
            if (uvout) {
                uvout[2 * (i * vs.k + k)] = ur;
                uvout[2 * (i * vs.k + k) + 1] = vr;
            }
        }
        float acc[3], wsum = wk > 0.f ? wk : 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] = wk > 0.f ? wk * rgb[c] : 0.f;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            wsum += __shfl_xor_sync(0xffffffffu, wsum, o, G);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], o, G);
        }
        if (k == 0 && i < nv) {
            if (rgbout) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float col = wsum > 0.f ? floorf(acc[c] / wsum + 0.5f) : 0.f;
                    col = fminf(fmaxf(col, 0.f), 255.f);
                    rgbout[3 * i + c] = (uint8_t)col;
                }
            }
            if (texout) texout[i] = wsum > 0.f ? 1 : 0;
        }
    }
}

}  // namespace

namespace {

cudaError_t run_texture(ftr_ctx* c, const ViewSet& vs, float depth_tol, const float* verts, int64_t nv,
                        const int* nv_dev, float* w, float* uv, uint8_t* rgb, uint8_t* textured) {
    if (nv <= 0) return cudaSuccess;
    prof_begin(c, ST_TEXTURE);
    const int G = vs.k <= 1 ? 1 : (vs.k <= 2 ? 2 : (vs.k <= 4 ? 4 : 8));
    // a thread per (vertex, camera) of the capacity: short CTAs that end at
    // once past the count fill in around concurrent frames' kernels (a
    // one-wave grid-stride launch measured 4-7 % slower with frames in flight)
    const unsigned blocks = (unsigned)((nv * G + 255) / 256);
    const double tau = (double)depth_tol;
    switch (G) {
        case 1: launch_pdl(k_texture<1>, blocks, 256, 0, c->stream, vs, verts, nv, nv_dev, tau, w, uv, rgb, textured); break;
        case 2: launch_pdl(k_texture<2>, blocks, 256, 0, c->stream, vs, verts, nv, nv_dev, tau, w, uv, rgb, textured); break;
        case 4: launch_pdl(k_texture<4>, blocks, 256, 0, c->stream, vs, verts, nv, nv_dev, tau, w, uv, rgb, textured); break;
        default: launch_pdl(k_texture<8>, blocks, 256, 0, c->stream, vs, verts, nv, nv_dev, tau, w, uv, rgb, textured); break;
    }
    c->launches++;
    prof_end(c, ST_TEXTURE);
    return cudaGetLastError();
}

}  // namespace

const void* texture_kernel(int k) {
    const int G = k <= 1 ? 1 : (k <= 2 ? 2 : (k <= 4 ? 4 : 8));
    switch (G) {
        case 1: return reinterpret_cast<const void*>(k_texture<1>);
        case 2: return reinterpret_cast<const void*>(k_texture<2>);
        case 4: return reinterpret_cast<const void*>(k_texture<4>);
        default: return reinterpret_cast<const void*>(k_texture<8>);
    }
}

cudaError_t launch_texture(ftr_ctx* c, const ViewSet& vs, float depth_tol, float* w, float* uv, uint8_t* rgb,
                           uint8_t* textured) {
    return run_texture(c, vs, depth_tol, c->d_verts, c->n_verts, nullptr, w, uv, rgb, textured);
}

cudaError_t launch_texture_vertices(ftr_ctx* c, const ViewSet& vs, float depth_tol, const float* verts, int64_t nv,
                                    float* w, float* uv, uint8_t* rgb, uint8_t* textured) {
    return run_texture(c, vs, depth_tol, verts, nv, nullptr, w, uv, rgb, textured);
}

cudaError_t launch_texture_bounded(ftr_ctx* c, const ViewSet& vs, float depth_tol, int64_t limit, const int* nv_dev,
                                   float* w, float* uv, uint8_t* rgb, uint8_t* textured) {
    return run_texture(c, vs, depth_tol, c->d_verts, limit, nv_dev, w, uv, rgb, textured);
}

}  // namespace ftr
