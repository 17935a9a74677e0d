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
// RGB samples, stored as floor(c + 1/2).  Projections and the blend run in
// float64 so that every discrete decision (pixel choice, visibility) matches
// a float64 evaluation of the same formulas.
#include <cuda_runtime.h>
#include <math.h>

#include "ftr_internal.h"

namespace ftr {
namespace {

__device__ __forceinline__ void project(const double* K, const double* RT, const double X[3], double& u, double& v,
                                        double& z) {
    const double xc = RT[0] * X[0] + RT[1] * X[1] + RT[2] * X[2] + RT[3];
    const double yc = RT[4] * X[0] + RT[5] * X[1] + RT[6] * X[2] + RT[7];
    const double zc = RT[8] * X[0] + RT[9] * X[1] + RT[10] * X[2] + RT[11];
    const double uu = K[0] * xc + K[1] * yc + K[2] * zc;
    const double vv = K[3] * xc + K[4] * yc + K[5] * zc;
    const double ww = K[6] * xc + K[7] * yc + K[8] * zc;
    u = uu / ww;
    v = vv / ww;
    z = zc;
}

__global__ void __launch_bounds__(256) k_texture(ViewSet vs, const float* __restrict__ verts, int64_t nv,
                                                 double tau, float* __restrict__ wout, float* __restrict__ uvout,
                                                 uint8_t* __restrict__ rgbout, uint8_t* __restrict__ texout) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const double X[3] = {verts[3 * i], verts[3 * i + 1], verts[3 * i + 2]};
    double acc[3] = {0.0, 0.0, 0.0};
    double wsum = 0.0;
    for (int k = 0; k < vs.k; ++k) {
        const ViewDev& vw = vs.v[k];
        double u, v, z;
        project(vw.K, vw.RT, X, u, v, z);
        double wk = 0.0;
        double ur = -1.0, vr = -1.0;
        if (z > 0.0) {
            const double px = floor(u + 0.5), py = floor(v + 0.5);
            if (px >= 0.0 && px < (double)vw.w && py >= 0.0 && py < (double)vw.h) {
                const int64_t pi = (int64_t)py * vw.w + (int64_t)px;
                const double D = vw.depth[pi];
                if (D > 0.0 && fabs(D - z) <= tau) wk = vw.conf[pi];
            }
        }
        if (wk > 0.0) {
            double zr;
            project(vw.Krgb, vw.RTrgb, X, ur, vr, zr);
            if (!(zr > 0.0 && ur >= 0.0 && ur <= (double)(vw.rgb_w - 1) && vr >= 0.0 &&
                  vr <= (double)(vw.rgb_h - 1)))
                wk = 0.0;
        }
        if (wk > 0.0) {
            const double fx0 = floor(ur), fy0 = floor(vr);
            const double fx = ur - fx0, fy = vr - fy0;
            const int x0 = (int)fx0, y0 = (int)fy0;
            const int xa = min(max(x0, 0), vw.rgb_w - 1), xb = min(max(x0 + 1, 0), vw.rgb_w - 1);
            const int ya = min(max(y0, 0), vw.rgb_h - 1), yb = min(max(y0 + 1, 0), vw.rgb_h - 1);
            const uint8_t* p00 = vw.rgb + 3 * ((int64_t)ya * vw.rgb_w + xa);
            const uint8_t* p10 = vw.rgb + 3 * ((int64_t)ya * vw.rgb_w + xb);
            const uint8_t* p01 = vw.rgb + 3 * ((int64_t)yb * vw.rgb_w + xa);
            const uint8_t* p11 = vw.rgb + 3 * ((int64_t)yb * vw.rgb_w + xb);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double s = (1.0 - fx) * (1.0 - fy) * p00[c] + fx * (1.0 - fy) * p10[c] +
                                 (1.0 - fx) * fy * p01[c] + fx * fy * p11[c];
                acc[c] += wk * s;
            }
            wsum += wk;
        } else {
            ur = -1.0;
            vr = -1.0;
        }
        if (wout) wout[i * vs.k + k] = (float)wk;
        if (uvout) {
            uvout[2 * (i * vs.k + k)] = (float)ur;
            uvout[2 * (i * vs.k + k) + 1] = (float)vr;
        }
    }
    if (rgbout) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double col = wsum > 0.0 ? floor(acc[c] / wsum + 0.5) : 0.0;
            col = col < 0.0 ? 0.0 : (col > 255.0 ? 255.0 : col);
            rgbout[3 * i + c] = (uint8_t)col;
        }
    }
    if (texout) texout[i] = wsum > 0.0 ? 1 : 0;
}

}  // namespace

cudaError_t launch_texture(ftr_ctx* c, const ViewSet& vs, float depth_tol, float* w, float* uv, uint8_t* rgb,
                           uint8_t* textured) {
    if (c->n_verts == 0) return cudaSuccess;
    prof_begin(c, ST_TEXTURE);
    k_texture<<<(unsigned)((c->n_verts + 255) / 256), 256, 0, c->stream>>>(vs, c->d_verts, c->n_verts,
                                                                           (double)depth_tol, w, uv, rgb, textured);
    c->launches++;
    prof_end(c, ST_TEXTURE);
    return cudaGetLastError();
}

}  // namespace ftr
