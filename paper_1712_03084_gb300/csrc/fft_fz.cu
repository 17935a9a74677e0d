// z pass: forward transform, integration filter, inverse transform, fused.
//
// Sec. III-B: A^(w) = j (w_x V^_x + w_y V^_y + w_z V^_z) / |w|^2, then the
// inverse 3D FFT.  After the y pass two fields remain per (k_x, k_y, z):
// W = j w_x V^_x + j w_y V^_y and V^_z (each transformed along x and y).  A CTA
// takes 16 z lines (k_y0..k_y0+15 at one k_x), transforms both along z,
// forms A^ = (W^ + j w_z V^_z^) / |w|^2 / M (numerator w_z = 0 at the Nyquist
// bin, |k| = n/2 in the denominator, A^(0) = 0), and transforms A^ back along
// z while it is still in registers.  The result overwrites the W line in
// place.  z-planes outside the slab that the splat touched are zero and are
// not read.
#include "fft_common.cuh"
#include "ftr_internal.h"
#include "tc_sm100.cuh"

namespace ftr {
namespace {

// Load line f's elements z = N2 n1 + r (zero outside [zl, zh)) and run step 1.
template <int N, int F>
__device__ __forceinline__ void load_step1(const float2* __restrict__ src, int r, int f, int zl, int zh,
                                           float2* smem, const float2* __restrict__ tw) {
    using X = Xchg<N, F>;
    float2 v[X::N1];
#pragma unroll
    for (int n1 = 0; n1 < X::N1; ++n1) {
        const int z = X::N2 * n1 + r;
        v[n1] = (z >= zl && z < zh) ? src[z] : make_float2(0.f, 0.f);
    }
    fft_step1<N, F, -1>(v, f, r, smem, tw);
}

// F lines per CTA (the tile plan; 8, 16 or 32).
template <int N, int F>
__global__ void __launch_bounds__(F * Xchg<N, F>::NT, MinCtasF<N, F>::value)
    k_fz(GridDev g, float2* __restrict__ s1, int64_t Mh, const float2* __restrict__ tw, float wx_scale,
         float wy_scale, float wz_scale, float inv_m, const int* __restrict__ meta) {
    pdl_wait();
    using X = Xchg<N, F>;
    extern __shared__ float2 smem[];
    const int ny = g.n[1], nx = g.n[0];
    const int ky0 = blockIdx.x * F;
    const int kx = blockIdx.y;
    const int tid = threadIdx.x;
    const int f = tid / X::NT, r = tid % X::NT;
    int zl, zh;
    live_z_range(meta, zl, zh);
    const size_t line = (size_t)N * ((size_t)(ky0 + f) + (size_t)ny * kx);
    // field 1 goes to L2 while field 0 is transformed
    if (r < X::N2 && (r & 15) == 0) {
#pragma unroll
        for (int n1 = 0; n1 < X::N1; ++n1) {
            const int z = X::N2 * n1 + r;
            if (z >= zl && z < zh) prefetch_l2(s1 + Mh + line + z);
        }
    }
    // forward z transforms of W (field 0) and of the x/y-transformed V_z (field 1)
    if (r < X::N2) load_step1<N, F>(s1 + line, r, f, zl, zh, smem, tw);
    __syncthreads();
    // the transformed W waits in shared memory (the same thread reads it back)
    float2* stash = smem + X::SIZE;
    float2 xw[X::N2];
    if (r < X::N1) {
        fft_step2<N, F, -1>(xw, f, r, smem);
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) stash[f + (F + 1) * (r + X::N1 * k2)] = xw[k2];
    }
    __syncthreads();
    if (r < X::N2) load_step1<N, F>(s1 + Mh + line, r, f, zl, zh, smem, tw);
    __syncthreads();
    float2 xh[X::N2];
    if (r < X::N1) fft_step2<N, F, -1>(xh, f, r, smem);
    __syncthreads();
    if (r < X::N1) {
        const int ky = ky0 + f;
        const float wxd = wx_scale * (float)kx;                 // |k_x| <= n_x/2 already
        const float wyd = wy_scale * (float)signed_bin(ky, ny);
        const float base = wxd * wxd + wyd * wyd;
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) {
            const int kz = r + X::N1 * k2;
            const float wzd = wz_scale * (float)signed_bin(kz, N);
            const float wzn = (kz == N / 2) ? 0.f : wzd;
            const float den = base + wzd * wzd;
            const float s = den > 0.f ? inv_m / den : 0.f;
            // S = W^ + j w_z V^_z
            const float2 w = stash[f + (F + 1) * kz];
            const float2 sv = make_float2(w.x - wzn * xh[k2].y, w.y + wzn * xh[k2].x);
            xw[k2] = make_float2(sv.x * s, sv.y * s);
        }
        (void)nx;
        fft_step1_swapped<N, F, +1>(xw, f, r, smem, tw);
    }
    __syncthreads();
    if (r < X::N2) {
        float2 o[X::N1];
        fft_step2_swapped<N, F, +1>(o, f, r, smem);
        float2* dst = s1 + line;
#pragma unroll
        for (int k2 = 0; k2 < X::N1; ++k2) dst[r + X::N2 * k2] = o[k2];
    }
}

// The same pass with both fields' tiles fetched by bulk asynchronous copies
// at the start (per line, only the live z range [zl, zh); the rest of the
// staged line is never read), so that all of the CTA's input is in flight
// at once.  Each field's buffer then serves as its exchange buffer, field
// 0's also as the stash.  Waits are bounded (a timeout sets *err and waits
// once more, so no copy is left in flight).
template <int N, int F>
__global__ void __launch_bounds__(F * Xchg<N, F>::NT, MinCtasF<N, F>::value)
    k_fz_bulk(GridDev g, float2* __restrict__ s1, int64_t Mh, const float2* __restrict__ tw, float wx_scale,
              float wy_scale, float wz_scale, float inv_m, const int* __restrict__ meta, int* err) {
    pdl_wait();
    using X = Xchg<N, F>;
    constexpr int BUF = cmax(X::SIZE, (F + 1) * N);
    extern __shared__ __align__(16) float2 smem[];
    __shared__ uint64_t mbar[2];
    const int ny = g.n[1];
    const int ky0 = blockIdx.x * F;
    const int kx = blockIdx.y;
    const int tid = threadIdx.x;
    const int f = tid / X::NT, r = tid % X::NT;
    int zl, zh;
    live_z_range(meta, zl, zh);
    const uint32_t bytes = (uint32_t)(zh - zl) * (uint32_t)sizeof(float2);
    const size_t tile = (size_t)N * ((size_t)ky0 + (size_t)ny * kx);
    float2* B0 = smem;
    float2* B1 = smem + BUF;
    if (tid < 32) {
        if (tid == 0) {
            tc::mbar_init(&mbar[0], 1);
            tc::mbar_init(&mbar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            tc::mbar_expect_tx(&mbar[0], F * bytes);
            tc::mbar_expect_tx(&mbar[1], F * bytes);
        }
        __syncwarp();
        if (tid < F && bytes > 0) {
            const size_t at = tile + (size_t)N * tid + zl;
            tc::bulk_g2s(B0 + N * tid + zl, s1 + at, bytes, &mbar[0]);
            tc::bulk_g2s(B1 + N * tid + zl, s1 + Mh + at, bytes, &mbar[1]);
        }
    }
    __syncthreads();                              // the barriers are initialised before anyone waits
    auto wait = [&](uint64_t* b) {
        if (!tc::mbar_wait(b, 0, 1u << 22)) {
            atomicExch(err, 1);
            tc::mbar_wait(b, 0, 1u << 22);
        }
    };
    auto staged_step1 = [&](float2* B) {
        float2 v[X::N1];
        if (r < X::N2) {
#pragma unroll
            for (int n1 = 0; n1 < X::N1; ++n1) {
                const int z = X::N2 * n1 + r;
                v[n1] = (z >= zl && z < zh) ? B[f * N + z] : make_float2(0.f, 0.f);
            }
        }
        __syncthreads();                          // the staged lines are in registers: B becomes the exchange
        if (r < X::N2) fft_step1<N, F, -1>(v, f, r, B, tw);
    };
    // forward z transforms of W (field 0) and of the x/y-transformed V_z (field 1)
    wait(&mbar[0]);
    staged_step1(B0);
    __syncthreads();
    float2 xw[X::N2];
    if (r < X::N1) fft_step2<N, F, -1>(xw, f, r, B0);
    __syncthreads();                              // every exchange read done: B0 becomes the stash
    float2* stash = B0;
    if (r < X::N1) {
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) stash[f + (F + 1) * (r + X::N1 * k2)] = xw[k2];
    }
    wait(&mbar[1]);
    staged_step1(B1);
    __syncthreads();
    float2 xh[X::N2];
    if (r < X::N1) fft_step2<N, F, -1>(xh, f, r, B1);
    __syncthreads();
    if (r < X::N1) {
        const int ky = ky0 + f;
        const float wxd = wx_scale * (float)kx;                 // |k_x| <= n_x/2 already
        const float wyd = wy_scale * (float)signed_bin(ky, ny);
        const float base = wxd * wxd + wyd * wyd;
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) {
            const int kz = r + X::N1 * k2;
            const float wzd = wz_scale * (float)signed_bin(kz, N);
            const float wzn = (kz == N / 2) ? 0.f : wzd;
            const float den = base + wzd * wzd;
            const float s = den > 0.f ? inv_m / den : 0.f;
            const float2 w = stash[f + (F + 1) * kz];
            const float2 sv = make_float2(w.x - wzn * xh[k2].y, w.y + wzn * xh[k2].x);
            xw[k2] = make_float2(sv.x * s, sv.y * s);
        }
        fft_step1_swapped<N, F, +1>(xw, f, r, B1, tw);
    }
    __syncthreads();
    if (r < X::N2) {
        float2 o[X::N1];
        fft_step2_swapped<N, F, +1>(o, f, r, B1);
        float2* dst = s1 + tile + (size_t)N * f;
#pragma unroll
        for (int k2 = 0; k2 < X::N1; ++k2) dst[r + X::N2 * k2] = o[k2];
    }
}

template <int N, int F>
cudaError_t run_fz_bulk(ftr_ctx* c) {
    using X = Xchg<N, F>;
    const size_t smem = sizeof(float2) * 2 * cmax(X::SIZE, (F + 1) * N);
    cudaError_t e = ensure_smem(k_fz_bulk<N, F>, smem, c->device);
    if (e != cudaSuccess) return e;
    if (c->occ_query)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(c->occ_query, k_fz_bulk<N, F>, F * X::NT, smem);
    dim3 grid(c->g.n[1] / F, c->g.n[0] / 2 + 1);
    const double two_pi = 2.0 * 3.14159265358979323846;
    const float wx = (float)(two_pi / (c->g.n[0] * c->g.h[0]));
    const float wy = (float)(two_pi / (c->g.n[1] * c->g.h[1]));
    const float wz = (float)(two_pi / (c->g.n[2] * c->g.h[2]));
    const float inv_m = (float)(1.0 / (double)c->M);
    launch_pdl(k_fz_bulk<N, F>, grid, F * X::NT, smem, c->stream, c->g, c->d_s1, c->Mh, c->d_tw[2], wx, wy, wz,
               inv_m, c->d_meta, c->d_kerr);
    c->launches++;
    return cudaGetLastError();
}

template <int N, int F>
cudaError_t run_fz_f(ftr_ctx* c) {
    using X = Xchg<N, F>;
    const size_t smem = sizeof(float2) * (X::SIZE + (F + 1) * N);
    cudaError_t e = ensure_smem(k_fz<N, F>, smem, c->device);
    if (e != cudaSuccess) return e;
    if (c->occ_query)   // the autotuner asks how many CTAs of this plan fit on an SM
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(c->occ_query, k_fz<N, F>, F * X::NT, smem);
    dim3 grid(c->g.n[1] / F, c->g.n[0] / 2 + 1);
    const double two_pi = 2.0 * 3.14159265358979323846;
    const float wx = (float)(two_pi / (c->g.n[0] * c->g.h[0]));
    const float wy = (float)(two_pi / (c->g.n[1] * c->g.h[1]));
    const float wz = (float)(two_pi / (c->g.n[2] * c->g.h[2]));
    const float inv_m = (float)(1.0 / (double)c->M);
    launch_pdl(k_fz<N, F>, grid, F * X::NT, smem, c->stream, c->g, c->d_s1, c->Mh, c->d_tw[2], wx, wy, wz, inv_m,
                                                       c->d_meta);
    c->launches++;
    return cudaGetLastError();
}

template <int N>
cudaError_t run_fz(ftr_ctx* c) {
    switch (c->plan_lines[1]) {
        case 8: return run_fz_f<N, 8>(c);
        case 32: return run_fz_f<N, 32>(c);
        case -16: return run_fz_bulk<N, 16>(c);
        default: return run_fz_f<N, 16>(c);
    }
}

}  // namespace

cudaError_t fft_fz_init(const float2* w96) { return upload_w96_table(w96); }

cudaError_t launch_fz(ftr_ctx* c) {
    if (c->p.precision != FTR_PREC_FP32) return launch_tc_pass(c, 2);
    switch (c->g.n[2]) {
        case 32: return run_fz<32>(c);
        case 48: return run_fz<48>(c);
        case 64: return run_fz<64>(c);
        case 96: return run_fz<96>(c);
        case 128: return run_fz<128>(c);
        case 192: return run_fz<192>(c);
        case 256: return run_fz<256>(c);
        case 384: return run_fz<384>(c);
        case 512: return run_fz<512>(c);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ftr
