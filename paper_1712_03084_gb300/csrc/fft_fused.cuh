// Plane transforms: the forward x and y passes, and the inverse y and x
// passes, of Sec. III-B's 3D FFT, each fused into one kernel per z-plane.
//
// A z-plane of the half spectrum is (n_x/2 + 1) x n_y complex values (264 KB
// at 256^2), too large for one CTA, so one thread-block cluster of C CTAs
// takes a plane and the transpose between the two axes goes through
// distributed shared memory instead of HBM:
//
//   forward (k_fxy), for each component c of V in turn:
//     X  CTA r transforms its n_y / C rows along x (two real rows per complex
//        transform, separated by Hermitian symmetry), multiplies the x
//        component by j w_x, and keeps the row spectra [k_x][y] in its own
//        shared memory;
//     -- cluster barrier --
//     Y  CTA r gathers its k_x columns (all y) from the C CTAs' shared memory,
//        transforms them along y and writes, for c = y, W = X^ + j w_y Y^
//        (the transform of the x component waits in the output field, read
//        back by the thread that wrote it) and for c = z the transform
//        itself: two fields, layout [z][k_x][k_y].
//   Two component buffers alternate, so one cluster barrier per component
//   (plus one before exit) orders every write before the peers' reads and
//   every read before the buffer is written again.
//
//   inverse (k_iyx): CTA r transforms its k_x columns of A^ (after the
//   inverse z pass, layout [z][k_x][k_y]) back along y into its shared
//   memory; -- cluster barrier --; then it gathers, for its pairs of rows,
//   every k_x from the C CTAs and runs the complex-to-real x transform (two
//   rows per complex inverse), writing A[z][y][x].
//
// The k_x columns split evenly (n_x / 2 / C per CTA) and the last CTA also
// takes the Nyquist column k_x = n_x / 2.  Per line the arithmetic is the
// same four-step transform as the separate axis passes (fft_common.cuh).
#pragma once

#include <cooperative_groups.h>

#include "fft_common.cuh"
#include "ftr_internal.h"

namespace ftr {
namespace fused {

namespace cg = cooperative_groups;

// CTAs per cluster for an n_x x n_y plane: 16 from 384^2, 8 from 128 x 256,
// 4 from 64 x 128, else 2, halved until every CTA gets an even number of
// rows and the same number of k_x columns.
__host__ __device__ constexpr int cluster_for(int nx, int ny) {
    int c = nx * ny >= 384 * 384 ? 16 : (nx * ny >= 128 * 256 ? 8 : (nx * ny >= 64 * 128 ? 4 : 2));
    while (c > 1 && ((ny % (2 * c)) != 0 || ((nx / 2) % c) != 0)) c /= 2;
    return c;
}

__host__ __device__ constexpr int round_up32(int v) { return (v + 31) / 32 * 32; }

template <int NX, int NY, int CF = 0>
struct Cfg {
    static constexpr int C = CF > 0 ? CF : cluster_for(NX, NY);
    static constexpr int RPC = NY / C;            // rows of the plane per CTA
    static constexpr int LX = RPC / 2;            // complex x lines per CTA (pairs of real rows)
    static constexpr int UPC = (NX / 2) / C;      // k_x columns per CTA (the last CTA: one more)
    static constexpr int LY = UPC + 1;            // y lines per CTA, at most
    static constexpr int NKX = NX / 2 + 1;
    static constexpr int NTX = Xchg<NX, LX>::NT;  // threads per x line
    static constexpr int NTY = Xchg<NY, LY>::NT;  // threads per y line
    static constexpr int THREADS = round_up32(cmax(LX * NTX, LY * NTY));
    static constexpr int XS = cmax(Xchg<NX, LX>::SIZE, Xchg<NY, LY>::SIZE);   // exchange, float2
    static constexpr int BUF = NKX * RPC;         // forward: one component's row spectra [k_x][y_local]
    static constexpr int NYP = NY + 2;            // inverse: column stride (16-byte pad)
    static constexpr int GBUF = LY * NYP;         // inverse: the CTA's inverse-y columns [u][y]
    static constexpr size_t SMEM_FWD = sizeof(float2) * (size_t)(2 * BUF + XS);
    static constexpr size_t SMEM_INV = sizeof(float2) * (size_t)(GBUF + XS);
    static_assert(RPC % 2 == 0 && (NX / 2) % C == 0 && NY % C == 0, "plane split");
    static_assert(XS >= LX * (NX + 1), "the exchange buffer also parks the x spectra");
    static_assert(BUF % 2 == 0 && GBUF % 2 == 0, "16-byte alignment of the buffers after them");
};

// ---------------------------------------------------------------------------
// forward x and y, x/y filter terms, one z-plane per cluster
template <int NX, int NY, int CF = 0>
__global__ void __launch_bounds__(Cfg<NX, NY, CF>::THREADS)
    k_fxy(GridDev g, const int* __restrict__ slot_tab, const float* __restrict__ vpool, float2* out,
          int64_t Mh, const float2* __restrict__ twx, const float2* __restrict__ twy, float wx_scale, float wy_scale,
          const int* __restrict__ meta) {
    using K = Cfg<NX, NY, CF>;
    constexpr int N1X = Plan<NX>::N1, N2X = Plan<NX>::N2;
    constexpr int N1Y = Plan<NY>::N1, N2Y = Plan<NY>::N2;
    constexpr int NBX = NX / kBrick;
    constexpr int NBR = K::RPC / kBrick + 2;
    pdl_wait();
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int z = blockIdx.y;
    // planes outside the slab of touched bricks are zero and never read by
    // the z pass: the whole cluster (one plane) leaves before any barrier
    int zl, zh;
    live_z_range(meta, zl, zh);
    if (z < zl || z >= zh) return;
    extern __shared__ __align__(16) float2 smem[];
    float2* const buf0 = smem;
    float2* const buf1 = smem + K::BUF;
    float2* const xs = smem + 2 * K::BUF;
    __shared__ int s_slot[NBR][NBX];
    const int tid = threadIdx.x;
    const int y0 = r * K::RPC;
    const int by0 = y0 >> 3, nbr = ((y0 + K::RPC - 1) >> 3) - by0 + 1;
    const int bz = z >> 3, lz = z & 7;
    for (int k = tid; k < nbr * NBX; k += K::THREADS) {
        const int rr = k / NBX, bx = k % NBX;
        s_slot[rr][bx] = slot_tab[bx + g.nb[0] * ((by0 + rr) + g.nb[1] * bz)];
    }
    __syncthreads();
    // x lines: element index fastest (the brick rows are contiguous along x)
    const int fx = tid / K::NTX, jx = tid % K::NTX;
    // y lines: element index fastest (a k_x column is contiguous along y)
    const int fy = tid / K::NTY, jy = tid % K::NTY;
    const bool y_line = fy < K::UPC || (fy == K::UPC && r == K::C - 1);
    const int kxl = fy < K::UPC ? r * K::UPC + fy : NX / 2;
    const size_t obase = ((size_t)z * K::NKX + kxl) * NY;
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
        float2* const B = (c & 1) ? buf1 : buf0;
        // ---- X: rows y0 + 2 fx and y0 + 2 fx + 1 of component c as one complex line
        if (fx < K::LX && jx < N2X) {
            const int ya = y0 + 2 * fx, yb = ya + 1;
            const int ra = (ya >> 3) - by0, rb = (yb >> 3) - by0;
            const int la = 8 * ((ya & 7) + 8 * lz), lb = 8 * ((yb & 7) + 8 * lz);
            float2 v[N1X];
#pragma unroll
            for (int n1 = 0; n1 < N1X; ++n1) {
                const int x = N2X * n1 + jx;
                const int sa = s_slot[ra][x >> 3], sb = s_slot[rb][x >> 3];
                const float a = sa >= 0 ? vpool[(size_t)sa * 3 * kBrickVox + c * kBrickVox + la + (x & 7)] : 0.f;
                const float b = sb >= 0 ? vpool[(size_t)sb * 3 * kBrickVox + c * kBrickVox + lb + (x & 7)] : 0.f;
                v[n1] = make_float2(a, b);
            }
            fft_step1<NX, K::LX, -1>(v, fx, jx, xs, twx);
        }
        __syncthreads();
        {
            float2 o[N2X];
            const bool act = fx < K::LX && jx < N1X;
            if (act) fft_step2<NX, K::LX, -1>(o, fx, jx, xs);
            __syncthreads();                           // exchange reads done: park the line spectra
            if (act) {
#pragma unroll
                for (int k2 = 0; k2 < N2X; ++k2) xs[fx * (NX + 1) + jx + N1X * k2] = o[k2];
            }
        }
        __syncthreads();
        // the two real rows' half spectra (Z = a + i b: A = (Z[k] + conj Z[-k]) / 2,
        // B = (Z[k] - conj Z[-k]) / 2i); the x component times j w_x (0 at Nyquist)
        for (int k = tid; k < K::LX * K::NKX; k += K::THREADS) {
            const int p = k % K::LX, kx = k / K::LX;
            const float2 za = xs[p * (NX + 1) + kx];
            const float2 zb = cconj(xs[p * (NX + 1) + (kx == 0 ? 0 : NX - kx)]);
            float2 a = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y + zb.y));
            const float2 d = csub(za, zb);
            float2 b = make_float2(0.5f * d.y, -0.5f * d.x);
            if (c == 0) {
                const float w = (kx == NX / 2) ? 0.f : wx_scale * (float)kx;
                a = make_float2(-w * a.y, w * a.x);
                b = make_float2(-w * b.y, w * b.x);
            }
            reinterpret_cast<float4*>(B)[(kx * K::RPC + 2 * p) >> 1] = make_float4(a.x, a.y, b.x, b.y);
        }
        cl.sync();
        // ---- Y: this CTA's k_x columns, every y from the CTA that holds it
        if (y_line && jy < N2Y) {
            float2 v[N1Y];
#pragma unroll
            for (int n1 = 0; n1 < N1Y; ++n1) {
                const int y = N2Y * n1 + jy;
                const int owner = y / K::RPC;
                const float2* rb = cl.map_shared_rank(B, owner);
                v[n1] = rb[kxl * K::RPC + (y - owner * K::RPC)];
            }
            fft_step1<NY, K::LY, -1>(v, fy, jy, xs, twy);
        }
        __syncthreads();
        if (y_line && jy < N1Y) {
            float2 o[N2Y];
            fft_step2<NY, K::LY, -1>(o, fy, jy, xs);
            if (c == 0) {
                // the x term waits in field 0 (this thread reads it back for c = 1:
                // from L2, without holding registers across the next component)
#pragma unroll
                for (int k2 = 0; k2 < N2Y; ++k2) out[obase + jy + N1Y * k2] = o[k2];
            } else if (c == 1) {
#pragma unroll
                for (int k2 = 0; k2 < N2Y; ++k2) {
                    const int ky = jy + N1Y * k2;
                    const float wy = (ky == NY / 2) ? 0.f : wy_scale * (float)signed_bin(ky, NY);
                    const float2 w = out[obase + ky];
                    out[obase + ky] = make_float2(w.x - wy * o[k2].y, w.y + wy * o[k2].x);
                }
            } else {
#pragma unroll
                for (int k2 = 0; k2 < N2Y; ++k2) out[Mh + obase + jy + N1Y * k2] = o[k2];
            }
        }
        __syncthreads();                               // exchange reads done before the next component
    }
    cl.sync();                                         // no CTA leaves while its buffer may be read
}

// ---------------------------------------------------------------------------
// inverse y and complex-to-real x, one z-plane per cluster
template <int NX, int NY, int CF = 0>
__global__ void __launch_bounds__(Cfg<NX, NY, CF>::THREADS)
    k_iyx(const float2* __restrict__ in, float* __restrict__ A, const float2* __restrict__ twx,
          const float2* __restrict__ twy) {
    using K = Cfg<NX, NY, CF>;
    constexpr int N1X = Plan<NX>::N1, N2X = Plan<NX>::N2;
    constexpr int N1Y = Plan<NY>::N1, N2Y = Plan<NY>::N2;
    pdl_wait();
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int z = blockIdx.y;
    extern __shared__ __align__(16) float2 smem[];
    float2* const G = smem;                    // [u][y], column stride NYP
    float2* const xs = smem + K::GBUF;
    const int tid = threadIdx.x;
    // ---- Y: inverse y of this CTA's k_x columns
    const int fy = tid / K::NTY, jy = tid % K::NTY;
    const bool y_line = fy < K::UPC || (fy == K::UPC && r == K::C - 1);
    const int kxl = fy < K::UPC ? r * K::UPC + fy : NX / 2;
    if (y_line && jy < N2Y) {
        const float2* src = in + ((size_t)z * K::NKX + kxl) * NY;
        float2 v[N1Y];
#pragma unroll
        for (int n1 = 0; n1 < N1Y; ++n1) v[n1] = src[N2Y * n1 + jy];
        fft_step1<NY, K::LY, +1>(v, fy, jy, xs, twy);
    }
    __syncthreads();
    if (y_line && jy < N1Y) {
        float2 o[N2Y];
        fft_step2<NY, K::LY, +1>(o, fy, jy, xs);
#pragma unroll
        for (int k2 = 0; k2 < N2Y; ++k2) G[fy * K::NYP + jy + N1Y * k2] = o[k2];
    }
    cl.sync();
    // ---- X: rows ya = y0 + 2 fx, yb = ya + 1 as Z = X_a + i X_b over every k_x
    const int fx = tid / K::NTX, jx = tid % K::NTX;
    const int ya = r * K::RPC + 2 * fx;
    if (fx < K::LX && jx < N2X) {
        float2 v[N1X];
#pragma unroll
        for (int n1 = 0; n1 < N1X; ++n1) {
            const int k = N2X * n1 + jx;
            const int kk = k <= NX / 2 ? k : NX - k;
            const int owner = kk == NX / 2 ? K::C - 1 : kk / K::UPC;
            const int u = kk == NX / 2 ? K::UPC : kk - owner * K::UPC;
            const float4 q = reinterpret_cast<const float4*>(cl.map_shared_rank(G, owner))[(u * K::NYP + ya) >> 1];
            float2 xa = make_float2(q.x, q.y), xb = make_float2(q.z, q.w);
            if (k == 0 || k == NX / 2) {               // real for an exactly Hermitian spectrum
                xa.y = 0.f;
                xb.y = 0.f;
            } else if (k > NX / 2) {                   // X[n - k] = conj X[k]
                xa = cconj(xa);
                xb = cconj(xb);
            }
            v[n1] = make_float2(xa.x - xb.y, xa.y + xb.x);
        }
        fft_step1<NX, K::LX, +1>(v, fx, jx, xs, twx);
    }
    __syncthreads();
    if (fx < K::LX && jx < N1X) {
        float2 o[N2X];
        fft_step2<NX, K::LX, +1>(o, fx, jx, xs);
        float* ra = A + (size_t)NX * ((size_t)ya + (size_t)NY * z);
        float* rb = ra + NX;
#pragma unroll
        for (int k2 = 0; k2 < N2X; ++k2) {
            ra[jx + N1X * k2] = o[k2].x;
            rb[jx + N1X * k2] = o[k2].y;
        }
    }
    cl.sync();                                 // no CTA leaves while its columns may be read
}

// ---------------------------------------------------------------------------
// z pass on the plane-major fields: forward z of W and of Y^X^V_z, the
// integration filter A^ = (W^ + j w_z V^_z) / |w|^2 / M (numerator w_z = 0 at
// Nyquist, A^(0) = 0), inverse z; A^ overwrites W, layout [z][k_x][k_y].  A
// CTA takes F consecutive k_y at one k_x; line index fastest, so each z of a
// line tile is one F x 8-byte run.  Planes outside [zl, zh) are zero.
template <int N, int F>
__global__ void __launch_bounds__(F * Xchg<N, F>::NT, MinCtasF<N, F>::value)
    k_fz2(GridDev g, float2* __restrict__ s, int64_t Mh, const float2* __restrict__ tw, float wx_scale,
          float wy_scale, float wz_scale, float inv_m, const int* __restrict__ meta) {
    pdl_wait();
    using X = Xchg<N, F>;
    extern __shared__ float2 smem[];
    const int ny = g.n[1], nkx = g.n[0] / 2 + 1;
    const int ky0 = blockIdx.x * F;
    const int kx = blockIdx.y;
    const int tid = threadIdx.x;
    const int f = tid % F, r = tid / F;
    int zl, zh;
    live_z_range(meta, zl, zh);
    const size_t zs = (size_t)nkx * ny;
    const size_t col = (size_t)kx * ny + ky0 + f;
    if (f == 0 && r < X::N2) {              // field 1 goes to L2 while field 0 is transformed
#pragma unroll
        for (int n1 = 0; n1 < X::N1; ++n1) {
            const int z = X::N2 * n1 + r;
            if (z >= zl && z < zh) prefetch_l2(s + Mh + col + z * zs);
        }
    }
    if (r < X::N2) {
        float2 v[X::N1];
#pragma unroll
        for (int n1 = 0; n1 < X::N1; ++n1) {
            const int z = X::N2 * n1 + r;
            v[n1] = (z >= zl && z < zh) ? s[col + z * zs] : make_float2(0.f, 0.f);
        }
        fft_step1<N, F, -1>(v, f, r, smem, tw);
    }
    __syncthreads();
    float2* stash = smem + X::SIZE;
    float2 xw[X::N2];
    if (r < X::N1) {
        fft_step2<N, F, -1>(xw, f, r, smem);
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) stash[f + (F + 1) * (r + X::N1 * k2)] = xw[k2];
    }
    __syncthreads();
    if (r < X::N2) {
        float2 v[X::N1];
#pragma unroll
        for (int n1 = 0; n1 < X::N1; ++n1) {
            const int z = X::N2 * n1 + r;
            v[n1] = (z >= zl && z < zh) ? s[Mh + col + z * zs] : make_float2(0.f, 0.f);
        }
        fft_step1<N, F, -1>(v, f, r, smem, tw);
    }
    __syncthreads();
    float2 xh[X::N2];
    if (r < X::N1) fft_step2<N, F, -1>(xh, f, r, smem);
    __syncthreads();
    if (r < X::N1) {
        const int ky = ky0 + f;
        const float wxd = wx_scale * (float)kx;
        const float wyd = wy_scale * (float)signed_bin(ky, ny);
        const float base = wxd * wxd + wyd * wyd;
#pragma unroll
        for (int k2 = 0; k2 < X::N2; ++k2) {
            const int kz = r + X::N1 * k2;
            const float wzd = wz_scale * (float)signed_bin(kz, N);
            const float wzn = (kz == N / 2) ? 0.f : wzd;
            const float den = base + wzd * wzd;
            const float sc = den > 0.f ? inv_m / den : 0.f;
            const float2 w = stash[f + (F + 1) * kz];
            const float2 sv = make_float2(w.x - wzn * xh[k2].y, w.y + wzn * xh[k2].x);
            xw[k2] = make_float2(sv.x * sc, sv.y * sc);
        }
        fft_step1_swapped<N, F, +1>(xw, f, r, smem, tw);
    }
    __syncthreads();
    if (r < X::N2) {
        float2 o[X::N1];
        fft_step2_swapped<N, F, +1>(o, f, r, smem);
#pragma unroll
        for (int k2 = 0; k2 < X::N1; ++k2) s[col + (size_t)(r + X::N2 * k2) * zs] = o[k2];
    }
}

}  // namespace fused
}  // namespace ftr

namespace ftr {
namespace fused {

// Launch with a cluster of cx CTAs along x, with programmatic dependent launch.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_cluster(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, int cx,
                                  Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = (unsigned)cx;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// Clusters of the kernel that fit on the device at once (0: the launch would fail).
template <typename... KArgs>
inline cudaError_t max_clusters(void (*kernel)(KArgs...), int threads, size_t smem, int cx, int* n) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cx, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cx;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(n, (const void*)kernel, &cfg);
}

// Shared-memory limit and (above 8 CTAs) the non-portable cluster size, once
// per kernel and device.
template <class Kern>
inline cudaError_t prepare(Kern kernel, size_t smem, int cx, int device) {
    cudaError_t e = ensure_smem(kernel, smem, device);
    if (e != cudaSuccess || cx <= 8) return e;
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair((const void*)kernel, device);
    if (done.count(key)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

// which: 0 launch the forward plane kernel, 1 the inverse one; 2 / 3 store
// in *n the clusters of the forward / inverse kernel that fit at once.
template <int NX, int NY>
cudaError_t run_pair(ftr_ctx* c, int which, int* n) {
    using K = Cfg<NX, NY>;
    cudaError_t e;
    if (which == 0 || which == 2) {
        if ((e = prepare(k_fxy<NX, NY>, K::SMEM_FWD, K::C, c->device)) != cudaSuccess) return e;
        if (which == 2) return max_clusters(k_fxy<NX, NY>, K::THREADS, K::SMEM_FWD, K::C, n);
        const double two_pi = 2.0 * 3.14159265358979323846;
        const float wx = (float)(two_pi / (c->g.n[0] * c->g.h[0]));
        const float wy = (float)(two_pi / (c->g.n[1] * c->g.h[1]));
        e = launch_cluster(k_fxy<NX, NY>, dim3(K::C, c->g.n[2]), dim3(K::THREADS), K::SMEM_FWD, c->stream, K::C, c->g,
                           (const int*)c->d_brick_slot, (const float*)c->d_vpool, c->d_s1, c->Mh,
                           (const float2*)c->d_tw[0], (const float2*)c->d_tw[1], wx, wy, (const int*)c->d_meta);
    } else {
        if ((e = prepare(k_iyx<NX, NY>, K::SMEM_INV, K::C, c->device)) != cudaSuccess) return e;
        if (which == 3) return max_clusters(k_iyx<NX, NY>, K::THREADS, K::SMEM_INV, K::C, n);
        e = launch_cluster(k_iyx<NX, NY>, dim3(K::C, c->g.n[2]), dim3(K::THREADS), K::SMEM_INV, c->stream, K::C,
                           (const float2*)c->d_s1, c->d_A, (const float2*)c->d_tw[0], (const float2*)c->d_tw[1]);
    }
    if (e != cudaSuccess) return e;
    c->launches++;
    return cudaGetLastError();
}

// the instantiated planes, split over two translation units (build time)
bool dispatch_a(ftr_ctx* c, int which, int* n, cudaError_t* e);
bool dispatch_b(ftr_ctx* c, int which, int* n, cudaError_t* e);

}  // namespace fused
}  // namespace ftr
