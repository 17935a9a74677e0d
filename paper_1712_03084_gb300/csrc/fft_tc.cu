// Split-precision tensor-core variant of the five FFT passes (Sec. III-B
// transforms, the same data flow and fusions as the fp32 passes).
//
// Every small DFT of the four-step decomposition N = N1 N2 (see
// fft_common.cuh) becomes a real matrix product on the fifth-generation
// tensor cores.  A batch of length-R complex vectors is a row-major real
// matrix X (rows x 2R, re/im interleaved) and the DFT a fixed real 2R x 2R
// matrix D_R (for W = exp(s 2 pi i / R): [re im] blocks [c -w; w c] of the
// entries w = W^{mq}).  Both operands are split into two 16-bit parts,
// x = x_hi + x_lo with x_hi = round16(x), x_lo = round16(x - x_hi), and the
// product is accumulated in fp32 Tensor Memory as
//   X D ~ X_lo D_hi + X_hi D_lo + X_hi D_hi
// (the dropped X_lo D_lo term is 2^-16 (bf16) or 2^-22 (fp16) of the result).
// bf16 parts keep the fp32 exponent range; fp16 parts do not, so in the fp16
// variant every line is first scaled by a power of two that brings its
// largest component into [1/2, 1) and scaled back after the transform
// (exact).  The twiddles W_N^{j k1} between the two steps, the filter and
// all other arithmetic stay fp32.
//
// One CTA keeps the fp32 passes' tile of F lines.  Step 1: thread (f, j)
// writes its row x[N2 n1 + j] (n1 < N1) of the operand, one thread issues the
// MMAs of all 128-row tiles, every thread reads its row back from Tensor
// Memory (warp w owns lanes 32 (w % 4) ..  of tile w / 4), applies the
// twiddles and scatters the values into the step-2 operand (the exchange
// transpose); step 2 the same with the roles of N1 and N2 exchanged.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <mutex>
#include <set>
#include <utility>
#include <vector>

#include "fft_common.cuh"
#include "ftr_internal.h"
#include "tc_sm100.cuh"

namespace ftr {
namespace {

// Layout of the DFT-matrix table on the device: one 8 KiB block per
// (R in {8, 16, 24, 32}, sign, part) in the canonical K-major layout.
constexpr int kTcBlock = 8192;
__host__ __device__ constexpr int tc_rindex(int R) { return R / 8 - 1; }
__host__ __device__ constexpr int tc_block(int R, int sign, int part) {
    return ((tc_rindex(R) * 2 + (sign > 0 ? 1 : 0)) * 2 + part) * kTcBlock;
}
constexpr size_t kTcTableBytes = 4 * 2 * 2 * kTcBlock;

// Byte offset of element (row, k) of a K-major operand with 2R columns.
__host__ __device__ constexpr int tc_off(int R, int row, int k) {
    return (row >> 3) * (32 * R) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// The A operands (the data) use padded core-matrix strides: core matrices
// adjacent along K are LBO_A bytes apart and 8-row groups SBO_A bytes apart,
// chosen so that the stores that fill them spread over the 32 shared-memory
// banks (the step-2 operand is written 4 bytes per row by threads that hold
// one K column each; with the dense strides 128 / 32 R those stores conflict
// 8-fold).  The MMA reads any such strides; only the B operands (the DFT
// matrices) keep the dense layout of the table.
__host__ __device__ constexpr int lbo_a(int R) { return R == 8 ? 192 : (R == 16 ? 160 : 144); }
__host__ __device__ constexpr int sbo_a(int R) { return R == 8 ? 336 : (R == 16 ? 624 : (R == 24 ? 880 : 1168)); }
__host__ __device__ constexpr int a_off(int R, int row, int k) {
    return (row >> 3) * sbo_a(R) + (k >> 3) * lbo_a(R) + (row & 7) * 16 + (k & 7) * 2;
}

template <int P> struct Half16;
template <> struct Half16<FTR_PREC_BF16X3> {
    __device__ static unsigned short rn(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
    __device__ static float back(unsigned short b) { return __bfloat162float(__ushort_as_bfloat16(b)); }
};
template <> struct Half16<FTR_PREC_FP16X3> {
    __device__ static unsigned short rn(float x) { return __half_as_ushort(__float2half_rn(x)); }
    __device__ static float back(unsigned short b) { return __half2float(__ushort_as_half(b)); }
};

template <int P>
__device__ __forceinline__ void split16(float x, unsigned short& hi, unsigned short& lo) {
    hi = Half16<P>::rn(x);
    lo = Half16<P>::rn(x - Half16<P>::back(hi));
}

constexpr int cpow2(int v) { return v <= 32 ? 32 : (v <= 64 ? 64 : (v <= 128 ? 128 : (v <= 256 ? 256 : 512))); }
constexpr uint32_t kWaitPolls = 1u << 22;

// Per-CTA tensor-core DFT engine for lines of length N, F lines per CTA,
// F * N1 threads.  FWD / INV: which DFT signs the kernel uses.
template <int N, int F, int P, bool FWD, bool INV>
struct Tc {
    static constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    static_assert(N1 >= N2 && N1 % 8 == 0 && N2 % 8 == 0, "tensor-core plan needs N1 >= N2, both multiples of 8");
    static constexpr int T = F * N1;
    static constexpr int tiles(int rows) { return (rows + 127) / 128; }
    static constexpr int TA = tiles(F * N2);   // rows carrying length-N1 vectors
    static constexpr int TB = tiles(F * N1);   // rows carrying length-N2 vectors
    static constexpr int APART = cmax(TA * 16 * sbo_a(N1), TB * 16 * sbo_a(N2));
    static constexpr int COLS = cpow2(cmax(TA * 2 * N1, TB * 2 * N2));
    static constexpr int NSIGN = (FWD ? 1 : 0) + (INV ? 1 : 0);
    static constexpr int BR1 = 16 * N1 * N1;
    static constexpr int BR2 = (N1 == N2) ? 0 : 16 * N2 * N2;
    static constexpr int BBYTES = NSIGN * (BR1 + BR2);
    static constexpr int TWBYTES = 8 * N;                  // W_N^m, m < N
    static constexpr int HDR = 16 + ((4 * F + 15) / 16) * 16;
    static constexpr int BYTES = HDR + BBYTES + TWBYTES + 2 * APART;

    unsigned char* base;
    uint32_t tmem;
    uint32_t phase;
    int* err;

    __device__ uint64_t* mbar() const { return (uint64_t*)base; }
    __device__ unsigned* linemax() const { return (unsigned*)(base + 16); }
    __device__ unsigned char* bmat(int R, int sign) const {
        const int s = (FWD && INV && sign > 0) ? 1 : 0;
        return base + HDR + s * (BR1 + BR2) + (R == N1 ? 0 : BR1);
    }
    __device__ const float2* twsm() const { return (const float2*)(base + HDR + BBYTES); }
    __device__ unsigned char* ahi() const { return base + HDR + BBYTES + TWBYTES; }
    __device__ unsigned char* alo() const { return base + HDR + BBYTES + TWBYTES + APART; }

    __device__ void copy_b(const unsigned char* __restrict__ table, int R, int sign) {
        const int bytes = 8 * R * R;
        unsigned char* dst = bmat(R, sign);
        for (int part = 0; part < 2; ++part) {
            const uint4* s = (const uint4*)(table + tc_block(R, sign, part));
            uint4* d = (uint4*)(dst + part * bytes);
            for (int i = threadIdx.x; i < bytes / 16; i += blockDim.x) d[i] = s[i];
        }
    }

    // Collective: stage the DFT matrices and the twiddles W_N^m (tw, m < N),
    // allocate Tensor Memory, set up the completion barrier.
    __device__ void init(unsigned char* smem, const unsigned char* __restrict__ table,
                         const float2* __restrict__ tw, int* err_flag) {
        base = smem;
        phase = 0;
        err = err_flag;
        {
            float2* t = (float2*)(base + HDR + BBYTES);
            for (int i = threadIdx.x; i < N; i += blockDim.x) t[i] = tw[i];
        }
        if (FWD) {
            copy_b(table, N1, -1);
            if (N2 != N1) copy_b(table, N2, -1);
        }
        if (INV) {
            copy_b(table, N1, +1);
            if (N2 != N1) copy_b(table, N2, +1);
        }
        if (threadIdx.x < 32) tc::tmem_alloc((uint32_t*)(base + 8), COLS);
        if (threadIdx.x == 0) {
            tc::mbar_init(mbar(), 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        tmem = *(volatile uint32_t*)(base + 8);
    }

    // Collective: release Tensor Memory (every CTA path that called init
    // must reach this).
    __device__ void finish() {
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (threadIdx.x < 32) tc::tmem_dealloc(tmem, COLS);
    }

    // Row `row` of the length-R operand from R complex values times `scale`.
    template <int R>
    __device__ void put_row(int row, const float2 (&v)[R], float scale) {
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            unsigned short h[8], l[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                split16<P>(v[4 * q + i].x * scale, h[2 * i], l[2 * i]);
                split16<P>(v[4 * q + i].y * scale, h[2 * i + 1], l[2 * i + 1]);
            }
            uint4 H, L;
            H.x = h[0] | ((uint32_t)h[1] << 16); H.y = h[2] | ((uint32_t)h[3] << 16);
            H.z = h[4] | ((uint32_t)h[5] << 16); H.w = h[6] | ((uint32_t)h[7] << 16);
            L.x = l[0] | ((uint32_t)l[1] << 16); L.y = l[2] | ((uint32_t)l[3] << 16);
            L.z = l[4] | ((uint32_t)l[5] << 16); L.w = l[6] | ((uint32_t)l[7] << 16);
            const int o = a_off(R, row, 8 * q);
            *(uint4*)(ahi() + o) = H;
            *(uint4*)(alo() + o) = L;
        }
    }

    // Complex value m of row `row` of the length-R operand.
    template <int R>
    __device__ void put1(int row, int m, float2 v) {
        unsigned short hr, lr, hi, li;
        split16<P>(v.x, hr, lr);
        split16<P>(v.y, hi, li);
        const int o = a_off(R, row, 2 * m);
        *(uint32_t*)(ahi() + o) = hr | ((uint32_t)hi << 16);
        *(uint32_t*)(alo() + o) = lr | ((uint32_t)li << 16);
    }

    // Collective: D_t = A_t D_R (sign) for every 128-row tile t of `rows`
    // rows, into Tensor Memory columns [t 2R, t 2R + 2R).
    template <int R, int SIGN>
    __device__ void run(int rows) {
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (threadIdx.x == 0) {
            constexpr uint32_t SBO = 32 * R;                 // B: dense
            constexpr uint32_t LA = lbo_a(R), SA = sbo_a(R);  // A: padded
            const uint32_t id = tc::idesc_f16(P == FTR_PREC_BF16X3, 128, 2 * R);
            const uint32_t a0 = tc::smem_u32(ahi()), a1 = tc::smem_u32(alo());
            const uint32_t b0 = tc::smem_u32(bmat(R, SIGN)), b1 = b0 + 8 * R * R;
            const int nt = tiles(rows);
            for (int t = 0; t < nt; ++t) {
#pragma unroll
                for (int s = 0; s < R / 8; ++s) {
                    const uint32_t ao = t * 16 * SA + s * 2 * LA, bo = s * 256;
                    const uint32_t d = tmem + t * 2 * R;
                    tc::mma_f16(d, tc::desc_kmajor(a1 + ao, LA, SA), tc::desc_kmajor(b0 + bo, 128, SBO), id, s > 0);
                    tc::mma_f16(d, tc::desc_kmajor(a0 + ao, LA, SA), tc::desc_kmajor(b1 + bo, 128, SBO), id, 1);
                    tc::mma_f16(d, tc::desc_kmajor(a0 + ao, LA, SA), tc::desc_kmajor(b0 + bo, 128, SBO), id, 1);
                }
            }
            tc::mma_commit(mbar());
        }
        if (!tc::mbar_wait(mbar(), phase, kWaitPolls)) atomicExch(err, 1);
        phase ^= 1u;
        tc::fence_after_sync();
    }

    // This thread's row (threadIdx.x) of the last product, 2R floats; false
    // when the row lies beyond `rows`.
    template <int R>
    __device__ bool get(int rows, float (&buf)[2 * R]) {
        const int w = threadIdx.x >> 5, t = w >> 2;
        if (t < tiles(rows)) {
            const uint32_t a = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(t * 2 * R);
            if ((2 * R) % 32 == 0) {
#pragma unroll
                for (int c = 0; c < 2 * R / 32; ++c) tc::tmem_ld32(a + 32 * c, buf + 32 * c);
            } else {
#pragma unroll
                for (int c = 0; c < 2 * R / 16; ++c) tc::tmem_ld16(a + 16 * c, buf + 16 * c);
            }
        }
        return (int)threadIdx.x < rows;
    }

    // Collective length-R1 R2 transform of F lines.  In: thread with `act`
    // holds x[R2 n1 + j] (n1 < R1) of line f, j < R2.  Out: thread t < F R1
    // holds X[k1 + R1 k2] (k2 < R2) of line t / R1 with k1 = t % R1, or (with
    // LINE_FAST) of line t % F with k1 = t / F.  tw: W_{R1 R2}^m, m < R1 R2.
    template <int R1, int R2, int SIGN, bool LINE_FAST>
    __device__ void dft(const float2 (&v)[R1], bool act, int f, int j, float2 (&out)[R2]) {
        constexpr int NN = R1 * R2;
        const int tid = threadIdx.x;
        float scale = 1.f;
        if (P == FTR_PREC_FP16X3) {
            __syncthreads();
            if (tid < F) linemax()[tid] = 0u;
            __syncthreads();
            if (act) {
                float m = 0.f;
#pragma unroll
                for (int i = 0; i < R1; ++i) m = fmaxf(m, fmaxf(fabsf(v[i].x), fabsf(v[i].y)));
                atomicMax(&linemax()[f], __float_as_uint(m));
            }
            __syncthreads();
            if (act) {
                int e;
                const float m = __uint_as_float(linemax()[f]);
                if (m > 0.f) {
                    frexpf(m, &e);
                    scale = ldexpf(1.f, -e);
                }
            }
        }
        if (act) put_row<R1>(f * R2 + j, v, scale);
        run<R1, SIGN>(F * R2);
        {
            float buf[2 * R1];
            if (get<R1>(F * R2, buf)) {
                const int f1 = tid / R2, j1 = tid % R2;
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) {
                    float2 y = make_float2(buf[2 * k1], buf[2 * k1 + 1]);
                    if (k1 != 0 && j1 != 0) {
                        float2 w = twsm()[(j1 * k1) % NN];
                        if (SIGN > 0) w.y = -w.y;
                        y = cmul(y, w);
                    }
                    const int row = LINE_FAST ? k1 * F + f1 : f1 * R1 + k1;
                    put1<R2>(row, j1, y);
                }
            }
        }
        run<R2, SIGN>(F * R1);
        float buf[2 * R2];
        if (get<R2>(F * R1, buf)) {
            float inv = 1.f;
            if (P == FTR_PREC_FP16X3) {
                const int fo = LINE_FAST ? tid % F : tid / R1;
                const float m = __uint_as_float(linemax()[fo]);
                if (m > 0.f) {
                    int e;
                    frexpf(m, &e);
                    inv = ldexpf(1.f, e);
                }
            }
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) out[k2] = make_float2(buf[2 * k2] * inv, buf[2 * k2 + 1] * inv);
        }
    }
};

// ---------------------------------------------------------------- x forward
// Same as the fp32 x pass: 16 rows (y0.., z) of the three components from the
// brick pool, two real rows per complex line (16 (V_x, V_y) + 8 (V_z, V_z)
// lines), half spectra out in [c][k_x][z][y], j w_x applied to c = x.
constexpr int kFxRows = 16;
constexpr int kFxLines = 24;

template <int N, int P>
__global__ void __launch_bounds__(kFxLines * Plan<N>::N1)
    k_tc_fx(GridDev g, const int* __restrict__ slot_tab, const float* __restrict__ vpool, float2* __restrict__ s0,
            int64_t Mh, const float2* __restrict__ tw, float wx_scale, const int* __restrict__ meta,
            const unsigned char* __restrict__ table, int* err) {
    pdl_wait();
    using E = Tc<N, kFxLines, P, true, false>;
    constexpr int N1 = E::N1, N2 = E::N2;
    constexpr int NB = N / kBrick;
    constexpr int NKX = N / 2 + 1;
    constexpr int ZS = kFxLines + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_slot[2][NB];
    __shared__ int s_any;
    const int ny = g.n[1], nz = g.n[2];
    const int y0 = blockIdx.x * kFxRows;
    const int z = blockIdx.y;
    const int tid = threadIdx.x;
    int zl, zh;
    live_z_range(meta, zl, zh);
    if (z < zl || z >= zh) return;
    if (tid == 0) s_any = 0;
    __syncthreads();
    const int bz = z >> 3;
    for (int k = tid; k < 2 * NB; k += blockDim.x) {
        const int r = k / NB, bx = k % NB;
        const int s = slot_tab[bx + g.nb[0] * ((y0 >> 3) + r + g.nb[1] * bz)];
        s_slot[r][bx] = s;
        if (s >= 0) s_any = 1;
    }
    __syncthreads();
    if (!s_any) {
        const float2 zero = make_float2(0.f, 0.f);
        for (int k = tid; k < kFxRows * NKX; k += blockDim.x) {
            const int r = k & (kFxRows - 1), kx = k >> 4;
            const size_t o = (size_t)(y0 + r) + (size_t)ny * (z + (size_t)nz * kx);
            s0[o] = zero;
            s0[Mh + o] = zero;
            s0[2 * Mh + o] = zero;
        }
        return;
    }
    E e;
    e.init(smem_raw, table, tw, err);
    // the transformed lines are parked in the operand buffers, which are free
    // once the last product has been read back
    static_assert(sizeof(float2) * ZS * N <= 2 * E::APART, "park fits the operand buffers");
    float2* park = (float2*)e.ahi();
    const int f = tid / N1, r = tid % N1;
    const int lz = z & 7;
    const bool act = r < N2;
    float2 v[N1];
    if (act) {
        const int ra = f < 16 ? f : f - 16;
        const int rb = f < 16 ? f : f - 8;
        const int ca = f < 16 ? 0 : 2;
        const int cb = f < 16 ? 1 : 2;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const int x = N2 * n1 + r;
            const int sa = s_slot[ra >> 3][x >> 3];
            const int sb = s_slot[rb >> 3][x >> 3];
            const int la = (x & 7) + 8 * ((ra & 7) + 8 * lz);
            const int lb = (x & 7) + 8 * ((rb & 7) + 8 * lz);
            const float a = sa >= 0 ? vpool[(size_t)sa * 3 * kBrickVox + ca * kBrickVox + la] : 0.f;
            const float b = sb >= 0 ? vpool[(size_t)sb * 3 * kBrickVox + cb * kBrickVox + lb] : 0.f;
            v[n1] = make_float2(a, b);
        }
    }
    float2 o[N2];
    e.template dft<N1, N2, -1, false>(v, act, f, r, o);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) park[f + ZS * (r + N1 * k2)] = o[k2];
    __syncthreads();
    for (int k = tid; k < kFxRows * NKX; k += blockDim.x) {
        const int row = k & (kFxRows - 1), kx = k >> 4;
        const int km = kx == 0 ? 0 : N - kx;
        const float2 za = park[row + ZS * kx];
        const float2 zb = cconj(park[row + ZS * km]);
        float2 vx = make_float2(0.5f * (za.x + zb.x), 0.5f * (za.y + zb.y));
        const float2 dy = csub(za, zb);
        const float2 vy = make_float2(0.5f * dy.y, -0.5f * dy.x);
        const int fz = 16 + (row & 7);
        const float2 zc = park[fz + ZS * kx];
        const float2 zd = cconj(park[fz + ZS * km]);
        float2 vz;
        if (row < 8) {
            vz = make_float2(0.5f * (zc.x + zd.x), 0.5f * (zc.y + zd.y));
        } else {
            const float2 dz = csub(zc, zd);
            vz = make_float2(0.5f * dz.y, -0.5f * dz.x);
        }
        const float wx = (kx == N / 2) ? 0.f : wx_scale * (float)kx;
        vx = make_float2(-wx * vx.y, wx * vx.x);
        const size_t oi = (size_t)(y0 + row) + (size_t)ny * (z + (size_t)nz * kx);
        s0[oi] = vx;
        s0[Mh + oi] = vy;
        s0[2 * Mh + oi] = vz;
    }
    e.finish();
}

// Lines per CTA of the y, inverse-y and z passes: 16; the z pass takes 8
// where the step-1 DFT is longer than 16 (384 points: a CTA of 8 x 24
// threads, three of which fit an SM; measured faster there, and slower for
// the y passes).
template <int N>
struct TcLines {
    static constexpr int value = 16;
};
template <int N>
struct TcLinesZ {
    static constexpr int value = Plan<N>::N1 > 16 ? 8 : 16;
};

// ---------------------------------------------------------------- y forward
// Same as the fp32 y pass: F y lines per component, W = Y[j w_x X V_x] +
// j w_y Y[X V_y] and Y[X V_z] out in [k_x][k_y][z].

template <int N, int P>
__global__ void __launch_bounds__(TcLines<N>::value * Plan<N>::N1, TcLines<N>::value * Plan<N>::N1 <= 256 ? 2 : 1)
    k_tc_fy(GridDev g, const float2* __restrict__ s0, float2* __restrict__ s1, int64_t Mh,
            const float2* __restrict__ tw, float wy_scale, const int* __restrict__ meta,
            const unsigned char* __restrict__ table, int* err) {
    pdl_wait();
    using E = Tc<N, TcLines<N>::value, P, true, false>;
    constexpr int N1 = E::N1, N2 = E::N2;
    constexpr int F = TcLines<N>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nz = g.n[2];
    const int z0 = blockIdx.x * F;
    const int kx = blockIdx.y;
    const int tid = threadIdx.x;
    int zl, zh;
    live_z_range(meta, zl, zh);
    if (z0 < zl || z0 >= zh) return;
    E e;
    e.init(smem_raw, table, tw, err);
    float2* stash = (float2*)(smem_raw + E::BYTES);
    const int f1 = tid / N1, r1 = tid % N1;
    const bool act = r1 < N2;
    const int f2 = tid % F, i2 = tid / F;
    const size_t out_base = (size_t)(z0 + f2) + (size_t)nz * ((size_t)N * kx);
    const float2* line = s0 + (size_t)N * (z0 + f1 + (size_t)nz * kx);
    float2 v[N1], o[N2];
    for (int c = 0; c < 3; ++c) {
        if (act) {
#pragma unroll
            for (int n1 = 0; n1 < N1; ++n1) v[n1] = line[(size_t)c * Mh + N2 * n1 + r1];
        }
        e.template dft<N1, N2, -1, true>(v, act, f1, r1, o);
        if (c == 0) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) stash[f2 + (F + 1) * (i2 + N1 * k2)] = o[k2];
        } else if (c == 1) {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) {
                const int ky = i2 + N1 * k2;
                const float wy = (ky == N / 2) ? 0.f : wy_scale * (float)signed_bin(ky, N);
                const float2 w = stash[f2 + (F + 1) * ky];
                s1[out_base + (size_t)nz * ky] = make_float2(w.x - wy * o[k2].y, w.y + wy * o[k2].x);
            }
        } else {
#pragma unroll
            for (int k2 = 0; k2 < N2; ++k2) s1[Mh + out_base + (size_t)nz * (i2 + N1 * k2)] = o[k2];
        }
    }
    e.finish();
}

// ------------------------------------------- z forward + filter + z inverse
template <int N, int P>
__global__ void __launch_bounds__(TcLinesZ<N>::value * Plan<N>::N1, TcLinesZ<N>::value * Plan<N>::N1 <= 256 ? 3 : 1)
    k_tc_fz(GridDev g, float2* __restrict__ s1, int64_t Mh, const float2* __restrict__ tw, float wx_scale,
            float wy_scale, float wz_scale, float inv_m, const int* __restrict__ meta,
            const unsigned char* __restrict__ table, int* err) {
    pdl_wait();
    using E = Tc<N, TcLinesZ<N>::value, P, true, true>;
    constexpr int N1 = E::N1, N2 = E::N2;
    constexpr int F = TcLinesZ<N>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ny = g.n[1];
    const int ky0 = blockIdx.x * F;
    const int kx = blockIdx.y;
    const int tid = threadIdx.x;
    const int f = tid / N1, r = tid % N1;
    const bool act = r < N2;
    int zl, zh;
    live_z_range(meta, zl, zh);
    E e;
    e.init(smem_raw, table, tw, err);
    const size_t line = (size_t)N * ((size_t)(ky0 + f) + (size_t)ny * kx);
    float2 v[N1], xw[N2], xh[N2];
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
        const int z = N2 * n1 + r;
        v[n1] = (act && z >= zl && z < zh) ? s1[line + z] : make_float2(0.f, 0.f);
    }
    e.template dft<N1, N2, -1, false>(v, act, f, r, xw);
#pragma unroll
    for (int n1 = 0; n1 < N1; ++n1) {
        const int z = N2 * n1 + r;
        v[n1] = (act && z >= zl && z < zh) ? s1[Mh + line + z] : make_float2(0.f, 0.f);
    }
    e.template dft<N1, N2, -1, false>(v, act, f, r, xh);
    // thread (f, r): bins k_z = r + N1 k2 of line f
    {
        const int ky = ky0 + f;
        const float wxd = wx_scale * (float)kx;
        const float wyd = wy_scale * (float)signed_bin(ky, ny);
        const float base = wxd * wxd + wyd * wyd;
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) {
            const int kz = r + N1 * k2;
            const float wzd = wz_scale * (float)signed_bin(kz, N);
            const float wzn = (kz == N / 2) ? 0.f : wzd;
            const float den = base + wzd * wzd;
            const float s = den > 0.f ? inv_m / den : 0.f;
            const float2 sv = make_float2(xw[k2].x - wzn * xh[k2].y, xw[k2].y + wzn * xh[k2].x);
            xw[k2] = make_float2(sv.x * s, sv.y * s);
        }
    }
    // inverse along z, N = N2 x N1: thread (f, r) holds x[r + N1 k2]
    float2 o[N1];
    e.template dft<N2, N1, +1, false>(xw, true, f, r, o);
    if (tid < F * N2) {
        const int fo = tid / N2, ko = tid % N2;
        float2* dst = s1 + (size_t)N * ((size_t)(ky0 + fo) + (size_t)ny * kx);
#pragma unroll
        for (int k2 = 0; k2 < N1; ++k2) dst[ko + N2 * k2] = o[k2];
    }
    e.finish();
}

// ---------------------------------------------------------------- y inverse
template <int N, int P>
__global__ void __launch_bounds__(TcLines<N>::value * Plan<N>::N1)
    k_tc_iy(GridDev g, const float2* __restrict__ src, float2* __restrict__ dst, const float2* __restrict__ tw,
            const unsigned char* __restrict__ table, int* err) {
    pdl_wait();
    using E = Tc<N, TcLines<N>::value, P, false, true>;
    constexpr int N1 = E::N1, N2 = E::N2;
    constexpr int F = TcLines<N>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nz = g.n[2];
    const int z0 = blockIdx.x * F;
    const int kx = blockIdx.y;
    const int tid = threadIdx.x;
    E e;
    e.init(smem_raw, table, tw, err);
    const int f1 = tid % F, j1 = tid / F;
    const bool act = j1 < N2;
    float2 v[N1], o[N2];
    if (act) {
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const int ky = N2 * n1 + j1;
            v[n1] = src[(size_t)(z0 + f1) + (size_t)nz * ((size_t)ky + (size_t)N * kx)];
        }
    }
    e.template dft<N1, N2, +1, false>(v, act, f1, j1, o);
    const int f2 = tid / N1, i2 = tid % N1;
    float2* out = dst + (size_t)N * ((size_t)(z0 + f2) + (size_t)nz * kx);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) out[i2 + N1 * k2] = o[k2];
    e.finish();
}

// ---------------------------------------------------------------- x inverse
constexpr int kIxRows = 16;
constexpr int kIxLines = 8;
constexpr int kHs = kIxRows + 1;

template <int N, int P>
__global__ void __launch_bounds__(kIxLines * Plan<N>::N1)
    k_tc_ix(GridDev g, const float2* __restrict__ src, float* __restrict__ A, const float2* __restrict__ tw,
            const unsigned char* __restrict__ table, int* err) {
    pdl_wait();
    using E = Tc<N, kIxLines, P, false, true>;
    constexpr int N1 = E::N1, N2 = E::N2;
    constexpr int NKX = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int ny = g.n[1], nz = g.n[2];
    const int y0 = blockIdx.x * kIxRows;
    const int z = blockIdx.y;
    const int tid = threadIdx.x;
    E e;
    e.init(smem_raw, table, tw, err);
    // the half-spectrum rows are staged in the operand buffers, which the
    // transform fills only after every thread has read its inputs
    static_assert(sizeof(float2) * kHs * (N / 2 + 1) <= 2 * E::APART, "staging fits the operand buffers");
    float2* hs = (float2*)e.ahi();
    for (int k = tid; k < kIxRows * NKX; k += blockDim.x) {
        const int row = k & (kIxRows - 1), kx = k >> 4;
        hs[kx * kHs + row] = src[(size_t)(y0 + row) + (size_t)ny * (z + (size_t)nz * kx)];
    }
    __syncthreads();
    const int f1 = tid % kIxLines, j1 = tid / kIxLines;
    const bool act = j1 < N2;
    float2 v[N1], o[N2];
    if (act) {
        const int ra = f1, rb = f1 + kIxLines;
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) {
            const int k = N2 * n1 + j1;
            float2 xa, xb;
            if (k <= N / 2) {
                xa = hs[k * kHs + ra];
                xb = hs[k * kHs + rb];
                if (k == 0 || k == N / 2) {
                    xa.y = 0.f;
                    xb.y = 0.f;
                }
            } else {
                xa = cconj(hs[(N - k) * kHs + ra]);
                xb = cconj(hs[(N - k) * kHs + rb]);
            }
            v[n1] = make_float2(xa.x - xb.y, xa.y + xb.x);
        }
    }
    __syncthreads();                             // every input is in registers: the staging area becomes the operand
    e.template dft<N1, N2, +1, false>(v, act, f1, j1, o);
    const int f2 = tid / N1, i2 = tid % N1;
    float* ra = A + (size_t)N * ((size_t)(y0 + f2) + (size_t)ny * z);
    float* rb = A + (size_t)N * ((size_t)(y0 + f2 + kIxLines) + (size_t)ny * z);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) {
        ra[i2 + N1 * k2] = o[k2].x;
        rb[i2 + N1 * k2] = o[k2].y;
    }
    e.finish();
}

// ---------------------------------------------------------------- launchers
// Raise a kernel's dynamic shared-memory limit once per device.
std::mutex g_smem_mu;
std::set<std::pair<const void*, int>> g_smem_done;

template <class K>
cudaError_t set_smem(K kernel, size_t bytes, int device) {
    std::lock_guard<std::mutex> lk(g_smem_mu);
    const auto key = std::make_pair((const void*)kernel, device);
    if (g_smem_done.count(key)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g_smem_done.insert(key);
    return e;
}

template <int N, int P>
cudaError_t run_pass(ftr_ctx* c, int pass, bool launch) {
    const double two_pi = 2.0 * 3.14159265358979323846;
    const unsigned char* tab = c->d_tc_table;
    int* err = c->d_tc_err;
    cudaError_t e;
    switch (pass) {
        case 0: {
            using E = Tc<N, kFxLines, P, true, false>;
            const size_t smem = E::BYTES;
            if ((e = set_smem(k_tc_fx<N, P>, smem, c->device)) != cudaSuccess) return e;
            if (!launch) return cudaSuccess;
            dim3 grid(c->g.n[1] / kFxRows, c->g.n[2]);
            const float wx = (float)(two_pi / (c->g.n[0] * c->g.h[0]));
            launch_pdl(k_tc_fx<N, P>, grid, E::T, smem, c->stream, c->g, c->d_brick_slot, c->d_vpool, c->d_s0, c->Mh,
                                                          c->d_tw[0], wx, c->d_meta, tab, err);
            break;
        }
        case 1: {
            using E = Tc<N, TcLines<N>::value, P, true, false>;
            const size_t smem = E::BYTES + sizeof(float2) * (TcLines<N>::value + 1) * N;
            if ((e = set_smem(k_tc_fy<N, P>, smem, c->device)) != cudaSuccess) return e;
            if (!launch) return cudaSuccess;
            dim3 grid(c->g.n[2] / TcLines<N>::value, c->g.n[0] / 2 + 1);
            const float wy = (float)(two_pi / (c->g.n[1] * c->g.h[1]));
            launch_pdl(k_tc_fy<N, P>, grid, E::T, smem, c->stream, c->g, c->d_s0, c->d_s1, c->Mh, c->d_tw[1], wy,
                                                          c->d_meta, tab, err);
            break;
        }
        case 2: {
            using E = Tc<N, TcLinesZ<N>::value, P, true, true>;
            const size_t smem = E::BYTES;
            if ((e = set_smem(k_tc_fz<N, P>, smem, c->device)) != cudaSuccess) return e;
            if (!launch) return cudaSuccess;
            dim3 grid(c->g.n[1] / TcLinesZ<N>::value, c->g.n[0] / 2 + 1);
            const float wx = (float)(two_pi / (c->g.n[0] * c->g.h[0]));
            const float wy = (float)(two_pi / (c->g.n[1] * c->g.h[1]));
            const float wz = (float)(two_pi / (c->g.n[2] * c->g.h[2]));
            const float inv_m = (float)(1.0 / (double)c->M);
            launch_pdl(k_tc_fz<N, P>, grid, E::T, smem, c->stream, c->g, c->d_s1, c->Mh, c->d_tw[2], wx, wy, wz, inv_m,
                                                          c->d_meta, tab, err);
            break;
        }
        case 3: {
            using E = Tc<N, TcLines<N>::value, P, false, true>;
            const size_t smem = E::BYTES;
            if ((e = set_smem(k_tc_iy<N, P>, smem, c->device)) != cudaSuccess) return e;
            if (!launch) return cudaSuccess;
            dim3 grid(c->g.n[2] / TcLines<N>::value, c->g.n[0] / 2 + 1);
            launch_pdl(k_tc_iy<N, P>, grid, E::T, smem, c->stream, c->g, c->d_s1, c->d_s0, c->d_tw[1], tab, err);
            break;
        }
        default: {
            using E = Tc<N, kIxLines, P, false, true>;
            const size_t smem = E::BYTES;
            if ((e = set_smem(k_tc_ix<N, P>, smem, c->device)) != cudaSuccess) return e;
            if (!launch) return cudaSuccess;
            dim3 grid(c->g.n[1] / kIxRows, c->g.n[2]);
            launch_pdl(k_tc_ix<N, P>, grid, E::T, smem, c->stream, c->g, c->d_s0, c->d_A, c->d_tw[0], tab, err);
            break;
        }
    }
    c->launches++;
    return cudaGetLastError();
}

template <int P>
cudaError_t run_pass_n(ftr_ctx* c, int pass, int n, bool launch) {
    switch (n) {
        case 64: return run_pass<64, P>(c, pass, launch);
        case 128: return run_pass<128, P>(c, pass, launch);
        case 256: return run_pass<256, P>(c, pass, launch);
        case 384: return run_pass<384, P>(c, pass, launch);
        default: return cudaErrorInvalidValue;
    }
}

int pass_axis(int pass) { return pass == 0 || pass == 4 ? 0 : (pass == 1 || pass == 3 ? 1 : 2); }

}  // namespace

bool tc_supported_n(int n) { return n == 64 || n == 128 || n == 256 || n == 384; }

size_t tc_table_bytes() { return kTcTableBytes; }

namespace {

// The real 2R x 2R DFT matrices (B operand, K-major: element (output column
// nn, input row kk)) of R = 8, 16, 24, 32 and both signs, split into hi / lo
// 16-bit parts: one thread per complex entry (R, sign, q, m), the cos / sin
// of 2 pi (m q mod R) / R in float64 (sincospi: exact at the quarter points).
template <int P>
__global__ void k_tc_table(unsigned char* __restrict__ out) {
    const int Rs[4] = {8, 16, 24, 32};
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    for (int ri = 0; ri < 4; ++ri) {
        const int R = Rs[ri];
        const int per_sign = R * R;
        if (t >= 2 * per_sign) {
            t -= 2 * per_sign;
            continue;
        }
        const int sign = t < per_sign ? -1 : 1;
        const int u = t % per_sign;
        const int q = u / R, m = u % R;
        const int jm = (m * q) % R;
        double sn, cs;
        sincospi(2.0 * (double)jm / (double)R, &sn, &cs);
        const double cr = cs, ci = (double)sign * sn;
        // y_re = sum x_re cr - x_im ci; y_im = sum x_re ci + x_im cr
        const double ent[2][2] = {{cr, -ci}, {ci, cr}};   // [c_out][c_in]
        unsigned short* hi = (unsigned short*)(out + tc_block(R, sign, 0));
        unsigned short* lo = (unsigned short*)(out + tc_block(R, sign, 1));
        for (int co = 0; co < 2; ++co) {
            for (int cin = 0; cin < 2; ++cin) {
                const double x = ent[co][cin];
                const unsigned short h = Half16<P>::rn((float)x);
                const unsigned short l = Half16<P>::rn((float)(x - (double)Half16<P>::back(h)));
                const int o = tc_off(R, 2 * q + co, 2 * m + cin) / 2;
                hi[o] = h;
                lo[o] = l;
            }
        }
        return;
    }
}

}  // namespace

cudaError_t tc_build_table(int precision, unsigned char* table_dev, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(table_dev, 0, kTcTableBytes, st);
    if (e != cudaSuccess) return e;
    const int entries = 2 * (8 * 8 + 16 * 16 + 24 * 24 + 32 * 32);
    if (precision == FTR_PREC_BF16X3)
        k_tc_table<FTR_PREC_BF16X3><<<(entries + 127) / 128, 128, 0, st>>>(table_dev);
    else
        k_tc_table<FTR_PREC_FP16X3><<<(entries + 127) / 128, 128, 0, st>>>(table_dev);
    return cudaGetLastError();
}

cudaError_t launch_tc_pass(ftr_ctx* c, int pass) {
    const int n = c->g.n[pass_axis(pass)];
    if (c->p.precision == FTR_PREC_BF16X3) return run_pass_n<FTR_PREC_BF16X3>(c, pass, n, true);
    return run_pass_n<FTR_PREC_FP16X3>(c, pass, n, true);
}

// Shared-memory limits of the context's five kernels, raised up front so that
// no attribute call falls inside a stream capture.
cudaError_t tc_prepare(ftr_ctx* c) {
    for (int pass = 0; pass < 5; ++pass) {
        const int n = c->g.n[pass_axis(pass)];
        cudaError_t e = c->p.precision == FTR_PREC_BF16X3 ? run_pass_n<FTR_PREC_BF16X3>(c, pass, n, false)
                                                          : run_pass_n<FTR_PREC_FP16X3>(c, pass, n, false);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace ftr
