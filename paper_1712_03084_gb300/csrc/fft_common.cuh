// Register/shared-memory building blocks of the batched 1D FFT passes.
//
// The 3D transforms of Sec. III-B (forward FFT of the three components of V,
// inverse FFT of the filtered spectrum) are done as one pass per axis.  Every
// pass moves tiles of F independent length-N lines through one CTA:
//
//   N = N1 * N2,  n = N2 n1 + j,  k = k1 + N1 k2
//   X[k1 + N1 k2] = sum_j W_N^{j k1} W_N2^{j k2} sum_n1 x[N2 n1 + j] W_N1^{n1 k1}
//
// step 1: thread j of a line holds x[N2 n1 + j] (n1 < N1) in registers, does
//         a length-N1 DFT, multiplies by W_N^{j k1} and parks the values in
//         shared memory;
// step 2: thread k1 of a line gathers the N2 values for its k1 and does a
//         length-N2 DFT, ending with X[k1 + N1 k2] (k2 < N2) in registers.
// The small DFTs are unrolled Cooley-Tukey compositions of radix-2/3/4
// butterflies whose twiddles are compile-time indices into a 96-entry table
// (every small length used divides 96).  Forward transforms use
// exp(-2 pi i nk/N); inverse ones exp(+2 pi i nk/N) without scaling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <set>
#include <utility>

namespace ftr {

// W_96^j = exp(-2 pi i j / 96), a constant table of each translation unit,
// copied once per device by the unit's init function from the table the
// device computed in float64 (launch_twiddle, n = 96).
static __constant__ float2 c_w96[96];

static inline cudaError_t upload_w96_table(const float2* w96_dev) {
    return cudaMemcpyToSymbol(c_w96, w96_dev, 96 * sizeof(float2), 0, cudaMemcpyDeviceToDevice);
}

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// i * a
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }

// Multiply by W_R^m (SIGN = -1 forward, +1 inverse) with m, R compile-time
// after unrolling.
template <int R, int SIGN>
__device__ __forceinline__ float2 tw_small(float2 v, int m) {
    const int j = ((m % R) * (96 / R)) % 96;
    if (j == 0) return v;
    if (j == 48) return make_float2(-v.x, -v.y);
    if (j == 24) return SIGN < 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);   // -i / +i
    if (j == 72) return SIGN < 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);   // +i / -i
    float2 w = c_w96[j];
    if (SIGN > 0) w.y = -w.y;
    return cmul(v, w);
}

template <int R, int SIGN>
struct Dft;

template <int SIGN>
struct Dft<1, SIGN> {
    __device__ __forceinline__ static void run(float2 (&)[1]) {}
};

template <int SIGN>
struct Dft<2, SIGN> {
    __device__ __forceinline__ static void run(float2 (&x)[2]) {
        float2 a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};

template <int SIGN>
struct Dft<3, SIGN> {
    __device__ __forceinline__ static void run(float2 (&x)[3]) {
        // W_3 = -1/2 + SIGN i sqrt(3)/2
        const float s3 = 0.866025403784438647f * (float)SIGN;
        float2 a = x[0], b = x[1], c = x[2];
        float2 t1 = cadd(b, c);
        float2 t2 = make_float2(a.x - 0.5f * t1.x, a.y - 0.5f * t1.y);
        float2 d = csub(b, c);
        float2 t3 = make_float2(-d.y * s3, d.x * s3);   // i * SIGN * sqrt(3)/2 * (b - c)
        x[0] = cadd(a, t1);
        x[1] = cadd(t2, t3);
        x[2] = csub(t2, t3);
    }
};

template <int SIGN>
struct Dft<4, SIGN> {
    __device__ __forceinline__ static void run(float2 (&x)[4]) {
        float2 a = x[0], b = x[1], c = x[2], d = x[3];
        float2 s0 = cadd(a, c), s1 = csub(a, c);
        float2 s2 = cadd(b, d), s3 = csub(b, d);
        float2 r = cmuli(s3);                 // i (b - d)
        if (SIGN < 0) r = make_float2(-r.x, -r.y);
        x[0] = cadd(s0, s2);
        x[2] = csub(s0, s2);
        x[1] = cadd(s1, r);                   // (a - c) + SIGN i (b - d)
        x[3] = csub(s1, r);
    }
};

template <int R>
struct FirstFactor {
    static constexpr int value = (R % 4 == 0) ? 4 : ((R % 2 == 0) ? 2 : 3);
};

// Composite length: R = P Q, n = Q n1 + n2, k = k1 + P k2.
template <int R, int SIGN>
struct Dft {
    static constexpr int P = FirstFactor<R>::value;
    static constexpr int Q = R / P;
    __device__ __forceinline__ static void run(float2 (&x)[R]) {
        float2 y[R];
#pragma unroll
        for (int n2 = 0; n2 < Q; ++n2) {
            float2 t[P];
#pragma unroll
            for (int n1 = 0; n1 < P; ++n1) t[n1] = x[Q * n1 + n2];
            Dft<P, SIGN>::run(t);
#pragma unroll
            for (int k1 = 0; k1 < P; ++k1) y[n2 * P + k1] = tw_small<R, SIGN>(t[k1], n2 * k1);
        }
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) {
            float2 u[Q];
#pragma unroll
            for (int n2 = 0; n2 < Q; ++n2) u[n2] = y[n2 * P + k1];
            Dft<Q, SIGN>::run(u);
#pragma unroll
            for (int k2 = 0; k2 < Q; ++k2) x[k1 + P * k2] = u[k2];
        }
    }
};

// Split of each supported line length into N1 (step-1 DFT) x N2 (step-2 DFT).
template <int N> struct Plan;
template <> struct Plan<32>  { static constexpr int N1 = 4,  N2 = 8; };
template <> struct Plan<48>  { static constexpr int N1 = 6,  N2 = 8; };
template <> struct Plan<64>  { static constexpr int N1 = 8,  N2 = 8; };
template <> struct Plan<96>  { static constexpr int N1 = 12, N2 = 8; };
template <> struct Plan<128> { static constexpr int N1 = 16, N2 = 8; };
template <> struct Plan<192> { static constexpr int N1 = 12, N2 = 16; };
template <> struct Plan<256> { static constexpr int N1 = 16, N2 = 16; };
template <> struct Plan<384> { static constexpr int N1 = 24, N2 = 16; };
template <> struct Plan<512> { static constexpr int N1 = 32, N2 = 16; };

__host__ __device__ constexpr int cmax(int a, int b) { return a > b ? a : b; }

// Minimum resident CTAs per SM requested from the register allocator for the
// 16-line passes: three (24 warps) while the transform still fits in 80
// registers without spilling (n <= 256), one above.
template <int N>
struct MinCtas {
    static constexpr int value = N <= 256 ? 3 : 1;
};
// The same register budget per thread for other tile heights F (lines per
// CTA): F = 8 asks for twice the CTAs of F = 16, F = 32 half (at least one).
template <int N, int F>
struct MinCtasF {
    static constexpr int raw = MinCtas<N>::value * 16 / F;
    static constexpr int value = raw < 1 ? 1 : raw;
};

// Raise a kernel's dynamic shared-memory limit to `bytes`, once per device.
template <class K>
inline cudaError_t ensure_smem(K kernel, size_t bytes, int device) {
    static std::mutex mu;
    static std::set<std::pair<const void*, int>> done;
    std::lock_guard<std::mutex> lk(mu);
    const auto key = std::make_pair((const void*)kernel, device);
    if (done.count(key)) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done.insert(key);
    return e;
}

__host__ __device__ constexpr int make_odd(int v) { return (v & 1) ? v : v + 1; }

// Shared-memory exchange layout for F lines of length N: element (f, j, k1)
// at f + P1 k1 + P2 j.  P1 and P2 are odd so that 16 consecutive lanes that
// vary any one of f, j or k1 touch 16 different 8-byte bank pairs.
template <int N, int F>
struct Xchg {
    static constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    static constexpr int NT = cmax(N1, N2);               // threads per line
    static constexpr int P1 = make_odd(F + 1);
    static constexpr int P2 = make_odd(P1 * N1);          // forward layout (j < N2, k1 < N1)
    static constexpr int P2R = make_odd(P1 * N2);         // swapped layout (j < N1, k1 < N2)
    static constexpr int SIZE = cmax(P2 * N2, P2R * N1);  // float2 elements
    __device__ __forceinline__ static int idx(int f, int j, int k1) { return f + P1 * k1 + P2 * j; }
    __device__ __forceinline__ static int idxr(int f, int j, int k1) { return f + P1 * k1 + P2R * j; }
};

// Step 1 of a length-N transform: regs hold x[N2 n1 + j]; afterwards the
// twiddled step-1 results sit in the exchange buffer.  tw = the axis table
// (W_N^m, then W_N^(j k1) as [k1 < N1][j < N2], then as [k1 < N2][j < N1]).
template <int N, int F, int SIGN>
__device__ __forceinline__ void fft_step1(float2 (&v)[Plan<N>::N1], int f, int j, float2* xs,
                                          const float2* __restrict__ tw) {
    using X = Xchg<N, F>;
    Dft<X::N1, SIGN>::run(v);
#pragma unroll
    for (int k1 = 0; k1 < X::N1; ++k1) {
        float2 w = (k1 == 0 || j == 0) ? make_float2(1.f, 0.f) : __ldg(&tw[N + k1 * X::N2 + j]);
        if (SIGN > 0) w.y = -w.y;
        xs[X::idx(f, j, k1)] = (k1 == 0) ? v[k1] : cmul(v[k1], w);
    }
}

// Step 2: thread i (< N1) of line f gathers its column and ends with
// X[i + N1 k2] in out[k2].
template <int N, int F, int SIGN>
__device__ __forceinline__ void fft_step2(float2 (&out)[Plan<N>::N2], int f, int i, const float2* xs) {
    using X = Xchg<N, F>;
#pragma unroll
    for (int j = 0; j < X::N2; ++j) out[j] = xs[X::idx(f, j, i)];
    Dft<X::N2, SIGN>::run(out);
}

// Swapped-role steps (N = N2 * N1) used to run a second transform straight
// from the registers that step 2 left: thread i holds x[i + N1 n1'] (n1' < N2).
template <int N, int F, int SIGN>
__device__ __forceinline__ void fft_step1_swapped(float2 (&v)[Plan<N>::N2], int f, int j, float2* xs,
                                                  const float2* __restrict__ tw) {
    using X = Xchg<N, F>;
    Dft<X::N2, SIGN>::run(v);
#pragma unroll
    for (int k1 = 0; k1 < X::N2; ++k1) {
        float2 w = (k1 == 0 || j == 0) ? make_float2(1.f, 0.f) : __ldg(&tw[2 * N + k1 * X::N1 + j]);
        if (SIGN > 0) w.y = -w.y;
        xs[X::idxr(f, j, k1)] = (k1 == 0) ? v[k1] : cmul(v[k1], w);
    }
}

template <int N, int F, int SIGN>
__device__ __forceinline__ void fft_step2_swapped(float2 (&out)[Plan<N>::N1], int f, int i, const float2* xs) {
    using X = Xchg<N, F>;
#pragma unroll
    for (int j = 0; j < X::N1; ++j) out[j] = xs[X::idxr(f, j, i)];
    Dft<X::N1, SIGN>::run(out);
}

// z-planes [zl, zh) that can hold non-zero data after the splat: the slab of
// touched bricks (meta[2] .. meta[3]) widened to multiples of 16 planes, the
// tile height of the y and z passes.  Empty when no brick was touched.
__device__ __forceinline__ void live_z_range(const int* __restrict__ meta, int& zl, int& zh) {
    const int bmin = meta[2], bmax = meta[3];
    if (bmax < 0) {
        zl = zh = 0;
        return;
    }
    zl = (bmin * 8) & ~15;
    zh = ((bmax + 1) * 8 + 15) & ~15;
}

// Ask L2 to fetch the 128-byte line holding p (no register is written, so
// later loads of the line find it in L2 instead of DRAM).
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// L2 eviction priorities for the passes' intermediates: a pass reads its
// input once (evict first: the lines are dead after) and writes the next
// pass's input (evict last: kept in L2 in preference, so that more of it is
// still there when the next pass reads it).
__device__ __forceinline__ uint64_t l2_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t l2_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ float2 ld_l2hint(const float2* a, uint64_t pol) {
    float2 v;
    asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_l2hint(float2* a, float2 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;" ::"l"(a), "f"(v.x), "f"(v.y), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void st_l2hint(float* a, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}

// Signed frequency index of bin k on an axis of length n (Nyquist -> -n/2).
__device__ __forceinline__ int signed_bin(int k, int n) { return k < n / 2 ? k : k - n; }

}  // namespace ftr
