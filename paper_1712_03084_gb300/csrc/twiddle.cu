// Twiddle tables generated on the device in float64.
//
// W_n^m = exp(-2 pi i m / n) for the axis passes (stored float32) and the
// 96-entry table of the small register DFTs are evaluated with the float64
// sincospi of the CUDA math library (exact at the quarter points), then
// rounded once to float32.
//
// An axis table holds 3 n entries: W_n^m (m < n), then the same values in
// the order the two twiddle steps of the four-step transform read them
// (n = N1 N2): [N1][N2] with entry (k1, j) = W_n^(j k1 mod n), then
// [N2][N1] likewise (the swapped step).  A warp of step 1 reads, for one
// k1, consecutive j: one contiguous run of the table instead of N2 values
// spread over it.
#include <cuda_runtime.h>

#include "fft_common.cuh"
#include "ftr_internal.h"

namespace ftr {
namespace {

__global__ void k_twiddle(float2* __restrict__ tw, int n) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n) return;
    double s, c;
    sincospi(2.0 * (double)m / (double)n, &s, &c);
    tw[m] = make_float2((float)c, (float)(-s));
}

// The two step-ordered copies of W_n^m, gathered from the first n entries.
template <int N>
__global__ void k_twiddle_steps(float2* __restrict__ tw) {
    constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * N) return;
    const bool swapped = e >= N;
    const int i = swapped ? e - N : e;
    const int cols = swapped ? N1 : N2;
    const int k1 = i / cols, j = i % cols;
    tw[N + e] = tw[(j * k1) % N];
}

template <int N>
cudaError_t steps(float2* tw, cudaStream_t st) {
    k_twiddle_steps<N><<<(2 * N + 127) / 128, 128, 0, st>>>(tw);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_twiddle(float2* tw, int n, cudaStream_t st) {
    k_twiddle<<<(n + 127) / 128, 128, 0, st>>>(tw, n);
    return cudaGetLastError();
}

cudaError_t launch_axis_twiddles(float2* tw, int n, cudaStream_t st) {
    cudaError_t e = launch_twiddle(tw, n, st);
    if (e != cudaSuccess) return e;
    switch (n) {
        case 32: return steps<32>(tw, st);
        case 48: return steps<48>(tw, st);
        case 64: return steps<64>(tw, st);
        case 96: return steps<96>(tw, st);
        case 128: return steps<128>(tw, st);
        case 192: return steps<192>(tw, st);
        case 256: return steps<256>(tw, st);
        case 384: return steps<384>(tw, st);
        case 512: return steps<512>(tw, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ftr
