// Twiddle tables generated on the device in float64.
//
// W_n^m = exp(-2 pi i m / n) for the axis passes (stored float32) and the
// 96-entry table of the small register DFTs are evaluated with the float64
// sincospi of the CUDA math library (exact at the quarter points), then
// rounded once to float32.
#include <cuda_runtime.h>

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

}  // namespace

cudaError_t launch_twiddle(float2* tw, int n, cudaStream_t st) {
    k_twiddle<<<(n + 127) / 128, 128, 0, st>>>(tw, n);
    return cudaGetLastError();
}

}  // namespace ftr
