// Plane transforms of the larger grids (see fft_fused.cuh).
#include "fft_fused.cuh"

namespace ftr {

// the small-DFT twiddle constants of this translation unit
cudaError_t fft_fused_a_init(const float2* w96) { return upload_w96_table(w96); }

namespace fused {

bool dispatch_a(ftr_ctx* c, int which, int* n, cudaError_t* e) {
    const int nx = c->g.n[0], ny = c->g.n[1];
#define FTR_PLANE(X, Y)                        \
    if (nx == X && ny == Y) {                  \
        *e = run_pair<X, Y>(c, which, n);      \
        return true;                           \
    }
    FTR_PLANE(256, 256)
    FTR_PLANE(384, 384)
    FTR_PLANE(192, 192)
    FTR_PLANE(128, 256)
    FTR_PLANE(128, 128)
#undef FTR_PLANE
    return false;
}

}  // namespace fused
}  // namespace ftr
