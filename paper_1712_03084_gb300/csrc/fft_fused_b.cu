// Plane transforms of the smaller and the elongated grids (see fft_fused.cuh).
#include "fft_fused.cuh"

namespace ftr {

// the small-DFT twiddle constants of this translation unit
cudaError_t fft_fused_b_init(const float2* w96) { return upload_w96_table(w96); }

namespace fused {

bool dispatch_b(ftr_ctx* c, int which, int* n, cudaError_t* e) {
    const int nx = c->g.n[0], ny = c->g.n[1];
#define FTR_PLANE(X, Y)                        \
    if (nx == X && ny == Y) {                  \
        *e = run_pair<X, Y>(c, which, n);      \
        return true;                           \
    }
    FTR_PLANE(32, 32)
    FTR_PLANE(48, 48)
    FTR_PLANE(64, 64)
    FTR_PLANE(96, 96)
    FTR_PLANE(48, 96)
    FTR_PLANE(32, 64)
    FTR_PLANE(64, 128)
    FTR_PLANE(384, 48)
    FTR_PLANE(192, 48)
    FTR_PLANE(32, 384)
    FTR_PLANE(32, 192)
    FTR_PLANE(48, 32)
#undef FTR_PLANE
    return false;
}

}  // namespace fused
}  // namespace ftr
