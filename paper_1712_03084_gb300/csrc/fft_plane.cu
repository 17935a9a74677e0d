// Launchers of the plane-fused transform path (fft_fused.cuh): forward x+y
// per z-plane, the z pass on the plane-major fields, inverse y+x per z-plane.
#include "fft_fused.cuh"

namespace ftr {

namespace {

cudaError_t plane(ftr_ctx* c, int which, int* n) {
    cudaError_t e = cudaErrorInvalidValue;
    if (fused::dispatch_a(c, which, n, &e)) return e;
    if (fused::dispatch_b(c, which, n, &e)) return e;
    return cudaErrorInvalidValue;
}

template <int N, int F>
cudaError_t run_fz2_f(ftr_ctx* c) {
    using X = Xchg<N, F>;
    const size_t smem = sizeof(float2) * (X::SIZE + (F + 1) * N);
    cudaError_t e = ensure_smem(fused::k_fz2<N, F>, smem, c->device);
    if (e != cudaSuccess) return e;
    if (c->occ_query)   // the autotuner asks how many CTAs of this plan fit on an SM
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(c->occ_query, fused::k_fz2<N, F>, F * X::NT, smem);
    dim3 grid(c->g.n[1] / F, c->g.n[0] / 2 + 1);
    const double two_pi = 2.0 * 3.14159265358979323846;
    const float wx = (float)(two_pi / (c->g.n[0] * c->g.h[0]));
    const float wy = (float)(two_pi / (c->g.n[1] * c->g.h[1]));
    const float wz = (float)(two_pi / (c->g.n[2] * c->g.h[2]));
    const float inv_m = (float)(1.0 / (double)c->M);
    launch_pdl(fused::k_fz2<N, F>, grid, F * X::NT, smem, c->stream, c->g, c->d_s1, c->Mh, (const float2*)c->d_tw[2], wx,
               wy, wz, inv_m, (const int*)c->d_meta);
    c->launches++;
    return cudaGetLastError();
}

template <int N>
cudaError_t run_fz2(ftr_ctx* c) {
    switch (c->plan_lines[1]) {
        case 8: return run_fz2_f<N, 8>(c);
        case 32: return run_fz2_f<N, 32>(c);
        default: return run_fz2_f<N, 16>(c);
    }
}

}  // namespace

cudaError_t fft_plane_init(const float2* w96) { return upload_w96_table(w96); }

bool fused_available(ftr_ctx* c) {
    int nf = 0, ni = 0;
    if (plane(c, 2, &nf) != cudaSuccess || plane(c, 3, &ni) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return nf > 0 && ni > 0;
}

cudaError_t launch_fxy(ftr_ctx* c) { return plane(c, 0, nullptr); }

cudaError_t launch_iyx(ftr_ctx* c) { return plane(c, 1, nullptr); }

cudaError_t launch_fz2(ftr_ctx* c) {
    switch (c->g.n[2]) {
        case 32: return run_fz2<32>(c);
        case 48: return run_fz2<48>(c);
        case 64: return run_fz2<64>(c);
        case 96: return run_fz2<96>(c);
        case 128: return run_fz2<128>(c);
        case 192: return run_fz2<192>(c);
        case 256: return run_fz2<256>(c);
        case 384: return run_fz2<384>(c);
        case 512: return run_fz2<512>(c);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ftr
