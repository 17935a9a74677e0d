// C ABI of the reconstruction library: context lifetime, staging of host
// inputs, the per-frame call sequence and the inspection hooks.  See
// include/ftr.h for the contract of every entry point.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <array>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "ftr_internal.h"

using namespace ftr;

namespace ftr {

int set_err(ftr_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int cuda_fail(ftr_ctx* c, cudaError_t e, const char* what) {
    return set_err(c, e == cudaErrorMemoryAllocation ? FTR_ENOMEM : FTR_ECUDA, "%s: %s (%s)", what,
                   cudaGetErrorString(e), cudaGetErrorName(e));
}

// After a stream synchronisation: FTR_ETIMEOUT if a tensor-core completion
// wait of the split-precision passes gave up since the last check.
int tc_check(ftr_ctx* c, const char* who) {
    // the flags reached c->h_flags with the frame's last copy (see launch_flags)
    if (!c->h_flags || (!c->h_flags[0] && !c->h_flags[1])) return FTR_OK;
    c->h_flags[0] = c->h_flags[1] = 0;
    if (c->d_tc_err) cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream);
    if (c->d_kerr) cudaMemsetAsync(c->d_kerr, 0, sizeof(int), c->stream);
    return set_err(c, FTR_ETIMEOUT, "%s: a device completion wait timed out", who);
}

// Enqueue the copy of the device wait flags into pinned host memory.
cudaError_t launch_flags(ftr_ctx* c) {
    cudaError_t e = cudaSuccess;
    if (c->d_tc_err) e = cudaMemcpyAsync(&c->h_flags[0], c->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && c->d_kerr)
        e = cudaMemcpyAsync(&c->h_flags[1], c->d_kerr, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    return e;
}

void prof_begin(ftr_ctx* c, int st) {
    if (!c->prof) return;
    if (c->ev_pending[st]) {
        float ms = 0.f;
        cudaEventSynchronize(c->ev_stop[st]);
        if (cudaEventElapsedTime(&ms, c->ev_start[st], c->ev_stop[st]) == cudaSuccess) {
            c->prof_ms[st] += ms;
            c->prof_n[st] += 1;
        }
        c->ev_pending[st] = false;
    }
    cudaEventRecord(c->ev_start[st], c->stream);
}

void prof_end(ftr_ctx* c, int st) {
    if (!c->prof) return;
    cudaEventRecord(c->ev_stop[st], c->stream);
    c->ev_pending[st] = true;
}

}  // namespace ftr

namespace {

const char* kStageNames[ST_COUNT] = {"ingest", "splat_bin", "splat_accum", "fft_x_fwd", "fft_y_fwd",
                                     "fft_z_filter_inv", "fft_y_inv", "fft_x_inv", "level", "mc_count",
                                     "mc_scan", "mc_emit", "mc_tris", "texture", "fft_xy_fwd",
                                     "fft_yx_inv", "fft_yz_fwd_filter_inv"};

bool supported_n(int n) {
    switch (n) {
        case 32: case 48: case 64: case 96: case 128: case 192: case 256: case 384: case 512: return true;
        default: return false;
    }
}

// one-time per-device constant setup (twiddle constants of every FFT unit, MC table)
std::mutex g_init_mu;
bool g_dev_ready[64] = {};

cudaError_t ensure_device_ready(int dev) {
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (dev >= 0 && dev < 64 && g_dev_ready[dev]) return cudaSuccess;
    cudaError_t e;
    // the small-DFT twiddles W_96^j, computed on the device in float64, then
    // copied into every transform unit's constant table
    float2* w96 = nullptr;
    if ((e = cudaMalloc(&w96, 96 * sizeof(float2))) != cudaSuccess) return e;
    if ((e = launch_twiddle(w96, 96, 0)) != cudaSuccess || (e = cudaStreamSynchronize(0)) != cudaSuccess ||
        (e = fft_fx_init(w96)) != cudaSuccess || (e = fft_fy_init(w96)) != cudaSuccess ||
        (e = fft_fz_init(w96)) != cudaSuccess || (e = fft_iy_init(w96)) != cudaSuccess ||
        (e = fft_ix_init(w96)) != cudaSuccess || (e = fft_fused_a_init(w96)) != cudaSuccess ||
        (e = fft_fused_b_init(w96)) != cudaSuccess || (e = fft_plane_init(w96)) != cudaSuccess ||
        (e = fft_yz_init(w96)) != cudaSuccess) {
        cudaFree(w96);
        return e;
    }
    cudaFree(w96);
    if ((e = mc_init()) != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) g_dev_ready[dev] = true;
    return cudaSuccess;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, count * sizeof(T));
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

cudaError_t ensure_stage(ftr_ctx* c, void** buf, size_t* cap, size_t bytes) {
    if (*cap >= bytes) return cudaSuccess;
    if (*buf) cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    size_t want = bytes + bytes / 4 + 256;
    cudaError_t e = cudaMalloc(buf, want);
    if (e == cudaSuccess) *cap = want;
    return e;
}

cudaError_t grow_points(ftr_ctx* c, int64_t need) {
    if (need <= c->pts.cap) return cudaSuccess;
    c->graph_valid = false;
    int64_t cap = c->pts.cap ? c->pts.cap : 1 << 16;
    while (cap < need) cap *= 2;
    int4* b;
    float4 *f, *n;
    cudaError_t e;
    if ((e = dalloc(&b, cap)) != cudaSuccess) return e;
    if ((e = dalloc(&f, cap)) != cudaSuccess) { cudaFree(b); return e; }
    if ((e = dalloc(&n, cap)) != cudaSuccess) { cudaFree(b); cudaFree(f); return e; }
    if (c->n_pts > 0) {
        cudaMemcpyAsync(b, c->pts.base, sizeof(int4) * c->n_pts, cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(f, c->pts.frac, sizeof(float4) * c->n_pts, cudaMemcpyDeviceToDevice, c->stream);
        cudaMemcpyAsync(n, c->pts.nrm, sizeof(float4) * c->n_pts, cudaMemcpyDeviceToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
    }
    dfree(c->pts.base);
    dfree(c->pts.frac);
    dfree(c->pts.nrm);
    c->pts.base = b;
    c->pts.frac = f;
    c->pts.nrm = n;
    c->pts.cap = cap;
    return cudaSuccess;
}

int64_t heavy_capacity(int64_t points) {
    int64_t cap = 64;
    while (cap < 8 * points / kSplatChunk + 1) cap *= 2;
    return cap;
}

cudaError_t grow_entries(ftr_ctx* c, int64_t need) {
    if (need <= c->cap_entries) return cudaSuccess;
    c->graph_valid = false;
    int64_t cap = c->cap_entries ? c->cap_entries : 1 << 18;
    while (cap < need) cap *= 2;
    cudaStreamSynchronize(c->stream);
    dfree(c->d_entries);
    cudaError_t e = dalloc(&c->d_entries, cap);
    if (e != cudaSuccess) return e;
    c->cap_entries = cap;
    // chunks: one per touched brick plus at most cap / chunk more
    const int64_t units = (int64_t)c->n_bricks + cap / kSplatChunk + 2;
    if (units > c->cap_units) {
        dfree(c->d_unit_slot);
        if ((e = dalloc(&c->d_unit_slot, (size_t)units)) != cudaSuccess) return e;
        c->cap_units = units;
    }
    return e;
}

// Accumulators of the heavy bricks (more than one chunk of pairs): at most
// pairs / chunk of them, with at most 8 pairs per point (every point's stencil
// overlaps at most 8 bricks); the capacity grows in powers of two.
cudaError_t grow_heavy(ftr_ctx* c, int64_t points) {
    const int64_t heavy = heavy_capacity(points);
    cudaError_t e = cudaSuccess;
    if (heavy > c->cap_heavy) {
        c->graph_valid = false;
        cudaStreamSynchronize(c->stream);
        dfree(c->d_heavy_acc);
        dfree(c->d_heavy_done);
        if ((e = dalloc(&c->d_heavy_acc, (size_t)heavy * 4 * kBrickVox)) != cudaSuccess) return e;
        if ((e = dalloc(&c->d_heavy_done, (size_t)heavy)) != cudaSuccess) return e;
        if ((e = cudaMemset(c->d_heavy_acc, 0, sizeof(unsigned long long) * heavy * 4 * kBrickVox)) != cudaSuccess)
            return e;
        if ((e = cudaMemset(c->d_heavy_done, 0, sizeof(int) * heavy)) != cudaSuccess) return e;
        c->cap_heavy = heavy;
    }
    return e;
}

void free_all(ftr_ctx* c) {
    dfree(c->pts.base);
    dfree(c->pts.frac);
    dfree(c->pts.nrm);
    dfree(c->d_dropped);
    dfree(c->d_npts);
    dfree(c->d_wild);
    if (c->d_stage) cudaFree(c->d_stage);
    dfree(c->d_brick_cnt);
    dfree(c->d_brick_off);
    dfree(c->d_brick_cursor);
    dfree(c->d_brick_slot);
    dfree(c->d_active);
    dfree(c->d_meta);
    dfree(c->d_tile);
    dfree(c->d_unit_off);
    dfree(c->d_unit_slot);
    dfree(c->d_heavy_idx);
    dfree(c->d_heavy_acc);
    dfree(c->d_heavy_done);
    dfree(c->d_entries);
    dfree(c->d_vpool);
    dfree(c->d_s0);
    dfree(c->d_s1);
    dfree(c->d_A);
    for (int a = 0; a < 3; ++a) dfree(c->d_tw[a]);
    dfree(c->d_tc_table);
    eval_free(c);
    dfree(c->d_raw);
    dfree(c->d_raw_tiles);
    dfree(c->d_raw_total);
    if (c->h_raw_total) cudaFreeHost(c->h_raw_total);
    dfree(c->d_tc_err);
    dfree(c->d_kerr);
    dfree(c->d_ring);
    dfree(c->d_yz_sync);
    dfree(c->d_level);
    dfree(c->d_levelf);
    dfree(c->d_level_part);
    dfree(c->d_ticket);
    dfree(c->d_mc_blk);
    dfree(c->d_mc_bits);
    dfree(c->d_rowmm);
    dfree(c->d_mc_word);
    dfree(c->d_mc_off);
    if (c->h_mc_tot) cudaFreeHost(c->h_mc_tot);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    dfree(c->d_mc_nodes);
    dfree(c->d_verts);
    dfree(c->d_vnrm);
    dfree(c->d_tris);
    if (c->d_tex_stage) cudaFree(c->d_tex_stage);
    for (int s = 0; s < ST_COUNT; ++s) {
        if (c->ev_start[s]) cudaEventDestroy(c->ev_start[s]);
        if (c->ev_stop[s]) cudaEventDestroy(c->ev_stop[s]);
    }
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
}

}  // namespace

extern "C" {

void ftr_default_params(ftr_params* p) {
    if (!p) return;
    p->sigma1_scale = 1.0f;
    p->sigma2_ratio2 = 1.5f;
    p->splat_mode = FTR_SPLAT_WEIGHTED;
    p->precision = FTR_PREC_FP32;
    p->stream = nullptr;
}

int ftr_create(const int grid_n[3], const float bbox[6], const ftr_params* p, ftr_ctx** out) {
    if (!out) return FTR_EINVAL;
    *out = nullptr;
    if (!grid_n || !bbox) return FTR_EINVAL;
    for (int a = 0; a < 3; ++a) {
        if (!supported_n(grid_n[a])) return FTR_EINVAL;
        if (!(bbox[3 + a] > bbox[a]) || !isfinite(bbox[a]) || !isfinite(bbox[3 + a])) return FTR_EINVAL;
    }
    ftr_params prm;
    ftr_default_params(&prm);
    if (p) prm = *p;
    if (!(prm.sigma1_scale > 0.f) || !(prm.sigma2_ratio2 > 1.0f)) return FTR_EINVAL;
    if (prm.splat_mode != FTR_SPLAT_WEIGHTED && prm.splat_mode != FTR_SPLAT_SIMPLE) return FTR_EINVAL;
    if (prm.precision != FTR_PREC_FP32 && prm.precision != FTR_PREC_BF16X3 && prm.precision != FTR_PREC_FP16X3)
        return FTR_EINVAL;
    if (prm.precision != FTR_PREC_FP32) {
        for (int a = 0; a < 3; ++a)
            if (!tc_supported_n(grid_n[a])) return FTR_EINVAL;
    }

    ftr_ctx* c = new (std::nothrow) ftr_ctx();
    if (!c) return FTR_ENOMEM;
    c->p = prm;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) { delete c; return FTR_ECUDA; }
    if ((e = ensure_device_ready(c->device)) != cudaSuccess) { delete c; return FTR_ECUDA; }

    GridDev& g = c->g;
    double diag2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        g.n[a] = grid_n[a];
        g.nb[a] = grid_n[a] / kBrick;
        g.bmin[a] = (double)bbox[a];
        g.h[a] = ((double)bbox[3 + a] - (double)bbox[a]) / grid_n[a];
        g.inv_h[a] = 1.0 / g.h[a];
        g.hf[a] = (float)g.h[a];
        g.inv_hf[a] = (float)g.inv_h[a];
        g.inv_h_lo[a] = (float)(g.inv_h[a] - (double)g.inv_hf[a]);
        g.bminf[a] = bbox[a];
        diag2 += g.h[a] * g.h[a];
    }
    const double s1 = (double)prm.sigma1_scale * 0.5 * sqrt(diag2);
    const double s2 = sqrt((double)prm.sigma2_ratio2) * s1;
    g.inv_s1sq = (float)(1.0 / (s1 * s1));
    g.inv_s2sq = (float)(1.0 / (s2 * s2));
    g.mode = prm.splat_mode;
    g.v_scale = prm.splat_mode == FTR_SPLAT_WEIGHTED ? s2 / s1 : 1.0;
    g.v_scale_f = (float)g.v_scale;
    c->M = (int64_t)grid_n[0] * grid_n[1] * grid_n[2];
    c->Mh = (int64_t)(grid_n[0] / 2 + 1) * grid_n[1] * grid_n[2];
    c->n_bricks = g.nb[0] * g.nb[1] * g.nb[2];

    if (prm.stream) {
        c->stream = (cudaStream_t)prm.stream;
    } else {
        if ((e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking)) != cudaSuccess) {
            delete c;
            return FTR_ECUDA;
        }
        c->own_stream = true;
    }
#define ALLOC(ptr, n)                                       \
    if ((e = dalloc(&(ptr), (size_t)(n))) != cudaSuccess) { \
        free_all(c);                                        \
        delete c;                                           \
        return FTR_ENOMEM;                                  \
    }
    ALLOC(c->d_dropped, 1);
    ALLOC(c->d_npts, 1);
    ALLOC(c->d_wild, 1);
    ALLOC(c->d_brick_cnt, c->n_bricks);
    ALLOC(c->d_brick_off, c->n_bricks + 1);
    ALLOC(c->d_brick_cursor, c->n_bricks);
    ALLOC(c->d_brick_slot, c->n_bricks);
    ALLOC(c->d_active, c->n_bricks);
    ALLOC(c->d_meta, 8);
    ALLOC(c->d_kerr, 1);
    ALLOC(c->d_tile, (c->n_bricks + kBrickScanTile - 1) / kBrickScanTile + 1);
    ALLOC(c->d_unit_off, c->n_bricks + 1);
    ALLOC(c->d_heavy_idx, c->n_bricks);
    ALLOC(c->d_vpool, (size_t)c->n_bricks * 3 * kBrickVox);
    ALLOC(c->d_s0, 3 * c->Mh);
    ALLOC(c->d_s1, 2 * c->Mh);
    ALLOC(c->d_A, c->M);
    for (int a = 0; a < 3; ++a) ALLOC(c->d_tw[a], 3 * grid_n[a]);
    c->level_blocks = 304;
    ALLOC(c->d_level, 2);
    ALLOC(c->d_levelf, 2);
    ALLOC(c->d_level_part, 2 * c->level_blocks);
    ALLOC(c->d_ticket, 1);
    c->mc_blocks = grid_n[1] * grid_n[2];      // marching cubes counts per grid row
    ALLOC(c->d_mc_blk, 3 * c->mc_blocks);
    {
        int wp = 1;
        while (wp < (grid_n[0] + 31) / 32) wp <<= 1;
        ALLOC(c->d_mc_bits, (size_t)c->mc_blocks * wp);
        ALLOC(c->d_mc_word, (size_t)c->mc_blocks * wp);
    }
    ALLOC(c->d_mc_off, 3 * (c->mc_blocks + 1) + 3);
    ALLOC(c->d_rowmm, c->mc_blocks);
#undef ALLOC
    if ((e = cudaMallocHost((void**)&c->h_mc_tot, 4 * sizeof(int))) != cudaSuccess ||
        (e = cudaMallocHost((void**)&c->h_flags, 2 * sizeof(int))) != cudaSuccess) {
        free_all(c);
        delete c;
        return FTR_ENOMEM;
    }
    // W_n^m of each axis, computed on the device in float64
    for (int a = 0; a < 3; ++a) {
        if ((e = launch_axis_twiddles(c->d_tw[a], grid_n[a], c->stream)) != cudaSuccess) {
            free_all(c);
            delete c;
            return FTR_ECUDA;
        }
    }
    if (prm.precision != FTR_PREC_FP32) {
        if ((e = dalloc(&c->d_tc_table, tc_table_bytes())) != cudaSuccess || (e = dalloc(&c->d_tc_err, 1)) != cudaSuccess) {
            free_all(c);
            delete c;
            return FTR_ENOMEM;
        }
        // the split DFT matrices, built on the device from float64 cos / sin
        if ((e = tc_build_table(prm.precision, c->d_tc_table, c->stream)) != cudaSuccess ||
            (e = cudaMemset(c->d_tc_err, 0, sizeof(int))) != cudaSuccess || (e = tc_prepare(c)) != cudaSuccess) {
            free_all(c);
            delete c;
            return FTR_ECUDA;
        }
    }
    // the persistent y+z pass where it is built for this grid; its ring is
    // allocated only while that path is in use (or being timed)
    c->yz_ok = prm.precision == FTR_PREC_FP32 && yz_supported(c->g.n);
    // the plane-fused transforms where they are built for this grid and fit
    c->fused_ok = prm.precision == FTR_PREC_FP32 && fused_available(c);
    c->fused = 0;         // five axis passes until ftr_autotune times both paths
    for (int s = 0; s < ST_COUNT; ++s) {
        cudaEventCreate(&c->ev_start[s]);
        cudaEventCreate(&c->ev_stop[s]);
    }
    cudaMemsetAsync(c->d_dropped, 0, sizeof(unsigned long long), c->stream);
    // every brick empty (slot -1) until the first splat: the x passes read
    // this table, also when ftr_autotune times the transforms before any frame
    cudaMemsetAsync(c->d_brick_slot, 0xff, sizeof(int) * c->n_bricks, c->stream);
    {
        // no brick touched yet: an empty live z-slab (max brick z = -1)
        const int meta0[8] = {0, 0, 0, -1, 0, 0, 0, 0};
        cudaMemcpyAsync(c->d_meta, meta0, sizeof(meta0), cudaMemcpyHostToDevice, c->stream);
    }
    cudaMemsetAsync(c->d_wild, 0, sizeof(int), c->stream);
    cudaMemsetAsync(c->d_kerr, 0, sizeof(int), c->stream);
    c->h_flags[0] = c->h_flags[1] = 0;
    cudaMemsetAsync(c->d_ticket, 0, sizeof(unsigned), c->stream);
    cudaMemsetAsync(c->d_npts, 0, sizeof(int64_t), c->stream);
    cudaMemsetAsync(c->d_brick_cnt, 0, sizeof(int) * c->n_bricks, c->stream);
    {
        int wp = 1;
        while (wp < (c->g.n[0] + 31) / 32) wp <<= 1;
        cudaMemsetAsync(c->d_mc_word, 0, sizeof(int2) * (size_t)c->mc_blocks * wp, c->stream);
    }
    double zero2[2] = {0.0, 0.0};
    float zerof[2] = {0.f, 0.f};
    cudaMemcpyAsync(c->d_level, zero2, sizeof(zero2), cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(c->d_levelf, zerof, sizeof(zerof), cudaMemcpyHostToDevice, c->stream);
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
        free_all(c);
        delete c;
        return FTR_ECUDA;
    }
    *out = c;
    return FTR_OK;
}

void ftr_destroy(ftr_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_all(c);
    delete c;
}

int ftr_reset(ftr_ctx* c) {
    if (!c) return FTR_EINVAL;
    c->n_pts = 0;
    c->points_in = 0;
    c->depth_async = false;
    c->solved = false;
    c->v_external = false;
    c->meshed = false;
    c->n_verts = c->n_tris = 0;
    cudaError_t e = cudaMemsetAsync(c->d_dropped, 0, sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_wild, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_npts, 0, sizeof(int64_t), c->stream);
    // the ingest counts each point into the bricks its stencil overlaps
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_brick_cnt, 0, sizeof(int) * c->n_bricks, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_reset");
    return FTR_OK;
}

int ftr_splat(ftr_ctx* c, const float* points, const float* normals, const float* weights, int64_t n) {
    if (!c) return FTR_EINVAL;
    if (c->depth_async) return set_err(c, FTR_ESTATE, "ftr_splat: the frame's points come from ftr_splat_depth_async");
    if (n < 0) return set_err(c, FTR_EINVAL, "ftr_splat: n < 0");
    if (n == 0) return FTR_OK;
    if (!points || !normals) return set_err(c, FTR_EINVAL, "ftr_splat: points and normals are required");
    if (c->n_pts + n > (int64_t)0x3fffffff) return set_err(c, FTR_EINVAL, "ftr_splat: too many points per frame");
    cudaError_t e;
    if ((e = grow_points(c, c->n_pts + n)) != cudaSuccess) return cuda_fail(c, e, "ftr_splat: point store");
    const bool dp = is_device_ptr(points), dn = is_device_ptr(normals);
    const bool dw = weights ? is_device_ptr(weights) : true;
    const float* P = points;
    const float* N = normals;
    const float* W = weights;
    if (!dp || !dn || !dw) {
        const size_t need = sizeof(float) * (size_t)n * 7;
        if ((e = ensure_stage(c, &c->d_stage, &c->stage_cap, need)) != cudaSuccess)
            return cuda_fail(c, e, "ftr_splat: staging");
        float* st = (float*)c->d_stage;
        if (!dp) {
            if ((e = cudaMemcpyAsync(st, points, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, c->stream)))
                return cuda_fail(c, e, "ftr_splat: copy points");
            P = st;
        }
        if (!dn) {
            if ((e = cudaMemcpyAsync(st + 3 * n, normals, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, c->stream)))
                return cuda_fail(c, e, "ftr_splat: copy normals");
            N = st + 3 * n;
        }
        if (weights && !dw) {
            if ((e = cudaMemcpyAsync(st + 6 * n, weights, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream)))
                return cuda_fail(c, e, "ftr_splat: copy weights");
            W = st + 6 * n;
        }
    }
    prof_begin(c, ST_INGEST);
    e = launch_ingest(c, P, N, W, n);
    prof_end(c, ST_INGEST);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_splat: ingest");
    c->n_pts += n;
    c->points_in += n;
    // the staging buffer is reused by the next call: keep host-staged calls ordered
    if (!dp || !dn || !dw) {
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "ftr_splat");
    }
    return FTR_OK;
}

namespace {

// Validate the views and enqueue the raw reconstruction into the context's
// scratch; *pixels = the number of pixels (a bound on the points).
int raw_enqueue(ftr_ctx* c, const char* who, const ftr_view* views, int k, double step, double noise, int radius,
                float* const* conf_out, int64_t* pixels_out) {
    if (k < 1 || k > kMaxViews || !views) return set_err(c, FTR_EINVAL, "%s: 1 <= k <= 8 views", who);
    if (step < 0.0) step = 0.03;
    if (noise < 0.0) noise = 0.0012;
    if (radius < 0) radius = 10;
    if (radius > raw_max_radius() || !(step >= 0.0) || !(noise >= 0.0))
        return set_err(c, FTR_EINVAL, "%s: radius <= 16, finite step and noise", who);
    int64_t pixels = 0;
    for (int i = 0; i < k; ++i) {
        const ftr_view& v = views[i];
        if (v.w < 2 || v.h < 2 || v.w > 16384 || v.h > 16384 || !v.depth || !is_device_ptr(v.depth))
            return set_err(c, FTR_EINVAL, "%s: view %d needs a device depth map of at least 2 x 2", who, i);
        if (!(v.K[0] != 0.f) || !(v.K[4] != 0.f)) return set_err(c, FTR_EINVAL, "%s: view %d focal", who, i);
        if (conf_out && conf_out[i] && !is_device_ptr(conf_out[i]))
            return set_err(c, FTR_EINVAL, "%s: confidence maps must be device memory", who);
        pixels += (int64_t)v.w * v.h;
    }
    cudaError_t e;
    const int tiles = raw_tiles(views, k);
    if (pixels > c->raw_cap) {
        c->graph_valid = false;
        cudaStreamSynchronize(c->stream);
        dfree(c->d_raw);
        if ((e = dalloc(&c->d_raw, (size_t)pixels * 7)) != cudaSuccess) return cuda_fail(c, e, who);
        c->raw_cap = pixels;
    }
    if (tiles > c->raw_tiles_cap) {
        cudaStreamSynchronize(c->stream);
        dfree(c->d_raw_tiles);
        if ((e = dalloc(&c->d_raw_tiles, (size_t)tiles)) != cudaSuccess) return cuda_fail(c, e, who);
        c->raw_tiles_cap = tiles;
    }
    if (!c->d_raw_total) {
        if ((e = dalloc(&c->d_raw_total, 1)) != cudaSuccess) return cuda_fail(c, e, who);
        if ((e = cudaMallocHost((void**)&c->h_raw_total, sizeof(int))) != cudaSuccess) return cuda_fail(c, e, who);
    }
    RawParams rp;
    rp.step = step;
    rp.noise = noise;
    rp.step_f = (float)step;
    rp.noise_f = (float)noise;
    rp.radius = radius;
    float* P = c->d_raw;
    if ((e = launch_raw(c, rp, views, k, conf_out, P, P + 3 * pixels, P + 6 * pixels, c->d_raw_tiles,
                        c->d_raw_total)) != cudaSuccess)
        return cuda_fail(c, e, who);
    *pixels_out = pixels;
    return FTR_OK;
}

}  // namespace

int ftr_splat_sets(ftr_ctx* c, const ftr_point_set* sets, int k) {
    if (!c) return FTR_EINVAL;
    if (c->depth_async) return set_err(c, FTR_ESTATE, "ftr_splat_sets: the frame's points come from ftr_splat_depth_async");
    if (k < 1 || k > kMaxSets || !sets) return set_err(c, FTR_EINVAL, "ftr_splat_sets: 1 <= k <= %d sets", kMaxSets);
    IngestSets S{};
    S.k = k;
    S.base = c->n_pts;
    S.off[0] = 0;
    bool dev[kMaxSets][3];
    size_t host_floats = 0;
    for (int s = 0; s < k; ++s) {
        const ftr_point_set& p = sets[s];
        if (p.n < 0) return set_err(c, FTR_EINVAL, "ftr_splat_sets: set %d has n < 0", s);
        if (p.n > 0 && (!p.points || !p.normals))
            return set_err(c, FTR_EINVAL, "ftr_splat_sets: set %d needs points and normals", s);
        dev[s][0] = p.n == 0 || is_device_ptr(p.points);
        dev[s][1] = p.n == 0 || is_device_ptr(p.normals);
        dev[s][2] = p.n == 0 || !p.weights || is_device_ptr(p.weights);
        host_floats += (size_t)p.n * ((dev[s][0] ? 0 : 3) + (dev[s][1] ? 0 : 3) + (dev[s][2] ? 0 : 1));
        S.pts[s] = p.points;
        S.nrm[s] = p.normals;
        S.w[s] = p.weights;
        S.off[s + 1] = S.off[s] + p.n;
    }
    const int64_t n = S.off[k];
    if (n == 0) return FTR_OK;
    if (c->n_pts + n > (int64_t)0x3fffffff) return set_err(c, FTR_EINVAL, "ftr_splat_sets: too many points per frame");
    cudaError_t e;
    if ((e = grow_points(c, c->n_pts + n)) != cudaSuccess) return cuda_fail(c, e, "ftr_splat_sets: point store");
    // host arrays: copied into the staging buffer, then one launch for all sets
    if (host_floats > 0) {
        if ((e = ensure_stage(c, &c->d_stage, &c->stage_cap, sizeof(float) * host_floats)) != cudaSuccess)
            return cuda_fail(c, e, "ftr_splat_sets: staging");
        float* st = (float*)c->d_stage;
        for (int s = 0; s < k; ++s) {
            const int64_t m = S.off[s + 1] - S.off[s];
            const float* src[3] = {S.pts[s], S.nrm[s], S.w[s]};
            const int width[3] = {3, 3, 1};
            for (int a = 0; a < 3; ++a) {
                if (dev[s][a]) continue;
                if ((e = cudaMemcpyAsync(st, src[a], sizeof(float) * width[a] * m, cudaMemcpyHostToDevice,
                                         c->stream)) != cudaSuccess)
                    return cuda_fail(c, e, "ftr_splat_sets: copy");
                if (a == 0) S.pts[s] = st;
                if (a == 1) S.nrm[s] = st;
                if (a == 2) S.w[s] = st;
                st += width[a] * m;
            }
        }
    }
    prof_begin(c, ST_INGEST);
    e = launch_ingest_sets(c, S);
    prof_end(c, ST_INGEST);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_splat_sets: ingest");
    c->n_pts += n;
    c->points_in += n;
    // the staging buffer is reused by the next call: keep host-staged calls ordered
    if (host_floats > 0 && (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_splat_sets");
    return FTR_OK;
}

int ftr_splat_depth(ftr_ctx* c, const ftr_view* views, int k, double step, double noise, int radius,
                    float* const* conf_out) {
    if (!c) return FTR_EINVAL;
    if (c->depth_async) return set_err(c, FTR_ESTATE, "ftr_splat_depth: the frame's points came from the async call");
    int64_t pixels = 0;
    if (int st = raw_enqueue(c, "ftr_splat_depth", views, k, step, noise, radius, conf_out, &pixels)) return st;
    // the point count decides the ingest launch: one wait per call
    cudaError_t e;
    if ((e = cudaMemcpyAsync(c->h_raw_total, c->d_raw_total, sizeof(int), cudaMemcpyDeviceToHost, c->stream)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_splat_depth");
    float* P = c->d_raw;
    return ftr_splat(c, P, P + 3 * pixels, P + 6 * pixels, (int64_t)*c->h_raw_total);
}

int ftr_splat_depth_async(ftr_ctx* c, const ftr_view* views, int k, double step, double noise, int radius,
                          float* const* conf_out) {
    if (!c) return FTR_EINVAL;
    if (c->n_pts != 0 || c->depth_async)
        return set_err(c, FTR_ESTATE, "ftr_splat_depth_async: must be the frame's only point source (after ftr_reset)");
    int64_t pixels = 0;
    if (int st = raw_enqueue(c, "ftr_splat_depth_async", views, k, step, noise, radius, conf_out, &pixels)) return st;
    cudaError_t e;
    // capacity for the bound; the ingest reads the count on the device
    if ((e = grow_points(c, pixels)) != cudaSuccess) return cuda_fail(c, e, "ftr_splat_depth_async: point store");
    float* P = c->d_raw;
    prof_begin(c, ST_INGEST);
    e = launch_ingest(c, P, P + 3 * pixels, P + 6 * pixels, pixels, c->d_raw_total);
    prof_end(c, ST_INGEST);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_splat_depth_async: ingest");
    c->n_pts = pixels;        // a bound: every consumer reads the exact count on the device
    c->points_in = -1;
    c->depth_async = true;
    return FTR_OK;
}

namespace {

// The forward 3D FFT with the integration filter and the inverse 3D FFT
// (Sec. III-B): three plane-fused kernels, or five axis passes.
cudaError_t launch_transforms(ftr_ctx* c) {
    cudaError_t e;
    if (c->fused == 2 && c->p.precision == FTR_PREC_FP32) {
        prof_begin(c, ST_FX);
        e = launch_fx(c);
        prof_end(c, ST_FX);
        if (e != cudaSuccess) return e;
        prof_begin(c, ST_FYZ);
        e = launch_fyz(c);
        prof_end(c, ST_FYZ);
        if (e != cudaSuccess) return e;
        prof_begin(c, ST_IY);
        e = launch_iy(c);
        prof_end(c, ST_IY);
        if (e != cudaSuccess) return e;
        prof_begin(c, ST_IX);
        e = launch_ix(c);
        prof_end(c, ST_IX);
        return e;
    }
    if (c->fused == 1 && c->p.precision == FTR_PREC_FP32) {
        prof_begin(c, ST_FXY);
        e = launch_fxy(c);
        prof_end(c, ST_FXY);
        if (e != cudaSuccess) return e;
        prof_begin(c, ST_FZ);
        e = launch_fz2(c);
        prof_end(c, ST_FZ);
        if (e != cudaSuccess) return e;
        c->rowmm_valid = false;   // the plane-fused inverse writes no row bounds
        prof_begin(c, ST_IYX);
        e = launch_iyx(c);
        prof_end(c, ST_IYX);
        return e;
    }
    prof_begin(c, ST_FX);
    e = launch_fx(c);
    prof_end(c, ST_FX);
    if (e != cudaSuccess) return e;
    prof_begin(c, ST_FY);
    e = launch_fy(c);
    prof_end(c, ST_FY);
    if (e != cudaSuccess) return e;
    prof_begin(c, ST_FZ);
    e = launch_fz(c);
    prof_end(c, ST_FZ);
    if (e != cudaSuccess) return e;
    prof_begin(c, ST_IY);
    e = launch_iy(c);
    prof_end(c, ST_IY);
    if (e != cudaSuccess) return e;
    prof_begin(c, ST_IX);
    e = launch_ix(c);
    prof_end(c, ST_IX);
    return e;
}

}  // namespace

int ftr_solve(ftr_ctx* c, double* iso_level_out) {
    if (!c) return FTR_EINVAL;
    cudaError_t e;
    // each point touches at most 8 bricks
    if ((e = grow_entries(c, 8 * c->n_pts + 1)) != cudaSuccess) return cuda_fail(c, e, "ftr_solve: entries");
    if ((e = grow_heavy(c, c->n_pts)) != cudaSuccess) return cuda_fail(c, e, "ftr_solve: accumulators");
    c->solved = false;
    c->meshed = false;
    if (!c->v_external) {
        if ((e = launch_splat(c)) != cudaSuccess) return cuda_fail(c, e, "ftr_solve: splat");
    }
    if ((e = launch_transforms(c)) != cudaSuccess) return cuda_fail(c, e, "ftr_solve: transforms");
    prof_begin(c, ST_LEVEL);
    e = launch_level(c);
    prof_end(c, ST_LEVEL);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_solve: level");
    c->solved = true;
    if (iso_level_out) {
        if ((e = cudaMemcpyAsync(&c->level_host, c->d_level, sizeof(double), cudaMemcpyDeviceToHost, c->stream)) ||
            (e = launch_flags(c)))
            return cuda_fail(c, e, "ftr_solve: level copy");
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "ftr_solve");
        if (int st = tc_check(c, "ftr_solve")) return st;
        *iso_level_out = c->level_host;
    }
    return FTR_OK;
}

namespace {

// Grow the mesh buffers to hold at least (na, nv, nt) with 50 % headroom.
cudaError_t grow_mesh(ftr_ctx* c, int64_t na, int64_t nv, int64_t nt) {
    cudaError_t e = cudaSuccess;
    if (na > c->cap_mc_nodes || nv > c->cap_verts || nt > c->cap_tris) c->graph_valid = false;
    if (na > c->cap_mc_nodes) {
        cudaStreamSynchronize(c->stream);
        dfree(c->d_mc_nodes);
        const int64_t cap = na + na / 2 + 1024;
        if ((e = dalloc(&c->d_mc_nodes, cap)) != cudaSuccess) return e;
        c->cap_mc_nodes = cap;
    }
    if (nv > c->cap_verts) {
        cudaStreamSynchronize(c->stream);
        dfree(c->d_verts);
        dfree(c->d_vnrm);
        const int64_t cap = nv + nv / 2 + 1024;
        if ((e = dalloc(&c->d_verts, 3 * cap)) != cudaSuccess) return e;
        if ((e = dalloc(&c->d_vnrm, 3 * cap)) != cudaSuccess) return e;
        c->cap_verts = cap;
    }
    if (nt > c->cap_tris) {
        cudaStreamSynchronize(c->stream);
        dfree(c->d_tris);
        const int64_t cap = nt + nt / 2 + 1024;
        if ((e = dalloc(&c->d_tris, 3 * cap)) != cudaSuccess) return e;
        c->cap_tris = cap;
    }
    return e;
}

}  // namespace

int ftr_extract_mesh(ftr_ctx* c, ftr_mesh* out) {
    if (!c || !out) return FTR_EINVAL;
    if (!c->solved) return set_err(c, FTR_ESTATE, "ftr_extract_mesh: nothing solved");
    cudaError_t e;
    // first use: room for a surface of M / 256 vertices (grows on demand)
    if (c->cap_verts == 0) {
        const int64_t guess = c->M / 256 + 4096;
        if ((e = grow_mesh(c, guess, guess, 2 * guess)) != cudaSuccess) return cuda_fail(c, e, "ftr_extract_mesh");
    }
    // counts, offsets and the emission run back to back; the host waits once
    if ((e = launch_mc_count(c)) != cudaSuccess) return cuda_fail(c, e, "ftr_extract_mesh: count");
    if ((e = launch_mc_emit(c)) != cudaSuccess) return cuda_fail(c, e, "ftr_extract_mesh: emit");
    if ((e = launch_mc_totals(c)) != cudaSuccess || (e = launch_flags(c)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_extract_mesh: totals");
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "ftr_extract_mesh");
    if (int st = tc_check(c, "ftr_extract_mesh")) return st;
    const int64_t na = c->h_mc_tot[0], nv = c->h_mc_tot[1], nt = c->h_mc_tot[2];
    if (na > c->cap_mc_nodes || nv > c->cap_verts || nt > c->cap_tris) {
        // the buffers were too small: the kernels skipped the writes past them
        if ((e = grow_mesh(c, na, nv, nt)) != cudaSuccess) return cuda_fail(c, e, "ftr_extract_mesh: grow");
        if ((e = launch_mc_emit(c)) != cudaSuccess) return cuda_fail(c, e, "ftr_extract_mesh: emit");
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "ftr_extract_mesh");
    }
    c->n_verts = nv;
    c->n_tris = nt;
    c->meshed = true;
    out->vertices = c->d_verts;
    out->normals = c->d_vnrm;
    out->tris = c->d_tris;
    out->n_vertices = nv;
    out->n_tris = nt;
    return FTR_OK;
}

int ftr_mesh_copy(ftr_ctx* c, float* vertices, float* normals, int32_t* tris) {
    if (!c) return FTR_EINVAL;
    if (!c->meshed) return set_err(c, FTR_ESTATE, "ftr_mesh_copy: no mesh");
    cudaError_t e = cudaSuccess;
    if (vertices && c->n_verts)
        e = cudaMemcpyAsync(vertices, c->d_verts, sizeof(float) * 3 * c->n_verts, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && normals && c->n_verts)
        e = cudaMemcpyAsync(normals, c->d_vnrm, sizeof(float) * 3 * c->n_verts, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && tris && c->n_tris)
        e = cudaMemcpyAsync(tris, c->d_tris, sizeof(int32_t) * 3 * c->n_tris, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_mesh_copy");
    return FTR_OK;
}

int ftr_mesh_copy_async(ftr_ctx* c, float* vertices, float* normals, int32_t* tris) {
    if (!c) return FTR_EINVAL;
    if (!c->meshed) return set_err(c, FTR_ESTATE, "ftr_mesh_copy_async: no mesh");
    cudaError_t e = cudaSuccess;
    if (vertices && c->n_verts)
        e = cudaMemcpyAsync(vertices, c->d_verts, sizeof(float) * 3 * c->n_verts, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && normals && c->n_verts)
        e = cudaMemcpyAsync(normals, c->d_vnrm, sizeof(float) * 3 * c->n_verts, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess && tris && c->n_tris)
        e = cudaMemcpyAsync(tris, c->d_tris, sizeof(int32_t) * 3 * c->n_tris, cudaMemcpyDefault, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_mesh_copy_async");
    return FTR_OK;
}

int ftr_texture(ftr_ctx* c, const ftr_view* views, int k, float depth_tol, ftr_tex* out) {
    if (!c || !out) return FTR_EINVAL;
    if (k < 0 || k > kMaxViews || (k > 0 && !views)) return set_err(c, FTR_EINVAL, "ftr_texture: 0 <= k <= 8");
    if (!c->meshed) return set_err(c, FTR_ESTATE, "ftr_texture: no mesh");
    if (!(depth_tol >= 0.f)) return set_err(c, FTR_EINVAL, "ftr_texture: depth_tol < 0");
    cudaError_t e;
    ViewSet vs;
    memset(&vs, 0, sizeof(vs));
    vs.k = k;
    // staging layout: per view depth | conf | rgb, then the outputs
    size_t need = 0;
    std::vector<size_t> offs(3 * k + 4);
    for (int i = 0; i < k; ++i) {
        const ftr_view& v = views[i];
        if (v.w <= 0 || v.h <= 0 || v.rgb_w <= 0 || v.rgb_h <= 0 || !v.depth || !v.conf || !v.rgb)
            return set_err(c, FTR_EINVAL, "ftr_texture: view %d incomplete", i);
        offs[3 * i] = need;
        need += is_device_ptr(v.depth) ? 0 : ((sizeof(float) * v.w * v.h + 255) & ~(size_t)255);
        offs[3 * i + 1] = need;
        need += is_device_ptr(v.conf) ? 0 : ((sizeof(float) * v.w * v.h + 255) & ~(size_t)255);
        offs[3 * i + 2] = need;
        need += is_device_ptr(v.rgb) ? 0 : (((size_t)3 * v.rgb_w * v.rgb_h + 255) & ~(size_t)255);
    }
    const int64_t nv = c->n_verts;
    const bool hw = out->weights && !is_device_ptr(out->weights);
    const bool huv = out->uv && !is_device_ptr(out->uv);
    const bool hrgb = out->rgb && !is_device_ptr(out->rgb);
    const bool htex = out->textured && !is_device_ptr(out->textured);
    const size_t o_w = need;
    need += hw ? ((sizeof(float) * nv * k + 255) & ~(size_t)255) : 0;
    const size_t o_uv = need;
    need += huv ? ((sizeof(float) * nv * k * 2 + 255) & ~(size_t)255) : 0;
    const size_t o_rgb = need;
    need += hrgb ? (((size_t)3 * nv + 255) & ~(size_t)255) : 0;
    const size_t o_tex = need;
    need += htex ? (((size_t)nv + 255) & ~(size_t)255) : 0;
    if (need > 0 && (e = ensure_stage(c, &c->d_tex_stage, &c->tex_stage_cap, need)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_texture: staging");
    char* st = (char*)c->d_tex_stage;
    for (int i = 0; i < k; ++i) {
        const ftr_view& v = views[i];
        ViewDev& d = vs.v[i];
        d.w = v.w;
        d.h = v.h;
        d.rgb_w = v.rgb_w;
        d.rgb_h = v.rgb_h;
        for (int j = 0; j < 9; ++j) {
            d.K[j] = d.Kf[j] = v.K[j];
            d.Krgb[j] = d.Krgbf[j] = v.K_rgb[j];
        }
        for (int j = 0; j < 12; ++j) {
            d.RT[j] = d.RTf[j] = v.world_to_cam[j];
            d.RTrgb[j] = d.RTrgbf[j] = v.world_to_rgb[j];
        }
        d.depth = v.depth;
        d.conf = v.conf;
        d.rgb = v.rgb;
        if (!is_device_ptr(v.depth)) {
            float* dst = (float*)(st + offs[3 * i]);
            if ((e = cudaMemcpyAsync(dst, v.depth, sizeof(float) * v.w * v.h, cudaMemcpyHostToDevice, c->stream)))
                return cuda_fail(c, e, "ftr_texture: copy depth");
            d.depth = dst;
        }
        if (!is_device_ptr(v.conf)) {
            float* dst = (float*)(st + offs[3 * i + 1]);
            if ((e = cudaMemcpyAsync(dst, v.conf, sizeof(float) * v.w * v.h, cudaMemcpyHostToDevice, c->stream)))
                return cuda_fail(c, e, "ftr_texture: copy conf");
            d.conf = dst;
        }
        if (!is_device_ptr(v.rgb)) {
            uint8_t* dst = (uint8_t*)(st + offs[3 * i + 2]);
            if ((e = cudaMemcpyAsync(dst, v.rgb, (size_t)3 * v.rgb_w * v.rgb_h, cudaMemcpyHostToDevice, c->stream)))
                return cuda_fail(c, e, "ftr_texture: copy rgb");
            d.rgb = dst;
        }
    }
    float* w = hw ? (float*)(st + o_w) : out->weights;
    float* uv = huv ? (float*)(st + o_uv) : out->uv;
    uint8_t* rgb = hrgb ? (uint8_t*)(st + o_rgb) : out->rgb;
    uint8_t* tex = htex ? (uint8_t*)(st + o_tex) : out->textured;
    if ((e = launch_texture(c, vs, depth_tol, w, uv, rgb, tex)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_texture: kernel");
    bool host_out = false;
    if (hw && nv) { cudaMemcpyAsync(out->weights, w, sizeof(float) * nv * k, cudaMemcpyDeviceToHost, c->stream); host_out = true; }
    if (huv && nv) { cudaMemcpyAsync(out->uv, uv, sizeof(float) * nv * k * 2, cudaMemcpyDeviceToHost, c->stream); host_out = true; }
    if (hrgb && nv) { cudaMemcpyAsync(out->rgb, rgb, (size_t)3 * nv, cudaMemcpyDeviceToHost, c->stream); host_out = true; }
    if (htex && nv) { cudaMemcpyAsync(out->textured, tex, (size_t)nv, cudaMemcpyDeviceToHost, c->stream); host_out = true; }
    bool host_in = false;
    for (int i = 0; i < k; ++i)
        host_in = host_in || !is_device_ptr(views[i].depth) || !is_device_ptr(views[i].conf) ||
                  !is_device_ptr(views[i].rgb);
    if (host_out || host_in) {
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "ftr_texture");
    }
    return FTR_OK;
}

namespace {

// Device-only view set for the queued paths (images must already be on the device).
int device_viewset(ftr_ctx* c, const ftr_view* views, int k, ViewSet& vs, const char* who) {
    memset(&vs, 0, sizeof(vs));
    vs.k = k;
    for (int i = 0; i < k; ++i) {
        const ftr_view& v = views[i];
        if (v.w <= 0 || v.h <= 0 || v.rgb_w <= 0 || v.rgb_h <= 0 || !is_device_ptr(v.depth) ||
            !is_device_ptr(v.conf) || !is_device_ptr(v.rgb))
            return set_err(c, FTR_EINVAL, "%s: view %d needs device images", who, i);
        ViewDev& d = vs.v[i];
        d.w = v.w;
        d.h = v.h;
        d.rgb_w = v.rgb_w;
        d.rgb_h = v.rgb_h;
        for (int j = 0; j < 9; ++j) {
            d.K[j] = d.Kf[j] = v.K[j];
            d.Krgb[j] = d.Krgbf[j] = v.K_rgb[j];
        }
        for (int j = 0; j < 12; ++j) {
            d.RT[j] = d.RTf[j] = v.world_to_cam[j];
            d.RTrgb[j] = d.RTrgbf[j] = v.world_to_rgb[j];
        }
        d.depth = v.depth;
        d.conf = v.conf;
        d.rgb = v.rgb;
    }
    return FTR_OK;
}

// Enqueue solve + marching cubes + texture exactly as the separate calls do.
cudaError_t enqueue_frame(ftr_ctx* c, const ViewSet& vs, float tol, const ftr_tex& out, int64_t out_capacity) {
    cudaError_t e;
    if ((e = launch_splat(c)) != cudaSuccess) return e;
    if ((e = launch_transforms(c)) != cudaSuccess) return e;
    if ((e = launch_level(c)) != cudaSuccess) return e;
    if ((e = launch_mc_count(c)) != cudaSuccess) return e;
    if ((e = launch_mc_emit(c)) != cudaSuccess) return e;
    if (vs.k > 0) {
        const int64_t limit = out_capacity < c->cap_verts ? out_capacity : c->cap_verts;
        e = launch_texture_bounded(c, vs, tol, limit, c->d_mc_off + 3 * (c->mc_blocks + 1) + 1, out.weights, out.uv,
                                   out.rgb, out.textured);
        if (e != cudaSuccess) return e;
    }
    if ((e = launch_mc_totals(c)) != cudaSuccess) return e;
    return launch_flags(c);
}

}  // namespace

int ftr_frame_launch(ftr_ctx* c, const ftr_view* views, int k, float depth_tol, ftr_tex* out, int64_t out_capacity) {
    if (!c || !out) return FTR_EINVAL;
    if (c->v_external) return set_err(c, FTR_ESTATE, "ftr_frame_launch: works on splatted points only");
    if (c->mesh_pending) return set_err(c, FTR_ESTATE, "ftr_frame_launch: finish the previous frame first");
    if (k < 0 || k > kMaxViews || (k > 0 && !views)) return set_err(c, FTR_EINVAL, "ftr_frame_launch: 0 <= k <= 8");
    if (!(depth_tol >= 0.f) || out_capacity < 0) return set_err(c, FTR_EINVAL, "ftr_frame_launch: bad argument");
    ViewSet vs;
    int st = device_viewset(c, views, k, vs, "ftr_frame_launch");
    if (st != FTR_OK) return st;
    const void* outs[4] = {out->weights, out->uv, out->rgb, out->textured};
    for (int i = 0; i < 4; ++i)
        if (outs[i] && !is_device_ptr(outs[i]))
            return set_err(c, FTR_EINVAL, "ftr_frame_launch: outputs must be device memory");
    cudaError_t e;
    // every buffer the graph captures is sized here, outside the capture
    if ((e = grow_entries(c, 8 * c->n_pts + 1)) != cudaSuccess) return cuda_fail(c, e, "ftr_frame_launch");
    if ((e = grow_heavy(c, c->n_pts)) != cudaSuccess) return cuda_fail(c, e, "ftr_frame_launch");
    if (c->cap_verts == 0) {
        const int64_t guess = c->M / 256 + 4096;
        if ((e = grow_mesh(c, guess, guess, 2 * guess)) != cudaSuccess) return cuda_fail(c, e, "ftr_frame_launch");
        c->graph_valid = false;
    }
    const bool same_but_views = c->graph_valid && c->graph_tol == depth_tol && c->graph_cap == out_capacity &&
                                memcmp(c->graph_outs, outs, sizeof(outs)) == 0;
    bool same = same_but_views && memcmp(&c->graph_vs, &vs, sizeof(vs)) == 0;
    if (same_but_views && !same && c->graph_tex_node && vs.k == c->graph_vs.k && vs.k > 0) {
        // only the images or calibrations changed: give the graph's texture
        // node the new view set instead of capturing the frame again
        cudaKernelNodeParams kp;
        if (cudaGraphKernelNodeGetParams(c->graph_tex_node, &kp) == cudaSuccess && kp.kernelParams &&
            kp.func == texture_kernel(vs.k)) {
            void* args[9];
            for (int i = 0; i < 9; ++i) args[i] = kp.kernelParams[i];
            ViewSet vs_arg = vs;
            args[0] = &vs_arg;
            kp.kernelParams = args;
            if (cudaGraphExecKernelNodeSetParams(c->graph_exec, c->graph_tex_node, &kp) == cudaSuccess &&
                cudaGraphKernelNodeSetParams(c->graph_tex_node, &kp) == cudaSuccess) {
                c->graph_vs = vs;
                same = true;
            }
        }
        cudaGetLastError();
    }
    if (!same) {
        if (c->graph_exec) {
            cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
        }
        if (c->graph) {
            cudaGraphDestroy(c->graph);
            c->graph = nullptr;
        }
        c->graph_tex_node = nullptr;
        const bool prof = c->prof;
        c->prof = false;                 // no event records inside the capture
        const int64_t l0 = c->launches;
        cudaGraph_t graph = nullptr;
        e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_frame(c, vs, depth_tol, *out, out_capacity);
            e = cudaStreamEndCapture(c->stream, &graph);
            if (e2 != cudaSuccess) e = e2;
        }
        c->prof = prof;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
        if (e == cudaSuccess && vs.k > 0) {
            // remember the texture kernel node for views-only updates
            size_t n = 0;
            if (cudaGraphGetNodes(graph, nullptr, &n) == cudaSuccess && n > 0) {
                std::vector<cudaGraphNode_t> nodes(n);
                if (cudaGraphGetNodes(graph, nodes.data(), &n) == cudaSuccess) {
                    const void* tex_fn = texture_kernel(vs.k);
                    for (size_t i = 0; i < n; ++i) {
                        cudaGraphNodeType t;
                        cudaKernelNodeParams kp;
                        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel &&
                            cudaGraphKernelNodeGetParams(nodes[i], &kp) == cudaSuccess && kp.func == tex_fn) {
                            c->graph_tex_node = nodes[i];
                            break;
                        }
                    }
                }
            }
            cudaGetLastError();
        }
        if (e == cudaSuccess) {
            c->graph = graph;                 // kept: its texture node is updated in place
        } else if (graph) {
            cudaGraphDestroy(graph);
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "ftr_frame_launch: graph capture");
        c->graph_launches = c->launches - l0;
        c->launches = l0;
        c->graph_valid = true;
        c->graph_vs = vs;
        c->graph_tol = depth_tol;
        c->graph_cap = out_capacity;
        memcpy(c->graph_outs, outs, sizeof(outs));
    }
    if ((e = cudaGraphLaunch(c->graph_exec, c->stream)) != cudaSuccess) return cuda_fail(c, e, "ftr_frame_launch");
    c->launches += c->graph_launches;
    c->solved = true;
    c->meshed = false;
    c->mesh_pending = true;
    c->tex_pending = k > 0;
    c->tex_vs = vs;
    c->tex_tol = depth_tol;
    c->tex_capacity = out_capacity;
    c->tex_w = out->weights;
    c->tex_uv = out->uv;
    c->tex_rgb = out->rgb;
    c->tex_flag = out->textured;
    return FTR_OK;
}

int ftr_texture_vertices(ftr_ctx* c, const ftr_view* views, int k, float depth_tol, const float* vertices,
                         int64_t n_vertices, ftr_tex* out) {
    if (!c || !out) return FTR_EINVAL;
    if (k < 1 || k > kMaxViews || !views) return set_err(c, FTR_EINVAL, "ftr_texture_vertices: 1 <= k <= 8");
    if (!(depth_tol >= 0.f) || n_vertices < 0) return set_err(c, FTR_EINVAL, "ftr_texture_vertices: bad argument");
    if (n_vertices > 0 && !is_device_ptr(vertices))
        return set_err(c, FTR_EINVAL, "ftr_texture_vertices: vertices must be device memory");
    const void* outs[4] = {out->weights, out->uv, out->rgb, out->textured};
    for (int i = 0; i < 4; ++i)
        if (outs[i] && !is_device_ptr(outs[i]))
            return set_err(c, FTR_EINVAL, "ftr_texture_vertices: outputs must be device memory");
    ViewSet vs;
    int st = device_viewset(c, views, k, vs, "ftr_texture_vertices");
    if (st != FTR_OK) return st;
    cudaError_t e = launch_texture_vertices(c, vs, depth_tol, vertices, n_vertices, out->weights, out->uv, out->rgb,
                                            out->textured);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_texture_vertices");
    return FTR_OK;
}

int ftr_extract_mesh_async(ftr_ctx* c) {
    if (!c) return FTR_EINVAL;
    if (!c->solved) return set_err(c, FTR_ESTATE, "ftr_extract_mesh_async: nothing solved");
    cudaError_t e;
    if (c->cap_verts == 0) {
        const int64_t guess = c->M / 256 + 4096;
        if ((e = grow_mesh(c, guess, guess, 2 * guess)) != cudaSuccess) return cuda_fail(c, e, "extract_async");
    }
    if ((e = launch_mc_count(c)) != cudaSuccess) return cuda_fail(c, e, "ftr_extract_mesh_async: count");
    if ((e = launch_mc_emit(c)) != cudaSuccess) return cuda_fail(c, e, "ftr_extract_mesh_async: emit");
    if ((e = launch_mc_totals(c)) != cudaSuccess || (e = launch_flags(c)) != cudaSuccess)
        return cuda_fail(c, e, "ftr_extract_mesh_async: totals");
    c->meshed = false;
    c->mesh_pending = true;
    c->tex_pending = false;
    return FTR_OK;
}

int64_t ftr_mesh_capacity(const ftr_ctx* c) { return c ? c->cap_verts : 0; }

int ftr_texture_async(ftr_ctx* c, const ftr_view* views, int k, float depth_tol, ftr_tex* out,
                      int64_t out_capacity) {
    if (!c || !out) return FTR_EINVAL;
    if (!c->mesh_pending) return set_err(c, FTR_ESTATE, "ftr_texture_async: no pending mesh");
    if (k < 0 || k > kMaxViews || (k > 0 && !views)) return set_err(c, FTR_EINVAL, "ftr_texture_async: 0 <= k <= 8");
    if (!(depth_tol >= 0.f) || out_capacity < 0) return set_err(c, FTR_EINVAL, "ftr_texture_async: bad argument");
    ViewSet vs;
    memset(&vs, 0, sizeof(vs));
    vs.k = k;
    for (int i = 0; i < k; ++i) {
        const ftr_view& v = views[i];
        if (v.w <= 0 || v.h <= 0 || v.rgb_w <= 0 || v.rgb_h <= 0 || !is_device_ptr(v.depth) ||
            !is_device_ptr(v.conf) || !is_device_ptr(v.rgb))
            return set_err(c, FTR_EINVAL, "ftr_texture_async: view %d needs device images", i);
        ViewDev& d = vs.v[i];
        d.w = v.w;
        d.h = v.h;
        d.rgb_w = v.rgb_w;
        d.rgb_h = v.rgb_h;
        for (int j = 0; j < 9; ++j) {
            d.K[j] = d.Kf[j] = v.K[j];
            d.Krgb[j] = d.Krgbf[j] = v.K_rgb[j];
        }
        for (int j = 0; j < 12; ++j) {
            d.RT[j] = d.RTf[j] = v.world_to_cam[j];
            d.RTrgb[j] = d.RTrgbf[j] = v.world_to_rgb[j];
        }
        d.depth = v.depth;
        d.conf = v.conf;
        d.rgb = v.rgb;
    }
    const void* outs[4] = {out->weights, out->uv, out->rgb, out->textured};
    for (int i = 0; i < 4; ++i)
        if (outs[i] && !is_device_ptr(outs[i]))
            return set_err(c, FTR_EINVAL, "ftr_texture_async: outputs must be device memory");
    const int nr = c->mc_blocks;
    const int64_t limit = out_capacity < c->cap_verts ? out_capacity : c->cap_verts;
    cudaError_t e = launch_texture_bounded(c, vs, depth_tol, limit, c->d_mc_off + 3 * (nr + 1) + 1, out->weights,
                                           out->uv, out->rgb, out->textured);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_texture_async");
    c->tex_pending = true;
    c->tex_vs = vs;
    c->tex_tol = depth_tol;
    c->tex_capacity = out_capacity;
    c->tex_w = out->weights;
    c->tex_uv = out->uv;
    c->tex_rgb = out->rgb;
    c->tex_flag = out->textured;
    return FTR_OK;
}

int ftr_frame_finish(ftr_ctx* c, ftr_mesh* out) {
    if (!c || !out) return FTR_EINVAL;
    if (!c->mesh_pending) return set_err(c, FTR_ESTATE, "ftr_frame_finish: nothing pending");
    cudaError_t e;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "ftr_frame_finish");
    if (int st = tc_check(c, "ftr_frame_finish")) {
        c->mesh_pending = false;
        c->tex_pending = false;
        return st;
    }
    const int64_t na = c->h_mc_tot[0], nv = c->h_mc_tot[1], nt = c->h_mc_tot[2];
    if (na > c->cap_mc_nodes || nv > c->cap_verts || nt > c->cap_tris) {
        if ((e = grow_mesh(c, na, nv, nt)) != cudaSuccess) return cuda_fail(c, e, "ftr_frame_finish: grow");
        if ((e = launch_mc_emit(c)) != cudaSuccess) return cuda_fail(c, e, "ftr_frame_finish: emit");
        if (c->tex_pending && nv <= c->tex_capacity) {
            e = launch_texture_bounded(c, c->tex_vs, c->tex_tol, nv, nullptr, c->tex_w, c->tex_uv, c->tex_rgb,
                                       c->tex_flag);
            if (e != cudaSuccess) return cuda_fail(c, e, "ftr_frame_finish: texture");
        }
        if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "ftr_frame_finish");
    }
    c->n_verts = nv;
    c->n_tris = nt;
    c->meshed = true;
    c->mesh_pending = false;
    out->vertices = c->d_verts;
    out->normals = c->d_vnrm;
    out->tris = c->d_tris;
    out->n_vertices = nv;
    out->n_tris = nt;
    const bool tex_short = c->tex_pending && nv > c->tex_capacity;
    c->tex_pending = false;
    if (tex_short)
        return set_err(c, FTR_ECAPACITY, "ftr_frame_finish: %lld vertices exceed the texture outputs (%lld)",
                       (long long)nv, (long long)c->tex_capacity);
    return FTR_OK;
}

int ftr_stats(const ftr_ctx* c, int64_t* points_in, int64_t* points_dropped) {
    if (!c) return FTR_EINVAL;
    if (points_in) {
        *points_in = c->points_in;
        if (c->points_in < 0) {     // counted on the device (ftr_splat_depth_async)
            int64_t n = 0;
            cudaError_t e = cudaMemcpyAsync(&n, c->d_npts, sizeof(n), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return FTR_ECUDA;
            *points_in = n;
        }
    }
    if (points_dropped) {
        unsigned long long d = 0;
        cudaError_t e = cudaMemcpyAsync(&d, c->d_dropped, sizeof(d), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return FTR_ECUDA;
        *points_dropped = (int64_t)d;
    }
    return FTR_OK;
}

namespace {
std::mutex g_plan_mu;
// (device, n) -> lines per CTA of the y, z, inverse-y passes, transform path,
// marching-cubes tile size and triangle CTAs per SM (0, 0: not timed)
std::map<std::tuple<int, int, int, int>, std::array<int, 6>> g_plans;

bool valid_lines(int f) { return f == 8 || f == 16 || f == 32; }

// F lines per CTA must tile the axis the pass strides over (z for the y
// passes, y for the z pass).  -16: the y pass with bulk-copied tiles (16
// lines, lines of at most 256).
bool plan_fits(const ftr_ctx* c, int pass, int f) {
    const int n = pass == 1 ? c->g.n[1] : c->g.n[2];
    if (f == -16) return (pass == 0 && n % 16 == 0 && c->g.n[1] <= 256) || (pass == 1 && n % 16 == 0);
    return valid_lines(f) && n % f == 0;
}
}  // namespace

int ftr_get_plan(const ftr_ctx* c, int* plan) {
    if (!c || !plan) return FTR_EINVAL;
    for (int i = 0; i < 3; ++i) plan[i] = c->plan_lines[i];
    return FTR_OK;
}

int ftr_set_plan(ftr_ctx* c, const int* plan) {
    if (!c || !plan) return FTR_EINVAL;
    for (int i = 0; i < 3; ++i)
        if (!plan_fits(c, i, plan[i]))
            return set_err(c, FTR_EINVAL, "ftr_set_plan: lines per CTA must be 8, 16 or 32 and divide the grid");
    if (c->p.precision != FTR_PREC_FP32) return set_err(c, FTR_EINVAL, "ftr_set_plan: fp32 passes only");
    for (int i = 0; i < 3; ++i) c->plan_lines[i] = plan[i];
    c->graph_valid = false;
    return FTR_OK;
}

int ftr_get_mc_plan(const ftr_ctx* c, int* plan) {
    if (!c || !plan) return FTR_EINVAL;
    plan[0] = c->mc_tile;
    plan[1] = c->mc_tris_per_sm;
    return FTR_OK;
}

int ftr_set_mc_plan(ftr_ctx* c, const int* plan) {
    if (!c || !plan) return FTR_EINVAL;
    if (!mc_plan_valid(plan[0], plan[1]))
        return set_err(c, FTR_EINVAL, "ftr_set_mc_plan: tile 128, 256 or 512 and 1 to 16 triangle CTAs per SM");
    if (c->mesh_pending) return set_err(c, FTR_ESTATE, "ftr_set_mc_plan: a frame is pending");
    c->mc_tile = plan[0];
    c->mc_tris_per_sm = plan[1];
    c->graph_valid = false;
    return FTR_OK;
}

int ftr_get_transform_path(const ftr_ctx* c) {
    if (!c) return FTR_EINVAL;
    return c->fused;
}

namespace {
// The ring and counters of the persistent y+z pass, allocated on first use.
cudaError_t ensure_yz_ring(ftr_ctx* c) {
    if (c->d_ring && c->d_yz_sync) return cudaSuccess;
    cudaError_t e;
    if ((e = dalloc(&c->d_ring, yz_ring_elems(c->g.n))) != cudaSuccess ||
        (e = dalloc(&c->d_yz_sync, (size_t)yz_sync_ints(c->g.n))) != cudaSuccess) {
        dfree(c->d_ring);
        dfree(c->d_yz_sync);
        cudaGetLastError();
    }
    return e;
}

// Free them once another path is chosen (the context's graph is rebuilt
// before its next launch, so no captured launch refers to them).
void release_yz_ring(ftr_ctx* c) {
    if (!c->d_ring && !c->d_yz_sync) return;
    cudaStreamSynchronize(c->stream);
    dfree(c->d_ring);
    dfree(c->d_yz_sync);
}
}  // namespace

int ftr_set_transform_path(ftr_ctx* c, int fused) {
    if (!c || fused < 0 || fused > 2) return FTR_EINVAL;
    if (fused == 1 && !c->fused_ok)
        return set_err(c, FTR_EINVAL, "ftr_set_transform_path: no plane-fused kernels for this grid or precision");
    if (fused == 2 && !c->yz_ok)
        return set_err(c, FTR_EINVAL, "ftr_set_transform_path: no persistent y+z kernel for this grid or precision");
    if (c->mesh_pending) return set_err(c, FTR_ESTATE, "ftr_set_transform_path: a frame is pending");
    if (fused == 2) {
        if (ensure_yz_ring(c) != cudaSuccess)
            return set_err(c, FTR_ENOMEM, "ftr_set_transform_path: no device memory for the y+z ring");
    } else {
        release_yz_ring(c);
    }
    c->fused = fused;
    c->graph_valid = false;
    c->solved = false;
    c->meshed = false;
    return FTR_OK;
}

int ftr_autotune(ftr_ctx* c, float* report) {
    if (!c) return FTR_EINVAL;
    if (report)
        for (int i = 0; i < 16; ++i) report[i] = 0.f;
    if (c->mesh_pending) return set_err(c, FTR_ESTATE, "ftr_autotune: a frame is pending");
    if (c->p.precision != FTR_PREC_FP32) return FTR_OK;
    const auto key = std::make_tuple(c->device, c->g.n[0], c->g.n[1], c->g.n[2]);
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        auto it = g_plans.find(key);
        if (it != g_plans.end()) {
            for (int i = 0; i < 3; ++i) c->plan_lines[i] = it->second[i];
            int pth = it->second[3];
            if (pth == 2 && !(c->yz_ok && ensure_yz_ring(c) == cudaSuccess)) pth = 0;
            c->fused = (pth == 1 && c->fused_ok) || pth == 2 ? pth : 0;
            if (c->fused != 2) release_yz_ring(c);
            if (mc_plan_valid(it->second[4], it->second[5])) {
                c->mc_tile = it->second[4];
                c->mc_tris_per_sm = it->second[5];
            }
            c->graph_valid = false;
            return FTR_OK;
        }
    }
    cudaError_t e;
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) return cuda_fail(c, e, "ftr_autotune");
    // marching-cubes block sizes, timed on the last frame's indicator and level
    // while they are still valid (the transform timing below overwrites them):
    // the count and emit tiles and the triangle pass's CTAs per SM; every
    // choice gives the same mesh (records, vertices and triangles follow node
    // order)
    int mc_best[2] = {0, 0};
    if (c->solved && c->meshed && c->n_verts > 0) {
        cudaEvent_t m0, m1;
        cudaEventCreate(&m0);
        cudaEventCreate(&m1);
        const int tiles[3] = {128, 256, 512}, per_sm[3] = {2, 4, 8};
        float best_us = 1e30f;
        for (int ti = 0; ti < 3; ++ti)
            for (int mi = 0; mi < 3; ++mi) {
                c->mc_tile = tiles[ti];
                c->mc_tris_per_sm = per_sm[mi];
                auto run = [&]() {
                    cudaError_t r = launch_mc_count(c);
                    return r == cudaSuccess ? launch_mc_emit(c) : r;
                };
                if (run() != cudaSuccess) {
                    cudaGetLastError();
                    continue;
                }
                cudaEventRecord(m0, c->stream);
                for (int r = 0; r < 5; ++r) run();
                cudaEventRecord(m1, c->stream);
                if (cudaEventSynchronize(m1) != cudaSuccess) {
                    cudaEventDestroy(m0);
                    cudaEventDestroy(m1);
                    return cuda_fail(c, cudaGetLastError(), "ftr_autotune: marching cubes");
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, m0, m1);
                if (1000.f * ms / 5 < best_us) {
                    best_us = 1000.f * ms / 5;
                    mc_best[0] = tiles[ti];
                    mc_best[1] = per_sm[mi];
                }
            }
        cudaEventDestroy(m0);
        cudaEventDestroy(m1);
        c->mc_tile = mc_best[0] ? mc_best[0] : 256;
        c->mc_tris_per_sm = mc_best[1] ? mc_best[1] : 4;
    }
    // the live z-slab of the last solved frame when there is one (the forward
    // passes skip planes outside it), else every plane live; a later splat
    // rewrites these values
    if (!c->solved) {
        const int meta[4] = {c->n_bricks, 0, 0, c->g.nb[2] - 1};
        if ((e = cudaMemcpyAsync(c->d_meta, meta, sizeof(meta), cudaMemcpyHostToDevice, c->stream)) != cudaSuccess)
            return cuda_fail(c, e, "ftr_autotune");
    }
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    const int F[4] = {8, 16, 32, -16};
    const int reps = 5;
    // mean microseconds of `reps` runs of f (after one untimed run); < 0 if it does not launch
    auto time_us = [&](auto&& f) -> float {
        if (f() != cudaSuccess) {
            cudaGetLastError();
            return -1.f;
        }
        cudaEventRecord(t0, c->stream);
        for (int r = 0; r < reps; ++r) f();
        cudaEventRecord(t1, c->stream);
        if (cudaEventSynchronize(t1) != cudaSuccess) return -2.f;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        return 1000.f * ms / reps;
    };
    // candidates keep at least two CTAs per SM: a CTA that fills an SM
    // alone waits for a whole SM to drain when frames of other contexts run
    // concurrently
    auto fits_twice = [&](auto&& f) {
        int occ = 0;
        c->occ_query = &occ;
        const cudaError_t qe = f();
        c->occ_query = nullptr;
        if (qe != cudaSuccess) cudaGetLastError();
        return qe == cudaSuccess && occ >= 2;
    };
    // one tile height per pass of the five-pass transforms, and of the z pass
    // of the plane-fused ones
    std::array<int, 3> best = {16, 16, 16};
    int best_fz2 = 16;
    const int saved_path = c->fused;
    for (int pass = 0; pass < 4; ++pass) {
        if (pass == 3 && !c->fused_ok) break;
        const int slot = pass == 3 ? 1 : pass;
        c->fused = pass == 3 ? 1 : 0;
        float best_us = 1e30f;
        for (int v = 0; v < 4; ++v) {
            if (!plan_fits(c, slot, F[v]) || (pass == 3 && F[v] < 0)) continue;   // the fused z pass: 8, 16, 32
            c->plan_lines[slot] = F[v];
            auto run = [&]() {
                if (pass == 3) return launch_fz2(c);
                return pass == 0 ? launch_fy(c) : (pass == 1 ? launch_fz(c) : launch_iy(c));
            };
            if (!fits_twice(run)) continue;
            const float us = time_us(run);
            if (us == -2.f) {
                cudaEventDestroy(t0);
                cudaEventDestroy(t1);
                c->fused = saved_path;
                return cuda_fail(c, cudaGetLastError(), "ftr_autotune");
            }
            if (us < 0.f) continue;          // the variant does not fit: skip it
            if (report && pass < 3) report[4 * pass + v] = us;
            if (us < best_us) {
                best_us = us;
                if (pass == 3)
                    best_fz2 = F[v];
                else
                    best[pass] = F[v];
            }
        }
        c->plan_lines[slot] = best[slot];
    }
    // the transform path: both whole chains (forward, filter, inverse) at
    // their best tile heights; the faster one is kept
    int path = 0;
    c->fused = 0;
    for (int i = 0; i < 3; ++i) c->plan_lines[i] = best[i];
    const float five_us = time_us([&]() { return launch_transforms(c); });
    if (report) report[12] = five_us;
    float best_chain = five_us;
    if (c->fused_ok) {
        c->fused = 1;
        c->plan_lines[1] = best_fz2;
        const float fused_us = time_us([&]() { return launch_transforms(c); });
        if (report) report[13] = fused_us;
        if (fused_us > 0.f && (best_chain < 0.f || fused_us < best_chain)) {
            path = 1;
            best_chain = fused_us;
        }
        c->plan_lines[1] = best[1];
    }
    if (c->yz_ok && ensure_yz_ring(c) == cudaSuccess) {
        c->fused = 2;
        const float yz_us = time_us([&]() { return launch_transforms(c); });
        if (report) report[15] = yz_us;
        if (yz_us > 0.f && (best_chain < 0.f || yz_us < best_chain)) {
            path = 2;
            best_chain = yz_us;
        }
    }
    if (path == 1) best[1] = best_fz2;
    c->fused = path;
    if (path != 2) release_yz_ring(c);
    for (int i = 0; i < 3; ++i) c->plan_lines[i] = best[i];
    if (report) report[14] = (float)path;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(c, e, "ftr_autotune");
    c->graph_valid = false;
    c->solved = false;       // the timing runs overwrote the spectra and the indicator
    c->meshed = false;
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        g_plans[key] = {best[0], best[1], best[2], path, mc_best[0], mc_best[1]};
    }
    return FTR_OK;
}

namespace {
// Capacities that decide a context's device memory besides its grid.
struct Caps {
    int64_t pts = 0, stage = 0, tex_stage = 0, entries = 0, units = 0, heavy = 0, raw = 0, raw_tiles = 0;
    int64_t mc_nodes = 0, verts = 0, tris = 0;
    bool tc = false;
    bool yz = false;     // the persistent y+z pass's ring and counters
};

int64_t context_bytes(const int n[3], const Caps& k) {
    const int64_t M = (int64_t)n[0] * n[1] * n[2];
    const int64_t Mh = (int64_t)(n[0] / 2 + 1) * n[1] * n[2];
    const int64_t nb = (int64_t)(n[0] / kBrick) * (n[1] / kBrick) * (n[2] / kBrick);
    const int64_t mc_blocks = (int64_t)n[1] * n[2];
    const int64_t level_blocks = 304;
    int64_t b = 0;
    b += k.pts * (int64_t)(sizeof(int4) + 2 * sizeof(float4));
    b += k.stage + k.tex_stage;
    b += nb * (int64_t)sizeof(int) * 5 + (nb / kBrickScanTile + 1) * (int64_t)sizeof(int4) + 64;
    b += k.entries * (int64_t)sizeof(int);
    b += k.units * (int64_t)sizeof(int);
    b += k.heavy * (4 * kBrickVox * 8 + 4) + nb * 8;   // heavy-brick accumulators, chunk offsets
    b += nb * 3 * kBrickVox * (int64_t)sizeof(float);
    b += 5 * Mh * (int64_t)sizeof(float2) + M * (int64_t)sizeof(float);
    b += 3 * (int64_t)(n[0] + n[1] + n[2]) * (int64_t)sizeof(float2);
    if (k.tc) b += (int64_t)tc_table_bytes() + 16;
    if (k.yz) b += (int64_t)(yz_ring_elems(n) * sizeof(float2)) + (int64_t)yz_sync_ints(n) * (int64_t)sizeof(int);
    b += k.raw * 7 * (int64_t)sizeof(float) + k.raw_tiles * (int64_t)sizeof(int);
    b += (2 * level_blocks + 8) * (int64_t)sizeof(double);
    b += (6 * mc_blocks + 16) * (int64_t)sizeof(int);
    b += mc_blocks * 16 * (int64_t)sizeof(unsigned);   // inside bits (upper bound)
    b += mc_blocks * (int64_t)sizeof(float2);          // row min / max of A
    b += mc_blocks * 16 * (int64_t)sizeof(int2);       // per-word record index and mask (upper bound)
    b += k.mc_nodes * (int64_t)sizeof(int4) + k.verts * 6 * (int64_t)sizeof(float) +
         k.tris * 3 * (int64_t)sizeof(int32_t);
    return b;
}

int64_t pow2_cap(int64_t need, int64_t first) {
    int64_t cap = first;
    while (cap < need) cap *= 2;
    return cap;
}
}  // namespace

int64_t ftr_device_bytes(const ftr_ctx* c) {
    if (!c) return 0;
    Caps k;
    k.pts = c->pts.cap;
    k.stage = (int64_t)c->stage_cap;
    k.tex_stage = (int64_t)c->tex_stage_cap;
    k.entries = c->cap_entries;
    k.units = c->cap_units;
    k.heavy = c->cap_heavy;
    k.raw = c->raw_cap;
    k.raw_tiles = c->raw_tiles_cap;
    k.mc_nodes = c->cap_mc_nodes;
    k.verts = c->cap_verts;
    k.tris = c->cap_tris;
    k.tc = c->d_tc_table != nullptr;
    k.yz = c->d_ring != nullptr;
    return context_bytes(c->g.n, k);
}

int64_t ftr_estimate_bytes(const int grid_n[3], int64_t points, int64_t depth_pixels, int64_t vertices,
                           int64_t tris, int precision) {
    if (!grid_n || points < 0 || depth_pixels < 0 || vertices < 0 || tris < 0) return -1;
    for (int a = 0; a < 3; ++a)
        if (!supported_n(grid_n[a])) return -1;
    Caps k;
    // the growth rules of the point store, the (point, brick) pairs and the
    // accumulation chunks, at these sizes; device inputs need no staging
    const int64_t pts = points > depth_pixels ? points : depth_pixels;
    k.pts = pts > 0 ? pow2_cap(pts, 1 << 16) : 0;
    k.entries = pow2_cap(8 * pts + 1, 1 << 18);
    const int64_t nb = (int64_t)(grid_n[0] / kBrick) * (grid_n[1] / kBrick) * (grid_n[2] / kBrick);
    k.units = nb + k.entries / kSplatChunk + 2;
    k.heavy = heavy_capacity(pts);
    k.raw = depth_pixels;
    k.raw_tiles = depth_pixels > 0 ? depth_pixels / 128 + 16 * 1024 : 0;
    // mesh buffers grow to 1.5 x what a frame needs (+1024); active nodes <= vertices
    k.mc_nodes = vertices + vertices / 2 + 1024;
    k.verts = vertices + vertices / 2 + 1024;
    k.tris = tris + tris / 2 + 1024;
    k.tc = precision != FTR_PREC_FP32;
    k.yz = false;   // the y+z ring exists only while transform path 2 is in use
    return context_bytes(grid_n, k);
}

const char* ftr_last_error(const ftr_ctx* c) {
    if (!c) return "null context";
    return c->err.c_str();
}

int ftr_get_field_V(ftr_ctx* c, float* out) {
    if (!c || !out) return FTR_EINVAL;
    if (!c->solved) return set_err(c, FTR_ESTATE, "ftr_get_field_V: nothing solved");
    cudaError_t e;
    float* dst = out;
    float* tmp = nullptr;
    if (!is_device_ptr(out)) {
        if ((e = cudaMalloc(&tmp, sizeof(float) * 3 * c->M)) != cudaSuccess) return cuda_fail(c, e, "get_field_V");
        dst = tmp;
    }
    e = launch_dense_V(c, dst);
    if (e == cudaSuccess && tmp)
        e = cudaMemcpyAsync(out, tmp, sizeof(float) * 3 * c->M, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_get_field_V");
    return FTR_OK;
}

int ftr_get_field_A(ftr_ctx* c, float* out) {
    if (!c || !out) return FTR_EINVAL;
    if (!c->solved) return set_err(c, FTR_ESTATE, "ftr_get_field_A: nothing solved");
    cudaError_t e = cudaMemcpyAsync(out, c->d_A, sizeof(float) * c->M, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_get_field_A");
    return FTR_OK;
}

int ftr_set_field_V(ftr_ctx* c, const float* V) {
    if (!c || !V) return FTR_EINVAL;
    cudaError_t e;
    const float* src = V;
    float* tmp = nullptr;
    if (!is_device_ptr(V)) {
        if ((e = cudaMalloc(&tmp, sizeof(float) * 3 * c->M)) != cudaSuccess) return cuda_fail(c, e, "set_field_V");
        if ((e = cudaMemcpyAsync(tmp, V, sizeof(float) * 3 * c->M, cudaMemcpyHostToDevice, c->stream))) {
            cudaFree(tmp);
            return cuda_fail(c, e, "set_field_V");
        }
        src = tmp;
    }
    e = launch_load_dense_V(c, src);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_set_field_V");
    c->n_pts = 0;
    cudaMemsetAsync(c->d_npts, 0, sizeof(int64_t), c->stream);
    c->v_external = true;
    return FTR_OK;
}

int ftr_set_indicator(ftr_ctx* c, const float* A, double level) {
    if (!c || !A) return FTR_EINVAL;
    cudaError_t e = cudaMemcpyAsync(c->d_A, A, sizeof(float) * c->M, cudaMemcpyDefault, c->stream);
    double lv[2] = {level, 1.0};
    // float thresholds: rounded up (same decision as the float64 compare) and to nearest
    float up = (float)level;
    if ((double)up < level) up = nextafterf(up, INFINITY);
    float lvf[2] = {up, (float)level};
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_level, lv, sizeof(lv), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_levelf, lvf, sizeof(lvf), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_set_indicator");
    c->rowmm_valid = false;   // the row bounds belong to the transform's A
    c->solved = true;
    c->meshed = false;
    return FTR_OK;
}

int ftr_get_cube_classes(ftr_ctx* c, uint8_t* out) {
    if (!c || !out) return FTR_EINVAL;
    if (!c->solved) return set_err(c, FTR_ESTATE, "ftr_get_cube_classes: nothing solved");
    const size_t ncell = (size_t)(c->g.n[0] - 1) * (c->g.n[1] - 1) * (c->g.n[2] - 1);
    cudaError_t e;
    uint8_t* dst = out;
    uint8_t* tmp = nullptr;
    if (!is_device_ptr(out)) {
        if ((e = cudaMalloc(&tmp, ncell)) != cudaSuccess) return cuda_fail(c, e, "get_cube_classes");
        dst = tmp;
    }
    e = launch_mc_classes(c, dst);
    if (e == cudaSuccess && tmp) e = cudaMemcpyAsync(out, tmp, ncell, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_get_cube_classes");
    return FTR_OK;
}

int ftr_get_inside_mask(ftr_ctx* c, uint32_t* out) {
    if (!c || !out) return FTR_EINVAL;
    if (!c->solved) return set_err(c, FTR_ESTATE, "ftr_get_inside_mask: nothing solved");
    cudaError_t e = launch_mc_bits(c);
    const int wp = mc_words_per_row(c->g.n[0]);
    const int nw = (c->g.n[0] + 31) / 32;
    const cudaMemcpyKind kind = is_device_ptr(out) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(out, sizeof(uint32_t) * nw, c->d_mc_bits, sizeof(unsigned) * wp, sizeof(uint32_t) * nw,
                              (size_t)c->mc_blocks, kind, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_get_inside_mask");
    return FTR_OK;
}

int ftr_frame_info(ftr_ctx* c, int64_t* info, int n) {
    if (!c || !info || n < 0) return FTR_EINVAL;
    int meta[4] = {0, 0, 0, -1};
    unsigned long long dropped = 0;
    cudaError_t e = cudaMemcpyAsync(meta, c->d_meta, sizeof(meta), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&dropped, c->d_dropped, sizeof(dropped), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_frame_info");
    int zl = 0, zh = 0;
    if (meta[3] >= 0) {
        zl = (meta[2] * kBrick) & ~15;
        zh = ((meta[3] + 1) * kBrick + 15) & ~15;
    }
    int64_t pin = c->points_in;
    if (pin < 0) {
        cudaMemcpy(&pin, c->d_npts, sizeof(pin), cudaMemcpyDeviceToHost);
    }
    const int64_t v[8] = {pin, (int64_t)dropped, meta[0], meta[1], zl, zh, c->n_verts, c->n_tris};
    for (int i = 0; i < n && i < 8; ++i) info[i] = v[i];
    return FTR_OK;
}

int ftr_debug_buffer(ftr_ctx* c, int which, void* out, int64_t bytes) {
    if (!c || !out) return FTR_EINVAL;
    const void* src = nullptr;
    int64_t have = 0;
    switch (which) {
        case 0: src = c->d_s0; have = (int64_t)sizeof(float2) * 3 * c->Mh; break;
        case 1: src = c->d_s1; have = (int64_t)sizeof(float2) * 2 * c->Mh; break;
        case 2: src = c->d_raw; have = (int64_t)sizeof(float) * 7 * c->raw_cap; break;
        default: return set_err(c, FTR_EINVAL, "ftr_debug_buffer: unknown buffer %d", which);
    }
    if (!src) return set_err(c, FTR_ESTATE, "ftr_debug_buffer: buffer %d does not exist yet", which);
    if (bytes > have) return set_err(c, FTR_EINVAL, "ftr_debug_buffer: %lld > %lld bytes", (long long)bytes,
                                     (long long)have);
    cudaError_t e = cudaMemcpyAsync(out, src, (size_t)bytes, cudaMemcpyDefault, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_debug_buffer");
    return FTR_OK;
}

int ftr_debug_raise_wait_flag(ftr_ctx* c, int which) {
    if (!c) return FTR_EINVAL;
    int* flag = which == 0 ? c->d_tc_err : (which == 1 ? c->d_kerr : nullptr);
    if (!flag) return set_err(c, FTR_EINVAL, "ftr_debug_raise_wait_flag: no flag %d on this context", which);
    // the flag's lowest byte to 1: the value a kernel writes when a bounded wait gives up
    cudaError_t e = cudaMemsetAsync(flag, 1, 1, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "ftr_debug_raise_wait_flag");
    return FTR_OK;
}

int ftr_mc_table(int32_t* ntri, int32_t* tris) {
    if (!ntri || !tris) return FTR_EINVAL;
    mc_generate_table(ntri, tris);
    return FTR_OK;
}

int ftr_profile_enable(ftr_ctx* c, int on) {
    if (!c) return FTR_EINVAL;
    c->prof = on != 0;
    for (int s = 0; s < ST_COUNT; ++s) {
        c->ev_pending[s] = false;
        c->prof_ms[s] = 0.0;
        c->prof_n[s] = 0;
    }
    return FTR_OK;
}

int ftr_profile_read(ftr_ctx* c, double* ms, int64_t* counts, int max_stages) {
    if (!c) return FTR_EINVAL;
    for (int s = 0; s < ST_COUNT; ++s) {
        if (c->ev_pending[s]) {
            float t = 0.f;
            cudaEventSynchronize(c->ev_stop[s]);
            if (cudaEventElapsedTime(&t, c->ev_start[s], c->ev_stop[s]) == cudaSuccess) {
                c->prof_ms[s] += t;
                c->prof_n[s] += 1;
            }
            c->ev_pending[s] = false;
        }
    }
    for (int s = 0; s < ST_COUNT && s < max_stages; ++s) {
        if (ms) ms[s] = c->prof_ms[s];
        if (counts) counts[s] = c->prof_n[s];
        c->prof_ms[s] = 0.0;
        c->prof_n[s] = 0;
    }
    return ST_COUNT;
}

const char* ftr_stage_name(int s) {
    if (s < 0 || s >= ST_COUNT) return "";
    return kStageNames[s];
}

int64_t ftr_launch_count(const ftr_ctx* c) { return c ? c->launches : 0; }

}  // extern "C"
