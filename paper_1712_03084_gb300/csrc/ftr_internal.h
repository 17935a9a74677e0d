// Internal state and launch interfaces shared by the translation units of
// the reconstruction library.  Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ftr.h"

namespace ftr {

constexpr int kBrick = 8;                 // splat accumulation brick edge (nodes)
constexpr int kBrickVox = kBrick * kBrick * kBrick;
constexpr int kMaxViews = 8;
constexpr int kBrickScanTile = 256;   // bricks per tile of the brick-count scan (one block scan per CTA)
constexpr int kMcThreads = 256;           // CTA size of the inside-bit pass (8 grid rows, a warp each)
constexpr int kMaxTrisPerCase = 5;
constexpr int kSplatChunk = 1024;          // (point, brick) pairs per accumulation work unit

enum Stage {
    ST_INGEST = 0,
    ST_SPLAT_BIN,
    ST_SPLAT_ACC,
    ST_FX,
    ST_FY,
    ST_FZ,
    ST_IY,
    ST_IX,
    ST_LEVEL,
    ST_MC_COUNT,
    ST_MC_SCAN,
    ST_MC_EMIT,
    ST_MC_TRIS,
    ST_TEXTURE,
    ST_FXY,           // plane-fused forward x + y
    ST_IYX,           // plane-fused inverse y + x
    ST_FYZ,           // forward y + z pass (filter, inverse z) through an L2 ring
    ST_COUNT
};

// Geometry handed to kernels by value.
struct GridDev {
    int n[3];
    int nb[3];                 // bricks per axis
    double bmin[3];
    double h[3];
    double inv_h[3];
    float hf[3];
    float inv_hf[3];
    float inv_h_lo[3];         // inv_h - (float)inv_h: 1/h as a float pair (inv_hf, inv_h_lo)
    float bminf[3];
    float inv_s1sq, inv_s2sq;  // 1/sigma1^2, 1/sigma2^2 (world units)
    double v_scale;            // sigma2/sigma1 (weighted) or 1 (simple)
    float v_scale_f;           // the same in float32
    int mode;
};

// Per-point record written by the ingest kernel.
//   base: floor(t) per axis, .w = flags (bit 0 accepted, bits 1..3 round-up
//         of the nearest node per axis, i.e. floor(t + 1/2) - floor(t))
//   frac: t - floor(t) per axis, .w = W
//   nrm : N, .w unused
struct PointStore {
    int4* base = nullptr;
    float4* frac = nullptr;
    float4* nrm = nullptr;
    int64_t cap = 0;
};

struct ViewDev {
    int w, h, rgb_w, rgb_h;
    double K[9], RT[12], Krgb[9], RTrgb[12];
    float Kf[9], RTf[12], Krgbf[9], RTrgbf[12];
    const float* depth;
    const float* conf;
    const uint8_t* rgb;
};
struct ViewSet {
    int k;
    ViewDev v[kMaxViews];
};
struct EvalScratch;
}  // namespace ftr

struct ftr_ctx {
    int device = 0;
    ftr::GridDev g{};
    int64_t M = 0;             // voxels
    int64_t Mh = 0;            // half-spectrum bins (n_x/2 + 1) n_y n_z
    ftr_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;

    // points of the current frame
    ftr::PointStore pts;
    int64_t n_pts = 0;
    int64_t* d_npts = nullptr;         // the same count on the device (written by the ingest)
    int64_t points_in = 0;             // -1: the count is on the device only (ftr_splat_depth_async)
    bool depth_async = false;          // the frame's points come from ftr_splat_depth_async
    unsigned long long* d_dropped = nullptr;
    int* d_wild = nullptr;     // set when some accepted weight lies outside [0, 1]
    void* d_stage = nullptr;   // staging for host inputs
    size_t stage_cap = 0;

    // splat bricks
    int n_bricks = 0;
    int* d_brick_cnt = nullptr;
    int* d_brick_off = nullptr;
    int* d_brick_cursor = nullptr;
    int* d_brick_slot = nullptr;
    int* d_active = nullptr;
    int* d_meta = nullptr;     // [0] active bricks, [1] entries, [2] min bz, [3] max bz, [4] accumulation
                               // ticket, [5] accumulation chunks, [6] heavy bricks
    int4* d_tile = nullptr;    // per-tile sums / offsets of the brick scan (pairs, touched, chunks, heavy)
    int* d_unit_off = nullptr; // per touched brick: first accumulation chunk; [touched] = all chunks
    int* d_heavy_idx = nullptr;  // per touched brick: index of its global accumulator, -1 for one chunk
    int* d_unit_slot = nullptr;  // per accumulation chunk: its touched brick
    int64_t cap_units = 0;
    unsigned long long* d_heavy_acc = nullptr;   // 4 x 512 int64 per heavy brick (zero between frames)
    int* d_heavy_done = nullptr; // chunks finished per heavy brick (zero between frames)
    int64_t cap_heavy = 0;
    int* d_entries = nullptr;
    int64_t cap_entries = 0;
    float* d_vpool = nullptr;  // active bricks x 3 x 512 V values

    // spectra and indicator
    float2* d_s0 = nullptr;    // 3 x Mh  [kx][z][y] (five-pass path)
    float2* d_s1 = nullptr;    // 2 x Mh  [kx][ky][z] (five-pass path) or [z][kx][ky] (plane-fused path)
    float* d_A = nullptr;      // M       [z][y][x]
    float2* d_tw[3] = {nullptr, nullptr, nullptr};   // W_n^m per axis
    int plan_lines[3] = {16, 16, 16};      // lines per CTA of the y, z and inverse-y passes (-16: y pass
                                           // with bulk-copied tiles)
    int fused = 0;                         // transform path: 0 five axis passes, 1 plane-fused (x+y, z, y+x),
                                           // 2 five passes with the y and z passes in one persistent kernel
    bool fused_ok = false;                 // the plane-fused kernels exist for this grid and fit the device
    bool yz_ok = false;                    // the persistent y+z kernel exists for this grid
    float2* d_ring = nullptr;              // its ring of k_x planes (2 fields each)
    int* d_yz_sync = nullptr;              // its ticket and per-k_x tile counters
    int* occ_query = nullptr;              // set: the pass launchers report occupancy instead of launching
    unsigned char* d_tc_table = nullptr;   // split DFT matrices of the tensor-core passes
    int* d_tc_err = nullptr;               // set when a tensor-core completion wait gave up
    int* d_kerr = nullptr;                 // set when a bulk-copy completion wait gave up

    // raw reconstruction scratch (ftr_splat_depth)
    float* d_raw = nullptr;                // 7 floats per pixel capacity: P (3), N (3), W
    int64_t raw_cap = 0;                   // pixels
    int* d_raw_tiles = nullptr;            // per-tile counts / offsets
    int64_t raw_tiles_cap = 0;
    int* d_raw_total = nullptr;            // device total of the last call
    int* h_raw_total = nullptr;            // pinned copy

    // level
    double* d_level = nullptr;     // [0] L, [1] accepted count
    float* d_levelf = nullptr;     // [0] L rounded up to float32, [1] L rounded to nearest
    double* d_level_part = nullptr;
    unsigned* d_ticket = nullptr;   // last-CTA ticket of the level reduction (0 between launches)
    int level_blocks = 0;
    bool solved = false;
    bool v_external = false;   // V was set with ftr_set_field_V: solve skips the splat
    double level_host = 0.0;

    // marching cubes
    int mc_blocks = 0;             // grid rows n_y n_z
    int mc_tile = 256;             // (row, word) threads per tile of the count and emit passes: 128, 256, 512
    int mc_tris_per_sm = 4;        // CTAs per SM of the triangle pass (256 threads each, grid stride)
    int* d_mc_blk = nullptr;       // 3 x mc_blocks ints: tile and group sums of the marching-cubes count
    unsigned* d_mc_bits = nullptr; // inside bits, 32 nodes per word, rows padded to a power-of-two word count
    float2* d_rowmm = nullptr;     // per grid row (y + n_y z): min and max of A, written with A by the x inverse
    bool rowmm_valid = false;      // d_rowmm belongs to the current A (the fp32 five-pass x inverse wrote it)
    int* d_mc_off = nullptr;       // 3 x (mc_blocks + 1)
    int2* d_mc_word = nullptr;     // per (row, 32-node word) of a tile with surface: first record index, active mask
    int* h_mc_tot = nullptr;       // pinned: totals (active, verts, tris)
    int* h_flags = nullptr;        // pinned: the device wait flags (tensor-core, bulk copy) of the last frame
    int4* d_mc_nodes = nullptr;
    int64_t cap_mc_nodes = 0;
    float* d_verts = nullptr;
    float* d_vnrm = nullptr;
    int32_t* d_tris = nullptr;
    int64_t cap_verts = 0, cap_tris = 0;
    int64_t n_verts = 0, n_tris = 0;
    bool meshed = false;
    bool mesh_pending = false;     // ftr_extract_mesh_async enqueued, ftr_frame_finish not yet called
    bool tex_pending = false;      // ftr_texture_async enqueued for the pending mesh
    ftr::ViewSet tex_vs{};
    int64_t tex_capacity = 0;
    float tex_tol = 0.f;
    float* tex_w = nullptr;
    float* tex_uv = nullptr;
    uint8_t* tex_rgb = nullptr;
    uint8_t* tex_flag = nullptr;

    // texture staging (host views / outputs)
    void* d_tex_stage = nullptr;
    size_t tex_stage_cap = 0;

    // whole-frame CUDA graph (ftr_frame_launch)
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraph_t graph = nullptr;           // the captured graph graph_exec was instantiated from
    cudaGraphNode_t graph_tex_node = nullptr;   // its texture kernel node (views-only updates)
    int64_t graph_launches = 0;       // kernels per replay
    bool graph_valid = false;
    ftr::ViewSet graph_vs{};
    float graph_tol = 0.f;
    int64_t graph_cap = -1;
    void* graph_outs[4] = {nullptr, nullptr, nullptr, nullptr};

    // profiling
    bool prof = false;
    cudaEvent_t ev_start[ftr::ST_COUNT] = {};
    cudaEvent_t ev_stop[ftr::ST_COUNT] = {};
    bool ev_pending[ftr::ST_COUNT] = {};
    double prof_ms[ftr::ST_COUNT] = {};
    int64_t prof_n[ftr::ST_COUNT] = {};
    int64_t launches = 0;

    // rendering / evaluation scratch (render.cu, evaluate.cu)
    ftr::EvalScratch* ev = nullptr;
};

namespace ftr {

// Programmatic dependent launch.  Frame kernels are launched with
// launch_pdl: the launch of the next kernel in the stream may overlap the
// completion of its predecessor; every such kernel starts with pdl_wait()
// (returns once the predecessor has completed and its writes are visible; a
// no-op for a plain launch).  No kernel triggers its successor early: CTAs
// parked in the wait would hold SM resources that concurrent frames on other
// streams need.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// error helpers (api.cu)
int set_err(ftr_ctx* c, int code, const char* fmt, ...);
int cuda_fail(ftr_ctx* c, cudaError_t e, const char* what);
void prof_begin(ftr_ctx* c, int stage);
void prof_end(ftr_ctx* c, int stage);

// per translation unit one-time device setup; w96: the device table W_96^j
cudaError_t fft_fx_init(const float2* w96);
cudaError_t fft_fy_init(const float2* w96);
cudaError_t fft_fz_init(const float2* w96);
cudaError_t fft_iy_init(const float2* w96);
cudaError_t fft_ix_init(const float2* w96);
cudaError_t fft_fused_a_init(const float2* w96);
cudaError_t fft_fused_b_init(const float2* w96);
cudaError_t fft_plane_init(const float2* w96);
// W_n^m, m < n, in float64 on the device, stored float32 (twiddle.cu)
cudaError_t launch_twiddle(float2* tw, int n, cudaStream_t st);
// An axis table: W_n^m, then its copies in the order of the two twiddle steps (3 n entries).
cudaError_t launch_axis_twiddles(float2* tw, int n, cudaStream_t st);
cudaError_t mc_init();

// launchers (return cudaError_t of the launch)
cudaError_t launch_ingest(ftr_ctx* c, const float* pts, const float* nrm, const float* w, int64_t n,
                          const int* n_dev = nullptr);   // n_dev: device count, n its bound
// Point sets ingested in one launch (ftr_splat_sets): set s holds points
// off[s] .. off[s + 1] - 1 of the launch, stored from slot base on.
constexpr int kMaxSets = 16;
struct IngestSets {
    const float* pts[kMaxSets];
    const float* nrm[kMaxSets];
    const float* w[kMaxSets];
    int64_t off[kMaxSets + 1];
    int64_t base;
    int k;
};
cudaError_t launch_ingest_sets(ftr_ctx* c, const IngestSets& S);
cudaError_t launch_splat(ftr_ctx* c);          // bin + accumulate into d_vpool
cudaError_t launch_fx(ftr_ctx* c);
cudaError_t launch_fy(ftr_ctx* c);
cudaError_t launch_fz(ftr_ctx* c);
cudaError_t launch_iy(ftr_ctx* c);
cudaError_t launch_ix(ftr_ctx* c);
// plane-fused transform path (fft_plane.cu): forward x + y per z-plane, the
// z pass on plane-major fields, inverse y + x per z-plane
bool fused_available(ftr_ctx* c);
cudaError_t launch_fxy(ftr_ctx* c);
cudaError_t launch_fz2(ftr_ctx* c);
cudaError_t launch_iyx(ftr_ctx* c);
// forward y pass and z pass in one persistent kernel (fft_yz.cu)
cudaError_t fft_yz_init(const float2* w96);
bool yz_supported(const int n[3]);
int yz_ring_planes(const int n[3]);
size_t yz_ring_elems(const int n[3]);
int yz_sync_ints(const int n[3]);
cudaError_t launch_fyz(ftr_ctx* c);
cudaError_t launch_level(ftr_ctx* c);
// raw reconstruction (raw.cu): depth maps -> compacted points, normals, W
struct RawParams {
    double step, noise;      // depth-step threshold step + 3 noise z_max^2 (metres)
    float step_f, noise_f;
    int radius;              // W2 window radius
};
cudaError_t launch_raw(ftr_ctx* c, const RawParams& rp, const ftr_view* views, int k, float* const* conf_maps,
                       float* P, float* N, float* W, int* d_tile_cnt, int* d_total);
int raw_tiles(const ftr_view* views, int k);
int raw_max_radius();
// tensor-core split-precision passes (fft_tc.cu): pass 0 x fwd, 1 y fwd,
// 2 z fwd + filter + z inv, 3 y inv, 4 x inv
bool tc_supported_n(int n);
size_t tc_table_bytes();
cudaError_t tc_build_table(int precision, unsigned char* table_dev, cudaStream_t st);
cudaError_t launch_tc_pass(ftr_ctx* c, int pass);
cudaError_t tc_prepare(ftr_ctx* c);
cudaError_t launch_mc_bits(ftr_ctx* c);        // inside bits A >= L only
int mc_words_per_row(int nx);                  // padded words per grid row of the inside bits
bool mc_plan_valid(int tile, int tris_per_sm);
cudaError_t launch_mc_count(ftr_ctx* c);       // inside bits, then tile and group counts
cudaError_t launch_mc_emit(ftr_ctx* c);        // offsets and node records, then vertices and triangles
cudaError_t launch_mc_totals(ftr_ctx* c);      // totals (active, verts, tris) to h_mc_tot
cudaError_t launch_flags(ftr_ctx* c);          // device wait flags to h_flags (api.cu)
cudaError_t launch_mc_classes(ftr_ctx* c, uint8_t* out_dev);
cudaError_t launch_dense_V(ftr_ctx* c, float* out_dev);
cudaError_t launch_load_dense_V(ftr_ctx* c, const float* V_dev);

// The texture kernel instantiated for k views (the function a graph node launches).
const void* texture_kernel(int k);
cudaError_t launch_texture(ftr_ctx* c, const ViewSet& vs, float depth_tol, float* w, float* uv,
                           uint8_t* rgb, uint8_t* textured);
// Same, for nv caller-given vertices (device, nv x 3).
cudaError_t launch_texture_vertices(ftr_ctx* c, const ViewSet& vs, float depth_tol, const float* verts, int64_t nv,
                                    float* w, float* uv, uint8_t* rgb, uint8_t* textured);
// Same, for min(limit, *nv_dev) vertices with the count read on the device.
cudaError_t launch_texture_bounded(ftr_ctx* c, const ViewSet& vs, float depth_tol, int64_t limit,
                                   const int* nv_dev, float* w, float* uv, uint8_t* rgb, uint8_t* textured);

// rendering and objective evaluation (render.cu, evaluate.cu): scratch owned
// by the context, grown on demand, released by eval_free
struct EvalScratch {
    unsigned long long* zkey = nullptr;   // per pixel: (float32 z bits << 32) | triangle, ~0 = empty
    int64_t zkey_cap = 0;
    int* big = nullptr;                   // large triangles for the shared-pixel pass, then their count
    int64_t big_cap = 0;
    int* col = nullptr;                   // 2 x pixels: column distances to the sensor / rendered silhouette
    float4* pts = nullptr;                // 2 x pixels: compacted sensor and rendered points (.w = pixel)
    float* d2 = nullptr;                  // pixels: squared closest-point distance per sensor pixel
    int64_t pix_cap = 0;
    unsigned long long* cnt = nullptr;    // 8 counters (see evaluate.cu)
    double* part = nullptr;               // per-block partial sums
    int64_t part_cap = 0;
    double* h_res = nullptr;              // pinned results
    float* img = nullptr;                 // appearance planes: luma X, Y per scale
    unsigned char* mask = nullptr;        // silhouette per scale
    int64_t img_cap = 0;
};
EvalScratch* eval_scratch(ftr_ctx* c);          // created on first use; nullptr if that fails
void eval_free(ftr_ctx* c);
bool camera_ok(const ftr_camera* cam);         // 1 <= w, h <= 16384 and non-zero focal lengths

// marching-cubes table (mc_table.cpp), generated from the face rule
void mc_generate_table(int32_t ntri[256], int32_t tris[256 * kMaxTrisPerCase * 3]);

}  // namespace ftr
