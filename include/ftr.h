/*
 * ftr.h -- C ABI of the GB300 volumetric Fourier-transform reconstruction.
 *
 * The library implements, on one CUDA GPU (sm_103a), the per-frame
 * reconstruction of Section III of Alexiadis et al., "An Integrated Platform
 * for Live 3D Human Reconstruction and Motion Capturing" (IEEE TCSVT 2017,
 * arXiv 1712.03084):
 *
 *   splat oriented points into a gradient field V         (Sec. III-B, eq. 1-2)
 *   forward 3D FFT of V_x, V_y, V_z                       (Sec. III-B)
 *   integration filter F(w) = j w / |w|^2, component sum  (Sec. III-B)
 *   inverse 3D FFT -> indicator A                         (Sec. III-B)
 *   level L = mean of A at the input samples              (Sec. III-B)
 *   marching cubes on A = L -> mesh                       (Sec. III-B, [35])
 *   per-vertex visibility, weights W_k, UVs               (Sec. III-C)
 *
 * and, around it, the raw reconstruction of depth maps into oriented,
 * weighted points (Sec. III-A) and the rendering and objective evaluation
 * of a mesh against sensor views (Sec. III-E, eq. 3-7).
 *
 * Conventions shared by every entry point
 *   - Pointers marked "host or device" may point to device memory (cudaMalloc,
 *     torch CUDA tensors, managed memory) or to host memory (pinned or
 *     pageable); the library tells them apart with cudaPointerGetAttributes
 *     and stages host data through its own device buffers.  All arrays are
 *     C-contiguous float32 unless stated otherwise.
 *   - Every call is ordered on the context's stream.  Calls that return data
 *     to the host (iso_level_out, mesh counts, host output buffers) wait for
 *     the stream; the others only enqueue work.
 *   - Inputs are caller-owned and only read.  Mesh buffers are context-owned
 *     and stay valid until the next ftr_solve / ftr_reset / ftr_destroy.
 *   - Errors: a negative ftr_status, with a message from ftr_last_error().
 *     The context stays usable after FTR_EINVAL.
 *   - A context is used by one host thread at a time.
 *
 * Grid: n = (n_x, n_y, n_z), each n_c in {32, 48, 64, 96, 128, 192, 256, 384,
 * 512}; the field is indexed x-fastest (x + n_x (y + n_y z)).  Node q sits at
 * the cell centre p(q) = b_min + (q + 1/2) h with h_c = (b_max,c - b_min,c) / n_c.
 * A point is accepted iff t = (X - b_min) / h - 1/2 satisfies 1 <= t_c < n_c - 2
 * on every axis, i.e. its whole 4^3 splat stencil lies inside the grid; other
 * points are dropped and counted (not an error).
 */
#ifndef FTR_H
#define FTR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ftr_ctx ftr_ctx;

typedef enum {
    FTR_OK = 0,
    FTR_EINVAL = -1,    /* bad argument; nothing was enqueued                   */
    FTR_ENOMEM = -2,    /* device allocation failed                             */
    FTR_ECUDA = -3,     /* a CUDA call failed; the context may be unusable      */
    FTR_ETIMEOUT = -4,  /* a bounded device wait gave up (tensor-core completion) */
    FTR_ESTATE = -5,    /* call out of order (e.g. extract before solve)        */
    FTR_ECAPACITY = -6  /* caller buffers too small for the result (see ftr_frame_finish) */
} ftr_status;

enum { FTR_SPLAT_WEIGHTED = 0, FTR_SPLAT_SIMPLE = 1 };
/*
 * Arithmetic of the FFT passes.  FTR_PREC_FP32: fp32 register butterflies.
 * FTR_PREC_BF16X3 / FTR_PREC_FP16X3: every small DFT of the transforms runs
 * on the tensor cores with each operand split into two 16-bit parts (bf16 or
 * fp16) and three products accumulated in fp32; twiddles, filter and the rest
 * stay fp32.  Not in the paper (Sec. III-B uses fp32 FFTs); the split
 * variants need every grid size in {64, 128, 256, 384}.
 */
enum { FTR_PREC_FP32 = 0, FTR_PREC_BF16X3 = 1, FTR_PREC_FP16X3 = 2 };

typedef struct {
    float sigma1_scale;   /* sigma1 = scale * half voxel diagonal (Sec. III-B); default 1   */
    float sigma2_ratio2;  /* sigma2^2 / sigma1^2 (Sec. III-B: 3/2); default 1.5              */
    int splat_mode;       /* FTR_SPLAT_WEIGHTED eq.(1)(2) | FTR_SPLAT_SIMPLE nearest node   */
    int precision;        /* FTR_PREC_FP32 (default), FTR_PREC_BF16X3 or FTR_PREC_FP16X3       */
    void* stream;         /* cudaStream_t to order all work on; NULL = context-owned stream  */
} ftr_params;

/* Fill *p with the defaults above. */
void ftr_default_params(ftr_params* p);

/*
 * Create a context on the current CUDA device (Sec. III-B grid "inside the
 * foreground object's bounding box", padded by the caller against circular
 * convolution).  grid_n[3] = (n_x, n_y, n_z); bbox[6] = (min x, min y, min z,
 * max x, max y, max z) in world units, max > min.  p may be NULL (defaults).
 * Allocates every device buffer the grid needs (about 37 bytes per voxel:
 * the spectra, the indicator and the brick pool; see ftr_estimate_bytes).
 * Returns FTR_EINVAL for an unsupported grid, FTR_ENOMEM if allocation fails.
 */
int ftr_create(const int grid_n[3], const float bbox[6], const ftr_params* p, ftr_ctx** out);

/* Release every resource of the context (NULL is a no-op). */
void ftr_destroy(ftr_ctx* ctx);

/* Start a new frame: forget the points of the previous frame. */
int ftr_reset(ftr_ctx* ctx);

/*
 * Add n oriented points to the current frame (Sec. III-A/III-B: the raw
 * X_k(u), N_k(u), W_k(u) of one or more cameras; call once per camera or
 * once for all).  points, normals: n x 3 float32 (host or device);
 * weights: n float32 (host or device), or NULL for W = 1.  The points are
 * copied; the splat itself (eq. 1-2) runs in ftr_solve.  n = 0 is allowed.
 */
int ftr_splat(ftr_ctx* ctx, const float* points, const float* normals, const float* weights, int64_t n);

typedef struct {
    const float* points;   /* n x 3 float32, host or device */
    const float* normals;  /* n x 3 float32, host or device */
    const float* weights;  /* n float32, host or device, or NULL for W = 1 */
    int64_t n;
} ftr_point_set;

/*
 * The same as k calls of ftr_splat, one per set (e.g. one per camera), in
 * one kernel launch: the sets' points are appended in set order, exactly as
 * the separate calls would store them.  1 <= k <= 16.  Device arrays are
 * read in stream order (reuse them once the stream has passed this call);
 * host arrays are copied into the context's staging buffer first and the
 * call then waits for the stream.  FTR_EINVAL for k out of range, n < 0 or
 * missing points / normals, before anything is enqueued.
 */
int ftr_splat_sets(ftr_ctx* ctx, const ftr_point_set* sets, int k);

/*
 * Run the reconstruction of Sec. III-B on the points added since the last
 * ftr_reset: splat eq.(1)(2) (or the simple nearest-node splat), forward 3D
 * FFT of the three components, filter j w / |w|^2 with the components summed,
 * inverse 3D FFT into A, and L = mean of trilinear A over the accepted points
 * (0 when none).  If iso_level_out is not NULL, waits and stores L there.
 */
int ftr_solve(ftr_ctx* ctx, double* iso_level_out);

typedef struct {
    const float* vertices;   /* device, n_vertices x 3 (world units)                    */
    const float* normals;    /* device, n_vertices x 3 (unit, outward = -grad A)        */
    const int32_t* tris;     /* device, n_tris x 3 vertex ids (outward winding)          */
    int64_t n_vertices;
    int64_t n_tris;
} ftr_mesh;

/*
 * Marching cubes (Sec. III-B, [35]) on the last solved indicator at level L.
 * A vertex lies on every grid edge whose end values straddle L (inside iff
 * A >= L); vertex ids follow (node index, axis) order and triangles follow
 * cell order, so the mesh is deterministic.  Waits for the stream (the counts
 * are returned).  *out stays valid until the next solve/reset/destroy.
 * FTR_ESTATE if nothing was solved.
 */
int ftr_extract_mesh(ftr_ctx* ctx, ftr_mesh* out);

/* Copy the extracted mesh into caller buffers (host or device, any may be NULL). */
int ftr_mesh_copy(ftr_ctx* ctx, float* vertices, float* normals, int32_t* tris);

/*
 * The same copies, only enqueued on the context's stream: the data is in the
 * caller's buffers once the stream has reached them (an event or a stream
 * synchronisation).  Host destinations must be page-locked for the copies to
 * overlap other work (pageable memory makes CUDA stage them synchronously).
 * The buffers must hold n_vertices x 3 and n_tris x 3 elements of the mesh
 * that ftr_extract_mesh / ftr_frame_finish last reported.
 */
int ftr_mesh_copy_async(ftr_ctx* ctx, float* vertices, float* normals, int32_t* tris);

typedef struct {
    int w, h;                 /* depth image size                                         */
    float K[9];               /* depth intrinsics, row-major 3x3                          */
    float world_to_cam[12];   /* [R | t], row-major 3x4: x_cam = R X + t                 */
    int rgb_w, rgb_h;         /* RGB image size                                           */
    float K_rgb[9];
    float world_to_rgb[12];
    const float* depth;       /* h x w metres, 0 = background (host or device)            */
    const float* conf;        /* h x w confidence W_k (Sec. III-A) (host or device)       */
    const uint8_t* rgb;       /* rgb_h x rgb_w x 3 (host or device)                       */
} ftr_view;

/*
 * Raw reconstruction on the device (Sec. III-A), appended to the frame like
 * ftr_splat: for each of the k views (1..8; w, h, K, world_to_cam and depth
 * are read, the RGB fields are not), every foreground pixel (depth > 0)
 * that lies on a kept triangle of the organised triangulation of its depth
 * map gives the point X = R^T (x_c - t) with x_c = ((u - c_x) / f_x D,
 * (v - c_y) / f_y D, D), the normal R^T N (N = the normalised sum of the
 * camera-facing unit normals of the kept triangles containing the pixel;
 * each 2 x 2 pixel quad gives the triangles (p00, p01, p10) and
 * (p01, p11, p10), kept iff all three pixels are foreground, the largest
 * corner depth difference is <= step + 3 noise z_max^2 and the area is not
 * zero) and the confidence W = W1 W2, W1 = max(<-x_c / |x_c|, N>, 0), W2 = the
 * mean of the silhouette over a (2 radius + 1)^2 window (zero outside).
 * Points are appended in view order, row-major pixel order.  depth: device
 * memory, h x w float32 metres, 0 = background.  step, noise: metres
 * (negative = 0.03 and 0.0012); radius: 0..16 (negative = 10).  conf_out
 * (nullable; entries nullable): per view a device h x w float32 map that
 * receives W per pixel (0 where no point): the W_k of the texture stage.
 * Waits for the stream once (the point count sizes the ingest).
 */
int ftr_splat_depth(ftr_ctx* ctx, const ftr_view* views, int k, double step, double noise, int radius,
                    float* const* conf_out);

/*
 * The same without any host wait: the ingest reads the point count on the
 * device, so a whole frame (ftr_reset, this call, ftr_frame_launch) is
 * queued at once.  It must be the frame's only point source: FTR_ESTATE if
 * points were added since ftr_reset, and ftr_splat / ftr_splat_depth refuse
 * until the next ftr_reset.  ftr_stats then reads the count from the device.
 */
int ftr_splat_depth_async(ftr_ctx* ctx, const ftr_view* views, int k, double step, double noise, int radius,
                          float* const* conf_out);

typedef struct {
    float* weights;           /* n_vertices x k: W_k at the vertex, 0 if not visible       */
    float* uv;                /* n_vertices x k x 2: RGB pixel coords, (-1,-1) if w = 0    */
    uint8_t* rgb;             /* n_vertices x 3: sum_k w_k RGB_k(uv_k) / sum_k w_k         */
    uint8_t* textured;        /* n_vertices: 1 iff sum_k w_k > 0                           */
} ftr_tex;                    /* caller-owned; host or device; any member may be NULL     */

/*
 * Per-vertex texture data of Sec. III-C for the extracted mesh and k <= 8
 * views.  Vertex X is visible in camera k iff x_cam.z > 0, its nearest depth
 * pixel floor(u + 1/2), floor(v + 1/2) is inside the image and foreground
 * (D > 0), and |D - x_cam.z| <= depth_tol; its weight is W_k at that pixel,
 * set to 0 when the RGB projection falls outside the RGB image.  Projections
 * run in float32; a decision that falls inside its float32 error guard band
 * (the pixel choice, the depth test, the RGB bounds) is taken again from that
 * quantity in float64, so every decision equals the float64 one.  The blend
 * accumulates in float32; the colour is floor(c + 1/2).
 */
int ftr_texture(ftr_ctx* ctx, const ftr_view* views, int k, float depth_tol, ftr_tex* out);

/*
 * The same per-vertex texture data for caller-given vertices instead of the
 * extracted mesh: vertices n_vertices x 3 float32, the views' images and
 * every output DEVICE memory (k = 1..8).  Only enqueues.
 */
int ftr_texture_vertices(ftr_ctx* ctx, const ftr_view* views, int k, float depth_tol, const float* vertices,
                         int64_t n_vertices, ftr_tex* out);

/* ---- frames without a host wait in the middle --------------------------------
 *
 * ftr_extract_mesh and ftr_texture return counts or host data, so the host
 * waits for the GPU between them.  The three calls below enqueue the same
 * work with no wait until ftr_frame_finish, so a whole frame (splat, solve,
 * mesh, texture) is queued at once:
 *
 *   ftr_extract_mesh_async  marching cubes into the context's mesh buffers
 *                           sized by ftr_mesh_capacity() (grown from earlier
 *                           frames); nothing is written past them.
 *   ftr_texture_async       per-vertex texture data (as ftr_texture) for that
 *                           mesh; views' images and all outputs must be device
 *                           memory with room for out_capacity vertices, and
 *                           must stay valid until ftr_frame_finish.
 *   ftr_frame_finish        waits; if the mesh outgrew the buffers, grows them
 *                           and redoes the marching cubes (and the texture, if
 *                           out_capacity suffices); fills *out.  Returns
 *                           FTR_ECAPACITY, with *out valid, when the mesh has
 *                           more vertices than out_capacity (call ftr_texture
 *                           with larger outputs).
 */
int ftr_extract_mesh_async(ftr_ctx* ctx);
int ftr_texture_async(ftr_ctx* ctx, const ftr_view* views, int k, float depth_tol, ftr_tex* out,
                      int64_t out_capacity);
int ftr_frame_finish(ftr_ctx* ctx, ftr_mesh* out);
/*
 * ftr_solve + ftr_extract_mesh_async + ftr_texture_async (k = 0: no texture)
 * as one CUDA graph replay on the context stream, for the points added since
 * ftr_reset; complete it with ftr_frame_finish.  The graph is captured on the
 * first call and again whenever depth_tol, the outputs, the output capacity,
 * the number of views or a context buffer changed (a buffer grows when a
 * frame has more points or a larger mesh than any before).  When only the
 * views' image pointers or calibrations changed, the graph's texture node is
 * given the new views in place (no capture).  Same results as the separate
 * calls; does not return L (see ftr_frame_info / ftr_solve).
 */
int ftr_frame_launch(ftr_ctx* ctx, const ftr_view* views, int k, float depth_tol, ftr_tex* out,
                     int64_t out_capacity);
/* Vertex capacity of the context's mesh buffers (0 before the first mesh). */
int64_t ftr_mesh_capacity(const ftr_ctx* ctx);

/* Points added since the last reset, and how many of them were dropped. */
int ftr_stats(const ftr_ctx* ctx, int64_t* points_in, int64_t* points_dropped);

/* Facts about the current frame (waits for the stream): info[0] points in,
 * [1] dropped, [2] bricks touched by the splat, [3] (point, brick) pairs,
 * [4], [5] the slab of z-planes z_lo <= z < z_hi that can hold non-zero V
 * (the forward x/y passes work on it only), [6] vertices, [7] triangles of
 * the last mesh.  Writes min(n, 8) values. */
int ftr_frame_info(ftr_ctx* ctx, int64_t* info, int n);

/* Device memory the context holds right now, in bytes (grids, FFT workspaces,
 * brick tables, point store, mesh buffers and staging). */
int64_t ftr_device_bytes(const ftr_ctx* ctx);

/* The device bytes a context on grid_n will hold once it has run frames of
 * at most `points` oriented points (or `depth_pixels` depth pixels through
 * ftr_splat_depth*) and meshes of at most `vertices` / `tris`, with device
 * inputs (no staging), at `precision` (an FTR_PREC_* code): the same
 * accounting as ftr_device_bytes, applied to the capacities the library's
 * growth rules give at those sizes.  Allocates nothing and needs no device,
 * so a server can refuse a session before creating anything for it.  The
 * ring of transform path 2 (about 40 MB, only while that path is in use) is
 * not included.  Returns -1 for an unsupported grid or a negative size. */
int64_t ftr_estimate_bytes(const int grid_n[3], int64_t points, int64_t depth_pixels, int64_t vertices,
                           int64_t tris, int precision);

/*
 * Tile plans (no counterpart in the paper, which gives no kernel design).
 * The y, z and inverse-y FFT passes each move F lines per CTA, F in
 * {8, 16, 32}; F = -16 means 16 lines whose input tiles are fetched by bulk
 * asynchronous copies at the CTA's start: the y pass's three component
 * tiles (lines of at most 256), or the z pass's two fields, each line's
 * live z range only.  Every plan computes bit-identical results (each
 * line's arithmetic does not depend on the plan), only the speed differs.
 * The plane-fused path's z pass takes 8, 16 or 32 (-16 runs it with 16).
 *
 * ftr_autotune times each pass's candidate F on this context's grid (a few
 * launches each, on the context's own buffers, so no frame may be pending:
 * FTR_ESTATE; the last solved frame's live z-slab is used when there is one,
 * else every plane; the fields of that frame are overwritten, so solve again
 * before extracting) and keeps the fastest.  Candidates are the F that
 * divide the grid and leave at least two CTAs resident per SM (one CTA that
 * fills an SM stalls when other contexts' frames run concurrently).  The
 * choice is cached per device and grid for the process: later contexts of
 * the same grid take it without timing.  Then it times the whole forward
 * filter inverse transform chain of both transform paths (see
 * ftr_set_transform_path), each at its best tile heights, and keeps the
 * faster path (cached with the plan).  report (nullable): 16 floats,
 * [0..11] microseconds per launch of F = 8, 16, 32, -16 for the y, z and
 * inverse-y passes of the five-pass path (0 = not timed: cached or not a
 * candidate), [12], [13] and [15] microseconds of the five-pass, the
 * plane-fused and the persistent y+z chain (0: not timed), [14] the path
 * kept.  Before the transform timing, when the last frame was solved and
 * meshed, it also times the marching-cubes block sizes (ftr_set_mc_plan).
 * Waits for the stream.  Split precision contexts keep F = 16 and the five
 * passes (their passes have no variants).
 */
int ftr_autotune(ftr_ctx* ctx, float* report);

/* The plan in use: plan[0..2] = lines per CTA of the y, z and inverse-y passes. */
int ftr_get_plan(const ftr_ctx* ctx, int* plan);

/* Force a plan: each entry 8, 16 or 32 and a divisor of the axis the pass
 * tiles (n_z for the y passes, n_y for the z pass), or -16 for the y pass
 * when 16 divides n_z and n_y <= 256, or for the z pass when 16 divides
 * n_y; else FTR_EINVAL. */
int ftr_set_plan(ftr_ctx* ctx, const int* plan);

/*
 * Marching-cubes block sizes (Sec. III-B, marching cubes [35]; the sizes are
 * this library's, the paper names none): plan[0] = (row, 32-node word)
 * threads per tile of the count and emit passes (128, 256 or 512), plan[1] =
 * CTAs per SM of the triangle pass (1 to 16, 256 threads each, grid stride).
 * Every choice gives the same mesh bit for bit: node records, vertex ids and
 * triangles follow node order, not the tiling.  Defaults 256 and 4;
 * ftr_autotune times 128/256/512 x 2/4/8 on the last frame's indicator and
 * level when that frame was solved and meshed and the grid's plans are not
 * cached yet, and keeps the fastest (cached with the tile plan).  Set:
 * FTR_EINVAL outside those ranges, FTR_ESTATE while a frame is pending; the
 * next extraction uses it.
 */
int ftr_get_mc_plan(const ftr_ctx* ctx, int* plan);
int ftr_set_mc_plan(ftr_ctx* ctx, const int* plan);

/*
 * Transform path of the FP32 transforms: 0 = five axis passes, 1 =
 * plane-fused, 2 = the five passes with the forward y pass and the z pass
 * (filter, inverse z) in one persistent kernel whose y tiles hand each k_x
 * plane to its z tiles through a ring of k_x planes that stays in L2
 * (about 40 MB; grids with n_y = n_z in {64, 96, 128, 192, 256, 384}; the
 * per-line arithmetic of path 0 with 16-line y and z tiles, equal to it
 * within rounding).  The plane-fused path runs the forward x and y transforms of a
 * z-plane in one kernel (a thread-block cluster per plane: each CTA
 * transforms its rows along x into its shared memory, then its k_x columns
 * along y, reading every y from the cluster's shared memory), the z pass with
 * the filter and the inverse z transform, and the inverse y and x transforms
 * of a z-plane in one kernel the same way: the half spectrum moves through
 * HBM twice per frame instead of four times.  It exists for the cubic grids
 * 32 ... 384 and the elongated grids 32 x 64, 64 x 128, 128 x 256, 48 x 96,
 * 384 x 48, 192 x 48, 32 x 384, 32 x 192, 48 x 32 (n_x x n_y) where its
 * clusters fit the device.  A context starts on the five-pass path;
 * ftr_autotune times both and keeps the faster (on a GB300 at 256^3 the
 * five passes: each plane's CTAs wait on one another at every cluster
 * barrier, where the independent tiles of the axis passes overlap).
 * The z-pass plan (plan[1]) applies to both paths; plan[0] and plan[2] only
 * to the five-pass path.  The paths agree within rounding (A rel-L2 ~1e-7),
 * not bit for bit (the x transforms pair other rows).  Set: FTR_EINVAL if 1
 * is asked where the fused kernels do not exist (2 likewise), FTR_ESTATE
 * while a frame is pending; the next solve uses it.  The ring of path 2 is
 * allocated when the path is set (FTR_ENOMEM if it does not fit) and freed
 * when another is set; ftr_autotune allocates it to time the path and frees
 * it unless the path is kept.  ftr_device_bytes counts it while it exists;
 * ftr_estimate_bytes does not.  Get: the path (or FTR_EINVAL).
 */
int ftr_get_transform_path(const ftr_ctx* ctx);
int ftr_set_transform_path(ftr_ctx* ctx, int fused);

/* Message of the last error on this context (never NULL). */
const char* ftr_last_error(const ftr_ctx* ctx);

/* ---- inspection hooks used by the tests and the benchmark ------------------ */

/* Dense V (3 x n_z x n_y x n_x float32, component-major) of the last solve. */
int ftr_get_field_V(ftr_ctx* ctx, float* out);
/* Replace the splat: the next ftr_solve transforms this dense V (3 x n_z x n_y
 * x n_x float32, host or device) instead of splatting points; L is then 0
 * (no samples).  Cleared by ftr_reset. */
int ftr_set_field_V(ftr_ctx* ctx, const float* V);
/* Indicator A (n_z x n_y x n_x float32) of the last solve. */
int ftr_get_field_A(ftr_ctx* ctx, float* out);
/* Replace A and L (e.g. with another implementation's) before ftr_extract_mesh. */
int ftr_set_indicator(ftr_ctx* ctx, const float* A, double level);
/*
 * The binarised volume of the last solve (Sec. IV feeds it to the skeleton
 * extraction): bit = 1 iff A >= L (the marching-cubes inside test).  Layout:
 * grid row r = y + n_y z holds ceil(n_x / 32) words, bit i of word w is node
 * x = 32 w + i (bits past n_x are 0); out (host or device) holds
 * n_y n_z ceil(n_x / 32) words.  FTR_ESTATE before a solve.  Waits.
 */
int ftr_get_inside_mask(ftr_ctx* ctx, uint32_t* out);
/* Cube class (uint8) per cell, (n_z-1) x (n_y-1) x (n_x-1), of the current A, L. */
int ftr_get_cube_classes(ftr_ctx* ctx, uint8_t* out);
/* Raw copy of an internal buffer (first `bytes` bytes; waits): which = 0 the
 * x-pass / inverse-y buffer of the five-pass transforms (3 x (n_x/2+1) n_y
 * n_z complex64), which = 1 the buffer of the two fields the z pass reads (2
 * x (n_x/2+1) n_y n_z complex64; layout [k_x][k_y][z] on the five-pass
 * path, [z][k_x][k_y] on the plane-fused one, field 0 overwritten by the
 * filtered, inverse-z transformed spectrum), both after ftr_solve; which = 2 the output of the last ftr_splat_depth call over P
 * depth pixels in all: points (3 P float32), normals (3 P) and W (P), each
 * array's first (point count) entries valid, in pixel order (FTR_ESTATE
 * before the first such call). */
int ftr_debug_buffer(ftr_ctx* ctx, int which, void* out, int64_t bytes);
/* Raise, on the stream, the device flag a kernel sets when one of its bounded
 * waits gives up (which = 0: the tensor-core completion wait of the split
 * precision passes, 1: the bulk-copy wait of the y pass), as if a wait had
 * timed out: the next call that reads the flags (ftr_solve with a level
 * output, ftr_extract_mesh, ftr_frame_finish) returns FTR_ETIMEOUT and
 * clears them; the context stays usable.  For tests of that error path
 * without making a GPU wait run out.  FTR_EINVAL if the context has no such
 * flag (which = 0 on an FP32 context). */
int ftr_debug_raise_wait_flag(ftr_ctx* ctx, int which);
/* The generated marching-cubes table: ntri[256] and tris[256 * 5 * 3] (-1 padded). */
int ftr_mc_table(int32_t* ntri, int32_t* tris);
/* Per-stage device time accounting (CUDA events on the context stream). */
int ftr_profile_enable(ftr_ctx* ctx, int on);
/* Accumulated ms and launch counts per stage since the last read; returns #stages. */
int ftr_profile_read(ftr_ctx* ctx, double* ms, int64_t* counts, int max_stages);
const char* ftr_stage_name(int stage);
/* Number of kernels this context has launched so far. */
int64_t ftr_launch_count(const ftr_ctx* ctx);

/* ---- rendering and objective evaluation (Sec. III-C, III-E) ------------------
 *
 * Sec. III-E scores a reconstruction by projecting the mesh into the K + K'
 * sensor views (K used by the reconstruction, K' held out) and comparing the
 * rendered depth and colour with what each sensor captured.  Every pointer
 * in this section is DEVICE memory; the render only enqueues, the two
 * evaluations wait for the stream and return host values.
 */

typedef struct {
    int w, h;                 /* image size, pixels                                       */
    float K[9];               /* intrinsics, row-major 3x3                                */
    float world_to_cam[12];   /* [R | t], row-major 3x4: x_cam = R X + t                 */
} ftr_camera;

typedef struct {
    const float* vertices;    /* n_vertices x 3 world coordinates                         */
    const int32_t* tris;      /* n_tris x 3 vertex indices (each < n_vertices)            */
    int64_t n_vertices, n_tris;
    /* colour source: at most one of vertex_rgb / tex_weights (both NULL = depth only)    */
    const uint8_t* vertex_rgb;  /* n_vertices x 3: colour-per-vertex rendering             */
    const float* tex_weights;   /* n_vertices x tex_k: W_k per vertex (ftr_tex.weights)    */
    const float* tex_uv;        /* n_vertices x tex_k x 2: RGB pixel coords (ftr_tex.uv)   */
    const ftr_view* tex_views;  /* tex_k views: only rgb_w, rgb_h and rgb are read         */
    int tex_k;                  /* 1..8 with tex_weights                                    */
} ftr_render_src;

/*
 * Render a triangle mesh into a pinhole camera (the depth and colour buffers
 * of Sec. III-E; the multitexture blend of Sec. III-C).  Pixel (i, j) samples
 * the image point (i, j).  A triangle is drawn unless a vertex has camera
 * z < 0.01 or its screen area is 0; a pixel is covered iff its three edge
 * functions have one sign (edges belong to both neighbours; no culling).
 * The depth is the camera z where the pixel's ray meets the triangle's
 * plane; the nearest surface wins (smallest (float32 z, triangle index)).
 * Projection, coverage and depth are evaluated in float64 in a fixed
 * operation order, so the drawn set and the depth are deterministic.
 * depth_out: h x w float32, 0 where nothing is drawn.  rgb_out: h x w x 3
 * u8 or NULL; with vertex_rgb the perspective-correct barycentric mean of
 * the vertex colours; with tex_weights the blend sum_k w_k RGB_k(uv_k) /
 * sum_k w_k over the views weighted at all three vertices, w_k and uv_k
 * interpolated across the triangle, RGB_k sampled bilinearly (clamped);
 * floor(c + 1/2), black where nothing is drawn or no view applies.
 * Returns FTR_EINVAL for bad sizes, host pointers, n_tris >= 2^31 or a
 * colour source without rgb_out.  Triangle indices are checked on the device:
 * a triangle with an index outside [0, n_vertices) is not drawn.
 */
int ftr_render(ftr_ctx* ctx, const ftr_render_src* src, const ftr_camera* cam, float* depth_out,
               uint8_t* rgb_out);

typedef struct {
    int64_t rendered_px;      /* |S_r|: pixels with rendered depth > 0                    */
    int64_t sensor_px;        /* |S_g|: pixels with sensor depth > 0                      */
    int64_t xor_px, or_px;    /* |S_r xor S_g|, |S_r or S_g|                              */
    double vre;               /* eq. (3): xor / or (0 when both are empty)                */
    double hausdorff_px;      /* eq. (4): symmetric 2D Hausdorff distance, pixels;
                                 0 when both are empty, +inf when one is                  */
    int64_t sensor_points;    /* I_k                                                       */
    int64_t rendered_points;  /* J_k                                                       */
    double cp_rmse;           /* eq. (5), depth units; nan if I_k = 0, +inf if J_k = 0    */
} ftr_geometry_eval;

/*
 * Volume and geometry metrics of Sec. III-E (eq. (3)-(5)) for one view:
 * rendered_depth (ftr_render of the mesh into cam) against sensor_depth,
 * both h x w float32 (0 = background).  The points of eq. (5) are the
 * back-projections X = z (dx, dy, 1), dy = (j - K12)/K11,
 * dx = ((i - K02) - K01 dy)/K00, of the foreground pixels (camera
 * coordinates).  cp_d2_out (nullable): h x w float32 receiving, per sensor
 * pixel, the squared distance to the closest rendered point (+inf without
 * rendered points), 0 elsewhere.  Counts and the Hausdorff distance are
 * exact; the closest-point distances are float32, their mean is summed in
 * float64 in a fixed order (deterministic).  Waits for the stream.
 */
int ftr_eval_geometry(ftr_ctx* ctx, const ftr_camera* cam, const float* rendered_depth, const float* sensor_depth,
                      float* cp_d2_out, ftr_geometry_eval* out);

typedef struct {
    double l[3], c[3], s[3];  /* weighted means of the SSIM terms per scale, eq. (7)      */
    double wms3im;            /* prod_j l_j^a_j c_j^b_j s_j^g_j                           */
} ftr_appearance_eval;

/*
 * Appearance metric of Sec. III-E3 (eq. (6)(7)): WMS3IM between a rendered
 * colour image and the sensor's, over the rendered silhouette S_r
 * (rendered_depth > 0), at J = 3 scales with exponents a = (0, 0, 0.1333),
 * b = g = (0.0448, 0.3001, 0.1333).  Luma Y = 0.299 R + 0.587 G + 0.114 B;
 * N(u) = the 11 x 11 window with Gaussian weights (sigma 1.5 pixels per
 * axis) cut at the image border and renormalised; C1 = (0.01 * 255)^2,
 * C2 = (0.03 * 255)^2, C3 = C2 / 2; s = (sigma_XY + C3) / (sigma_X sigma_Y
 * + C3); w(u) = silhouette pixels in the cut 11 x 11 window.  Scale j + 1
 * is the 2 x 2 block mean (silhouette: block AND), floor(n / 2) pixels.
 * A weighted mean <= 0 contributes 0 to the product; without silhouette
 * pixels at some scale every field is nan.  Images h x w x 3 u8,
 * rendered_depth h x w float32, w, h >= 1.  Waits for the stream.
 */
int ftr_eval_appearance(ftr_ctx* ctx, int w, int h, const float* rendered_depth, const uint8_t* rendered_rgb,
                        const uint8_t* sensor_rgb, ftr_appearance_eval* out);

/* ---- allocation-free variant ------------------------------------------------ */

/*
 * Iso-level L = mean over the accepted points of trilinear A, without any
 * device allocation.  Every point gets the same accept / reject decision as
 * in ftr_solve (both follow the float64 quotient (X - b_min) / h - 1/2), and
 * the value matches ftr_solve's level within |dL| / (max A - min A) <= 1e-5,
 * but it is not bit-identical: the fractions are rounded from float64 rather
 * than through the ingest's float pair, and the partial sums are reduced in
 * a different tree (1024 points per CTA, then one warp).  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory where they need the level -- a per-frame loop with a hard
 * latency budget (cudaMalloc/cudaFree may synchronise the device), or a host
 * framework that owns every allocation and gives the library none.
 *
 * A: n_z x n_y x n_x float32 indicator (device); grid_n, bbox as in
 * ftr_create; points: n x 3 float32 (device); level_out: one double, host or
 * device (a host pointer makes the call wait for the stream, so with a host
 * level_out on a stream that is being captured the call returns FTR_EINVAL
 * and enqueues nothing); stream: the cudaStream_t to use, NULL = the default
 * stream.  Needs no context.
 *
 * Scratch: a static 64 KB device array inside the library (one per device
 * that loads it, kept until the process exits), so n is limited to
 * 4,194,304 points; larger n returns FTR_EINVAL before any work.  The first
 * call on each device looks up that array's device address; make that first
 * call before any stream capture.  All calls share the array: calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race and must be serialised by the caller.  Every scratch slot a call reads
 * is written by that call first, so nothing needs clearing between calls.
 * Returns FTR_EINVAL for bad arguments, FTR_ECUDA if a CUDA call fails.
 */
int ftr_iso_level_noalloc(const float* A, const int grid_n[3], const float bbox[6], const float* points,
                          int64_t n, double* level_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FTR_H */
