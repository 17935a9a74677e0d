"""Python binding of the C ABI in include/ftr.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: all the reconstruction work runs in the CUDA kernels
of libftr.so.  Arrays may be numpy arrays (host memory) or torch tensors
(host or CUDA); they must be C-contiguous with the dtype the C ABI states.
Loading fails loudly when the library has not been built: there is no CPU
fallback.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libftr.so")

FTR_OK = 0
FTR_SPLAT_WEIGHTED = 0
FTR_SPLAT_SIMPLE = 1
FTR_PREC_FP32 = 0
FTR_PREC_BF16X3 = 1
FTR_PREC_FP16X3 = 2
FTR_ETIMEOUT = -4
MAX_TRIS_PER_CASE = 5

_lib = None


class FtrError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ftr error {code}: {msg}")
        self.code = code


class ftr_params(ctypes.Structure):
    _fields_ = [("sigma1_scale", ctypes.c_float), ("sigma2_ratio2", ctypes.c_float),
                ("splat_mode", ctypes.c_int), ("precision", ctypes.c_int), ("stream", ctypes.c_void_p)]


class ftr_mesh(ctypes.Structure):
    _fields_ = [("vertices", ctypes.c_void_p), ("normals", ctypes.c_void_p), ("tris", ctypes.c_void_p),
                ("n_vertices", ctypes.c_int64), ("n_tris", ctypes.c_int64)]


class ftr_view(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int), ("h", ctypes.c_int), ("K", ctypes.c_float * 9),
                ("world_to_cam", ctypes.c_float * 12), ("rgb_w", ctypes.c_int), ("rgb_h", ctypes.c_int),
                ("K_rgb", ctypes.c_float * 9), ("world_to_rgb", ctypes.c_float * 12),
                ("depth", ctypes.c_void_p), ("conf", ctypes.c_void_p), ("rgb", ctypes.c_void_p)]


class ftr_tex(ctypes.Structure):
    _fields_ = [("weights", ctypes.c_void_p), ("uv", ctypes.c_void_p), ("rgb", ctypes.c_void_p),
                ("textured", ctypes.c_void_p)]


class ftr_point_set(ctypes.Structure):
    _fields_ = [("points", ctypes.c_void_p), ("normals", ctypes.c_void_p), ("weights", ctypes.c_void_p),
                ("n", ctypes.c_int64)]


class ftr_camera(ctypes.Structure):
    _fields_ = [("w", ctypes.c_int), ("h", ctypes.c_int), ("K", ctypes.c_float * 9),
                ("world_to_cam", ctypes.c_float * 12)]


class ftr_render_src(ctypes.Structure):
    _fields_ = [("vertices", ctypes.c_void_p), ("tris", ctypes.c_void_p), ("n_vertices", ctypes.c_int64),
                ("n_tris", ctypes.c_int64), ("vertex_rgb", ctypes.c_void_p), ("tex_weights", ctypes.c_void_p),
                ("tex_uv", ctypes.c_void_p), ("tex_views", ctypes.POINTER(ftr_view)), ("tex_k", ctypes.c_int)]


class ftr_geometry_eval(ctypes.Structure):
    _fields_ = [("rendered_px", ctypes.c_int64), ("sensor_px", ctypes.c_int64), ("xor_px", ctypes.c_int64),
                ("or_px", ctypes.c_int64), ("vre", ctypes.c_double), ("hausdorff_px", ctypes.c_double),
                ("sensor_points", ctypes.c_int64), ("rendered_points", ctypes.c_int64),
                ("cp_rmse", ctypes.c_double)]


class ftr_appearance_eval(ctypes.Structure):
    _fields_ = [("l", ctypes.c_double * 3), ("c", ctypes.c_double * 3), ("s", ctypes.c_double * 3),
                ("wms3im", ctypes.c_double)]


# (name, restype, argtypes) of every exported symbol
_SIGNATURES = [
    ("ftr_default_params", None, [ctypes.POINTER(ftr_params)]),
    ("ftr_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_float),
                                  ctypes.POINTER(ftr_params), ctypes.POINTER(ctypes.c_void_p)]),
    ("ftr_destroy", None, [ctypes.c_void_p]),
    ("ftr_reset", ctypes.c_int, [ctypes.c_void_p]),
    ("ftr_splat", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 ctypes.c_int64]),
    ("ftr_splat_sets", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_point_set), ctypes.c_int]),
    ("ftr_splat_depth", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_view), ctypes.c_int, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    ("ftr_splat_depth_async", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_view), ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p]),
    ("ftr_solve", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    ("ftr_extract_mesh", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_mesh)]),
    ("ftr_mesh_copy", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_mesh_copy_async", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_texture", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_view), ctypes.c_int, ctypes.c_float,
                                   ctypes.POINTER(ftr_tex)]),
    ("ftr_texture_vertices", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_view), ctypes.c_int,
                                            ctypes.c_float, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ftr_tex)]),
    ("ftr_extract_mesh_async", ctypes.c_int, [ctypes.c_void_p]),
    ("ftr_texture_async", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_view), ctypes.c_int, ctypes.c_float,
                                         ctypes.POINTER(ftr_tex), ctypes.c_int64]),
    ("ftr_frame_finish", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_mesh)]),
    ("ftr_frame_launch", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_view), ctypes.c_int, ctypes.c_float,
                                        ctypes.POINTER(ftr_tex), ctypes.c_int64]),
    ("ftr_mesh_capacity", ctypes.c_int64, [ctypes.c_void_p]),
    ("ftr_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    ("ftr_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("ftr_frame_info", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("ftr_device_bytes", ctypes.c_int64, [ctypes.c_void_p]),
    ("ftr_estimate_bytes", ctypes.c_int64, [ctypes.POINTER(ctypes.c_int), ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_int64, ctypes.c_int64, ctypes.c_int]),
    ("ftr_autotune", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_get_plan", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_set_plan", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_get_mc_plan", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_set_mc_plan", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_get_transform_path", ctypes.c_int, [ctypes.c_void_p]),
    ("ftr_set_transform_path", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("ftr_get_field_V", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_get_field_A", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_set_field_V", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_set_indicator", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double]),
    ("ftr_get_cube_classes", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_get_inside_mask", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_debug_buffer", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64]),
    ("ftr_debug_raise_wait_flag", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("ftr_mc_table", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_profile_enable", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    ("ftr_profile_read", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("ftr_stage_name", ctypes.c_char_p, [ctypes.c_int]),
    ("ftr_launch_count", ctypes.c_int64, [ctypes.c_void_p]),
    ("ftr_render", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_render_src), ctypes.POINTER(ftr_camera),
                                  ctypes.c_void_p, ctypes.c_void_p]),
    ("ftr_eval_geometry", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ftr_camera), ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ftr_geometry_eval)]),
    ("ftr_eval_appearance", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ftr_appearance_eval)]),
    ("ftr_iso_level_noalloc", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                             ctypes.POINTER(ctypes.c_float), ctypes.c_void_p, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.c_void_p]),
]

EXPORTED = [s[0] for s in _SIGNATURES]


def load():
    """Load libftr.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1712_03084_gb300.build.build() "
                           "(the reconstruction has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a, dtype=None):
    """Raw address of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and a.dtype != dtype:
            raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if dtype is not None:
            want = {np.float32: "torch.float32", np.uint8: "torch.uint8", np.int32: "torch.int32"}[dtype]
            if str(a.dtype) != want:
                raise TypeError(f"expected {want}, got {a.dtype}")
        return a.data_ptr()
    if isinstance(a, int):
        return a
    raise TypeError(f"unsupported buffer type {type(a)}")


def _check(code, ctx=None):
    if code != FTR_OK:
        msg = load().ftr_last_error(ctx).decode() if ctx else ""
        raise FtrError(code, msg)


# ---------------------------------------------------------------- C-named calls

def ftr_default_params():
    p = ftr_params()
    load().ftr_default_params(ctypes.byref(p))
    return p


def ftr_create(grid_n, bbox, params=None):
    lib = load()
    g = (ctypes.c_int * 3)(*[int(v) for v in grid_n])
    b = (ctypes.c_float * 6)(*[float(v) for v in bbox])
    out = ctypes.c_void_p()
    code = lib.ftr_create(g, b, ctypes.byref(params) if params is not None else None, ctypes.byref(out))
    if code != FTR_OK:
        raise FtrError(code, "ftr_create failed (unsupported grid, bad box or no device memory)")
    return out.value


def ftr_destroy(ctx):
    load().ftr_destroy(ctx)


def ftr_reset(ctx):
    _check(load().ftr_reset(ctx), ctx)


def ftr_splat(ctx, points, normals, weights=None):
    n = int(points.shape[0])
    _check(load().ftr_splat(ctx, _ptr(points, np.float32), _ptr(normals, np.float32),
                            _ptr(weights, np.float32), n), ctx)


def ftr_splat_sets(ctx, sets):
    """sets: list of (points, normals, weights-or-None) arrays or tensors (host
    or device); one ingest launch."""
    arr = (ftr_point_set * len(sets))()
    for i, (p, n, w) in enumerate(sets):
        arr[i].points = _ptr(p, np.float32)
        arr[i].normals = _ptr(n, np.float32)
        arr[i].weights = _ptr(w, np.float32)
        arr[i].n = int(p.shape[0])
        if n.shape[0] != p.shape[0] or (w is not None and w.shape[0] != p.shape[0]):
            raise ValueError("points, normals and weights of a set must have the same length")
    _check(load().ftr_splat_sets(ctx, arr, len(sets)), ctx)


def ftr_solve(ctx, want_level=True):
    lv = ctypes.c_double(0.0)
    _check(load().ftr_solve(ctx, ctypes.byref(lv) if want_level else None), ctx)
    return lv.value if want_level else None


def ftr_extract_mesh(ctx):
    m = ftr_mesh()
    _check(load().ftr_extract_mesh(ctx, ctypes.byref(m)), ctx)
    return m


def ftr_mesh_copy(ctx, vertices=None, normals=None, tris=None):
    _check(load().ftr_mesh_copy(ctx, _ptr(vertices, np.float32), _ptr(normals, np.float32),
                                _ptr(tris, np.int32)), ctx)


def ftr_mesh_copy_async(ctx, vertices=None, normals=None, tris=None):
    _check(load().ftr_mesh_copy_async(ctx, _ptr(vertices, np.float32), _ptr(normals, np.float32),
                                      _ptr(tris, np.int32)), ctx)


def make_view(view):
    """ftr_view from a dict(depth, conf, rgb, K, world_to_cam, K_rgb, world_to_rgb)."""
    v = ftr_view()
    depth, conf, rgb = view["depth"], view.get("conf"), view.get("rgb")
    v.h, v.w = int(depth.shape[0]), int(depth.shape[1])
    if rgb is not None:
        v.rgb_h, v.rgb_w = int(rgb.shape[0]), int(rgb.shape[1])
    v.K[:] = [float(x) for x in np.asarray(view["K"], dtype=np.float32).reshape(-1)]
    v.world_to_cam[:] = [float(x) for x in np.asarray(view["world_to_cam"], dtype=np.float32).reshape(-1)]
    if "K_rgb" in view:
        v.K_rgb[:] = [float(x) for x in np.asarray(view["K_rgb"], dtype=np.float32).reshape(-1)]
        v.world_to_rgb[:] = [float(x) for x in np.asarray(view["world_to_rgb"], dtype=np.float32).reshape(-1)]
    v.depth = _ptr(depth, np.float32)
    v.conf = _ptr(conf, np.float32)
    v.rgb = _ptr(rgb, np.uint8)
    return v


def ftr_splat_depth(ctx, views, step=-1.0, noise=-1.0, radius=-1, conf_out=None, wait=True):
    """Raw reconstruction of the views' device depth maps, appended to the
    frame (wait=False: ftr_splat_depth_async, the frame's only point source)."""
    arr = (ftr_view * max(1, len(views)))(*[make_view(v) for v in views])
    confs = None
    if conf_out is not None:
        confs = (ctypes.c_void_p * len(views))(*[_ptr(c, np.float32) for c in conf_out])
    fn = load().ftr_splat_depth if wait else load().ftr_splat_depth_async
    _check(fn(ctx, arr, len(views), float(step), float(noise), int(radius), confs), ctx)


def make_camera(K, world_to_cam, w, h):
    cam = ftr_camera()
    cam.w, cam.h = int(w), int(h)
    cam.K[:] = [float(x) for x in np.asarray(K, dtype=np.float32).reshape(-1)]
    cam.world_to_cam[:] = [float(x) for x in np.asarray(world_to_cam, dtype=np.float32).reshape(-1)]
    return cam


def ftr_render(ctx, vertices, tris, camera, depth_out, rgb_out=None, vertex_rgb=None, tex_weights=None,
               tex_uv=None, tex_views=None, n_vertices=None, n_tris=None):
    """Render a device mesh into ``camera`` (an ftr_camera); all buffers are
    CUDA tensors or device addresses."""
    src = ftr_render_src()
    src.vertices = _ptr(vertices, np.float32)
    src.tris = _ptr(tris, np.int32)
    src.n_vertices = int(n_vertices if n_vertices is not None else vertices.shape[0])
    src.n_tris = int(n_tris if n_tris is not None else tris.shape[0])
    src.vertex_rgb = _ptr(vertex_rgb, np.uint8)
    keep = None
    if tex_weights is not None:
        keep = (ftr_view * len(tex_views))(*[make_view(v) for v in tex_views])
        src.tex_weights = _ptr(tex_weights, np.float32)
        src.tex_uv = _ptr(tex_uv, np.float32)
        src.tex_views = keep
        src.tex_k = len(tex_views)
    _check(load().ftr_render(ctx, ctypes.byref(src), ctypes.byref(camera), _ptr(depth_out, np.float32),
                             _ptr(rgb_out, np.uint8)), ctx)
    del keep


def ftr_eval_geometry(ctx, camera, rendered_depth, sensor_depth, cp_d2_out=None):
    out = ftr_geometry_eval()
    _check(load().ftr_eval_geometry(ctx, ctypes.byref(camera), _ptr(rendered_depth, np.float32),
                                    _ptr(sensor_depth, np.float32), _ptr(cp_d2_out, np.float32),
                                    ctypes.byref(out)), ctx)
    return {f: getattr(out, f) for f, _ in ftr_geometry_eval._fields_}


def ftr_eval_appearance(ctx, rendered_depth, rendered_rgb, sensor_rgb):
    out = ftr_appearance_eval()
    h, w = int(rendered_depth.shape[0]), int(rendered_depth.shape[1])
    _check(load().ftr_eval_appearance(ctx, w, h, _ptr(rendered_depth, np.float32), _ptr(rendered_rgb, np.uint8),
                                      _ptr(sensor_rgb, np.uint8), ctypes.byref(out)), ctx)
    return {"wms3im": out.wms3im, "l": list(out.l), "c": list(out.c), "s": list(out.s)}


def ftr_texture(ctx, views, depth_tol, weights=None, uv=None, rgb=None, textured=None):
    arr = (ftr_view * max(1, len(views)))(*[make_view(v) for v in views])
    t = ftr_tex(_ptr(weights, np.float32), _ptr(uv, np.float32), _ptr(rgb, np.uint8), _ptr(textured, np.uint8))
    _check(load().ftr_texture(ctx, arr, len(views), float(depth_tol), ctypes.byref(t)), ctx)


def ftr_texture_vertices(ctx, views, depth_tol, vertices, weights=None, uv=None, rgb=None, textured=None):
    """Per-vertex texture data of caller-given device vertices (all device buffers)."""
    arr = (ftr_view * max(1, len(views)))(*[make_view(v) for v in views])
    t = ftr_tex(_ptr(weights, np.float32), _ptr(uv, np.float32), _ptr(rgb, np.uint8), _ptr(textured, np.uint8))
    _check(load().ftr_texture_vertices(ctx, arr, len(views), float(depth_tol), _ptr(vertices, np.float32),
                                       int(vertices.shape[0]), ctypes.byref(t)), ctx)


def ftr_extract_mesh_async(ctx):
    _check(load().ftr_extract_mesh_async(ctx), ctx)


def ftr_texture_async(ctx, views, depth_tol, weights, uv, rgb, textured, out_capacity):
    arr = (ftr_view * max(1, len(views)))(*[make_view(v) for v in views])
    t = ftr_tex(_ptr(weights, np.float32), _ptr(uv, np.float32), _ptr(rgb, np.uint8), _ptr(textured, np.uint8))
    _check(load().ftr_texture_async(ctx, arr, len(views), float(depth_tol), ctypes.byref(t), int(out_capacity)), ctx)


def ftr_frame_launch(ctx, views, depth_tol, weights=None, uv=None, rgb=None, textured=None, out_capacity=0):
    arr = (ftr_view * max(1, len(views)))(*[make_view(v) for v in views])
    t = ftr_tex(_ptr(weights, np.float32), _ptr(uv, np.float32), _ptr(rgb, np.uint8), _ptr(textured, np.uint8))
    _check(load().ftr_frame_launch(ctx, arr, len(views), float(depth_tol), ctypes.byref(t), int(out_capacity)), ctx)


def ftr_frame_finish(ctx):
    """Wait for the queued frame; returns the mesh (raises FtrError on FTR_ECAPACITY too)."""
    m = ftr_mesh()
    _check(load().ftr_frame_finish(ctx, ctypes.byref(m)), ctx)
    return m


def ftr_mesh_capacity(ctx):
    return int(load().ftr_mesh_capacity(ctx))


def ftr_stats(ctx):
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().ftr_stats(ctx, ctypes.byref(a), ctypes.byref(b)), ctx)
    return a.value, b.value


FRAME_INFO_KEYS = ("points_in", "dropped", "bricks", "pairs", "z_lo", "z_hi", "n_vertices", "n_tris")


def ftr_frame_info(ctx):
    out = np.zeros(8, np.int64)
    _check(load().ftr_frame_info(ctx, out.ctypes.data, 8), ctx)
    return dict(zip(FRAME_INFO_KEYS, (int(v) for v in out)))


def ftr_device_bytes(ctx):
    return int(load().ftr_device_bytes(ctx))


def ftr_estimate_bytes(grid_n, points, depth_pixels, vertices, tris, precision=FTR_PREC_FP32):
    """Device bytes of a context at these sizes (allocates nothing)."""
    g = (ctypes.c_int * 3)(*[int(v) for v in grid_n])
    b = load().ftr_estimate_bytes(g, int(points), int(depth_pixels), int(vertices), int(tris), int(precision))
    if b < 0:
        raise FtrError(-1, "ftr_estimate_bytes: unsupported grid or negative size")
    return int(b)


def ftr_autotune(ctx):
    """Time the tile plans and the transform paths; returns the 16-float
    report of include/ftr.h ([0..11]: microseconds per launch, rows y, z,
    inverse-y passes x columns 8, 16, 32 lines per CTA and the bulk-copied
    16-line y pass; [12], [13], [15]: the five-pass, plane-fused and
    persistent y+z chains; [14]: the path kept; 0 = not timed)."""
    rep = np.zeros(16, np.float32)
    _check(load().ftr_autotune(ctx, rep.ctypes.data), ctx)
    return rep


def ftr_get_plan(ctx):
    plan = np.zeros(3, np.int32)
    _check(load().ftr_get_plan(ctx, plan.ctypes.data), ctx)
    return tuple(int(v) for v in plan)


def ftr_set_plan(ctx, plan):
    arr = np.ascontiguousarray(plan, dtype=np.int32)
    _check(load().ftr_set_plan(ctx, arr.ctypes.data), ctx)


def ftr_get_mc_plan(ctx):
    """(count/emit tile threads, triangle-pass CTAs per SM)."""
    plan = np.zeros(2, np.int32)
    _check(load().ftr_get_mc_plan(ctx, plan.ctypes.data), ctx)
    return tuple(int(v) for v in plan)


def ftr_set_mc_plan(ctx, plan):
    arr = np.ascontiguousarray(plan, dtype=np.int32)
    if arr.shape != (2,):
        raise ValueError("ftr_set_mc_plan: two ints (tile threads, triangle CTAs per SM)")
    _check(load().ftr_set_mc_plan(ctx, arr.ctypes.data), ctx)


def ftr_get_transform_path(ctx):
    """0: five axis passes, 1: plane-fused, 2: five passes with the y and z
    passes in one persistent kernel."""
    v = load().ftr_get_transform_path(ctx)
    if v < 0:
        _check(v, ctx)
    return int(v)


def ftr_set_transform_path(ctx, fused):
    _check(load().ftr_set_transform_path(ctx, int(fused)), ctx)


def ftr_last_error(ctx):
    return load().ftr_last_error(ctx).decode()


def ftr_get_field_V(ctx, out):
    _check(load().ftr_get_field_V(ctx, _ptr(out, np.float32)), ctx)


def ftr_get_field_A(ctx, out):
    _check(load().ftr_get_field_A(ctx, _ptr(out, np.float32)), ctx)


def ftr_set_field_V(ctx, V):
    _check(load().ftr_set_field_V(ctx, _ptr(V, np.float32)), ctx)


def ftr_set_indicator(ctx, A, level):
    _check(load().ftr_set_indicator(ctx, _ptr(A, np.float32), float(level)), ctx)


def ftr_get_cube_classes(ctx, out):
    _check(load().ftr_get_cube_classes(ctx, _ptr(out, np.uint8)), ctx)


def ftr_debug_buffer(ctx, which, out):
    _check(load().ftr_debug_buffer(ctx, int(which), _ptr(out), int(out.nbytes)), ctx)


def ftr_debug_raise_wait_flag(ctx, which):
    _check(load().ftr_debug_raise_wait_flag(ctx, int(which)), ctx)


def ftr_mc_table():
    ntri = np.zeros(256, np.int32)
    tris = np.zeros(256 * MAX_TRIS_PER_CASE * 3, np.int32)
    _check(load().ftr_mc_table(ntri.ctypes.data, tris.ctypes.data))
    return ntri, tris.reshape(256, MAX_TRIS_PER_CASE, 3)


def ftr_profile_enable(ctx, on=True):
    _check(load().ftr_profile_enable(ctx, 1 if on else 0), ctx)


def ftr_profile_read(ctx):
    ms = np.zeros(64, np.float64)
    cnt = np.zeros(64, np.int64)
    n = load().ftr_profile_read(ctx, ms.ctypes.data, cnt.ctypes.data, 64)
    if n < 0:
        _check(n, ctx)
    return {ftr_stage_name(s): (float(ms[s]), int(cnt[s])) for s in range(n)}


def ftr_stage_name(s):
    return load().ftr_stage_name(int(s)).decode()


def ftr_launch_count(ctx):
    return int(load().ftr_launch_count(ctx))


def ftr_iso_level_noalloc(A, grid_n, bbox, points, n=None, level_out=None, stream=None):
    """Level without device allocation (see include/ftr.h); returns L when level_out is None.

    The kernel reads ``A`` and ``points`` on the device, so both must be CUDA
    float32 tensors on one device, ``A`` with n_x n_y n_z elements and
    ``points`` with at least ``n`` rows of 3; ``level_out`` (optional) is a
    float64 numpy array or tensor with at least one element.  Anything else
    raises ValueError before the library is called."""
    g = [int(v) for v in grid_n]
    if len(g) != 3 or len(bbox) != 6:
        raise ValueError("grid_n needs 3 sizes and bbox 6 coordinates")
    for name, t in (("A", A), ("points", points)):
        if not (hasattr(t, "is_cuda") and t.is_cuda and str(t.dtype) == "torch.float32" and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA float32 tensor")
    if A.device != points.device:
        raise ValueError("A and points must be on the same device")
    if A.numel() != g[0] * g[1] * g[2]:
        raise ValueError(f"A has {A.numel()} elements, the grid {g[0] * g[1] * g[2]}")
    if points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points must be n x 3")
    n = int(points.shape[0]) if n is None else int(n)
    if not 0 <= n <= int(points.shape[0]):
        raise ValueError(f"n = {n} outside [0, {int(points.shape[0])}]")
    if level_out is None:
        out = np.zeros(1, np.float64)
    else:
        out = level_out
        if isinstance(out, np.ndarray):
            ok = out.dtype == np.float64 and out.size >= 1 and out.flags["C_CONTIGUOUS"]
        else:
            ok = (hasattr(out, "data_ptr") and str(out.dtype) == "torch.float64" and out.numel() >= 1
                  and (not out.is_cuda or out.device == A.device))
        if not ok:
            raise ValueError("level_out must hold at least one float64 (host, or on the device of A)")
    gc = (ctypes.c_int * 3)(*g)
    b = (ctypes.c_float * 6)(*[float(v) for v in bbox])
    code = load().ftr_iso_level_noalloc(A.data_ptr(), gc, b, points.data_ptr(), n, _ptr(out), stream)
    if code != FTR_OK:
        raise FtrError(code, "ftr_iso_level_noalloc failed")
    return float(out[0]) if level_out is None else None


# ---------------------------------------------------------------- convenience

class Context:
    """Owns one ftr_ctx; methods forward to the C-named calls above."""

    def __init__(self, grid_n, bbox, sigma1_scale=1.0, sigma2_ratio2=1.5, splat_mode=FTR_SPLAT_WEIGHTED,
                 stream=None, precision=FTR_PREC_FP32):
        p = ftr_default_params()
        p.sigma1_scale = sigma1_scale
        p.sigma2_ratio2 = sigma2_ratio2
        p.splat_mode = splat_mode
        p.precision = precision
        p.stream = stream
        self.grid_n = tuple(int(v) for v in grid_n)
        self.bbox = tuple(float(v) for v in bbox)
        self.h = ftr_create(self.grid_n, self.bbox, p)

    def close(self):
        if self.h:
            ftr_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def reset(self):
        ftr_reset(self.h)

    def splat(self, points, normals, weights=None):
        ftr_splat(self.h, points, normals, weights)

    def splat_sets(self, sets):
        ftr_splat_sets(self.h, sets)

    def solve(self, want_level=True):
        return ftr_solve(self.h, want_level)

    def extract_mesh(self):
        return ftr_extract_mesh(self.h)

    def mesh_numpy(self):
        m = ftr_extract_mesh(self.h)
        v = np.zeros((m.n_vertices, 3), np.float32)
        n = np.zeros((m.n_vertices, 3), np.float32)
        t = np.zeros((m.n_tris, 3), np.int32)
        ftr_mesh_copy(self.h, v, n, t)
        return {"vertices": v, "normals": n, "tris": t}

    def texture_numpy(self, views, depth_tol, n_vertices):
        k = len(views)
        w = np.zeros((n_vertices, k), np.float32)
        uv = np.zeros((n_vertices, k, 2), np.float32)
        rgb = np.zeros((n_vertices, 3), np.uint8)
        tex = np.zeros(n_vertices, np.uint8)
        ftr_texture(self.h, views, depth_tol, w, uv, rgb, tex)
        return {"weights": w, "uv": uv, "rgb": rgb, "textured": tex}

    def stats(self):
        return ftr_stats(self.h)

    def autotune(self):
        """Per-pass tile timings as 3 x 4 microseconds (the whole report is
        kept in ``tune_report``)."""
        self.tune_report = ftr_autotune(self.h)
        return self.tune_report[:12].reshape(3, 4)

    def plan(self):
        return ftr_get_plan(self.h)

    def set_plan(self, plan):
        ftr_set_plan(self.h, plan)

    def mc_plan(self):
        return ftr_get_mc_plan(self.h)

    def set_mc_plan(self, plan):
        ftr_set_mc_plan(self.h, plan)

    def transform_path(self):
        return ftr_get_transform_path(self.h)

    def set_transform_path(self, fused):
        ftr_set_transform_path(self.h, fused)

    def frame_info(self):
        return ftr_frame_info(self.h)

    def field_V(self):
        nx, ny, nz = self.grid_n
        out = np.zeros((3, nz, ny, nx), np.float32)
        ftr_get_field_V(self.h, out)
        return out

    def field_A(self):
        nx, ny, nz = self.grid_n
        out = np.zeros((nz, ny, nx), np.float32)
        ftr_get_field_A(self.h, out)
        return out

    def set_field_V(self, V):
        ftr_set_field_V(self.h, np.ascontiguousarray(V, dtype=np.float32))

    def set_indicator(self, A, level):
        ftr_set_indicator(self.h, np.ascontiguousarray(A, dtype=np.float32), level)

    def inside_mask(self):
        """Binarised volume A >= L as bool [n_z, n_y, n_x]."""
        nx, ny, nz = self.grid_n
        nw = (nx + 31) // 32
        words = np.zeros((nz, ny, nw), np.uint32)
        _check(load().ftr_get_inside_mask(self.h, words.ctypes.data), self.h)
        bits = np.unpackbits(words.view(np.uint8), axis=-1, bitorder="little")
        return bits[..., :nx].astype(bool)

    def cube_classes(self):
        nx, ny, nz = self.grid_n
        out = np.zeros((nz - 1, ny - 1, nx - 1), np.uint8)
        ftr_get_cube_classes(self.h, out)
        return out

    def profile_enable(self, on=True):
        ftr_profile_enable(self.h, on)

    def profile_read(self):
        return ftr_profile_read(self.h)

    def launch_count(self):
        return ftr_launch_count(self.h)
