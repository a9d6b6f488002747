"""ctypes binding of libhyrf (include/hyrf.h): same call names, argument
marshalling only. Tensors are torch CUDA tensors; every call is enqueued on
the current torch stream (or `stream`). The library is loaded from this
package directory; importing this module on a machine without it, or
without CUDA, raises.
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhyrf.so")

HYRF_OK = 0
HYRF_ERR_INVALID_ARG = 1
HYRF_ERR_UNSUPPORTED = 2
HYRF_ERR_CUDA = 4
HYRF_ERR_OVERFLOW = 8
HYRF_ERR_BOUNDS = 16
HYRF_ERR_TIMEOUT = 32
HYRF_F32 = 0
HYRF_BF16 = 1
HYRF_U8 = 2
HYRF_F16 = 3
TILE = 16

_vp = C.c_void_p


class hyrf_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("z_near", C.c_float), ("cull_tol", C.c_float)]


class hyrf_grid(C.Structure):
    _fields_ = [("table", _vp), ("n_levels", C.c_int32), ("log2_T", C.c_int32),
                ("n_feat", C.c_int32), ("base_res", C.c_int32), ("growth", C.c_float),
                ("dtype", C.c_int32), ("qparams", _vp)]


class hyrf_mlp(C.Structure):
    _fields_ = [("W", _vp * 3), ("b", _vp * 3), ("n_in", C.c_int32), ("width", C.c_int32),
                ("n_hidden", C.c_int32), ("n_out", C.c_int32), ("dtype", C.c_int32)]


class hyrf_fields(C.Structure):
    _fields_ = [("box_lo", C.c_float * 3), ("box_hi", C.c_float * 3), ("geo", hyrf_grid),
                ("rad", hyrf_grid), ("geo_mlp", hyrf_mlp), ("col_mlp", hyrf_mlp),
                ("pe_freq", C.c_int32), ("pe_pad", C.c_int32)]


class hyrf_field_grads(C.Structure):
    _fields_ = [("geo_table", _vp), ("rad_table", _vp), ("geo_W", _vp * 3), ("geo_b", _vp * 3),
                ("col_W", _vp * 3), ("col_b", _vp * 3)]


class hyrf_query_fields_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", _vp), ("alpha_e", _vp), ("scale_e", _vp),
                ("color_e", _vp), ("cam", hyrf_camera), ("fields", hyrf_fields),
                ("vis_ids", _vp), ("n_vis", _vp), ("alpha", _vp), ("scale", _vp), ("quat", _vp),
                ("color", _vp), ("status", _vp), ("features", _vp), ("explicit_only", C.c_int32),
                ("vis_ready", C.c_int32)]


class hyrf_precull_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", _vp), ("cam", hyrf_camera), ("vis_ids", _vp), ("n_vis", _vp)]


class hyrf_query_fields_backward_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", _vp), ("alpha_e", _vp), ("scale_e", _vp),
                ("color_e", _vp), ("cam", hyrf_camera), ("fields", hyrf_fields),
                ("vis_ids", _vp), ("n_vis", _vp), ("d_alpha", _vp), ("d_scale", _vp),
                ("d_quat", _vp), ("d_color", _vp), ("d_pos", _vp), ("d_alpha_e", _vp),
                ("d_scale_e", _vp), ("d_color_e", _vp), ("grads", hyrf_field_grads),
                ("loss_scale", C.c_float), ("status", _vp), ("features", _vp), ("explicit_only", C.c_int32)]


class hyrf_project_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", _vp), ("vis_ids", _vp), ("n_vis", _vp), ("scale", _vp),
                ("quat", _vp), ("cam", hyrf_camera), ("tile", C.c_int32), ("mean2d", _vp),
                ("conic", _vp), ("depth", _vp), ("rect", _vp), ("ntiles", _vp),
                ("fp64_flag", _vp), ("status", _vp), ("alpha", _vp), ("footprint", _vp)]


class hyrf_project_backward_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", _vp), ("vis_ids", _vp), ("n_vis", _vp), ("scale", _vp),
                ("quat", _vp), ("cam", hyrf_camera), ("d_mean2d", _vp), ("d_conic", _vp),
                ("d_pos", _vp), ("d_scale", _vp), ("d_quat", _vp), ("status", _vp)]


class hyrf_bin_sort_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_vis", _vp), ("rect", _vp), ("ntiles", _vp), ("depth", _vp),
                ("tiles_x", C.c_int32), ("tiles_y", C.c_int32), ("capacity", C.c_int64),
                ("keys", _vp), ("vals", _vp), ("ranges", _vp), ("n_instances", _vp),
                ("status", _vp), ("depth_order", _vp), ("mean2d", _vp), ("footprint", _vp)]


class hyrf_depth_order_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", _vp), ("vis_ids", _vp), ("n_vis", _vp), ("cam", hyrf_camera),
                ("order", _vp), ("status", _vp)]


class hyrf_rasterize_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("n_vis", _vp), ("ranges", _vp), ("vals", _vp), ("mean2d", _vp),
                ("conic", _vp), ("alpha", _vp), ("color", _vp), ("width", C.c_int32),
                ("height", C.c_int32), ("tile", C.c_int32), ("C_fg", _vp), ("T_final", _vp),
                ("n_contrib", _vp), ("status", _vp), ("tile_order", _vp), ("records", _vp)]


class hyrf_tile_order_args(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("tile", C.c_int32), ("n_contrib", _vp),
                ("order", _vp)]


class hyrf_rasterize_backward_args(C.Structure):
    _fields_ = [("fwd", hyrf_rasterize_args), ("d_C_fg", _vp), ("d_T_final", _vp),
                ("d_mean2d", _vp), ("d_conic", _vp), ("d_alpha", _vp), ("d_color", _vp), ("C", _vp)]


class hyrf_background(C.Structure):
    _fields_ = [("mode", C.c_int32), ("map_h", C.c_int32), ("map_w", C.c_int32),
                ("radius", C.c_float), ("tau_T", C.c_float)]


class hyrf_composite_background_args(C.Structure):
    _fields_ = [("cam", hyrf_camera), ("fields", hyrf_fields), ("bg", hyrf_background),
                ("C_fg", _vp), ("T_final", _vp), ("C", _vp), ("status", _vp), ("features", _vp),
                ("features_ready", C.c_int32)]


class hyrf_composite_background_backward_args(C.Structure):
    _fields_ = [("fwd", hyrf_composite_background_args), ("d_C", _vp), ("d_C_fg", _vp),
                ("d_T_final", _vp), ("grads", hyrf_field_grads), ("loss_scale", C.c_float),
                ("scatter_stream", _vp)]


class hyrf_loss_args(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("C", _vp), ("target", _vp),
                ("lambda_", C.c_float), ("grad_scale", C.c_float), ("loss", _vp), ("d_C", _vp)]


class hyrf_densify_stats_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("vis_ids", _vp), ("n_vis", _vp), ("d_mean2d", _vp), ("ntiles", _vp),
                ("width", C.c_int32), ("height", C.c_int32), ("accum", _vp), ("count", _vp)]


class hyrf_densify_plan_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("vis_ids", _vp), ("n_vis", _vp), ("alpha", _vp), ("scale", _vp),
                ("accum", _vp), ("count", _vp), ("grad_threshold", C.c_float), ("dense_scale", C.c_float),
                ("min_opacity", C.c_float), ("action", _vp), ("row", _vp), ("offset", _vp), ("n_out", _vp)]


class hyrf_remap_array(C.Structure):
    _fields_ = [("src", _vp), ("dst", _vp), ("width", C.c_int32), ("kind", C.c_int32)]


REMAP_MAX = 24
DENSIFY_KEEP, DENSIFY_PRUNE, DENSIFY_CLONE, DENSIFY_SPLIT = 0, 1, 2, 3
REMAP_PARAM, REMAP_STATE, REMAP_POSITION, REMAP_SCALE_LOGIT = 0, 1, 2, 3


class hyrf_densify_apply_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("action", _vp), ("row", _vp), ("offset", _vp), ("scale", _vp),
                ("quat", _vp), ("noise", _vp), ("split_log_scale", C.c_float), ("n_arrays", C.c_int32),
                ("arrays", hyrf_remap_array * REMAP_MAX)]


class hyrf_spatial_order_args(C.Structure):
    _fields_ = [("n", C.c_int32), ("pos", _vp), ("box_lo", C.c_float * 3), ("box_hi", C.c_float * 3),
                ("perm", _vp)]


_ARGS = {
    "hyrf_spatial_order": hyrf_spatial_order_args,
    "hyrf_densify_plan": hyrf_densify_plan_args,
    "hyrf_query_fields": hyrf_query_fields_args,
    "hyrf_query_fields_backward": hyrf_query_fields_backward_args,
    "hyrf_project": hyrf_project_args,
    "hyrf_project_backward": hyrf_project_backward_args,
    "hyrf_bin_sort": hyrf_bin_sort_args,
    "hyrf_bin_sort_backward": hyrf_bin_sort_args,
    "hyrf_rasterize": hyrf_rasterize_args,
    "hyrf_rasterize_backward": hyrf_rasterize_backward_args,
    "hyrf_tile_order": hyrf_tile_order_args,
    "hyrf_precull": hyrf_precull_args,
    "hyrf_depth_order": hyrf_depth_order_args,
    "hyrf_composite_background": hyrf_composite_background_args,
    "hyrf_composite_background_backward": hyrf_composite_background_backward_args,
    "hyrf_loss": hyrf_loss_args,
}
_WS = {k: (k + "_workspace_size") for k in _ARGS if k != "hyrf_bin_sort_backward"}
_WS["hyrf_bin_sort_backward"] = None

_lib = None


class HyrfError(RuntimeError):
    pass


def lib():
    """Load libhyrf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise HyrfError(f"{LIB_PATH} is missing: build it with paper_2509_17083_gb300/build.py")
        L = C.CDLL(LIB_PATH)
        for name, st in _ARGS.items():
            fn = getattr(L, name)
            fn.argtypes = [C.POINTER(st), _vp, C.c_size_t, _vp]
            fn.restype = C.c_int32
            ws = _WS.get(name)
            if ws:
                f = getattr(L, ws)
                f.argtypes = [C.POINTER(st)]
                f.restype = C.c_size_t
        L.hyrf_read_status.argtypes = [_vp, _vp, C.POINTER(C.c_int32)]
        L.hyrf_read_status.restype = C.c_int32
        L.hyrf_error_string.argtypes = [C.c_int32]
        L.hyrf_error_string.restype = C.c_char_p
        L.hyrf_densify_stats.argtypes = [C.POINTER(hyrf_densify_stats_args), _vp]
        L.hyrf_densify_stats.restype = C.c_int32
        L.hyrf_densify_apply.argtypes = [C.POINTER(hyrf_densify_apply_args), _vp]
        L.hyrf_densify_apply.restype = C.c_int32
        L.hyrf_gather_background.argtypes = [C.POINTER(hyrf_composite_background_args), _vp]
        L.hyrf_gather_background.restype = C.c_int32
        L.hyrf_permute_rows.argtypes = [_vp, C.c_int32, C.POINTER(hyrf_remap_array), C.c_int32, _vp]
        L.hyrf_permute_rows.restype = C.c_int32
        L.hyrf_quantize_grid.argtypes = [_vp, C.c_int32, C.c_int32, C.c_int32, _vp, _vp, _vp]
        L.hyrf_quantize_grid.restype = C.c_int32
        L.hyrf_reset_opacity.argtypes = [_vp, C.c_int64, C.c_float, _vp, _vp, _vp]
        L.hyrf_reset_opacity.restype = C.c_int32
        L.hyrf_bin_sort_noalloc.argtypes = [C.POINTER(hyrf_bin_sort_args), _vp]
        L.hyrf_bin_sort_noalloc.restype = C.c_int32
        L.hyrf_launch_count.argtypes = []
        L.hyrf_launch_count.restype = C.c_uint64
        L.hyrf_adam_step.argtypes = [C.POINTER(hyrf_adam_tensor), C.c_int32, C.POINTER(hyrf_adam_hparams), _vp]
        L.hyrf_adam_step.restype = C.c_int32
        L.hyrf_timer_enable.argtypes = [C.c_int]
        L.hyrf_timer_enable.restype = None
        L.hyrf_timer_read.argtypes = [C.POINTER(hyrf_kernel_time), C.c_int]
        L.hyrf_timer_read.restype = C.c_int
        L.hyrf_check_bounded_wait.argtypes = [_vp, C.c_uint32, _vp]
        L.hyrf_check_bounded_wait.restype = C.c_int32
        _lib = L
    return _lib


EXPORTED = list(_ARGS) + [k + "_workspace_size" for k in _ARGS if k != "hyrf_bin_sort_backward"] + [
    "hyrf_read_status", "hyrf_error_string", "hyrf_launch_count", "hyrf_bin_sort_noalloc"]
NOALLOC_MAX_GAUSSIANS = 65536
NOALLOC_MAX_INSTANCES = 262144


def ptr(t):
    """Device address of a tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise HyrfError("tensor must be contiguous")
    return t.data_ptr()


def stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Workspace:
    """Grow-only device scratch buffer handed to the library as `workspace`."""

    def __init__(self, device="cuda"):
        self.device = device
        self.buf = None

    def get(self, nbytes):
        if nbytes == 0:
            return None, 0
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        return self.buf.data_ptr(), self.buf.numel()


def call(name, args, ws: Workspace = None, stream=None):
    """Invoke hyrf_<name>(&args, workspace, bytes, stream); raise on a host-side error."""
    L = lib()
    size_fn = _WS.get(name)
    need = getattr(L, size_fn)(C.byref(args)) if size_fn else 0
    if need and ws is None:
        ws = Workspace()
    wp, wb = ws.get(need) if need else (None, 0)
    st = getattr(L, name)(C.byref(args), wp, wb, stream_handle(stream))
    if st != HYRF_OK:
        raise HyrfError(f"{name}: {L.hyrf_error_string(st).decode()} ({st})")
    return st


def read_status(status, stream=None):
    out = C.c_int32(0)
    lib().hyrf_read_status(ptr(status), stream_handle(stream), C.byref(out))
    return out.value


def error_string(st):
    return lib().hyrf_error_string(st).decode()


def hyrf_check_bounded_wait(status, polls, stream=None):
    """One CTA's bounded wait on a barrier nothing completes (sets
    HYRF_ERR_TIMEOUT in the device status word after `polls` polls)."""
    _check("hyrf_check_bounded_wait",
           lib().hyrf_check_bounded_wait(ptr(status), int(polls), stream_handle(stream)))


def launch_count():
    return int(lib().hyrf_launch_count())


class hyrf_adam_tensor(C.Structure):
    _fields_ = [("param", _vp), ("grad", _vp), ("m", _vp), ("v", _vp), ("shadow", _vp),
                ("n", C.c_int64), ("lr_scale", C.c_float)]


class hyrf_adam_hparams(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("step", C.c_int32), ("grad_scale", C.c_float)]


ADAM_MAX_TENSORS = 32


def hyrf_adam_step(tensors, lr, beta1, beta2, eps, step, grad_scale=1.0, stream=None):
    """One fused Adam step. tensors: list of dicts with param, grad, m, v
    (float32 tensors of equal size), optional shadow (bfloat16) and lr_scale."""
    L = lib()
    for c0 in range(0, len(tensors), ADAM_MAX_TENSORS):
        chunk = tensors[c0:c0 + ADAM_MAX_TENSORS]
        arr = (hyrf_adam_tensor * len(chunk))()
        for d, t in zip(arr, chunk):
            d.param, d.grad, d.m, d.v = ptr(t["param"]), ptr(t["grad"]), ptr(t["m"]), ptr(t["v"])
            d.shadow = ptr(t["shadow"]) if t.get("shadow") is not None else None
            d.n = int(t["param"].numel())
            d.lr_scale = float(t.get("lr_scale", 1.0))
        hp = hyrf_adam_hparams(float(lr), float(beta1), float(beta2), float(eps), int(step), float(grad_scale))
        st = L.hyrf_adam_step(arr, len(chunk), C.byref(hp), stream_handle(stream))
        if st != HYRF_OK:
            raise HyrfError(f"hyrf_adam_step: {L.hyrf_error_string(st).decode()} ({st})")


class hyrf_kernel_time(C.Structure):
    _fields_ = [("name", C.c_char_p), ("launches", C.c_uint64), ("total_ms", C.c_double)]


def hyrf_timer_enable(on=True):
    """Time every kernel launch of the library with CUDA events on its stream."""
    lib().hyrf_timer_enable(1 if on else 0)


def hyrf_timer_read(max_entries=256):
    """Per-kernel totals since the last read: {name: (launches, total_ms)}; waits
    for the recorded events and clears the totals."""
    buf = (hyrf_kernel_time * max_entries)()
    n = lib().hyrf_timer_read(buf, max_entries)
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
            for i in range(min(n, max_entries))}


# ---------------------------------------------------------------- struct builders

def camera(cam):
    c = hyrf_camera()
    R = [float(x) for x in torch.as_tensor(cam.R, dtype=torch.float32).reshape(9)]
    t = [float(x) for x in torch.as_tensor(cam.t, dtype=torch.float32).reshape(3)]
    c.R[:] = R
    c.t[:] = t
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = cam.width, cam.height
    c.z_near, c.cull_tol = cam.z_near, cam.cull_tol
    return c


def grid(table, g, dtype, qparams=None):
    s = hyrf_grid()
    s.table = ptr(table)
    s.n_levels, s.log2_T, s.n_feat, s.base_res = g.n_levels, g.log2_T, g.n_feat, g.base_res
    s.growth = g.growth
    s.dtype = dtype
    s.qparams = ptr(qparams)
    return s


def hyrf_quantize_grid(table, dtype, n_levels, log2_T, codes, qparams, stream=None):
    """8-bit min-max codes of a hash table (per level lo and step)."""
    _check("hyrf_quantize_grid", lib().hyrf_quantize_grid(ptr(table), int(dtype), int(n_levels), int(log2_T),
                                                          ptr(codes), ptr(qparams), stream_handle(stream)))


def mlp(Ws, bs, m, dtype):
    s = hyrf_mlp()
    for l in range(m.n_hidden + 1):
        s.W[l] = ptr(Ws[l])
        s.b[l] = ptr(bs[l])
    s.n_in, s.width, s.n_hidden, s.n_out = m.n_in, m.width, m.n_hidden, m.n_out
    s.dtype = dtype
    return s


def field_grads(geo_table=None, rad_table=None, geo_W=(), geo_b=(), col_W=(), col_b=()):
    s = hyrf_field_grads()
    s.geo_table, s.rad_table = ptr(geo_table), ptr(rad_table)
    for l, t in enumerate(geo_W):
        s.geo_W[l] = ptr(t)
    for l, t in enumerate(geo_b):
        s.geo_b[l] = ptr(t)
    for l, t in enumerate(col_W):
        s.col_W[l] = ptr(t)
    for l, t in enumerate(col_b):
        s.col_b[l] = ptr(t)
    return s


def _fill(st, kw):
    for k, v in kw.items():
        if isinstance(v, torch.Tensor):
            v = ptr(v)
        setattr(st, k, v)
    return st


# ---------------------------------------------------------------- the calls

def hyrf_query_fields(ws=None, stream=None, **kw):
    return call("hyrf_query_fields", _fill(hyrf_query_fields_args(), kw), ws, stream)


def hyrf_query_fields_backward(ws=None, stream=None, **kw):
    return call("hyrf_query_fields_backward", _fill(hyrf_query_fields_backward_args(), kw), ws,
                stream)


def hyrf_project(ws=None, stream=None, **kw):
    return call("hyrf_project", _fill(hyrf_project_args(), kw), ws, stream)


def hyrf_project_backward(ws=None, stream=None, **kw):
    return call("hyrf_project_backward", _fill(hyrf_project_backward_args(), kw), ws, stream)


def hyrf_bin_sort(ws=None, stream=None, **kw):
    return call("hyrf_bin_sort", _fill(hyrf_bin_sort_args(), kw), ws, stream)


def hyrf_precull(ws=None, stream=None, **kw):
    """Pre-cull and ascending compaction alone (query_fields with vis_ready=1 then skips it)."""
    return call("hyrf_precull", _fill(hyrf_precull_args(), kw), ws, stream)


def hyrf_depth_order(ws=None, stream=None, **kw):
    """The visible rows in hyrf_bin_sort's depth order, from the positions."""
    return call("hyrf_depth_order", _fill(hyrf_depth_order_args(), kw), ws, stream)


def hyrf_bin_sort_backward(ws=None, stream=None, **kw):
    return call("hyrf_bin_sort_backward", _fill(hyrf_bin_sort_args(), kw), ws, stream)


def _check(name, st):
    if st != HYRF_OK:
        raise HyrfError(f"{name}: {lib().hyrf_error_string(st).decode()} ({st})")


def hyrf_densify_stats(stream=None, **kw):
    """Accumulate the view-space positional gradient statistics of one view."""
    _check("hyrf_densify_stats",
           lib().hyrf_densify_stats(C.byref(_fill(hyrf_densify_stats_args(), kw)), stream_handle(stream)))


def hyrf_densify_plan(ws=None, stream=None, **kw):
    """Per-Gaussian keep / prune / clone / split and the output offsets."""
    return call("hyrf_densify_plan", _fill(hyrf_densify_plan_args(), kw), ws, stream)


def hyrf_densify_apply(arrays, stream=None, **kw):
    """Rewrite per-Gaussian arrays: arrays = [(src, dst, kind), ...] with
    src [N, w] / dst [N', w] float32 tensors (w = 1 for flat tensors)."""
    a = _fill(hyrf_densify_apply_args(), kw)
    if len(arrays) > REMAP_MAX:
        raise HyrfError("too many arrays")
    a.n_arrays = len(arrays)
    for d, (src, dst, kind) in zip(a.arrays, arrays):
        d.src, d.dst = ptr(src), ptr(dst)
        d.width = 1 if src.dim() == 1 else int(src.shape[1])
        d.kind = int(kind)
    _check("hyrf_densify_apply", lib().hyrf_densify_apply(C.byref(a), stream_handle(stream)))


def hyrf_spatial_order(ws=None, stream=None, **kw):
    """Morton order of the contracted positions: fills perm."""
    a = hyrf_spatial_order_args()
    lo, hi = kw.pop("box_lo"), kw.pop("box_hi")
    a.box_lo[:] = [float(x) for x in lo]
    a.box_hi[:] = [float(x) for x in hi]
    return call("hyrf_spatial_order", _fill(a, kw), ws, stream)


def hyrf_gather_background(args, stream=None):
    """Fill args.features with the background hash features (ahead of
    hyrf_composite_background with features_ready = 1)."""
    _check("hyrf_gather_background", lib().hyrf_gather_background(C.byref(args), stream_handle(stream)))


def hyrf_permute_rows(perm, pairs, stream=None):
    """dst[k] = src[perm[k]] for every (src, dst) pair of float32 tensors."""
    arr = (hyrf_remap_array * max(1, len(pairs)))()
    for d, (src, dst) in zip(arr, pairs):
        d.src, d.dst = ptr(src), ptr(dst)
        d.width = 1 if src.dim() == 1 else int(src.shape[1])
    _check("hyrf_permute_rows", lib().hyrf_permute_rows(ptr(perm), int(perm.numel()), arr, len(pairs),
                                                        stream_handle(stream)))


def hyrf_reset_opacity(alpha_e, max_logit, m=None, v=None, stream=None):
    """alpha_e = min(alpha_e, max_logit); the Adam moments restart from zero."""
    _check("hyrf_reset_opacity", lib().hyrf_reset_opacity(ptr(alpha_e), int(alpha_e.numel()), float(max_logit),
                                                          ptr(m), ptr(v), stream_handle(stream)))


def hyrf_bin_sort_noalloc(stream=None, **kw):
    """hyrf_bin_sort with the library's fixed scratch array (no workspace)."""
    a = _fill(hyrf_bin_sort_args(), kw)
    L = lib()
    st = L.hyrf_bin_sort_noalloc(C.byref(a), stream_handle(stream))
    if st != HYRF_OK:
        raise HyrfError(f"hyrf_bin_sort_noalloc: {L.hyrf_error_string(st).decode()} ({st})")
    return st


def hyrf_rasterize(ws=None, stream=None, **kw):
    return call("hyrf_rasterize", _fill(hyrf_rasterize_args(), kw), ws, stream)


def hyrf_tile_order(ws=None, stream=None, **kw):
    """Tiles by decreasing bit length of their longest pixel list (n_contrib)."""
    kw.setdefault("tile", TILE)
    return call("hyrf_tile_order", _fill(hyrf_tile_order_args(), kw), ws, stream)


def hyrf_rasterize_backward(fwd, ws=None, stream=None, **kw):
    a = _fill(hyrf_rasterize_backward_args(), kw)
    a.fwd = fwd
    return call("hyrf_rasterize_backward", a, ws, stream)


def hyrf_composite_background(ws=None, stream=None, **kw):
    return call("hyrf_composite_background", _fill(hyrf_composite_background_args(), kw), ws,
                stream)


def hyrf_composite_background_backward(fwd, ws=None, stream=None, **kw):
    a = _fill(hyrf_composite_background_backward_args(), kw)
    a.fwd = fwd
    return call("hyrf_composite_background_backward", a, ws, stream)


def hyrf_loss(ws=None, stream=None, **kw):
    lam = kw.pop("lambda_", kw.pop("lam", 0.0))
    a = _fill(hyrf_loss_args(), kw)
    a.lambda_ = lam
    return call("hyrf_loss", a, ws, stream)
