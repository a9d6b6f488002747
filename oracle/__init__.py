"""HyRF FP64 oracle (arXiv 2509.17083): ctypes wrapper and stage composition.

TEST INFRASTRUCTURE. Only tests/, the smoke check and the CPU-baseline leg
of bench.py may import this package. It imports nothing from the product
package; inputs are plain numpy arrays or duck-typed objects with the fields
named below (camera: R, t, fx, fy, cx, cy, width, height, z_near, cull_tol;
grid: table, n_levels, log2_T, n_feat, base_res, growth; mlp: W, b, n_in,
width, n_hidden, n_out; fields: box_lo, box_hi, geo, rad, geo_mlp, col_mlp,
pe_freq, pe_pad; background: mode, map_h, map_w, radius).

Every function follows the section or equation named in its docstring; the
C++ sources carry the step-by-step definitions. Parity pins live in
tests/test_oracle_*.py.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_f64p = C.POINTER(C.c_double)
_f32p = C.POINTER(C.c_float)
_i32p = C.POINTER(C.c_int32)
_u8p = C.POINTER(C.c_uint8)
_u64p = C.POINTER(C.c_uint64)

TILE = 16


class _Camera(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("z_near", C.c_double),
                ("cull_tol", C.c_double)]


class _Aabb(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3)]


class _Grid(C.Structure):
    _fields_ = [("n_levels", C.c_int32), ("log2_T", C.c_int32), ("n_feat", C.c_int32),
                ("base_res", C.c_int32), ("growth", C.c_double), ("table", _f64p)]


class _Mlp(C.Structure):
    _fields_ = [("n_in", C.c_int32), ("width", C.c_int32), ("n_hidden", C.c_int32),
                ("n_out", C.c_int32), ("W", _f64p * 3), ("b", _f64p * 3),
                ("relu_replay", C.c_int32)]


class _MlpGrad(C.Structure):
    _fields_ = [("W", _f64p * 3), ("b", _f64p * 3)]


class _Fields(C.Structure):
    _fields_ = [("box", _Aabb), ("geo", _Grid), ("rad", _Grid), ("geo_mlp", _Mlp),
                ("col_mlp", _Mlp), ("pe_freq", C.c_int32), ("pe_pad", C.c_int32)]


class _Bg(C.Structure):
    _fields_ = [("mode", C.c_int32), ("map_h", C.c_int32), ("map_w", C.c_int32),
                ("radius", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _lib.orc_loss.restype = C.c_double
        _lib.orc_ssim.restype = C.c_double
        _lib.orc_bin_sort.restype = C.c_int64
        _lib.orc_level_index.restype = C.c_uint32
        _lib.orc_branch_sum.restype = C.c_uint64
    return _lib


def _d(a):
    """Contiguous float64 copy (kept alive by the caller) and its pointer."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


def _ptr(a, t):
    return a.ctypes.data_as(t)


class _Keep:
    """Holds the numpy buffers a ctypes struct points into."""

    def __init__(self):
        self.items = []

    def d(self, a):
        a, p = _d(a)
        self.items.append(a)
        return p


def camera(cam):
    c = _Camera()
    R = np.asarray(cam.R, dtype=np.float64).reshape(9)
    t = np.asarray(cam.t, dtype=np.float64).reshape(3)
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.z_near, c.cull_tol = float(cam.z_near), float(cam.cull_tol)
    return c


def _grid(g, keep):
    s = _Grid()
    s.n_levels, s.log2_T, s.n_feat, s.base_res = g.n_levels, g.log2_T, g.n_feat, g.base_res
    s.growth = float(g.growth)
    s.table = keep.d(np.asarray(g.table, dtype=np.float64).reshape(-1))
    return s


# Precision in which the decoders' ReLU branches are decided (orc_mlp.relu_replay).
_RELU_REPLAY = {"f64": 0, "bf16": 1}


def branch_sum_reset():
    lib().orc_branch_sum_reset()


def branch_sum():
    """Sum of a 64-bit mix of every decoder evaluation's ReLU branch pattern
    since the last branch_sum_reset (changes when any branch changes)."""
    return int(lib().orc_branch_sum())


def replay_relu(fields, precision="bf16"):
    """A shallow copy of `fields` whose decoders decide every hidden unit's
    ReLU branch as a kernel with `precision` operands does ("bf16": layer
    inputs and hidden outputs rounded to bfloat16, sums exact) and evaluate
    FP64 values on those branches; "f64" is the plain FP64 decoder. The
    reading: where floating point decides a branch, the oracle takes it in the
    kernel's precision (as the FP32 replays of the integer decisions do)."""
    import copy
    if precision not in _RELU_REPLAY:
        raise ValueError(precision)
    f = copy.copy(fields)
    f.relu_precision = precision
    return f


def _mlp(m, keep, relu="f64"):
    s = _Mlp()
    s.n_in, s.width, s.n_hidden, s.n_out = m.n_in, m.width, m.n_hidden, m.n_out
    s.relu_replay = _RELU_REPLAY[relu]
    for l in range(m.n_hidden + 1):
        s.W[l] = keep.d(np.asarray(m.W[l], dtype=np.float64))
        s.b[l] = keep.d(np.asarray(m.b[l], dtype=np.float64))
    return s


def fields_struct(fl, keep):
    s = _Fields()
    for k in range(3):
        s.box.lo[k] = float(fl.box_lo[k])
        s.box.hi[k] = float(fl.box_hi[k])
    s.geo = _grid(fl.geo, keep)
    s.rad = _grid(fl.rad, keep)
    relu = getattr(fl, "relu_precision", "f64")
    s.geo_mlp = _mlp(fl.geo_mlp, keep, relu)
    s.col_mlp = _mlp(fl.col_mlp, keep, relu)
    s.pe_freq, s.pe_pad = fl.pe_freq, fl.pe_pad
    return s


def _mlp_grad(m):
    """Zeroed gradient buffers shaped like m, and the struct pointing at them."""
    Ws = [np.zeros_like(np.asarray(w, dtype=np.float64)) for w in m.W]
    bs = [np.zeros_like(np.asarray(b, dtype=np.float64)) for b in m.b]
    s = _MlpGrad()
    for l in range(len(Ws)):
        s.W[l] = _ptr(Ws[l], _f64p)
        s.b[l] = _ptr(bs[l], _f64p)
    return s, Ws, bs


def _bg(bg):
    s = _Bg()
    s.mode, s.map_h, s.map_w, s.radius = int(bg.mode), int(bg.map_h), int(bg.map_w), float(bg.radius)
    return s


# ---------------------------------------------------------------- building blocks

def contract(box_lo, box_hi, p):
    """App. A.1 normalisation then Eq. 2 contraction; returns (y, dy/dp)."""
    b = _Aabb()
    for k in range(3):
        b.lo[k], b.hi[k] = float(box_lo[k]), float(box_hi[k])
    p, pp = _d(p)
    y = np.zeros(3)
    J = np.zeros(9)
    lib().orc_contract(C.byref(b), pp, _ptr(y, _f64p), _ptr(J, _f64p))
    return y, J.reshape(3, 3)


def hash_encode(grid, y):
    """Eq. 3 multi-resolution hash encoding of one point y in (0,1)^3."""
    keep = _Keep()
    g = _grid(grid, keep)
    y, yp = _d(y)
    f = np.zeros(grid.n_levels * grid.n_feat)
    lib().orc_hash_encode(C.byref(g), yp, _ptr(f, _f64p))
    return f


def level_res(grid, l):
    keep = _Keep()
    g = _grid(grid, keep)
    return lib().orc_level_res(C.byref(g), l)


def level_index(grid, l, ix, iy, iz):
    keep = _Keep()
    g = _grid(grid, keep)
    return lib().orc_level_index(C.byref(g), l, ix, iy, iz)


def mlp_forward(mlp, x, relu="f64"):
    keep = _Keep()
    m = _mlp(mlp, keep, relu)
    x, xp = _d(x)
    y = np.zeros(mlp.n_out)
    lib().orc_mlp_forward(C.byref(m), xp, _ptr(y, _f64p))
    return y


def pos_enc(d, n_freq):
    d, dp = _d(d)
    out = np.zeros(3 + 6 * n_freq)
    lib().orc_pos_enc(dp, n_freq, _ptr(out, _f64p))
    return out


# ---------------------------------------------------------------- stages

def precull_f32(pos, cam):
    """Eqs. 8-9 in the GPU's FP32 operation order; returns a bool mask."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    vis = np.zeros(len(pos), dtype=np.uint8)
    c = camera(cam)
    lib().orc_precull_f32(len(pos), _ptr(pos, _f32p), C.byref(c), _ptr(vis, _u8p))
    return vis.astype(bool)


def query_fields(pos, alpha_e, scale_e, color_e, cam, fields):
    """Eqs. 2-7 for visible Gaussians: alpha [n], scale [n,3], quat [n,4], color [n,3]."""
    n = len(pos)
    keep = _Keep()
    fl = fields_struct(fields, keep)
    c = camera(cam)
    out = [np.zeros(n), np.zeros((n, 3)), np.zeros((n, 4)), np.zeros((n, 3))]
    rc = lib().orc_query_fields(n, keep.d(pos), keep.d(alpha_e), keep.d(scale_e), keep.d(color_e),
                                C.byref(c), C.byref(fl), *[_ptr(o, _f64p) for o in out])
    assert rc == 0
    return tuple(out)


def query_fields_backward(pos, alpha_e, scale_e, color_e, cam, fields, d_alpha, d_scale, d_quat,
                          d_color):
    n = len(pos)
    keep = _Keep()
    fl = fields_struct(fields, keep)
    c = camera(cam)
    g = dict(pos=np.zeros((n, 3)), alpha_e=np.zeros(n), scale_e=np.zeros(n),
             color_e=np.zeros((n, 3)),
             geo_table=np.zeros(np.asarray(fields.geo.table).shape),
             rad_table=np.zeros(np.asarray(fields.rad.table).shape))
    gs, gW, gb = _mlp_grad(fields.geo_mlp)
    cs, cW, cb = _mlp_grad(fields.col_mlp)
    rc = lib().orc_query_fields_backward(
        n, keep.d(pos), keep.d(alpha_e), keep.d(scale_e), keep.d(color_e), C.byref(c), C.byref(fl),
        keep.d(d_alpha), keep.d(d_scale), keep.d(d_quat), keep.d(d_color),
        _ptr(g["pos"], _f64p), _ptr(g["alpha_e"], _f64p), _ptr(g["scale_e"], _f64p),
        _ptr(g["color_e"], _f64p), _ptr(g["geo_table"], _f64p), _ptr(g["rad_table"], _f64p),
        C.byref(gs), C.byref(cs))
    assert rc == 0
    g.update(geo_W=gW, geo_b=gb, col_W=cW, col_b=cb)
    return g


def decoder_margins(pos, cam, fields):
    """Smallest relative ReLU margin of each point's geometry and colour
    decoders: (margin_geo [n], margin_col [n])."""
    n = len(pos)
    keep = _Keep()
    fl = fields_struct(fields, keep)
    c = camera(cam)
    mg, mc = np.zeros(n), np.zeros(n)
    rc = lib().orc_decoder_margins(n, keep.d(pos), C.byref(c), C.byref(fl), _ptr(mg, _f64p),
                                   _ptr(mc, _f64p))
    assert rc == 0
    return mg, mc


def bg_margins(cam, fields, bg):
    """Per pixel, the smallest relative ReLU margin of the background's
    colour-decoder evaluations."""
    keep = _Keep()
    fl = fields_struct(fields, keep)
    c = camera(cam)
    b = _bg(bg)
    out = np.zeros((cam.height, cam.width))
    rc = lib().orc_bg_margins(C.byref(c), C.byref(fl), C.byref(b), _ptr(out, _f64p))
    assert rc == 0
    return out


def relu_safe_mask(g, fields, cam, vis_ids, geo_margin, col_margin):
    """Per visible Gaussian: 1 if no ReLU pre-activation of its decoders lies
    within the given relative margins of the kink, else 0."""
    pos = np.asarray(g.pos, np.float64)[vis_ids]
    mg, mc = decoder_margins(pos, cam, fields)
    return ((mg > geo_margin) & (mc > col_margin)).astype(np.float64)


def project(pos, scale, quat, cam):
    """EWA projection (3DGS conventions): mean2d [n,2], conic [n,3], depth [n] (FP64)."""
    n = len(pos)
    keep = _Keep()
    c = camera(cam)
    out = [np.zeros((n, 2)), np.zeros((n, 3)), np.zeros(n)]
    rc = lib().orc_project(n, keep.d(pos), keep.d(scale), keep.d(quat), C.byref(c),
                           *[_ptr(o, _f64p) for o in out])
    assert rc == 0
    return tuple(out)


def project_f32(pos, scale, quat, cam, tile=TILE):
    """FP32 replay of the projection's integer outputs: rect [n,4], ntiles [n]
    (rectangle areas), depth (float32) [n], near-singular flag [n]."""
    rect, ntiles, depth, flag, _, _ = _project_f32(pos, scale, quat, cam, tile, None, False)
    return rect, ntiles, depth, flag


def project_f32_footprint(pos, scale, quat, cam, alpha=None, tile=TILE):
    """FP32 replay of the projection with the binning's opacity-aware
    footprint (opacity alpha [n], or 1 when None): rect [n,4], ntiles [n]
    (tiles of the footprint), depth [n], flag [n], mean2d (float32) [n,2],
    footprint records (float32) [n,12]: Sigma' (a, b, c), t, and eight words
    of packed row spans (bit patterns)."""
    return _project_f32(pos, scale, quat, cam, tile, alpha, True)


def _project_f32(pos, scale, quat, cam, tile, alpha, footprint):
    n = len(pos)
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    scale = np.ascontiguousarray(scale, dtype=np.float32)
    quat = np.ascontiguousarray(quat, dtype=np.float32)
    al = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float32)
    c = camera(cam)
    rect = np.zeros((n, 4), dtype=np.int32)
    ntiles = np.zeros(n, dtype=np.int32)
    depth = np.zeros(n, dtype=np.float32)
    flag = np.zeros(n, dtype=np.uint8)
    mean2d = np.zeros((n, 2), dtype=np.float32) if footprint else None
    foot = np.zeros((n, 12), dtype=np.float32) if footprint else None
    rc = lib().orc_project_f32_fp(n, _ptr(pos, _f32p), _ptr(scale, _f32p), _ptr(quat, _f32p),
                                  None if al is None else _ptr(al, _f32p), C.byref(c), tile,
                                  _ptr(rect, _i32p), _ptr(ntiles, _i32p), _ptr(depth, _f32p),
                                  _ptr(flag, _u8p), None if mean2d is None else _ptr(mean2d, _f32p),
                                  None if foot is None else _ptr(foot, _f32p))
    assert rc == 0
    return rect, ntiles, depth, flag, mean2d, foot


def project_backward(pos, scale, quat, cam, d_mean2d, d_conic):
    n = len(pos)
    keep = _Keep()
    c = camera(cam)
    out = [np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 4))]
    rc = lib().orc_project_backward(n, keep.d(pos), keep.d(scale), keep.d(quat), C.byref(c),
                                    keep.d(d_mean2d), keep.d(d_conic),
                                    *[_ptr(o, _f64p) for o in out])
    assert rc == 0
    return tuple(out)


def tiles_of(width, height, tile=TILE):
    return (width + tile - 1) // tile, (height + tile - 1) // tile


def bin_sort(rect, depth_f32, tiles_x, tiles_y, mean2d=None, footprint=None, tile=TILE):
    """Stable sort of (tile << 32 | depth bits) instance keys: keys, vals,
    ranges [tiles,2]. With mean2d and footprint (project_f32_footprint) each
    rectangle row yields only its footprint's tiles."""
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    depth_f32 = np.ascontiguousarray(depth_f32, dtype=np.float32)
    n = len(rect)
    r = rect
    cnt = np.where((r[:, 2] > r[:, 0]) & (r[:, 3] > r[:, 1]),
                   (r[:, 2] - r[:, 0]) * (r[:, 3] - r[:, 1]), 0)
    cap = int(cnt.sum())
    keys = np.zeros(max(cap, 1), dtype=np.uint64)
    vals = np.zeros(max(cap, 1), dtype=np.int32)
    ranges = np.zeros((tiles_x * tiles_y, 2), dtype=np.int32)
    if footprint is None:
        m2 = fp = None
    else:
        m2 = np.ascontiguousarray(mean2d, dtype=np.float32)
        fp = np.ascontiguousarray(footprint, dtype=np.float32)
    K = lib().orc_bin_sort_fp(n, _ptr(rect, _i32p), _ptr(depth_f32, _f32p),
                              None if m2 is None else _ptr(m2, _f32p), None if fp is None else _ptr(fp, _f32p),
                              tile, tiles_x, tiles_y, cap, _ptr(keys, _u64p), _ptr(vals, _i32p),
                              _ptr(ranges, _i32p))
    assert 0 <= K <= cap and (footprint is not None or K == cap)
    return keys[:K], vals[:K], ranges


def rasterize(width, height, ranges, vals, mean2d, conic, opacity, color, tile=TILE):
    """Eq. 1 front-to-back compositing per tile list: C_fg, T_final, n_contrib, margin."""
    keep = _Keep()
    ranges = np.ascontiguousarray(ranges, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.int32)
    P = width * height
    C_fg, T, nc, mg = np.zeros((height, width, 3)), np.zeros((height, width)), \
        np.zeros((height, width), dtype=np.int32), np.zeros((height, width))
    rc = lib().orc_rasterize(width, height, tile, _ptr(ranges, _i32p), _ptr(vals, _i32p),
                             keep.d(mean2d), keep.d(conic), keep.d(opacity), keep.d(color),
                             _ptr(C_fg, _f64p), _ptr(T, _f64p), _ptr(nc, _i32p), _ptr(mg, _f64p))
    assert rc == 0 and P == T.size
    return C_fg, T, nc, mg


def rasterize_untiled(width, height, rect, depth_f32, mean2d, conic, opacity, color, tile=TILE):
    keep = _Keep()
    rect = np.ascontiguousarray(rect, dtype=np.int32)
    depth_f32 = np.ascontiguousarray(depth_f32, dtype=np.float32)
    C_fg, T = np.zeros((height, width, 3)), np.zeros((height, width))
    rc = lib().orc_rasterize_untiled(width, height, tile, len(rect), _ptr(rect, _i32p),
                                     _ptr(depth_f32, _f32p), keep.d(mean2d), keep.d(conic),
                                     keep.d(opacity), keep.d(color), _ptr(C_fg, _f64p),
                                     _ptr(T, _f64p))
    assert rc == 0
    return C_fg, T


def rasterize_backward(width, height, ranges, vals, mean2d, conic, opacity, color, d_C_fg,
                       d_T_final, tile=TILE):
    keep = _Keep()
    n = len(opacity)
    ranges = np.ascontiguousarray(ranges, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.int32)
    out = [np.zeros((n, 2)), np.zeros((n, 3)), np.zeros(n), np.zeros((n, 3))]
    rc = lib().orc_rasterize_backward(width, height, tile, _ptr(ranges, _i32p), _ptr(vals, _i32p),
                                      keep.d(mean2d), keep.d(conic), keep.d(opacity),
                                      keep.d(color), keep.d(d_C_fg), keep.d(d_T_final),
                                      *[_ptr(o, _f64p) for o in out])
    assert rc == 0
    return tuple(out)


def ray_sphere(cam, box_lo, box_hi, radius, i, j):
    """App. A.2: hit point p_s (normalised space), t, origin and direction."""
    c = camera(cam)
    b = _Aabb()
    for k in range(3):
        b.lo[k], b.hi[k] = float(box_lo[k]), float(box_hi[k])
    ps, o, d = np.zeros(3), np.zeros(3), np.zeros(3)
    t = C.c_double()
    lib().orc_ray_sphere(C.byref(c), C.byref(b), C.c_double(radius), i, j, _ptr(ps, _f64p),
                         C.byref(t), _ptr(o, _f64p), _ptr(d, _f64p))
    return ps, t.value, o, d


def background(cam, fields, bg, C_fg, T_final):
    """Eqs. 10-11: C = C_fg + T_final * c_s; returns (C, c_s)."""
    keep = _Keep()
    fl = fields_struct(fields, keep)
    c = camera(cam)
    b = _bg(bg)
    H, W = cam.height, cam.width
    Cout, cs = np.zeros((H, W, 3)), np.zeros((H, W, 3))
    rc = lib().orc_background(C.byref(c), C.byref(fl), C.byref(b), keep.d(C_fg), keep.d(T_final),
                              _ptr(Cout, _f64p), _ptr(cs, _f64p))
    assert rc == 0
    return Cout, cs


def background_backward(cam, fields, bg, T_final, d_C):
    keep = _Keep()
    fl = fields_struct(fields, keep)
    c = camera(cam)
    b = _bg(bg)
    H, W = cam.height, cam.width
    dCfg, dT = np.zeros((H, W, 3)), np.zeros((H, W))
    d_rad = np.zeros(np.asarray(fields.rad.table).shape)
    cs_, cW, cb = _mlp_grad(fields.col_mlp)
    rc = lib().orc_background_backward(C.byref(c), C.byref(fl), C.byref(b), keep.d(T_final),
                                       keep.d(d_C), _ptr(dCfg, _f64p), _ptr(dT, _f64p),
                                       _ptr(d_rad, _f64p), C.byref(cs_))
    assert rc == 0
    return dict(C_fg=dCfg, T_final=dT, rad_table=d_rad, col_W=cW, col_b=cb)


def loss(C_img, target, lam):
    """Eq. 12: (1 - lam) L1 + lam (1 - SSIM); returns (L, dL/dC)."""
    keep = _Keep()
    H, W = C_img.shape[:2]
    dC = np.zeros((H, W, 3))
    L = lib().orc_loss(W, H, keep.d(C_img), keep.d(target), C.c_double(lam), _ptr(dC, _f64p))
    return L, dC


def quantize_grid(table):
    """8-bit min-max codes of a [L, T, 2] table: (codes uint8, qparams
    [L, 2] float32, decoded float64)."""
    t = np.ascontiguousarray(table, dtype=np.float32)
    L = t.shape[0]
    per = t[0].size
    codes = np.zeros(t.shape, dtype=np.uint8)
    q = np.zeros((L, 2), dtype=np.float32)
    dec = np.zeros(t.shape)
    rc = lib().orc_quantize_grid(L, C.c_int64(per), _ptr(t, _f32p), _ptr(codes, _u8p), _ptr(q, _f32p),
                                 _ptr(dec, _f64p))
    assert rc == 0
    return codes, q, dec


def adam_step(p, grad, m, v, lr, b1, b2, eps, t, grad_scale=1.0):
    """One Adam step (Kingma & Ba, Algorithm 1) on float64 copies; returns
    the updated (p, m, v)."""
    p, m, v = [np.array(x, dtype=np.float64).ravel() for x in (p, m, v)]
    g = np.ascontiguousarray(grad, dtype=np.float64).ravel()
    rc = lib().orc_adam_step(C.c_int64(len(p)), _ptr(p, _f64p), _ptr(g, _f64p), _ptr(m, _f64p),
                             _ptr(v, _f64p), C.c_double(lr), C.c_double(b1), C.c_double(b2),
                             C.c_double(eps), C.c_int32(t), C.c_double(grad_scale))
    assert rc == 0
    return p, m, v


def densify_stats(n, vis_ids, d_mean2d, ntiles, width, height, accum, count):
    """Adds one view's positional-gradient statistics (FP32 replay); returns
    (accum, count) as new arrays."""
    vis = np.ascontiguousarray(vis_ids, dtype=np.int32)
    dm = np.ascontiguousarray(d_mean2d, dtype=np.float32)
    nt = np.ascontiguousarray(ntiles, dtype=np.int32)
    acc = np.array(accum, dtype=np.float32)
    cnt = np.array(count, dtype=np.int32)
    rc = lib().orc_densify_stats(n, len(vis), _ptr(vis, _i32p), _ptr(dm, _f32p), _ptr(nt, _i32p), width, height,
                                 _ptr(acc, _f32p), _ptr(cnt, _i32p))
    assert rc == 0
    return acc, cnt


def densify_plan(n, vis_ids, alpha, scale, accum, count, grad_threshold, dense_scale, min_opacity):
    """(action [n] u8, row [n] i32, offset [n+1] i64, new count)."""
    vis = np.ascontiguousarray(vis_ids, dtype=np.int32)
    al = np.ascontiguousarray(alpha, dtype=np.float32)
    sc = np.ascontiguousarray(scale, dtype=np.float32)
    acc = np.ascontiguousarray(accum, dtype=np.float32)
    cnt = np.ascontiguousarray(count, dtype=np.int32)
    action = np.zeros(n, dtype=np.uint8)
    row = np.zeros(n, dtype=np.int32)
    offset = np.zeros(n + 1, dtype=np.int64)
    f = lib().orc_densify_plan
    f.restype = C.c_int64
    total = f(n, len(vis), _ptr(vis, _i32p), _ptr(al, _f32p), _ptr(sc, _f32p), _ptr(acc, _f32p),
              _ptr(cnt, _i32p), C.c_float(grad_threshold), C.c_float(dense_scale), C.c_float(min_opacity),
              _ptr(action, _u8p), _ptr(row, _i32p), _ptr(offset, C.POINTER(C.c_int64)))
    assert total >= 0
    return action, row, offset, int(total)


def densify_apply(action, row, offset, scale, quat, noise, split_log_scale, src, kind):
    """New array for one per-Gaussian array src [n, w] (kind 0 parameter,
    1 optimiser state, 2 position, 3 explicit scale logit)."""
    n = len(action)
    src = np.ascontiguousarray(src, dtype=np.float64)
    w = 1 if src.ndim == 1 else src.shape[1]
    dst = np.zeros((int(offset[n]), w))
    keep = _Keep()
    a = np.ascontiguousarray(action, dtype=np.uint8)
    r = np.ascontiguousarray(row, dtype=np.int32)
    o = np.ascontiguousarray(offset, dtype=np.int64)
    rc = lib().orc_densify_apply(n, _ptr(a, _u8p), _ptr(r, _i32p), _ptr(o, C.POINTER(C.c_int64)),
                                 keep.d(scale), keep.d(quat), keep.d(noise), C.c_double(split_log_scale), w,
                                 kind, _ptr(src, _f64p), _ptr(dst, _f64p))
    assert rc == 0
    return dst if src.ndim > 1 else dst[:, 0]


def ssim(x, y):
    keep = _Keep()
    H, W = x.shape[:2]
    return lib().orc_ssim(W, H, keep.d(x), keep.d(y))


# ---------------------------------------------------------------- composition

def render(g, fields, cam, bg, tile=TILE):
    """Whole forward path of one view (Fig. 3): pre-cull, field query and
    aggregation, projection, binning, compositing, background."""
    pos32 = np.asarray(g.pos, dtype=np.float32)
    vis = precull_f32(pos32, cam)
    ids = np.nonzero(vis)[0].astype(np.int32)
    pos = np.asarray(g.pos, dtype=np.float64)[ids]
    alpha, scale, quat, color = query_fields(pos, np.asarray(g.alpha_e)[ids],
                                             np.asarray(g.scale_e)[ids],
                                             np.asarray(g.color_e)[ids], cam, fields)
    mean2d, conic, depth = project(pos, scale, quat, cam)
    # binning with the opacity-aware footprint, as the GPU path bins
    rect, ntiles, depth32, flag, m32, foot = project_f32_footprint(pos32[ids], scale, quat, cam, alpha, tile)
    TX, TY = tiles_of(cam.width, cam.height, tile)
    keys, vals, ranges = bin_sort(rect, depth32, TX, TY, m32, foot, tile)
    C_fg, T_final, n_contrib, margin = rasterize(cam.width, cam.height, ranges, vals, mean2d,
                                                 conic, alpha, color, tile)
    C_img, c_s = background(cam, fields, bg, C_fg, T_final)
    return dict(vis=vis, ids=ids, alpha=alpha, scale=scale, quat=quat, color=color,
                mean2d=mean2d, conic=conic, depth=depth, rect=rect, ntiles=ntiles,
                depth32=depth32, flag=flag, keys=keys, vals=vals, ranges=ranges, C_fg=C_fg,
                T_final=T_final, n_contrib=n_contrib, margin=margin, C=C_img, c_s=c_s)


def loss_and_grads(g, fields, cam, bg, target, lam, tile=TILE, dC_mask=None, query_mask=None):
    """Forward, Eq. 12 loss and the analytic reverse pass of every stage.
    Returns (loss, forward dict, gradient dict over all parameters).
    dC_mask (optional [H,W]) multiplies dL/dC before the reverse pass;
    query_mask (optional, one entry per visible Gaussian) multiplies the
    gradients entering the field-query reverse pass."""
    fw = render(g, fields, cam, bg, tile)
    L, dC = loss(fw["C"], target, lam)
    if dC_mask is not None:
        dC = dC * np.asarray(dC_mask, np.float64)[..., None]
    gb = background_backward(cam, fields, bg, fw["T_final"], dC)
    d_mean2d, d_conic, d_op, d_col = rasterize_backward(
        cam.width, cam.height, fw["ranges"], fw["vals"], fw["mean2d"], fw["conic"], fw["alpha"],
        fw["color"], gb["C_fg"], gb["T_final"], tile)
    ids = fw["ids"]
    pos = np.asarray(g.pos, dtype=np.float64)[ids]
    d_pos_p, d_scale, d_quat = project_backward(pos, fw["scale"], fw["quat"], cam, d_mean2d,
                                                d_conic)
    if query_mask is not None:
        qm = np.asarray(query_mask, np.float64)
        d_op, d_col = d_op * qm, d_col * qm[:, None]
        d_scale, d_quat = d_scale * qm[:, None], d_quat * qm[:, None]
    gq = query_fields_backward(pos, np.asarray(g.alpha_e)[ids], np.asarray(g.scale_e)[ids],
                               np.asarray(g.color_e)[ids], cam, fields, d_op, d_scale, d_quat,
                               d_col)
    N = len(g.pos)
    grads = dict(pos=np.zeros((N, 3)), alpha_e=np.zeros(N), scale_e=np.zeros(N),
                 color_e=np.zeros((N, 3)))
    grads["pos"][ids] = gq["pos"] + d_pos_p
    grads["alpha_e"][ids] = gq["alpha_e"]
    grads["scale_e"][ids] = gq["scale_e"]
    grads["color_e"][ids] = gq["color_e"]
    grads["geo_table"] = gq["geo_table"]
    grads["rad_table"] = gq["rad_table"] + gb["rad_table"]
    grads["geo_W"], grads["geo_b"] = gq["geo_W"], gq["geo_b"]
    grads["col_W"] = [a + b for a, b in zip(gq["col_W"], gb["col_W"])]
    grads["col_b"] = [a + b for a, b in zip(gq["col_b"], gb["col_b"])]
    inter = dict(d_mean2d=d_mean2d, d_conic=d_conic, d_alpha=d_op, d_color=d_col,
                 d_scale=d_scale, d_quat=d_quat, dC=dC, d_T_final=gb["T_final"],
                 d_C_fg=gb["C_fg"])
    return L, fw, grads, inter


def decision_safe_mask(fw, cam, tile=TILE, comp_margin=1e-4, rel_radius=1e-5, center_px=1e-4,
                       fields=None, bg=None, bg_relu_margin=0.0):
    """Pixels of a rendered view (the dict `render` returns) whose value is a
    smooth function of the inputs near this point: no compositing threshold
    test within `comp_margin` (relative) of its threshold, and not in a tile
    whose membership in a Gaussian's rectangle changes when 3 sqrt(lambda_max)
    moves by `rel_radius` (relative) or the centre by `center_px` pixels;
    with `bg_relu_margin` > 0, also not a pixel whose background decoder has a
    hidden pre-activation within that relative margin of the ReLU kink."""
    safe = fw["margin"] > comp_margin
    if bg_relu_margin > 0.0:
        safe &= bg_margins(cam, fields, bg) > bg_relu_margin
    con = np.asarray(fw["conic"])
    det = con[:, 0] * con[:, 2] - con[:, 1] ** 2
    sa, sb, sc = con[:, 2] / det, -con[:, 1] / det, con[:, 0] / det
    mid = 0.5 * (sa + sc)
    lam = mid + np.sqrt(np.maximum(mid * mid - (sa * sc - sb * sb), 0.0))
    r3 = 3.0 * np.sqrt(lam)
    m = np.asarray(fw["mean2d"])
    TX, TY = tiles_of(cam.width, cam.height, tile)
    lo, hi = None, None
    for dr in (-rel_radius, rel_radius):
        rad = np.ceil(r3 * (1.0 + dr))
        for du in (-center_px, center_px):
            x0 = np.clip(np.floor((m[:, 0] + du - rad) / tile), 0, TX)
            x1 = np.clip(np.floor((m[:, 0] + du + rad) / tile) + 1, 0, TX)
            y0 = np.clip(np.floor((m[:, 1] + du - rad) / tile), 0, TY)
            y1 = np.clip(np.floor((m[:, 1] + du + rad) / tile) + 1, 0, TY)
            r = np.stack([x0, y0, x1, y1], 1)
            lo = r if lo is None else np.minimum(lo, r)
            hi = r if hi is None else np.maximum(hi, r)
    bad = np.zeros((TY, TX), bool)
    for i in np.nonzero((lo != hi).any(1))[0]:
        ox0, oy0, ox1, oy1 = int(lo[i, 0]), int(lo[i, 1]), int(hi[i, 2]), int(hi[i, 3])
        ix0, iy0, ix1, iy1 = int(hi[i, 0]), int(hi[i, 1]), int(lo[i, 2]), int(lo[i, 3])
        outer = np.zeros((TY, TX), bool)
        outer[oy0:oy1, ox0:ox1] = True
        outer[iy0:max(iy0, iy1), ix0:max(ix0, ix1)] = False
        bad |= outer
    tile_bad = np.kron(bad, np.ones((tile, tile), bool))[:cam.height, :cam.width]
    return safe & ~tile_bad


__all__ = [n for n in dir() if not n.startswith("_")]
_ = os
