"""Seeded synthetic HyRF workloads (numpy only; no method arithmetic).

The paper's datasets (MipNeRF360, Tanks&Temples, DeepBlending, Mill19, ...)
are not available; these generators stand in for them with the shapes the
paper reports: Gaussian counts of 1-6 M (App. A.5), hash tables of 2^17-2^22
entries x 16 levels x 2 features and 2x64 decoders (Sec. 4.1), and image
sizes around one megapixel. All randomness comes from
numpy.random.Generator(PCG64(seed)); scene seed 0, target seed 1.

Both the CUDA path's tests and the oracle consume these objects; this module
holds only random draws, camera placement and parameter initialisation.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def bf16_round(a):
    """Round float32 values to the nearest bfloat16 (ties to even), kept as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).reshape(a.shape)


@dataclass
class Camera:
    R: np.ndarray            # [3,3] float32, world -> camera rotation
    t: np.ndarray            # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    z_near: float = 0.2
    cull_tol: float = 0.3

    def center(self):
        return -(self.R.astype(np.float64).T @ self.t.astype(np.float64))


@dataclass
class HashGrid:
    n_levels: int
    log2_T: int
    table: np.ndarray        # [L, T, F] float32 (bf16-representable in the BF16 path)
    n_feat: int = 2
    base_res: int = 16
    growth: float = 1.5


@dataclass
class MLP:
    n_in: int
    width: int
    n_hidden: int
    n_out: int
    W: List[np.ndarray]      # [out, in] float32
    b: List[np.ndarray]      # [out] float32


@dataclass
class Fields:
    box_lo: np.ndarray
    box_hi: np.ndarray
    geo: HashGrid
    rad: HashGrid
    geo_mlp: MLP
    col_mlp: MLP
    pe_freq: int = 4
    pe_pad: int = 32


@dataclass
class Gaussians:
    pos: np.ndarray          # [N,3] float32
    alpha_e: np.ndarray      # [N] float32, opacity logit
    scale_e: np.ndarray      # [N] float32, isotropic scale logit
    color_e: np.ndarray      # [N,3] float32, colour logits
    quat: Optional[np.ndarray] = None  # [N,4] unit quaternions for stage-level tests

    @property
    def n(self):
        return len(self.pos)


@dataclass
class Background:
    mode: int = 0            # 0 exact per-pixel query, 1 equirect map
    map_h: int = 0
    map_w: int = 0
    radius: float = 100.0


@dataclass
class Workload:
    name: str
    gaussians: Gaussians
    fields: Fields
    cams: List[Camera]
    bg: Background
    targets: List[np.ndarray]        # [H,W,3] float32 per camera
    ssim_lambda: float = 0.0
    precision: str = "f32"           # "f32" or "bf16" (grid tables + MLP weights)
    loss_scale: float = 1.0
    extra: dict = field(default_factory=dict)


def pinhole(width, height, fov_x_deg=None, fx=None, R=None, t=None):
    if fx is None:
        fx = (width / 2.0) / np.tan(np.radians(fov_x_deg) / 2.0)
    fx = float(np.float32(fx))
    R = np.eye(3, dtype=np.float32) if R is None else np.asarray(R, dtype=np.float32)
    t = np.zeros(3, dtype=np.float32) if t is None else np.asarray(t, dtype=np.float32)
    return Camera(R=R, t=t, fx=fx, fy=fx, cx=float(np.float32(width / 2.0)),
                  cy=float(np.float32(height / 2.0)), width=width, height=height)


def look_at(eye, target, width, height, fov_x_deg):
    """Camera at `eye` looking at `target`; camera y points along world +y
    ("down" in the image), z forward."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, f)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f]).astype(np.float32)
    t = (-(R.astype(np.float64) @ eye)).astype(np.float32)
    return pinhole(width, height, fov_x_deg, R=R, t=t)


def random_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def explicit_params(rng, pos):
    """Explicit 8-parameter Gaussians (Sec. 3.2): opacity logit N(0,1), scale
    logit with sigma(s_e) = e^u, u ~ U(-5,-2), colour logits N(0,1)."""
    n = len(pos)
    alpha_e = rng.standard_normal(n).astype(np.float32)
    u = rng.uniform(-5.0, -2.0, n)
    s = np.exp(u)
    scale_e = np.log(s / (1.0 - s)).astype(np.float32)
    color_e = rng.standard_normal((n, 3)).astype(np.float32)
    quat = random_quats(rng, n)
    return Gaussians(pos=np.ascontiguousarray(pos, dtype=np.float32), alpha_e=alpha_e,
                     scale_e=scale_e, color_e=color_e, quat=quat)


def hash_grid(rng, n_levels, log2_T, init=1e-4, n_feat=2):
    table = rng.uniform(-init, init, (n_levels, 1 << log2_T, n_feat)).astype(np.float32)
    return HashGrid(n_levels=n_levels, log2_T=log2_T, table=table, n_feat=n_feat)


def xavier_mlp(rng, n_in, width, n_hidden, n_out, out_bias=None):
    Ws, bs = [], []
    dims = [n_in] + [width] * n_hidden + [n_out]
    for l in range(n_hidden + 1):
        fi, fo = dims[l], dims[l + 1]
        a = np.sqrt(6.0 / (fi + fo))
        Ws.append(rng.uniform(-a, a, (fo, fi)).astype(np.float32))
        bs.append(np.zeros(fo, dtype=np.float32))
    if out_bias is not None:
        bs[-1] = np.asarray(out_bias, dtype=np.float32).copy()
    return MLP(n_in=n_in, width=width, n_hidden=n_hidden, n_out=n_out, W=Ws, b=bs)


# Geometry decoder output: (alpha_n, s_n[3], r_n[4]); the rotation part starts
# at the identity quaternion so that Normalize(r_n) is well conditioned.
GEO_BIAS = [0, 0, 0, 0, 1, 0, 0, 0]


def make_fields(rng, box_lo, box_hi, n_levels, log2_T, width, n_hidden, table_init=1e-4,
                pe_freq=4, pe_pad=32):
    geo = hash_grid(rng, n_levels, log2_T, table_init)
    rad = hash_grid(rng, n_levels, log2_T, table_init)
    nf = n_levels * 2
    gm = xavier_mlp(rng, nf, width, n_hidden, 8, GEO_BIAS)
    cm = xavier_mlp(rng, nf + pe_pad, width, n_hidden, 3)
    return Fields(box_lo=np.asarray(box_lo, np.float64), box_hi=np.asarray(box_hi, np.float64),
                  geo=geo, rad=rad, geo_mlp=gm, col_mlp=cm, pe_freq=pe_freq, pe_pad=pe_pad)


def f16_round(a):
    """Round float32 values to the nearest IEEE half (ties to even), kept as float32."""
    return np.ascontiguousarray(a, dtype=np.float32).astype(np.float16).astype(np.float32)


def to_f16(fields: Fields) -> Fields:
    """Same fields with tables and decoder weights rounded to IEEE half."""
    def g(h):
        return HashGrid(h.n_levels, h.log2_T, f16_round(h.table), h.n_feat, h.base_res, h.growth)

    def m(x):
        return MLP(x.n_in, x.width, x.n_hidden, x.n_out, [f16_round(w) for w in x.W],
                   [b.copy() for b in x.b])
    return Fields(fields.box_lo, fields.box_hi, g(fields.geo), g(fields.rad), m(fields.geo_mlp),
                  m(fields.col_mlp), fields.pe_freq, fields.pe_pad)


def to_bf16(fields: Fields) -> Fields:
    """Same fields with tables and decoder weights rounded to bfloat16."""
    def g(h):
        return HashGrid(h.n_levels, h.log2_T, bf16_round(h.table), h.n_feat, h.base_res, h.growth)

    def m(x):
        return MLP(x.n_in, x.width, x.n_hidden, x.n_out, [bf16_round(w) for w in x.W],
                   [b.copy() for b in x.b])
    return Fields(fields.box_lo, fields.box_hi, g(fields.geo), g(fields.rad), m(fields.geo_mlp),
                  m(fields.col_mlp), fields.pe_freq, fields.pe_pad)


def cluster_points(rng, n, n_clusters, cam, depth=(3.0, 15.0), far_frac=0.1,
                   far_depth=(20.0, 100.0), sigma=(0.05, 0.5)):
    """Anisotropic Gaussian clusters with centres uniform in the camera frustum
    plus a fraction of far points (uniform directions within 1.1 x the frustum)."""
    tx = (cam.width / 2.0) / cam.fx
    ty = (cam.height / 2.0) / cam.fy
    n_far = int(round(n * far_frac))
    n_cl = n - n_far
    z = rng.uniform(depth[0], depth[1], n_clusters)
    cx = rng.uniform(-1, 1, n_clusters) * z * tx
    cy = rng.uniform(-1, 1, n_clusters) * z * ty
    centres = np.stack([cx, cy, z], 1)
    sig = np.exp(rng.uniform(np.log(sigma[0]), np.log(sigma[1]), (n_clusters, 3)))
    # random orientations: Q factor of a Gaussian matrix, sign-fixed
    A = rng.standard_normal((n_clusters, 3, 3))
    Q, Rr = np.linalg.qr(A)
    Rm = Q * np.sign(np.diagonal(Rr, axis1=1, axis2=2))[:, None, :]
    lab = rng.integers(0, n_clusters, n_cl)
    gz = rng.standard_normal((n_cl, 3)) * sig[lab]
    pts = centres[lab] + np.einsum("nij,nj->ni", Rm[lab], gz)
    fz = rng.uniform(far_depth[0], far_depth[1], n_far)
    fx_ = rng.uniform(-1.1, 1.1, n_far) * fz * tx
    fy_ = rng.uniform(-1.1, 1.1, n_far) * fz * ty
    far = np.stack([fx_, fy_, fz], 1)
    pts = np.concatenate([pts, far], 0)
    pts = pts[rng.permutation(len(pts))]
    # camera frame -> world frame
    Rc = cam.R.astype(np.float64)
    tc = cam.t.astype(np.float64)
    world = (pts - tc) @ Rc
    return world.astype(np.float32)


def percentile_box(pos, lo=1.0, hi=99.0):
    """App. A.1 large-scene rule: the 1st-99th percentile box of the points."""
    return (np.percentile(pos, lo, axis=0).astype(np.float64),
            np.percentile(pos, hi, axis=0).astype(np.float64))


def noise_target(rng, cam):
    return rng.uniform(0.0, 1.0, (cam.height, cam.width, 3)).astype(np.float32)


def teacher_of(w, seed=2, sigma=0.3):
    """The workload's scene with its explicit colour and opacity logits moved
    by N(0, sigma^2) draws (a stand-in for the ground-truth image of a scene
    the student nearly fits): rendering it gives a target image a few tens of
    dB from the student's, against which PSNR differences of a hundredth of
    a dB are measurable."""
    import dataclasses
    rng = _rng(seed)
    g = w.gaussians
    g2 = dataclasses.replace(
        g, color_e=(g.color_e + sigma * rng.standard_normal(g.color_e.shape)).astype(np.float32),
        alpha_e=(g.alpha_e + sigma * rng.standard_normal(g.alpha_e.shape)).astype(np.float32))
    return dataclasses.replace(w, gaussians=g2)


# ---------------------------------------------------------------------------
# The five workloads. Each accepts size overrides so tests can run the same
# generator at sizes the oracle finishes in seconds.

def config1(n=4096, width=128, height=128, table_init=1e-4, seed=0):
    """Plain FP32, one view: centres U([-1,1]^2 x [2,4]) before a 128x128
    pinhole camera (fx = fy = 128 at 128 px), 8-level 2^12 grids, 16->32->out
    decoders, 16x16 background map, L1 loss."""
    rng = _rng(seed)
    pos = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 4, n)], 1)
    g = explicit_params(rng, pos)
    cam = pinhole(width, height, fx=128.0 * width / 128.0)
    fl = make_fields(rng, [-1, -1, 2], [1, 1, 4], 8, 12, 32, 1, table_init)
    tr = _rng(seed + 1)
    return Workload("config1: 4,096 Gaussians @128x128, FP32", g, fl, [cam],
                    Background(mode=1, map_h=16, map_w=16), [noise_target(tr, cam)], 0.0)


def config2(n=200_000, width=800, height=800, log2_T=17, n_clusters=64, table_init=1e-4, seed=0):
    """Plain FP32, one view: 64 anisotropic clusters + 10 % far points at
    depth 20-100, 800x800 at 60 deg fov, 16-level 2^17 grids, 32->64->64->out,
    64x128 background map, 0.8 L1 + 0.2 D-SSIM."""
    rng = _rng(seed)
    cam = pinhole(width, height, 60.0)
    pos = cluster_points(rng, n, n_clusters, cam)
    g = explicit_params(rng, pos)
    lo, hi = percentile_box(pos)
    fl = make_fields(rng, lo, hi, 16, log2_T, 64, 2, table_init)
    tr = _rng(seed + 1)
    return Workload("config2: 200k Gaussians @800x800, FP32", g, fl, [cam],
                    Background(mode=1, map_h=64, map_w=128), [noise_target(tr, cam)], 0.2)


def config3(n=1_000_000, width=1237, height=822, log2_T=19, n_clusters=256, precision="bf16",
            table_init=1e-4, seed=0):
    """1M Gaussians from 256 clusters, 1237x822 at 60 deg horizontal fov,
    16-level 2^19 grids, 32->64->64->out, exact background, L1; BF16 grids and
    decoders with loss scale 1024, or the plain FP32 variant."""
    rng = _rng(seed)
    cam = pinhole(width, height, 60.0)
    pos = cluster_points(rng, n, n_clusters, cam)
    g = explicit_params(rng, pos)
    lo, hi = percentile_box(pos)
    fl = make_fields(rng, lo, hi, 16, log2_T, 64, 2, table_init)
    if precision == "bf16":
        fl = to_bf16(fl)
    elif precision == "f16":
        fl = to_f16(fl)
    tr = _rng(seed + 1)
    return Workload(f"config3: 1M Gaussians @1237x822, {precision.upper()} fields", g, fl, [cam],
                    Background(mode=0), [noise_target(tr, cam)], 0.0, precision,
                    1024.0 if precision == "bf16" else 1.0)


def config3_360(n=1_000_000, width=1237, height=822, log2_T=19, n_clusters=256, precision="bf16",
                table_init=1e-4, seed=0):
    """The config-3 scene replicated around the camera: four groups of n/4
    Gaussians, group k turned by k x 90 deg about the camera's vertical axis,
    so that about a quarter lies in the view (a 360-degree capture, as the
    Tanks & Temples scenes of the paper's ablation, Tab. 5)."""
    rng = _rng(seed)
    cam = pinhole(width, height, 60.0)
    parts = []
    for k in range(4):
        p = cluster_points(rng, n // 4 + (1 if k < n % 4 else 0), n_clusters // 4, cam).astype(np.float64)
        a = k * 0.5 * np.pi
        Ry = np.array([[np.cos(a), 0.0, np.sin(a)], [0.0, 1.0, 0.0], [-np.sin(a), 0.0, np.cos(a)]])
        c = cam.center()
        parts.append(((p - c) @ Ry.T + c).astype(np.float32))
    pos = np.concatenate(parts, 0)
    pos = pos[rng.permutation(len(pos))]
    g = explicit_params(rng, pos)
    lo, hi = percentile_box(pos)
    fl = make_fields(rng, lo, hi, 16, log2_T, 64, 2, table_init)
    if precision == "bf16":
        fl = to_bf16(fl)
    tr = _rng(seed + 1)
    return Workload(f"config3-360: 1M Gaussians around the camera @1237x822, {precision.upper()}", g, fl,
                    [cam], Background(mode=0), [noise_target(tr, cam)], 0.0, precision,
                    1024.0 if precision == "bf16" else 1.0)


def config4(n=3_000_000, width=1297, height=840, log2_T=21, n_clusters=1024, n_views=8,
            precision="bf16", table_init=1e-4, seed=0):
    """3M Gaussians in 1024 clusters inside a radius-2 ball at the origin,
    8 cameras on a ring of radius 4 (1297x840, 60 deg), 2^21 BF16 grids."""
    rng = _rng(seed)
    cams = [look_at([4 * np.cos(a), 0.0, 4 * np.sin(a)], [0, 0, 0], width, height, 60.0)
            for a in np.arange(n_views) * 2 * np.pi / n_views]
    d = rng.standard_normal((n_clusters, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    centres = d * 2.0 * rng.uniform(0, 1, (n_clusters, 1)) ** (1 / 3)
    sig = np.exp(rng.uniform(np.log(0.02), np.log(0.2), (n_clusters, 3)))
    lab = rng.integers(0, n_clusters, n)
    pos = (centres[lab] + rng.standard_normal((n, 3)) * sig[lab]).astype(np.float32)
    g = explicit_params(rng, pos)
    lo, hi = percentile_box(pos)
    fl = make_fields(rng, lo, hi, 16, log2_T, 64, 2, table_init)
    if precision == "bf16":
        fl = to_bf16(fl)
    tr = _rng(seed + 1)
    return Workload(f"config4: 3M Gaussians x {n_views} views @1297x840, {precision.upper()}",
                    g, fl, cams, Background(mode=0), [noise_target(tr, c) for c in cams], 0.0,
                    precision, 1024.0 if precision == "bf16" else 1.0)


def config5(n=6_000_000, width=1920, height=1080, log2_T=22, n_clusters=1024, precision="bf16",
            degenerate_frac=0.01, table_init=1e-4, seed=0):
    """6M Gaussians, 40 % beyond depth 50 (background-dominated), 1920x1080,
    2^22 BF16 grids; 1 % near-degenerate Gaussians (scale ratio 1e4) whose
    scale is overwritten at the projection input."""
    rng = _rng(seed)
    cam = pinhole(width, height, 60.0)
    pos = cluster_points(rng, n, n_clusters, cam, far_frac=0.4, far_depth=(50.0, 100.0))
    g = explicit_params(rng, pos)
    lo, hi = percentile_box(pos)
    fl = make_fields(rng, lo, hi, 16, log2_T, 64, 2, table_init)
    if precision == "bf16":
        fl = to_bf16(fl)
    n_deg = int(round(n * degenerate_frac))
    deg_ids = np.sort(rng.choice(n, n_deg, replace=False)).astype(np.int32)
    deg_scale = np.tile(np.array([[1e-1, 1e-5, 1e-5]], np.float32), (n_deg, 1))
    tr = _rng(seed + 1)
    return Workload(f"config5: 6M Gaussians @1920x1080, {precision.upper()}", g, fl, [cam],
                    Background(mode=0), [noise_target(tr, cam)], 0.0, precision,
                    1024.0 if precision == "bf16" else 1.0,
                    extra=dict(degenerate_ids=deg_ids, degenerate_scale=deg_scale))
