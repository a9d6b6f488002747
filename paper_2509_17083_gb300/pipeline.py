"""One HyRF view, forward and backward, through the libhyrf C ABI.

DeviceModel holds the trainable state on the GPU (explicit Gaussians, the
two hash grids and decoders) and its float32 gradient buffers. ViewRenderer
holds every per-view buffer (sized once) and runs the path of Fig. 3:

  hyrf_query_fields -> hyrf_project -> hyrf_bin_sort -> hyrf_rasterize
  -> hyrf_composite_background -> hyrf_loss, then the reverse calls.

All arithmetic happens in the library's kernels; this module only allocates
tensors and fills the argument structs.
"""
import math

import torch

from . import hyrf as H


def _t(a, device, dtype=torch.float32):
    return torch.as_tensor(a).to(device=device, dtype=dtype).contiguous()


class DeviceModel:
    """coupled=True: one hash grid serves both decoders (Tab. 5 "w/o
    Decouple."): the geometry decoder reads the radiance grid and both
    gradients land in one buffer."""

    def __init__(self, workload, device="cuda", coupled=False):
        self.device = device
        self.workload = workload
        g = workload.gaussians
        fl = workload.fields
        self.n = g.n
        self.pos = _t(g.pos, device)
        self.alpha_e = _t(g.alpha_e, device)
        self.scale_e = _t(g.scale_e, device)
        self.color_e = _t(g.color_e, device)
        self.fl = fl
        self.bf16 = workload.precision == "bf16"
        self.f16 = workload.precision == "f16"  # render only
        tdt = torch.bfloat16 if self.bf16 else (torch.float16 if self.f16 else torch.float32)
        self.coupled = bool(coupled)
        self.rad_table = _t(fl.rad.table, device, tdt)
        self.geo_table = self.rad_table if self.coupled else _t(fl.geo.table, device, tdt)
        wdt = tdt
        self.geo_W = [_t(w, device, wdt) for w in fl.geo_mlp.W]
        self.geo_b = [_t(b, device) for b in fl.geo_mlp.b]
        self.col_W = [_t(w, device, wdt) for w in fl.col_mlp.W]
        self.col_b = [_t(b, device) for b in fl.col_mlp.b]
        self.dtype_code = H.HYRF_BF16 if self.bf16 else (H.HYRF_F16 if self.f16 else H.HYRF_F32)
        self.codes = None  # (geo codes, geo qparams, rad codes, rad qparams) once quantised
        self.grad = {}
        self.zero_grad()

    def zero_grad(self):
        """Zero every gradient buffer. They are f32 views of one flat buffer
        (each 256-byte aligned), so this is one fill; buffers replaced later
        (density control, storage order) are zeroed one by one."""
        d = self.device
        if not self.grad:
            shapes = dict(pos=self.pos.shape, alpha_e=self.alpha_e.shape, scale_e=self.scale_e.shape,
                          color_e=self.color_e.shape, rad_table=self.rad_table.shape)
            if not self.coupled:
                shapes["geo_table"] = self.geo_table.shape
            lists = dict(geo_W=[w.shape for w in self.geo_W], geo_b=[b.shape for b in self.geo_b],
                         col_W=[w.shape for w in self.col_W], col_b=[b.shape for b in self.col_b])
            flat = _FlatGrads([*shapes.values(), *[x for v in lists.values() for x in v]], d)
            views = iter(flat.views)
            self.grad = {k: next(views) for k in shapes}
            for k, v in lists.items():
                self.grad[k] = [next(views) for _ in v]
            if self.coupled:
                self.grad["geo_table"] = self.grad["rad_table"]
            self._flat = flat
            return
        self._flat.zero_()
        for v in self.grad.values():
            for x in (v if isinstance(v, list) else [v]):
                if not self._flat.owns(x):
                    x.zero_()

    def fields_struct(self):
        fl = self.fl
        s = H.hyrf_fields()
        s.box_lo[:] = [float(x) for x in fl.box_lo]
        s.box_hi[:] = [float(x) for x in fl.box_hi]
        if self.codes is not None:  # the 8-bit codec (render only)
            gc, gq, rc, rq = self.codes
            s.geo = H.grid(gc, fl.rad if self.coupled else fl.geo, H.HYRF_U8, gq)
            s.rad = H.grid(rc, fl.rad, H.HYRF_U8, rq)
        else:
            s.geo = H.grid(self.geo_table, fl.rad if self.coupled else fl.geo, self.dtype_code)
            s.rad = H.grid(self.rad_table, fl.rad, self.dtype_code)
        s.geo_mlp = H.mlp(self.geo_W, self.geo_b, fl.geo_mlp, self.dtype_code)
        s.col_mlp = H.mlp(self.col_W, self.col_b, fl.col_mlp, self.dtype_code)
        s.pe_freq, s.pe_pad = fl.pe_freq, fl.pe_pad
        return s

    def spatial_order(self):
        """Store the Gaussians in the Morton order of their contracted
        positions (hyrf_spatial_order; a layout step, the scene is unchanged).
        Returns perm: new index k holds the Gaussian that was perm[k].
        Gradient buffers restart from zero; call before building a Trainer."""
        n, d = self.n, self.device
        perm = torch.empty(max(n, 1), dtype=torch.int32, device=d)
        H.hyrf_spatial_order(n=n, pos=self.pos, box_lo=self.fl.box_lo, box_hi=self.fl.box_hi, perm=perm)
        pairs, new = [], []
        for name in ("pos", "alpha_e", "scale_e", "color_e"):
            src = getattr(self, name)
            dst = torch.empty_like(src)
            pairs.append((src.view(n, -1), dst.view(n, -1)))
            new.append((name, dst))
        H.hyrf_permute_rows(perm[:n], pairs)
        for name, dst in new:
            setattr(self, name, dst)
            self.grad[name].zero_()  # same shape: the buffer stays
        return perm[:n]

    def quantize_u8(self, on=True):
        """Switch the grids to their 8-bit min-max codes (render only; the
        float tables stay and are used again after quantize_u8(False))."""
        if not on:
            self.codes = None
            return
        out = []
        for t, g in ((self.geo_table, self.fl.geo), (self.rad_table, self.fl.rad)):
            codes = torch.empty(t.shape, dtype=torch.uint8, device=self.device)
            q = torch.empty(g.n_levels, 2, dtype=torch.float32, device=self.device)
            H.hyrf_quantize_grid(t, self.dtype_code, g.n_levels, g.log2_T, codes, q)
            out += [codes, q]
        self.codes = tuple(out)

    def grads_struct(self):
        g = self.grad
        return H.field_grads(g["geo_table"], g["rad_table"], g["geo_W"], g["geo_b"], g["col_W"],
                             g["col_b"])


class _FlatGrads:
    """f32 buffers of the given shapes as views of one zero-initialised
    allocation, each starting on a 256-byte boundary."""

    def __init__(self, shapes, device):
        offs, total = [], 0
        for sh in shapes:
            offs.append(total)
            total += (math.prod(sh) + 63) // 64 * 64
        self.buf = torch.zeros(max(total, 1), device=device)
        self.views = [self.buf.narrow(0, o, math.prod(sh)).view(sh) for o, sh in zip(offs, shapes)]
        self._ids = {id(v) for v in self.views}

    def zero_(self):
        self.buf.zero_()

    def owns(self, t):
        return id(t) in self._ids


def shared_workspaces(device="cuda"):
    """Scratch buffers of the library calls of one view. Pass the same dict to
    several ViewRenderers that run one after the other on one stream to share
    it (with save_features off, the gathered hash features then live only in
    this scratch: memory for time)."""
    return {k: H.Workspace(device) for k in ("q", "qb", "p", "s", "r", "rb", "b", "bb", "l", "to", "pc", "do")}


class ViewRenderer:
    """Buffers and calls for one camera of fixed size.

    save_features (BF16 fields only; default on for them): keep the hash
    features gathered by the forward (2 x 64 B per Gaussian, 64 B per pixel)
    for the backward, which then skips its gather; off = gather again
    (recompute). workspaces: a scratch dict shared with other views
    (shared_workspaces()).

    Ablations of Tab. 5: neural=False (explicit-only isotropic Gaussians),
    explicit=False (neural terms only), background=False (C = C_fg),
    precull=False (every Gaussian in front of the near plane is queried)."""

    def __init__(self, model: DeviceModel, cam, bg, lam=0.0, loss_scale=1.0, capacity=None,
                 save_features=None, workspaces=None, neural=True, explicit=True, background=True,
                 precull=True):
        self.m = model
        self.cam = cam
        self.bg = bg
        self.lam = float(lam)
        self.loss_scale = float(loss_scale)
        d = model.device
        n = model.n
        W, Hh = cam.width, cam.height
        self.W, self.H = W, Hh
        self.TX, self.TY = (W + H.TILE - 1) // H.TILE, (Hh + H.TILE - 1) // H.TILE
        i32, f32 = torch.int32, torch.float32
        z = lambda *s, dt=f32: torch.zeros(*s, dtype=dt, device=d)
        self.status = z(1, dt=i32)
        self.vis_ids, self.n_vis = z(max(n, 1), dt=i32), z(1, dt=i32)
        self.alpha, self.scale, self.quat, self.color = z(n), z(n, 3), z(n, 4), z(n, 3)
        self.mean2d, self.conic, self.depth = z(n, 2), z(n, 3), z(n)
        # the compositing records the forward packs and the reverse reuses
        self.records = z(max(n, 1), 12)
        self.rect, self.ntiles = z(n, 4, dt=i32), z(n, dt=i32)
        # opacity-aware footprint of each projected Gaussian (hyrf_project):
        # the binning keeps only the tiles it can show in
        self.footprint = z(max(n, 1), 12)
        self.flag = z(max(n, 1), dt=torch.uint8)
        self.ranges = z(self.TX * self.TY, 2, dt=i32)
        # the compositing passes take the tiles in this order: index order at
        # first, then longest pixel list first from the last forward's
        # n_contrib (the forward uses the previous frame's, the reverse the
        # current one)
        self.tile_order = torch.arange(self.TX * self.TY, dtype=i32, device=d)
        self.depth_order = z(max(n, 1), dt=i32)  # visible rows by depth (hyrf_depth_order)
        self._depth_ready = False
        self.n_inst = z(1, dt=i32)
        self.C_fg, self.T_final = z(Hh, W, 3), z(Hh, W)
        self.n_contrib = z(Hh, W, dt=i32)
        self.C = z(Hh, W, 3)
        self.loss = z(1)
        self.dC, self.dT = z(Hh, W, 3), z(Hh, W)
        self._dvis = _FlatGrads([(n, 2), (n, 3), (n,), (n, 3)], d)  # zeroed by one fill
        self.d_mean2d, self.d_conic, self.d_alpha, self.d_color = self._dvis.views
        self.d_scale, self.d_quat = z(n, 3), z(n, 4)
        # scratch of the library calls; views that run one after the other on
        # one stream may share one dict (see shared_workspaces)
        self.ws = workspaces if workspaces is not None else shared_workspaces(d)
        self.neural, self.explicit = bool(neural), bool(explicit)
        self.background, self.precull = bool(background), bool(precull)
        if save_features is None:
            save_features = model.bf16 and self.neural
        if save_features and not model.bf16:
            raise ValueError("save_features needs BF16 fields")
        self.save_features = bool(save_features)
        self.feat_q = self.feat_b = None
        # second stream: the background's feature gather ahead of the
        # foreground, and its table-gradient scatter behind it
        self.side = torch.cuda.Stream(device=d) if str(d).startswith("cuda") else None
        self._depth_done = torch.cuda.Event() if self.side is not None else None
        self.serial = False
        if self.save_features:
            self.feat_q = torch.empty(2 * max(n, 1) * 32, dtype=torch.bfloat16, device=d)
            if int(bg.mode) == 0 and self.background:
                self.feat_b = torch.empty(W * Hh * 32, dtype=torch.bfloat16, device=d)
        self.set_capacity(capacity if capacity is not None else max(4 * n, 1 << 16))
        self.ccam = H.camera(cam)
        # the field query's camera: without the pre-cull every Gaussian is
        # queried (the projection still drops those behind the near plane)
        self.ccam_q = H.camera(cam)
        if not self.precull:
            self.ccam_q.cull_tol = 1e30
            self.ccam_q.z_near = -1e30
        self.cbg = H.hyrf_background(int(bg.mode) if self.background else 2, int(bg.map_h), int(bg.map_w),
                                     float(bg.radius))

    def set_capacity(self, cap):
        self.capacity = int(cap)
        d = self.m.device
        self.keys = torch.zeros(self.capacity, dtype=torch.int64, device=d)
        self.vals = torch.zeros(self.capacity, dtype=torch.int32, device=d)

    # ------------------------------------------------------------- forward
    def _raster_args(self):
        a = H.hyrf_rasterize_args()
        H._fill(a, dict(n=self.m.n, n_vis=self.n_vis, ranges=self.ranges, vals=self.vals,
                        mean2d=self.mean2d, conic=self.conic, alpha=self.alpha, color=self.color,
                        width=self.W, height=self.H, tile=H.TILE, C_fg=self.C_fg,
                        T_final=self.T_final, n_contrib=self.n_contrib, status=self.status,
                        tile_order=self.tile_order, records=self.records))
        return a

    def rasterize(self):
        """Compositing forward, then the tile order of its n_contrib (for the
        reverse and the next forward)."""
        H.call("hyrf_rasterize", self._raster_args(), self.ws["r"])
        H.hyrf_tile_order(ws=self.ws["to"], width=self.W, height=self.H, n_contrib=self.n_contrib,
                          order=self.tile_order)

    def _bg_args(self, tau_T=0.0):
        a = H.hyrf_composite_background_args()
        a.cam = self.ccam
        a.fields = self.m.fields_struct()
        a.bg = self.cbg
        a.bg.tau_T = float(tau_T)
        H._fill(a, dict(C_fg=self.C_fg, T_final=self.T_final, C=self.C, status=self.status,
                        features=self.feat_b))
        return a

    def query_kwargs(self):
        """Arguments of hyrf_query_fields for this view."""
        m = self.m
        e = self.explicit
        return dict(n=m.n, pos=m.pos, alpha_e=m.alpha_e if e else None, scale_e=m.scale_e if e else None,
                    color_e=m.color_e if e else None, cam=self.ccam_q, fields=m.fields_struct(),
                    vis_ids=self.vis_ids, n_vis=self.n_vis, alpha=self.alpha, scale=self.scale, quat=self.quat,
                    color=self.color, status=self.status, features=self.feat_q,
                    explicit_only=0 if self.neural else 1)

    def query_backward_kwargs(self):
        """Arguments of hyrf_query_fields_backward for this view."""
        m = self.m
        e = self.explicit
        return dict(n=m.n, pos=m.pos, alpha_e=m.alpha_e if e else None, scale_e=m.scale_e if e else None,
                    color_e=m.color_e if e else None, cam=self.ccam_q, fields=m.fields_struct(),
                    vis_ids=self.vis_ids, n_vis=self.n_vis, d_alpha=self.d_alpha, d_scale=self.d_scale,
                    d_quat=self.d_quat, d_color=self.d_color, d_pos=m.grad["pos"],
                    d_alpha_e=m.grad["alpha_e"] if e else None, d_scale_e=m.grad["scale_e"] if e else None,
                    d_color_e=m.grad["color_e"] if e else None, grads=m.grads_struct(),
                    loss_scale=self.loss_scale, status=self.status, features=self.feat_q,
                    explicit_only=0 if self.neural else 1)

    def _overlap(self, tau_T=0.0):
        """The background's gather and reverse can run on the side stream
        (unless .serial is set: everything on the caller's stream)."""
        return self.feat_b is not None and self.side is not None and tau_T == 0.0 and not self.serial

    def forward(self, target=None, want_keys=True, tau_T=0.0):
        """The forward path; tau_T > 0 (render only) queries the background
        only where T_final >= tau_T. With the side stream, the depth order
        and the background's feature gather run beside the field query."""
        self.forward_fields(tau_T)
        self.project()
        self.bin_sort(want_keys)
        self.rasterize()
        self.composite(tau_T)
        if target is not None:
            self.loss_fn(target)
        return self.C

    def forward_fields(self, tau_T=0.0):
        """Pre-cull and field query of the Gaussians. With the side stream
        the pre-cull runs first (hyrf_precull); the depth order
        (hyrf_depth_order: positions only) and the background's feature
        gather then run on the side stream while the fields are queried."""
        self._depth_ready = self._overlap(tau_T)
        if not self._depth_ready:
            H.hyrf_query_fields(ws=self.ws["q"], **self.query_kwargs())
            return
        m = self.m
        H.hyrf_precull(ws=self.ws["pc"], n=m.n, pos=m.pos, cam=self.ccam_q, vis_ids=self.vis_ids, n_vis=self.n_vis)
        self.side.wait_stream(torch.cuda.current_stream())  # after the pre-cull and earlier table updates
        H.hyrf_depth_order(ws=self.ws["do"], stream=self.side, n=m.n, pos=m.pos, vis_ids=self.vis_ids,
                           n_vis=self.n_vis, cam=self.ccam, order=self.depth_order, status=self.status)
        self._depth_done.record(self.side)  # the binning waits for this, not for the gather
        H.hyrf_gather_background(self._bg_args(), stream=self.side)
        H.hyrf_query_fields(ws=self.ws["q"], vis_ready=1, **self.query_kwargs())

    def composite(self, tau_T=0.0):
        """The background blend (Eqs. 10-11); with the side stream, after its
        feature gather."""
        bg = self._bg_args(tau_T)
        if self._overlap(tau_T):
            torch.cuda.current_stream().wait_stream(self.side)
            bg.features_ready = 1
        H.call("hyrf_composite_background", bg, self.ws["b"])

    def project(self):
        m = self.m
        H.hyrf_project(ws=self.ws["p"], n=m.n, pos=m.pos, vis_ids=self.vis_ids, n_vis=self.n_vis,
                       scale=self.scale, quat=self.quat, cam=self.ccam, tile=H.TILE,
                       mean2d=self.mean2d, conic=self.conic, depth=self.depth, rect=self.rect,
                       ntiles=self.ntiles, fp64_flag=self.flag, status=self.status, alpha=self.alpha,
                       footprint=self.footprint)

    def bin_sort(self, want_keys=True):
        """Tile binning; takes the side stream's depth order when forward_fields
        started one (identical result)."""
        order = None
        if self._depth_ready:
            torch.cuda.current_stream().wait_event(self._depth_done)
            order = self.depth_order
            self._depth_ready = False  # one binning per depth order
        H.hyrf_bin_sort(ws=self.ws["s"], n=self.m.n, n_vis=self.n_vis, rect=self.rect,
                        ntiles=self.ntiles, depth=self.depth, tiles_x=self.TX, tiles_y=self.TY,
                        capacity=self.capacity, keys=self.keys if want_keys else None,
                        vals=self.vals, ranges=self.ranges, n_instances=self.n_inst,
                        status=self.status, depth_order=order, mean2d=self.mean2d, footprint=self.footprint)

    def loss_fn(self, target, grad=True):
        H.hyrf_loss(ws=self.ws["l"], width=self.W, height=self.H, C=self.C, target=target,
                    lam=self.lam, grad_scale=1.0, loss=self.loss, d_C=self.dC if grad else None)

    # ------------------------------------------------------------- backward
    def backward(self):
        """Reverse of every stage; dL/dC must be in self.dC. Adds into model.grad."""
        self.backward_render()
        self.backward_fields()
        self.join()

    def join(self):
        """Order the caller's stream after the side stream's work (the
        background table scatter of backward_render). Only when the side
        stream is in use: waiting on an idle stream would, during CUDA graph
        capture, depend on work outside the graph."""
        if self._overlap():
            torch.cuda.current_stream().wait_stream(self.side)

    def backward_render(self):
        """Reverse of background, compositing and projection: fills the
        visible Gaussians' dL/d(alpha, scale, quat, color) and adds the
        projection's dL/dpos."""
        m = self.m
        self._dvis.zero_()
        g = m.grads_struct()
        if self._overlap():
            # the background's whole reverse on the side stream, concurrently
            # with the compositing reverse, which takes dL/dT_final T_final
            # from the composited image (C - C_fg = T_final c_s, Eq. 11)
            # instead of waiting for the background's dL/dT_final
            self.side.wait_stream(torch.cuda.current_stream())
            H.hyrf_composite_background_backward(self._bg_args(), ws=self.ws["bb"], stream=self.side,
                                                 d_C=self.dC, d_C_fg=None, d_T_final=None, grads=g,
                                                 loss_scale=self.loss_scale)
            H.hyrf_rasterize_backward(self._raster_args(), ws=self.ws["rb"], d_C_fg=self.dC,
                                      d_T_final=None, C=self.C, d_mean2d=self.d_mean2d,
                                      d_conic=self.d_conic, d_alpha=self.d_alpha, d_color=self.d_color)
        else:
            H.hyrf_composite_background_backward(self._bg_args(), ws=self.ws["bb"], d_C=self.dC,
                                                 d_C_fg=None, d_T_final=self.dT, grads=g,
                                                 loss_scale=self.loss_scale)
            H.hyrf_rasterize_backward(self._raster_args(), ws=self.ws["rb"], d_C_fg=self.dC,
                                      d_T_final=self.dT, d_mean2d=self.d_mean2d, d_conic=self.d_conic,
                                      d_alpha=self.d_alpha, d_color=self.d_color)
        H.hyrf_project_backward(ws=self.ws["p"], n=m.n, pos=m.pos, vis_ids=self.vis_ids,
                                n_vis=self.n_vis, scale=self.scale, quat=self.quat, cam=self.ccam,
                                d_mean2d=self.d_mean2d, d_conic=self.d_conic, d_pos=m.grad["pos"],
                                d_scale=self.d_scale, d_quat=self.d_quat, status=self.status)

    def backward_fields(self):
        """Reverse of the field query (decoders, hash encodings, aggregation)."""
        H.hyrf_query_fields_backward(ws=self.ws["qb"], **self.query_backward_kwargs())

    def step(self, target):
        """One training iteration of the view: forward, loss, backward."""
        self.forward(target)
        self.backward()
        return self.loss

    def check_status(self):
        st = H.read_status(self.status)
        return st

    def fit_capacity(self, target=None, headroom=1.25):
        """Run the forward once and grow the instance capacity until it fits."""
        for _ in range(8):
            self.status.zero_()
            self.forward(target)
            st = H.read_status(self.status)
            if not st & H.HYRF_ERR_OVERFLOW:
                k = int(self.n_inst.item())
                if self.capacity > 3 * int(k * headroom) + (1 << 16):
                    self.set_capacity(int(k * headroom) + (1 << 16))
                    self.status.zero_()
                    self.forward(target)
                return st
            self.set_capacity(self.capacity * 2)
        raise H.HyrfError("instance capacity could not be fitted")


class StepGraph:
    """One iteration of a view captured once as a CUDA graph: training
    (model.zero_grad, forward with the loss over a fixed target buffer,
    every reverse call) or, with train=False, the render-only forward
    (tau_T as in ViewRenderer.forward). Every library call is asynchronous
    on its stream and reads no host value, so the graph replays exactly the
    eager work; replay() launches it on the current stream. Write each
    step's target into .target (same shape, device) before replaying.
    Capture after one eager iteration, so that capacities and workspaces
    are settled; capture again after changing the model's storage (e.g. the
    8-bit codes)."""

    def __init__(self, renderer, target=None, train=True, zero_grad=True, want_keys=False, tau_T=0.0):
        if train and target is None:
            raise ValueError("a training step needs a target buffer")
        self.r = renderer
        self.target = target
        self.graph = torch.cuda.CUDAGraph()
        main = torch.cuda.current_stream()
        cap = torch.cuda.Stream(device=renderer.C.device)
        cap.wait_stream(main)
        n0 = H.launch_count()
        with torch.cuda.stream(cap):
            with torch.cuda.graph(self.graph, stream=cap):
                if train and zero_grad:
                    renderer.m.zero_grad()
                renderer.forward(target if train else None, want_keys=want_keys, tau_T=tau_T)
                if train:
                    renderer.backward()
        main.wait_stream(cap)
        self.launches = H.launch_count() - n0  # library kernels per replay

    def replay(self):
        self.graph.replay()
        return self.r.loss


class Trainer:
    """Training iterations of several views with the fused Adam update
    (hyrf_adam_step). The gradients of all views are accumulated, averaged
    and applied in one launch over every trainable tensor.

    BF16 fields train float32 master copies of the tables and decoder
    weights; the Adam kernel refreshes the bf16 working copies the render
    kernels read. Learning rates (the paper keeps 3DGS's hyper-parameters,
    Sec. 4.1): explicit position 1.6e-4 x the scene extent, opacity 0.05,
    scale 5e-3, colour 2.5e-3 (3DGS); hash tables 1e-2 and decoders 1e-3
    (Instant-NGP); Adam betas (0.9, 0.999), eps 1e-15 for all.
    """

    LR = dict(pos=1.6e-4, alpha_e=0.05, scale_e=5e-3, color_e=2.5e-3, table=1e-2, mlp=1e-3)

    def __init__(self, model: DeviceModel, views, lr=None, betas=(0.9, 0.999), eps=1e-15):
        self.m = model
        self.views = list(views)
        self.betas, self.eps = betas, eps
        self.t = 0
        lr = dict(self.LR, **(lr or {}))
        fl = model.fl
        extent = float(max(fl.box_hi[k] - fl.box_lo[k] for k in range(3)))
        g = model.grad
        z = torch.zeros_like
        self.groups = []

        def add(param, grad, lr_v, shadow=None):
            master = param.float().clone() if shadow is not None else param
            self.groups.append(dict(param=master, grad=grad, m=z(master), v=z(master), shadow=shadow,
                                    lr_scale=lr_v))

        add(model.pos, g["pos"], lr["pos"] * extent)
        add(model.alpha_e, g["alpha_e"], lr["alpha_e"])
        add(model.scale_e, g["scale_e"], lr["scale_e"])
        add(model.color_e, g["color_e"], lr["color_e"])
        for name in ("geo_table", "rad_table"):
            if name == "geo_table" and model.coupled:
                continue  # one grid serves both decoders
            t = getattr(model, name)
            add(t, g[name], lr["table"], shadow=t if model.bf16 else None)
        for W, gW, b, gb in zip(model.geo_W + model.col_W, g["geo_W"] + g["col_W"],
                                model.geo_b + model.col_b, g["geo_b"] + g["col_b"]):
            add(W, gW, lr["mlp"], shadow=W if model.bf16 else None)
            add(b, gb, lr["mlp"])

        self._per_gaussian = 4  # the first four groups are [N]-shaped explicit parameters
        self.reset_stats()

    def reset_stats(self):
        n, d = self.m.n, self.m.device
        self.accum = torch.zeros(max(n, 1), device=d)
        self.count = torch.zeros(max(n, 1), dtype=torch.int32, device=d)

    def step(self, targets):
        """One iteration over all views; returns the per-view loss tensors.
        Also accumulates each view's densification statistics."""
        self.m.zero_grad()
        losses = []
        for r, tgt in zip(self.views, targets):
            r.step(tgt)
            H.hyrf_densify_stats(n=self.m.n, vis_ids=r.vis_ids, n_vis=r.n_vis, d_mean2d=r.d_mean2d,
                                 ntiles=r.ntiles, width=r.W, height=r.H, accum=self.accum, count=self.count)
            losses.append(r.loss)
        self.t += 1
        H.hyrf_adam_step(self.groups, 1.0, self.betas[0], self.betas[1], self.eps, self.t,
                         grad_scale=1.0 / len(self.views))
        return losses

    def reset_opacity(self, opacity=0.01):
        """Periodic reset of the explicit opacity (3DGS: to 0.01)."""
        g = self.groups[1]
        H.hyrf_reset_opacity(self.m.alpha_e, math.log(opacity / (1.0 - opacity)), g["m"], g["v"])

    def densify(self, targets, grad_threshold=2e-4, dense_scale=None, min_opacity=0.005, noise_seed=0):
        """Clone / split / prune (3DGS rules; decisions from the first view's
        last forward) and rebuild every per-Gaussian buffer. Returns the new
        Gaussian count. The views' buffers are re-created and re-fitted."""
        m, r = self.m, self.views[0]
        n, d = m.n, m.device
        fl = m.fl
        extent = float(max(fl.box_hi[k] - fl.box_lo[k] for k in range(3)))
        if dense_scale is None:
            dense_scale = 0.01 * extent  # 3DGS percent_dense x scene extent
        action = torch.empty(n, dtype=torch.uint8, device=d)
        row = torch.empty(n, dtype=torch.int32, device=d)
        offset = torch.empty(n + 1, dtype=torch.int64, device=d)
        n_out = torch.empty(1, dtype=torch.int64, device=d)
        H.hyrf_densify_plan(n=n, vis_ids=r.vis_ids, n_vis=r.n_vis, alpha=r.alpha, scale=r.scale,
                            accum=self.accum, count=self.count, grad_threshold=grad_threshold,
                            dense_scale=dense_scale, min_opacity=min_opacity, action=action, row=row,
                            offset=offset, n_out=n_out)
        n2 = int(n_out.item())
        gen = torch.Generator(device=d)
        gen.manual_seed(noise_seed)
        noise = torch.randn(n, 2, 3, device=d, generator=gen)
        kinds = [H.REMAP_POSITION, H.REMAP_PARAM, H.REMAP_SCALE_LOGIT, H.REMAP_PARAM]
        arrays, new = [], []
        for k, grp in enumerate(self.groups[:self._per_gaussian]):
            p = grp["param"].view(n, -1)
            trio = []
            for src, kind in ((p, kinds[k]), (grp["m"].view(n, -1), H.REMAP_STATE),
                              (grp["v"].view(n, -1), H.REMAP_STATE)):
                dst = torch.empty((n2, src.shape[1]), device=d)
                arrays.append((src, dst, kind))
                trio.append(dst)
            new.append(trio)
        H.hyrf_densify_apply(arrays, n=n, action=action, row=row, offset=offset, scale=r.scale, quat=r.quat,
                             noise=noise, split_log_scale=math.log(1.6))
        shapes = [(n2, 3), (n2,), (n2,), (n2, 3)]
        names = ["pos", "alpha_e", "scale_e", "color_e"]
        for k, (name, (p2, m2, v2)) in enumerate(zip(names, new)):
            p2, m2, v2 = (x.view(shapes[k]).contiguous() for x in (p2, m2, v2))
            setattr(m, name, p2)
            m.grad[name] = torch.zeros_like(p2)
            self.groups[k].update(param=p2, grad=m.grad[name], m=m2, v=v2)
        m.n = n2
        self.reset_stats()
        views = []
        for old, tgt in zip(self.views, targets):
            nr = ViewRenderer(m, old.cam, old.bg, lam=old.lam, loss_scale=old.loss_scale,
                              save_features=old.save_features, workspaces=old.ws)
            nr.fit_capacity(tgt)
            views.append(nr)
        self.views = views
        return n2
