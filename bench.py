"""HyRF hot-path benchmark: fwd+bwd iterations/s and render FPS of one view
of the 1M-Gaussian, 1237x822 workload (16-level 2^19 grids, 2x64 decoders,
exact neural background, L1 loss), on synthetic seeded data, BF16 fields
against the plain FP32 path.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|f32]
  python bench.py --config 1|2          # the plain FP32 workloads (128x128, 800x800)
  python bench.py --config 4|5          # 8-view CUDA-graph step; 6M Gaussians at 1920x1080
  python bench.py --ablation            # Tab. 5 variants
  python bench.py --impl reference ...  # the FP64 CPU oracle on seeded windows of the view

One "step" = gradient zeroing -> pre-cull -> query_fields (the depth order
and the background's feature gather beside it on a second stream) ->
project -> bin_sort -> rasterize -> composite_background -> loss -> every
reverse call (the background's on the second stream), inputs resident in
HBM, replayed as one CUDA graph (pipeline.StepGraph; --no-graph issues the
calls one by one). L2 is flushed (256 MiB write) between timed steps.
Prints one JSON line with the per-kernel rooflines (each kernel on its
binding axis: HBM bytes, tensor FLOPs or FP32 FLOPs), the PSNR of each path
against a teacher image, the end-to-end rate with host buffers and the
oracle timed on the host's cores. Multi-GPU: independent replicas (one view
per rank), no collective.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd iters/s & render FPS, 1M Gaussians @1237x822: BF16-field vs FP32 path"
WORKLOAD = "config3: 1M Gaussians (256 clusters + 10% far), 1237x822, 2x16-level 2^19 hash grids, 32->64->64 decoders, exact background, L1"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="auto", choices=["auto", "bf16", "f32"])
    p.add_argument("--n", type=int, default=1_000_000)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-graph", dest="graph", action="store_false",
                   help="issue every call of the timed step from the host instead of replaying the "
                        "step captured as one CUDA graph")
    p.add_argument("--cpu-sample-s", type=float, default=15.0)
    p.add_argument("--layout", default="morton", choices=["input", "morton"],
                   help="storage order of the Gaussians: morton = hyrf_spatial_order once at load (a "
                        "layout step outside the timed region), input = the generator's random order")
    p.add_argument("--config", type=int, default=3, choices=[1, 2, 3, 4, 5],
                   help="3: the headline line; 1, 2: the plain FP32 workloads (4,096 Gaussians at "
                        "128x128, 200k at 800x800); 4: 8-view step as one CUDA graph (3M Gaussians, "
                        "memory saved vs recompute); 5: 6M Gaussians at 1920x1080 with 1%% degenerate ones")
    p.add_argument("--ablation", action="store_true",
                   help="render FPS and fwd+bwd it/s of the Tab. 5 ablations on the 360-degree variant")
    return p.parse_args()


def replica_max(x, device="cpu"):
    """The maximum of x over the ranks of the default process group (the
    slowest replica sets the step time)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(ms_per_step, n_replicas):
    """Iterations per second of the whole job: every replica runs its own
    view, all finish within the slowest one's step time."""
    return n_replicas * 1000.0 / ms_per_step


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, out_dir=None):
        """Samples go to <out_dir>/clocks_rank<i>.csv (default: the system's
        temporary directory); the JSON line carries their summary."""
        self.idx = gpu_index
        self.proc = None
        out_dir = out_dir or os.environ.get("HYRF_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            t0 = time.time()
            while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nme, v in zip(names, parts[5:9]):
                if v.lower() in ("active", "0x1", "1"):
                    reasons.add(nme)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- workloads

# The single-view workloads bench.py times (--config 1, 2, 3; 3 is the
# headline line): metric, workload description and image size.
CONFIGS = {
    1: dict(metric="fwd+bwd iters/s & render FPS, 4,096 Gaussians @128x128: plain FP32 path",
            workload="config1: 4,096 Gaussians uniform in [-1,1]^2 x [2,4], 128x128 (fx = 128), 2x8-level "
                     "2^12 hash grids, 16->32->out decoders, 16x16 background map, L1",
            image="128x128", precisions=("f32",)),
    2: dict(metric="fwd+bwd iters/s & render FPS, 200k Gaussians @800x800: plain FP32 path",
            workload="config2: 200k Gaussians (64 clusters + 10% far at depth 20-100), 800x800 at 60 deg, "
                     "2x16-level 2^17 hash grids, 32->64->64 decoders, 64x128 background map, "
                     "0.8 L1 + 0.2 D-SSIM",
            image="800x800", precisions=("f32",)),
    3: dict(metric=METRIC, workload=WORKLOAD, image="1237x822", precisions=("bf16", "f32")),
}


def make_workload(config, n, precision, seed=0):
    """Seeded synthetic workload of a config (generators only)."""
    from paper_2509_17083_gb300 import synth
    if config == 1:
        return synth.config1(seed=seed)
    if config == 2:
        return synth.config2(seed=seed)
    return synth.config3(n=n, precision=precision, seed=seed)


def bench_config(args):
    """The `config` object of the JSON line (identical in both arms)."""
    c = CONFIGS[args.config]
    n = {1: 4096, 2: 200_000}.get(args.config, args.n)
    return {"workload": c["workload"], "gaussians": n, "image": c["image"],
            "l2": "flushed between timed steps (256 MiB write)"}


# ---------------------------------------------------------------- algorithmic work per kernel

# FP32 operations (FLOPs, a fused multiply-add counted as 2) per evaluated
# (pixel, Gaussian) pair of the compositing, from Eq. 1 as written:
#   forward: offset d = mean - pixel (2); exponent -1/2 (a dx^2 + c dy^2) -
#   b dx dy (9); alpha = min(0.99, o G) (2); the skip and stop tests with
#   T (1 - alpha) (4); C += c alpha T (7): 24, plus one exponential;
#   reverse: the same exponent and alpha (13), T before the Gaussian by
#   division (2), the colour behind S (3), c . dL/dC (5), dL/dc += alpha T
#   dL/dC (7), dL/dalpha (4), dL/dopacity (2), dL/dpower and its three
#   moments over the pixels (6): 42, plus one exponential.
# The pairs are those up to each pixel's last contributor (sum of n_contrib).
FP32_FLOPS_PER_PAIR = {"k_raster_fwd": 24, "k_raster_bwd": 42}


def decoder_macs(mlp):
    """Multiply-accumulates of one decoder evaluation (Eqs. 4 and 6)."""
    dims = [mlp.n_in] + [mlp.width] * mlp.n_hidden + [mlp.n_out]
    return sum(a * b for a, b in zip(dims, dims[1:]))


def kernel_work(nv, K, P, tiles, bf16, pairs=0, macs=(0, 0), active=None):
    """Algorithmic work per launch of the main kernels on the axis that
    bounds each: ("hbm", bytes) for the gathers, scatters, field kernels of
    the FP32 path and the sort (every input read once, every output written
    once, a table-gradient atomic counted as its 8-byte payload); ("tensor",
    FLOPs) for the decoders on the tensor cores (2 per multiply-accumulate;
    the reverse recomputes the forward and forms dX and dW: 3x); ("alu",
    FP32 FLOPs) for the compositing (FP32_FLOPS_PER_PAIR). Units: visible
    Gaussian (nv), tile instance (K), pixel (P), evaluated pair (pairs);
    macs = (geometry, colour) decoder multiply-accumulates per row; active =
    visible Gaussians with a non-zero upstream gradient (the Gaussian
    decoders' reverse and the scatter run on those rows only: the others
    add exactly zero)."""
    active = nv if active is None else active
    L = 16
    ent = 4 if bf16 else 8                     # bytes per 2-feature table entry
    gather = L * 8 * ent                       # one field, 8 corners per level
    scatter = L * 8 * 8                        # one field, float2 atomic per corner
    feat, dfeat = 64, 128                      # bf16 features / f32 gradients per row and field
    mg, mc = macs
    hbm = {
        # FP32 fused field kernels: vis id, position, both fields, explicit
        # params (20 B), outputs (44 B)
        "k_query_fwd": nv * (4 + 12 + 2 * gather + 20 + 44),
        # BF16 split path. gather: vis id, position, 8 corners x 16 levels per
        # field, features written
        "k_gather<gaussians>": nv * (4 + 12 + 2 * (gather + feat)),
        "k_gather<pixels>": P * (gather + feat),
        # scatter: feature gradients in, float2 atomics, corner values re-read
        # for dL/dp (Gaussians), d_pos RMW; rows without gradient read their
        # feature gradients only
        # (the rows with a gradient only: list, feature gradients, atomics)
        "k_scatter<gaussians>": active * (4 + 4 + 12 + 2 * (dfeat + scatter + gather) + 24),
        "k_scatter<pixels>": P * (dfeat + scatter),
        # radix scatter: 4-B key and 4-B value read and written per element
        # (depth passes over the visible Gaussians, tile passes over the
        # instances)
        "k_radix_scatter<depth>": nv * 16,
        "k_radix_scatter<tile>": K * 16,
        # instance expansion: offsets and depth order read per Gaussian, key
        # and value written per instance
        "k_expand": nv * 8 + K * 8,
    }
    tensor = {
        "k_query_fwd_tc": nv * (mg + mc) * 2,
        "k_bg_exact_fwd_tc": P * mc * 2,
        # the Gaussian reverse runs on the rows with a gradient only
        "k_decoder_bwd_tc<GeoGauss>": active * mg * 3 * 2,
        "k_decoder_bwd_tc<ColGauss>": active * mc * 3 * 2,
        "k_decoder_bwd_tc<BgPixel>": P * mc * 3 * 2,
    }
    alu = {k: pairs * f for k, f in FP32_FLOPS_PER_PAIR.items()}
    if not bf16:
        # the FP32 path's register-tiled decoders: 2 FP32 FLOPs per
        # multiply-accumulate, the reverse 3x (recomputed forward, dX, dW)
        alu.update({"k_query_dec_f32<geo>": nv * mg * 2, "k_query_dec_f32<col>": nv * mc * 2,
                    "k_bg_dec_f32": P * mc * 2, "k_bg_dec_bwd_f32": P * mc * 3 * 2,
                    "k_query_dec_bwd_f32<geo>": active * mg * 3 * 2,
                    "k_query_dec_bwd_f32<col>": active * mc * 3 * 2})
    out = {k: ("hbm", v) for k, v in hbm.items()}
    if bf16:
        out.update({k: ("tensor", v) for k, v in tensor.items()})
    out.update({k: ("alu", v) for k, v in alu.items()})
    return out


def fp32_peak_tflops(sm_mhz, n_sm):
    """FP32 peak of the GPU at the sampled SM clock: SMs x 128 FP32 lanes x 2
    FLOPs per fused multiply-add per clock (Blackwell SM: four partitions of
    32 FP32 lanes)."""
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the named kernel on this workload; an entry is removed when
# the kernel changes after its capture.
NCU_TRAFFIC = {
    # the compositing reverse (one launch of the step driver's config-3
    # training step, footprint-culled lists, paired two-pixel reverse):
    # 55,583,488 B read + 327,168 B written
    ("k_raster_bwd", "bf16"): 55_910_656,
}


def rooflines(R, peaks, prec, sm_mhz, n_sm):
    """Roofline of every kernel that has a work figure, from the library's
    own CUDA-event kernel timer over the steps of the timer pass (the timed
    step's calls issued on one stream), each on its binding axis: HBM GB/s
    against the measured copy bandwidth, tensor TFLOP/s against the measured
    sustained bf16 GEMM rate, FP32 TFLOP/s against the FP32 peak at the
    sampled clock. Returns (the dominant kernel's entry with the table
    under "per_kernel")."""
    hbm = peaks.get("hbm_gbs")
    hsrc = "of measured" if hbm else "of fallback"
    hbm = hbm or 6800.0
    ten = peaks.get("bf16_tflops_sustained")
    tsrc = "of measured (sustained)" if ten else "of fallback"
    ten = ten or 1700.0
    mhz = sm_mhz or peaks.get("sm_max_mhz") or 2070.0
    alu = fp32_peak_tflops(mhz, n_sm)
    table = {}
    for k, (n, avg_ms) in R["kernels"].items():
        if k not in R["work"]:
            continue
        axis, work = R["work"][k]
        if axis == "hbm":
            ach, peak, unit, src = work / (avg_ms * 1e-3) / 1e9, hbm, "GB/s", hsrc
        elif axis == "tensor":
            ach, peak, unit, src = work / (avg_ms * 1e-3) / 1e12, ten, "TFLOP/s", tsrc
        else:
            ach, peak, unit, src = work / (avg_ms * 1e-3) / 1e12, alu, "TFLOP/s", (
                f"derived: {n_sm} SMs x 128 FP32 lanes x 2 x {mhz:.0f} MHz (sampled median)")
        table[k] = {"bound": axis, "achieved": round(ach, 2), "peak": round(peak, 1), "unit": unit,
                    "frac": round(ach / peak, 4), "work_per_launch": int(work), "avg_launch_ms": round(avg_ms, 4),
                    "ms_per_step": round(n * avg_ms, 4), "peak_source": src,
                    "traffic": NCU_TRAFFIC.get((k, prec))}
    if not table:
        return {"kernel": None, "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s",
                "frac": None, "traffic": None, "per_kernel": {}}
    top = max(table, key=lambda k: table[k]["ms_per_step"])
    head = dict(table[top])
    head["kernel"] = top
    head["per_kernel"] = table
    return head


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    from paper_2509_17083_gb300 import hyrf as H
    from paper_2509_17083_gb300 import synth
    from paper_2509_17083_gb300.pipeline import DeviceModel, StepGraph, ViewRenderer

    ws, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(dev))
    H.lib()
    cfg = CONFIGS[args.config]
    precisions = [p for p in cfg["precisions"] if args.precision in ("auto", p)]
    if not precisions:
        raise SystemExit(f"config {args.config} has no {args.precision} path")
    results = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sampler = ClockSampler(local)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # teacher image: the scene with its explicit colour and opacity logits
    # moved (synth.teacher_of), rendered once on the FP32 path; the PSNR of
    # each path's render against it, and of the renders against each other,
    # measure what the reduced precision costs in image quality
    tw = synth.teacher_of(make_workload(args.config, args.n, "f32", seed=local))
    tm = DeviceModel(tw, device=dev)
    tr = ViewRenderer(tm, tw.cams[0], tw.bg)
    tr.fit_capacity()
    teacher = tr.forward(None).clone()
    del tr, tm, tw
    images = {}
    for prec in precisions:
        w = make_workload(args.config, args.n, prec, seed=local)
        m = DeviceModel(w, device=dev)
        if args.layout == "morton":
            m.spatial_order()  # one-time layout step at load, outside the timed region
        r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
        tgt = torch.as_tensor(w.targets[0]).to(dev)
        try:
            r.fit_capacity(tgt)
        except H.HyrfError as e:
            if prec == "bf16":
                results[prec] = {"unavailable": str(e)}
                continue
            raise
        stream = torch.cuda.current_stream()
        names = ["query_fwd", "project_fwd", "bin_sort", "raster_fwd", "bg_fwd", "loss",
                 "render_bwd", "query_bwd"]
        ev = {k: [] for k in names}

        def timed_step(record):
            m.zero_grad()
            evs = {}

            def mark(k):
                if record:
                    e0 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    evs.setdefault(k, []).append(e0)
            mark("query_fwd")
            r.forward_fields()
            mark("query_fwd"); mark("project_fwd")
            r.project()
            mark("project_fwd"); mark("bin_sort")
            r.bin_sort(want_keys=False)
            mark("bin_sort"); mark("raster_fwd")
            r.rasterize()
            mark("raster_fwd"); mark("bg_fwd")
            r.composite()
            mark("bg_fwd"); mark("loss")
            r.loss_fn(tgt)
            mark("loss")
            # reverse of background, compositing and projection (the
            # background's on the second stream), then of the field query
            mark("render_bwd")
            r.backward_render()
            mark("render_bwd"); mark("query_bwd")
            r.backward_fields()
            r.join()
            mark("query_bwd")
            return evs

        for _ in range(max(3, args.warmup)):
            timed_step(False)
        torch.cuda.synchronize()
        # the step as one CUDA graph (the pipeline's StepGraph: zero_grad,
        # forward with the loss, every reverse call), over a fixed target
        sg = StepGraph(r, tgt) if args.graph else None
        for _ in range(3 if sg else 0):
            sg.replay()
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()
        l0 = H.launch_count()
        step_ms = []
        if prec == precisions[0]:
            sampler.start()
        t_wall = time.perf_counter()
        for _ in range(args.steps):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if sg:
                sg.replay()
            else:
                evs = timed_step(True)
            e1.record(stream)
            torch.cuda.synchronize()
            step_ms.append(e0.elapsed_time(e1))
            if not sg:
                for k, (a, b) in evs.items():
                    ev[k].append(a.elapsed_time(b))
        t_wall = time.perf_counter() - t_wall
        launches = sg.launches * args.steps if sg else H.launch_count() - l0
        # eager issue of the same step with stage marks: stage times, and the
        # step time without the graph
        eager_ms = []
        for _ in range(max(3, args.steps // 2) if sg else 0):
            flush.fill_(1)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            evs = timed_step(True)
            e1.record(stream)
            torch.cuda.synchronize()
            eager_ms.append(e0.elapsed_time(e1))
            for k, (a, b) in evs.items():
                ev[k].append(a.elapsed_time(b))
        # the same steps again, every call on one stream (so that no kernel
        # shares the GPU with another), with the library's kernel timer on
        # (CUDA events around every launch, on its stream): per-kernel
        # durations
        r.serial = True
        for _ in range(3):
            timed_step(False)
        H.hyrf_timer_read()
        H.hyrf_timer_enable(True)
        for _ in range(args.steps):
            flush.fill_(1)
            timed_step(False)
        torch.cuda.synchronize()
        H.hyrf_timer_enable(False)
        r.serial = False
        ktimes = H.hyrf_timer_read()
        clocks = sampler.stop() if prec == precisions[0] else None
        st = H.read_status(r.status)
        nv = int(r.n_vis.item())
        K = int(r.n_inst.item())
        ms = float(np.mean(step_ms))
        if ws > 1:
            ms = replica_max(ms, dev)
        def render_ms(rr, tau_T=0.0):
            """Mean forward-only time (render FPS), same flush protocol; the
            forward replayed as one CUDA graph unless --no-graph."""
            for _ in range(3):
                rr.forward(None, want_keys=False, tau_T=tau_T)
            g = StepGraph(rr, train=False, tau_T=tau_T) if args.graph else None
            out = []
            for i in range(3 + max(3, args.steps // 2)):
                flush.fill_(1)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                if g:
                    g.replay()
                else:
                    rr.forward(None, want_keys=False, tau_T=tau_T)
                e1.record(stream)
                torch.cuda.synchronize()
                if i >= 3:
                    out.append(e0.elapsed_time(e1))
            return float(np.mean(out))

        # render-only (forward, no backward)
        fwd_ms = [render_ms(r)]
        # render-time background skip (tau_T = 0.2, the paper's value; BF16 only)
        tau_ms = [render_ms(r, 0.2)] if prec == "bf16" else []
        # the 8-bit grid codec (render only)
        u8_ms = []
        if prec == "bf16":
            m.quantize_u8()
            u8_ms = [render_ms(r)]
            m.quantize_u8(False)
        # the IEEE-half render path (f16 grids and decoders), same scene
        f16_ms = []
        if prec == "bf16":
            wf = synth.config3(n=args.n, precision="f16", seed=local)
            mf = DeviceModel(wf, device=dev)
            if args.layout == "morton":
                mf.spatial_order()
            rf = ViewRenderer(mf, wf.cams[0], wf.bg)
            rf.fit_capacity()
            f16_ms = [render_ms(rf)]
            del rf, mf
        # end to end through the pipeline API with host buffers: the step's
        # target copied host -> device into the graph's target buffer, the
        # step replayed, its loss copied device -> host
        pinned = torch.as_tensor(w.targets[0]).pin_memory()
        dev_tgt = sg.target if sg else torch.empty_like(tgt)
        host_loss = torch.empty(1, dtype=torch.float32).pin_memory()
        torch.cuda.synchronize()
        e2e_ms = []
        for _ in range(max(3, args.steps // 2)):
            flush.fill_(1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dev_tgt.copy_(pinned, non_blocking=True)
            if sg:
                sg.replay()
            else:
                r.forward(dev_tgt, want_keys=False)
                m.zero_grad()
                r.backward()
            host_loss.copy_(r.loss, non_blocking=True)
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        del sg
        stage_ms = {k: float(np.mean(v)) for k, v in ev.items() if v}
        r.forward(None, want_keys=False)
        torch.cuda.synchronize()
        C = r.C.float().clamp(0, 1).clone()
        images[prec] = C
        psnr = float(-10.0 * torch.log10(((C - teacher.clamp(0, 1)) ** 2).mean()).item())
        evals = int(r.n_contrib.sum().item())
        active = int(((r.d_alpha[:nv] != 0) | (r.d_color[:nv] != 0).any(1) | (r.d_scale[:nv] != 0).any(1)
                      | (r.d_quat[:nv] != 0).any(1)).sum().item())
        fl = w.fields
        results[prec] = dict(ms=ms, fwd_ms=float(np.mean(fwd_ms)), e2e_ms=float(np.mean(e2e_ms)),
                             eager_ms=float(np.mean(eager_ms)) if eager_ms else None,
                             tau_ms=float(np.mean(tau_ms)) if tau_ms else None,
                             u8_ms=float(np.mean(u8_ms)) if u8_ms else None,
                             f16_ms=float(np.mean(f16_ms)) if f16_ms else None,
                             stage_ms=stage_ms, launches_per_step=launches / args.steps,
                             n_vis=nv, instances=K, status=st, clocks=clocks, wall_s=t_wall,
                             loss=float(r.loss.item()),
                             h2d=int(pinned.numel() * 4), d2h=4, psnr=psnr, evals=evals,
                             kernels={k: (n / args.steps, t / n) for k, (n, t) in ktimes.items()},
                             work=kernel_work(nv, K, w.cams[0].width * w.cams[0].height,
                                              int(r.ranges.shape[0]), prec == "bf16", pairs=evals,
                                              macs=(decoder_macs(fl.geo_mlp), decoder_macs(fl.col_mlp)),
                                              active=active),
                             active=active)
        del r, m
        torch.cuda.empty_cache()
    head = "bf16" if "bf16" in results and "ms" in results["bf16"] else "f32"
    R = results[head]
    value = whole_job_rate(R["ms"], ws)
    roof = rooflines(R, peaks, head, (R["clocks"] or {}).get("sm_mhz"), n_sm)
    per_step = {k: n * t for k, (n, t) in R["kernels"].items()}
    tot = sum(per_step.values()) or 1.0
    top = sorted(per_step, key=per_step.get, reverse=True)[:12]
    kern = {k: {"ms_per_step": round(per_step[k], 4), "share": round(per_step[k] / tot, 4),
                "launches_per_step": round(R["kernels"][k][0], 2)} for k in top}
    rf = R["kernels"].get("k_raster_fwd")
    R_run_extra = {"gaussians_with_gradient": R.get("active")}
    out = {"metric": cfg["metric"], "value": round(value, 3), "unit": "iters/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(R["ms"], 4),
           "step_issue": "one CUDA graph per step" if args.graph else "eager",
           "eager_ms_per_step": round(R["eager_ms"], 4) if R.get("eager_ms") else None,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16" if head == "bf16" else "f32", "data": "synthetic",
           "config": bench_config(args),
           "run": {"precision": head, "visible": R["n_vis"], "instances": R["instances"],
                   "layout": args.layout, "parallelism": f"replicas x{ws}", "view": (
                       "one fixed camera: each forward takes its tiles in the order of the previous "
                       "replay's pixel lists, which on a fixed view are the current ones"), **R_run_extra},
           "render_fps": round(ws * 1000.0 / R["fwd_ms"], 2),
           "render_fps_tau_T_0.2": round(ws * 1000.0 / R["tau_ms"], 2) if R.get("tau_ms") else None,
           "render_fps_u8_grids": round(ws * 1000.0 / R["u8_ms"], 2) if R.get("u8_ms") else None,
           "render_fps_f16_fields": round(ws * 1000.0 / R["f16_ms"], 2) if R.get("f16_ms") else None,
           "stage_ms": {k: round(v, 4) for k, v in R["stage_ms"].items()},
           "kernels": kern,
           "psnr_db": round(R["psnr"], 4),
           "psnr_definition": ("PSNR of the path's render against a teacher image: the same scene with "
                               "its explicit colour and opacity logits moved by N(0, 0.3^2) draws, "
                               "rendered on the FP32 path"),
           "gaussian_pixel_evals_per_s": (round(R["evals"] / (rf[1] * 1e-3), 1) if rf else None),
           "e2e": {"value": round(ws * 1000.0 / R["e2e_ms"], 3), "unit": "iters/s",
                   "h2d_bytes_per_step": R["h2d"], "d2h_bytes_per_step": R["d2h"]},
           "gpu_launches": int(round(R["launches_per_step"] * args.steps)),
           "roofline": roof, "clocks": R["clocks"], "device_status": R["status"]}
    for p, v in results.items():
        if p != head:
            out[f"{p}_path"] = ({"iters_per_s": round(1000.0 / v["ms"], 3),
                                 "render_fps": round(1000.0 / v["fwd_ms"], 2),
                                 "psnr_db": round(v["psnr"], 4),
                                 "stage_ms": {k: round(x, 4) for k, x in v["stage_ms"].items()}}
                                if "ms" in v else v)
            if "psnr" in v:
                out["delta_psnr_db"] = round(R["psnr"] - v["psnr"], 5)
    if len(images) == 2:
        a, b = images.values()
        out["psnr_bf16_vs_f32_db"] = round(float(-10.0 * torch.log10(((a - b) ** 2).mean()).item()), 3)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, budget_s=args.cpu_sample_s)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# ---------------------------------------------------------------- configs 4 and 5 (multi-view, large)

def run_config(args):
    """Configs 4 and 5 (one JSON line each): the 8-view step as one CUDA graph
    with and without saved features (peak device memory of each), and the
    6M-Gaussian 1920x1080 view (fwd+bwd iterations/s and render FPS)."""
    import torch
    from paper_2509_17083_gb300 import hyrf as H
    from paper_2509_17083_gb300 import synth
    from paper_2509_17083_gb300.pipeline import DeviceModel, StepGraph, ViewRenderer, shared_workspaces

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    H.lib()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    steps = max(5, args.steps // 4)
    warm = max(3, args.warmup)
    sampler = ClockSampler(0)

    def timed(fn, k):
        for _ in range(warm):
            fn()
        ms = []
        for _ in range(k):
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return float(np.mean(ms))

    common = {"n_gpus": 1, "steps": steps, "warmup": warm, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "bf16", "data": "synthetic"}
    if args.config == 5:
        w = synth.config5()
        m = DeviceModel(w)
        m.spatial_order()
        r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
        tgt = torch.as_tensor(w.targets[0]).cuda()
        r.fit_capacity(tgt)
        for _ in range(3):
            m.zero_grad()
            r.step(tgt)
        torch.cuda.synchronize()
        sg = StepGraph(r, tgt)
        sampler.start()
        ms = timed(sg.replay, steps)
        del sg
        fwd_g = StepGraph(r, train=False)
        fwd = timed(fwd_g.replay, steps)
        del fwd_g
        tau_g = StepGraph(r, train=False, tau_T=0.2)
        tau = timed(tau_g.replay, steps)
        clocks = sampler.stop()
        del tau_g
        out = {"metric": "fwd+bwd iters/s & render FPS, 6M Gaussians @1920x1080, BF16 fields",
               "value": round(1000 / ms, 3), "unit": "iters/s", "ms_per_step": round(ms, 3), **common,
               "render_fps": round(1000 / fwd, 2), "render_fps_tau_T_0.2": round(1000 / tau, 2),
               "config": {"workload": "config5: 6M Gaussians (1024 clusters, 40% at depth 50-100, 1% "
                                      "near-degenerate with scale ratio 1e4), 1920x1080 at 60 deg, 2x16-level "
                                      "2^22 hash grids, 32->64->64 decoders, exact background, L1",
                          "gaussians": w.gaussians.n, "image": "1920x1080",
                          "l2": "flushed between timed steps (256 MiB write)"},
               "run": {"visible": int(r.n_vis.item()), "instances": int(r.n_inst.item()), "layout": "morton",
                       "step_issue": "one CUDA graph per step"},
               "device_status": H.read_status(r.status), "clocks": clocks}
        print(json.dumps(out))
        return
    # config 4: 8 views, one CUDA graph per step; saved features vs recompute
    res = {}
    sampler.start()
    for save in (True, False):
        torch.cuda.empty_cache()
        torch.cuda.reset_peak_memory_stats()
        w = synth.config4()
        m = DeviceModel(w)
        m.spatial_order()
        ws = shared_workspaces()
        views = []
        for cam, t in zip(w.cams, w.targets):
            r = ViewRenderer(m, cam, w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale, save_features=save,
                             workspaces=ws)
            tt = torch.as_tensor(t).cuda()
            r.fit_capacity(tt)
            views.append((r, tt))

        def step():
            m.zero_grad()
            for r, tt in views:
                r.step(tt)
        step()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                step()
        torch.cuda.current_stream().wait_stream(side)
        ms = timed(g.replay, steps)
        st = max(H.read_status(r.status) for r, _ in views)
        res["saved" if save else "recompute"] = dict(ms_per_step=round(ms, 3), views_per_s=round(8000 / ms, 2),
                                                     peak_gib=round(torch.cuda.max_memory_allocated() / 2**30, 2),
                                                     device_status=st)
        del g, views, m
    clocks = sampler.stop()
    print(json.dumps({"metric": "8-view fwd+bwd step as one CUDA graph, 3M Gaussians @1297x840, BF16 fields",
                      "value": res["saved"]["views_per_s"], "unit": "views/s",
                      "ms_per_step": res["saved"]["ms_per_step"], **common,
                      "config": {"workload": "config4: 3M Gaussians (1024 clusters in a radius-2 ball), 8 cameras "
                                             "on a ring of radius 4, 1297x840 at 60 deg, 2x16-level 2^21 hash "
                                             "grids, 32->64->64 decoders, exact background, L1",
                                 "gaussians": 3_000_000, "image": "1297x840 x 8 views",
                                 "l2": "flushed between timed steps (256 MiB write)"},
                      "run": {"layout": "morton", "step_issue": "one CUDA graph per 8-view step",
                              "tile_order": "each view keeps the tile order of its own previous forward"},
                      "features": res, "clocks": clocks}))


# ---------------------------------------------------------------- ablations (Tab. 5)

# The paper's Tab. 5 render FPS (Tanks & Temples, RTX 3090), for the ratios.
PAPER_TAB5_FPS = {"full": 106, "w/o Decouple.": 101, "w/o Explicit": 121, "w/o Neural": 127,
                  "w/o Background": 112, "w/o Pre-culling": 27}


def run_ablation(args):
    import torch
    from paper_2509_17083_gb300 import hyrf as H
    from paper_2509_17083_gb300 import synth
    from paper_2509_17083_gb300.pipeline import DeviceModel, ViewRenderer

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    H.lib()
    w = synth.config3_360(n=args.n, precision="bf16")
    tgt = torch.as_tensor(w.targets[0]).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    variants = [("full", {}, False), ("w/o Decouple.", {}, True), ("w/o Explicit", dict(explicit=False), False),
                ("w/o Neural", dict(neural=False), False), ("w/o Background", dict(background=False), False),
                ("w/o Pre-culling", dict(precull=False), False)]
    steps = max(5, args.steps // 4)
    out = {}
    for name, kw, coupled in variants:
        wv = w
        if not kw.get("explicit", True):
            # without explicit parts the decoders' output biases carry the
            # explicit initial values (mean logits), so that the neural-only
            # Gaussians start with the same opacities, sizes and colours
            import dataclasses
            fl = w.fields
            gb = [b.copy() for b in fl.geo_mlp.b]
            gb[-1][0] += float(np.mean(w.gaussians.alpha_e))
            gb[-1][1:4] += float(np.mean(w.gaussians.scale_e))
            wv = dataclasses.replace(w, fields=dataclasses.replace(
                fl, geo_mlp=dataclasses.replace(fl.geo_mlp, b=gb)))
        m = DeviceModel(wv, coupled=coupled)
        r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale, **kw)
        r.fit_capacity(tgt)
        res = {}
        for mode in ("render", "train"):
            for _ in range(3):
                r.forward(tgt) if mode == "render" else r.step(tgt)
            times = []
            for _ in range(steps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                if mode == "render":
                    r.forward(None, want_keys=False)
                else:
                    m.zero_grad()
                    r.step(tgt)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            res["render_fps" if mode == "render" else "iters_per_s"] = round(1000.0 / float(np.mean(times)), 2)
        res["visible"] = int(r.n_vis.item())
        res["status"] = H.read_status(r.status)
        out[name] = res
        del r, m
        torch.cuda.empty_cache()
    base = out["full"]
    for name, res in out.items():
        res["fps_ratio"] = round(res["render_fps"] / base["render_fps"], 3)
        res["its_ratio"] = round(res["iters_per_s"] / base["iters_per_s"], 3)
        res["paper_fps_ratio"] = round(PAPER_TAB5_FPS[name] / PAPER_TAB5_FPS["full"], 3)
    print(json.dumps({"metric": "Tab. 5 ablations: render FPS and fwd+bwd iters/s, BF16 fields",
                      "config": {"workload": "config3 scene replicated around the camera (360 deg, ~25 % "
                                             "in view), 1M Gaussians, 1237x822, 2^19 grids",
                                 "steps": steps, "l2": "flushed between timed steps"},
                      "variants": out}))


# ---------------------------------------------------------------- oracle arm

def cpu_info():
    """Host cores this process may use, and the CPU model."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    import platform
    return cores, model or platform.processor() or platform.machine()


# oracle sample windows: CROP_W x CROP_H windows of the view (the camera's
# principal point shifted; config 1's whole 128x128 view is one window); a
# window's pre-cull band, visible set, instances, pixels and background scale
# with its area like the full view's
CROP_W, CROP_H = 96, 64
_W_CACHE = {}


def _crop(config):
    return (128, 128) if config == 1 else (CROP_W, CROP_H)


def _oracle_windows(job):
    """FP64 oracle forward, loss and full reverse (oracle.loss_and_grads) of
    the given windows of a config's workload, one after the other on one
    core; returns [(pixels, seconds)] per window. Runs in a spawned worker
    process or in-process; the workload is generated once per process."""
    config, n, prec, windows = job
    import dataclasses as dc

    import oracle
    key = (config, n, prec)
    if key not in _W_CACHE:
        _W_CACHE.clear()
        _W_CACHE[key] = make_workload(config, n, prec)
    w = _W_CACHE[key]
    cam = w.cams[0]
    out = []
    CW, CH = _crop(config)
    for x0, y0 in windows:
        cw, ch = min(CW, cam.width - x0), min(CH, cam.height - y0)
        wc = dc.replace(cam, cx=cam.cx - x0, cy=cam.cy - y0, width=cw, height=ch)
        tgt = np.ascontiguousarray(w.targets[0][y0:y0 + ch, x0:x0 + cw])
        t = time.perf_counter()
        oracle.loss_and_grads(w.gaussians, w.fields, wc, w.bg, tgt, w.ssim_lambda)
        out.append((cw * ch, time.perf_counter() - t))
    return out


def _warm(job):
    """Generate the workload in a worker (untimed)."""
    _oracle_windows(tuple(job) + ([],))
    return os.getpid()


def _windows(config, n, rng, k):
    """k windows at seeded positions (window origins on the view)."""
    W, H = {1: (128, 128), 2: (800, 800)}.get(config, (1237, 822))
    CW, CH = _crop(config)
    return [(int(rng.integers(0, max(1, W - CW + 1))), int(rng.integers(0, max(1, H - CH + 1))))
            for _ in range(k)]


class OraclePool:
    """Worker processes (spawned: no fork after CUDA is initialised) that run
    the oracle on windows in parallel, one window per core at a time."""

    def __init__(self, config, n, prec, procs):
        import multiprocessing as mp
        self.job = (config, n, prec)
        self.procs = procs
        self.pool = mp.get_context("spawn").Pool(procs)
        self.pool.map(_warm, [self.job] * procs, chunksize=1)

    def run(self, windows):
        """Windows split over the workers; returns (pixels, wall seconds)."""
        parts = [windows[i::self.procs] for i in range(self.procs)]
        t = time.perf_counter()
        res = self.pool.map(_oracle_windows, [self.job + (p,) for p in parts if p], chunksize=1)
        wall = time.perf_counter() - t
        return sum(px for r in res for px, _ in r), wall

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_baseline(args, budget_s=15.0):
    """The FP64 oracle as it stands (oracle.loss_and_grads: forward, loss and
    the reverse of every stage, on the field outputs it computes itself), on
    a bounded sample of the workload: seeded CROP_W x CROP_H windows of the
    view, timed on one core (in-process, one window after another) and on
    every host core (one spawned process per core, one window each at a
    time); seconds per pixel scaled to the full view give iterations/s."""
    cfg = CONFIGS[args.config]
    prec = "bf16" if "bf16" in cfg["precisions"] and args.precision != "f32" else "f32"
    n = bench_config(args)["gaussians"]
    W, H = [int(x) for x in cfg["image"].split("x")]
    P = W * H
    rng = np.random.default_rng(7)
    cores, model = cpu_info()
    t_all = time.perf_counter()
    _oracle_windows((args.config, n, prec, []))  # workload generation, untimed
    # one core, in this process
    px1 = sec1 = 0.0
    k1 = 0
    while sec1 < budget_s / 2 or k1 < 2:
        r = _oracle_windows((args.config, n, prec, _windows(args.config, n, rng, 1)))
        px1 += r[0][0]
        sec1 += r[0][1]
        k1 += 1
        if k1 >= 64:
            break
    one = 1.0 / (sec1 / px1 * P)
    # every core, spawned workers
    pool = OraclePool(args.config, n, prec, cores)
    per = max(1, int(round(budget_s / 2 / max(sec1 / k1, 1e-3))))
    pxn, wall = pool.run(_windows(args.config, n, rng, per * cores))
    pool.close()
    many = 1.0 / (wall / pxn * P)
    return {"value": round(many, 6), "unit": "iters/s", "cores": cores, "kind": "oracle",
            "cpu_model": model,
            "sample": (f"FP64 oracle, forward + loss + reverse of every stage on seeded "
                       f"{'x'.join(map(str, _crop(args.config)))} windows of the {W}x{H} view (all {n} Gaussians pre-culled per window), seconds "
                       f"per pixel scaled to the full view: {cores} processes, {per * cores} windows"),
            "extrapolated": True,
            "single_core": {"value": round(one, 6), "unit": "iters/s", "cores": 1, "windows": k1,
                            "seconds_per_iter": round(sec1 / px1 * P, 2)},
            "seconds_per_iter": round(wall / pxn * P, 2), "wall_s": round(time.perf_counter() - t_all, 1)}


def run_reference(args):
    """The oracle arm: each step runs one window per host core in parallel
    (spawned processes) through the FP64 oracle; the rate is the windows'
    pixels per wall second scaled to the full view (extrapolated). Only rank
    0 works under torchrun."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    cfg = CONFIGS[args.config]
    prec = "bf16" if "bf16" in cfg["precisions"] and args.precision != "f32" else "f32"
    n = bench_config(args)["gaussians"]
    W, H = [int(x) for x in cfg["image"].split("x")]
    cores, model = cpu_info()
    rng = np.random.default_rng(11)
    pool = OraclePool(args.config, n, prec, cores)
    for _ in range(args.warmup):
        pool.run(_windows(args.config, n, rng, cores))
    px = wall = 0.0
    step_s = []
    for _ in range(args.steps):
        p_, w_ = pool.run(_windows(args.config, n, rng, cores))
        px += p_
        wall += w_
        step_s.append(w_)
    pool.close()
    v = (px / (W * H)) / wall if wall > 0 else 0.0
    frac = (px / args.steps) / (W * H) if args.steps else 0.0
    sample = (f"FP64 oracle, forward + loss + reverse of every stage, each step {cores} seeded "
              f"{'x'.join(map(str, _crop(args.config)))} windows of the {W}x{H} view in parallel ({cores} processes); "
              f"rate = windows' pixels per second / pixels of the view")
    out = {"metric": cfg["metric"], "value": round(v, 6), "unit": "iters/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1000.0 * float(np.mean(step_s)), 1) if step_s else None,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": bench_config(args), "impl": "reference",
           "extrapolated": True, "step_fraction_of_iteration": round(frac, 5),
           "cpu_baseline": {"value": round(v, 6), "unit": "iters/s", "cores": cores, "kind": "oracle",
                            "cpu_model": model, "sample": sample},
           "e2e": {"value": round(v, 6), "unit": "iters/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.ablation:
        run_ablation(a)
    elif a.config in (4, 5):
        run_config(a)
    else:
        run_ours(a)
