"""HyRF hot-path benchmark: fwd+bwd iterations/s and render FPS of one view
of the 1M-Gaussian, 1237x822 workload (16-level 2^19 grids, 2x64 decoders,
exact neural background, L1 loss), on synthetic seeded data.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision bf16|f32]
  python bench.py --impl reference ...   # the FP64 CPU oracle on a bounded sample

One "step" = gradient zeroing -> pre-cull -> query_fields (the depth order
and the background's feature gather beside it on a second stream) ->
project -> bin_sort -> rasterize -> composite_background -> loss -> every
reverse call (the background's on the second stream), inputs resident in
HBM, replayed as one CUDA graph (pipeline.StepGraph; --no-graph issues the
calls one by one). L2 is flushed (256 MiB write) between timed steps.
Prints one JSON line. Multi-GPU: independent replicas (one view per rank),
no collective.
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
    p.add_argument("--config", type=int, default=3, choices=[3, 4, 5],
                   help="3: the headline line; 4: 8-view step as one CUDA graph (3M Gaussians, memory "
                        "saved vs recompute); 5: 6M Gaussians at 1920x1080 with 1%% degenerate ones")
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


# ---------------------------------------------------------------- algorithmic work per stage

def kernel_work(nv, K, P, tiles, bf16):
    """Algorithmic HBM bytes per launch of the main kernels: every input read
    once, every output written once, each table-gradient atomic counted as its
    8-byte float2 payload. Per-unit figures: visible Gaussian (nv), tile
    instance (K), pixel (P)."""
    L = 16
    ent = 4 if bf16 else 8                     # bytes per 2-feature table entry
    gather = L * 8 * ent                       # one field, 8 corners per level
    scatter = L * 8 * 8                        # one field, float2 atomic per corner
    feat, dfeat = 64, 128                      # bf16 features / f32 gradients per row and field
    return {
        # FP32 fused field kernels: vis id, position, both fields, explicit
        # params (20 B), outputs (44 B)
        "k_query_fwd": nv * (4 + 12 + 2 * gather + 20 + 44),
        # BF16 split path. gather: vis id, position, 8 corners x 16 levels per
        # field, features written
        "k_gather<gaussians>": nv * (4 + 12 + 2 * (gather + feat)),
        "k_gather<pixels>": P * (gather + feat),
        # decoders on the tensor cores: features in, outputs / gradients out
        "k_query_fwd_tc": nv * (4 + 12 + 2 * feat + 20 + 44),
        "k_bg_exact_fwd_tc": P * (feat + 12 + 4 + 12),
        # vis id, features, dalpha/dscale/dquat, alpha_e/scale_e, their
        # gradients read-modify-write, feature gradients out
        "k_decoder_bwd_tc<GeoGauss>": nv * (4 + feat + 32 + 8 + 16 + dfeat),
        # vis id, features, position, dcolor, color_e, d_color_e and d_pos RMW,
        # feature gradients out
        "k_decoder_bwd_tc<ColGauss>": nv * (4 + feat + 12 + 12 + 12 + 24 + 24 + dfeat),
        # features, T_final, dC, dT out, feature gradients out
        "k_decoder_bwd_tc<BgPixel>": P * (feat + 4 + 12 + 4 + dfeat),
        # scatter: feature gradients in, float2 atomics, corner values re-read
        # for dL/dp (Gaussians), d_pos RMW
        "k_scatter<gaussians>": nv * (4 + 12 + 2 * (dfeat + scatter + gather) + 24),
        "k_scatter<pixels>": P * (dfeat + scatter),
        # 48-B record + 4-B id per instance, ranges, C_fg/T_final/n_contrib out
        "k_raster_fwd": K * 52 + tiles * 8 + P * 20,
        # as forward, plus dC/dT/T_final/n_contrib per pixel, 36-B grads RMW per Gaussian
        "k_raster_bwd": K * 52 + tiles * 8 + P * 24 + nv * 72,
    }


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
    precisions = []
    if args.precision in ("auto", "bf16"):
        precisions.append("bf16")
    if args.precision in ("auto", "f32"):
        precisions.append("f32")
    results = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sampler = ClockSampler(local)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    for prec in precisions:
        w = synth.config3(n=args.n, precision=prec, seed=local)
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
        C = r.C.float()
        psnr = float(-10.0 * torch.log10(((C - tgt) ** 2).mean()).item())
        evals = int(r.n_contrib.sum().item())
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
                                              int(r.ranges.shape[0]), prec == "bf16"))
        del r, m
        torch.cuda.empty_cache()
    head = "bf16" if "bf16" in results and "ms" in results["bf16"] else "f32"
    R = results[head]
    value = whole_job_rate(R["ms"], ws)
    roof = roofline(R, peaks, head)
    per_step = {k: n * t for k, (n, t) in R["kernels"].items()}
    tot = sum(per_step.values()) or 1.0
    top = sorted(per_step, key=per_step.get, reverse=True)[:12]
    kern = {k: {"ms_per_step": round(per_step[k], 4), "share": round(per_step[k] / tot, 4),
                "launches_per_step": round(R["kernels"][k][0], 2)} for k in top}
    rf = R["kernels"].get("k_raster_fwd")
    out = {"metric": METRIC, "value": round(value, 3), "unit": "iters/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(R["ms"], 4),
           "step_issue": "one CUDA graph per step" if args.graph else "eager",
           "eager_ms_per_step": round(R["eager_ms"], 4) if R.get("eager_ms") else None,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "bf16" if head == "bf16" else "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "precision": head, "gaussians": args.n,
                      "image": "1237x822", "visible": R["n_vis"], "instances": R["instances"],
                      "l2": "flushed between timed steps (256 MiB write)", "layout": args.layout,
                      "parallelism": f"replicas x{ws}"},
           "render_fps": round(ws * 1000.0 / R["fwd_ms"], 2),
           "render_fps_tau_T_0.2": round(ws * 1000.0 / R["tau_ms"], 2) if R.get("tau_ms") else None,
           "render_fps_u8_grids": round(ws * 1000.0 / R["u8_ms"], 2) if R.get("u8_ms") else None,
           "render_fps_f16_fields": round(ws * 1000.0 / R["f16_ms"], 2) if R.get("f16_ms") else None,
           "stage_ms": {k: round(v, 4) for k, v in R["stage_ms"].items()},
           "kernels": kern,
           "psnr_db": round(R["psnr"], 4),
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
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args, budget_s=args.cpu_sample_s)
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the named kernel on this workload; an entry is removed when
# the kernel changes after its capture.
NCU_TRAFFIC = {
    # profiles/kernels_config3_bf16.md (traffic of the compositing reverse):
    # 57.57 MB read + 0.04-0.25 MB written per launch, two launches
    ("k_raster_bwd", "bf16"): 57_720_000,
}


def roofline(R, peaks, prec):
    """Roofline of the kernel with the largest time per step, from the
    library's own CUDA-event kernel timer over the steps of the timer pass
    (the timed step's calls, issued on one stream)."""
    hbm = peaks.get("hbm_gbs")
    src = "of measured" if hbm else "of fallback"
    hbm = hbm or 6800.0
    per_step = {k: n * t for k, (n, t) in R["kernels"].items()}
    if not per_step:
        return {"kernel": None, "bound": "hbm", "achieved": None, "peak": hbm, "unit": "GB/s",
                "frac": None, "traffic": None}
    k = max(per_step, key=per_step.get)
    n, avg_ms = R["kernels"][k]
    work = R["work"].get(k)
    gbs = work / (avg_ms * 1e-3) / 1e9 if work else None
    tr = NCU_TRAFFIC.get((k, prec))
    return {"kernel": k, "bound": "hbm", "achieved": round(gbs, 1) if gbs else None, "peak": hbm,
            "unit": "GB/s", "frac": round(gbs / hbm, 4) if gbs else None,
            "traffic": tr, "algorithmic_bytes": work, "avg_launch_ms": round(avg_ms, 4),
            "peak_source": src}


# ---------------------------------------------------------------- configs 4 and 5

def run_config(args):
    import torch
    from paper_2509_17083_gb300 import hyrf as H
    from paper_2509_17083_gb300 import synth
    from paper_2509_17083_gb300.pipeline import DeviceModel, ViewRenderer, shared_workspaces

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    H.lib()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    steps = max(3, args.steps // 10)

    def timed(fn, k):
        for _ in range(max(3, args.warmup // 5)):
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

    if args.config == 5:
        w = synth.config5()
        m = DeviceModel(w)
        m.spatial_order()
        r = ViewRenderer(m, w.cams[0], w.bg, lam=w.ssim_lambda, loss_scale=w.loss_scale)
        tgt = torch.as_tensor(w.targets[0]).cuda()
        r.fit_capacity(tgt)

        def step():
            m.zero_grad()
            r.step(tgt)
        ms = timed(step, steps)
        fwd = timed(lambda: r.forward(None, want_keys=False), steps)
        tau = timed(lambda: r.forward(None, want_keys=False, tau_T=0.2), steps)
        out = {"metric": "fwd+bwd iters/s & render FPS, 6M Gaussians @1920x1080, BF16 fields", "value": round(1000 / ms, 3),
               "unit": "iters/s", "ms_per_step": round(ms, 3), "render_fps": round(1000 / fwd, 2),
               "render_fps_tau_T_0.2": round(1000 / tau, 2), "visible": int(r.n_vis.item()),
               "instances": int(r.n_inst.item()), "status": H.read_status(r.status),
               "config": {"workload": "config5: 6M Gaussians (40 % beyond depth 50), 1920x1080, 2^22 grids",
                          "layout": "morton", "steps": steps}}
        print(json.dumps(out))
        return
    # config 4: 8 views, one CUDA graph per step; saved features vs recompute
    res = {}
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
        res["saved" if save else "recompute"] = dict(ms_per_step=round(ms, 3), views_per_s=round(8000 / ms, 2),
                                                     peak_gib=round(torch.cuda.max_memory_allocated() / 2**30, 2))
        del g, views, m
    print(json.dumps({"metric": "8-view fwd+bwd step as one CUDA graph, 3M Gaussians @1297x840, BF16 fields",
                      "value": res["saved"]["views_per_s"], "unit": "views/s",
                      "config": {"workload": "config4: 3M Gaussians in a radius-2 ball, 8 ring cameras, 2^21 grids",
                                 "layout": "morton", "steps": steps},
                      "features": res}))


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

def cpu_baseline(args, budget_s=15.0, w=None, frac=1.0):
    """The FP64 oracle, single-threaded, on a bounded sample of the workload;
    per-stage sample times are scaled to one full iteration. `frac` shrinks
    the sample (the reference arm runs several such steps)."""
    import oracle
    from paper_2509_17083_gb300 import synth

    if w is None:
        w = synth.config3(n=args.n, precision="bf16" if args.precision != "f32" else "f32")
    g, fl, cam, bg = w.gaussians, w.fields, w.cams[0], w.bg
    rng = np.random.default_rng(0)
    t_all = time.perf_counter()
    parts = {}
    vis = oracle.precull_f32(g.pos, cam)
    ids = np.nonzero(vis)[0]
    nv = len(ids)
    # field query fwd+bwd on a sample of visible Gaussians
    ns = max(50, min(nv, int(2000 * frac)))
    sid = np.sort(rng.choice(ids, ns, replace=False))
    pos = g.pos[sid].astype(np.float64)
    t = time.perf_counter()
    a, s, q, c = oracle.query_fields(pos, g.alpha_e[sid], g.scale_e[sid], g.color_e[sid], cam, fl)
    oracle.query_fields_backward(pos, g.alpha_e[sid], g.scale_e[sid], g.color_e[sid], cam, fl,
                                 np.ones(ns), np.ones((ns, 3)), np.ones((ns, 4)), np.ones((ns, 3)))
    parts["query"] = (time.perf_counter() - t) * nv / ns
    # projection fwd+bwd on the sample
    t = time.perf_counter()
    m2, cn, d = oracle.project(pos, s, q, cam)
    oracle.project_backward(pos, s, q, cam, np.ones((ns, 2)), np.ones((ns, 3)))
    parts["project"] = (time.perf_counter() - t) * nv / ns
    # binning on all visible Gaussians (isotropic FP64 query replaced by the
    # explicit scales, which is what the field outputs are at initialisation)
    sv = (1 / (1 + np.exp(-g.scale_e[ids].astype(np.float64))))[:, None].repeat(3, 1)
    qv = np.tile([1.0, 0, 0, 0], (nv, 1))
    t = time.perf_counter()
    rect, ntiles, d32, _ = oracle.project_f32(g.pos[ids], sv, qv, cam)
    TX, TY = oracle.tiles_of(cam.width, cam.height)
    keys, vals, ranges = oracle.bin_sort(rect, d32, TX, TY)
    parts["bin_sort"] = time.perf_counter() - t
    # compositing fwd+bwd on a sample of tiles
    mall, call_, _ = oracle.project(g.pos[ids].astype(np.float64), sv, qv, cam)
    op = 1 / (1 + np.exp(-g.alpha_e[ids].astype(np.float64)))
    col = 1 / (1 + np.exp(-g.color_e[ids].astype(np.float64)))
    nt = TX * TY
    tsel = rng.choice(nt, max(1, int(nt // 100 * frac)), replace=False)
    rs = np.zeros_like(ranges)
    rs[tsel] = ranges[tsel]
    t = time.perf_counter()
    Cfg, T, _, _ = oracle.rasterize(cam.width, cam.height, rs, vals, mall, call_, op, col)
    oracle.rasterize_backward(cam.width, cam.height, rs, vals, mall, call_, op, col,
                              np.ones((cam.height, cam.width, 3)), np.ones((cam.height, cam.width)))
    parts["rasterize"] = (time.perf_counter() - t) * nt / len(tsel)
    # background fwd+bwd on a small sub-image, scaled by pixel count
    sub = synth.pinhole(64, 48, fx=cam.fx)
    sub.cx, sub.cy = cam.cx - 300, cam.cy - 200
    t = time.perf_counter()
    oracle.background(sub, fl, bg, np.zeros((48, 64, 3)), np.ones((48, 64)))
    oracle.background_backward(sub, fl, bg, np.ones((48, 64)), np.ones((48, 64, 3)))
    parts["background"] = (time.perf_counter() - t) * (cam.width * cam.height) / (64 * 48)
    t = time.perf_counter()
    oracle.loss(np.zeros((cam.height, cam.width, 3)), w.targets[0], 0.0)
    parts["loss"] = time.perf_counter() - t
    sec = sum(parts.values())
    return {"value": round(1.0 / sec, 6), "unit": "iters/s", "cores": 1, "kind": "oracle",
            "sample": (f"FP64 oracle single-threaded: field query+project fwd/bwd on {ns} of {nv} "
                       f"visible Gaussians, compositing fwd/bwd on {len(tsel)} of {nt} tiles, "
                       f"background fwd/bwd on 64x48 of 1237x822 pixels, each scaled to the "
                       f"full workload; binning and loss in full"),
            "seconds_per_iter": round(sec, 2), "stage_s": {k: round(v, 2) for k, v in parts.items()},
            "wall_s": round(time.perf_counter() - t_all, 1)}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from paper_2509_17083_gb300 import synth
    w = synth.config3(n=args.n, precision="bf16" if args.precision != "f32" else "f32")
    vals = []
    cb = None
    for k in range(args.warmup + args.steps):
        cb = cpu_baseline(args, w=w, frac=0.25)
        if k >= args.warmup:
            vals.append(cb["value"])
    v = float(np.mean(vals)) if vals else 0.0
    out = {"metric": METRIC, "value": round(v, 6), "unit": "iters/s", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(1000.0 / v, 1) if v else None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "sample": "bounded; see cpu_baseline"},
           "impl": "reference",
           "cpu_baseline": {"value": round(v, 6), "unit": "iters/s", "cores": 1, "kind": "oracle",
                            "sample": cb["sample"] if cb else ""},
           "e2e": {"value": round(v, 6), "unit": "iters/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.ablation:
        run_ablation(a)
    elif a.config != 3:
        run_config(a)
    else:
        run_ours(a)
