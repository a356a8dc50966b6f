#!/usr/bin/env python
"""Benchmark: fwd+bwd rasterize (+ L1 and Adam) ms/view on the GB300.

Workload (one step = one view through the whole hot path): a seeded 2M-Gaussian
scene of textured planes/spheres plus a background shell (the 2M ground-truth
scene of the plain full-resolution training configuration), optimised at the
full 1237x822 resolution, one view per step:
    project -> bin (depth order, pair emission, tile sort, ranges) ->
    render fwd -> L1 loss -> render bwd -> project bwd -> Adam (all 59 rows).
The optimised state is the ground truth with Gaussian noise on every
parameter; targets are the ground truth rendered at the same 16 views.  The
working set (params, grads, Adam moments: 1.9 GB) is larger than L2, so no
flush is needed between steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on the same workload (a bounded sample per step, scaled to ms/view).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

W_FULL, H_FULL = 1237, 822
N_GAUSS = 2_000_000
N_VIEWS = 16
BENCH_TILE = 8  # tile edge of the workload (the autotuner picks the rest of the launch shape)
METRIC = "fwd+bwd rasterize ms/view (full-res training step incl. L1 + D-SSIM + Adam)"
# training leg: the plain FP32 full-resolution arm (one view per iteration) and
# the scheduled arms: 16 views per step in one launch per pass, each step one
# CUDA-graph replay, mixed-precision records; a = 2 and the paper's a = 4
TRAIN_RUNS = ("plain", "scheduled:a=2:v=16:graph=1:record=mixed", "scheduled:a=4:v=16:graph=1:record=mixed")
# Algorithmic FP32 work of the compositing passes (Eq. 1 and its adjoint), per
# (pixel, list entry): every entry a pixel examines needs its alpha test --
# offsets, quadratic form, exponential, clamp, threshold; a blended entry adds
# the transmittance and colour update (forward) or the gradient (backward).
FLOPS_TEST = 12
FLOPS_FWD_BLEND = 7
FLOPS_BWD_BLEND = 38
# the same passes counted per examined entry as the hot-path scope table does
# (forward about 18 FP32 operations per examined entry, backward about 50)
FLOPS_FWD_PER_E = 18
FLOPS_BWD_PER_E = 50
SM_COUNT, FP32_LANES, MAX_MHZ = 152, 128, 2070.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=int(os.environ.get("WORLD_SIZE", "1")))
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n-gauss", type=int, default=N_GAUSS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--record", choices=["fp32", "mixed"], default="fp32",
                    help="render-side record storage (mixed: float16 conic/opacity, bfloat16 colour)")
    ap.add_argument("--graph", action="store_true",
                    help="also time the step captured as one CUDA graph (graph_ms_per_view)")
    ap.add_argument("--shape", default=None,
                    help="render launch shape, e.g. t8f1b1s0 (tile, pixels per thread fwd/bwd, split); "
                         "default: autotuned over the candidates")
    ap.add_argument("--separate-adam", action="store_true",
                    help="projection adjoint and Adam as two kernels (default: one fused kernel)")
    ap.add_argument("--no-train", action="store_true",
                    help="skip the 30k-iteration training leg (plain FP32 arm vs scheduled batched mixed arm)")
    ap.add_argument("--train-runs", nargs="*", default=list(TRAIN_RUNS),
                    help="training runs of the training leg (train.py run specs; the first is the baseline)")
    ap.add_argument("--bins", choices=["tight", "paper"], default="tight",
                    help="pair lists: tight (tiles where the Gaussian can reach alpha 1/255; same images and "
                         "gradients) or paper (every tile of the 3-sigma rect)")
    ap.add_argument("--no-c4-crop", action="store_true",
                    help="skip the CPU baseline's 6M-Gaussian crop measurement (scene generation takes ~30 s)")
    return ap.parse_args()


def parse_shape(label: str):
    """Shape from its label t<tile>f<ppt fwd>b<ppt bwd>s<split>."""
    import re
    from paper_2503_18402_gb300.autotune import Shape
    mt = re.fullmatch(r"t(\d+)f(\d+)b(\d+)s(-?\d+)", label)
    if not mt:
        raise SystemExit(f"bad --shape {label!r}: want e.g. t8f1b1s0")
    return Shape(*(int(x) for x in mt.groups()))


# source file of each timed stage's kernels (for the ncu summaries' hash check)
STAGE_SOURCE = {"render_fwd": "render.cu", "render_bwd": "render.cu", "project": "project.cu",
                "project_bwd": "project.cu", "project_bwd_adam": "project.cu", "adam": "optim.cu"}


def measured_traffic(stage: str, root: str = ROOT):
    """DRAM bytes per launch of the stage's kernel from a committed ncu summary
    under profiles/ (lines 'stage:', 'source_sha1:', 'dram_bytes_per_launch:'),
    or None when there is none or it was taken on another version of the
    kernel's source file."""
    import glob
    import hashlib
    src = STAGE_SOURCE.get(stage)
    if src is None:
        return None
    try:
        with open(os.path.join(root, "paper_2503_18402_gb300", "csrc", src), "rb") as f:
            sha = hashlib.sha1(f.read()).hexdigest()
    except OSError:
        return None
    for path in sorted(glob.glob(os.path.join(root, "profiles", "*.md"))):
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith((" ", "|", "#")):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("stage") == stage and kv.get("source_sha1") == sha and "dram_bytes_per_launch" in kv:
            return int(kv["dram_bytes_per_launch"])
    return None


def config(args, n_gauss):
    prec = "mixed" if args.record == "mixed" else "fp32"
    return {"workload": f"textured-{n_gauss // 1000}k-gaussians-{W_FULL}x{H_FULL}-1view-{prec}",
            "n_gaussians": n_gauss, "width": W_FULL, "height": H_FULL, "views_per_step": 1,
            "tile": BENCH_TILE, "sh_degree": 3, "loss": "0.8 L1 + 0.2 D-SSIM",
            "step": "project+bin+render_fwd+loss+render_bwd+project_bwd+adam",
            "adjoint_adam": "two kernels" if args.separate_adam else "fused",
            "render_records": "mixed fp16/bf16" if args.record == "mixed" else "fp32",
            "pair_lists": "tight (kept tiles of rects up to 8x8 tiles)" if args.bins == "tight" else "3-sigma rect",
            "l2": "working set 1.9 GB > L2 (no flush)", "parallelism": f"replicas{args.gpus}"}


# --------------------------------------------------------------------------- ranks
def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest value of x over the ranks (replicas run in lockstep between
    barriers, so the job takes as long as its slowest rank)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_ms_per_view(elapsed_ms: float, steps: int, world: int) -> float:
    """Whole-job figure: every rank renders `steps` views (weak scaling), the
    job takes the slowest rank's time."""
    return elapsed_ms / (steps * world)


# --------------------------------------------------------------------------- scene
def make_scene(n_gauss, rank):
    from paper_2503_18402_gb300 import synth
    gt = synth.textured_scene(n_gauss, 1001)
    model = synth.jitter(gt, 3001)
    cams = synth.ring_cameras(160, W_FULL, H_FULL, 5.0, 2001)
    views = [cams[(rank * N_VIEWS + j * 10) % 160] for j in range(N_VIEWS)]
    return gt, model, views


# --------------------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------------------- ours
def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2503_18402_gb300 import capi
    from paper_2503_18402_gb300.autotune import CANDIDATES, RenderTuner
    from paper_2503_18402_gb300.raster import Rasterizer, make_camera

    world = args.gpus
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    gt, model, views = make_scene(args.n_gauss, rank)
    P = gt.shape[0]
    gcams = [make_camera(np.asarray(v["viewmat"], np.float32).reshape(-1), v["intr"], v["width"], v["height"])
             for v in views]
    opts = capi.raster_opts(tile=16, sh_degree=3, record=1 if args.record == "mixed" else 0,
                            tight_bins=1 if args.bins == "tight" else 0)
    rz = Rasterizer(dev, capi.raster_opts(tile=16, sh_degree=3))
    gt_t = torch.from_numpy(np.ascontiguousarray(gt.T)).to(dev)
    targets = []
    for c in gcams:
        fr = rz.forward(gt_t, P, c)
        targets.append(fr.img.clone())
    del gt_t
    params = torch.from_numpy(np.ascontiguousarray(model.T)).to(dev)
    grads = torch.zeros_like(params)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    stride = params.stride(0)
    extent = 5.0
    lr = [1.6e-4 * extent] * 3 + [0.005] * 3 + [0.001] * 4 + [0.025] + [0.0025] * 3 + [0.0025 / 20] * 45
    dL = torch.empty((3, H_FULL, W_FULL), dtype=torch.float32, device=dev)
    loss = torch.zeros(2, dtype=torch.float32, device=dev)
    sws = torch.empty(capi.dg_ssim_workspace_size([(W_FULL, H_FULL)]), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    adam_t = [0]

    def step_with(r, i, tgt=None, mark=None):
        j = i % N_VIEWS
        r.mark = mark
        if mark:
            mark("start")
        fr = r.forward(params, P, gcams[j])
        capi.dg_loss_l1_dssim(fr.img, targets[j] if tgt is None else tgt, [(W_FULL, H_FULL)], 0.2, dL, loss, sws,
                              sws.numel(), stream)
        if mark:
            mark("loss")
        r.backward_render(fr, dL, stream)
        adam_t[0] += 1
        if args.separate_adam:
            capi.dg_project_bwd(params, stride, P, gcams[j], 1, r.opts, r.radius, r.clamp, r.grad2d, grads, stream)
            if mark:
                mark("project_bwd")
            capi.dg_adam_step(params, grads, m, v, stride, P, lr, 0.9, 0.999, 1e-15, adam_t[0], stream)
            if mark:
                mark("adam")
        else:
            r.project_bwd_adam(params, stride, fr, m, v, lr, adam_t[0], stream=stream)
        return fr

    # launch-shape autotuning: time each candidate on a few steps, keep the fastest
    tuner = RenderTuner(dev, opts)
    tune_ms = {}
    for shape in ([parse_shape(args.shape)] if args.shape else [c for c in CANDIDATES if c.tile == BENCH_TILE]):
        r = tuner.rasterizer(shape)
        for i in range(2):
            step_with(r, i)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for i in range(4):
            step_with(r, 2 + i)
        e1.record(stream)
        torch.cuda.synchronize()
        tune_ms[shape] = e0.elapsed_time(e1) / 4
    shape = min(tune_ms, key=tune_ms.get)
    rz = tuner.rasterizer(shape)
    # restart the optimisation from the same state for the timed run
    params.copy_(torch.from_numpy(np.ascontiguousarray(model.T)).to(dev))
    m.zero_(); v.zero_(); adam_t[0] = 0

    # algorithmic work per view, counted on the paper's lists (every tile of
    # the rect): entries examined by the forward, entries the backward walks
    # (up to each pixel's last blended one), blended entries; and the pairs of
    # the lists the timed step sorts
    po = capi.RasterOpts.from_buffer_copy(rz.opts)
    po.tight_bins = 0
    rzp = Rasterizer(dev, po, ppt_fwd=shape.ppt_fwd, ppt_bwd=shape.ppt_bwd)
    E_f, E_l, E_b, M_paper, M_tot = [], [], [], [], []
    for c in gcams:
        fr = rzp.forward(params, P, c, examined=True)
        E_f.append(int(rzp.examined.sum().item()))
        E_l.append(int(fr.last.sum().item()))
        E_b.append(int(rzp.blended.sum().item()))
        M_paper.append(fr.M)
        M_tot.append(rz.forward(params, P, c).M)
    del rzp, fr
    torch.cuda.empty_cache()

    events = []
    rz.mark = None

    def mark(name):
        e = torch.cuda.Event(enable_timing=True)
        e.record(stream)
        events.append((name, e))

    def step(i, tgt=None, stage_events=False):
        return step_with(rz, i, tgt, mark if stage_events else None)

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()

    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = capi.dg_kernel_launches()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.nvtx.range_push("timed")
    t0.record(stream)
    for i in range(args.steps):
        events.clear() if i == 0 else None
        step(args.warmup + i, stage_events=True)
    t1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    launches = capi.dg_kernel_launches() - launches0
    clk = clocks.stop()
    elapsed_ms = t0.elapsed_time(t1)
    # per-stage device time between consecutive marks
    stage_ms = {}
    prev = None
    for name, e in events:
        if name == "start":
            prev = e
            continue
        stage_ms[name] = stage_ms.get(name, 0.0) + prev.elapsed_time(e)
        prev = e
    elapsed_ms = max_over_ranks(elapsed_ms, world, dev)

    # the same step captured once as a CUDA graph and replayed per view (new
    # camera, Adam hyper-parameters and target written to device buffers)
    graph_ms = None
    if args.graph:
        from paper_2503_18402_gb300.graphstep import StepGraph
        gshape = shape
        gr = tuner.rasterizer(gshape)
        fr0 = gr.forward(params, P, gcams[0])
        M_cap = int(max(M_tot) * 1.25) + 4096
        sg = StepGraph(dev, gr.opts, gshape.ppt_fwd, gshape.ppt_bwd, params, m, v, grads, stride, P, [gcams[0]],
                       M_cap, 0.2, fused=not args.separate_adam)
        adam_t[0] += 1
        sg.capture([gcams[0]], capi.dg_adam_hparams_fill(lr, 0.9, 0.999, 1e-15, adam_t[0]), [targets[0]])
        for i in range(args.warmup):
            adam_t[0] += 1
            sg.replay([gcams[i % N_VIEWS]], capi.dg_adam_hparams_fill(lr, 0.9, 0.999, 1e-15, adam_t[0]),
                      [targets[i % N_VIEWS]])
        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        hps = [capi.dg_adam_hparams_fill(lr, 0.9, 0.999, 1e-15, adam_t[0] + 1 + i) for i in range(args.steps)]
        g0.record(stream)
        for i in range(args.steps):
            sg.replay([gcams[i % N_VIEWS]], hps[i], [targets[i % N_VIEWS]])
        g1.record(stream)
        torch.cuda.synchronize()
        adam_t[0] += args.steps
        graph_ms = g0.elapsed_time(g1) / args.steps
        status, _ = sg.result()
        if status != 0:
            graph_ms = None  # a step exceeded the graph's pair capacity: no valid number
        del sg

    # end to end through the public API: each step's target is copied from
    # pinned host memory and its loss read back to the host.  The copy of step
    # i + 1's target runs on a side stream into the other of two buffers while
    # step i computes (as a data loader would), and the host reads step i's
    # loss, copied to pinned memory asynchronously, after launching step i + 1.
    pinned = [t.cpu().pin_memory() for t in targets]
    tbuf = [torch.empty_like(targets[0]) for _ in range(2)]
    copy_stream = torch.cuda.Stream(dev)
    ready = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    loss_host = torch.zeros((args.steps + 2, 2), dtype=torch.float32).pin_memory()
    loss_done = [torch.cuda.Event() for _ in range(args.steps + 2)]

    def e2e_run(n):
        losses = []
        with torch.cuda.stream(copy_stream):
            tbuf[0].copy_(pinned[0], non_blocking=True)
            ready[0].record(copy_stream)
        for i in range(n):
            k = i % 2
            if i + 1 < n:
                with torch.cuda.stream(copy_stream):
                    if i >= 1:
                        copy_stream.wait_event(freed[1 - k])  # step i - 1 has consumed that buffer
                    tbuf[1 - k].copy_(pinned[(i + 1) % N_VIEWS], non_blocking=True)
                    ready[1 - k].record(copy_stream)
            stream.wait_event(ready[k])
            step(i, tgt=tbuf[k])
            freed[k].record(stream)
            loss_host[i].copy_(loss, non_blocking=True)
            loss_done[i].record(stream)
            if i >= 1:
                loss_done[i - 1].synchronize()
                losses.append(float(loss_host[i - 1, 1]))
        loss_done[n - 1].synchronize()
        losses.append(float(loss_host[n - 1, 1]))
        return losses

    e2e_run(2)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = time.perf_counter()
    e2e_losses = e2e_run(args.steps)
    torch.cuda.synchronize()
    assert len(e2e_losses) == args.steps and all(np.isfinite(e2e_losses)), e2e_losses
    e2e_ms = (time.perf_counter() - e0) * 1e3
    e2e_ms = max_over_ranks(e2e_ms, world, dev)

    views_total = args.steps * world
    ms_per_view = job_ms_per_view(elapsed_ms, args.steps, world)
    out = {
        "metric": METRIC,
        "value": round(ms_per_view, 4), "unit": "ms/view", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded textured scene)",
        "config": config(args, P), "impl": "ours", "render_shape": shape.label(),
        "autotune_ms_per_step": {s.label(): round(t, 4) for s, t in tune_ms.items()},
    }
    tot = sum(stage_ms.values())
    stages = {k: {"ms": round(v / args.steps, 4), "share": round(v / tot, 4)} for k, v in stage_ms.items()}
    out["stages"] = stages
    pf = sum(E_f) / len(E_f)
    pl = sum(E_l) / len(E_l)
    pb = sum(E_b) / len(E_b)
    work = {"render_fwd": ("alu", pf * FLOPS_TEST + pb * FLOPS_FWD_BLEND),
            "render_bwd": ("alu", pl * FLOPS_TEST + pb * FLOPS_BWD_BLEND),
            "project": ("hbm", P * 297.0), "project_bwd": ("hbm", P * 525.0), "adam": ("hbm", P * 1652.0),
            "project_bwd_adam": ("hbm", P * 1469.0)}
    dom = max((k for k in stages if k in work), key=lambda k: stages[k]["ms"])
    kind, units = work[dom]
    dur_s = stages[dom]["ms"] * 1e-3
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    if kind == "alu":
        peak = SM_COUNT * FP32_LANES * 2 * MAX_MHZ * 1e6 / 1e12
        ach = units / dur_s / 1e12
        out["roofline"] = {"bound": "alu", "kernel": dom, "achieved": round(ach, 3), "peak": round(peak, 2),
                           "unit": "TFLOP/s", "frac": round(ach / peak, 4), "traffic": measured_traffic(dom),
                           "peak_source": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz"}
    else:
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        ach = units / dur_s / 1e9
        out["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                           "frac": round(ach / hbm, 4), "traffic": measured_traffic(dom),
                           "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks
                           else "fallback 6800 GB/s"}
    # every timed stage against its bound: HBM stages by algorithmic bytes, the
    # compositing passes by FP32 work (both counts: the per-examined-entry count
    # and the count of the operations the algorithm needs per walked/blended entry)
    alu_peak = SM_COUNT * FP32_LANES * 2 * MAX_MHZ * 1e6 / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    by_stage = {}
    for k, st in stages.items():
        dur = st["ms"] * 1e-3
        if dur <= 0 or k not in work:
            continue
        kind_k, units_k = work[k]
        if kind_k == "alu":
            per_e = {"render_fwd": FLOPS_FWD_PER_E * pf, "render_bwd": FLOPS_BWD_PER_E * pf}[k]
            by_stage[k] = {"bound": "alu", "unit": "TFLOP/s", "peak": round(alu_peak, 2),
                           "achieved": round(units_k / dur / 1e12, 3), "frac": round(units_k / dur / 1e12 / alu_peak, 4),
                           "achieved_per_examined_count": round(per_e / dur / 1e12, 3),
                           "frac_per_examined_count": round(per_e / dur / 1e12 / alu_peak, 4)}
        else:
            by_stage[k] = {"bound": "hbm", "unit": "GB/s", "peak": hbm_peak,
                           "achieved": round(units_k / dur / 1e9, 1), "frac": round(units_k / dur / 1e9 / hbm_peak, 4)}
    out["roofline_by_stage"] = by_stage
    out["work"] = {"pairs_per_view": int(sum(M_tot) / len(M_tot)),
                   "pairs_per_view_rect_lists": int(sum(M_paper) / len(M_paper)), "examined_per_view": int(pf),
                   "walked_back_per_view": int(pl), "blended_per_view": int(pb)}
    # the rasterizer's forward and backward: projection, binning, both compositing passes
    out["fwd_bwd_ms_per_view"] = round(sum(stages[k]["ms"] for k in stages
                                           if k in ("project", "bin_count", "host_sync", "bin_sort", "render_fwd",
                                                    "render_bwd")), 4)
    out["e2e"] = {"value": round(e2e_ms / views_total, 4), "unit": "ms/view",
                  "h2d_bytes_per_step": int(targets[0].numel() * 4),
                  "d2h_bytes_per_step": 8 + 8}  # the loss (2 floats) and the pair count
    out["gpu_launches"] = int(launches)
    if graph_ms is not None:
        out["graph_ms_per_view"] = round(graph_ms, 4)
    out["clocks"] = clk
    if not args.no_train:
        out["training"] = training_leg(gt, dev, args, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(model, views[0], targets[0].double().cpu().numpy(), BENCH_TILE,
                                           c4_scene=not args.no_c4_crop)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------- training
def training_leg(gt, dev, args, gpu_index):
    """The metric's first half: seconds to 30k iterations and held-out PSNR of
    the plain FP32 full-resolution arm and of the scheduled arms, on this
    scene (160 ring views at 1237x822 rendered from the ground truth, every
    8th held out, 100k perturbed points to start).  Wall-clock of each run
    includes the schedule's spectrum pass, excludes scene generation."""
    import types

    import torch

    from paper_2503_18402_gb300 import synth, train
    targs = types.SimpleNamespace(iters=30000, p_cap=3_000_000, a=4.0, gamma=0.98, ssim_lambda=0.2,
                                  no_autotune=False, views_per_step=1, cuda_graph=False, record="fp32",
                                  sparse_adam=False, mip2d=0.0, log_every=0)
    _, cams, imgs, tr_idx, te_idx = train.make_dataset(gt.shape[0], 160, W_FULL, H_FULL, dev, gt=gt)
    init = synth.perturb(gt, 3001, n_keep=100_000)
    runs = {}
    clocks = Clocks(gpu_index)
    clocks.start()
    for spec in args.train_runs:
        res, _ = train.train_run(spec, targs, init, cams, imgs, tr_idx, te_idx, dev)
        runs[spec] = {"s": round(res["seconds"], 2), "psnr_db": round(res["psnr_test"], 3),
                      "P_final": res["P_final"], "steps": res["steps"],
                      "r_m": round(res["schedule"]["r_m"], 2) if "schedule" in res else None,
                      "skipped_steps": res["skipped_steps"]}
    clk = clocks.stop()
    del imgs
    torch.cuda.empty_cache()
    base = runs[args.train_runs[0]]
    for spec, r in runs.items():
        if spec != args.train_runs[0]:
            r["psnr_gap_db"] = round(r["psnr_db"] - base["psnr_db"], 3)
            r["time_ratio"] = round(r["s"] / base["s"], 3)
            r["matched"] = bool(r["psnr_db"] >= base["psnr_db"] - 0.1 and r["s"] < base["s"])
    return {"metric": "s to 30k iterations at matched PSNR (held-out, within 0.1 dB of the first run)",
            "scene": "textured 2M-Gaussian ground truth, 140 train / 20 held-out views at 1237x822, init 100k",
            "baseline": args.train_runs[0], "runs": runs, "clocks": clk}


# --------------------------------------------------------------------------- oracle (CPU)
def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _bands(H, tile, n):
    """[y0, y1) pixel-row bands of whole tile rows, at most n of them."""
    TY = (H + tile - 1) // tile
    n = max(1, min(n, TY))
    edges = [round(i * TY / n) for i in range(n + 1)]
    return [(edges[i] * tile, min(H, edges[i + 1] * tile)) for i in range(n) if edges[i + 1] > edges[i]]


def oracle_step(model, view, W, H, tile, target, pool, threads, lam=0.2, bg=(0.0, 0.0, 0.0), keep=False):
    """Wall seconds of one training step of the FP64 oracle on one view, the
    bench's step: projection, binning, Eq. 1, (1 - lam) L1 + lam D-SSIM,
    adjoint, projection adjoint, Adam.  The oracle's functions run unmodified
    on independent parts of the step, one part per host thread (ctypes and
    numpy release the GIL):
      * per-Gaussian stages on `threads` contiguous chunks of the Gaussians;
      * per-pixel stages on bands of whole tile rows (4 per thread, for
        balance): each band is binned and composited as a view of its own, the
        band's Gaussians' v shifted by the band's first row (a multiple of the
        tile edge, so the tile grid is the full view's and every band list is
        the full list restricted to its tiles), and the bands' 2D gradients
        summed per Gaussian;
      * the SSIM term on the same bands with a 10-row halo (the window's
        reach, 5 rows, twice: statistics, then the adjoint filter), so each
        band's interior rows are exact.
    Returns (seconds, info); with keep, info also holds the image, the loss
    gradient, the 2D gradients and the parameter gradients."""
    import oracle
    from oracle import ssim as ossim
    k = oracle.consts(tile=tile)
    fx, fy, cx, cy = view["intr"]
    cam = oracle.camera(view["viewmat"], fx, fy, cx, cy, W, H)
    P = model.shape[0]
    g64 = np.asarray(model, np.float64)
    cuts = np.linspace(0, P, threads + 1).astype(np.int64)
    chunks = [(int(cuts[i]), int(cuts[i + 1])) for i in range(threads) if cuts[i + 1] > cuts[i]]
    bands = _bands(H, tile, 4 * threads)
    bg = np.asarray(bg, np.float64)
    t0 = time.perf_counter()
    prs = list(pool.map(lambda c: oracle.project(g64[c[0]:c[1]], cam, k), chunks))
    feat = np.concatenate([p["feat"] for p in prs])
    radius = np.concatenate([p["radius"] for p in prs])
    dkey = np.concatenate([p["depth_key"] for p in prs])
    vis = radius > 0
    v_lo = feat[:, 1] - radius
    v_hi = feat[:, 1] + radius

    def fwd(band):
        y0, y1 = band
        idx = np.flatnonzero(vis & (v_hi >= y0 - tile) & (v_lo < y1 + tile))
        fb = feat[idx].copy()
        fb[:, 1] -= y0
        bs = oracle.bin_sort(fb[:, :2], radius[idx], dkey[idx], W, y1 - y0, tile)
        rf = oracle.render_fwd(fb, W, y1 - y0, tile, bs["gid"], bs["ranges"], bg, k)
        return idx, fb, bs, rf
    parts = list(pool.map(fwd, bands))
    img = np.concatenate([p[3]["img"] for p in parts], axis=1)
    n = img.size

    def loss(band):
        y0, y1 = band
        a0, a1 = max(0, y0 - 10), min(H, y1 + 10)
        xb, yb = img[:, a0:a1], target[:, a0:a1]
        smap = ossim.ssim_map(xb, yb)[:, y0 - a0:y1 - a0]
        sg = ossim.ssim_grad(xb, yb)[:, y0 - a0:y1 - a0] * (xb.size / n)
        d = img[:, y0:y1] - target[:, y0:y1]
        return np.abs(d).sum(), smap.sum(), (1 - lam) * np.sign(d) / n - lam * sg
    ls = list(pool.map(loss, bands))
    loss_val = (1 - lam) * sum(x[0] for x in ls) / n + lam * (1 - sum(x[1] for x in ls) / n)

    def bwd(i):
        (y0, y1), (idx, fb, bs, rf) = bands[i], parts[i]
        return idx, oracle.render_bwd(fb, W, y1 - y0, tile, bs["gid"], bs["ranges"], bg, k, ls[i][2])
    g2 = np.zeros((P, 9))
    for idx, gb in pool.map(bwd, range(len(bands))):
        g2[idx] += gb
    grads = list(pool.map(lambda c: oracle.project_bwd(g64[c[0]:c[1]], cam, k, g2[c[0]:c[1]]), chunks))

    def adam(ci):
        c = chunks[ci]
        pm = g64[c[0]:c[1]].copy()
        mm = np.zeros_like(pm)
        vv = np.zeros_like(pm)
        oracle.adam(pm, grads[ci], mm, vv, 1e-3, 0.9, 0.999, 1e-15, 1)
    list(pool.map(adam, range(len(chunks))))
    dt = time.perf_counter() - t0
    M = int(sum(p[2]["M"] for p in parts))
    info = dict(loss=float(loss_val), pairs=M, bands=len(bands), chunks=len(chunks))
    if keep:
        info.update(img=img, dL=np.concatenate([x[2] for x in ls], axis=1), grad2d=g2,
                    grad=np.concatenate(grads))
    return dt, info


def _cfg0_step():
    """Config 0 in full: 1,000 Gaussians, 64x64, tile 16, L1 against a uniform
    target, one thread (seconds)."""
    import oracle
    from paper_2503_18402_gb300 import synth
    g = np.asarray(synth.random_gaussians(1000, 1000), np.float64)
    cam = synth.camera_cfg0(64, 64, 4.0)
    tgt = synth.target_image(64, 64, 3000)
    fx, fy, cx, cy = cam["intr"]
    ocam = oracle.camera(cam["viewmat"], fx, fy, cx, cy, 64, 64)
    k = oracle.consts(tile=16)
    t = time.perf_counter()
    f = oracle.forward(g, ocam, k)
    _, dL = oracle.loss_l1(f["img"], tgt)
    oracle.backward(g, ocam, k, f, dL)
    return time.perf_counter() - t


def cpu_baseline(model, view, targets_np, tile, c4_scene=True):
    """The oracle on the host cores (all of them), measured on whole views:
    the bench view (value), and the four reference measurements: config 0 in
    full, one 309x205 and one 1237x822 view of the 2M-Gaussian scene, the
    64x64 centre crop of a 1600x1063 view of a 6M-Gaussian scene."""
    from concurrent.futures import ThreadPoolExecutor
    threads = host_threads()
    with ThreadPoolExecutor(threads) as pool:
        t_full, info = oracle_step(model, view, W_FULL, H_FULL, tile, targets_np, pool, threads)
        c0 = {"cfg0_64x64_1k_ms": round(_cfg0_step() * 1e3, 2),
              "view_1237x822_2M_ms": round(t_full * 1e3, 1)}
        w4, h4 = W_FULL // 4, H_FULL // 4
        fx, fy, cx, cy = view["intr"]
        s4 = w4 / W_FULL
        v4 = dict(viewmat=view["viewmat"], intr=(fx * s4, fy * h4 / H_FULL, cx * s4, cy * h4 / H_FULL))
        tgt4 = targets_np[:, :h4 * 4:4, :w4 * 4:4].copy()
        t4, _ = oracle_step(model, v4, w4, h4, tile, tgt4, pool, threads)
        c0[f"view_{w4}x{h4}_2M_ms"] = round(t4 * 1e3, 1)
        if c4_scene:
            from paper_2503_18402_gb300 import synth
            g6 = synth.textured_scene(6_000_000, 1004)
            cams = synth.ring_cameras(300, 1600, 1063, 5.0, 2004)
            fx, fy, cx, cy = cams[0]["intr"]
            crop = dict(viewmat=cams[0]["viewmat"], intr=(fx, fy, cx - (1600 - 64) / 2, cy - (1063 - 64) / 2))
            tgt = np.random.default_rng(4).uniform(size=(3, 64, 64))
            tc, _ = oracle_step(g6, crop, 64, 64, tile, tgt, pool, threads)
            c0["crop_64x64_of_1600x1063_6M_ms"] = round(tc * 1e3, 1)
            del g6
    return {"value": round(t_full * 1e3, 1), "unit": "ms/view", "cores": threads, "kind": "oracle",
            "sample": (f"one whole {W_FULL}x{H_FULL} view of the bench workload (no extrapolation): FP64 oracle, "
                       f"{threads} host threads over {info['chunks']} Gaussian chunks and {info['bands']} "
                       f"tile-row bands, tile {tile}, 0.8 L1 + 0.2 D-SSIM, {info['pairs']} pairs"),
            "measurements": c0}


def run_reference(args):
    """The reference arm: the FP64 oracle on all host cores, one whole view of
    the bench workload per step (same scene, views, tile, loss)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from concurrent.futures import ThreadPoolExecutor
    from paper_2503_18402_gb300 import synth
    gt = synth.textured_scene(args.n_gauss, 1001)
    model = synth.jitter(gt, 3001)
    cams = synth.ring_cameras(160, W_FULL, H_FULL, 5.0, 2001)
    views = [cams[(j * 10) % 160] for j in range(N_VIEWS)]
    threads = host_threads()
    rng = np.random.default_rng(5)
    target = rng.uniform(size=(3, H_FULL, W_FULL))
    times = []
    info = None
    with ThreadPoolExecutor(threads) as pool:
        for i in range(args.warmup + args.steps):
            t, info = oracle_step(model, views[i % N_VIEWS], W_FULL, H_FULL, BENCH_TILE, target, pool, threads)
            if i >= args.warmup:
                times.append(t)
    ms = 1e3 * sum(times) / len(times)
    sample = (f"every step one whole {W_FULL}x{H_FULL} view (no extrapolation); FP64 oracle on {threads} host "
              f"threads ({info['chunks']} Gaussian chunks, {info['bands']} tile-row bands), tile {BENCH_TILE}, "
              f"0.8 L1 + 0.2 D-SSIM")
    out = {"metric": METRIC, "value": round(ms, 1),
           "unit": "ms/view", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(ms, 1), "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic (seeded textured scene)", "config": config(args, model.shape[0]),
           "impl": "reference",
           "cpu_baseline": {"value": round(ms, 1), "unit": "ms/view", "cores": threads, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(ms, 1), "unit": "ms/view", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
