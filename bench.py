#!/usr/bin/env python
"""Benchmark of the Gaussian-splatting hot path on one GB300 (or N, one
process per GPU under torchrun, each rendering its own copy of the workload:
weak scaling, no collective on the data path).

One step = project -> bin/sort -> blend forward (tensor-core variant) ->
blend backward over the 1280x720, 200k-Gaussian, SH-degree-3 synthetic scene
(seed 0), inputs resident in HBM.  The metric is Gaussian-pixel evaluations
per second, evaluations = sum over pixels of n_contrib (the pairs Eq. 1 with
the skip/stop rules must examine), counted once per forward and once per
backward.  L2 is flushed (256 MB write) before every timed step.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead (the reference arm), on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "blend ms/frame & Gaussian-pixel evals/s (fwd, fwd+bwd) TC vs FP32 CUDA-core"
UNIT = "Gaussian-pixel evals/s"
WORKLOADS = {
    0: "256x256, 10k Gaussians, SH degree 0, seed 0",
    1: "1280x720, 200k Gaussians, SH degree 3, seed 0",
    2: "1920x1080, 1M Gaussians in 64 anisotropic clusters, SH degree 0, seed 0",
    3: "ring camera 0 of 16 (resolution drawn from 640x480..1920x1080), 1.5M clustered Gaussians, seed 0",
    4: "3840x2160, 3M Gaussians, heavy-tailed scales, Beta(0.5, 0.5) opacity, SH degree 3, seed 0",
}
WORKLOAD_NOTE = " (synthetic stand-in for the paper's trained scenes)"

# DRAM traffic per launch from ncu captures, keyed by kernel, with the SHA-256 of
# the kernel's source when it was measured and the workload it was measured on
# (entries for another source or workload are not reported).
KNOWN_TRAFFIC = {
    # profiles/k_blend_tc_fp16split_1280x720_200k.md, profiles/k_blend_tc_bwd_fp16split_1280x720_200k.md
    # (dram__bytes_read.sum + dram__bytes_write.sum, median over the captured launches; forward at chunk 32).
    # Since the captures only the host-side launch wrappers changed (launch shapes cached under a lock):
    # the kernels' device code and their grids are the captured ones.
    "k_blend_tc<fp16_split>": {"bytes": 9740672, "src": "758192731a592fb3", "config": 1},
    "k_blend_tc_bwd<fp16_split>": {"bytes": 31102976, "src": "134ba8c991a6bcf0", "config": 1},
}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--variant", default="fp16_split")
    p.add_argument("--config", type=int, default=1)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--quick", action="store_true", help="skip the per-variant blend sweep")
    return p.parse_args()


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type); never raises."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:  # lscpu missing or failing: fall through
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine() or "unknown"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock/throttle sampling every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [x.strip() for x in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if "Active" in r[5 + i] and "Not" not in r[5 + i]})
        load = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(load) if load else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons, "samples": len(rows)}


def read_hbm_peak():
    """Measured copy bandwidth (GB/s) of this machine's GPUs, else None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return None


def source_digest(*names):
    import hashlib
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2604_02120_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------ ours ----

def run_ours(args):
    import torch
    from paper_2604_02120_gb300 import gs, scenes

    ws_n, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws_n > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gs.load()
    sc = scenes.make_config(args.config, seed=0)
    cam = sc.cameras[0]
    W, H = cam.width, cam.height
    dev = gs.scene_to_device(sc)
    fp32 = gs.make_opts("fp32")
    dL = torch.from_numpy(scenes.upstream_grad(0, [cam])[0]).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    # capacity from one synchronising bin/sort; the timed steps then never
    # synchronise the host (gs_bin_sort_views in graph mode)
    proj0 = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    count0 = gs.BinSorter("cuda", 1 << 20).run(proj0["mean2d"], proj0["radius"], proj0["depth"], W, H)["n_instances"]
    capacity = int(count0 * 1.25) + 4096
    n = sc.n
    ws = torch.empty(gs.gs_bin_sort_workspace_size(n, capacity, W, H) + 256, dtype=torch.uint8, device="cuda")
    ids = torch.empty(capacity, dtype=torch.int32, device="cuda")  # the blends need no sorted keys
    ranges = torch.empty(2 * gs.num_tiles(W, H), dtype=torch.int32, device="cuda")
    count_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    # the opacity-aware step sorts into buffers of its own, so the full lists
    # (and the forward outputs that index them) stay intact for the timings below
    t_ids = torch.empty_like(ids)
    t_ranges, t_count = torch.empty_like(ranges), torch.zeros_like(count_dev)
    # longest tile lists first (gs_tile_order after every bin/sort)
    order, t_order = torch.empty(gs.num_tiles(W, H), dtype=torch.int32, device="cuda"), \
        torch.empty(gs.num_tiles(W, H), dtype=torch.int32, device="cuda")
    opts = gs.make_opts(args.variant, tile_order=order)
    t_opts = gs.make_opts(args.variant, tile_order=t_order)

    def step(ev=None, tight=False):
        if ev:
            ev[0].record(stream)
        proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
        if ev:
            ev[1].record(stream)
        # opacity-aware lists: the exponent each splat must reach in a tile (gs_alpha_power_min)
        pmin = gs.alpha_power_min(dev["opacities"]) if tight else None
        i_, r_, c_ = (t_ids, t_ranges, t_count) if tight else (ids, ranges, count_dev)
        gs.gs_bin_sort_views(1, n, proj["mean2d"], proj["radius"], proj["depth"], [W], [H], capacity, ws, None, i_,
                             r_, count_dev=c_, conic=proj["conic"] if tight else None, power_min=pmin)
        o_ = t_opts if tight else opts
        gs.tile_order(r_, [W], [H], out=t_order if tight else order)
        bs = dict(tile_ranges=r_, ids=i_)
        if ev:
            ev[2].record(stream)
        fwd = gs.blend_forward(W, H, bs, proj, dev["opacities"], o_)
        if ev:
            ev[3].record(stream)
        g = gs.blend_backward(W, H, bs, proj, dev["opacities"], o_, fwd, dL)
        if ev:
            ev[4].record(stream)
        bs["n_instances"] = count0
        return proj, bs, fwd, g

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    proj, bs, fwd, _ = step()
    tuned = None
    if args.variant != "fp32":  # the forward's pipeline shape by the library's own measurement
        gs.gs_blend_autotune([W], [H], n, ranges, ids, proj["mean2d"], proj["conic"], dev["opacities"], proj["rgb"],
                             opts, fwd["image"], fwd["T_final"], fwd["n_contrib"])
        t_opts.chunk, t_opts.stages = opts.chunk, opts.stages
        tuned = {"chunk": opts.chunk, "stages": opts.stages}
        proj, bs, fwd, _ = step()
    evals_fwd = int(fwd["n_contrib"].sum().item())
    n_inst = bs["n_instances"]

    # ---- the step as four CUDA graphs (projection; bin/sort and tile order;
    # forward; backward), replayed with CUDA events between them on the
    # launching stream: the stage chain without per-launch host and queue gaps
    graphs = []

    # with a process group, its watchdog thread queries CUDA events while the
    # main thread captures: only this thread's calls are checked then
    mode = {"capture_error_mode": "thread_local"} if dist else {}

    def capture(fn):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, **mode):
            r = fn()
        graphs.append(g)
        return r

    launches_c = gs.gs_launch_count()
    g_proj = capture(lambda: gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam))

    def sort_stage():
        gs.gs_bin_sort_views(1, n, g_proj["mean2d"], g_proj["radius"], g_proj["depth"], [W], [H], capacity, ws, None,
                             ids, ranges, count_dev=count_dev)
        gs.tile_order(ranges, [W], [H], out=order)

    capture(sort_stage)
    g_bs = dict(tile_ranges=ranges, ids=ids)
    g_fwd = capture(lambda: gs.blend_forward(W, H, g_bs, g_proj, dev["opacities"], opts))
    capture(lambda: gs.blend_backward(W, H, g_bs, g_proj, dev["opacities"], opts, g_fwd, dL))
    launches_per_step = gs.gs_launch_count() - launches_c  # the library's kernels in the four graphs
    for _ in range(3):
        for g in graphs:
            g.replay()
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    assert torch.equal(g_fwd["image"], fwd["image"]) and torch.equal(g_fwd["n_contrib"], fwd["n_contrib"])

    K = args.steps
    E = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    st_ev = [(E(), E()) for _ in range(K)]
    k_ev = [tuple(E() for _ in range(5)) for _ in range(K)]
    with ClockSampler(local) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for k in range(K):
            flush.zero_()
            st_ev[k][0].record(stream)
            k_ev[k][0].record(stream)
            for i, g in enumerate(graphs):
                g.replay()
                k_ev[k][i + 1].record(stream)
            st_ev[k][1].record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall = time.perf_counter() - wall0
    launches = launches_per_step * K
    clocks = clk.summary()
    assert gs.gs_sync_status() == gs.GS_OK  # also catches a capacity overflow of the bin/sort
    step_ms = [a.elapsed_time(b) for a, b in st_ev]
    proj_ms = [e[0].elapsed_time(e[1]) for e in k_ev]
    sort_ms = [e[1].elapsed_time(e[2]) for e in k_ev]
    fwd_ms = [e[2].elapsed_time(e[3]) for e in k_ev]
    bwd_ms = [e[3].elapsed_time(e[4]) for e in k_ev]
    dev_ms = sum(step_ms)
    if dist:
        t = torch.tensor([dev_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_ms = float(t.item())
    evals_step = 2 * evals_fwd  # forward and backward each examine sum(n_contrib) pairs
    value = ws_n * evals_step * K / (dev_ms / 1e3)

    # ---- the same step launched call by call (no graphs), for comparison
    Ke = min(K, 200)
    e_ev = [(E(), E()) for _ in range(Ke)]
    for k in range(Ke):
        flush.zero_()
        e_ev[k][0].record(stream)
        step()
        e_ev[k][1].record(stream)
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    eager_ms = statistics.mean(a.elapsed_time(b) for a, b in e_ev)

    # ---- the same step with opacity-aware tile lists (same image; fewer instances)
    for _ in range(3):
        step(tight=True)
    _, tbs, tfwd, _ = step(tight=True)
    t_inst = int(t_count.item())
    t_evals = 2 * int(tfwd["n_contrib"].sum().item())
    Kt = min(K, 200)
    t_ev = [tuple(E() for _ in range(5)) for _ in range(Kt)]
    for k in range(Kt):
        flush.zero_()
        step(t_ev[k], tight=True)
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    t_ms = statistics.mean(e[0].elapsed_time(e[4]) for e in t_ev)
    tight_line = {"ms_per_step": round(t_ms, 5), "instances": t_inst, "evals_per_step": t_evals,
                  "breakdown_ms": {"project": round(statistics.mean(e[0].elapsed_time(e[1]) for e in t_ev), 5),
                                   "bin_sort": round(statistics.mean(e[1].elapsed_time(e[2]) for e in t_ev), 5),
                                   "blend_forward": round(statistics.mean(e[2].elapsed_time(e[3]) for e in t_ev), 5),
                                   "blend_backward": round(statistics.mean(e[3].elapsed_time(e[4]) for e in t_ev), 5)},
                  "steps": Kt, "note": "gs_bin_sort_views with conic + gs_alpha_power_min: a splat keeps a tile "
                                       "only if alpha can reach 1/255 there; the image equals the full lists' "}

    # ---- issued pairs: every chunk a tile evaluates before its exit, at all 256 pixels
    issued_line = None
    if args.variant != "fp32":
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        o_cnt = gs.make_opts(args.variant, chunk=opts.chunk, stages=opts.stages, tile_order=order, issued_pairs=cnt)
        out_c = gs.blend_forward(W, H, bs, proj, dev["opacities"], o_cnt)
        issued = int(cnt.item())
        assert gs.gs_sync_status() == gs.GS_OK and torch.equal(out_c["n_contrib"], fwd["n_contrib"])
        issued_line = {"evaluated_per_frame": evals_fwd, "issued_per_frame": issued,
                       "issued_over_evaluated": round(issued / max(evals_fwd, 1), 3),
                       "note": "evaluated = sum of n_contrib (the metric's pairs); issued = 256 x the splats of "
                               "every chunk the tensor-core forward evaluates before a tile's exit"}

    # ---- projection backward: dL/d(means, scales, quats, sh) from the blend's
    # splat gradients (HBM-bound, one thread per Gaussian)
    pproj, _, _, gb = step()
    pb_args = (dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam, pproj["radius"],
               gb["mean2d"], gb["conic"], gb["rgb"])
    for _ in range(3):
        gs.project_backward(*pb_args)
    pb_ev = []
    for _ in range(min(K, 200)):
        flush.zero_()
        a, b = E(), E()
        a.record(stream)
        gs.project_backward(*pb_args)
        b.record(stream)
        pb_ev.append((a, b))
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    pb_ms = statistics.median(a.elapsed_time(b) for a, b in pb_ev)
    Ksh = (sc.sh_degree + 1) ** 2
    # per Gaussian: means, scales, quats, sh, radius, dmean2d, dconic, drgb read; dmeans, dscales, dquats, dsh written
    pb_bytes = n * (4 * (3 + 3 + 4 + 3 * Ksh + 1 + 2 + 3 + 3) + 4 * (3 + 3 + 4 + 3 * Ksh))
    hbm = read_hbm_peak()
    pb_line = {"ms": round(pb_ms, 5), "bytes_per_gaussian": pb_bytes // n,
               "achieved_gb_per_s": round(pb_bytes / pb_ms / 1e6, 1),
               "peak_gb_per_s": hbm, "frac": round(pb_bytes / pb_ms / 1e6 / hbm, 4) if hbm else None,
               "note": "gs_project_backward alone (k_project_bwd), L2 flushed before each launch, median of "
                       f"{len(pb_ev)}; peak = measured copy bandwidth"}

    # ---- small scene: projection + bin/sort fused into one cooperative launch
    small_line = run_small_fused(gs, torch, gs.make_opts(args.variant), flush, min(K, 200))
    # ---- all cameras of the ring scene in one batched step (one launch per stage over every view)
    batched_line = run_batched(gs, torch, sc, dev, args.variant, flush, min(K, 50)) if args.config == 3 else None

    # ---- blend-only ms/frame per variant (forward), tensor core vs FP32 CUDA core
    blend = {}
    if not args.quick:
        for name in ["fp32", "fp16", "bf16", "fp16_split", "bf16_split", "fp8_split"]:
            o = gs.make_opts(name, tile_order=order)  # the main step's lists and order
            for _ in range(3):
                gs.blend_forward(W, H, bs, proj, dev["opacities"], o)
            times = []
            for _ in range(min(max(K, 10), 50)):
                flush.zero_()
                a, b = E(), E()
                a.record(stream)
                out = gs.blend_forward(W, H, bs, proj, dev["opacities"], o)
                b.record(stream)
                times.append((a, b))
            torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(b) for a, b in times)
            ev = int(out["n_contrib"].sum().item())
            blend[name] = {"ms_per_frame": round(ms, 5), "evals_per_s": ev / (ms / 1e3)}
        # backward (FP32 CUDA-core recompute) alone
        times = []
        for _ in range(min(max(K, 10), 50)):
            flush.zero_()
            a, b = E(), E()
            a.record(stream)
            gs.blend_backward(W, H, bs, proj, dev["opacities"], fp32, fwd, dL)
            b.record(stream)
            times.append((a, b))
        torch.cuda.synchronize()
        ms = statistics.median(a.elapsed_time(b) for a, b in times)
        blend["backward_fp32"] = {"ms_per_frame": round(ms, 5), "evals_per_s": evals_fwd / (ms / 1e3)}

    # ---- end to end through the public API with host buffers
    e2e = run_e2e(args, gs, torch, sc, cam, opts, capacity, dL, flush, evals_step, ws_n, dist)

    # ---- roofline of the dominant blend kernel (MUFU-bound: the forward pass
    # takes one exp2 per evaluated pair, the backward pass an exp2 and a reciprocal)
    # MUFU rates measured on this GPU by the library's own microbenchmark
    mp = gs.gs_measure_peaks()
    ex2_g, rcp_g = mp["ex2_per_s"] / 1e9, mp["rcp_per_s"] / 1e9
    f_ms, b_ms = statistics.mean(fwd_ms), statistics.mean(bwd_ms)
    tc = args.variant != "fp32"
    if f_ms >= b_ms:
        kern, t_ms, per_pair = (f"k_blend_tc<{args.variant}>" if tc else "k_blend_fp32_fwd"), f_ms, 1
        src = ("blend_tc.cuh",) if tc else ("blend_fp32.cu",)
    else:
        kern, t_ms, per_pair = (f"k_blend_tc_bwd<{args.variant}>" if tc else "k_blend_fp32_bwd"), b_ms, 2
        src = ("blend_tc_bwd.cuh", "blend_tc.cuh") if tc else ("blend_fp32.cu",)
    achieved = evals_fwd / (t_ms / 1e3) / 1e9
    # pairs/s if MUFU were the only limit: an ex2 per pair, plus a reciprocal in the backward pass
    peak = ex2_g if per_pair == 1 else 1.0 / (1.0 / ex2_g + 1.0 / rcp_g)
    tr = KNOWN_TRAFFIC.get(kern)
    traffic = tr["bytes"] if tr and tr["src"] == source_digest(*src) and tr["config"] == args.config else None
    roofline = {"bound": "alu", "kernel": kern, "achieved": round(achieved, 2), "peak": round(peak, 1),
                "unit": "G evals/s (MUFU-bound)", "frac": round(achieved / peak, 4), "traffic": traffic,
                "peak_source": f"gs_measure_peaks on this GPU: {ex2_g:.0f} G ex2/s, {rcp_g:.0f} G rcp/s at "
                               f"{mp['sm_mhz']:.0f} MHz ({mp['sms']} SMs); "
                               + ("1 ex2 per pair" if per_pair == 1 else "1 ex2 + 1 rcp per pair"),
                "launch_ms": round(t_ms, 5)}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_n, "steps": K, "warmup": args.warmup,
        "ms_per_step": dev_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config] + WORKLOAD_NOTE, "blend_variant": args.variant,
                   "step": "project + bin_sort + tile_order + blend_forward + blend_backward",
                   "tile_order": "longest list first (gs_tile_order)",
                   "blend_shape": tuned or "per-tile FP32 blocks",
                   "evals_per_step": evals_step, "instances": n_inst, "pixels": W * H,
                   "l2": "flushed before every timed step (256 MB write)", "parallelism": f"replica x{ws_n}",
                   "bin_sort": "no host synchronisation (fixed capacity, count on the device)",
                   "launch": "each stage (project; bin_sort + tile_order; forward; backward) replayed as a CUDA "
                             "graph, CUDA events between the stages"},
        "breakdown_ms": {"project": round(statistics.mean(proj_ms), 5), "bin_sort": round(statistics.mean(sort_ms), 5),
                         "blend_forward": round(f_ms, 5), "blend_backward": round(b_ms, 5),
                         "gaps": round(dev_ms / K - f_ms - b_ms - statistics.mean(proj_ms)
                                       - statistics.mean(sort_ms), 5)},
        "wall_ms_per_step": wall * 1e3 / K,
        "eager_ms_per_step": round(eager_ms, 5),
        "launches_per_step": launches_per_step,
        "blend_forward_by_variant": blend,
        "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
        "opacity_aware_lists": tight_line,
        "projection_backward": pb_line,
        **({"forward_pairs": issued_line} if issued_line else {}),
        "small_scene_fused": small_line,
        **({"batched_views": batched_line} if batched_line else {}),
    }
    if rank == 0 and ws_n == 1 and not args.no_cpu_baseline:  # the oracle on the host cores: N = 1 only
        line["cpu_baseline"] = cpu_baseline(cam, proj, bs, sc, dL, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_small_fused(gs, torch, opts, flush, K):
    """The 256x256, 10k-Gaussian scene (the launch-bound case): the step with
    gs_project + gs_bin_sort_views (graph mode, 9 launches) against the step
    with gs_project_bin_small (one cooperative launch), both followed by the
    same blend forward and backward; L2 flushed before every step."""
    from paper_2604_02120_gb300 import scenes
    sc = scenes.make_config(0, seed=0)
    cam = sc.cameras[0]
    W, H, n = cam.width, cam.height, sc.n
    dev = gs.scene_to_device(sc)
    dL = torch.from_numpy(scenes.upstream_grad(0, [cam])[0]).cuda()
    stream = torch.cuda.current_stream()
    capacity = 1 << 20
    ws = torch.empty(gs.gs_bin_sort_workspace_size(n, capacity, W, H) + 256, dtype=torch.uint8, device="cuda")
    ids = torch.empty(capacity, dtype=torch.int32, device="cuda")
    ranges = torch.empty(2 * gs.num_tiles(W, H), dtype=torch.int32, device="cuda")
    count = torch.zeros(1, dtype=torch.int64, device="cuda")
    args3 = (dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)

    def unfused():
        proj = gs.project(*args3)
        gs.gs_bin_sort_views(1, n, proj["mean2d"], proj["radius"], proj["depth"], [W], [H], capacity, ws, None, ids,
                             ranges, count_dev=count)
        return proj, dict(tile_ranges=ranges, ids=ids)

    def fused():
        return gs.project_bin_small(*args3, max_per_tile=1024)

    out = {}
    for name, front in (("unfused", unfused), ("fused", fused)):
        def step():
            proj, bs = front()
            fwd = gs.blend_forward(W, H, bs, proj, dev["opacities"], opts)
            gs.blend_backward(W, H, bs, proj, dev["opacities"], opts, fwd, dL)
        for _ in range(3):
            step()
        ev = []
        for _ in range(K):
            flush.zero_()
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            proj, bs = front()
            b.record(stream)
            fwd = gs.blend_forward(W, H, bs, proj, dev["opacities"], opts)
            gs.blend_backward(W, H, bs, proj, dev["opacities"], opts, fwd, dL)
            c.record(stream)
            ev.append((a, b, c))
        torch.cuda.synchronize()
        assert gs.gs_sync_status() == gs.GS_OK
        out[name] = {"ms_per_step": round(statistics.median(a.elapsed_time(c) for a, b, c in ev), 5),
                     "project_bin_ms": round(statistics.median(a.elapsed_time(b) for a, b, c in ev), 5)}
    out["workload"] = "256x256, 10k Gaussians, SH degree 0, seed 0; step = project + bin + blend fwd + bwd"
    return out


def run_batched(gs, torch, sc, dev, variant, flush, K):
    """Every camera of the scene in one BatchRenderer step (gs_project_views ->
    gs_bin_sort_views -> tile order -> one persistent forward and one backward
    over the tiles of all views), replayed as a CUDA graph, against the views
    rendered one after another with the single-view calls (same step each)."""
    from paper_2604_02120_gb300 import scenes
    cams = sc.cameras
    V, n = len(cams), sc.n
    stream = torch.cuda.current_stream()
    # capacity from one synchronising sort of all views
    f32 = dict(device="cuda", dtype=torch.float32)
    m2, co = torch.empty(V * n, 2, **f32), torch.empty(V * n, 3, **f32)
    de, rg = torch.empty(V * n, **f32), torch.empty(V * n, 3, **f32)
    ra, tt = (torch.empty(V * n, device="cuda", dtype=torch.int32) for _ in range(2))
    gs.gs_project_views(n, dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cams, m2, co, de,
                        ra, rg, tt)
    widths, heights = [c.width for c in cams], [c.height for c in cams]
    cap0 = 1 << 20  # an overflowing synchronising sort still reports the instance count
    ws = torch.empty(gs.gs_bin_sort_workspace_size(V * n, cap0, widths[0], heights[0]) + 256, dtype=torch.uint8,
                     device="cuda")
    ids = torch.empty(cap0, dtype=torch.int32, device="cuda")
    rng = torch.empty(2 * sum(gs.num_tiles(w, h) for w, h in zip(widths, heights)), dtype=torch.int32, device="cuda")
    st, count = gs.gs_bin_sort_views(V, n, m2, ra, de, widths, heights, cap0, ws, None, ids, rng, check=False)
    assert st in (gs.GS_OK, gs.GS_ERR_CAPACITY) and count > 0
    del ws, ids, rng, m2, co, de, rg, ra, tt
    capacity = int(count * 1.25) + 4096
    dL = torch.from_numpy(np.concatenate([g.reshape(-1) for g in scenes.upstream_grad(0, cams)])).cuda()
    br = gs.BatchRenderer(dev, cams, gs.make_opts(variant), capacity)
    br.dL.copy_(dL)
    br.step()
    br.capture()
    for _ in range(3):
        br.graph.replay()
    ev = []
    for _ in range(K):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        br.graph.replay()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    batched = statistics.median(a.elapsed_time(b) for a, b in ev)
    evals = 2 * int(br.nc.sum().item())
    del br
    # the same views one after another (single-view calls, each sorted and blended on its own)
    opts = gs.make_opts(variant)
    sorters = [gs.BinSorter("cuda", 1 << 22) for _ in cams]
    dls = [torch.from_numpy(g).cuda() for g in scenes.upstream_grad(0, cams)]

    def seq():
        for cam, so, g in zip(cams, sorters, dls):
            proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
            bs = so.run(proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height)
            fwd = gs.blend_forward(cam.width, cam.height, bs, proj, dev["opacities"], opts)
            gs.blend_backward(cam.width, cam.height, bs, proj, dev["opacities"], opts, fwd, g)
    for _ in range(2):
        seq()
    ev = []
    for _ in range(min(K, 10)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        seq()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    sequential = statistics.median(a.elapsed_time(b) for a, b in ev)
    return {"views": V, "instances": int(count), "evals_per_step": evals, "batched_ms": round(batched, 4),
            "batched_evals_per_s": evals / (batched / 1e3), "sequential_ms": round(sequential, 4),
            "note": "batched: BatchRenderer step of all views captured in a CUDA graph; sequential: per view "
                    "gs_project + gs_bin_sort (synchronising) + blend forward + backward; L2 flushed before each"}


def run_e2e(args, gs, torch, sc, cam, opts, capacity, dL, flush, evals_step, ws, dist):
    """Same step through the public API from pinned host buffers: every step
    copies the scene host-to-device and the image and the four gradient
    arrays device-to-host.  Timed twice: serialised (BatchRenderer: copy in,
    compute, copy out) and pipelined (PipelinedRenderer: step k+1's upload
    and step k-1's download overlap step k's compute, as for independent
    frames); `value` is the pipelined figure."""
    W, H = cam.width, cam.height
    host = {k: torch.from_numpy(getattr(sc, k)).pin_memory() for k in ("means", "scales", "quats", "opacities", "sh")}
    n = sc.n
    out_h = {"image": torch.empty(3, H, W).pin_memory(), "mean2d": torch.empty(n, 2).pin_memory(),
             "conic": torch.empty(n, 3).pin_memory(), "opacity": torch.empty(n).pin_memory(),
             "rgb": torch.empty(n, 3).pin_memory()}
    h2d = sum(v.numel() * v.element_size() for v in host.values())
    d2h = sum(v.numel() * v.element_size() for v in out_h.values())

    def timed(step):
        for k in range(max(args.warmup, 3)):
            step(k)
        torch.cuda.synchronize()
        K = args.steps
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(K):
            flush.zero_()
            step(k)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t = time.perf_counter() - t0
        if dist:
            tt = torch.tensor([t], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        return t

    # serialised
    devb = {k: v.to("cuda") for k, v in host.items()}
    br = gs.BatchRenderer(dict(devb, sh_degree=sc.sh_degree), [cam], opts, capacity)
    br.dL.copy_(dL.reshape(-1))
    br.capture()  # the step replayed as one CUDA graph

    def step_serial(k):
        for key, v in host.items():
            devb[key].copy_(v, non_blocking=True)
        br.graph.replay()
        out_h["image"].copy_(br.image.view(3, H, W), non_blocking=True)
        out_h["mean2d"].copy_(br.g_mean2d, non_blocking=True)
        out_h["conic"].copy_(br.g_conic, non_blocking=True)
        out_h["opacity"].copy_(br.g_opac, non_blocking=True)
        out_h["rgb"].copy_(br.g_rgb, non_blocking=True)

    t_serial = timed(step_serial)
    del br, devb
    # pipelined
    pr = gs.PipelinedRenderer(host, sc.sh_degree, [cam], opts, capacity, dL, graphs=True)
    t = timed(lambda k: pr.submit(k, host, out_h))
    K = args.steps
    return {"value": ws * evals_step * K / t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": t * 1e3 / K, "serialised_ms_per_step": t_serial * 1e3 / K,
            "timing": "host wall clock around K steps incl. L2 flush writes; every step copies its inputs in and its "
                      "image and gradients out; pipelined: step k+1's upload and step k-1's download overlap step "
                      "k's compute (independent frames); serialised_ms_per_step: copy in, compute, copy out; "
                      "the compute of a step is one CUDA graph replay (gs.BatchRenderer.capture)"}


# ------------------------------------------------------------ CPU oracle ----

def _oracle_sample(oracle, W, H, ranges, ids, mean2d, conic, opac, rgb, dL, tiles, threads):
    t0 = time.perf_counter()
    r = oracle.blend(W, H, ranges, ids, mean2d, conic, opac, rgb, n_threads=threads, tile_subset=tiles)
    oracle.blend_grad(W, H, ranges, ids, mean2d, conic, opac, rgb, dL, n_threads=threads, tile_subset=tiles)
    dt = time.perf_counter() - t0
    mask = np.zeros((H, W), bool)
    tx = (W + 15) // 16
    for t in tiles:
        mask[16 * (t // tx):16 * (t // tx) + 16, 16 * (t % tx):16 * (t % tx) + 16] = True
    evals = 2 * int(r["n_contrib"][mask].sum())
    return evals, dt


def _calibrate(run, order, threads, seconds):
    """Number of tiles (a prefix of `order`) whose oracle run takes about
    `seconds`: grow a probe until it takes >= 1 s (or covers everything)."""
    k = min(len(order), max(threads, 8))
    while True:
        dt = run(order[:k])
        if dt >= 1.0 or k == len(order):
            break
        k = min(len(order), 4 * k)
    return int(min(len(order), max(k, k * seconds / max(dt, 1e-3))))


def _busy_tiles(ranges):
    lens = ranges[1::2].astype(np.int64) - ranges[0::2]
    return np.nonzero(lens > 0)[0]


def cpu_baseline(cam, proj, bs, sc, dL, seconds):
    """The FP64 oracle (forward blend + gradient) on a random sample of the
    workload's tiles, on all host cores; evals/s over the sampled pixels."""
    import oracle
    W, H = cam.width, cam.height
    ranges = bs["tile_ranges"].cpu().numpy().view(np.uint32)
    ids = bs["ids"].cpu().numpy().view(np.uint32)
    m2 = proj["mean2d"].cpu().numpy().astype(np.float64)
    co = proj["conic"].cpu().numpy().astype(np.float64)
    rgb = proj["rgb"].cpu().numpy().astype(np.float64)
    op = sc.opacities.astype(np.float64)
    g = dL.cpu().numpy().astype(np.float64)
    threads = os.cpu_count() or 1
    busy = _busy_tiles(ranges)
    order = np.random.default_rng(0).permutation(busy)
    k = _calibrate(lambda t: _oracle_sample(oracle, W, H, ranges, ids, m2, co, op, rgb, g, t, threads)[1],
                   order, threads, seconds)
    # the sample, repeated while it takes less than `seconds` in all (a whole small workload)
    ev = reps = 0
    dt = 0.0
    while reps == 0 or dt < seconds:
        e1, d1 = _oracle_sample(oracle, W, H, ranges, ids, m2, co, op, rgb, g, order[:k], threads)
        ev, dt, reps = ev + e1, dt + d1, reps + 1
    return {"value": ev / dt, "unit": UNIT, "cores": threads, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"{k} of {len(busy)} non-empty tiles (random, seed 0) x {reps}, FP64 blend forward + "
                      f"gradient, {dt:.1f} s", "seconds": dt}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2604_02120_gb300 import scenes
    sc = scenes.make_config(args.config, seed=0)
    cam = sc.cameras[0]
    W, H = cam.width, cam.height
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam)
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], pr["depth"].astype(np.float32), W, H)
    dL = scenes.upstream_grad(0, [cam])[0].astype(np.float64)
    op = sc.opacities.astype(np.float64)
    threads = os.cpu_count() or 1
    busy = _busy_tiles(bs["tile_ranges"])
    order = np.random.default_rng(0).permutation(busy)
    per_step_s = min(6.0, 150.0 / max(1, args.steps + args.warmup))
    k = _calibrate(lambda t: _oracle_sample(oracle, W, H, bs["tile_ranges"], bs["ids"], pr["mean2d"], pr["conic"],
                                            op, pr["rgb"], dL, t, threads)[1], order, threads, per_step_s)
    evals_total, t_total = 0, 0.0
    for s in range(args.warmup + args.steps):
        tiles = np.roll(order, -s * k)[:k]
        ev, dt = _oracle_sample(oracle, W, H, bs["tile_ranges"], bs["ids"], pr["mean2d"], pr["conic"], op,
                                pr["rgb"], dL, tiles, threads)
        if s >= args.warmup:
            evals_total += ev
            t_total += dt
    value = evals_total / t_total
    sample = f"{k} of {len(busy)} non-empty tiles per step (rotating), FP64 blend forward + gradient"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_total * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOADS[args.config] + WORKLOAD_NOTE,
                       "step": "FP64 oracle blend forward + gradient on a tile sample"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "cpu_model": cpu_model(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
