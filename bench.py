#!/usr/bin/env python
"""Benchmark of the Gaussian-splatting hot path on one GB300 (or N, one
process per GPU under torchrun).

One step = project -> bin/sort (opacity-aware lists) -> tile order -> blend
forward (tensor-core variant) -> blend backward over the 3840x2160,
3M-Gaussian synthetic scene with heavy-tailed scales (seed 0), inputs resident
in HBM.  The metric is Gaussian-pixel evaluations per second, evaluations =
sum over pixels of n_contrib (the pairs Eq. 1 with the skip/stop rules must
examine), counted once per forward and once per backward.  L2 is flushed
(256 MB write) before every timed step.  With N > 1 ranks the blend is
sharded by tiles (rank r blends tiles t = r mod N) and the per-Gaussian
gradients are all-reduced over NCCL: the frame's work is fixed (strong
scaling).

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

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# ncu captures, keyed by kernel (or stage), with the SHA-256 prefix of the
# sources it was measured with and the workload; an entry whose sources or
# workload differ from the run's is not reported.
KNOWN_TRAFFIC = {}

# Algorithmic work per unit (the roofline numerators; the derivations are in
# the design notes):
#  - FP32 operations per evaluated pair: compositing, skip and stop tests with
#    the exponent from the tensor cores (10), the CUDA-core forward that also
#    evaluates Eq. 3 (16), the backward pass (25);
#  - bytes per instance a blend touches: the id and the splat's record
#    (mean2d 8, conic 12, opacity 4, rgb 12); per pixel written or read:
#    image 12, T_final 4, n_contrib 4 (forward), plus dL/dimage 12 (backward);
#    the backward adds 9 gradient floats per (instance, tile half);
#  - bin/sort: per Gaussian its inputs (mean2d, radius, depth, conic,
#    power_min: 32 bytes) and per instance the sorted id (4 bytes), per tile
#    its range (8 bytes): the least a binning must move.
FP32_OPS = {"forward_tc": 10, "forward_fp32": 16, "backward": 25}
REC_BYTES = 4 + 36
K_OF = {"fp16": 16, "bf16": 16, "fp16_split": 16, "bf16_split": 32, "fp8_split": 64}
DTYPE_OF = {"fp32": "f32 (CUDA-core Eq. 3)", "fp16": "fp16 operands, f32 accumulate",
            "bf16": "bf16 operands, f32 accumulate", "fp16_split": "fp16 hi+lo split operands, f32 accumulate",
            "bf16_split": "bf16 hi+mid+lo split operands, f32 accumulate",
            "fp8_split": "e4m3 5-term split operands (trial), f32 accumulate"}


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--variant", default="bf16_split")
    p.add_argument("--config", type=int, default=4)
    p.add_argument("--full-lists", action="store_true", help="full 3-sigma rectangles instead of opacity-aware lists")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--sustained-seconds", type=float, default=5.0)
    p.add_argument("--quick", action="store_true", help="skip the per-variant sweeps and the 1920x1080 leg")
    p.add_argument("--step-only", action="store_true",
                   help="time the step alone: no sweeps, no side legs (for profiler captures)")
    p.add_argument("--resolution", default=None,
                   help="WxH: render the configuration's scene from the same camera position at this resolution "
                        "(smaller captures of the same kernels); the line then names the resolution")
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
    """nvidia-smi clock/throttle sampling (every interval_ms) while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, interval_ms=50):
        self.gpu = gpu_index
        self.interval = int(interval_ms)
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", str(self.interval)],
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

class Step:
    """Buffers and stages of one step on one camera: project -> (opacity-aware)
    bin/sort -> tile order -> blend forward -> blend backward."""

    def __init__(self, gs, torch, dev, cam, variant, tight, shard=(1, 0)):
        self.gs, self.torch, self.dev, self.cam = gs, torch, dev, cam
        self.W, self.H, self.n = cam.width, cam.height, int(dev["means"].shape[0])
        self.tight = tight
        W, H, n = self.W, self.H, self.n
        self.pmin = torch.empty(n, device="cuda") if tight else None
        # capacity from one synchronising bin/sort; the timed steps then never
        # synchronise the host (gs_bin_sort_views in graph mode)
        proj = self.project()
        cap = 1 << 20
        while True:
            ws = torch.empty(gs.gs_bin_sort_workspace_size(n, cap, W, H) + 256, dtype=torch.uint8, device="cuda")
            ids = torch.empty(cap, dtype=torch.int32, device="cuda")
            ranges = torch.empty(2 * gs.num_tiles(W, H), dtype=torch.int32, device="cuda")
            if tight:
                gs.gs_alpha_power_min(n, dev["opacities"], self.pmin)
            st, count = gs.gs_bin_sort_views(1, n, proj["mean2d"], proj["radius"], proj["depth"], [W], [H], cap, ws,
                                             None, ids, ranges, check=False, conic=proj["conic"] if tight else None,
                                             power_min=self.pmin)
            if st == gs.GS_OK:
                break
            assert st == gs.GS_ERR_CAPACITY, st
            del ws, ids
            cap = count + 1024
        self.count0 = count
        self.capacity = int(count * 1.1) + 4096
        self.ws = torch.empty(gs.gs_bin_sort_workspace_size(n, self.capacity, W, H) + 256, dtype=torch.uint8,
                              device="cuda")
        self.ids = torch.empty(self.capacity, dtype=torch.int32, device="cuda")
        self.ranges = ranges
        self.count_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.order = torch.empty(gs.num_tiles(W, H), dtype=torch.int32, device="cuda")
        self.bs = dict(tile_ranges=self.ranges, ids=self.ids)
        # packed splat records for the TMA-staged forward (measured against the
        # default per-thread loads; the step uses the faster, per-thread loads)
        self.rec = torch.empty(n, 16, device="cuda") if n > 0 else None
        self.opts = gs.make_opts(variant, tile_order=self.order, shard_count=shard[0], shard_index=shard[1])
        del ws, ids

    def project(self):
        d = self.dev
        self.proj = self.gs.project(d["means"], d["scales"], d["quats"], d["sh"], d["sh_degree"], self.cam)
        return self.proj

    def sort(self, proj=None):
        gs, proj = self.gs, proj or self.proj
        if self.tight:
            gs.gs_alpha_power_min(self.n, self.dev["opacities"], self.pmin)
        gs.gs_bin_sort_views(1, self.n, proj["mean2d"], proj["radius"], proj["depth"], [self.W], [self.H],
                             self.capacity, self.ws, None, self.ids, self.ranges, count_dev=self.count_dev,
                             conic=proj["conic"] if self.tight else None, power_min=self.pmin)
        gs.tile_order(self.ranges, [self.W], [self.H], out=self.order)

    def forward(self, proj=None, opts=None):
        self.fwd = self.gs.blend_forward(self.W, self.H, self.bs, proj or self.proj, self.dev["opacities"],
                                         opts or self.opts)
        return self.fwd

    def backward(self, dL, proj=None, fwd=None, opts=None):
        return self.gs.blend_backward(self.W, self.H, self.bs, proj or self.proj, self.dev["opacities"],
                                      opts or self.opts, fwd or self.fwd, dL)

    def eager(self, dL, ev=None, stream=None):
        if ev:
            ev[0].record(stream)
        self.project()
        if ev:
            ev[1].record(stream)
        self.sort()
        if ev:
            ev[2].record(stream)
        self.forward()
        if ev:
            ev[3].record(stream)
        g = self.backward(dL)
        if ev:
            ev[4].record(stream)
        return g


def _events(torch, k):
    return [torch.cuda.Event(enable_timing=True) for _ in range(k)]


def supertile_pairs(torch, gs, st):
    """(Gaussian, supertile of 4 x 4 tiles) pairs of the step's lists: the
    coarse duplication's output count, from the sorted ids and tile ranges."""
    r = st.ranges.view(-1, 2).long()
    lens = (r[:, 1] - r[:, 0]).clamp_min(0)
    tiles = torch.repeat_interleave(torch.arange(lens.numel(), device=lens.device), lens)
    tx = (st.W + 15) // 16
    stx = (tx + 3) // 4
    sup = (tiles // tx // 4) * stx + (tiles % tx) // 4
    ids = st.ids[: int(lens.sum())].long()  # the lists are contiguous, in tile order
    return int(torch.unique(sup * st.n + ids).numel())


def _timed(torch, flush, stream, fn, reps):
    """Median ms of fn() over reps launches, L2 flushed before each."""
    ev = []
    for _ in range(reps):
        flush.zero_()
        a, b = _events(torch, 2)
        a.record(stream)
        fn()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev)


def backward_issued_pairs(torch, n_contrib, chunk=16):
    """Pairs the tensor-core backward evaluates: every pixel of a tile, in
    chunks of 16 splats, up to the tile's longest n_contrib."""
    H, W = n_contrib.shape
    ty, tx = (H + 15) // 16, (W + 15) // 16
    nc = torch.zeros(ty * 16, tx * 16, dtype=torch.int32, device=n_contrib.device)
    nc[:H, :W] = n_contrib
    mx = nc.view(ty, 16, tx, 16).amax(dim=(1, 3)).to(torch.int64)
    return int((((mx + chunk - 1) // chunk) * chunk * 256).sum().item())


def blend_roofline(kind, variant, t_ms, evals, issued, pixels, peaks):
    """Every roofline term of one blend launch, as Gaussian-pixel evals/s the
    term alone would allow, and the achieved rate; bound = the smallest."""
    ex2, rcp, fma = peaks["ex2_per_s"], peaks["rcp_per_s"], peaks["fma_per_s"]
    tc = variant != "fp32"
    achieved = evals / (t_ms / 1e3)
    terms = {}
    if kind == "forward":
        terms["mufu"] = {"per_s": ex2, "note": "1 ex2 per evaluated pair"}
        ops = FP32_OPS["forward_tc" if tc else "forward_fp32"]
        bytes_ = issued / 256 * REC_BYTES + pixels * 20 if tc else evals / 256 * REC_BYTES + pixels * 20
        flops_pair = 2 * K_OF.get(variant, 0) * issued / max(evals, 1)
    else:
        terms["mufu"] = {"per_s": 1.0 / (1.0 / ex2 + 1.0 / rcp), "note": "1 ex2 + 1 rcp per evaluated pair"}
        ops = FP32_OPS["backward"]
        bytes_ = issued / 256 * (REC_BYTES + 2 * 36) + pixels * 32
        flops_pair = (256 + 2 * K_OF.get(variant, 0)) * issued / max(evals, 1)
    terms["fp32_issue"] = {"per_s": fma / ops, "note": f"{ops} FP32 operations per evaluated pair at the measured "
                                                       f"FMA rate {fma / 1e12:.1f} T/s"}
    hbm = read_peaks().get("hbm_gbs")
    if hbm:
        terms["hbm"] = {"per_s": hbm * 1e9 / (bytes_ / max(evals, 1)),
                        "note": f"{bytes_ / max(evals, 1):.3f} algorithmic bytes per evaluated pair at "
                                f"{hbm:.0f} GB/s (measured copy)", "bytes_per_launch": int(bytes_)}
    tf = read_peaks().get("bf16_tflops")
    if tc and tf and flops_pair > 0:
        tpeak = tf * 1e12 * (2.0 if variant == "fp8_split" else 1.0)
        terms["tensor"] = {"per_s": tpeak / flops_pair,
                           "note": f"{flops_pair:.1f} MMA FLOPs per evaluated pair at {tpeak / 1e12:.0f} TFLOP/s "
                                   f"(measured bf16{' x 2, e4m3 nominal ratio' if variant == 'fp8_split' else ''})",
                           "achieved_tflops": round(flops_pair * achieved / 1e12, 2),
                           "frac": round(flops_pair * achieved / tpeak, 4)}
    bound = min(terms, key=lambda k: terms[k]["per_s"])
    for v in terms.values():
        v["per_s"] = round(v["per_s"] / 1e9, 1)  # G evals/s
    return {"kernel": kind, "variant": variant, "launch_ms": round(t_ms, 5), "achieved_g_evals_per_s":
            round(achieved / 1e9, 2), "terms_g_evals_per_s": terms, "bound": bound,
            "frac_of_bound": round(achieved / 1e9 / terms[bound]["per_s"], 4),
            "issued_over_evaluated": round(issued / max(evals, 1), 3)}


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def variant_sweep(gs, torch, st, dL, flush, stream, reps, variants):
    """Blend-only ms/frame of each variant on the step's lists (forward, and
    backward from that variant's own forward), TC against FP32 CUDA-core."""
    out = {}
    for name in variants:
        o = gs.make_opts(name, tile_order=st.order)
        fwd = st.forward(opts=o)
        bwd_ok = name != "fp32_persistent"  # forward only
        if name != "fp32":  # each variant's pipeline shapes by the library's own measurement
            gs.gs_blend_autotune([st.W], [st.H], st.n, st.ranges, st.ids, st.proj["mean2d"], st.proj["conic"],
                                 st.dev["opacities"], st.proj["rgb"], o, fwd["image"], fwd["T_final"],
                                 fwd["n_contrib"], reps=3)
            fwd = st.forward(opts=o)
            if bwd_ok:
                scratch = {k: torch.empty(st.n * c, device="cuda") for k, c in (("mean2d", 2), ("conic", 3),
                                                                                  ("opacity", 1), ("rgb", 3))}
                gs.gs_blend_autotune_backward([st.W], [st.H], st.n, st.ranges, st.ids, st.proj["mean2d"],
                                              st.proj["conic"], st.dev["opacities"], st.proj["rgb"], o,
                                              fwd["T_final"], fwd["n_contrib"], dL, scratch, reps=3)
                del scratch
        for _ in range(2):
            fwd = st.forward(opts=o)
            if bwd_ok:
                st.backward(dL, fwd=fwd, opts=o)
        f_ms = _timed(torch, flush, stream, lambda: st.forward(opts=o), reps)
        fwd = st.forward(opts=o)
        b_ms = _timed(torch, flush, stream, lambda: st.backward(dL, fwd=fwd, opts=o), reps) if bwd_ok else None
        torch.cuda.synchronize()
        ev = int(fwd["n_contrib"].sum().item())
        out[name] = {"forward_ms": round(f_ms, 5), "backward_ms": round(b_ms, 5) if b_ms else None,
                     "shape": None if name == "fp32" else {"chunk": o.chunk, "stages": o.stages,
                                                           "bwd_stages": o.bwd_stages},
                     "forward_evals_per_s": ev / (f_ms / 1e3),
                     "backward_evals_per_s": ev / (b_ms / 1e3) if b_ms else None}
    assert gs.gs_sync_status() == gs.GS_OK
    if "fp32" in out:
        for name, v in out.items():
            v["forward_speedup_vs_fp32"] = round(out["fp32"]["forward_ms"] / v["forward_ms"], 3)
            if v["backward_ms"]:
                v["backward_speedup_vs_fp32"] = round(out["fp32"]["backward_ms"] / v["backward_ms"], 3)
    if "fp32_persistent" in out:  # the tensor cores against CUDA cores inside the same kernel
        for name, v in out.items():
            v["forward_speedup_vs_persistent_fp32"] = round(out["fp32_persistent"]["forward_ms"] / v["forward_ms"], 3)
    return out


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
    if args.resolution:
        rw, rh = (int(x) for x in args.resolution.lower().split("x"))
        cam = scenes.look_at_camera((0.0, 0.0, -3.0), (0.0, 0.0, 0.0), rw, rh)
    W, H = cam.width, cam.height
    dev = gs.scene_to_device(sc)
    tight = not args.full_lists
    dL = torch.from_numpy(scenes.upstream_grad(0, [cam])[0]).cuda()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    # with N ranks each blends the tiles t = rank (mod N) of the longest-first order
    st = Step(gs, torch, dev, cam, args.variant, tight, shard=(ws_n, rank))
    n = sc.n

    for _ in range(max(args.warmup, 3)):
        st.eager(dL)
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    tuned = None
    if args.variant != "fp32":  # the pipeline shapes by the library's own measurement
        gs.gs_blend_autotune([W], [H], n, st.ranges, st.ids, st.proj["mean2d"], st.proj["conic"], dev["opacities"],
                             st.proj["rgb"], st.opts, st.fwd["image"], st.fwd["T_final"], st.fwd["n_contrib"])
        scratch = {k: torch.empty(n * c, device="cuda") for k, c in (("mean2d", 2), ("conic", 3), ("opacity", 1),
                                                                       ("rgb", 3))}
        gs.gs_blend_autotune_backward([W], [H], n, st.ranges, st.ids, st.proj["mean2d"], st.proj["conic"],
                                      dev["opacities"], st.proj["rgb"], st.opts, st.fwd["T_final"],
                                      st.fwd["n_contrib"], dL, scratch)
        del scratch
        tuned = {"chunk": st.opts.chunk, "stages": st.opts.stages, "bwd_stages": st.opts.bwd_stages}
    g_eager = st.eager(dL)
    torch.cuda.synchronize()
    evals_fwd = int(st.fwd["n_contrib"].sum().item())
    if dist:  # each rank holds its tiles' pixels: the frame's evaluations are the sum
        t = torch.tensor([evals_fwd], device="cuda", dtype=torch.int64)
        dist.all_reduce(t)
        evals_fwd = int(t.item())
    n_inst = int(st.count_dev.item())

    # ---- the step as four CUDA graphs (projection; bin/sort and tile order;
    # forward; backward + gradient all-reduce), replayed with CUDA events
    # between them on the launching stream
    graphs = []
    mode = {"capture_error_mode": "thread_local"} if dist else {}

    def capture(fn):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, **mode):
            r = fn()
        graphs.append(g)
        return r

    launches_c = gs.gs_launch_count()
    g_proj = capture(st.project)
    capture(lambda: st.sort(g_proj))
    g_fwd = capture(lambda: st.forward(g_proj))
    g_grad = capture(lambda: st.backward(dL, proj=g_proj, fwd=g_fwd))
    launches_per_step = gs.gs_launch_count() - launches_c  # the library's kernels in the four graphs

    def replay_step(ev=None):
        if ev:
            ev[0].record(stream)
        for i, g in enumerate(graphs):
            g.replay()
            if i == 3 and dist:  # the one exchange: the per-Gaussian gradient buffer (N x 9 floats)
                dist.all_reduce(g_grad["mean2d"]._base, op=dist.ReduceOp.SUM)
            if ev:
                ev[i + 1].record(stream)

    for _ in range(3):
        replay_step()
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    assert torch.equal(g_fwd["image"], st.fwd["image"]) and torch.equal(g_fwd["n_contrib"], st.fwd["n_contrib"])

    K = args.steps
    k_ev = [_events(torch, 5) for _ in range(K)]
    with ClockSampler(local, 50) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        wall0 = time.perf_counter()
        for k in range(K):
            flush.zero_()
            replay_step(k_ev[k])
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        wall = time.perf_counter() - wall0
    clocks = clk.summary()
    assert gs.gs_sync_status() == gs.GS_OK  # also catches a capacity overflow of the bin/sort
    launches = launches_per_step * K
    stage = lambda i, j: [e[i].elapsed_time(e[j]) for e in k_ev]  # noqa: E731
    proj_ms, sort_ms, fwd_ms, bwd_ms = stage(0, 1), stage(1, 2), stage(2, 3), stage(3, 4)
    dev_ms = sum(stage(0, 4))
    if dist:
        t = torch.tensor([dev_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_ms = float(t.item())
    evals_step = 2 * evals_fwd  # forward and backward each examine sum(n_contrib) pairs
    value = evals_step * K / (dev_ms / 1e3)

    # ---- the same replays for a few seconds: clocks over a long window
    sus = None
    if args.sustained_seconds > 0:
        Ks = max(K, int(args.sustained_seconds * 1e3 / max(dev_ms / K, 1e-3)))
        s_ev = _events(torch, 2)
        with ClockSampler(local, 100) as sclk:
            if dist:
                dist.barrier()
            s_ev[0].record(stream)
            for _ in range(Ks):
                flush.zero_()
                replay_step()
            s_ev[1].record(stream)
            torch.cuda.synchronize()
        sus = {"steps": Ks, "ms_per_step": round(s_ev[0].elapsed_time(s_ev[1]) / Ks, 5), "clocks": sclk.summary(),
               "note": "the same graph replays (L2 flush included) for several seconds, clocks sampled every 100 ms"}

    # ---- the same step launched call by call (no graphs), for comparison
    Ke = min(K, 100)
    e_ev = [_events(torch, 5) for _ in range(Ke)]
    for k in range(Ke):
        flush.zero_()
        st.eager(dL, e_ev[k], stream)
        if dist:
            pass  # the eager comparison leaves the gradients per rank
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    eager_ms = statistics.mean(e[0].elapsed_time(e[4]) for e in e_ev)

    # ---- issued pairs: the chunks the tensor-core forward evaluates before a tile's exit
    issued_fwd = evals_fwd
    if args.variant != "fp32":
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        o_cnt = gs.make_opts(args.variant, chunk=st.opts.chunk, stages=st.opts.stages, tile_order=st.order,
                             issued_pairs=cnt, shard_count=ws_n, shard_index=rank)
        out_c = st.forward(opts=o_cnt)
        issued_fwd = int(cnt.item())
        assert gs.gs_sync_status() == gs.GS_OK and torch.equal(out_c["n_contrib"], g_fwd["n_contrib"])
        st.forward()
    issued_bwd = backward_issued_pairs(torch, g_fwd["n_contrib"]) if args.variant != "fp32" else evals_fwd

    # ---- the forward's splat staging: TMA gathers of packed records against per-thread loads
    producer = None
    if args.variant != "fp32" and st.rec is not None and not args.step_only:
        gs.pack_splats(st.proj, dev["opacities"], out=st.rec)
        o_tma = gs.make_opts(args.variant, chunk=st.opts.chunk, stages=st.opts.stages, tile_order=st.order,
                             shard_count=ws_n, shard_index=rank, splat_records=st.rec)
        reps = min(max(K, 10), 50)
        for _ in range(2):
            st.forward(opts=o_tma)
        t_tma = _timed(torch, flush, stream, lambda: st.forward(opts=o_tma), reps)
        t_ldg = _timed(torch, flush, stream, lambda: st.forward(), reps)
        producer = {"tma_gather4_ms": round(t_tma, 5), "per_thread_loads_ms": round(t_ldg, 5),
                    "note": "blend forward alone, median of %d, L2 flushed; the step uses per-thread loads, the "
                            "faster" % reps}

    # ---- rooflines: the library's own MUFU / FMA microbenchmark, the measured HBM and tensor peaks
    mp = gs.gs_measure_peaks()
    f_ms, b_ms = statistics.mean(fwd_ms), statistics.mean(bwd_ms)
    p_ms, s_ms = statistics.mean(proj_ms), statistics.mean(sort_ms)
    rf = blend_roofline("forward", args.variant, f_ms, evals_fwd, issued_fwd, W * H, mp)
    rb = blend_roofline("backward", args.variant, b_ms, evals_fwd, issued_bwd, W * H, mp)
    hbm = read_peaks().get("hbm_gbs")
    sort_bytes = 32 * n + 4 * n_inst + 8 * gs.num_tiles(W, H)
    stages = {"project": p_ms, "bin_sort": s_ms, "blend_forward": f_ms, "blend_backward": b_ms}
    # the largest bin/sort kernel, the coarse duplication, timed live inside its stage: the stage
    # captured again with events around that launch (gs_set_kernel_events), replayed after the
    # projection with L2 flushed first, as in the step
    e_dup = _events(torch, 2)
    gs.set_kernel_events(gs.KERNEL_DUPLICATE, *e_dup)
    try:
        g_sort_t = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g_sort_t, **mode):
            st.sort(g_proj)
    finally:
        gs.set_kernel_events(gs.KERNEL_DUPLICATE, None, None)
    dup_runs = []
    for _ in range(min(max(K, 10), 50)):
        flush.zero_()
        graphs[0].replay()
        g_sort_t.replay()
        torch.cuda.synchronize()
        dup_runs.append(e_dup[0].elapsed_time(e_dup[1]))
    assert gs.gs_sync_status() == gs.GS_OK
    dup_ms = statistics.median(dup_runs)
    # its algorithmic bytes: per Gaussian the depth rank and inputs read (perm, mean2d, radius, conic,
    # power_min: 32 bytes), per (Gaussian, supertile) pair the 8 bytes written
    n_pairs = supertile_pairs(torch, gs, st)
    dup_bytes = 32 * n + 8 * n_pairs

    # the dominant kernel, by live duration: the backward or forward blend (each its stage's one
    # kernel) or the coarse duplication; the bin/sort stage as a whole is reported beside
    cand = {"blend_backward": b_ms, "blend_forward": f_ms, "dup": dup_ms}
    dom = max(cand, key=cand.get)
    if dom == "dup":
        ach = dup_bytes / (dup_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": "k_dup_coarse (bin/sort's coarse duplication)",
                    "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(ach / hbm, 4) if hbm else None, "traffic": None, "launch_ms": round(dup_ms, 5),
                    "algorithmic_bytes": dup_bytes, "pairs": n_pairs,
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, burst) of measured",
                    "note": "bound by instruction issue and latency, not by HBM (ncu: issue 56% busy, 4 blocks "
                            "per SM); algorithmic bytes: 32 per Gaussian read, 8 per supertile pair written"}
    else:
        r = rf if dom == "blend_forward" else rb
        b = r["terms_g_evals_per_s"][r["bound"]]
        tr = KNOWN_TRAFFIC.get(r["kernel"] + "/" + args.variant)
        roofline = {"bound": "alu" if r["bound"] in ("mufu", "fp32_issue") else r["bound"],
                    "kernel": f"k_blend_tc_bwd ({args.variant})" if r is rb else f"k_blend_tc ({args.variant})",
                    "achieved": r["achieved_g_evals_per_s"], "peak": b["per_s"], "unit": "G evals/s",
                    "frac": r["frac_of_bound"],
                    "traffic": tr["bytes"] if tr and tr["config"] == args.config and not args.resolution else None,
                    "launch_ms": r["launch_ms"],
                    "terms": {k: v["per_s"] for k, v in r["terms_g_evals_per_s"].items()},
                    "peak_source": b["note"] + " (measured on this GPU); the min of the MUFU, FP32-issue, HBM "
                                   "and tensor terms"}
    roofline["kernel_ms"] = {k: round(v, 5) for k, v in cand.items()}
    achieved = sort_bytes / (s_ms / 1e3) / 1e9
    stage_roofline = {"stage": "bin/sort (gs_alpha_power_min + gs_bin_sort_views + gs_tile_order, one CUDA graph)",
                      "bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                      "frac": round(achieved / hbm, 4) if hbm else None, "algorithmic_bytes": sort_bytes,
                      "launch_ms": round(s_ms, 5),
                      "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, burst) of measured",
                      "note": "algorithmic bytes: 32 per Gaussian (inputs), 4 per instance (the sorted id), 8 per "
                              "tile (range): the least a binning moves"}
    roofline["stage_ms"] = {k: round(v, 5) for k, v in stages.items()}

    # ---- blend-only ms/frame per variant, TC vs FP32 CUDA core, and the 1920x1080 workload
    sweep, sweep_c2, sweep_c1 = None, None, None
    if not args.quick and not args.step_only:
        reps = min(max(K, 10), 30)
        sweep = variant_sweep(gs, torch, st, dL, flush, stream, reps,
                              ["fp32", "fp32_persistent", "fp16", "bf16", "fp16_split", "bf16_split", "fp8_split"])
        if args.config == 4 and ws_n == 1:
            sweep_c2 = run_config2(gs, torch, scenes, flush, stream, reps, args.variant)
            sweep_c1 = run_config1(gs, torch, scenes, flush, stream, reps)

    # ---- projection backward (§8(f) row 1) and the small-scene fused front end (row 4)
    side = not args.step_only
    pb_line = run_project_backward(gs, torch, dev, sc, cam, st, g_eager, flush, stream, min(K, 100)) if side else None
    small_line = run_small_fused(gs, torch, gs.make_opts(args.variant), flush, min(K, 100)) if side else None
    batched_line = (run_batched(gs, torch, sc, dev, args.variant, flush, min(K, 50))
                    if args.config == 3 and side else None)

    # ---- end to end through the public API with host buffers
    e2e = run_e2e(args, gs, torch, sc, cam, st.opts, st.capacity, dL, flush, evals_step, ws_n, dist, tight) \
        if side else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_n, "steps": K, "warmup": args.warmup,
        "ms_per_step": dev_ms / K, "higher_is_better": True, "scaling": "strong" if ws_n > 1 else "weak",
        "vs_baseline": None, "dtype": DTYPE_OF.get(args.variant, args.variant), "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config] + WORKLOAD_NOTE
                   + (f" (rendered at {W}x{H})" if args.resolution else ""), "blend_variant": args.variant,
                   "step": "project + bin_sort + tile_order + blend_forward + blend_backward",
                   "lists": "opacity-aware (gs_alpha_power_min + conics): a splat keeps a tile only if alpha can "
                            "reach 1/255 there; same image as the full 3-sigma rectangles" if tight
                            else "full 3-sigma rectangles",
                   "tile_order": "longest list first (gs_tile_order)",
                   "blend_shape": tuned or "per-tile FP32 blocks",
                   "evals_per_step": evals_step, "instances": n_inst, "pixels": W * H,
                   "l2": "flushed before every timed step (256 MB write)",
                   "parallelism": f"tile shards x{ws_n} + NCCL all-reduce of the gradients" if ws_n > 1 else "1 GPU",
                   "bin_sort": "no host synchronisation (fixed capacity, count on the device)",
                   "launch": "each stage (project; bin_sort + tile_order; forward; backward) replayed as a CUDA "
                             "graph, CUDA events between the stages"},
        "breakdown_ms": {k: round(v, 5) for k, v in stages.items()},
        "wall_ms_per_step": wall * 1e3 / K,
        "eager_ms_per_step": round(eager_ms, 5),
        "launches_per_step": launches_per_step,
        **({"e2e": e2e} if e2e else {}), "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
        "bin_sort_roofline": stage_roofline,
        "blend_rooflines": {"forward": rf, "backward": rb},
        **({"forward_splat_staging": producer} if producer else {}),
        **({"sustained": sus} if sus else {}),
        **({"blend_by_variant": sweep} if sweep else {}),
        **({"workload_1920x1080": sweep_c2} if sweep_c2 else {}),
        **({"workload_1280x720": sweep_c1} if sweep_c1 else {}),
        "forward_pairs": {"evaluated_per_frame": evals_fwd, "issued_per_frame": issued_fwd,
                          "backward_issued_per_frame": issued_bwd,
                          "note": "evaluated = sum of n_contrib (the metric's pairs); issued = 256 x the splats of "
                                  "every chunk the tensor-core kernels evaluate before a tile's exit"},
        **({"projection_backward": pb_line} if pb_line else {}),
        **({"small_scene_fused": small_line} if small_line else {}),
        **({"batched_views": batched_line} if batched_line else {}),
    }
    if ws_n > 1:
        line["all_reduce_bytes_per_step"] = int(g_grad["mean2d"]._base.numel() * 4)
    if rank == 0 and ws_n == 1 and not args.no_cpu_baseline and side:  # the oracle on the host cores: N = 1 only
        line["cpu_baseline"] = cpu_baseline(cam, st.proj, st.bs, sc, dL, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_project_backward(gs, torch, dev, sc, cam, st, g, flush, stream, K):
    """dL/d(means, scales, quats, sh) from the blend's splat gradients alone
    (k_project_bwd: HBM-bound, one thread per Gaussian)."""
    args_ = (dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam, st.proj["radius"],
             g["mean2d"], g["conic"], g["rgb"])
    for _ in range(3):
        gs.project_backward(*args_)
    ms = _timed(torch, flush, stream, lambda: gs.project_backward(*args_), K)
    assert gs.gs_sync_status() == gs.GS_OK
    n = sc.n
    Ksh = (sc.sh_degree + 1) ** 2
    # per Gaussian: means, scales, quats, sh, radius, dmean2d, dconic, drgb read; dmeans, dscales, dquats, dsh written
    b = n * (4 * (3 + 3 + 4 + 3 * Ksh + 1 + 2 + 3 + 3) + 4 * (3 + 3 + 4 + 3 * Ksh))
    hbm = read_hbm_peak()
    return {"ms": round(ms, 5), "bytes_per_gaussian": b // n, "achieved_gb_per_s": round(b / ms / 1e6, 1),
            "peak_gb_per_s": hbm, "frac": round(b / ms / 1e6 / hbm, 4) if hbm else None,
            "note": f"gs_project_backward alone (k_project_bwd), L2 flushed before each launch, median of {K}; "
                    "peak = measured copy bandwidth"}


def run_config2(gs, torch, scenes, flush, stream, reps, variant):
    """The 1920x1080, 1M clustered-Gaussian workload (full 3-sigma lists, as
    its description states): the step time and every variant's blend."""
    sc = scenes.make_config(2, seed=0)
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    dL = torch.from_numpy(scenes.upstream_grad(0, [cam])[0]).cuda()
    st = Step(gs, torch, dev, cam, variant, tight=False)
    for _ in range(3):
        st.eager(dL)
    ev = [_events(torch, 5) for _ in range(reps)]
    for e in ev:
        flush.zero_()
        st.eager(dL, e, stream)
    torch.cuda.synchronize()
    assert gs.gs_sync_status() == gs.GS_OK
    out = {"workload": WORKLOADS[2] + WORKLOAD_NOTE, "lists": "full 3-sigma rectangles", "instances": st.count0,
           "step_ms_eager": round(statistics.median(e[0].elapsed_time(e[4]) for e in ev), 5),
           "evals_per_frame": int(st.fwd["n_contrib"].sum().item())}
    out["blend_by_variant"] = variant_sweep(gs, torch, st, dL, flush, stream, reps,
                                            ["fp32", "fp32_persistent", "bf16", "fp16_split", "bf16_split",
                                             "fp8_split"])
    del st
    return out


def run_config1(gs, torch, scenes, flush, stream, reps):
    """The 1280x720, 200k-Gaussian workload (full 3-sigma lists): every
    variant's blend, FP32 Alg. 1 and the persistent kernel on CUDA cores
    beside the tensor-core variants."""
    sc = scenes.make_config(1, seed=0)
    cam = sc.cameras[0]
    dev = gs.scene_to_device(sc)
    dL = torch.from_numpy(scenes.upstream_grad(0, [cam])[0]).cuda()
    st = Step(gs, torch, dev, cam, "bf16_split", tight=False)
    for _ in range(3):
        st.eager(dL)
    torch.cuda.synchronize()
    out = {"workload": WORKLOADS[1] + WORKLOAD_NOTE, "lists": "full 3-sigma rectangles", "instances": st.count0,
           "evals_per_frame": int(st.fwd["n_contrib"].sum().item())}
    out["blend_by_variant"] = variant_sweep(gs, torch, st, dL, flush, stream, reps,
                                            ["fp32", "fp32_persistent", "fp16_split", "bf16_split"])
    del st
    return out


def run_small_fused(gs, torch, opts, flush, K):
    """The 256x256, 10k-Gaussian scene (the launch-bound case), three ways,
    each step (project, lists, blend forward and backward) captured once as a
    CUDA graph and replayed K times, L2 flushed before every replay, CUDA
    events around the replay: gs_project + gs_bin_sort_views (graph mode, 9
    launches) then the blends; gs_project_bin_small (one cooperative launch)
    then the blends; gs_render_small (projection, lists and the forward blend
    in one cooperative launch) then the backward."""
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
    fwd_opts = gs.make_opts("fp16_split", bg=tuple(opts.bg))

    def unfused():
        proj = gs.project(*args3)
        gs.gs_bin_sort_views(1, n, proj["mean2d"], proj["radius"], proj["depth"], [W], [H], capacity, ws, None, ids,
                             ranges, count_dev=count)
        bs = dict(tile_ranges=ranges, ids=ids)
        fwd = gs.blend_forward(W, H, bs, proj, dev["opacities"], opts)
        gs.blend_backward(W, H, bs, proj, dev["opacities"], opts, fwd, dL)

    def fused_lists():
        proj, bs = gs.project_bin_small(*args3, max_per_tile=1024)
        fwd = gs.blend_forward(W, H, bs, proj, dev["opacities"], opts)
        gs.blend_backward(W, H, bs, proj, dev["opacities"], opts, fwd, dL)

    def fused_render():
        proj, bs, fwd = gs.render_small(*args3[:5], dev["opacities"], cam, bg=tuple(opts.bg), max_per_tile=1024)
        gs.blend_backward(W, H, bs, proj, dev["opacities"], fwd_opts, fwd, dL)

    out = {}
    for name, step in (("unfused", unfused), ("fused", fused_lists), ("fused_render", fused_render)):
        for _ in range(3):
            step()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            step()
        for _ in range(3):
            g.replay()
        ev = []
        for _ in range(K):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g.replay()
            b.record(stream)
            ev.append((a, b))
        torch.cuda.synchronize()
        assert gs.gs_sync_status() == gs.GS_OK
        out[name] = {"ms_per_step": round(statistics.median(a.elapsed_time(b) for a, b in ev), 5)}
    out["workload"] = "256x256, 10k Gaussians, SH degree 0, seed 0; step = project + bin + blend fwd + bwd"
    out["note"] = ("unfused: 9 bin/sort launches; fused: gs_project_bin_small then the persistent blends; "
                   "fused_render: gs_render_small (project, lists and the fp16-split tensor-core forward in one "
                   "launch) then the backward; each step one CUDA graph replay")
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


def run_e2e(args, gs, torch, sc, cam, opts, capacity, dL, flush, evals_step, ws, dist, tight=False):
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
    br = gs.BatchRenderer(dict(devb, sh_degree=sc.sh_degree), [cam], opts, capacity, opacity_aware=tight)
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
    pr = gs.PipelinedRenderer(host, sc.sh_degree, [cam], opts, capacity, dL, graphs=True, opacity_aware=tight)
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
    threads = os.cpu_count() or 1
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam)
    d32 = pr["depth"].astype(np.float32)
    tight = not args.full_lists
    # the opacity-aware lists of the GPU arm, from the oracle's FP64 definition
    kw = {}
    if tight:
        o = sc.opacities.astype(np.float64)
        keep = sc.opacities >= np.float32(1.0) / np.float32(255.0)
        kw = dict(conic=pr["conic"].astype(np.float32),
                  power_min=np.where(keep, -np.log(255 * o) - 2e-3, np.inf).astype(np.float32))
    # a large image gets lists for a random tile sample only (the timed steps visit no other tile)
    ntiles = cam.num_tiles
    mask = None
    if ntiles > 8192:
        mask = np.zeros(ntiles, bool)
        mask[np.random.default_rng(0).choice(ntiles, size=4096, replace=False)] = True
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], d32, W, H, tile_mask=mask, **kw)
    dL = scenes.upstream_grad(0, [cam])[0].astype(np.float64)
    op = sc.opacities.astype(np.float64)
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
    pool = f"{len(busy)} non-empty tiles" + (f" of a random sample of 4096 of {ntiles}" if mask is not None else "")
    sample = (f"{k} of {pool} per step (rotating), FP64 blend forward + gradient over "
              + ("opacity-aware lists (FP64 definition)" if tight else "full 3-sigma lists"))
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
