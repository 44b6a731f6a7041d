"""The reference arm of bench.py (the FP64 oracle timed on the host cores)
keeps the JSON-line contract, on the CPU: one line with the metric, unit and
workload of the GPU arm, a cpu_baseline describing the run, an e2e object
with no host copies; under a multi-rank launch only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env, *args):
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK")}
    env.update(extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line(oracle_lib):
    p = _run({}, "--config", "0", "--steps", "2", "--warmup", "1")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"].startswith("256x256, 10k Gaussians")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert isinstance(cb["cpu_model"], str) and cb["cpu_model"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    p = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--config", "0", "--steps", "1", "--warmup", "0")
    assert p.returncode == 0, p.stderr[-2000:]
    assert not [l for l in p.stdout.splitlines() if l.startswith("{")]


def test_gpu_arm_cpu_baseline_leg(oracle_lib):
    """bench.cpu_baseline (the GPU arm's oracle leg) on CPU tensors of the
    256x256 workload: a bounded run that reports its sample, threads and CPU model."""
    import numpy as np
    import torch

    import bench
    import oracle
    from paper_2604_02120_gb300 import scenes

    sc = scenes.make_config(0)
    cam = sc.cameras[0]
    pr = oracle.project(sc.means, sc.scales, sc.quats, sc.sh, sc.sh_degree, cam)
    d32 = pr["depth"].astype(np.float32)
    bs = oracle.bin_sort(pr["mean2d"], pr["radius"], d32, cam.width, cam.height)
    proj = {k: torch.from_numpy(np.ascontiguousarray(pr[k], np.float32)) for k in ("mean2d", "conic", "rgb")}
    tb = dict(tile_ranges=torch.from_numpy(bs["tile_ranges"].view(np.int32)), ids=torch.from_numpy(bs["ids"].view(np.int32)))
    dL = torch.from_numpy(scenes.upstream_grad(0, [cam])[0])
    cb = bench.cpu_baseline(cam, proj, tb, sc, dL, 0.5)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1 and cb["cpu_model"]
    assert cb["seconds"] >= 0.5 and "non-empty tiles" in cb["sample"]
