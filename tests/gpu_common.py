"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
(binding in paper_2604_02120_gb300.gs) and the FP64 oracle on the same seeded
inputs."""
import os

import numpy as np
import torch

import oracle
from paper_2604_02120_gb300 import gs, scenes

CORES = os.cpu_count() or 4
# Rounding model of each blend variant, for the oracle's ambiguity flags and
# colour error bounds (oracle.blend's margins):
#  - alpha: relative error of alpha (absolute error of the exponent) that does
#    not grow with the size of Eq. 3's terms: exp2 and constants; for the split
#    tensor-core variants about twice the largest measured exponent error
#    (4.7e-6 at 1280x720; the tile-power tests check it);
#  - sum: exponent error per unit of the magnitude sum of Eq. 3's terms, the
#    float32 evaluation of a sum (it dominates for nearly singular conics far
#    from the splat's centre: needle-shaped splats of the clustered and heavy-
#    tailed scenes), with offsets enlarged by `slack` px where the exponent is
#    taken relative to a half-tile's reference pixel;
#  - t: relative error of the transmittance product after a few hundred steps.
U32 = 2.0 ** -24  # float32 unit roundoff
SPLIT_EXP_ERR = 1e-5
FP8_EXP_ERR = 1e-3  # the FP8-e4m3 split trial (measured max 7.4e-4; the stated bound is 2e-3)
FP32_ALPHA_ERR = 2e-6
T_PRODUCT_ERR = 1e-5
MARGINS = {
    "fp32": dict(alpha_margin=FP32_ALPHA_ERR, t_margin=T_PRODUCT_ERR, sum_margin=4 * U32, sum_slack=0.0),
    "split": dict(alpha_margin=SPLIT_EXP_ERR, t_margin=T_PRODUCT_ERR, sum_margin=2 * U32, sum_slack=8.0),
    "fp8_split": dict(alpha_margin=FP8_EXP_ERR, t_margin=T_PRODUCT_ERR, sum_margin=2 * U32, sum_slack=8.0),
}


def margins(variant):
    """The rounding model of a variant: the FP32 CUDA-core blend, or the Eq. 6
    contraction with FP32 accumulation (split tensor-core operands, or FP32
    FMAs in the persistent kernel), or the FP8 trial."""
    return MARGINS.get(variant, MARGINS["split"])


# Largest share of pixels with a decision within those margins of its threshold.
# Measured with the oracle's own lists: 1280x720 0.025% FP32, 0.093% split;
# 1920x1080 (1M clustered, many needle splats) 0.15% and 0.26%.
# 3840x2160 (3M heavy-tailed: Student-t scales make many splats needles whose
# float32 exponent is ill-conditioned over much of the image): 3.5% and 2.1%
# on the sampled tiles, where the colour error still stays within its bound.
MAX_AMB_FP32 = 5e-4
MAX_AMB_SPLIT = 1e-3
LARGE_MAX_AMB = {"1920x1080_1M": {"fp32": 3e-3, "split": 5e-3},
                 "3840x2160_3M": {"fp32": 6e-2, "split": 4e-2}}
# Plain (unsplit) operands carry the operand type's rounding into the exponent
# (up to 0.1 for fp16 and 0.8 for bf16 on far splats): per-pixel bounds, about
# twice the largest measured.
PLAIN_MAX_ERR = {"fp16": 0.02, "bf16": 0.1}
_REPORT = {}


def report(key, value):
    """Record a measured number; written as JSON to $GS_TEST_REPORT at exit."""
    _REPORT[key] = value
    path = os.environ.get("GS_TEST_REPORT")
    if path:
        import json
        with open(path, "w") as f:
            json.dump(_REPORT, f, indent=1, sort_keys=True)


def gpu_pipeline(scene, cam_index=0, capacity=1 << 20):
    dev = gs.scene_to_device(scene)
    cam = scene.cameras[cam_index]
    proj = gs.project(dev["means"], dev["scales"], dev["quats"], dev["sh"], dev["sh_degree"], cam)
    sorter = gs.BinSorter("cuda", capacity)
    bs = sorter.run(proj["mean2d"], proj["radius"], proj["depth"], cam.width, cam.height)
    torch.cuda.synchronize()
    return dev, cam, proj, bs


def to_np(d):
    return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in d.items()}


def oracle_blend_on_gpu_params(cam, proj_np, bs_np, opac, bg=(0.0, 0.0, 0.0), variant=None, tile_subset=None):
    """Oracle blend over the GPU's sorted lists and FP32 splat parameters (cast
    to double), with the rounding model of `variant` (None: no margins)."""
    m = margins(variant) if variant else {}
    return oracle.blend(cam.width, cam.height, bs_np["tile_ranges"].view(np.uint32),
                        bs_np["ids"].view(np.uint32), proj_np["mean2d"].astype(np.float64),
                        proj_np["conic"].astype(np.float64), np.asarray(opac, np.float64),
                        proj_np["rgb"].astype(np.float64), bg=bg, n_threads=CORES, tile_subset=tile_subset, **m)


def blend_gpu(cam, proj, bs, opac, variant="fp32", bg=(0.0, 0.0, 0.0), chunk=0, stages=0, ref_origin=0):
    opts = gs.make_opts(variant, chunk=chunk, stages=stages, ref_origin=ref_origin, bg=bg)
    out = gs.blend_forward(cam.width, cam.height, bs, proj, opac, opts)
    st = gs.gs_sync_status()
    assert st == gs.GS_OK, f"device status {st}"
    return to_np(out)


def pixel_mask_tiles(cam, tiles):
    """Boolean H x W mask of the pixels of the given tiles."""
    m = np.zeros((cam.height, cam.width), bool)
    tx = cam.tiles_x
    for t in tiles:
        x0, y0 = 16 * (t % tx), 16 * (t // tx)
        m[y0:y0 + 16, x0:x0 + 16] = True
    return m


def check_tight_lists(got, ref, full, max_amb_frac=1e-3):
    """GPU opacity-aware lists against the oracle's FP64 definition.

    got, ref, full: dicts with tile_ranges (2 per tile, [start, end)), ids and
    optionally keys; `ref` from oracle.bin_sort with conic and power_min (its
    ``ambiguous`` rows are the pairs whose decision lies within rounding of
    the threshold), `full` the full-rectangle lists (GPU or oracle: they are
    bit-exact).  Asserts that
      * every tile's GPU list is a sub-sequence of its full list (same order),
        and the ranges tile the id array in tile order;
      * the GPU keeps exactly the pairs the definition keeps, except pairs
        reported ambiguous;
      * ambiguous pairs are at most max_amb_frac of the kept pairs;
      * keys, where given, are those of the full list at the same pairs.
    Returns (number of ambiguous pairs, number of pairs decided otherwise)."""
    def codes(d):
        r = np.asarray(d["tile_ranges"]).view(np.uint32).astype(np.int64)
        lens = r[1::2] - r[0::2]
        tiles = np.repeat(np.arange(lens.size, dtype=np.int64), np.maximum(lens, 0))
        n = int(lens.sum())
        ids = np.asarray(d["ids"]).view(np.uint32)[:n].astype(np.int64)
        starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
        assert (r[0::2][lens > 0] == starts[lens > 0]).all(), "ranges do not tile the id array in tile order"
        return (tiles << 32) | ids

    g, rf, fl = codes(got), codes(ref), codes(full)
    amb = np.asarray(ref["ambiguous"], np.int64).reshape(-1, 3)
    amb_codes = (amb[:, 0] << 32) | amb[:, 1]
    diff = np.setxor1d(g, rf)
    assert np.isin(diff, amb_codes).all(), \
        f"{int((~np.isin(diff, amb_codes)).sum())} pairs decided otherwise than the FP64 definition and not ambiguous"
    assert amb.shape[0] <= max_amb_frac * max(rf.size, 1), f"{amb.shape[0]} ambiguous pairs of {rf.size}"
    order = np.argsort(fl, kind="stable")
    pos = order[np.clip(np.searchsorted(fl[order], g), 0, max(fl.size - 1, 0))]
    assert fl.size > 0 or g.size == 0
    if g.size:
        assert (fl[pos] == g).all(), "a kept pair is not on the splat's rectangle"
        assert (np.diff(pos) > 0).all(), "opacity-aware lists are not sub-sequences of the full lists"
    if got.get("keys") is not None and full.get("keys") is not None and g.size:
        np.testing.assert_array_equal(np.asarray(got["keys"]).view(np.uint64)[:g.size],
                                      np.asarray(full["keys"]).view(np.uint64)[pos])
    return int(amb.shape[0]), int(diff.size)


def compare_to_oracle(out, ref, tol, nc_exact=True, max_amb=0.01):
    """Every pixel whose decisions are clear of their thresholds: colour and
    T_final within tol plus the first-order bound of the variant's own
    rounding (ref["err_bound"]), n_contrib exact; ambiguous pixels bounded."""
    amb = ref["ambiguous"]
    ok = ~amb
    assert amb.mean() <= max_amb, f"{amb.mean():.4%} ambiguous pixels"
    bound = tol + ref["err_bound"][ok]
    err = np.abs(out["image"] - ref["image"])[:, ok]
    assert (err <= bound).all(), f"max abs {err.max():.3e} beyond {tol} + bound"
    assert (np.abs(out["T_final"] - ref["T_final"])[ok] <= bound).all()
    if nc_exact:
        np.testing.assert_array_equal(out["n_contrib"][ok], ref["n_contrib"][ok])
    return err
