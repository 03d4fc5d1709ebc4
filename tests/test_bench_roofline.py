"""The bench's roofline arithmetic on made-up stage times (no GPU): achieved =
algorithmic bytes of one launch / the mean CUDA-event time of a launch, and
frac = achieved / the measured HBM peak, for the sort pass (16 B per pair per
pass, one launch per pass or one cooperative launch for all passes), the
projection (pool record + 64 B splat per drawn Gaussian) and the blend
(44 B per pair + 12 B per pixel)."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

STAGES = ("feedback", "residency", "stream", "project", "scan_emit", "sort", "ranges", "blend", "prefetch", "sort_prep")


def _stage(frames, sort_launches_per_view, sort_us, project_us, blend_us):
    ms = [0.0] * len(STAGES)
    n = [0] * len(STAGES)
    ms[STAGES.index("sort")] = frames * sort_launches_per_view * sort_us / 1e3
    n[STAGES.index("sort")] = frames * sort_launches_per_view
    ms[STAGES.index("project")] = frames * project_us / 1e3
    n[STAGES.index("project")] = frames
    ms[STAGES.index("blend")] = frames * blend_us / 1e3
    n[STAGES.index("blend")] = frames
    return ms, n


@pytest.mark.parametrize("coop", [False, True])
def test_roofline_arithmetic(coop):
    import bench
    v = types.SimpleNamespace(STAGES=STAGES)
    frames, pairs, gauss, rec16, W, H = 20, 2_900_000, 1_750_000, 128, 1920, 1080
    per_view = 1 if coop else 5   # 13 tile + 27 depth bits: five 8-bit passes
    stats = {"acc_frames": frames, "acc_views": frames, "acc_pairs": frames * pairs,
             "acc_drawn_gaussians": frames * gauss, "key_tile_bits": 13, "key_depth_bits": 27}
    peaks = {"hbm_gbs": 6000.0}
    rl = bench.roofline(v, _stage(frames, per_view, 30.0 * (5 if coop else 1), 100.0, 80.0), stats, peaks, rec16, W, H)
    k = rl["kernels"]
    # the sort: a launch moves 16 B per pair per pass it runs (five passes per cooperative launch)
    passes_per_launch = 5 if coop else 1
    sort_t = 30e-6 * passes_per_launch
    assert k["sort"]["algorithmic_bytes_per_launch"] == int(pairs * 16 * passes_per_launch)
    assert k["sort"]["us_per_launch"] == pytest.approx(sort_t * 1e6)
    assert k["sort"]["achieved"] == pytest.approx(pairs * 16 * passes_per_launch / sort_t / 1e9, abs=0.1)
    assert rl["frac"] == pytest.approx(k["sort"]["achieved"] / 6000.0, abs=1e-4)
    assert rl["achieved"] == k["sort"]["achieved"] and rl["peak"] == 6000.0 and rl["bound"] == "hbm"
    assert ("coop" in rl["kernel"]) == coop
    # the projection: record read + 64 B written per drawn Gaussian, one launch per frame
    assert k["project"]["algorithmic_bytes_per_launch"] == int(gauss * (rec16 + 64))
    assert k["project"]["achieved"] == pytest.approx(gauss * (rec16 + 64) / 100e-6 / 1e9, abs=0.1)
    # the blend: 44 B per pair read + 12 B per pixel written, one launch per view
    assert k["blend"]["algorithmic_bytes_per_launch"] == int(pairs * 44 + W * H * 12)
    assert k["blend"]["achieved"] == pytest.approx((pairs * 44 + W * H * 12) / 80e-6 / 1e9, abs=0.1)
    assert set(rl) >= {"bound", "achieved", "peak", "unit", "frac", "traffic"}
