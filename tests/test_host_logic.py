"""Host-side logic that needs no GPU: the Python binding's argument
marshalling (binning-mode names, camera and tuning structs, tensor checks,
the capacity guess) and bench.py's roofline bookkeeping (algorithmic work per
kernel, the dominant kernel, fractions of the measured peaks, traffic scaled
from the ncu captures)."""
import json
import os

import numpy as np
import pytest
import torch

import bench
from paper_2605_04844_gb300 import _native as N
from paper_2605_04844_gb300 import rasterizer as R
from paper_2605_04844_gb300 import synth


def test_mode_names_and_the_unclamped_flag():
    for name, v in N.MODE_NAMES.items():
        assert R.mode_id(name) == v
        assert R.mode_id(name.upper()) == v
        assert R.mode_id(name + "+noclamp") == v | N.QB_BIN_NO_CLAMP
    assert R.mode_id(N.MODE_NAMES["adr"]) == N.MODE_NAMES["adr"]
    with pytest.raises(KeyError):
        R.mode_id("hexbox")


def test_camera_struct_copies_every_field():
    cam = synth.pinhole(64, 48)
    c = R.camera_struct(cam)
    np.testing.assert_allclose(np.array(c.viewmat[:]), np.asarray(cam["viewmat"], dtype=np.float64).reshape(16),
                               rtol=1e-6)
    assert (c.width, c.height) == (64, 48)
    assert c.fx == pytest.approx(cam["fx"], rel=1e-6) and c.cy == pytest.approx(cam["cy"], rel=1e-6)
    assert c.tan_fovx == pytest.approx(cam["tan_fovx"], rel=1e-6)
    assert c.znear == pytest.approx(0.2)


def test_tune_struct_defaults_and_overrides():
    t = R.tune_struct()
    assert (t.tiles_per_fetch, t.render_batch, t.sort_digit_bits, t.blocks_per_sm) == (2, 128, 8, 0)
    t = R.tune_struct({"sort_digit_bits": 10, "render_batch": 64})
    assert (t.sort_digit_bits, t.render_batch, t.tiles_per_fetch) == (10, 64, 2)


def test_scene_struct_rejects_host_tensors_and_bad_shapes():
    n = 5
    scene = {"means": torch.zeros(n, 3), "scales": torch.zeros(n, 3), "quats": torch.zeros(n, 4),
             "opacities": torch.zeros(n), "sh": torch.zeros(n, 1, 3), "sh_degree": 0}
    with pytest.raises(ValueError, match="CUDA"):
        R.scene_struct(scene)  # host memory: the library takes device pointers only
    with pytest.raises(ValueError):
        R._check_tensor(torch.zeros(n, 3, dtype=torch.float64), "means", (3,), n)


def test_capacity_guess_bounds():
    assert R.estimate_capacity(0, 16, 16) == 1 << 16
    assert R.estimate_capacity(1_000_000, 1920, 1080) == 8_000_000
    assert R.estimate_capacity(10**9, 1920, 1080) == 2**30
    assert R.estimate_capacity(10, 16000, 16000) == 4 * 1000 * 1000


def test_kernel_work_figures():
    P, n, E, Ep = 34_613_290, 1_000_000, 123_456_789, 23_456_789
    w = bench.kernel_work(P, n, (E, Ep))
    assert w["tile_sort_pass"] == ("hbm", 16 * P)
    assert w["tile_sort_pass_values"] == ("hbm", 12 * P)
    wp = bench.kernel_work(P, n, (E, Ep), packed=True)  # one packed word between the passes
    assert wp["tile_sort_pass"] == ("hbm", 12 * P)
    assert wp["tile_sort_pass_values"] == ("hbm", 8 * P)
    # 1080p: 8160 tiles, 13-bit ids sorted as 7 + 6 bits, indices below 2^26
    assert bench.tile_sort_packed(1_000_000, 1920, 1080, 8)
    assert not bench.tile_sort_packed(2 ** 26 + 1, 1920, 1080, 8)
    assert not bench.tile_sort_packed(1_000, 64, 64, 8)  # 16 tiles: one pass
    assert not bench.tile_sort_packed(1_000, 16384, 16384, 8)  # 20-bit ids: three passes
    assert w["emit_warp_kernel"] == ("hbm", 8 * P + 28 * n)
    assert w["render_kernel"] == ("alu", 9 * E + 12 * Ep)  # power test on every entry, alpha and blend on passes
    assert w["preprocess_kernel"] == ("hbm", n * bench.PREPROCESS_BYTES)
    # every captured kernel's traffic refers to a kernel with algorithmic work
    assert set(bench.TRAFFIC_PER_UNIT) <= set(w)


def test_roofline_picks_the_dominant_kernel_and_uses_the_measured_peaks():
    path = os.path.join(bench.ROOT, "MEASURED_PEAKS.json")
    # the driver writes the measured peaks; without them bench.py falls back to 6800 GB/s
    peaks = json.load(open(path)) if os.path.exists(path) else {"hbm_gbs": 6800.0}
    P, n, E = 20_000_000, 600_000, 400_000_000
    kernels = {
        "render_kernel": {"ms_per_launch": 0.30, "ms_per_step": 0.30},
        "tile_sort_pass": {"ms_per_launch": 0.10, "ms_per_step": 0.10},
        "preprocess_kernel": {"ms_per_launch": 0.05, "ms_per_step": 0.05},
        "not_a_kernel_of_ours": {"ms_per_launch": 9.0, "ms_per_step": 9.0},
    }
    clk = {"sm_mhz": 2000.0}
    Ep = 100_000_000
    r = bench.roofline({}, kernels, P, n, 1920, 1080, 8, (E, Ep), clk, "depth_first", sms=148)
    assert r["kernel"] == "render_kernel" and r["bound"] == "alu"
    alu_peak = 148 * 128 * 2 * 2000.0 * 1e6 / 1e12  # the SM count passed in, not a constant
    assert r["peak"] == pytest.approx(alu_peak, rel=1e-3)
    assert r["achieved"] == pytest.approx((9 * E + 12 * Ep) / 0.30e-3 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    unit, per = bench.TRAFFIC_PER_UNIT["render_kernel"]
    assert unit == "eval" and r["traffic"] == int(per * E)
    sp = r["kernels"]["tile_sort_pass"]
    assert sp["bound"] == "hbm" and sp["peak"] == peaks["hbm_gbs"]
    assert sp["achieved"] == pytest.approx(12 * P / 0.10e-3 / 1e9, rel=1e-3)  # 600k at 1080p: packed
    assert sp["traffic"] == int(bench.TRAFFIC_PER_UNIT["tile_sort_pass"][1] * P)
    assert "not_a_kernel_of_ours" not in r["kernels"]


def test_autotune_cache_round_trip_and_corrupt_file(tmp_path, monkeypatch):
    from paper_2605_04844_gb300 import autotune
    monkeypatch.setenv("QUADBOX_CACHE_DIR", str(tmp_path / "cache"))
    assert autotune._load() == {}  # no file yet
    db = {"GB300|n=10|64x48|quadbox": {"digit_bits": 9, "ms": {"8": 1.0, "9": 0.9}}}
    autotune._save(db)
    assert autotune._load() == db
    (tmp_path / "cache" / "tune.json").write_text("{ not json")
    assert autotune._load() == {}  # a damaged cache is ignored, not fatal


def _full_result_like_a_default_run():
    """A result dict shaped like bench.py's full default run, with the long
    sections (30 zoom views x 6 modes, every kernel row) filled in."""
    kern = {f"kernel_{i}": {"ms_per_launch": 0.1234, "launches_per_step": 1.0, "ms_per_step": 0.1234}
            for i in range(12)}
    views = [{"view": k, "distance": 40.0, **{m: {"pairs": 123456789, "fwd_ms": 7.123, "fps": 140.4}
                                             for m in ("quadbox", "aabb3s", "adr", "quadbox_naive", "dualbox",
                                                       "quadbox+noclamp")}} for k in range(30)]
    stage = {s: 0.1234 for s in ("preprocess", "emit", "sort", "render", "backward")}
    return {
        "metric": bench.METRIC, "value": 948.123, "unit": "FPS", "n_gpus": 1, "steps": 20, "warmup": 5,
        "ms_per_step": 1.0551, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded 1M-Gaussian clustered scene; stands in for Mip-NeRF 360 / DB / T&T)",
        "config": {"workload": "1M Gaussians, 1920x1080, SH degree 3, 16x16 tiles, QuadBox binning (clamped to "
                               "3-sigma) vs 3-sigma AABB on the same kernels", "n_gaussians": 1000000,
                   "width": 1920, "height": 1080, "sh_degree": 3,
                   "l2": "L2 flushed (258 MB write) between timed steps; scene inputs 236 MB > L2",
                   "sort_digit_bits": 8, "sort_mode": "depth_first", "parallelism": "replicas x1"},
        "quadbox": {"fwd_fps": 948.1, "fwd_ms": 1.0551, "fwd_bwd_ms": 1.7512, "pairs_per_frame": 34613290,
                    "stage_ms": stage},
        "aabb3s": {"fwd_fps": 432.1, "fwd_ms": 2.3123, "fwd_bwd_ms": 3.3312, "pairs_per_frame": 101012345,
                   "stage_ms": stage},
        "speedup_vs_aabb": {"fwd": 2.191, "fwd_bwd": 1.902, "pair_ratio": 2.918},
        "quadbox_other_sort_modes": {"full_key": {"fwd_ms": 2.52, "stage_ms": stage}},
        "e2e": {"value": 431.123, "unit": "FPS", "h2d_bytes_per_step": 236000000, "d2h_bytes_per_step": 24883200},
        "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 123},
        "roofline": {"kernel": "render_kernel", "bound": "alu", "achieved": 26.512, "peak": 80.486,
                     "unit": "TFLOP/s", "frac": 0.3294, "traffic": 15000000,
                     "peak_source": "148 SMs x 128 FP32 lanes x 2 x 2070 MHz (median sampled SM clock)"},
        "roofline_kernels": kern, "kernels_fwd": kern, "gpu_launches": 12345,
        "c3_zoom": {"workload": "x" * 200, "views": views},
        "batch64": {"workload": "x" * 200, "graph_fwd_ms": 52.3, "graph_fwd_bwd_ms": 85.8, "speedup_fwd": 1.07,
                    "speedup_fwd_bwd": 1.18, "tune": {"tiles_per_fetch": 2}},
        "cpu_baseline": {"value": 0.25114, "unit": "FPS", "cores": 16, "kind": "oracle",
                         "sample": "one 1M-Gaussian 1920x1080 QuadBox frame: FP64 projection, binning and sort in "
                                   "full, compositing of every 16th tile row (129600 pixels) scaled to the frame",
                         "seconds_per_frame": 3.98},
    }


def test_bench_headline_is_the_last_line_and_stays_compact():
    """The run's last output line is the headline and stays under 2 KB (a
    reader that keeps only the tail of the output must be able to parse it);
    every detail section is on an earlier line of its own."""
    res = _full_result_like_a_default_run()
    lines = bench.output_lines(res)
    last = lines[-1]
    assert len(last.encode()) <= 2048
    h = json.loads(last)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "dtype",
              "e2e", "clocks", "roofline", "cpu_baseline", "gpu_launches"):
        assert k in h, k
    assert h["config"]["workload"].startswith("1M Gaussians, 1920x1080")
    assert h["quadbox"]["pairs_per_frame"] == 34613290 and h["aabb3s"]["fwd_bwd_ms"] == 3.3312
    assert h["roofline"]["frac"] == 0.3294 and h["cpu_baseline"]["cores"] == 16
    sections = [json.loads(x)["section"] for x in lines[:-1]]
    assert "c3_zoom" in sections and "kernels_fwd" in sections and "batch64" in sections
    # a result with still longer strings is trimmed, never over the bound
    res["cpu_baseline"]["sample"] = "y" * 3000
    assert len(bench.output_lines(res)[-1].encode()) <= 2048
