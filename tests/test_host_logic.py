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
    P, n, E = 34_613_290, 1_000_000, 123_456_789
    w = bench.kernel_work(P, n, E)
    assert w["tile_sort_pass"] == ("hbm", 16 * P)
    assert w["tile_sort_pass_values"] == ("hbm", 12 * P)
    assert w["emit_warp_kernel"] == ("hbm", 8 * P + 28 * n)
    assert w["render_kernel"] == ("alu", E * bench.RENDER_FLOPS_PER_EVAL)
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
    r = bench.roofline({}, kernels, P, n, 1920, 1080, 8, E, clk, "depth_first")
    assert r["kernel"] == "render_kernel" and r["bound"] == "alu"
    alu_peak = 152 * 128 * 2 * 2000.0 * 1e6 / 1e12
    assert r["peak"] == pytest.approx(alu_peak, rel=1e-3)
    assert r["achieved"] == pytest.approx(E * bench.RENDER_FLOPS_PER_EVAL / 0.30e-3 / 1e12, rel=1e-3)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-3)
    unit, per = bench.TRAFFIC_PER_UNIT["render_kernel"]
    assert unit == "eval" and r["traffic"] == int(per * E)
    sp = r["kernels"]["tile_sort_pass"]
    assert sp["bound"] == "hbm" and sp["peak"] == peaks["hbm_gbs"]
    assert sp["achieved"] == pytest.approx(16 * P / 0.10e-3 / 1e9, rel=1e-3)
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
