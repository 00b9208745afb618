"""Autotuner for the rasteriser's launch parameters.

Times the candidates on the caller's own scene and camera and keeps the
fastest: the sort's radix digit width (8..11 bits, which sets the number of
onesweep passes).  Results are cached as JSON under
$QUADBOX_CACHE_DIR (default ~/.cache/quadbox/tune.json), keyed by GPU name,
Gaussian count, image size and binning mode.
"""
from __future__ import annotations

import json
import os

import torch

from . import rasterizer as R

DIGIT_CANDIDATES = (8, 9, 10, 11)


def _cache_path():
    d = os.environ.get("QUADBOX_CACHE_DIR", os.path.join(os.path.expanduser("~"), ".cache", "quadbox"))
    os.makedirs(d, exist_ok=True)
    return os.path.join(d, "tune.json")


def _load():
    try:
        return json.load(open(_cache_path()))
    except Exception:
        return {}


def _save(db):
    tmp = _cache_path() + ".tmp"
    with open(tmp, "w") as f:
        json.dump(db, f, indent=1, sort_keys=True)
    os.replace(tmp, _cache_path())


def _time(fn, reps):
    s = torch.cuda.current_stream()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_frame(scene, cam, mode="quadbox", reps=5, use_cache=True):
    """Pick the sort digit width for this scene and camera."""
    n = int(scene["means"].shape[0])
    W, H = int(cam["width"]), int(cam["height"])
    key = f"{torch.cuda.get_device_name()}|n={n}|{W}x{H}|{mode}"
    db = _load() if use_cache else {}
    if key in db:
        return dict(db[key], cached=True)
    _, fr = R.forward(scene, cam, mode)
    scene_s, cam_s = R.scene_struct(scene), R.camera_struct(cam)
    timings = {}
    for d in DIGIT_CANDIDATES:
        fr.set_tuning(digit_bits=d)

        def run():
            fr.preprocess(scene_s, cam_s, mode)
            fr.bin_emit(sync=False)
            fr.sort()
        run()
        timings[d] = _time(run, reps)
    best = min(timings, key=timings.get)
    res = {"digit_bits": int(best), "ms": {str(k): round(v, 4) for k, v in timings.items()}}
    if use_cache:
        db[key] = res
        _save(db)
    return dict(res, cached=False)
