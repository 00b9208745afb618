"""Autotuner for the rasteriser's launch parameters.

Times the candidates on the caller's own scene and camera and keeps the
fastest.  For a frame: the tile sort's radix digit width (8..11 bits, which
sets the number of onesweep passes), then the render's per-tile batch depth
(Gaussians staged in shared memory per step).  For a batch of cameras: the
digit width, batch depth, tiles a persistent render block takes per fetch
from the global queue and persistent blocks per SM, by coordinate descent.
Results are cached as JSON under
$QUADBOX_CACHE_DIR (default ~/.cache/quadbox/tune.json), keyed by GPU name,
Gaussian count, image size and binning mode.
"""
from __future__ import annotations

import json
import os

import torch

from . import rasterizer as R

DIGIT_CANDIDATES = (8, 9, 10, 11)
RENDER_BATCH_CANDIDATES = (64, 128, 256)


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
    """Pick the sort digit width (timing preprocess, emit and sort), then the
    render's batch depth (timing the render), for this scene and camera."""
    n = int(scene["means"].shape[0])
    W, H = int(cam["width"]), int(cam["height"])
    key = f"{torch.cuda.get_device_name()}|frame2|n={n}|{W}x{H}|{mode}"
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
    fr.set_tuning(digit_bits=best)
    fr.preprocess(scene_s, cam_s, mode)
    fr.bin_emit(sync=False)
    fr.sort()
    img = torch.empty((3, H, W), dtype=torch.float32, device=fr.ws.device)
    rtimes = {}
    for rb in RENDER_BATCH_CANDIDATES:
        fr.set_tuning(render_batch=rb)
        fr.render(None, img)
        rtimes[rb] = _time(lambda: fr.render(None, img), reps)
    fr.check()
    best_rb = min(rtimes, key=rtimes.get)
    res = {"digit_bits": int(best), "render_batch": int(best_rb),
           "ms": {str(k): round(v, 4) for k, v in timings.items()},
           "render_ms": {str(k): round(v, 4) for k, v in rtimes.items()}}
    if use_cache:
        db[key] = res
        _save(db)
    return dict(res, cached=False)


BATCH_SPACE = {
    "sort_digit_bits": (8, 10, 11),
    "render_batch": (64, 128, 256),
    "tiles_per_fetch": (1, 2, 4),
    "blocks_per_sm": (0, 2, 4),
}


def tune_batch(batch, scene, cams, mode="quadbox", reps=2, use_cache=True):
    """Coordinate descent over the batched path's launch parameters (sort
    digit width, staging batch depth, tiles per queue fetch, persistent
    blocks per SM), timing qb_render_batch on the caller's scene and cameras."""
    key = (f"{torch.cuda.get_device_name()}|batch|n={batch.n}|cams={batch.n_cams}|group={batch.group}|"
           f"{'-'.join(f'{w}x{h}' for w, h in zip(batch.widths, batch.heights))[:200]}|{mode}")
    db = _load() if use_cache else {}
    if key in db:
        return dict(db[key], cached=True)
    scene_s, cams_arr = R.scene_struct(scene), R.camera_array(cams)
    best = {"sort_digit_bits": 8, "render_batch": 128, "tiles_per_fetch": 2, "blocks_per_sm": 0}
    timings = {}
    for name, values in BATCH_SPACE.items():
        res = {}
        for v in values:
            cand = dict(best, **{name: v})
            batch.render(scene_s, cams_arr, mode, cand)  # warm
            res[v] = _time(lambda: batch.render(scene_s, cams_arr, mode, cand), reps)
        best[name] = min(res, key=res.get)
        timings[name] = {str(k): round(t, 3) for k, t in res.items()}
    batch.check()
    out = {"tune": best, "ms": timings}
    if use_cache:
        db[key] = out
        _save(db)
    return dict(out, cached=False)
