"""Helpers shared by the GPU tests: move seeded numpy scenes to the device,
run the library's stages and read back its arrays."""
import numpy as np

from oracle import oracle as O


def to_device(scene):
    import torch
    out = {}
    for k, v in scene.items():
        if isinstance(v, np.ndarray):
            out[k] = torch.from_numpy(np.ascontiguousarray(v, dtype=np.float32)).cuda()
        else:
            out[k] = v
    return out


def f64(scene):
    return {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in scene.items()}


def run_forward(scene, cam, mode="quadbox", bg=None, digit_bits=8, capacity=None, sort_mode="depth_first"):
    """sort_mode: a rasterizer sort mode, or "depth_first_fused" (depth-first
    with the emit fused with the first tile-sort pass)."""
    from paper_2605_04844_gb300 import rasterizer as R
    fused = sort_mode == "depth_first_fused"
    img, fr = R.forward(to_device(scene), cam, mode, bg=bg, digit_bits=digit_bits, capacity=capacity,
                        sort_mode="depth_first" if fused else sort_mode, emit_fused=fused)
    import torch
    torch.cuda.synchronize()
    fr.check()
    A = {k: v.cpu().numpy() for k, v in fr.arrays().items()}
    A["full_keys"] = gpu_full_keys(A, sort_mode)
    return img.cpu().numpy(), fr, A


def gpu_full_keys(A, sort_mode):
    """The sorted (tile << 31) | depth-bits keys: read directly in the full-key
    mode, rebuilt from the tile keys and each value's depth in depth-first mode."""
    if sort_mode == "full_key":
        return A["keys"].view(np.uint64)
    d = A["rgbd"][:, 3].astype(np.float32).view(np.uint32).astype(np.uint64) & np.uint64(0x7FFFFFFF)
    tiles = A["tile_keys"].view(np.uint32).astype(np.uint64)
    return (tiles << np.uint64(31)) | d[A["vals"].view(np.uint32).astype(np.int64)]


def oracle_keys_from_gpu_boxes(A, mode, clamp, W, H):
    """The oracle's integer traversal fed the GPU's float32 box parameters:
    rects, per-Gaussian counts, stably sorted keys and values, ranges."""
    meta = A["meta"]
    valid = (meta & 1).astype(np.int32)
    orient = ((meta >> 1) & 1).astype(np.int32)
    rects = O.rects_f32(A["xy"], A["box"], A["r3"], orient, valid, mode, clamp, W, H)
    tx, ty = O.grid(W, H)
    counts, offsets, tiles, gids = O.tile_lists(rects, mode != O.QUADBOX_NAIVE, tx)
    keys = O.keys_from_lists(tiles, gids, A["rgbd"][:, 3])
    sk, sv = O.sort_pairs(keys, gids)
    ranges = O.ranges_from_sorted_tiles((sk >> np.uint64(31)).astype(np.int64), tx * ty)
    return {"rects": rects, "counts": counts, "keys": sk, "vals": sv, "ranges": ranges}


def image_parity(img_gpu, ref, max_abs=2e-3, mean_abs=1e-5, max_flip_frac=1e-4):
    """North-star image bar: per channel max-abs and mean-abs, with pixels
    whose discrete decisions sit inside the float32 band of a threshold
    (flagged by the oracle) allowed to differ, counted and bounded."""
    diff = np.abs(img_gpu.astype(np.float64) - ref["img"])
    bad = diff.max(axis=0) > max_abs
    amb = ref["amb"] != 0
    unexplained = bad & ~amb
    flips = bad & amb
    HW = bad.size
    keep = ~flips
    stats = {"max_abs": float(diff[:, keep].max()) if keep.any() else 0.0,
             "mean_abs": [float(diff[c][keep].mean()) for c in range(3)],
             "flips": int(flips.sum()), "unexplained": int(unexplained.sum()), "pixels": HW}
    ok = (stats["unexplained"] == 0 and stats["max_abs"] <= max_abs and max(stats["mean_abs"]) <= mean_abs
          and stats["flips"] <= max(1, int(max_flip_frac * HW)))
    return ok, stats
