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


def perturbed_sensitivity(scene, cam, trials=4, rel=2.0 ** -22, seed=0):
    """Per-entry sensitivity of the oracle's projection records to ulp-sized
    relative perturbations of the float32 inputs (means, scales, quaternions,
    opacities): the largest change over a few random perturbations.  It
    measures how much rounding at the inputs' own precision can move each
    output, i.e. the part of a float32 evaluation's error that no backward-
    stable float32 algorithm avoids."""
    base = f64(scene)
    ref = O.project(base, cam)
    rng = np.random.default_rng(seed)
    sens = np.zeros_like(ref)
    for _ in range(trials):
        s2 = dict(base)
        for k in ("means", "scales", "quats", "opacities"):
            v = base[k]
            s2[k] = v * (1.0 + rel * rng.choice((-1.0, 1.0), size=v.shape))
        r2 = O.project(s2, cam)
        both = (r2[:, O.F_VALID] != 0) & (ref[:, O.F_VALID] != 0)
        d = np.where(both[:, None], np.abs(r2 - ref), 0.0)
        sens = np.maximum(sens, d)
    return ref, sens


def assert_projection_parity(A, scene, cam, max_sens_frac=1e-3):
    """The preprocess's per-Gaussian records against the oracle, entry by
    entry.  Visibility must agree except where the deciding quantity lies
    within float32 rounding of its threshold (view depth vs the near plane,
    opacity vs 1/255).  Conic and extents: relative error <= 1e-5 per entry
    (b against sqrt(a c), its bound by positive definiteness), mu^2D within
    1e-6 of |mu| + |c|, depth 1e-6, opacity 1e-6, colour 2e-5 absolute;
    where an entry's sensitivity to ulp-sized input perturbations exceeds
    that bar (an ill-conditioned projection), the error may reach 4x the
    sensitivity instead, and at most max_sens_frac of the entries may use it.
    Returns the statistics."""
    ref, sens = perturbed_sensitivity(scene, cam)
    vis_g = (A["meta"] & 1) != 0
    vis_o = ref[:, O.F_VALID] != 0
    diff = np.nonzero(vis_g != vis_o)[0]
    if len(diff):
        s64 = f64(scene)
        V = np.asarray(cam["viewmat"], np.float64).reshape(4, 4)
        tz = s64["means"][diff] @ V[2, :3] + V[2, 3]
        raw = int(s64.get("raw", 1))
        o = 1.0 / (1.0 + np.exp(-s64["opacities"][diff])) if raw else s64["opacities"][diff]
        near = np.abs(tz / cam.get("znear", 0.2) - 1.0) < 1e-6
        faint = np.abs(o * 255.0 - 1.0) < 1e-6
        assert np.all(near | faint), f"visibility differs without a threshold tie: {diff[~(near | faint)][:5]}"
    m = vis_g & vis_o
    r, sv = ref[m], sens[m]
    cx, cy = cam["cx"], cam["cy"]
    a, b, c = r[:, O.F_A], r[:, O.F_B], r[:, O.F_C]
    checks = [
        ("mu_x", A["xy"][m, 0], r[:, O.F_X], 1e-6 * (np.abs(r[:, O.F_X]) + abs(cx)), sv[:, O.F_X]),
        ("mu_y", A["xy"][m, 1], r[:, O.F_Y], 1e-6 * (np.abs(r[:, O.F_Y]) + abs(cy)), sv[:, O.F_Y]),
        ("depth", A["rgbd"][m, 3], r[:, O.F_DEPTH], 1e-6 * np.abs(r[:, O.F_DEPTH]), sv[:, O.F_DEPTH]),
        ("conic_a", A["conic_o"][m, 0], a, 1e-5 * a, sv[:, O.F_A]),
        ("conic_b", A["conic_o"][m, 1], b, 1e-5 * np.sqrt(a * c), sv[:, O.F_B]),
        ("conic_c", A["conic_o"][m, 2], c, 1e-5 * c, sv[:, O.F_C]),
        ("opacity", A["conic_o"][m, 3], r[:, O.F_O], 1e-6 * r[:, O.F_O], sv[:, O.F_O]),
        ("x_max", A["box"][m, 0], r[:, O.F_XMAX], 1e-5 * r[:, O.F_XMAX], sv[:, O.F_XMAX]),
        ("y_max", A["box"][m, 1], r[:, O.F_YMAX], 1e-5 * r[:, O.F_YMAX], sv[:, O.F_YMAX]),
        ("f_x_max", A["box"][m, 2], r[:, O.F_XMIN], 1e-5 * r[:, O.F_XMIN], sv[:, O.F_XMIN]),
        ("f_y_max", A["box"][m, 3], r[:, O.F_YMIN], 1e-5 * r[:, O.F_YMIN], sv[:, O.F_YMIN]),
    ]
    stats = {"visible": int(m.sum()), "visibility_ties": int(len(diff))}
    for ch, f in enumerate((O.F_R, O.F_G, O.F_BL)):
        e = np.abs(A["rgbd"][m, ch].astype(np.float64) - r[:, f])
        assert np.all(e <= 2e-5 + 4 * sv[:, f]), ("colour", ch, float(e.max()))
    for name, got, want, tol, s in checks:
        e = np.abs(got.astype(np.float64) - want)
        strict = e <= tol
        loose = e <= 4.0 * s
        assert np.all(strict | loose), (name, float((e / tol).max()), int((~(strict | loose)).sum()))
        used = int((~strict).sum())
        assert used <= max_sens_frac * len(e), (name, used)
        stats[name] = {"max_err_over_tol": float((e / tol).max()), "over_tol_within_sensitivity": used}
    return stats
