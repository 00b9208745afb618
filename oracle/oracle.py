"""FP64 CPU oracle for the QuadBox tile rasteriser -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code with the CUDA library
and never imports the product package; inputs arrive as plain numpy arrays.

The arithmetic lives in ``qb_oracle.c`` (double precision, one Gaussian or one
pixel at a time).  This file only marshals arrays and performs the steps that
are library primitives: a stable sort of the (tile | depth) keys (Sec. 2,
"SortPairs") and the derivation of per-tile ranges from the sorted keys.

Scene dict: means [n,3], scales [n,3] (log-scales when raw), quats [n,4]
(w,x,y,z), opacities [n] (logits when raw), sh [n,K,3], sh_degree, raw.
Camera dict: viewmat [4,4] row-major world->view, fx, fy, cx, cy, tan_fovx,
tan_fovy, campos [3], width, height, znear.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_DIR = os.path.join(_HERE, "lib")
LIB_PATH = os.path.join(LIB_DIR, "liboracle.so")
SRC_PATH = os.path.join(_HERE, "qb_oracle.c")

TILE = 16
NF = 32
# projection record fields (mirrors the enum in qb_oracle.c)
F_VALID, F_X, F_Y, F_DEPTH = 0, 1, 2, 3
F_S11, F_S12, F_S22 = 4, 5, 6
F_A, F_B, F_C = 7, 8, 9
F_O, F_R, F_G, F_BL, F_CLAMP = 10, 11, 12, 13, 14
F_GAMMA, F_GAMMAB = 15, 16
F_XMAX, F_YMAX, F_XMIN, F_YMIN = 17, 18, 19, 20
F_F, F_R3, F_ORIENT = 21, 22, 23

AABB3S, QUADBOX, ADR, QUADBOX_NAIVE, DUALBOX = 0, 1, 2, 3, 4

_lib = None


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile qb_oracle.c into lib/liboracle.so with gcc (OpenMP when available)."""
    os.makedirs(LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB_PATH)
            and os.path.getmtime(LIB_PATH) >= os.path.getmtime(SRC_PATH)):
        return LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", "-o", LIB_PATH + ".tmp", SRC_PATH, "-lm"]
    for extra in (["-fopenmp"], []):
        r = subprocess.run(base[:1] + extra + base[1:], capture_output=True, text=True)
        if r.returncode == 0:
            os.replace(LIB_PATH + ".tmp", LIB_PATH)
            if verbose:
                print("built", LIB_PATH, "with", extra)
            return LIB_PATH
    raise RuntimeError("oracle build failed:\n" + r.stderr)


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(LIB_PATH)
    return _lib


def set_threads(n: int) -> None:
    """Threads of the C oracle's OpenMP loops (for timing; results do not depend on it)."""
    lib().orc_set_threads(ctypes.c_int(int(n)))


def max_threads() -> int:
    return int(lib().orc_max_threads())


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def camera_array(cam) -> np.ndarray:
    """26 doubles: viewmat[16], fx, fy, cx, cy, tan_fovx, tan_fovy, campos[3], znear."""
    v = np.zeros(26, dtype=np.float64)
    v[:16] = np.asarray(cam["viewmat"], dtype=np.float64).reshape(16)
    v[16:22] = [cam["fx"], cam["fy"], cam["cx"], cam["cy"], cam["tan_fovx"], cam["tan_fovy"]]
    v[22:25] = np.asarray(cam["campos"], dtype=np.float64)
    v[25] = cam.get("znear", 0.2)
    return v


def sh_basis(deg: int, dirs: np.ndarray) -> np.ndarray:
    """Real SH basis values [m, (deg+1)^2] for unit directions [m, 3]."""
    dirs = _f64(dirs).reshape(-1, 3)
    K = (deg + 1) ** 2
    out = np.zeros((dirs.shape[0], 16), dtype=np.float64)
    f = lib().orc_sh_basis
    for i in range(dirs.shape[0]):
        f(ctypes.c_int(deg), _p(dirs[i]), _p(out[i]))
    return out[:, :K]


def project(scene, cam) -> np.ndarray:
    """Projection records [n, NF] (Sec. 2 EWA projection + Sec. 3.1 box terms)."""
    n = int(scene["means"].shape[0])
    deg = int(scene["sh_degree"])
    out = np.zeros((n, NF), dtype=np.float64)
    if n == 0:
        return out
    means, scales, quats = _f64(scene["means"]), _f64(scene["scales"]), _f64(scene["quats"])
    opac, sh = _f64(scene["opacities"]), _f64(scene["sh"])
    c = camera_array(cam)
    lib().orc_project(ctypes.c_int(n), _p(means), _p(scales), _p(quats), _p(opac), _p(sh),
                      ctypes.c_int(deg), ctypes.c_int(int(scene.get("raw", 1))), _p(c), _p(out))
    return out


def rects_f32(xy, ext, r3, orient, valid, mode, clamp3s, W, H) -> np.ndarray:
    """Tile rectangles [n,4,4] (x0,y0,x1,y1) from float32 box parameters,
    replaying the float32 rounding of the tile mapping exactly."""
    xy = np.ascontiguousarray(xy, dtype=np.float32)
    ext = np.ascontiguousarray(ext, dtype=np.float32)
    r3 = np.ascontiguousarray(r3, dtype=np.float32)
    orient, valid = _i32(orient), _i32(valid)
    n = int(valid.shape[0])
    out = np.zeros((n, 4, 4), dtype=np.int32)
    if n:
        lib().orc_rects_f32(ctypes.c_int(n), _p(xy), _p(ext), _p(r3), _p(orient), _p(valid),
                            ctypes.c_int(mode), ctypes.c_int(int(clamp3s)), ctypes.c_int(W),
                            ctypes.c_int(H), _p(out))
    return out


def rects_f64(proj, mode, clamp3s, W, H) -> np.ndarray:
    proj = _f64(proj)
    n = int(proj.shape[0])
    out = np.zeros((n, 4, 4), dtype=np.int32)
    if n:
        lib().orc_rects_f64(ctypes.c_int(n), _p(proj), ctypes.c_int(mode), ctypes.c_int(int(clamp3s)),
                            ctypes.c_int(W), ctypes.c_int(H), _p(out))
    return out


def tile_lists(rects, use_qpass: bool, tiles_x: int):
    """Per-Gaussian tile lists: counts [n], offsets [n] (exclusive prefix),
    tiles [P], gids [P], in Gaussian-index order."""
    rects = _i32(rects)
    n = int(rects.shape[0])
    counts = np.zeros(n, dtype=np.int64)
    if n:
        lib().orc_count(ctypes.c_int(n), _p(rects), ctypes.c_int(int(use_qpass)), _p(counts))
    offsets = np.zeros(n, dtype=np.int64)
    if n:
        offsets[1:] = np.cumsum(counts)[:-1]
    P = int(counts.sum())
    tiles = np.zeros(max(P, 1), dtype=np.uint32)
    gids = np.zeros(max(P, 1), dtype=np.uint32)
    if n:
        lib().orc_emit(ctypes.c_int(n), _p(rects), ctypes.c_int(int(use_qpass)), ctypes.c_int(tiles_x),
                       _p(offsets), _p(tiles), _p(gids))
    return counts, offsets, tiles[:P], gids[:P]


def depth_bits(depth_f32) -> np.ndarray:
    return np.ascontiguousarray(depth_f32, dtype=np.float32).view(np.uint32).astype(np.uint64)


def keys_from_lists(tiles, gids, depth_f32) -> np.ndarray:
    """key = (tile << 31) | (float32 depth bits & 0x7fffffff)."""
    d = depth_bits(depth_f32)[gids.astype(np.int64)] & np.uint64(0x7FFFFFFF)
    return (tiles.astype(np.uint64) << np.uint64(31)) | d


def sort_pairs(keys, vals):
    """Stable sort of the pairs by key (SortPairs, Sec. 2)."""
    order = np.argsort(keys, kind="stable")
    return keys[order], vals[order]


def ranges_from_sorted_tiles(sorted_tiles, ntiles: int) -> np.ndarray:
    """ranges[t] = [first, last+1) of tile t in the sorted list; [0,0) if absent."""
    r = np.zeros((ntiles, 2), dtype=np.int64)
    if sorted_tiles.size == 0:
        return r
    t = sorted_tiles.astype(np.int64)
    starts = np.searchsorted(t, np.arange(ntiles), side="left")
    ends = np.searchsorted(t, np.arange(ntiles), side="right")
    present = ends > starts
    r[present, 0] = starts[present]
    r[present, 1] = ends[present]
    return r


def render(W, H, ranges, vals, proj, bg=(0.0, 0.0, 0.0)):
    """Per-pixel compositing (Eq. 2) over tile lists.  Returns
    (img [3,H,W], T_final [H,W], n_contrib [H,W], ambiguous [H,W])."""
    ranges = np.ascontiguousarray(ranges, dtype=np.int64)
    vals = _i32(vals) if len(vals) else np.zeros(1, dtype=np.int32)
    proj = _f64(proj)
    bgv = _f64(bg)
    img = np.zeros((3, H, W), dtype=np.float64)
    T = np.zeros((H, W), dtype=np.float64)
    nc = np.zeros((H, W), dtype=np.int32)
    amb = np.zeros((H, W), dtype=np.int32)
    lib().orc_render(ctypes.c_int(W), ctypes.c_int(H), _p(ranges), _p(vals), _p(proj), _p(bgv),
                     _p(img), _p(T), _p(nc), _p(amb))
    return img, T, nc, amb


def render_pixels(W, H, pxs, pys, ranges, vals, proj, bg=(0.0, 0.0, 0.0)):
    pxs, pys = _i32(pxs), _i32(pys)
    ranges = np.ascontiguousarray(ranges, dtype=np.int64)
    vals = _i32(vals) if len(vals) else np.zeros(1, dtype=np.int32)
    proj = _f64(proj)
    bgv = _f64(bg)
    m = int(pxs.shape[0])
    rgb = np.zeros((m, 3), dtype=np.float64)
    T = np.zeros(m, dtype=np.float64)
    nc = np.zeros(m, dtype=np.int32)
    amb = np.zeros(m, dtype=np.int32)
    lib().orc_render_pixels(ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(m), _p(pxs), _p(pys),
                            _p(ranges), _p(vals), _p(proj), _p(bgv), _p(rgb), _p(T), _p(nc), _p(amb))
    return rgb, T, nc, amb


def render_brute(W, H, rects, proj, bg=(0.0, 0.0, 0.0)):
    rects = _i32(rects)
    proj = _f64(proj)
    n = int(proj.shape[0])
    bgv = _f64(bg)
    img = np.zeros((3, H, W), dtype=np.float64)
    T = np.zeros((H, W), dtype=np.float64)
    nc = np.zeros((H, W), dtype=np.int32)
    amb = np.zeros((H, W), dtype=np.int32)
    lib().orc_render_brute(ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(n), _p(rects), _p(proj),
                           _p(bgv), _p(img), _p(T), _p(nc), _p(amb))
    return img, T, nc, amb


def render_backward(W, H, ranges, vals, proj, dL_dimg, bg=(0.0, 0.0, 0.0)):
    """Gradients w.r.t. (mu2D [n,2], conic (a,b,c) [n,3], o [n], colour [n,3])."""
    ranges = np.ascontiguousarray(ranges, dtype=np.int64)
    vals = _i32(vals) if len(vals) else np.zeros(1, dtype=np.int32)
    proj = _f64(proj)
    n = int(proj.shape[0])
    g_xy = np.zeros((n, 2)); g_con = np.zeros((n, 3)); g_o = np.zeros(n); g_rgb = np.zeros((n, 3))
    lib().orc_render_backward(ctypes.c_int(W), ctypes.c_int(H), _p(ranges), _p(vals), _p(proj),
                              _p(_f64(bg)), _p(_f64(dL_dimg)), _p(g_xy), _p(g_con), _p(g_o), _p(g_rgb))
    return g_xy, g_con, g_o, g_rgb


def render_backward_pixels(W, H, pxs, pys, dL, ranges, vals, proj, bg=(0.0, 0.0, 0.0), magnitudes=False):
    """render_backward restricted to the listed pixels (dL [m,3] their loss
    gradients): equal to render_backward with dL_dimg zero elsewhere.  With
    magnitudes, also returns the per-entry sums of the terms' absolute
    values (same shapes), the scale of a float32 evaluation's rounding error."""
    pxs, pys = _i32(pxs), _i32(pys)
    ranges = np.ascontiguousarray(ranges, dtype=np.int64)
    vals = _i32(vals) if len(vals) else np.zeros(1, dtype=np.int32)
    proj = _f64(proj)
    n = int(proj.shape[0])
    g_xy = np.zeros((n, 2)); g_con = np.zeros((n, 3)); g_o = np.zeros(n); g_rgb = np.zeros((n, 3))
    a = [np.zeros((n, 2)), np.zeros((n, 3)), np.zeros(n), np.zeros((n, 3))] if magnitudes else None
    ap = [_p(x) for x in a] if magnitudes else [None] * 4
    lib().orc_render_backward_pixels(ctypes.c_int(W), ctypes.c_int(H), ctypes.c_int(int(pxs.shape[0])), _p(pxs),
                                     _p(pys), _p(ranges), _p(vals), _p(proj), _p(_f64(bg)),
                                     _p(_f64(np.asarray(dL).reshape(-1, 3))), _p(g_xy), _p(g_con), _p(g_o),
                                     _p(g_rgb), *ap)
    if magnitudes:
        return (g_xy, g_con, g_o, g_rgb), tuple(a)
    return g_xy, g_con, g_o, g_rgb


def project_backward(scene, cam, g_xy, g_con, g_o, g_rgb):
    """Chain the screen-space gradients to the raw parameters."""
    n = int(scene["means"].shape[0])
    deg = int(scene["sh_degree"])
    K = (deg + 1) ** 2
    gm = np.zeros((n, 3)); gs = np.zeros((n, 3)); gq = np.zeros((n, 4)); go = np.zeros(n)
    gsh = np.zeros((n, K, 3))
    lib().orc_project_backward(
        ctypes.c_int(n), _p(_f64(scene["means"])), _p(_f64(scene["scales"])), _p(_f64(scene["quats"])),
        _p(_f64(scene["opacities"])), _p(_f64(scene["sh"])), ctypes.c_int(deg),
        ctypes.c_int(int(scene.get("raw", 1))), _p(camera_array(cam)), _p(_f64(g_xy)), _p(_f64(g_con)),
        _p(_f64(g_o)), _p(_f64(g_rgb)), _p(gm), _p(gs), _p(gq), _p(go), _p(gsh))
    return {"means": gm, "scales": gs, "quats": gq, "opacities": go, "sh": gsh}


# --------------------------------------------------------------------------
# Convenience pipelines
# --------------------------------------------------------------------------

def grid(W, H):
    tx = (W + TILE - 1) // TILE
    ty = (H + TILE - 1) // TILE
    return tx, ty


def own_lists(proj, W, H, mode=QUADBOX, clamp3s=True):
    """The oracle's own FP64 binning: rects, per-tile lists sorted by
    (tile, depth, index) and ranges."""
    tx, ty = grid(W, H)
    rects = rects_f64(proj, mode, clamp3s, W, H)
    use_qpass = mode != QUADBOX_NAIVE
    counts, offsets, tiles, gids = tile_lists(rects, use_qpass, tx)
    depth = proj[:, F_DEPTH][gids.astype(np.int64)] if len(gids) else np.zeros(0)
    order = np.lexsort((gids, depth, tiles)) if len(gids) else np.zeros(0, dtype=np.int64)
    st, sg = tiles[order], gids[order]
    ranges = ranges_from_sorted_tiles(st, tx * ty)
    return {"rects": rects, "counts": counts, "tiles": st, "vals": sg.astype(np.int32), "ranges": ranges}


def image(scene, cam, mode=QUADBOX, clamp3s=True, bg=(0.0, 0.0, 0.0)):
    """Full FP64 forward: projection, binning, sort, ranges, compositing."""
    W, H = int(cam["width"]), int(cam["height"])
    proj = project(scene, cam)
    L = own_lists(proj, W, H, mode, clamp3s)
    img, T, nc, amb = render(W, H, L["ranges"], L["vals"], proj, bg)
    return {"proj": proj, "img": img, "T": T, "n_contrib": nc, "amb": amb, **L}


def gradients(scene, cam, dL_dimg, mode=QUADBOX, clamp3s=True, bg=(0.0, 0.0, 0.0)):
    """Analytic FP64 gradients of sum(dL_dimg * image) w.r.t. the raw parameters."""
    W, H = int(cam["width"]), int(cam["height"])
    proj = project(scene, cam)
    L = own_lists(proj, W, H, mode, clamp3s)
    g_xy, g_con, g_o, g_rgb = render_backward(W, H, L["ranges"], L["vals"], proj, dL_dimg, bg)
    g = project_backward(scene, cam, g_xy, g_con, g_o, g_rgb)
    g["screen"] = {"xy": g_xy, "conic": g_con, "o": g_o, "rgb": g_rgb}
    return g
