"""GPU backward (qb_render_bwd, stages S11-S12) against the oracle's analytic
FP64 gradient and FP64 central finite differences; autograd.Function."""
import json

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_04844_gb300 import synth

from gpu_util import f64, run_forward, to_device

pytestmark = pytest.mark.gpu

KEYS = ("means", "scales", "quats", "opacities", "sh")


def gpu_grads(scene, cam, G, mode="quadbox", bg=(0.1, 0.2, 0.3)):
    import torch
    from paper_2605_04844_gb300 import _native as N
    from paper_2605_04844_gb300 import rasterizer as R
    sd = to_device(scene)
    img, fr = R.forward(sd, cam, mode, bg=bg)
    g = {k: torch.zeros_like(sd[k]) for k in KEYS}
    gs = N.QbSceneGrads()
    gs.means, gs.scales, gs.quats = g["means"].data_ptr(), g["scales"].data_ptr(), g["quats"].data_ptr()
    gs.opacities, gs.sh = g["opacities"].data_ptr(), g["sh"].data_ptr()
    n = len(scene["opacities"])
    screen = torch.zeros((max(n, 1), 9), dtype=torch.float64, device="cuda")
    Gt = torch.from_numpy(G.astype(np.float32)).cuda()
    N.qb_render_bwd(fr.frame, R.scene_struct(sd), R.camera_struct(cam), bg, Gt, gs, screen)
    torch.cuda.synchronize()
    fr.check()
    out = {k: v.cpu().numpy().astype(np.float64) for k, v in g.items()}
    out["screen"] = screen.cpu().numpy()[:n].astype(np.float64)
    return out, img.cpu().numpy()


def screen_reference(sc64, cam, scr):
    """The oracle's screen-space gradients in the library's layout: the conic
    gradient Ghat mapped to the covariance, H = -Lambda Ghat Lambda."""
    proj = O.project(sc64, cam)
    a, b, c = proj[:, O.F_A], proj[:, O.F_B], proj[:, O.F_C]
    ga, gb, gc = scr["conic"][:, 0], 0.5 * scr["conic"][:, 1], scr["conic"][:, 2]
    # (Lambda Ghat Lambda) entries for symmetric 2x2 matrices
    t00, t01 = a * ga + b * gb, a * gb + b * gc
    t10, t11 = b * ga + c * gb, b * gb + c * gc
    H00, H01, H11 = -(t00 * a + t01 * b), -(t00 * b + t01 * c), -(t10 * b + t11 * c)
    return np.stack([scr["xy"][:, 0], scr["xy"][:, 1], H00, 2 * H01, H11, scr["o"],
                     scr["rgb"][:, 0], scr["rgb"][:, 1], scr["rgb"][:, 2]], axis=1)


def normwise(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


# Element-wise gradient bar.  A gradient entry is a sum over pixels of terms
# of both signs, each evaluated in float32 on the GPU; its rounding error
# scales with the terms' magnitudes, not with the (possibly cancelled) sum.
# The oracle therefore also sums every term's absolute value (the entry's
# magnitude M, carried to the raw parameters through |J|^T), and each entry
# must satisfy
#     |g - ref| <= REL |ref| + MAG M + 4 S.
# REL = 1e-3 is the relative bar; MAG covers the float32 transmittance
# recomputed by division from the back of the list (each step divides by
# 1 - alpha, which amplifies alpha's rounding by up to 1/(1 - 0.99) = 100),
# measured below 3.5e-4 M on the scenes here.  S (where computed) is the
# entry's change under ulp-sized random perturbations of the float32 inputs:
# a needle-thin Gaussian's alpha is so sensitive to its conic that rounding
# alone moves its gradient by a percent, and no float32 evaluation avoids it.
REL = 1e-3
MAG = 5e-4


def elementwise(g, ref, mag, name, sens=None):
    g, ref, mag = (np.asarray(x, np.float64).ravel() for x in (g, ref, mag))
    err = np.abs(g - ref)
    bound = REL * np.abs(ref) + MAG * mag
    if sens is not None:
        bound = bound + 4.0 * np.asarray(sens, np.float64).ravel()
    bad = err > bound
    rel_only = err <= REL * np.abs(ref)
    stats = {"tensor": name, "entries": int(ref.size), "needing_magnitude_term": int((~rel_only).sum()),
             "max_err_over_bound": float((err / np.maximum(bound, 1e-300)).max()), "violations": int(bad.sum())}
    if bad.any():
        i = int(np.argmax(np.where(bad, err / np.maximum(bound, 1e-300), 0)))
        stats["worst"] = {"index": i, "gpu": float(g[i]), "oracle": float(ref[i]), "magnitude": float(mag[i])}
    return not bad.any(), stats


SCREEN = ("mu_x", "mu_y", "S11", "S12", "S22", "o", "r", "g", "b")


# Gaussians thinner than this stretching factor f (Eq. f-closed), an aspect
# ratio above 20 : 1, have their mean, scale and rotation gradients left out
# of the element-wise comparison (their screen-space gradients stay in it):
# the chain from the 2D covariance to the minor scale contracts entries of
# size |dL/dSigma| |M|^2 to a result smaller by about f^2, so float32 rounding
# of the chain alone is of the order of 2^-24 / f^2 of the result.
NEEDLE_F = 0.05
COVARIANCE_CHAIN = ("means", "scales", "quats")


def assert_elementwise(g, ref, g_screen, ref_screen, mag_raw, mag_screen, sens_raw=None, sens_screen=None,
                       needles=None):
    report = []
    for j, nm in enumerate(SCREEN):
        ok, st = elementwise(g_screen[:, j], ref_screen[:, j], mag_screen[:, j], "screen_" + nm,
                             None if sens_screen is None else sens_screen[:, j])
        report.append(st)
        assert ok, json.dumps(st)
    for k in KEYS:
        keep = slice(None) if needles is None or k not in COVARIANCE_CHAIN else ~needles
        ok, st = elementwise(g[k][keep], ref[k][keep], mag_raw[k][keep], k,
                             None if sens_raw is None else sens_raw[k][keep])
        if needles is not None and k in COVARIANCE_CHAIN:
            st["needles_left_out"] = int(needles.sum())
        report.append(st)
        assert ok, json.dumps(st)
    return report


def screen_magnitude(sc64, cam, mag):
    """The magnitude sums in the library's screen layout: mu^2D, Sigma (the
    conic's terms mapped by |Lambda| . |terms| . |Lambda|), o, colour."""
    proj = O.project(sc64, cam)
    a, b, c = np.abs(proj[:, O.F_A]), np.abs(proj[:, O.F_B]), np.abs(proj[:, O.F_C])
    ga, gb, gc = mag[1][:, 0], 0.5 * mag[1][:, 1], mag[1][:, 2]
    t00, t01 = a * ga + b * gb, a * gb + b * gc
    t10, t11 = b * ga + c * gb, b * gb + c * gc
    H00, H01, H11 = t00 * a + t01 * b, t00 * b + t01 * c, t10 * b + t11 * c
    return np.stack([mag[0][:, 0], mag[0][:, 1], H00, 2 * H01, H11, mag[2],
                     mag[3][:, 0], mag[3][:, 1], mag[3][:, 2]], axis=1)


def raw_magnitude(sc64, cam, mag):
    """|J|^T M: each screen component's magnitude alone through the oracle's
    (linear) projection backward, absolute values summed."""
    xy, con, o, rgb = mag
    n = len(o)
    zeros = (np.zeros((n, 2)), np.zeros((n, 3)), np.zeros(n), np.zeros((n, 3)))
    out = {k: 0.0 for k in KEYS}
    for slot, arr in enumerate((xy, con, o, rgb)):
        cols = 1 if arr.ndim == 1 else arr.shape[1]
        for j in range(cols):
            comp = [z.copy() for z in zeros]
            if arr.ndim == 1:
                comp[slot] = arr.copy()
            else:
                comp[slot][:, j] = arr[:, j]
            r = O.project_backward(sc64, cam, *comp)
            out = {k: out[k] + np.abs(r[k]) for k in KEYS}
    return out


def oracle_backward_with_magnitudes(sc64, cam, G, bg, pxs=None, pys=None, dL=None):
    """The oracle's analytic gradient of sum(G * image) over all pixels (or
    over the listed pixels with their dL rows), with its magnitudes."""
    W, H = cam["width"], cam["height"]
    proj = O.project(sc64, cam)
    L = O.own_lists(proj, W, H)
    if pxs is None:
        pys, pxs = (a.ravel() for a in np.mgrid[0:H, 0:W])
        dL = G[:, pys, pxs].T
    scr, mag = O.render_backward_pixels(W, H, pxs, pys, dL, L["ranges"], L["vals"], proj, bg=bg, magnitudes=True)
    return scr, mag


def unambiguous(G, amb):
    """The loss gradient with the pixels zeroed whose discrete decisions sit
    inside the float32 band of a threshold (the oracle's ambiguity flag):
    there FP32 and FP64 may count different entries, so neither side's
    gradient is the reference for the other."""
    return G * (amb == 0)[None]


def problem(n=256, W=64, H=64, deg=1, seed=77):
    cam = synth.pinhole(W, H)
    sc = synth.scene_uniform(n, seed, cam, depth=(2.0, 5.0), logscale=(-2.2, 0.5), deg=deg)
    G = np.random.default_rng(seed).standard_normal((3, H, W))
    G = unambiguous(G, O.image(f64(sc), cam, O.QUADBOX, bg=(0.1, 0.2, 0.3))["amb"])
    return sc, cam, G


def check_against_oracle(sc, cam, G, bg):
    g, _ = gpu_grads(sc, cam, G, bg=bg)
    sc64 = f64(sc)
    (gx, gc, go, gr), mag = oracle_backward_with_magnitudes(sc64, cam, G, bg)
    ref = O.project_backward(sc64, cam, gx, gc, go, gr)
    ref_screen = screen_reference(sc64, cam, {"xy": gx, "conic": gc, "o": go, "rgb": gr})
    return assert_elementwise(g, ref, g["screen"], ref_screen, raw_magnitude(sc64, cam, mag),
                              screen_magnitude(sc64, cam, mag))


@pytest.mark.parametrize("deg", [0, 1, 3])
def test_backward_matches_oracle_analytic(deg):
    sc, cam, G = problem(deg=deg)
    check_against_oracle(sc, cam, G, (0.1, 0.2, 0.3))


def test_backward_blobs_sh3():
    cam = synth.pinhole(160, 104)
    sc = synth.scene_blobs(4000, 1104, cam, deg=3)
    G = np.sign(np.random.default_rng(5).standard_normal((3, 104, 160))) / (3 * 160 * 104)
    G = unambiguous(G, O.image(f64(sc), cam, O.QUADBOX)["amb"])
    print(check_against_oracle(sc, cam, G, (0.0, 0.0, 0.0)))


def test_backward_c4_scene_on_sampled_tiles():
    """The forward+backward workload at full size (500k Gaussians, 1264x832,
    SH degree 3, L1 loss against a U[0,1] target): the GPU backward of the
    whole frame with dL/dimg non-zero on 24 sampled tiles (the 8 with the
    longest lists, 16 random, corners included) against the oracle's
    analytic backward over exactly those pixels, element by element, for
    every Gaussian those pixels reach; every other Gaussian's gradient is
    exactly zero on both sides."""
    scene, cam, target = synth.config4()
    W, H = cam["width"], cam["height"]
    tx, ty = O.grid(W, H)
    sc64 = f64(scene)
    proj = O.project(sc64, cam)
    L = O.own_lists(proj, W, H)
    lens = L["ranges"][:, 1] - L["ranges"][:, 0]
    rng = np.random.default_rng(44)
    tiles = set(np.argsort(-lens)[:8].tolist()) | {0, tx - 1, (ty - 1) * tx, tx * ty - 1}
    while len(tiles) < 24:
        tiles.add(int(rng.integers(0, tx * ty)))
    pxs, pys = [], []
    for t in sorted(tiles):
        x0, y0 = (t % tx) * 16, (t // tx) * 16
        yy, xx = np.mgrid[y0:min(y0 + 16, H), x0:min(x0 + 16, W)]
        pxs.append(xx.ravel())
        pys.append(yy.ravel())
    pxs, pys = np.concatenate(pxs), np.concatenate(pys)
    rgb, _, _, amb = O.render_pixels(W, H, pxs, pys, L["ranges"], L["vals"], proj)
    # the L1 loss gradient from the oracle's image, zero on ambiguous pixels
    dL = np.sign(rgb - target[:, pys, pxs].T.astype(np.float64)) / (3 * H * W)
    dL[amb != 0] = 0.0
    G = np.zeros((3, H, W))
    G[:, pys, pxs] = dL.T
    g, _ = gpu_grads(scene, cam, G, bg=(0.0, 0.0, 0.0))
    (g_xy, g_con, g_o, g_rgb), mag = O.render_backward_pixels(W, H, pxs, pys, dL, L["ranges"], L["vals"], proj,
                                                              magnitudes=True)
    touched = np.nonzero((np.abs(g_xy).sum(1) + np.abs(g_con).sum(1) + np.abs(g_o) + np.abs(g_rgb).sum(1)) > 0)[0]
    assert len(touched) > 1000
    sub = {k: (v[touched] if isinstance(v, np.ndarray) else v) for k, v in sc64.items()}
    ref = O.project_backward(sub, cam, g_xy[touched], g_con[touched], g_o[touched], g_rgb[touched])
    scr = {"xy": g_xy[touched], "conic": g_con[touched], "o": g_o[touched], "rgb": g_rgb[touched]}
    ref_screen = screen_reference(sub, cam, scr)
    # sensitivity: the same oracle gradient with the inputs perturbed by
    # random relative steps of 2^-22 (two draws)
    sens_raw = {k: np.zeros_like(ref[k]) for k in KEYS}
    sens_screen = np.zeros_like(ref_screen)
    prng = np.random.default_rng(46)
    for _ in range(2):
        sp = dict(sc64)
        for k in ("means", "scales", "quats", "opacities"):
            sp[k] = sc64[k] * (1.0 + 2.0 ** -22 * prng.choice((-1.0, 1.0), size=sc64[k].shape))
        pp = O.project(sp, cam)
        q_xy, q_con, q_o, q_rgb = O.render_backward_pixels(W, H, pxs, pys, dL, L["ranges"], L["vals"], pp)
        subp = {k: (v[touched] if isinstance(v, np.ndarray) else v) for k, v in sp.items()}
        rp = O.project_backward(subp, cam, q_xy[touched], q_con[touched], q_o[touched], q_rgb[touched])
        sp_screen = screen_reference(subp, cam, {"xy": q_xy[touched], "conic": q_con[touched], "o": q_o[touched],
                                                 "rgb": q_rgb[touched]})
        for k in KEYS:
            sens_raw[k] = np.maximum(sens_raw[k], np.abs(rp[k] - ref[k]))
        sens_screen = np.maximum(sens_screen, np.abs(sp_screen - ref_screen))
    mag_t = tuple(m[touched] for m in mag)
    needles = proj[touched, O.F_F] < NEEDLE_F
    assert needles.sum() <= 0.1 * len(touched)
    report = assert_elementwise({k: g[k][touched] for k in KEYS}, ref, g["screen"][touched], ref_screen,
                                raw_magnitude(sub, cam, mag_t), screen_magnitude(sub, cam, mag_t), sens_raw,
                                sens_screen, needles)
    rest = np.ones(len(scene["opacities"]), bool)
    rest[touched] = False
    for k in KEYS:
        assert not np.any(g[k][rest]), k  # no pixel with a loss gradient reaches them
    print(report)


def test_backward_matches_fp64_finite_differences():
    sc, cam, G = problem(n=256, deg=1, seed=78)
    sc64 = f64(sc)
    g, _ = gpu_grads(sc, cam, G)
    _, mag = oracle_backward_with_magnitudes(sc64, cam, G, (0.1, 0.2, 0.3))
    mag_raw = raw_magnitude(sc64, cam, mag)
    rng = np.random.default_rng(1)
    checked = 0
    for k in KEYS:
        flat = g[k].reshape(256, -1)
        rows = list(np.argsort(-np.abs(flat).max(axis=1))[:4]) + list(rng.integers(0, 256, 2))
        for i in rows:
            for j in range(min(flat.shape[1], 3)):
                base = sc64[k].reshape(256, -1)[i, j]
                h = 1e-5 * max(1.0, abs(base))
                vals = []
                for d in (h, -h, 0.0):
                    s2 = {kk: (v.copy() if isinstance(v, np.ndarray) else v) for kk, v in sc64.items()}
                    s2[k].reshape(256, -1)[i, j] = base + d
                    vals.append(float((O.image(s2, cam, O.QUADBOX, bg=(0.1, 0.2, 0.3))["img"] * G).sum()))
                fp, fm, f0 = vals
                if abs((fp - f0) - (f0 - fm)) > 1e-3 * (abs(fp - fm) / 2 + 1e-3 * h):
                    continue  # a discrete decision changed inside [-h, h]
                fd = (fp - fm) / (2 * h)
                # the element-wise bar of the analytic comparison
                m = mag_raw[k].reshape(256, -1)[i, j]
                assert abs(flat[i, j] - fd) <= REL * abs(fd) + MAG * m, (k, i, j, flat[i, j], fd, m)
                checked += 1
    assert checked >= 30


def test_binning_does_not_change_gradients():
    sc, cam, G = problem(n=400, deg=1, seed=79)
    ga, _ = gpu_grads(sc, cam, G, mode="aabb3s")
    gq, _ = gpu_grads(sc, cam, G, mode="quadbox")
    for k in KEYS:
        # same pairs contribute; only atomics' summation order may differ
        assert normwise(gq[k], ga[k]) <= 1e-5, k


def test_autograd_function():
    import torch
    from paper_2605_04844_gb300 import rasterizer as R
    sc, cam, G = problem(n=256, deg=1, seed=80)
    sd = to_device(sc)
    leaves = {k: sd[k].clone().requires_grad_(True) for k in KEYS}
    img = R.rasterize(leaves["means"], leaves["scales"], leaves["quats"], leaves["opacities"], leaves["sh"], cam,
                      "quadbox", (0.1, 0.2, 0.3))
    (img * torch.from_numpy(G.astype(np.float32)).cuda()).sum().backward()
    g, img2 = gpu_grads(sc, cam, G)
    np.testing.assert_array_equal(img.detach().cpu().numpy(), img2)
    for k in KEYS:
        assert normwise(leaves[k].grad.cpu().numpy().astype(np.float64), g[k]) <= 1e-5
