"""GPU backward (qb_render_bwd, stages S11-S12) against the oracle's analytic
FP64 gradient and FP64 central finite differences; autograd.Function."""
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


def problem(n=256, W=64, H=64, deg=1, seed=77):
    cam = synth.pinhole(W, H)
    sc = synth.scene_uniform(n, seed, cam, depth=(2.0, 5.0), logscale=(-2.2, 0.5), deg=deg)
    G = np.random.default_rng(seed).standard_normal((3, H, W))
    return sc, cam, G


@pytest.mark.parametrize("deg", [0, 1, 3])
def test_backward_matches_oracle_analytic(deg):
    sc, cam, G = problem(deg=deg)
    g, _ = gpu_grads(sc, cam, G)
    ref = O.gradients(f64(sc), cam, G, bg=(0.1, 0.2, 0.3))
    ref_screen = screen_reference(f64(sc), cam, ref["screen"])
    assert normwise(g["screen"], ref_screen) <= 1e-3
    for k in KEYS:
        assert normwise(g[k], ref[k]) <= 1e-3, (k, normwise(g[k], ref[k]))


def test_backward_blobs_sh3():
    cam = synth.pinhole(160, 104)
    sc = synth.scene_blobs(4000, 1104, cam, deg=3)
    G = np.sign(np.random.default_rng(5).standard_normal((3, 104, 160))) / (3 * 160 * 104)
    g, _ = gpu_grads(sc, cam, G, bg=(0.0, 0.0, 0.0))
    ref = O.gradients(f64(sc), cam, G, bg=(0.0, 0.0, 0.0))
    for k in KEYS:
        assert normwise(g[k], ref[k]) <= 1e-3, (k, normwise(g[k], ref[k]))


def test_backward_matches_fp64_finite_differences():
    sc, cam, G = problem(n=256, deg=1, seed=78)
    sc64 = f64(sc)
    g, _ = gpu_grads(sc, cam, G)
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
                assert flat[i, j] == pytest.approx(fd, rel=1e-3, abs=1e-3 * np.abs(flat).max()), (k, i, j)
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
