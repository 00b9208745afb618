"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks an oracle function against something other than itself:
closed forms of the QuadBox paper (Eq. support, extents-closed, f-closed),
brute-force maximisation over the ellipse, library routines (scipy's
spherical harmonics and rotations, numpy's matrix inverse), invariants of
Sec. 3 (conservativeness, QuadBox within the 3-sigma box, QPass = naive
union, binning-independent images) and finite differences.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_04844_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# helpers written independently of the oracle
# ---------------------------------------------------------------------------

def ellipse_extent_bruteforce(a, b, c, gamma, n=200001):
    """max |x| and |y| over {u : u^T Lambda u = gamma} by dense sampling of
    u = sqrt(gamma) L^-T (cos t, sin t) with Lambda = L L^T."""
    L = np.linalg.cholesky(np.array([[a, b], [b, c]]))
    t = np.linspace(0, 2 * np.pi, n)
    circ = np.stack([np.cos(t), np.sin(t)])
    u = math.sqrt(gamma) * np.linalg.solve(L.T, circ)
    return np.abs(u[0]).max(), np.abs(u[1]).max(), u


def axis_intercepts_bruteforce(a, c, gamma):
    """Roots of a x^2 = gamma and c y^2 = gamma by bisection (not a closed form)."""
    def root(coef):
        lo, hi = 0.0, 1.0
        while coef * hi * hi < gamma:
            hi *= 2
        for _ in range(200):
            mid = 0.5 * (lo + hi)
            if coef * mid * mid < gamma:
                lo = mid
            else:
                hi = mid
        return 0.5 * (lo + hi)
    return root(a), root(c)


def identity_cam(W=64, H=64, fx=100.0):
    return {"viewmat": np.eye(4, dtype=np.float32), "fx": fx, "fy": fx, "cx": (W - 1) / 2, "cy": (H - 1) / 2,
            "tan_fovx": W / (2 * fx), "tan_fovy": H / (2 * fx), "campos": np.zeros(3, np.float32),
            "width": W, "height": H, "znear": 0.2}


def one_gaussian_scene(mean, scales, quat, opac, deg=0, raw=0, rgb=(0.7, 0.2, 0.4)):
    K = (deg + 1) ** 2
    sh = np.zeros((1, K, 3))
    sh[0, 0] = (np.asarray(rgb) - 0.5) / synth.SH_C0
    return {"means": np.array([mean], float), "scales": np.array([scales], float),
            "quats": np.array([quat], float), "opacities": np.array([opac], float), "sh": sh,
            "sh_degree": deg, "raw": raw}


def small_scene(n=1500, seed=7, W=96, H=80, deg=0, logscale=(-2.5, 0.9)):
    cam = synth.pinhole(W, H)
    return synth.scene_uniform(n, seed, cam, depth=(1.0, 6.0), logscale=logscale, deg=deg), cam


# ---------------------------------------------------------------------------
# spherical harmonics
# ---------------------------------------------------------------------------

def test_sh_basis_matches_scipy_complex_harmonics():
    sp = pytest.importorskip("scipy.special")
    rng = np.random.default_rng(0)
    d = rng.standard_normal((40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = O.sh_basis(3, d)
    theta = np.arccos(np.clip(d[:, 2], -1, 1))  # polar
    phi = np.arctan2(d[:, 1], d[:, 0])
    for l in range(4):
        for m in range(-l, l + 1):
            am = abs(m)
            Yc = sp.sph_harm_y(l, am, theta, phi)  # includes the Condon-Shortley phase
            if m == 0:
                ref = Yc.real
            elif m > 0:
                ref = math.sqrt(2) * Yc.real
            else:
                ref = math.sqrt(2) * Yc.imag
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, rtol=1e-12, atol=1e-12)


def test_sh_basis_orthonormal_under_quadrature():
    # Gauss-Legendre in cos(theta) x uniform in phi integrates these polynomials exactly
    x, w = np.polynomial.legendre.leggauss(16)
    phis = np.linspace(0, 2 * np.pi, 32, endpoint=False)
    dirs, wts = [], []
    for xi, wi in zip(x, w):
        s = math.sqrt(1 - xi * xi)
        for ph in phis:
            dirs.append([s * math.cos(ph), s * math.sin(ph), xi])
            wts.append(wi * 2 * np.pi / len(phis))
    Y = O.sh_basis(3, np.array(dirs))
    G = (Y * np.array(wts)[:, None]).T @ Y
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_degree0_colour():
    cam = identity_cam()
    sc = one_gaussian_scene([0.1, -0.2, 10.0], [0.1, 0.1, 0.1], [1, 0, 0, 0], 0.5, rgb=(0.7, 0.2, 0.4))
    p = O.project(sc, cam)[0]
    np.testing.assert_allclose(p[[O.F_R, O.F_G, O.F_BL]], [0.7, 0.2, 0.4], atol=1e-14)


# ---------------------------------------------------------------------------
# rotation and projection
# ---------------------------------------------------------------------------

def test_rotation_matches_scipy_and_sign_flip():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    import ctypes
    rng = np.random.default_rng(1)
    for _ in range(20):
        q = rng.standard_normal(4)
        R = np.zeros(9)
        O.lib().orc_quat_to_rot(O._p(np.ascontiguousarray(q)), O._p(R))
        ref = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()  # scipy is (x, y, z, w)
        np.testing.assert_allclose(R.reshape(3, 3), ref, atol=1e-13)
        R2 = np.zeros(9)
        O.lib().orc_quat_to_rot(O._p(np.ascontiguousarray(-q)), O._p(R2))
        np.testing.assert_allclose(R2, R, atol=1e-15)


def test_projection_isotropic_on_axis_closed_form():
    cam = identity_cam(W=64, H=48, fx=120.0)
    s, tz = 0.05, 4.0
    sc = one_gaussian_scene([0.0, 0.0, tz], [s, s, s], [1, 0, 0, 0], 0.8)
    p = O.project(sc, cam)[0]
    k = 120.0 * s / tz
    np.testing.assert_allclose(p[[O.F_S11, O.F_S12, O.F_S22]], [k * k + 0.3, 0.0, k * k + 0.3], rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(p[[O.F_X, O.F_Y]], [cam["cx"], cam["cy"]], atol=1e-12)
    assert p[O.F_F] == pytest.approx(1.0, abs=1e-14)  # circle -> f = 1 (Sec. 3.1.2)


def test_projection_matches_numerical_jacobian_ewa():
    """Sigma2D = J W Sigma3 W^T J^T + 0.3 I with J the numerical Jacobian of the
    perspective map (unclamped means only) and Sigma3 built with scipy."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    scene, cam = small_scene(n=50, seed=3)
    V = cam["viewmat"].astype(np.float64)
    proj = O.project(scene, cam)
    fx, fy = cam["fx"], cam["fy"]
    for i in range(50):
        p = proj[i]
        if p[O.F_VALID] == 0 or p[24] != 0 or p[25] != 0:
            continue
        m = scene["means"][i].astype(np.float64)
        t = V[:3, :3] @ m + V[:3, 3]

        def pi(v):
            return np.array([fx * v[0] / v[2] + cam["cx"], fy * v[1] / v[2] + cam["cy"]])
        J = np.zeros((2, 3))
        for j in range(3):
            e = np.zeros(3); e[j] = 1e-6 * t[2]
            J[:, j] = (pi(t + e) - pi(t - e)) / (2e-6 * t[2])
        q = scene["quats"][i].astype(np.float64)
        R = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S = np.diag(np.exp(scene["scales"][i].astype(np.float64)))
        S3 = R @ S @ S @ R.T
        S2 = J @ V[:3, :3] @ S3 @ V[:3, :3].T @ J.T + 0.3 * np.eye(2)
        np.testing.assert_allclose(p[[O.F_S11, O.F_S12, O.F_S22]], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-6)
        np.testing.assert_allclose(p[[O.F_X, O.F_Y]], pi(t), rtol=1e-12)
        inv = np.linalg.inv(S2)
        np.testing.assert_allclose(p[[O.F_A, O.F_B, O.F_C]], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-5)


# ---------------------------------------------------------------------------
# Sec. 3.1: gamma, extents, support function, f
# ---------------------------------------------------------------------------

def test_golden_closed_form_case():
    g = json.load(open(os.path.join(GOLDEN, "quadbox_closed_form.json")))
    c = g["camera"]
    cam = identity_cam(W=c["width"], H=c["height"], fx=c["fx"])
    gg = g["gaussian"]
    sc = one_gaussian_scene(gg["mean"], gg["scales"], gg["quat_wxyz"], gg["opacity"])
    p = O.project(sc, cam)[0]
    e = g["expected"]
    np.testing.assert_allclose(p[[O.F_S11, O.F_S12, O.F_S22]], e["sigma2d"], rtol=1e-6)
    np.testing.assert_allclose(p[[O.F_A, O.F_B, O.F_C]], e["conic"], rtol=1e-6)
    assert p[O.F_F] == pytest.approx(e["f"], rel=1e-6)
    gb = p[O.F_GAMMAB]
    assert p[O.F_XMAX] / math.sqrt(gb) == pytest.approx(e["x_max_over_sqrt_gamma"], rel=1e-6)
    assert p[O.F_XMIN] / math.sqrt(gb) == pytest.approx(e["x_inter_over_sqrt_gamma"], rel=1e-6)
    assert int(p[O.F_ORIENT]) == e["orient_major_in_quadrants_I_III"]
    # gamma = 2 ln(o / alpha_min) at o = 1 (Eq. 3)
    assert p[O.F_GAMMA] == pytest.approx(2 * math.log(255.0), rel=1e-14)


def test_extents_and_f_against_bruteforce_and_closed_forms():
    scene, cam = small_scene(n=300, seed=11)
    proj = O.project(scene, cam)
    checked = 0
    for p in proj:
        if p[O.F_VALID] == 0:
            continue
        a, b, c, gb = p[O.F_A], p[O.F_B], p[O.F_C], p[O.F_GAMMAB]
        xm, ym, _ = ellipse_extent_bruteforce(a, b, c, gb)
        assert p[O.F_XMAX] == pytest.approx(xm, rel=1e-9)
        assert p[O.F_YMAX] == pytest.approx(ym, rel=1e-9)
        # Eq. extents-closed
        assert p[O.F_XMAX] == pytest.approx(math.sqrt(gb * c / (a * c - b * b)), rel=1e-10)
        assert p[O.F_YMAX] == pytest.approx(math.sqrt(gb * a / (a * c - b * b)), rel=1e-10)
        # intercepts and Eq. f-closed
        xi, yi = axis_intercepts_bruteforce(a, c, gb)
        assert p[O.F_XMIN] == pytest.approx(xi, rel=1e-10)
        assert p[O.F_YMIN] == pytest.approx(yi, rel=1e-10)
        f = p[O.F_F]
        assert 0 < f <= 1 + 1e-15
        assert f == pytest.approx(xi / xm, rel=1e-8) and f == pytest.approx(yi / ym, rel=1e-8)
        # the two other forms of Eq. f-closed (Lambda^-1 = Sigma2D)
        assert f == pytest.approx(1 / math.sqrt(c * p[O.F_S22]), rel=1e-10)
        assert f == pytest.approx(1 / math.sqrt(a * p[O.F_S11]), rel=1e-10)
        checked += 1
    assert checked > 200


def test_support_function_identity():
    """Eq. support: max_{u^T Lambda u = gamma} v^T u = sqrt(gamma v^T Lambda^-1 v)."""
    rng = np.random.default_rng(5)
    for _ in range(30):
        A = rng.standard_normal((2, 2))
        Lam = A @ A.T + 0.1 * np.eye(2)
        gamma = rng.uniform(0.5, 11.0)
        v = rng.standard_normal(2)
        _, _, u = ellipse_extent_bruteforce(Lam[0, 0], Lam[0, 1], Lam[1, 1], gamma)
        best = (v @ u).max()
        closed = math.sqrt(gamma * v @ np.linalg.inv(Lam) @ v)
        assert best == pytest.approx(closed, rel=1e-9)


def test_f_is_one_for_axis_aligned_and_circles():
    cam = identity_cam()
    for quat in ([1, 0, 0, 0], [0, 0, 0, 1]):  # axis aligned
        sc = one_gaussian_scene([0.0, 0.0, 100.0], [3.0, 1.0, 0.01], quat, 0.9)
        p = O.project(sc, cam)[0]
        assert p[O.F_F] == pytest.approx(1.0, abs=1e-12)
        np.testing.assert_allclose(p[O.F_XMIN], p[O.F_XMAX], rtol=1e-12)


def test_gamma_cull_below_alpha_min():
    cam = identity_cam()
    sc = one_gaussian_scene([0.0, 0.0, 100.0], [1.0, 1.0, 1.0], [1, 0, 0, 0], 0.9 / 255)
    assert O.project(sc, cam)[0][O.F_VALID] == 0
    sc = one_gaussian_scene([0.0, 0.0, 0.1], [1.0, 1.0, 1.0], [1, 0, 0, 0], 0.9)  # behind near plane
    assert O.project(sc, cam)[0][O.F_VALID] == 0


# ---------------------------------------------------------------------------
# Sec. 3.1.2 / 3.2: tile sets
# ---------------------------------------------------------------------------

def tile_sets(rects, use_qpass, tiles_x):
    counts, offsets, tiles, gids = O.tile_lists(rects, use_qpass, tiles_x)
    out = []
    for i in range(len(counts)):
        out.append(list(tiles[offsets[i]:offsets[i] + counts[i]]))
    return out


def adversarial_scene(n=2000, seed=21, W=160, H=96):
    """Uniform scene plus strongly anisotropic, diagonal and huge Gaussians and
    some straddling the image border."""
    cam = synth.pinhole(W, H)
    sc = synth.scene_uniform(n, seed, cam, depth=(1.0, 8.0), logscale=(-2.5, 1.2), deg=0)
    rng = np.random.default_rng(seed + 1)
    k = n // 4
    sc["scales"][:k, 0] += 3.0  # needles
    sc["scales"][:k, 1] -= 1.0
    sc["opacities"][:k // 2] = 4.0  # opaque: gamma > 9, the QuadBox exceeds 3 sigma
    sc["means"][-50:, 0] *= 1.4  # some off the image edge
    return sc, cam


@pytest.mark.parametrize("mode", [O.QUADBOX, O.ADR, O.DUALBOX, O.AABB3S])
def test_qpass_equals_naive_union(mode):
    sc, cam = adversarial_scene()
    W, H = cam["width"], cam["height"]
    tx, _ = O.grid(W, H)
    proj = O.project(sc, cam)
    for clamp in (True, False):
        rects = O.rects_f64(proj, mode, clamp, W, H)
        qp = tile_sets(rects, True, tx)
        nv = tile_sets(rects, False, tx)
        for i, (a, b) in enumerate(zip(qp, nv)):
            assert len(a) == len(set(a)), f"QPass visited a tile twice for Gaussian {i}"
            assert len(b) == len(set(b))
            assert set(a) == set(b), f"QPass != naive union for Gaussian {i}"
            # the naive union is the set union of the rectangles
            u = set()
            for q in range(4):
                x0, y0, x1, y1 = rects[i, q]
                for yy in range(y0, y1 + 1):
                    for xx in range(x0, x1 + 1):
                        u.add(yy * tx + xx)
            assert u == set(a)


def test_quadbox_within_3sigma_and_adr():
    sc, cam = adversarial_scene()
    W, H = cam["width"], cam["height"]
    tx, _ = O.grid(W, H)
    proj = O.project(sc, cam)
    S = tile_sets(O.rects_f64(proj, O.AABB3S, True, W, H), True, tx)
    Q = tile_sets(O.rects_f64(proj, O.QUADBOX, True, W, H), True, tx)
    A = tile_sets(O.rects_f64(proj, O.ADR, True, W, H), True, tx)
    Qn = tile_sets(O.rects_f64(proj, O.QUADBOX, False, W, H), True, tx)
    An = tile_sets(O.rects_f64(proj, O.ADR, False, W, H), True, tx)
    fewer = 0
    for s, q, a, qn, an in zip(S, Q, A, Qn, An):
        assert set(q) <= set(s)
        assert set(q) <= set(a)
        assert set(qn) <= set(an)  # QuadBox lies inside the AdR box (Sec. 3.1.2)
        fewer += len(q) < len(a)
    assert fewer > 0


def test_conservative_bruteforce():
    """Every tile holding a pixel with alpha >= (1/255)(1 + 1e-6) is covered
    (within the 3-sigma rectangle when clamped; everywhere without the clamp)."""
    sc, cam = adversarial_scene(n=1200, seed=33)
    W, H = cam["width"], cam["height"]
    tx, _ = O.grid(W, H)
    proj = O.project(sc, cam)
    ys, xs = np.mgrid[0:H, 0:W]
    for clamp in (True, False):
        Q = tile_sets(O.rects_f64(proj, O.QUADBOX, clamp, W, H), True, tx)
        S = tile_sets(O.rects_f64(proj, O.AABB3S, True, W, H), True, tx)
        for i, p in enumerate(proj):
            if p[O.F_VALID] == 0:
                continue
            dx, dy = p[O.F_X] - xs, p[O.F_Y] - ys
            q = p[O.F_A] * dx * dx + 2 * p[O.F_B] * dx * dy + p[O.F_C] * dy * dy
            alpha = p[O.F_O] * np.exp(-0.5 * q)
            hit = alpha >= (1 / 255) * (1 + 1e-6)
            tiles = set(((ys[hit] // 16) * tx + xs[hit] // 16).tolist())
            if clamp:
                tiles &= set(S[i])
            assert tiles <= set(Q[i]), f"Gaussian {i}: uncovered tiles {sorted(tiles - set(Q[i]))[:5]}"


def _three_sigma_scene():
    """The adversarial scene plus isotropic Gaussians of several sizes (equal
    eigenvalues: the discriminant floor of the radius binds there)."""
    sc, cam = adversarial_scene(n=1200, seed=44)
    iso = 40
    rng = np.random.default_rng(45)
    z = rng.uniform(1.5, 6.0, iso)
    xy = rng.uniform(-0.3, 0.3, (iso, 2)) * z[:, None]
    means = np.concatenate([xy, z[:, None]], axis=1)
    s = np.repeat(rng.uniform(-4.0, -1.0, iso)[:, None], 3, axis=1)  # equal log-scales
    quats = np.tile([1.0, 0.0, 0.0, 0.0], (iso, 1))
    sc = dict(sc)
    for k, v in (("means", means), ("scales", s), ("quats", quats), ("opacities", np.full(iso, 2.0)),
                 ("sh", np.zeros((iso,) + sc["sh"].shape[1:]))):
        sc[k] = np.concatenate([np.asarray(sc[k], np.float64), v.astype(np.float64)])
    return sc, cam, iso


def test_3sigma_radius_against_eigenvalues():
    """The vanilla box of Sec. 2 has side 6 sqrt(lambda_max), lambda_max the
    largest eigenvalue of Sigma^2D: the oracle's integer radius is
    ceil(3 sqrt(lambda_max)) with lambda_max from numpy's symmetric eigen-
    solver.  The discriminant of the 2x2 eigenvalue formula is floored at 0.1
    (the 3DGS convention, reading C2): where ((l1 - l2) / 2)^2 < 0.1 the
    radius is ceil(3 sqrt(trace / 2 + sqrt(0.1))), which still covers
    lambda_max."""
    sc, cam, iso = _three_sigma_scene()
    proj = O.project(sc, cam)
    checked = floored = 0
    for i, p in enumerate(proj):
        if p[O.F_VALID] == 0:
            continue
        S = np.array([[p[O.F_S11], p[O.F_S12]], [p[O.F_S12], p[O.F_S22]]])
        lam = np.linalg.eigvalsh(S)  # ascending
        half_gap2 = (0.5 * (lam[1] - lam[0])) ** 2
        if half_gap2 >= 0.1 * (1 + 1e-9):
            want = 3.0 * math.sqrt(lam[1])
        elif half_gap2 <= 0.1 * (1 - 1e-9):
            want = 3.0 * math.sqrt(0.5 * (lam[0] + lam[1]) + math.sqrt(0.1))
            assert want >= 3.0 * math.sqrt(lam[1])
            floored += 1
        else:
            continue
        if abs(want - round(want)) < 1e-9:
            continue  # ceil undecidable at the rounding of the eigenvalues
        assert p[O.F_R3] == math.ceil(want), f"Gaussian {i}: r3 {p[O.F_R3]} vs ceil({want})"
        checked += 1
    assert checked > 1000 and floored >= iso


def test_3sigma_rect_holds_the_3sigma_ellipse_bruteforce():
    """Every pixel centre inside the 3-sigma ellipse d^T Sigma^-1 d <= 9 (the
    inverse by numpy, not the oracle's conic) lies in the 3-sigma pixel
    interval [ceil(mu) - r3, floor(mu) + r3] on both axes and in a tile of the
    AABB3S tile set, and the interval is no wider than one pixel plus
    3 sqrt(lambda_max) on each side (so r3 is not inflated either)."""
    sc, cam, _ = _three_sigma_scene()
    W, H = cam["width"], cam["height"]
    tx, _ = O.grid(W, H)
    proj = O.project(sc, cam)
    S3 = tile_sets(O.rects_f64(proj, O.AABB3S, True, W, H), True, tx)
    ys, xs = np.mgrid[0:H, 0:W]
    inside_px = 0
    for i, p in enumerate(proj):
        if p[O.F_VALID] == 0:
            continue
        S = np.array([[p[O.F_S11], p[O.F_S12]], [p[O.F_S12], p[O.F_S22]]])
        Si = np.linalg.inv(S)
        dx, dy = xs - p[O.F_X], ys - p[O.F_Y]
        m = Si[0, 0] * dx * dx + 2 * Si[0, 1] * dx * dy + Si[1, 1] * dy * dy
        hit = m <= 9.0
        r3 = p[O.F_R3]
        assert np.all(np.abs(dx[hit]) <= r3) and np.all(np.abs(dy[hit]) <= r3), f"Gaussian {i}"
        tiles = set(((ys[hit] // 16) * tx + xs[hit] // 16).tolist())
        assert tiles <= set(S3[i]), f"Gaussian {i}: 3-sigma pixels outside the AABB3S tiles"
        inside_px += int(hit.sum())
        lmax = np.linalg.eigvalsh(S)[1]
        assert r3 <= 3.0 * math.sqrt(lmax + math.sqrt(0.1)) + 1.0
    assert inside_px > 10000


def test_dualbox_is_not_conservative():
    sc, cam = adversarial_scene(n=1200, seed=33)
    W, H = cam["width"], cam["height"]
    r_q = O.image(sc, cam, O.QUADBOX)
    r_d = O.image(sc, cam, O.DUALBOX)
    assert len(r_d["vals"]) < len(r_q["vals"])
    assert np.abs(r_q["img"] - r_d["img"]).max() > 1e-3


def test_float32_rect_replay_matches_f64_rule_on_exact_inputs():
    """With inputs exactly representable in float32 the two rect builders agree."""
    sc, cam = adversarial_scene(n=500, seed=44)
    W, H = cam["width"], cam["height"]
    proj = O.project(sc, cam)
    f = lambda a: a.astype(np.float32).astype(np.float64)
    p32 = proj.copy()
    for col in (O.F_X, O.F_Y, O.F_XMAX, O.F_YMAX, O.F_XMIN, O.F_YMIN, O.F_R3):
        p32[:, col] = f(proj[:, col])
    # make every sub-box endpoint exact in float32 too: quantise to 1/256 px
    for col in (O.F_X, O.F_Y, O.F_XMAX, O.F_YMAX, O.F_XMIN, O.F_YMIN):
        p32[:, col] = np.round(p32[:, col] * 256) / 256
    for mode in (O.QUADBOX, O.AABB3S, O.ADR, O.DUALBOX):
        r64 = O.rects_f64(p32, mode, True, W, H)
        r32 = O.rects_f32(p32[:, [O.F_X, O.F_Y]], p32[:, [O.F_XMAX, O.F_YMAX, O.F_XMIN, O.F_YMIN]],
                          p32[:, O.F_R3], p32[:, O.F_ORIENT].astype(np.int32), p32[:, O.F_VALID].astype(np.int32),
                          mode, True, W, H)
        np.testing.assert_array_equal(r32, r64)


# ---------------------------------------------------------------------------
# Eq. 2: compositing
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("mode", [O.AABB3S, O.QUADBOX, O.ADR])
def test_tiled_render_equals_tile_free_bruteforce(mode):
    sc, cam = small_scene(n=900, seed=5)
    W, H = cam["width"], cam["height"]
    r = O.image(sc, cam, mode)
    b = O.render_brute(W, H, r["rects"], r["proj"])
    np.testing.assert_array_equal(r["img"], b[0])
    np.testing.assert_array_equal(r["n_contrib"], b[2])


def test_image_identical_across_conservative_binnings():
    sc, cam = adversarial_scene(n=1500, seed=9)
    imgs = [O.image(sc, cam, m)["img"] for m in (O.AABB3S, O.QUADBOX, O.ADR, O.QUADBOX_NAIVE)]
    for im in imgs[1:]:
        np.testing.assert_array_equal(im, imgs[0])


def test_single_gaussian_pixel_closed_form():
    cam = identity_cam(W=64, H=64, fx=100.0)
    g = json.load(open(os.path.join(GOLDEN, "quadbox_closed_form.json")))["gaussian"]
    sc = one_gaussian_scene(g["mean"], g["scales"], g["quat_wxyz"], 0.6, rgb=(0.9, 0.3, 0.1))
    r = O.image(sc, cam, O.QUADBOX, bg=(0.1, 0.2, 0.3))
    Lam = np.array([[0.625, -0.375], [-0.375, 0.625]])
    for (px, py) in [(31, 31), (33, 30), (29, 34), (40, 31)]:
        d = np.array([31.5 - px, 31.5 - py])
        alpha = min(0.99, 0.6 * math.exp(-0.5 * d @ Lam @ d))
        if alpha < 1 / 255:
            expect = np.array([0.1, 0.2, 0.3])
        else:
            expect = alpha * np.array([0.9, 0.3, 0.1]) + (1 - alpha) * np.array([0.1, 0.2, 0.3])
        np.testing.assert_allclose(r["img"][:, py, px], expect, rtol=1e-5, atol=1e-7)


def test_keys_sort_by_tile_then_depth_then_index():
    sc, cam = small_scene(n=600, seed=12)
    W, H = cam["width"], cam["height"]
    tx, ty = O.grid(W, H)
    proj = O.project(sc, cam)
    rects = O.rects_f64(proj, O.QUADBOX, True, W, H)
    counts, offsets, tiles, gids = O.tile_lists(rects, True, tx)
    depth32 = proj[:, O.F_DEPTH].astype(np.float32)
    depth32[5] = depth32[6]  # force a depth tie between two Gaussians
    keys = O.keys_from_lists(tiles, gids, depth32)
    sk, sv = O.sort_pairs(keys, gids)
    ref = np.lexsort((gids, depth32[gids.astype(np.int64)], tiles))
    np.testing.assert_array_equal(sv, gids[ref])
    rg = O.ranges_from_sorted_tiles((sk >> np.uint64(31)).astype(np.int64), tx * ty)
    for t in range(tx * ty):
        s, e = rg[t]
        assert np.all((sk[s:e] >> np.uint64(31)) == t)
    assert rg[:, 1].max() == len(sk)


# ---------------------------------------------------------------------------
# backward
# ---------------------------------------------------------------------------

def _loss_and_grads(sc, cam, G, mode=O.QUADBOX, bg=(0.1, 0.2, 0.3)):
    r = O.image(sc, cam, mode, bg=bg)
    return float((r["img"] * G).sum()), r


def test_projection_backward_matches_finite_differences():
    """Chain rule of the projection vs central differences of the projection."""
    sc, cam = small_scene(n=40, seed=8, deg=3, logscale=(-2.0, 0.6))
    n = 40
    proj = O.project(sc, cam)
    rng = np.random.default_rng(1)
    gxy, gcon, go, grgb = rng.standard_normal((n, 2)), rng.standard_normal((n, 3)), rng.standard_normal(n), \
        rng.standard_normal((n, 3))
    g = O.project_backward(sc, cam, gxy, gcon, go, grgb)

    def L(s):
        p = O.project(s, cam)
        m = p[:, O.F_VALID] != 0
        v = (gxy * p[:, [O.F_X, O.F_Y]]).sum(1) + (gcon * p[:, [O.F_A, O.F_B, O.F_C]]).sum(1) \
            + go * p[:, O.F_O] + (grgb * p[:, [O.F_R, O.F_G, O.F_BL]]).sum(1)
        return v, m

    base_valid = proj[:, O.F_VALID] != 0
    for key in ("means", "scales", "quats", "opacities", "sh"):
        arr = sc[key]
        flat = arr.reshape(n, -1)
        for i in range(n):
            if not base_valid[i] or proj[i, 24] or proj[i, 25]:
                continue
            for j in range(min(flat.shape[1], 6)):
                h = 1e-6 * max(1.0, abs(flat[i, j]))
                sp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
                sm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
                sp[key] = sp[key].astype(np.float64); sm[key] = sm[key].astype(np.float64)
                sp[key].reshape(n, -1)[i, j] += h
                sm[key].reshape(n, -1)[i, j] -= h
                vp, mp = L(sp)
                vm, mm = L(sm)
                if not (mp[i] and mm[i]):
                    continue
                fd = (vp[i] - vm[i]) / (2 * h)
                an = g[key].reshape(n, -1)[i, j]
                assert an == pytest.approx(fd, rel=2e-5, abs=2e-6 * (1 + abs(fd))), (key, i, j)


def test_render_backward_matches_finite_differences_fp64():
    """Full-pipeline gradient (render backward + projection backward) vs FP64
    central differences on a 64x64, 256-Gaussian problem, skipping entries
    whose +-h perturbation crosses a discrete threshold (detected by
    disagreeing one-sided differences)."""
    W, H = 64, 64
    cam = synth.pinhole(W, H)
    sc = synth.scene_uniform(256, 77, cam, depth=(2.0, 5.0), logscale=(-2.2, 0.5), deg=1)
    sc = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    G = np.random.default_rng(3).standard_normal((3, H, W))
    g = O.gradients(sc, cam, G, bg=(0.1, 0.2, 0.3))
    rng = np.random.default_rng(4)
    checked = 0
    for key in ("means", "scales", "quats", "opacities", "sh"):
        flat_g = g[key].reshape(256, -1)
        # probe the entries with the largest analytic gradients plus random ones
        order = np.argsort(-np.abs(flat_g).max(axis=1))[:6]
        for i in list(order) + list(rng.integers(0, 256, 3)):
            for j in range(min(flat_g.shape[1], 4)):
                base = sc[key].reshape(256, -1)[i, j]
                h = 1e-5 * max(1.0, abs(base))
                vals = []
                for dlt in (h, -h, 0.0):
                    s2 = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
                    s2[key].reshape(256, -1)[i, j] = base + dlt
                    vals.append(_loss_and_grads(s2, cam, G)[0])
                fp, fm, f0 = vals
                d_plus, d_minus = (fp - f0) / h, (f0 - fm) / h
                fd = (fp - fm) / (2 * h)
                if abs(d_plus - d_minus) > 1e-3 * (abs(fd) + 1e-3):
                    continue  # a discrete decision changed inside [-h, h]
                an = flat_g[i, j]
                assert an == pytest.approx(fd, rel=1e-4, abs=1e-6), (key, i, j, an, fd)
                checked += 1
    assert checked > 40


def test_pixel_subset_backward_equals_the_masked_full_backward():
    """render_backward_pixels over a pixel subset equals render_backward with
    dL/dimg zero outside the subset, exactly (the same per-pixel sums in the
    same order)."""
    sc, cam = small_scene(n=600, seed=12, W=48, H=40, deg=0)
    W, H = cam["width"], cam["height"]
    proj = O.project(sc, cam)
    L = O.own_lists(proj, W, H)
    rng = np.random.default_rng(3)
    G = rng.standard_normal((3, H, W))
    mask = rng.random((H, W)) < 0.3
    Gm = G * mask
    full = O.render_backward(W, H, L["ranges"], L["vals"], proj, Gm, bg=(0.1, 0.2, 0.3))
    pys, pxs = np.nonzero(mask)
    sub = O.render_backward_pixels(W, H, pxs, pys, G[:, pys, pxs].T, L["ranges"], L["vals"], proj,
                                   bg=(0.1, 0.2, 0.3))
    for a, b in zip(full, sub):
        assert np.any(a != 0)
        np.testing.assert_array_equal(a, b)
    # the magnitude sums bound the gradients (triangle inequality), and with
    # a non-negative dL every colour term is non-negative, so there they agree
    g, mag = O.render_backward_pixels(W, H, pxs, pys, G[:, pys, pxs].T, L["ranges"], L["vals"], proj,
                                      bg=(0.1, 0.2, 0.3), magnitudes=True)
    for a, m in zip(g, mag):
        assert np.all(np.abs(a) <= m * (1 + 1e-12))
    gp, magp = O.render_backward_pixels(W, H, pxs, pys, np.abs(G[:, pys, pxs].T), L["ranges"], L["vals"], proj,
                                        magnitudes=True)
    np.testing.assert_allclose(gp[3], magp[3], rtol=1e-12)
