"""The training-step integration: the L1 loss gradient and the fused Adam
update against their textbook definitions (numpy), and a short optimisation
that fits a scene to a rendered target."""
import numpy as np
import pytest

from paper_2605_04844_gb300 import synth

from gpu_util import to_device

pytestmark = pytest.mark.gpu


def test_l1_loss_grad_matches_numpy():
    import torch
    from paper_2605_04844_gb300 import _native as N
    rng = np.random.default_rng(3)
    a = rng.normal(size=100_003).astype(np.float32)
    b = rng.normal(size=100_003).astype(np.float32)
    b[:10] = a[:10]  # exact ties: zero gradient
    A, B = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    dL = torch.empty_like(A)
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    scale = 1.0 / a.size
    N.qb_l1_loss_grad(A, B, dL, scale, loss)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(dL.cpu().numpy(), (np.sign(a - b) * np.float32(scale)).astype(np.float32))
    ref = np.abs(a.astype(np.float64) - b.astype(np.float64)).sum() * np.float32(scale)
    assert abs(loss.item() - ref) <= 1e-6 * ref


def _adam_reference(p, g_seq, lr, b1, b2, eps):
    """Kingma & Ba's update with bias correction, in float64."""
    p = p.astype(np.float64).copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    for t, g in enumerate(g_seq, start=1):
        g = g.astype(np.float64)
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        p -= lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
    return p


def test_adam_matches_reference():
    import torch
    from paper_2605_04844_gb300 import _native as N
    rng = np.random.default_rng(5)
    n = 65_537
    p0 = rng.normal(size=n).astype(np.float32)
    gs = [rng.normal(size=n).astype(np.float32) * 10.0 ** rng.uniform(-3, 1, n).astype(np.float32)
          for _ in range(4)]
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-8
    P = torch.from_numpy(p0).cuda()
    M, V = torch.zeros_like(P), torch.zeros_like(P)
    for t, g in enumerate(gs, start=1):
        N.qb_adam_step(P, torch.from_numpy(g).cuda(), M, V, lr, b1, b2, eps, t)
    torch.cuda.synchronize()
    ref = _adam_reference(p0, gs, lr, b1, b2, eps)
    np.testing.assert_allclose(P.cpu().numpy(), ref, rtol=1e-5, atol=1e-6)
    # the first step moves every parameter by lr against the sign of its gradient
    P1 = torch.from_numpy(p0).cuda()
    N.qb_adam_step(P1, torch.from_numpy(gs[0]).cuda(), torch.zeros_like(P1), torch.zeros_like(P1), lr, b1, b2, eps, 1)
    step1 = P1.cpu().numpy() - p0
    big = np.abs(gs[0]) > 1e-3
    np.testing.assert_allclose(step1[big], -lr * np.sign(gs[0][big]), rtol=1e-4)


def test_adam_rejects_bad_arguments():
    import torch
    from paper_2605_04844_gb300 import _native as N
    P = torch.zeros(4, device="cuda")
    with pytest.raises(N.QbError):
        N.qb_adam_step(P, P, P, P, 1e-3, 0.9, 0.999, 1e-8, 0)
    with pytest.raises(N.QbError):
        N.qb_adam_step(P, P, P, P, 1e-3, 1.0, 0.999, 1e-8, 1)


def test_training_fits_a_rendered_target():
    """Colours of a scene are perturbed; Adam steps through the library's own
    forward, L1 gradient and backward bring the render back to the target."""
    import torch
    from paper_2605_04844_gb300 import rasterizer as R
    cam = synth.pinhole(160, 120)
    scene = synth.scene_blobs(6000, 1201, cam, deg=1)
    ref = to_device(scene)
    target, _ = R.forward(ref, cam, "quadbox")
    moved = dict(scene)
    moved["sh"] = scene["sh"] + np.random.default_rng(9).normal(0.0, 0.3, scene["sh"].shape).astype(np.float32)
    sd = to_device(moved)
    tr = R.Trainer(sd, cam, "quadbox", lr={"means": 0.0, "scales": 0.0, "quats": 0.0, "opacities": 0.0,
                                           "sh": 2e-2})
    losses = [float(tr.step(target).item()) for _ in range(40)]
    assert losses[-1] < 0.5 * losses[0], losses[::8]
