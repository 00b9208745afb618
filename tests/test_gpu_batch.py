"""The batched multi-camera path (qb_render_batch / qb_render_batch_bwd):
identical images and matching gradients to one frame per camera, CUDA-graph
capture, grouping, tuning variants and overflow handling."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_04844_gb300 import synth

from gpu_util import f64, image_parity, to_device

pytestmark = pytest.mark.gpu

KEYS = ("means", "scales", "quats", "opacities", "sh")


def problem(n=20_000, seed=55, sizes=((96, 64), (130, 70), (64, 64), (200, 120), (50, 90))):
    scene = synth.scene_ball(n, seed, radius=3.0, deg=3)
    rng = np.random.default_rng(seed)
    cams = []
    for k, (W, H) in enumerate(sizes):
        d = rng.standard_normal(3)
        pos = 6.0 * d / np.linalg.norm(d)
        cams.append(synth.pinhole(W, H, viewmat=synth.look_at(pos, (0.0, 0.0, 0.0))))
    return scene, cams


def frame_images(sd, cams, bg):
    from paper_2605_04844_gb300 import rasterizer as R
    out = []
    for c in cams:
        img, fr = R.forward(sd, c, "quadbox", bg=bg)
        out.append(img.cpu().numpy())
    return out


@pytest.mark.parametrize("group", [1, 2, 16])
def test_batch_images_identical_to_frames(group):
    import torch
    from paper_2605_04844_gb300 import rasterizer as R
    scene, cams = problem()
    sd = to_device(scene)
    bg = (0.1, 0.2, 0.3)
    b = R.calibrated_batch(sd, cams, group=group)
    b.render(R.scene_struct(sd), R.camera_array(cams), "quadbox", bg=bg)
    torch.cuda.synchronize()
    assert len(b.check()) == len(cams)
    ref = frame_images(sd, cams, bg)
    for k in range(len(cams)):
        np.testing.assert_array_equal(b.image(k).cpu().numpy(), ref[k])


def test_batch_image_parity_with_oracle():
    import torch
    from paper_2605_04844_gb300 import rasterizer as R
    scene, cams = problem(n=8000)
    sd = to_device(scene)
    b = R.calibrated_batch(sd, cams, group=4)
    b.render(R.scene_struct(sd), R.camera_array(cams), "quadbox", bg=(0.1, 0.2, 0.3))
    torch.cuda.synchronize()
    for k in (0, 3):
        ref = O.image(f64(scene), cams[k], O.QUADBOX, bg=(0.1, 0.2, 0.3))
        ok, st = image_parity(b.image(k).cpu().numpy(), ref)
        assert ok, (k, st)


@pytest.mark.parametrize("tune", [{"tiles_per_fetch": 1, "render_batch": 64, "sort_digit_bits": 8},
                                  {"tiles_per_fetch": 4, "render_batch": 256, "sort_digit_bits": 11,
                                   "blocks_per_sm": 2},
                                  {"tiles_per_fetch": 8, "render_batch": 128, "sort_digit_bits": 10}])
def test_batch_tuning_does_not_change_images(tune):
    import torch
    from paper_2605_04844_gb300 import rasterizer as R
    scene, cams = problem(n=10_000)
    sd = to_device(scene)
    b = R.calibrated_batch(sd, cams, group=3)
    s, ca = R.scene_struct(sd), R.camera_array(cams)
    b.render(s, ca, "quadbox")
    base = b.images.clone()
    b.render(s, ca, "quadbox", tune=tune)
    torch.cuda.synchronize()
    b.check()
    assert torch.equal(b.images, base)


def test_batch_cuda_graph_replay():
    import torch
    from paper_2605_04844_gb300 import rasterizer as R
    scene, cams = problem(n=10_000)
    sd = to_device(scene)
    b = R.calibrated_batch(sd, cams, group=2)
    s, ca = R.scene_struct(sd), R.camera_array(cams)
    b.render(s, ca, "quadbox")  # first call outside capture
    torch.cuda.synchronize()
    ref = b.images.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        b.stream = side
        with torch.cuda.graph(g, stream=side):
            b.render(s, ca, "quadbox")
    b.stream = None
    for _ in range(2):
        b.images.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(b.images, ref)
    b.check()


def test_batch_backward_matches_frames():
    import torch
    from paper_2605_04844_gb300 import _native as N
    from paper_2605_04844_gb300 import rasterizer as R
    scene, cams = problem(n=6000, sizes=((64, 48), (80, 60), (48, 48)))
    sd = to_device(scene)
    bg = (0.1, 0.2, 0.3)
    b = R.calibrated_batch(sd, cams, group=2)
    s, ca = R.scene_struct(sd), R.camera_array(cams)
    b.render(s, ca, "quadbox", bg=bg)
    dL = torch.randn(b.images.shape, generator=torch.Generator("cuda").manual_seed(3), device="cuda")
    gb = {k: torch.zeros_like(sd[k]) for k in KEYS}
    gsb = N.QbSceneGrads()
    gsb.means, gsb.scales, gsb.quats = gb["means"].data_ptr(), gb["scales"].data_ptr(), gb["quats"].data_ptr()
    gsb.opacities, gsb.sh = gb["opacities"].data_ptr(), gb["sh"].data_ptr()
    b.backward(s, ca, dL, gsb, bg=bg)
    torch.cuda.synchronize()
    b.check()
    gf = {k: torch.zeros_like(sd[k]) for k in KEYS}
    for k, c in enumerate(cams):
        img, fr = R.forward(sd, c, "quadbox", bg=bg)
        gs = N.QbSceneGrads()
        gs.means, gs.scales, gs.quats = gf["means"].data_ptr(), gf["scales"].data_ptr(), gf["quats"].data_ptr()
        gs.opacities, gs.sh = gf["opacities"].data_ptr(), gf["sh"].data_ptr()
        N.qb_render_bwd(fr.frame, s, R.camera_struct(c), bg, b.image(k, dL).contiguous(), gs, None)
    torch.cuda.synchronize()
    for k in KEYS:
        a, r = gb[k].double(), gf[k].double()
        assert (torch.linalg.norm(a - r) / torch.linalg.norm(r)).item() <= 1e-5, k


def test_batch_capacity_overflow_is_flagged():
    import torch
    from paper_2605_04844_gb300 import _native as N
    from paper_2605_04844_gb300 import rasterizer as R
    scene, cams = problem(n=10_000)
    sd = to_device(scene)
    b = R.Batch(10_000, cams, group=2, pair_capacity=1000)
    b.render(R.scene_struct(sd), R.camera_array(cams), "quadbox", bg=(0.1, 0.2, 0.3))
    torch.cuda.synchronize()
    with pytest.raises(N.QbCapacityError):
        b.check()
    # every overflowing camera rendered as background, nothing read out of bounds
    img = b.image(0).cpu().numpy()
    np.testing.assert_allclose(img[0], 0.1, atol=1e-7)
    b.check()  # flags were cleared


def test_batch_at_the_benchmark_resolutions_matches_frames():
    """Sixteen cameras of the batched benchmark's resolutions (800x800,
    1264x832, 1600x900, 1920x1080, four of each) around a 200k-Gaussian
    scene in one group, 81,872 tiles in the render's global queue; every
    camera's tile sort takes two digit passes.  Every camera's image is
    bit-identical to its single-frame render (whose keys the frame tests hold
    bit-exact to the oracle)."""
    import torch
    from paper_2605_04844_gb300 import rasterizer as R
    sizes = [(800, 800), (1264, 832), (1600, 900), (1920, 1080)] * 4
    scene, cams = problem(n=200_000, seed=57, sizes=sizes)
    sd = to_device(scene)
    b = R.calibrated_batch(sd, cams, group=16)
    b.render(R.scene_struct(sd), R.camera_array(cams), "quadbox")
    torch.cuda.synchronize()
    pairs = b.check()
    assert len(pairs) == 16 and sum(pairs) > 5_000_000
    tiles = sum(((w + 15) // 16) * ((h + 15) // 16) for w, h in sizes)
    assert tiles == 81_872
    ref = frame_images(sd, cams, None)
    for k in range(len(cams)):
        np.testing.assert_array_equal(b.image(k).cpu().numpy(), ref[k])
