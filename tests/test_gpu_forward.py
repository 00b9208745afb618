"""GPU parity of the forward path (stages S1-S10) against the FP64 oracle,
called through the C ABI."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_04844_gb300 import synth

from gpu_util import assert_projection_parity, f64, image_parity, oracle_keys_from_gpu_boxes, run_forward, to_device

pytestmark = pytest.mark.gpu

MODES = [("aabb3s", O.AABB3S), ("quadbox", O.QUADBOX), ("adr", O.ADR), ("quadbox_naive", O.QUADBOX_NAIVE),
         ("dualbox", O.DUALBOX)]


def c1_small(n=10_000, W=256, H=256):
    return synth.config1(n, W, H)


def c2_small(n=20_000, W=200, H=120, deg=3):
    cam = synth.pinhole(W, H)
    return synth.scene_blobs(n, 1102, cam, deg=deg), cam


def rel_err(a, b, scale):
    return np.abs(a - b) / scale


@pytest.mark.parametrize("maker", [c1_small, c2_small])
def test_preprocess_parity(maker):
    scene, cam = maker()
    img, fr, A = run_forward(scene, cam, "quadbox")
    assert_projection_parity(A, scene, cam)
    ref = O.project(f64(scene), cam)
    m = ((A["meta"] & 1) != 0) & (ref[:, O.F_VALID] != 0)
    r = ref[m]
    # 3-sigma radius: an integer ceil, equal except where 3 sqrt(lambda_max)
    # lies within float32 rounding of an integer (then off by one at most)
    s11, s12_, s22 = r[:, O.F_S11], r[:, O.F_S12], r[:, O.F_S22]
    mid = 0.5 * (s11 + s22)
    w3 = 3.0 * np.sqrt(mid + np.sqrt(np.maximum(0.1, mid * mid - (s11 * s22 - s12_ * s12_))))
    differ = A["r3"][m] != r[:, O.F_R3]
    assert np.all(np.abs(w3[differ] - np.round(w3[differ])) <= 1e-5 * w3[differ])
    assert np.all(np.abs(A["r3"][m] - r[:, O.F_R3]) <= 1)
    orient_g = ((A["meta"][m] >> 1) & 1)
    s12 = r[:, O.F_S12]
    ok = (orient_g == (s12 >= 0)) | (np.abs(s12) < 1e-5 * np.sqrt(r[:, O.F_S11] * r[:, O.F_S22]))
    assert ok.all()


@pytest.mark.parametrize("name,mode", MODES)
@pytest.mark.parametrize("clamp", [True, False])
@pytest.mark.parametrize("sort_mode", ["depth_first", "depth_first_fused", "full_key"])
def test_keys_and_ranges_bit_exact(name, mode, clamp, sort_mode):
    scene, cam = c2_small()
    W, H = cam["width"], cam["height"]
    m = name if clamp else name + "+noclamp"
    img, fr, A = run_forward(scene, cam, m, sort_mode=sort_mode)
    o = oracle_keys_from_gpu_boxes(A, mode, clamp, W, H)
    np.testing.assert_array_equal(A["counts"].astype(np.int64), o["counts"])
    P = fr.n_pairs
    assert P == len(o["keys"])
    np.testing.assert_array_equal(A["full_keys"], o["keys"])
    np.testing.assert_array_equal(A["vals"].astype(np.uint32), o["vals"])
    np.testing.assert_array_equal(A["ranges"].astype(np.int64), o["ranges"])


@pytest.mark.parametrize("digit_bits", [8, 9, 10, 11])
@pytest.mark.parametrize("sort_mode", ["depth_first", "depth_first_fused", "full_key"])
def test_keys_bit_exact_all_digit_widths(digit_bits, sort_mode):
    scene, cam = c1_small()
    img, fr, A = run_forward(scene, cam, "quadbox", digit_bits=digit_bits, sort_mode=sort_mode)
    o = oracle_keys_from_gpu_boxes(A, O.QUADBOX, True, cam["width"], cam["height"])
    np.testing.assert_array_equal(A["full_keys"], o["keys"])
    np.testing.assert_array_equal(A["vals"].astype(np.uint32), o["vals"])


def test_depth_order_is_stable_depth_sort():
    scene, cam = c2_small()
    img, fr, A = run_forward(scene, cam, "quadbox")
    d = A["rgbd"][:, 3].astype(np.float32).view(np.uint32) & np.uint32(0x7FFFFFFF)
    key = np.where(A["counts"] > 0, d, np.uint32(0x7FFFFFFF))
    np.testing.assert_array_equal(A["depth_order"].view(np.uint32), np.argsort(key, kind="stable").astype(np.uint32))


def test_sort_modes_identical_images():
    scene, cam = c2_small()
    a = run_forward(scene, cam, "quadbox", sort_mode="depth_first")
    for other in ("depth_first_fused", "full_key"):
        b = run_forward(scene, cam, "quadbox", sort_mode=other)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[2]["vals"], b[2]["vals"])
        np.testing.assert_array_equal(a[2]["ranges"], b[2]["ranges"])


@pytest.mark.parametrize("mode", ["quadbox", "aabb3s"])
def test_grid_beyond_the_tile_histogram_takes_the_fused_emit(mode):
    """A 3840x2160 frame has 32400 tiles, more than the shared-memory tile
    histogram holds, so the emit performs the first digit pass with per-tile
    counts from the preprocess: keys, values and ranges bit-exact against the
    oracle's traversal of the GPU machines, several million pairs."""
    cam = synth.pinhole(3840, 2160)
    scene = synth.scene_blobs(300_000, 1077, cam, deg=0)
    img, fr, A = run_forward(scene, cam, mode)
    assert fr.frame.tiles_x * fr.frame.tiles_y > 24576 and fr.n_pairs > 1_000_000
    o = oracle_keys_from_gpu_boxes(A, O.QUADBOX if mode == "quadbox" else O.AABB3S, True, 3840, 2160)
    np.testing.assert_array_equal(A["full_keys"], o["keys"])
    np.testing.assert_array_equal(A["vals"].astype(np.uint32), o["vals"])
    np.testing.assert_array_equal(A["ranges"].astype(np.int64), o["ranges"])


def test_quadbox_fewer_pairs_than_aabb():
    scene, cam = c2_small()
    P = {name: run_forward(scene, cam, name)[1].n_pairs for name in ("aabb3s", "adr", "quadbox", "dualbox")}
    assert P["quadbox"] < P["adr"] < P["aabb3s"]
    assert P["dualbox"] <= P["quadbox"]


@pytest.mark.parametrize("sort_mode", ["depth_first", "depth_first_fused", "full_key"])
def test_ragged_image_and_tiny_scenes(sort_mode):
    # image sizes that are not multiples of 16, a one-pixel image, one Gaussian, no Gaussian
    for (W, H, n) in [(37, 23, 300), (1, 1, 5), (17, 16, 1), (64, 48, 0)]:
        cam = synth.pinhole(W, H)
        scene = synth.scene_uniform(n, 5 + W, cam, depth=(1.0, 4.0), logscale=(-1.5, 0.5))
        img, fr, A = run_forward(scene, cam, "quadbox", bg=(0.2, 0.3, 0.4), sort_mode=sort_mode)
        ref = O.image(f64(scene), cam, O.QUADBOX, bg=(0.2, 0.3, 0.4))
        ok, st = image_parity(img, ref)
        assert ok, (W, H, n, st)
        if n:
            o = oracle_keys_from_gpu_boxes(A, O.QUADBOX, True, W, H)
            np.testing.assert_array_equal(A["full_keys"], o["keys"])


@pytest.mark.parametrize("sort_mode", ["depth_first", "depth_first_fused"])
def test_huge_gaussian_covering_everything(sort_mode):
    cam = synth.pinhole(300, 200)
    scene = synth.scene_uniform(50, 9, cam, depth=(1.0, 3.0), logscale=(-3.0, 0.3))
    scene["scales"][0] = [1.5, -0.5, 0.2]  # several hundred pixels
    scene["opacities"][0] = 3.0
    img, fr, A = run_forward(scene, cam, "quadbox", sort_mode=sort_mode)
    o = oracle_keys_from_gpu_boxes(A, O.QUADBOX, True, 300, 200)
    np.testing.assert_array_equal(A["full_keys"], o["keys"])
    ok, st = image_parity(img, O.image(f64(scene), cam, O.QUADBOX))
    assert ok, st


@pytest.mark.parametrize("sort_mode", ["depth_first", "depth_first_fused"])
def test_capacity_overflow_is_reported_not_written(sort_mode):
    import torch
    from paper_2605_04844_gb300 import _native as N
    from paper_2605_04844_gb300 import rasterizer as R
    scene, cam = c1_small(2000, 128, 128)
    sd = to_device(scene)
    fr = R.Frame(2000, 128, 128, pair_capacity=64)
    fr.set_tuning(sort_mode=sort_mode.replace("_fused", ""), emit_fused=sort_mode.endswith("_fused"))
    s, c = R.scene_struct(sd), R.camera_struct(cam)
    fr.preprocess(s, c, "quadbox")
    with pytest.raises(N.QbCapacityError):
        fr.bin_emit(sync=True)
    # device-side path: no host sync, the emit writes nothing and flags it
    keys_before = fr.arrays(n_pairs=64)["keys"].clone()
    fr.preprocess(s, c, "quadbox")
    fr.bin_emit(sync=False)
    torch.cuda.synchronize()
    with pytest.raises(N.QbCapacityError):
        fr.check()
    assert torch.equal(fr.arrays(n_pairs=64)["keys"], keys_before)
    fr.check()  # flags were cleared
    # and the render after an overflowed, unsynchronised emit sees empty tiles
    fr.sort()
    img = fr.render((0.25, 0.5, 0.75))
    torch.cuda.synchronize()
    assert torch.equal(img[0], torch.full_like(img[0], 0.25))
    # the forward helper grows the buffer and succeeds
    img, fr2 = R.forward(sd, cam, "quadbox", capacity=64)
    assert fr2.pair_capacity >= fr2.n_pairs


@pytest.mark.parametrize("sort_mode", ["depth_first", "depth_first_fused"])
def test_unsynchronised_pipeline_matches_synchronised(sort_mode):
    """qb_bin_emit without the host read-back (capacity-sized sort) gives the
    same image and keys."""
    import torch
    from paper_2605_04844_gb300 import rasterizer as R
    scene, cam = c2_small()
    img_a, fr_a, A = run_forward(scene, cam, "quadbox")
    sd = to_device(scene)
    fr = R.Frame(len(scene["opacities"]), cam["width"], cam["height"], pair_capacity=fr_a.n_pairs + 70000)
    fr.set_tuning(sort_mode=sort_mode.replace("_fused", ""), emit_fused=sort_mode.endswith("_fused"))
    fr.preprocess(R.scene_struct(sd), R.camera_struct(cam), "quadbox")
    fr.bin_emit(sync=False)
    fr.sort()
    img_b = fr.render(None)
    torch.cuda.synchronize()
    fr.check()
    np.testing.assert_array_equal(img_b.cpu().numpy(), img_a)
    B = fr.arrays(n_pairs=fr_a.n_pairs)
    np.testing.assert_array_equal(B["vals"].cpu().numpy(), A["vals"])
    np.testing.assert_array_equal(B["tile_keys"].cpu().numpy(), A["tile_keys"])


def test_invalid_arguments_rejected():
    from paper_2605_04844_gb300 import _native as N
    from paper_2605_04844_gb300 import rasterizer as R
    scene, cam = c1_small(100, 64, 64)
    sd = to_device(scene)
    fr = R.Frame(100, 64, 64, pair_capacity=10000)
    with pytest.raises(N.QbError):
        fr.sort()  # before preprocess / emit
    bad = dict(cam)
    bad["width"] = 65
    with pytest.raises(N.QbError):
        fr.preprocess(R.scene_struct(sd), R.camera_struct(bad), "quadbox")
    with pytest.raises(N.QbError):
        fr.preprocess(R.scene_struct(sd), R.camera_struct(cam), 17)


def test_tile_keys_accessor_is_bounded_by_its_output():
    """qb_frame_tile_keys writes only the positions its output holds."""
    import torch
    from paper_2605_04844_gb300 import _native as N
    scene, cam = c1_small(2000, 128, 128)
    _, fr, A = run_forward(scene, cam, "quadbox")
    buf = torch.full((16,), -7, dtype=torch.int32, device="cuda")
    N.qb_frame_tile_keys(fr.frame, buf[:10])
    torch.cuda.synchronize()
    got = buf.cpu().numpy()
    np.testing.assert_array_equal(got[:10], A["tile_keys"][:10])
    assert (got[10:] == -7).all()


def test_counted_render_is_the_same_render_and_counts_its_work():
    """qb_render_fwd_counted (measurement only) writes the same image and
    per-pixel state as qb_render_fwd, the per-pixel evaluation counts (n_eval,
    which only it writes) summing to its first count, and counts power-test
    passes between the pixels' contributors and their evaluations."""
    import torch
    from paper_2605_04844_gb300 import _native as N
    scene, cam = c2_small()
    img, fr, A = run_forward(scene, cam, "quadbox", bg=(0.2, 0.1, 0.0))
    out = torch.empty_like(torch.from_numpy(img)).cuda()
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda")
    N.qb_render_fwd_counted(fr.frame, (0.2, 0.1, 0.0), out, cnt)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), img)
    B = {k: v.cpu().numpy() for k, v in fr.arrays().items()}
    np.testing.assert_array_equal(B["n_contrib"], A["n_contrib"])
    np.testing.assert_array_equal(B["t_final"], A["t_final"])
    n_eval, n_pass = (int(x) for x in cnt.cpu().tolist())
    assert n_eval == int(B["n_eval"].astype(np.int64).sum())
    # a pixel evaluates at least up to its last contributor, at most its tile's list
    assert np.all(B["n_eval"] >= B["n_contrib"])
    # every contributing entry passed the power test; far from all evaluated ones did
    assert n_pass <= n_eval
    assert n_pass >= int((A["n_contrib"] > 0).sum())


@pytest.mark.parametrize("maker", [c2_small, lambda: c1_small(n=3000, W=250, H=190)])
def test_tile_orders_file_every_tile_once_by_its_work(maker):
    """The render files every tile once into the render's order (by the work
    estimate) and once into the backward's (64 buckets of 16 entries, heaviest
    first); the backward's bucket of a tile follows from its pixels' largest
    n_contrib, exactly."""
    scene, cam = maker()
    img, fr, A = run_forward(scene, cam, "quadbox")
    B = {k: v.cpu().numpy() for k, v in fr.arrays().items()}
    tiles = fr.frame.tiles_x * fr.frame.tiles_y
    cnt, lists = B["order_counts"].astype(np.int64), B["order_lists"]
    for o in range(2):
        assert int(cnt[o].sum()) == tiles
        filed = np.concatenate([lists[o, j, :cnt[o, j]] for j in range(64)])
        np.testing.assert_array_equal(np.sort(filed), np.arange(tiles))
    H, W = B["n_contrib"].shape
    tx, ty = fr.frame.tiles_x, fr.frame.tiles_y
    nc = np.zeros((ty * 16, tx * 16), np.int64)
    nc[:H, :W] = B["n_contrib"]
    work = nc.reshape(ty, 16, tx, 16).max(axis=(1, 3)).reshape(-1)
    want = 63 - np.minimum(work // 16, 63)
    got = np.empty(tiles, np.int64)
    for j in range(64):
        got[lists[1, j, :cnt[1, j]]] = j
    np.testing.assert_array_equal(got, want)
