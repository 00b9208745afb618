"""The bounded spin-waits of the decoupled look-back (Sec. 2's SortPairs as
a onesweep radix sort): a wait that nothing satisfies must end with the
TIMEOUT status, with every kernel returned and the frame usable afterwards.

The frame's test-only word (qb_frame_arrays.err_flags[1]) makes the second
block of the last tile-sort pass find its predecessor unpublished and give up
after a few polls.  No GPU fault is involved: the wait is an ordinary bounded
loop, and the pass's writes stay inside the value buffer."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2605_04844_gb300 import synth
from gpu_util import oracle_keys_from_gpu_boxes, to_device

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("emit_fused", [False, True])
@pytest.mark.parametrize("size", [(256, 256), (1920, 1080)])
def test_lookback_wait_runs_out_reports_timeout_and_recovers(size, emit_fused):
    import torch
    from paper_2605_04844_gb300 import _native as N
    from paper_2605_04844_gb300 import rasterizer as R
    W, H = size
    cam = synth.pinhole(W, H)
    scene = synth.scene_blobs(20_000, 606, cam, deg=0)
    sd = to_device(scene)
    s, c = R.scene_struct(sd), R.camera_struct(cam)
    _, ref = R.forward(sd, cam, "quadbox", emit_fused=emit_fused)
    fr = R.Frame(20_000, W, H, pair_capacity=ref.n_pairs + 4096)
    fr.set_tuning(digit_bits=8, emit_fused=emit_fused)
    flags = fr.arrays(n_pairs=0)["err_flags"]
    assert int(flags[1].item()) == 0  # zero after qb_frame_init
    flags[1] = 64  # the stalled block gives up after 64 polls
    t0 = time.time()
    fr.preprocess(s, c, "quadbox")
    fr.bin_emit(sync=False)
    fr.sort()
    torch.cuda.synchronize()  # every kernel has returned
    assert time.time() - t0 < 30.0
    with pytest.raises(N.QbError) as ei:
        fr.check()
    assert ei.value.status == N.QB_ERR_TIMEOUT
    assert "iteration limit" in str(ei.value)
    fr.check()  # the flag was cleared with the report

    # with the test word back at zero the same frame renders correctly
    flags[1] = 0
    img, fr2 = R.forward(sd, cam, "quadbox", frame=fr, emit_fused=emit_fused)
    torch.cuda.synchronize()
    fr2.check()
    A = {k: v.cpu().numpy() for k, v in fr2.arrays().items()}
    o = oracle_keys_from_gpu_boxes(A, O.QUADBOX, True, W, H)
    np.testing.assert_array_equal(A["vals"].astype(np.uint32), o["vals"])
    np.testing.assert_array_equal(A["ranges"].astype(np.int64), o["ranges"])
    img_ref = R.forward(sd, cam, "quadbox", emit_fused=emit_fused)[0]
    assert torch.equal(img, img_ref)
