"""ctypes binding of libquadbox (include/quadbox.h).

Argument marshalling only: every step of the rasteriser runs in the CUDA
library.  Functions keep the C names; tensors are passed as device pointers,
streams as ``torch.cuda.Stream.cuda_stream`` handles.  If the library is
missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

c_f = ctypes.c_float
c_i32 = ctypes.c_int32
c_u64 = ctypes.c_uint64
c_vp = ctypes.c_void_p
c_size = ctypes.c_size_t

QB_OK, QB_ERR_INVALID_ARG, QB_ERR_CUDA, QB_ERR_CAPACITY, QB_ERR_TIMEOUT, QB_ERR_STATE = range(6)
QB_BIN_AABB3S, QB_BIN_QUADBOX, QB_BIN_ADR, QB_BIN_QUADBOX_NAIVE, QB_BIN_DUALBOX = range(5)
QB_BIN_NO_CLAMP = 0x100
QB_SORT_DEPTH_FIRST, QB_SORT_FULL_KEY = 0, 1
MODE_NAMES = {"aabb3s": 0, "quadbox": 1, "adr": 2, "quadbox_naive": 3, "dualbox": 4}
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "CUDA", 3: "CAPACITY", 4: "TIMEOUT", 5: "STATE"}


class QbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class QbCapacityError(QbError):
    pass


class QbCamera(ctypes.Structure):
    _fields_ = [("viewmat", c_f * 16), ("fx", c_f), ("fy", c_f), ("cx", c_f), ("cy", c_f),
                ("tan_fovx", c_f), ("tan_fovy", c_f), ("campos", c_f * 3), ("width", c_i32),
                ("height", c_i32), ("znear", c_f)]


class QbScene(ctypes.Structure):
    _fields_ = [("means", c_vp), ("scales", c_vp), ("quats", c_vp), ("opacities", c_vp), ("sh", c_vp),
                ("n", c_i32), ("sh_degree", c_i32), ("params_raw", c_i32)]


class QbSceneGrads(ctypes.Structure):
    _fields_ = [("means", c_vp), ("scales", c_vp), ("quats", c_vp), ("opacities", c_vp), ("sh", c_vp)]


class QbFrame(ctypes.Structure):
    _fields_ = [("n", c_i32), ("width", c_i32), ("height", c_i32), ("tiles_x", c_i32), ("tiles_y", c_i32),
                ("pair_capacity", c_u64), ("workspace", c_vp), ("workspace_bytes", c_size),
                ("bin_mode", c_i32), ("sh_degree", c_i32), ("key_bits", c_i32), ("stage", c_i32),
                ("n_pairs", c_u64), ("sort_digit_bits", c_i32), ("render_batch", c_i32),
                ("sorted_in_alt", c_i32), ("sort_mode", c_i32), ("depth_in_alt", c_i32), ("emit_fused", c_i32),
                ("reserved", c_i32 * 3)]


QB_MAX_CAMERAS = 256
QB_GROUP_MAX = 16


class QbTune(ctypes.Structure):
    _fields_ = [("tiles_per_fetch", c_i32), ("render_batch", c_i32), ("sort_digit_bits", c_i32),
                ("blocks_per_sm", c_i32)]


class QbBatch(ctypes.Structure):
    _fields_ = [("n", c_i32), ("n_cams", c_i32), ("group", c_i32), ("n_groups", c_i32), ("pair_capacity", c_u64),
                ("workspace", c_vp), ("workspace_bytes", c_size), ("widths", c_i32 * QB_MAX_CAMERAS),
                ("heights", c_i32 * QB_MAX_CAMERAS), ("image_offset", c_u64 * QB_MAX_CAMERAS),
                ("total_floats", c_u64), ("sh_degree", c_i32), ("bin_mode", c_i32), ("stage", c_i32),
                ("sorted_tile_bits", c_i32), ("reserved", c_i32 * 8)]


class QbFrameArrays(ctypes.Structure):
    _fields_ = [(name, c_vp) for name in ("xy", "conic_o", "rgbd", "box", "r3", "meta", "counts", "offsets",
                                          "keys", "tile_keys", "vals", "depth_order", "ranges", "t_final",
                                          "n_contrib", "n_eval", "n_pairs", "err_flags", "order_counts",
                                          "order_lists")]


_lib = None

# (name, restype, argtypes)
_SIGS = [
    ("qb_last_error", ctypes.c_char_p, []),
    ("qb_version", ctypes.c_char_p, []),
    ("qb_kernel_launches", c_u64, []),
    ("qb_set_launch_hook", None, [c_vp, c_vp]),
    ("qb_frame_workspace_bytes", c_size, [c_i32, c_i32, c_i32, c_u64]),
    ("qb_frame_init", c_i32, [ctypes.POINTER(QbFrame), c_i32, c_i32, c_i32, c_u64, c_vp, c_size, c_vp]),
    ("qb_frame_arrays_get", c_i32, [ctypes.POINTER(QbFrame), ctypes.POINTER(QbFrameArrays)]),
    ("qb_frame_check", c_i32, [ctypes.POINTER(QbFrame), c_vp]),
    ("qb_frame_tile_keys", c_i32, [ctypes.POINTER(QbFrame), c_vp, c_u64, c_vp]),
    ("qb_preprocess", c_i32, [ctypes.POINTER(QbFrame), ctypes.POINTER(QbScene), ctypes.POINTER(QbCamera),
                              c_i32, c_vp]),
    ("qb_bin_emit", c_i32, [ctypes.POINTER(QbFrame), ctypes.POINTER(c_u64), c_vp]),
    ("qb_sort", c_i32, [ctypes.POINTER(QbFrame), c_vp]),
    ("qb_render_fwd", c_i32, [ctypes.POINTER(QbFrame), ctypes.POINTER(c_f), c_vp, c_vp]),
    ("qb_render_fwd_counted", c_i32, [ctypes.POINTER(QbFrame), ctypes.POINTER(c_f), c_vp, c_vp, c_vp]),
    ("qb_render_bwd", c_i32, [ctypes.POINTER(QbFrame), ctypes.POINTER(QbScene), ctypes.POINTER(QbCamera),
                              ctypes.POINTER(c_f), c_vp, ctypes.POINTER(QbSceneGrads), c_vp, c_vp]),
    ("qb_l1_loss_grad", c_i32, [c_vp, c_vp, c_vp, c_u64, ctypes.c_float, c_vp, c_vp]),
    ("qb_adam_step", c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                             ctypes.c_float, c_i32, c_vp]),
    ("qb_sort_scratch_bytes", c_size, [c_u64, c_i32, c_i32]),
    ("qb_sort_pairs", c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, c_i32, c_i32, c_vp, c_size,
                              ctypes.POINTER(c_i32), c_vp]),
    ("qb_batch_workspace_bytes", c_size, [c_i32, c_i32, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32), c_i32, c_u64]),
    ("qb_batch_init", c_i32, [ctypes.POINTER(QbBatch), c_i32, c_i32, ctypes.POINTER(c_i32), ctypes.POINTER(c_i32),
                              c_i32, c_u64, c_vp, c_size, c_vp]),
    ("qb_render_batch", c_i32, [ctypes.POINTER(QbBatch), ctypes.POINTER(QbScene), ctypes.POINTER(QbCamera), c_i32,
                                ctypes.POINTER(QbTune), ctypes.POINTER(c_f), c_vp, c_vp]),
    ("qb_render_batch_bwd", c_i32, [ctypes.POINTER(QbBatch), ctypes.POINTER(QbScene), ctypes.POINTER(QbCamera),
                                    ctypes.POINTER(c_f), c_vp, ctypes.POINTER(QbSceneGrads), c_vp]),
    ("qb_batch_check", c_i32, [ctypes.POINTER(QbBatch), ctypes.POINTER(c_u64), c_vp]),
    ("qb_batch_release", c_i32, [ctypes.POINTER(QbBatch)]),
    ("qb_sort_pairs_noalloc_max_scratch", c_size, []),
    ("qb_sort_pairs_noalloc", c_i32, [c_vp, c_vp, c_vp, c_vp, c_u64, c_i32, c_i32, ctypes.POINTER(c_i32), c_vp]),
]

# Every symbol include/quadbox.h declares (checked by the CPU test suite).
EXPORTED = [s[0] for s in _SIGS]


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libquadbox.so (building it first if allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB_PATH):
        if not build_if_missing:
            raise RuntimeError(f"libquadbox not built: {_build.LIB_PATH} is missing")
        _build.build()
    lib = ctypes.CDLL(_build.LIB_PATH)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int):
    if status != QB_OK:
        msg = load().qb_last_error().decode()
        if status == QB_ERR_CAPACITY:
            raise QbCapacityError(status, msg)
        raise QbError(status, msg)


def stream_handle(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


# ---------------------------------------------------------------------------
# Thin wrappers with the C names
# ---------------------------------------------------------------------------

def qb_frame_workspace_bytes(n, width, height, pair_capacity) -> int:
    return int(load().qb_frame_workspace_bytes(n, width, height, pair_capacity))


def qb_frame_init(frame: QbFrame, n, width, height, pair_capacity, workspace, stream=None):
    check(load().qb_frame_init(ctypes.byref(frame), n, width, height, pair_capacity, ptr(workspace),
                               workspace.numel() * workspace.element_size(), stream_handle(stream)))


def qb_frame_arrays_get(frame: QbFrame) -> QbFrameArrays:
    out = QbFrameArrays()
    check(load().qb_frame_arrays_get(ctypes.byref(frame), ctypes.byref(out)))
    return out


def qb_frame_check(frame: QbFrame, stream=None):
    check(load().qb_frame_check(ctypes.byref(frame), stream_handle(stream)))


def qb_kernel_launches() -> int:
    return int(load().qb_kernel_launches())


LAUNCH_HOOK = ctypes.CFUNCTYPE(None, ctypes.c_char_p, ctypes.c_void_p, ctypes.c_void_p)
_hook_ref = None


def qb_set_launch_hook(fn):
    """fn(kernel: str, stream_handle: int) or None; called before each launch."""
    global _hook_ref
    if fn is None:
        load().qb_set_launch_hook(None, None)
        _hook_ref = None
        return
    _hook_ref = LAUNCH_HOOK(lambda name, stream, user: fn(name.decode(), stream or 0))
    load().qb_set_launch_hook(ctypes.cast(_hook_ref, c_vp), None)


def qb_frame_tile_keys(frame: QbFrame, out, stream=None):
    """Fills the device uint32/int32 tensor `out` (its length bounds the writes)."""
    check(load().qb_frame_tile_keys(ctypes.byref(frame), ptr(out), out.numel(), stream_handle(stream)))


def qb_preprocess(frame: QbFrame, scene: QbScene, camera: QbCamera, mode: int, stream=None):
    check(load().qb_preprocess(ctypes.byref(frame), ctypes.byref(scene), ctypes.byref(camera), mode,
                               stream_handle(stream)))


def qb_bin_emit(frame: QbFrame, sync: bool = True, stream=None):
    """Returns P when sync, else None."""
    if sync:
        P = c_u64(0)
        check(load().qb_bin_emit(ctypes.byref(frame), ctypes.byref(P), stream_handle(stream)))
        return int(P.value)
    check(load().qb_bin_emit(ctypes.byref(frame), None, stream_handle(stream)))
    return None


def qb_sort(frame: QbFrame, stream=None):
    check(load().qb_sort(ctypes.byref(frame), stream_handle(stream)))


def _bg(bg):
    return (c_f * 3)(*(bg if bg is not None else (0.0, 0.0, 0.0)))


def qb_render_fwd(frame: QbFrame, bg, img, stream=None):
    check(load().qb_render_fwd(ctypes.byref(frame), _bg(bg), ptr(img), stream_handle(stream)))


def qb_render_fwd_counted(frame: QbFrame, bg, img, counts, stream=None):
    """counts: device int64 tensor of 2 entries, accumulated (zero it first)."""
    check(load().qb_render_fwd_counted(ctypes.byref(frame), _bg(bg), ptr(img), ptr(counts), stream_handle(stream)))


def qb_render_bwd(frame: QbFrame, scene: QbScene, camera: QbCamera, bg, dL_dimg, grads: QbSceneGrads,
                  grad_screen=None, stream=None):
    check(load().qb_render_bwd(ctypes.byref(frame), ctypes.byref(scene), ctypes.byref(camera), _bg(bg),
                               ptr(dL_dimg), ctypes.byref(grads), ptr(grad_screen), stream_handle(stream)))


def qb_l1_loss_grad(img, target, dL, scale, loss=None, stream=None):
    check(load().qb_l1_loss_grad(ptr(img), ptr(target), ptr(dL), img.numel(), scale, ptr(loss),
                                 stream_handle(stream)))


def qb_adam_step(param, grad, m, v, lr, beta1, beta2, eps, step, stream=None):
    check(load().qb_adam_step(ptr(param), ptr(grad), ptr(m), ptr(v), param.numel(), lr, beta1, beta2, eps, step,
                              stream_handle(stream)))


def qb_sort_scratch_bytes(n, end_bit, digit_bits) -> int:
    return int(load().qb_sort_scratch_bytes(n, end_bit, digit_bits))


def qb_sort_pairs(keys, vals, keys_alt, vals_alt, n, end_bit, digit_bits, scratch, stream=None) -> bool:
    """Returns True when the result is in the *_alt buffers."""
    alt = c_i32(0)
    check(load().qb_sort_pairs(ptr(keys), ptr(vals), ptr(keys_alt), ptr(vals_alt), n, end_bit, digit_bits,
                               ptr(scratch), scratch.numel() * scratch.element_size(), ctypes.byref(alt),
                               stream_handle(stream)))
    return bool(alt.value)


def qb_sort_pairs_noalloc(keys, vals, keys_alt, vals_alt, n, end_bit, digit_bits, stream=None) -> bool:
    """Sort with the library's static scratch array (no allocation).
    Returns True when the result is in the *_alt buffers."""
    alt = c_i32(0)
    check(load().qb_sort_pairs_noalloc(ptr(keys), ptr(vals), ptr(keys_alt), ptr(vals_alt), n, end_bit, digit_bits,
                                       ctypes.byref(alt), stream_handle(stream)))
    return bool(alt.value)


# ---------------------------------------------------------------------------
# Batched multi-camera rendering
# ---------------------------------------------------------------------------

def _int_array(vals):
    arr = (c_i32 * len(vals))(*[int(v) for v in vals])
    return arr


def qb_batch_workspace_bytes(n, widths, heights, group, pair_capacity) -> int:
    return int(load().qb_batch_workspace_bytes(n, len(widths), _int_array(widths), _int_array(heights), group,
                                               pair_capacity))


def qb_batch_init(batch: QbBatch, n, widths, heights, group, pair_capacity, workspace, stream=None):
    check(load().qb_batch_init(ctypes.byref(batch), n, len(widths), _int_array(widths), _int_array(heights), group,
                               pair_capacity, ptr(workspace), workspace.numel() * workspace.element_size(),
                               stream_handle(stream)))


def qb_render_batch(batch: QbBatch, scene: QbScene, cams_array, mode: int, tune: QbTune, bg, images, stream=None):
    check(load().qb_render_batch(ctypes.byref(batch), ctypes.byref(scene), cams_array, mode,
                                 ctypes.byref(tune) if tune is not None else None, _bg(bg), ptr(images),
                                 stream_handle(stream)))


def qb_render_batch_bwd(batch: QbBatch, scene: QbScene, cams_array, bg, dL_dimages, grads: QbSceneGrads,
                        stream=None):
    check(load().qb_render_batch_bwd(ctypes.byref(batch), ctypes.byref(scene), cams_array, _bg(bg),
                                     ptr(dL_dimages), ctypes.byref(grads), stream_handle(stream)))


def qb_batch_release(batch: QbBatch):
    check(load().qb_batch_release(ctypes.byref(batch)))


def qb_batch_check(batch: QbBatch, stream=None):
    """Returns the pairs of every camera (synchronises)."""
    out = (c_u64 * max(1, batch.n_cams))()
    check(load().qb_batch_check(ctypes.byref(batch), out, stream_handle(stream)))
    return [int(out[i]) for i in range(batch.n_cams)]
