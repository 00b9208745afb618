"""PyTorch-facing layer over libquadbox: frames, the forward pipeline and a
``torch.autograd.Function``.  PyTorch provides device memory and streams;
every stage runs in the library's CUDA kernels.

Pipeline (Sec. 2 of the QuadBox paper): qb_preprocess -> qb_bin_emit ->
qb_sort -> qb_render_fwd; backward: qb_render_bwd.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _native as N

MODES = N.MODE_NAMES


def mode_id(mode) -> int:
    if isinstance(mode, str):
        m = mode.lower()
        no_clamp = m.endswith("+noclamp")
        m = m.replace("+noclamp", "")
        return MODES[m] | (N.QB_BIN_NO_CLAMP if no_clamp else 0)
    return int(mode)


def camera_struct(cam) -> N.QbCamera:
    c = N.QbCamera()
    vm = [float(v) for v in torch.as_tensor(cam["viewmat"], dtype=torch.float64).reshape(16).tolist()]
    for i in range(16):
        c.viewmat[i] = vm[i]
    c.fx, c.fy, c.cx, c.cy = float(cam["fx"]), float(cam["fy"]), float(cam["cx"]), float(cam["cy"])
    c.tan_fovx, c.tan_fovy = float(cam["tan_fovx"]), float(cam["tan_fovy"])
    cp = [float(v) for v in torch.as_tensor(cam["campos"], dtype=torch.float64).reshape(3).tolist()]
    for i in range(3):
        c.campos[i] = cp[i]
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.znear = float(cam.get("znear", 0.2))
    return c


def _check_tensor(t, name, shape_tail, n):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    if t.shape[0] != n or tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected ({n}, {shape_tail})")


def scene_struct(scene) -> N.QbScene:
    """scene: dict of CUDA float32 tensors means [n,3], scales [n,3], quats [n,4],
    opacities [n], sh [n,K,3], plus sh_degree and raw."""
    n = int(scene["means"].shape[0])
    deg = int(scene["sh_degree"])
    K = (deg + 1) ** 2
    _check_tensor(scene["means"], "means", (3,), n)
    _check_tensor(scene["scales"], "scales", (3,), n)
    _check_tensor(scene["quats"], "quats", (4,), n)
    _check_tensor(scene["opacities"], "opacities", (), n)
    _check_tensor(scene["sh"], "sh", (K, 3), n)
    s = N.QbScene()
    s.means, s.scales, s.quats = scene["means"].data_ptr(), scene["scales"].data_ptr(), scene["quats"].data_ptr()
    s.opacities, s.sh = scene["opacities"].data_ptr(), scene["sh"].data_ptr()
    s.n, s.sh_degree, s.params_raw = n, deg, int(scene.get("raw", 1))
    return s


SORT_MODES = {"depth_first": 0, "full_key": 1}


class Frame:
    """One rasterisation frame: a workspace plus the qb_frame handle."""

    def __init__(self, n, width, height, pair_capacity, device="cuda", stream=None):
        self.n, self.width, self.height = int(n), int(width), int(height)
        self.pair_capacity = int(pair_capacity)
        nbytes = N.qb_frame_workspace_bytes(self.n, self.width, self.height, self.pair_capacity)
        if nbytes == 0:
            raise ValueError("invalid frame sizes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.workspace.data_ptr()) % 256
        self.ws = self.workspace[off:off + nbytes]
        self.frame = N.QbFrame()
        self.stream = stream
        N.qb_frame_init(self.frame, self.n, self.width, self.height, self.pair_capacity, self.ws, stream)

    # -- configuration ------------------------------------------------------
    def set_tuning(self, digit_bits=None, render_batch=None, sort_mode=None, emit_fused=None):
        if digit_bits is not None:
            self.frame.sort_digit_bits = int(digit_bits)
        if sort_mode is not None:
            self.frame.sort_mode = SORT_MODES.get(sort_mode, sort_mode)
        if render_batch is not None:
            self.frame.render_batch = int(render_batch)
        if emit_fused is not None:
            self.frame.emit_fused = int(bool(emit_fused))

    # -- stages -----------------------------------------------------------------
    def preprocess(self, scene_s: N.QbScene, cam_s: N.QbCamera, mode):
        N.qb_preprocess(self.frame, scene_s, cam_s, mode_id(mode), self.stream)

    def bin_emit(self, sync=True):
        return N.qb_bin_emit(self.frame, sync, self.stream)

    def sort(self):
        N.qb_sort(self.frame, self.stream)

    def render(self, bg=None, out=None):
        if out is None:
            out = torch.empty((3, self.height, self.width), dtype=torch.float32, device=self.ws.device)
        N.qb_render_fwd(self.frame, bg, out, self.stream)
        return out

    def check(self):
        N.qb_frame_check(self.frame, self.stream)

    @property
    def n_pairs(self):
        v = self.frame.n_pairs
        return None if v == 2 ** 64 - 1 else int(v)

    # -- inspection ----------------------------------------------------------------
    def sorted_tile_keys(self, n_pairs=None):
        """The tile id of every sorted pair (from the per-tile ranges)."""
        P = n_pairs if n_pairs is not None else (self.n_pairs or 0)
        out = torch.empty(P, dtype=torch.int32, device=self.ws.device)
        N.qb_frame_tile_keys(self.frame, out, self.stream)
        return out

    def _view(self, p, dtype, shape):
        off = p - self.ws.data_ptr()
        nbytes = int(math.prod(shape)) * torch.empty((), dtype=dtype).element_size()
        return self.ws[off:off + nbytes].view(dtype).view(*shape)

    def arrays(self, n_pairs=None):
        a = N.qb_frame_arrays_get(self.frame)
        n, H, W = self.n, self.height, self.width
        P = n_pairs if n_pairs is not None else (self.n_pairs or 0)
        tiles = self.frame.tiles_x * self.frame.tiles_y
        return {
            "xy": self._view(a.xy, torch.float32, (n, 2)),
            "conic_o": self._view(a.conic_o, torch.float32, (n, 4)),
            "rgbd": self._view(a.rgbd, torch.float32, (n, 4)),
            "box": self._view(a.box, torch.float32, (n, 4)),
            "r3": self._view(a.r3, torch.float32, (n,)),
            "meta": self._view(a.meta, torch.int32, (n,)),
            "counts": self._view(a.counts, torch.int32, (n,)),
            "offsets": self._view(a.offsets, torch.int32, (n,)),
            "keys": self._view(a.keys, torch.int64, (P,)),
            "tile_keys": self.sorted_tile_keys(P) if self.frame.stage >= 3 else self._view(a.tile_keys, torch.int32, (P,)),
            "vals": self._view(a.vals, torch.int32, (P,)),
            "depth_order": self._view(a.depth_order, torch.int32, (n,)),
            "ranges": self._view(a.ranges, torch.int32, (tiles, 2)),
            "t_final": self._view(a.t_final, torch.float32, (H, W)),
            "n_contrib": self._view(a.n_contrib, torch.int32, (H, W)),
            "n_eval": self._view(a.n_eval, torch.int32, (H, W)),
            "err_flags": self._view(a.err_flags, torch.int32, (2,)),
            "order_counts": self._view(a.order_counts, torch.int32, (2, 64)),
            "order_lists": self._view(a.order_lists, torch.int32, (2, 64, tiles)),
        }


def estimate_capacity(n, width, height):
    """A first guess at the pair capacity; the forward grows it on overflow."""
    tiles = ((width + 15) // 16) * ((height + 15) // 16)
    return int(min(2 ** 30, max(1 << 16, 8 * n, 4 * tiles)))


def forward(scene, cam, mode="quadbox", bg=None, frame: Frame | None = None, digit_bits=8, capacity=None,
            sort_mode="depth_first", emit_fused=False):
    """Full forward pass.  Returns (image [3,H,W], frame).  Grows the pair
    buffer when the tile pairs exceed it (the count is read back once)."""
    scene_s = scene_struct(scene)
    cam_s = camera_struct(cam)
    n, W, H = scene_s.n, cam_s.width, cam_s.height
    if frame is None or frame.n != n or frame.width != W or frame.height != H:
        frame = Frame(n, W, H, capacity or estimate_capacity(n, W, H))
    frame.set_tuning(digit_bits=digit_bits, sort_mode=sort_mode, emit_fused=emit_fused)
    while True:
        frame.preprocess(scene_s, cam_s, mode)
        try:
            frame.bin_emit(sync=True)
            break
        except N.QbCapacityError:
            P = _read_pairs(frame)
            frame = Frame(n, W, H, min(2 ** 30, int(P * 1.25) + 1024))
            frame.set_tuning(digit_bits=digit_bits, sort_mode=sort_mode, emit_fused=emit_fused)
    frame.sort()
    img = frame.render(bg)
    return img, frame


def _read_pairs(frame: Frame) -> int:
    a = N.qb_frame_arrays_get(frame.frame)
    return int(frame._view(a.n_pairs, torch.int64, (1,)).item())


class QuadBoxRasterize(torch.autograd.Function):
    """Differentiable rasterisation of raw Gaussian parameters.

    forward(means, log_scales, quats, opacity_logits, sh, cam, mode, bg)
    -> image [3,H,W].  The backward is libquadbox's hand-written backward
    (qb_render_bwd)."""

    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, cam, mode="quadbox", bg=None):
        deg = int(round(math.sqrt(sh.shape[1]))) - 1
        scene = {"means": means.contiguous(), "scales": scales.contiguous(), "quats": quats.contiguous(),
                 "opacities": opacities.contiguous(), "sh": sh.contiguous(), "sh_degree": deg, "raw": 1}
        img, frame = forward(scene, cam, mode, bg)
        ctx.frame = frame
        ctx.cam = cam
        ctx.bg = bg
        ctx.deg = deg
        ctx.save_for_backward(scene["means"], scene["scales"], scene["quats"], scene["opacities"], scene["sh"])
        return img

    @staticmethod
    def backward(ctx, grad_img):
        means, scales, quats, opacities, sh = ctx.saved_tensors
        scene = {"means": means, "scales": scales, "quats": quats, "opacities": opacities, "sh": sh,
                 "sh_degree": ctx.deg, "raw": 1}
        g = {k: torch.zeros_like(v) for k, v in scene.items() if isinstance(v, torch.Tensor)}
        gs = N.QbSceneGrads()
        gs.means, gs.scales, gs.quats = g["means"].data_ptr(), g["scales"].data_ptr(), g["quats"].data_ptr()
        gs.opacities, gs.sh = g["opacities"].data_ptr(), g["sh"].data_ptr()
        N.qb_render_bwd(ctx.frame.frame, scene_struct(scene), camera_struct(ctx.cam), ctx.bg,
                        grad_img.contiguous(), gs, None, ctx.frame.stream)
        return g["means"], g["scales"], g["quats"], g["opacities"], g["sh"], None, None, None


def rasterize(means, scales, quats, opacities, sh, cam, mode="quadbox", bg=None):
    return QuadBoxRasterize.apply(means, scales, quats, opacities, sh, cam, mode, bg)


def camera_array(cams):
    """A C array of qb_camera structs for the batch entry points."""
    arr = (N.QbCamera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera_struct(c)
    return arr


def tune_struct(tune=None) -> N.QbTune:
    t = N.QbTune()
    d = {"tiles_per_fetch": 2, "render_batch": 128, "sort_digit_bits": 8, "blocks_per_sm": 0}
    d.update(tune or {})
    t.tiles_per_fetch, t.render_batch = int(d["tiles_per_fetch"]), int(d["render_batch"])
    t.sort_digit_bits, t.blocks_per_sm = int(d["sort_digit_bits"]), int(d["blocks_per_sm"])
    return t


class Batch:
    """Many cameras of one scene rendered with the batched entry points.

    The preprocess runs per group of `group` cameras; `pair_capacity` bounds
    the Gaussian-tile pairs of one camera (see calibrated_batch()).  Images
    are packed in one buffer; image(k) is camera k's [3, H, W] view."""

    def __init__(self, n, cams, group=16, pair_capacity=None, device="cuda", stream=None):
        self.n = int(n)
        self.widths = [int(c["width"]) for c in cams]
        self.heights = [int(c["height"]) for c in cams]
        self.group = int(min(group, N.QB_GROUP_MAX, len(cams)))
        if pair_capacity is None:
            tiles = max(((w + 15) // 16) * ((h + 15) // 16) for w, h in zip(self.widths, self.heights))
            pair_capacity = min(2 ** 30, max(8 * self.n, 4 * tiles))
        self.pair_capacity = int(pair_capacity)
        self.device = device
        self.stream = stream
        nbytes = N.qb_batch_workspace_bytes(self.n, self.widths, self.heights, self.group, self.pair_capacity)
        if nbytes == 0:
            raise ValueError("invalid batch sizes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.workspace.data_ptr()) % 256
        self.ws = self.workspace[off:off + nbytes]
        self.batch = N.QbBatch()
        N.qb_batch_init(self.batch, self.n, self.widths, self.heights, self.group, self.pair_capacity, self.ws, stream)
        self.images = torch.empty(int(self.batch.total_floats), dtype=torch.float32, device=device)

    def __del__(self):
        # the library's side streams of this batch (the workspace is torch's)
        try:
            if self.batch.workspace:
                N.qb_batch_release(self.batch)
        except Exception:
            pass

    @property
    def n_cams(self):
        return len(self.widths)

    def image(self, k, buf=None):
        buf = self.images if buf is None else buf
        o = int(self.batch.image_offset[k])
        H, W = self.heights[k], self.widths[k]
        return buf[o:o + 3 * H * W].view(3, H, W)

    def render(self, scene_s: N.QbScene, cams_arr, mode="quadbox", tune=None, bg=None):
        N.qb_render_batch(self.batch, scene_s, cams_arr, mode_id(mode), tune_struct(tune), bg, self.images,
                          self.stream)
        return self.images

    def backward(self, scene_s: N.QbScene, cams_arr, dL_dimages, grads: N.QbSceneGrads, bg=None):
        N.qb_render_batch_bwd(self.batch, scene_s, cams_arr, bg, dL_dimages, grads, self.stream)

    def check(self):
        return N.qb_batch_check(self.batch, self.stream)


def calibrated_batch(scene, cams, mode="quadbox", group=16, headroom=1.1, tune=None):
    """A Batch whose pair capacity fits this scene and these cameras: one
    render with a generous capacity measures the pairs of every camera."""
    scene_s, cams_arr = scene_struct(scene), camera_array(cams)
    n = scene_s.n
    probe = Batch(n, cams, group, pair_capacity=None)
    while True:
        probe.render(scene_s, cams_arr, mode, tune)
        try:
            pairs = probe.check()
            break
        except N.QbCapacityError:
            cap = min(2 ** 30, probe.pair_capacity * 4)
            if cap == probe.pair_capacity:
                raise
            probe = Batch(n, cams, group, pair_capacity=cap)
    cap = min(2 ** 30, int(max(pairs) * headroom) + 4096)
    del probe
    return Batch(n, cams, group, pair_capacity=cap)


# Per-array Adam learning rates (3DGS's defaults for raw parameters; the mean's
# is for a scene of unit extent).
DEFAULT_LR = {"means": 1.6e-4, "scales": 5e-3, "quats": 1e-3, "opacities": 5e-2, "sh": 2.5e-3}


class Trainer:
    """Adam on the raw scene parameters against a target image with the L1
    loss, every step in the library's kernels: forward, loss gradient,
    backward, update.  `scene` holds the (mutable, raw) device arrays."""

    KEYS = ("means", "scales", "quats", "opacities", "sh")

    def __init__(self, scene, cam, mode="quadbox", lr=None, betas=(0.9, 0.999), eps=1e-15, bg=None, stream=None):
        self.scene, self.cam, self.mode, self.bg = scene, cam, mode, bg
        self.lr = dict(DEFAULT_LR, **(lr or {}))
        self.betas, self.eps = betas, eps
        self.stream = stream
        self.scene_s, self.cam_s = scene_struct(scene), camera_struct(cam)
        dev = scene["means"].device
        self.grads = {k: torch.zeros_like(scene[k]) for k in self.KEYS}
        self.m = {k: torch.zeros_like(scene[k]) for k in self.KEYS}
        self.v = {k: torch.zeros_like(scene[k]) for k in self.KEYS}
        self.gs = N.QbSceneGrads()
        for k in self.KEYS:
            setattr(self.gs, k, self.grads[k].data_ptr())
        H, W = cam["height"], cam["width"]
        self.img = torch.empty((3, H, W), dtype=torch.float32, device=dev)
        self.dL = torch.empty_like(self.img)
        self.loss = torch.zeros((), dtype=torch.float64, device=dev)
        _, self.frame = forward(scene, cam, mode, bg=bg)
        self.t = 0

    def step(self, target):
        """One step; returns the loss (mean absolute error) as a device scalar
        of the image before the update."""
        fr, s = self.frame, self.stream
        fr.preprocess(self.scene_s, self.cam_s, self.mode)
        try:
            fr.bin_emit(sync=True)
        except N.QbCapacityError:  # the scene moved: grow the pair buffer
            _, self.frame = forward(self.scene, self.cam, self.mode, bg=self.bg)
            fr = self.frame
            fr.preprocess(self.scene_s, self.cam_s, self.mode)
            fr.bin_emit(sync=True)
        fr.sort()
        fr.render(self.bg, self.img)
        self.loss.zero_()
        N.qb_l1_loss_grad(self.img, target, self.dL, 1.0 / self.img.numel(), self.loss, s)
        for g in self.grads.values():
            g.zero_()
        N.qb_render_bwd(fr.frame, self.scene_s, self.cam_s, self.bg, self.dL, self.gs, None, s)
        self.t += 1
        for k in self.KEYS:
            N.qb_adam_step(self.scene[k], self.grads[k], self.m[k], self.v[k], self.lr[k], self.betas[0],
                           self.betas[1], self.eps, self.t, s)
        return self.loss
