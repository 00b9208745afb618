#!/usr/bin/env python
"""Benchmark of the QuadBox tile rasteriser on one GB300 (or N replicas).

Workload: 1M Gaussians, 1920x1080, SH degree 3, clustered synthetic scene
(64 blobs + 20% background at depth 1-50, 10% anisotropic), QuadBox binning
versus the 3-sigma AABB binning on the same kernels.

A step is one pass of the rasteriser's hot path over the scene: preprocess
(projection, SH colour, QuadBox, QPass count), scan + emit, onesweep sort +
ranges, render; the fwd+bwd step adds the hand-written backward.  `value` is
the QuadBox forward frame rate summed over ranks; the AABB path, fwd+bwd
times, per-stage times and tile pairs per frame are reported beside it.

--impl reference times the FP64 CPU oracle on the host cores instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FPS fwd & fwd+bwd ms @1M Gaussians 1080p, QuadBox vs AABB; tile pairs/frame"
UNIT = "FPS"
L2_BYTES = 129 * 1024 * 1024


# ---- replicas: one process per GPU, no data-path collective -----------------
# Each rank renders its own copy of the workload; the timing collectives below
# are the only communication.  A step takes as long as the slowest rank, and
# the job's frame rate is every rank's frames over that time.

def ranks_barrier(world):
    if world > 1:
        import torch
        torch.distributed.barrier()


def max_over_ranks(x, world, device):
    """The largest x over all ranks (x itself at world size 1)."""
    if world == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_fps(ms_per_frame_max, world):
    """Frames per second of the whole job: world replicas, each one frame per
    step of the slowest rank's duration."""
    return world * 1000.0 / ms_per_frame_max


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--width", type=int, default=1920)
    ap.add_argument("--height", type=int, default=1080)
    ap.add_argument("--digit-bits", type=int, default=None)
    ap.add_argument("--sort-mode", default="depth_first", choices=["depth_first", "full_key"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the 64-camera batched comparison")
    ap.add_argument("--no-c3", action="store_true", help="skip the 3M-Gaussian zoom sweep")
    ap.add_argument("--no-c4", action="store_true", help="skip the 500k forward+backward (L1 loss) case")
    ap.add_argument("--batch-cams", type=int, default=64)
    ap.add_argument("--batch-n", type=int, default=1_000_000)
    ap.add_argument("--out", default=None, help="also write the JSON line here")
    return ap.parse_args()


# --------------------------------------------------------------------------
# clocks
# --------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2605_04844_gb300 import _native as N
    from paper_2605_04844_gb300 import rasterizer as R
    from paper_2605_04844_gb300 import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)
    scene_np, cam = synth.config2(args.n, args.width, args.height)
    W, H, n = cam["width"], cam["height"], args.n
    pinned = {k: torch.from_numpy(v).pin_memory() for k, v in scene_np.items() if isinstance(v, np.ndarray)}
    sd = {k: v.to(dev) for k, v in pinned.items()}
    sd["sh_degree"], sd["raw"] = scene_np["sh_degree"], 1
    scene_s, cam_s = R.scene_struct(sd), R.camera_struct(cam)
    bg = (0.0, 0.0, 0.0)

    # autotuned sort digit width and render batch depth unless the digit
    # width is given
    digit_bits = args.digit_bits
    render_batch = 128
    tune = None
    if digit_bits is None:
        from paper_2605_04844_gb300 import autotune
        tune = autotune.tune_frame(sd, cam, mode="quadbox")
        digit_bits = tune["digit_bits"]
        render_batch = tune.get("render_batch", render_batch)

    frames, pairs = {}, {}
    for mode in ("quadbox", "aabb3s"):
        _, fr = R.forward(sd, cam, mode, bg=bg, digit_bits=digit_bits, sort_mode=args.sort_mode)
        pairs[mode] = fr.n_pairs
        cap = int(fr.n_pairs * 1.1) + 4096
        frames[mode] = R.Frame(n, W, H, cap)
        frames[mode].set_tuning(digit_bits=digit_bits, sort_mode=args.sort_mode, render_batch=render_batch)
    # the same QuadBox frame with the other pair-ordering schemes, for comparison
    other_modes = [m for m in ("depth_first", "full_key") if m != args.sort_mode]
    for m in other_modes:
        frames["quadbox_" + m] = R.Frame(n, W, H, int(pairs["quadbox"] * 1.1) + 4096)
        frames["quadbox_" + m].set_tuning(digit_bits=8, sort_mode=m, render_batch=render_batch)
    img = torch.empty((3, H, W), dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=dev)
    grads = {k: torch.zeros_like(sd[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    gs = N.QbSceneGrads()
    gs.means, gs.scales, gs.quats = grads["means"].data_ptr(), grads["scales"].data_ptr(), grads["quats"].data_ptr()
    gs.opacities, gs.sh = grads["opacities"].data_ptr(), grads["sh"].data_ptr()
    dL = torch.full((3, H, W), 1.0 / (3 * H * W), dtype=torch.float32, device=dev)

    STAGES = ("preprocess", "emit", "sort", "render", "backward")

    # per-kernel timeline: the library calls the hook just before each launch;
    # an event recorded there on the launching stream ends the previous kernel
    timeline = [None]
    ext_streams = {}

    def on_launch(name, handle):
        if timeline[0] is None:
            return
        st = stream if handle in (0, stream.cuda_stream) else ext_streams.setdefault(
            handle, torch.cuda.ExternalStream(handle))
        e = torch.cuda.Event(enable_timing=True)
        e.record(st)
        timeline[0].append((name, e))

    N.qb_set_launch_hook(on_launch)

    def mark(e):
        e.record(stream)
        if timeline[0] is not None:
            timeline[0].append(("", e))

    def step(fr, with_bwd, ev):
        mark(ev[0])
        fr.preprocess(scene_s, cam_s, mode_of[id(fr)])
        mark(ev[1])
        fr.bin_emit(sync=False)
        mark(ev[2])
        fr.sort()
        mark(ev[3])
        fr.render(bg, img)
        mark(ev[4])
        if with_bwd:
            for g in grads.values():
                g.zero_()
            N.qb_render_bwd(fr.frame, scene_s, cam_s, bg, dL, gs, None)
            mark(ev[5])

    mode_of = {id(fr): ("aabb3s" if name == "aabb3s" else "quadbox") for name, fr in frames.items()}

    def run_phase(mode, with_bwd, steps, warmup, kernels=None):
        """Times `steps` steps; with a dict `kernels`, also every kernel of the
        library launched in them (per name: launches and ms per step, ms per
        launch), from the events recorded at each launch."""
        fr = frames[mode]
        nev = 6 if with_bwd else 5
        for _ in range(warmup):
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(nev)]
            step(fr, with_bwd, evs)
        torch.cuda.synchronize()
        recs, lines = [], []
        for _ in range(steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            evs = [torch.cuda.Event(enable_timing=True) for _ in range(nev)]
            l0 = N.qb_kernel_launches()
            if kernels is not None:
                # the GPU spins while the host queues the step and its per-launch
                # events, so the kernels then run back to back between them
                torch.cuda._sleep(KERNEL_TIMING_SPIN_CYCLES)
                timeline[0] = []
            step(fr, with_bwd, evs)
            if kernels is not None:
                lines.append(timeline[0])
                timeline[0] = None
            launches[0] += N.qb_kernel_launches() - l0
            recs.append(evs)
        torch.cuda.synchronize()
        fr.check()
        per_stage = {s: 0.0 for s in STAGES}
        total = 0.0
        for evs in recs:
            for i in range(nev - 1):
                dt = evs[i].elapsed_time(evs[i + 1])
                per_stage[STAGES[i]] += dt
                total += dt
        if kernels is not None:
            for tl in lines:
                for i, (name, e) in enumerate(tl):
                    if name and i + 1 < len(tl):
                        k = kernels.setdefault(name, {"launches": 0, "ms": 0.0})
                        k["launches"] += 1
                        k["ms"] += e.elapsed_time(tl[i + 1][1])
            for k in kernels.values():
                k["ms_per_launch"] = round(k["ms"] / max(1, k["launches"]), 4)
                k["launches_per_step"] = k["launches"] / steps
                k["ms_per_step"] = round(k["ms"] / steps, 4)
                del k["ms"], k["launches"]
        return total / steps, {s: v / steps for s, v in per_stage.items()}

    def barrier():
        ranks_barrier(world)

    def rank_max(x):
        return max_over_ranks(x, world, dev)

    launches = [0]  # kernels of the library launched inside the timed steps
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    t_wall0 = time.time()
    fwd_ms, fwd_stages = run_phase("quadbox", False, args.steps, args.warmup)
    fb_ms, fb_stages = run_phase("quadbox", True, args.steps, args.warmup)
    afwd_ms, afwd_stages = run_phase("aabb3s", False, args.steps, args.warmup)
    afb_ms, afb_stages = run_phase("aabb3s", True, args.steps, args.warmup)
    others = {m: run_phase("quadbox_" + m, False, args.steps, args.warmup) for m in other_modes}
    # per-kernel durations of the QuadBox forward (for the roofline)
    fwd_kernels = {}
    run_phase("quadbox", False, args.steps, 1, kernels=fwd_kernels)
    torch.cuda.synchronize()
    barrier()
    wall = time.time() - t_wall0
    clk = clocks.stop()
    fwd_ms_max = rank_max(fwd_ms)

    # ---- render statistics for the ALU roofline (outside the timed region) ----
    fr = frames["quadbox"]
    fr.preprocess(scene_s, cam_s, "quadbox")
    fr.bin_emit(sync=False)
    fr.sort()
    fr.render(bg, img)
    torch.cuda.synchronize()
    # the method's render work: (pixel, entry) evaluations and those whose
    # power test passed, counted by the counted variant of the same render
    cnt = torch.zeros(2, dtype=torch.int64, device=dev)
    N.qb_render_fwd_counted(fr.frame, bg, img, cnt)
    torch.cuda.synchronize()
    n_eval, n_pass = (int(x) for x in cnt.cpu().tolist())

    # ---- end to end through the public API with host buffers ----
    # (as a user calls it: no per-launch timing hook)
    N.qb_set_launch_hook(None)
    host_img = torch.empty((3, H, W), dtype=torch.float32).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in pinned.values())
    d2h = host_img.numel() * 4
    e2e_times = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        l0 = N.qb_kernel_launches()
        for k, v in pinned.items():
            sd[k].copy_(v, non_blocking=True)
        fr.preprocess(scene_s, cam_s, "quadbox")
        fr.bin_emit(sync=False)
        fr.sort()
        fr.render(bg, img)
        host_img.copy_(img, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            e2e_times.append(e0.elapsed_time(e1))
            launches[0] += N.qb_kernel_launches() - l0
    fr.check()
    e2e_serial_ms = rank_max(statistics.mean(e2e_times))

    # streamed: frame i+1's scene upload and frame i-1's image download run on
    # copy streams while frame i renders (scene and image double-buffered on
    # the device); every frame still copies its whole scene in and its image
    # out, through the same API calls
    up_s, down_s = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    bufs = [sd, {k: (torch.empty_like(v) if torch.is_tensor(v) else v) for k, v in sd.items()}]
    structs = [R.scene_struct(bb) for bb in bufs]
    imgs = [img, torch.empty_like(img)]
    host_imgs = [host_img, torch.empty_like(host_img).pin_memory()]
    ev_copied = [torch.cuda.Event() for _ in range(2)]
    ev_rendered = [torch.cuda.Event() for _ in range(2)]
    ev_down = [torch.cuda.Event() for _ in range(2)]

    def streamed(frames, count_launches):
        for i in range(frames):
            b = i % 2
            with torch.cuda.stream(up_s):
                if i >= 2:
                    up_s.wait_event(ev_rendered[b])  # frame i-2 has read buffer b
                for k, v in pinned.items():
                    bufs[b][k].copy_(v, non_blocking=True)
                ev_copied[b].record(up_s)
            stream.wait_event(ev_copied[b])
            if i >= 2:
                stream.wait_event(ev_down[b])  # frame i-2's image has left buffer b
            l0 = N.qb_kernel_launches()
            fr.preprocess(structs[b], cam_s, "quadbox")
            fr.bin_emit(sync=False)
            fr.sort()
            fr.render(bg, imgs[b])
            if count_launches:
                launches[0] += N.qb_kernel_launches() - l0
            ev_rendered[b].record(stream)
            with torch.cuda.stream(down_s):
                down_s.wait_event(ev_rendered[b])
                host_imgs[b].copy_(imgs[b], non_blocking=True)
                ev_down[b].record(down_s)

    streamed(args.warmup, False)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(up_s)
    streamed(args.steps, True)
    down_s.wait_event(ev_rendered[(args.steps - 1) % 2])
    t1.record(down_s)
    torch.cuda.synchronize()
    fr.check()
    e2e_ms = rank_max(t0.elapsed_time(t1) / args.steps)

    P = pairs["quadbox"]
    result = {
        "metric": METRIC,
        "value": round(replica_fps(fwd_ms_max, world), 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(fwd_ms_max, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded 1M-Gaussian clustered scene; stands in for Mip-NeRF 360 / DB / T&T)",
        "config": {"workload": "1M Gaussians, 1920x1080, SH3, 16x16 tiles (C2): QuadBox vs 3-sigma AABB binning, "
                               "same kernels",
                   "n_gaussians": n, "width": W, "height": H, "sh_degree": 3,
                   "l2": "flushed between timed steps (258 MB write); scene 236 MB > L2",
                   "sort_digit_bits": digit_bits, "render_batch": render_batch, "sort_mode": args.sort_mode,
                   "parallelism": f"replicas x{world}"},
        "quadbox": {"fwd_fps": round(1000.0 / fwd_ms, 2), "fwd_ms": round(fwd_ms, 4),
                    "fwd_bwd_ms": round(fb_ms, 4), "pairs_per_frame": P,
                    "stage_ms": {k: round(v, 4) for k, v in fb_stages.items()}},
        "aabb3s": {"fwd_fps": round(1000.0 / afwd_ms, 2), "fwd_ms": round(afwd_ms, 4),
                   "fwd_bwd_ms": round(afb_ms, 4), "pairs_per_frame": pairs["aabb3s"],
                   "stage_ms": {k: round(v, 4) for k, v in afb_stages.items()}},
        "speedup_vs_aabb": {"fwd": round(afwd_ms / fwd_ms, 3), "fwd_bwd": round(afb_ms / fb_ms, 3),
                            "pair_ratio": round(pairs["aabb3s"] / max(P, 1), 3)},
        "quadbox_other_sort_modes": {m: {"fwd_ms": round(v[0], 4), "stage_ms": {k: round(x, 4) for k, x in v[1].items()}}
                                     for m, v in others.items()},
        "paper_context": "paper: 1.85x FPS over 3DGS, mean over Mip-NeRF 360/DB/T&T on NVIDIA A100 (Table 1)",
        "e2e": {"value": round(replica_fps(e2e_ms, world), 3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "mode": "streamed, double-buffered",
                "serial_value": round(replica_fps(e2e_serial_ms, world), 3)},
        "clocks": clk,
        "wall_s_timed": round(wall, 2),
    }
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    result["roofline"] = roofline(fwd_stages, fwd_kernels, P, n, W, H, digit_bits, (n_eval, n_pass), clk,
                                  args.sort_mode, sms=sms)
    result["render_work"] = {"evaluations": n_eval, "power_test_passed": n_pass,
                             "flops": RENDER_FLOPS_POWER_TEST * n_eval + RENDER_FLOPS_PASSED * n_pass}
    result["roofline_kernels"] = result["roofline"].pop("kernels", {})
    result["kernels_fwd"] = fwd_kernels
    # counted by the library at each launch, inside the timed steps of every
    # phase and of the end-to-end loop
    result["gpu_launches"] = int(launches[0])
    if tune:
        result["autotune"] = tune
    return result


def tile_sort_packed(n, W, H, digit_bits):
    """Whether the library's two-pass tile sort of this frame carries packed
    words between its passes: two passes whose first digit has 5 to 8 bits,
    and Gaussian indices below 2^(32 - second digit's bits)."""
    tiles = -(-W // 16) * -(-H // 16)
    tile_bits = max(1, (tiles - 1).bit_length())
    if -(-tile_bits // digit_bits) != 2:
        return False
    b0, b1 = -(-tile_bits // 2), tile_bits // 2
    return 5 <= b0 <= 8 and n <= 2 ** (32 - b1)


def kernel_work(P, n, evals, packed=False):
    """Algorithmic work per launch of each forward kernel at this frame: HBM
    bytes (what the kernel must move at least) or FP32 operations.  evals:
    (pixel-entry evaluations, those whose power test passed) of the render.
    packed: the tile sort's passes exchange one packed word per pair."""
    n_eval, n_pass = evals if evals else (0, 0)
    return {
        "preprocess_kernel": ("hbm", n * PREPROCESS_BYTES),
        "sort_hist_kernel": ("hbm", n * 4),              # the depth keys once
        "onesweep_kernel": ("hbm", n * 16),              # a depth-sort pass: key + value read and written
        "scan_onepass_kernel": ("hbm", n * 12),        # depth order read, counts gathered, offsets written
        "emit_warp_kernel": ("hbm", P * 8 + n * 28),     # pairs written; depth order, offset, count, segments
        "tile_count_kernel": ("hbm", P * 4),             # the tile ids once
        # key + value read, and written (packed: one word written)
        "tile_sort_pass": ("hbm", P * (12 if packed else 16)),
        # key + value (packed: one word) read, value written
        "tile_sort_pass_values": ("hbm", P * (8 if packed else 12)),
        "render_kernel": ("alu", n_eval * RENDER_FLOPS_POWER_TEST + n_pass * RENDER_FLOPS_PASSED),
    }


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per unit of
# work, from the ncu --set full captures of the 600k-Gaussian 1080p frame
# (20,633,099 pairs, 398,728,138 evaluations) summarised under profiles/,
# scaled to a launch of this frame by its units; valid for the kernels as
# captured (kernel -> (unit, bytes per unit)).  A kernel changed since its
# capture has no entry.
TRAFFIC_PER_UNIT = {
    "render_kernel": ("eval", (13.032192e6 + 0.436224e6) / 398728138),
    "tile_sort_pass": ("pair", (165.526528e6 + 34.277120e6) / 20633099),
    "tile_sort_pass_values": ("pair", (82.809600e6 + 35.105536e6) / 20633099),
    "emit_warp_kernel": ("pair", (52.036864e6 + 118.226176e6) / 20633099),
    "preprocess_kernel": ("gaussian", (147.195648e6 + 41.842176e6) / 600000),
    "tile_count_kernel": ("pair", (82.591232e6 + 1.410816e6) / 20633099),
}


def roofline(fwd_stages, kernels, P, n, W, H, digit_bits, evals, clk, sort_mode, sms=152):
    """Roofline of the dominant kernel of the forward step: its algorithmic
    work per launch over its average launch duration, both measured in the
    timed steps (CUDA events recorded at each launch on the launching
    stream); every other kernel of the step is listed the same way."""
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    sm_mhz = clk.get("sm_mhz") or float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    work = kernel_work(P, n, evals, packed=sort_mode != "full_key" and tile_sort_packed(n, W, H, digit_bits))
    n_eval = evals[0] if evals else 0
    rows = {}
    for name, k in kernels.items():
        if name not in work or not k.get("ms_per_launch"):
            continue
        bound, amount = work[name]
        secs = k["ms_per_launch"] * 1e-3
        if bound == "hbm":
            ach = amount / secs / 1e9
            rows[name] = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                          "frac": round(ach / hbm, 4), "bytes_per_launch": amount,
                          "ms_per_launch": k["ms_per_launch"], "ms_per_step": k["ms_per_step"]}
        elif amount:
            ach = amount / secs / 1e12
            rows[name] = {"bound": "alu", "achieved": round(ach, 3), "peak": round(alu_peak, 3), "unit": "TFLOP/s",
                          "frac": round(ach / alu_peak, 4), "flops_per_launch": amount,
                          "ms_per_launch": k["ms_per_launch"], "ms_per_step": k["ms_per_step"]}
    if not rows:
        return {"kernel": None}
    for name, r in rows.items():
        if name in TRAFFIC_PER_UNIT:
            unit, per = TRAFFIC_PER_UNIT[name]
            units = n_eval if unit == "eval" else (n if unit == "gaussian" else P)
            r["traffic"] = int(per * units) if units else None
    dom = max(rows, key=lambda r: rows[r]["ms_per_step"])
    d = rows[dom]
    traffic = d.get("traffic")
    out = {"kernel": dom, "bound": d["bound"], "achieved": d["achieved"], "peak": d["peak"], "unit": d["unit"],
           "frac": d["frac"], "traffic": traffic,
           "peak_source": ("MEASURED_PEAKS.json hbm_gbs (of measured)" if d["bound"] == "hbm" else
                           f"{sms} SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz (median sampled SM clock)"),
           "kernels": rows}
    return out


def _time_ms(fn, steps, warmup, stream):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / steps


def run_c3(args, dev):
    """Zoom sweep (Fig. 1 analogue): 3M Gaussians at 2560x1440, 30 views from
    distance 40 to 2; tile pairs and forward FPS per view for every binning
    mode on the same kernels (QuadBox and the 3-sigma AABB, plus AdR,
    QuadBox without QPass, DualBox and the unclamped QuadBox)."""
    import numpy as np
    import torch

    from paper_2605_04844_gb300 import _native as N
    from paper_2605_04844_gb300 import rasterizer as R
    from paper_2605_04844_gb300 import synth

    scene_np, cams = synth.config3()
    sd = {k: (torch.from_numpy(v).to(dev) if isinstance(v, np.ndarray) else v) for k, v in scene_np.items()}
    s = R.scene_struct(sd)
    stream = torch.cuda.current_stream(dev)
    frames = {}
    views = []
    modes = ("quadbox", "aabb3s", "adr", "quadbox_naive", "dualbox", "quadbox+noclamp")
    for k, cam in enumerate(cams):
        d = float(-cam["viewmat"][2][3]) if "viewmat" in cam else None
        row = {"view": k, "distance": round(abs(d), 3) if d is not None else None}
        cs = R.camera_struct(cam)
        for mode in modes:
            # the two headline modes keep their own frames; the others share one
            slot = mode if mode in ("quadbox", "aabb3s") else "other"
            try:
                _, fr = R.forward(sd, cam, mode, frame=frames.get(slot))
            except N.QbCapacityError:
                row[mode] = {"pairs": None, "note": "over 2^30 pairs"}
                continue
            frames[slot] = fr
            pairs = fr.n_pairs
            img = torch.empty((3, cam["height"], cam["width"]), device=dev)

            def fwd(fr=fr, mode=mode):
                fr.preprocess(s, cs, mode)
                fr.bin_emit(sync=False)
                fr.sort()
                fr.render(None, img)
            ms = _time_ms(fwd, 3, 1, stream)
            fr.check()
            row[mode] = {"pairs": pairs, "fwd_ms": round(ms, 3), "fps": round(1000.0 / ms, 1)}
        if row.get("quadbox", {}).get("pairs") and row.get("aabb3s", {}).get("pairs"):
            row["pair_ratio"] = round(row["aabb3s"]["pairs"] / max(1, row["quadbox"]["pairs"]), 3)
            row["speedup"] = round(row["aabb3s"]["fwd_ms"] / row["quadbox"]["fwd_ms"], 3)
        views.append(row)
    return {"workload": "3M Gaussians (ball of radius 10 at the origin), 2560x1440, SH3, 30 views on -z from "
                        "distance 40 to 2 (geometric); every binning mode on the same kernels", "views": views}


def run_modes(args, dev):
    """The paper's ablation (Table 3) on C2: pairs per frame and forward time
    of every binning mode on the same kernels, and each mode's image against
    the clamped QuadBox image (the conservative modes must match it bit for
    bit; DualBox is not conservative and the unclamped boxes reach beyond the
    3-sigma rectangle, so those two differ by design)."""
    import numpy as np
    import torch

    from paper_2605_04844_gb300 import rasterizer as R
    from paper_2605_04844_gb300 import synth

    scene_np, cam = synth.config2(args.n, args.width, args.height)
    sd = {k: (torch.from_numpy(v).to(dev) if isinstance(v, np.ndarray) else v) for k, v in scene_np.items()}
    s, cs = R.scene_struct(sd), R.camera_struct(cam)
    stream = torch.cuda.current_stream(dev)
    img = torch.empty((3, cam["height"], cam["width"]), device=dev)
    out = {"workload": "C2 (1M Gaussians, 1920x1080, SH3), forward per binning mode, same kernels; image delta "
                       "against the clamped QuadBox image"}
    ref = None
    for mode in ("quadbox", "aabb3s", "adr", "quadbox_naive", "dualbox", "quadbox+noclamp", "adr+noclamp"):
        _, fr = R.forward(sd, cam, mode)
        pairs = fr.n_pairs

        def fwd(fr=fr, mode=mode):
            fr.preprocess(s, cs, mode)
            fr.bin_emit(sync=False)
            fr.sort()
            fr.render(None, img)
        ms = _time_ms(fwd, 10, 3, stream)
        fr.check()
        row = {"pairs": pairs, "fwd_ms": round(ms, 4), "fps": round(1000.0 / ms, 1)}
        if ref is None:
            ref = img.clone()
        else:
            diff = (img - ref).abs()
            row["image_vs_quadbox"] = {"identical": bool(torch.equal(img, ref)),
                                       "max_abs": round(float(diff.max().item()), 6),
                                       "pixels_differing": int((diff.amax(dim=0) > 0).sum().item())}
        out[mode] = row
        del fr
    return out


def run_c4(args, dev):
    """500k Gaussians, 1264x832, SH3: forward + backward with an L1 loss against
    a random target (dL/dimg = sign(img - target) / (3 H W))."""
    import numpy as np
    import torch

    from paper_2605_04844_gb300 import _native as N
    from paper_2605_04844_gb300 import rasterizer as R
    from paper_2605_04844_gb300 import synth

    scene_np, cam, target_np = synth.config4()
    sd = {k: (torch.from_numpy(v).to(dev) if isinstance(v, np.ndarray) else v) for k, v in scene_np.items()}
    target = torch.from_numpy(target_np).to(dev)
    s, cs = R.scene_struct(sd), R.camera_struct(cam)
    H, W = cam["height"], cam["width"]
    stream = torch.cuda.current_stream(dev)
    grads = {k: torch.zeros_like(sd[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    gs = N.QbSceneGrads()
    gs.means, gs.scales, gs.quats = grads["means"].data_ptr(), grads["scales"].data_ptr(), grads["quats"].data_ptr()
    gs.opacities, gs.sh = grads["opacities"].data_ptr(), grads["sh"].data_ptr()
    img = torch.empty((3, H, W), device=dev)
    dL = torch.empty_like(img)
    out = {"workload": "500k Gaussians, 1264x832, SH3, L1 loss against a U[0,1] target (seed 2004); "
                       "train_step_ms: forward + loss gradient + backward + Adam on all raw parameters "
                       "(one host read of the pair count per step)"}
    for mode in ("quadbox", "aabb3s"):
        _, fr = R.forward(sd, cam, mode)
        pairs = fr.n_pairs

        def step(fr=fr, mode=mode):
            fr.preprocess(s, cs, mode)
            fr.bin_emit(sync=False)
            fr.sort()
            fr.render(None, img)
            torch.sub(img, target, out=dL)
            dL.sign_().mul_(1.0 / (3 * H * W))
            for g in grads.values():
                g.zero_()
            N.qb_render_bwd(fr.frame, s, cs, None, dL, gs, None)

        def fwd(fr=fr, mode=mode):
            fr.preprocess(s, cs, mode)
            fr.bin_emit(sync=False)
            fr.sort()
            fr.render(None, img)
        fb = _time_ms(step, 10, 3, stream)
        f = _time_ms(fwd, 10, 3, stream)
        fr.check()
        # a whole training step: forward, L1 gradient, backward and Adam on
        # every raw parameter array, on a copy of the scene
        sd_t = {k: (v.clone() if torch.is_tensor(v) else v) for k, v in sd.items()}
        tr = R.Trainer(sd_t, cam, mode)
        ts = _time_ms(lambda: tr.step(target), 10, 3, stream)
        out[mode] = {"pairs": pairs, "fwd_ms": round(f, 3), "fwd_bwd_ms": round(fb, 3),
                     "fwd_bwd_per_s": round(1000.0 / fb, 1), "train_step_ms": round(ts, 3),
                     "loss_after_13_steps": round(float(tr.loss.item()), 6)}
    out["speedup_fwd_bwd"] = round(out["aabb3s"]["fwd_bwd_ms"] / out["quadbox"]["fwd_bwd_ms"], 3)
    return out


def run_batch(args, dev):
    """64 cameras of uneven resolution around a 1M-Gaussian scene: one
    graph-captured qb_render_batch (fwd, and fwd+bwd with an L1 loss against a
    random target) versus 64 separate single-frame launch sequences."""
    import numpy as np
    import torch

    from paper_2605_04844_gb300 import _native as N
    from paper_2605_04844_gb300 import autotune
    from paper_2605_04844_gb300 import rasterizer as R
    from paper_2605_04844_gb300 import synth

    scene_np, cams = synth.config5(args.batch_n, args.batch_cams)
    sd = {k: (torch.from_numpy(v).to(dev) if isinstance(v, np.ndarray) else v) for k, v in scene_np.items()}
    s = R.scene_struct(sd)
    ca = R.camera_array(cams)
    b = R.calibrated_batch(sd, cams, group=16)
    tune = autotune.tune_batch(b, sd, cams)
    t = tune["tune"]
    stream = torch.cuda.current_stream(dev)
    target = torch.rand(b.images.shape, device=dev, generator=torch.Generator(dev).manual_seed(2005))
    npix = sum(w * h for w, h in zip(b.widths, b.heights))
    grads = {k: torch.zeros_like(sd[k]) for k in ("means", "scales", "quats", "opacities", "sh")}
    gs = N.QbSceneGrads()
    gs.means, gs.scales, gs.quats = grads["means"].data_ptr(), grads["scales"].data_ptr(), grads["quats"].data_ptr()
    gs.opacities, gs.sh = grads["opacities"].data_ptr(), grads["sh"].data_ptr()
    dL = torch.empty_like(b.images)

    def fwd():
        b.render(s, ca, "quadbox", t)

    def fwd_bwd():
        b.render(s, ca, "quadbox", t)
        torch.sub(b.images, target, out=dL)
        dL.sign_().mul_(1.0 / (3 * npix))
        for g in grads.values():
            g.zero_()
        b.backward(s, ca, dL, gs)

    fwd_bwd()  # first calls outside capture
    torch.cuda.synchronize()
    pairs = b.check()
    graphs = {}
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    for name, fn in (("fwd", fwd), ("fwd_bwd", fwd_bwd)):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            b.stream = side
            with torch.cuda.graph(g, stream=side):
                fn()
        b.stream = None
        graphs[name] = g
    torch.cuda.synchronize()

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / steps

    steps = max(3, min(args.steps, 10))
    g_fwd = timed(graphs["fwd"].replay, steps, 2)
    g_fb = timed(graphs["fwd_bwd"].replay, steps, 2)
    b.check()

    # the same cameras as separate single-frame launch sequences
    frames = {}
    for c in cams:  # one frame per resolution, grown to the largest camera's pairs
        key = (c["width"], c["height"])
        _, frames[key] = R.forward(sd, c, "quadbox", frame=frames.get(key), digit_bits=t["sort_digit_bits"])
    for fr in frames.values():
        fr.set_tuning(render_batch=t["render_batch"])
    imgs = {key: torch.empty((3, key[1], key[0]), device=dev) for key in frames}
    dls = {key: torch.full((3, key[1], key[0]), 1.0 / (3 * npix), device=dev) for key in frames}
    cam_structs = [R.camera_struct(c) for c in cams]

    def separate(with_bwd):
        for c, cs in zip(cams, cam_structs):
            key = (c["width"], c["height"])
            fr = frames[key]
            fr.preprocess(s, cs, "quadbox")
            fr.bin_emit(sync=False)
            fr.sort()
            fr.render(None, imgs[key])
            if with_bwd:
                N.qb_render_bwd(fr.frame, s, cs, None, dls[key], gs, None)

    sep_fwd = timed(lambda: separate(False), max(2, steps // 2), 1)
    sep_fb = timed(lambda: separate(True), max(2, steps // 2), 1)
    for fr in frames.values():
        fr.check()
    K = len(cams)
    return {"workload": f"{args.batch_n} Gaussians, {K} cameras on a radius-8 sphere, resolutions from "
                        "800x800/1264x832/1600x900/1920x1080, preprocess in groups of 16, one global render queue",
            "pairs_total": int(sum(pairs)), "pairs_max_camera": int(max(pairs)), "tune": t,
            "graph_fwd_ms": round(g_fwd, 3), "graph_fwd_bwd_ms": round(g_fb, 3),
            "separate_fwd_ms": round(sep_fwd, 3), "separate_fwd_bwd_ms": round(sep_fb, 3),
            "graph_fwd_cams_per_s": round(K * 1000.0 / g_fwd, 1),
            "graph_fwd_bwd_cams_per_s": round(K * 1000.0 / g_fb, 1),
            "speedup_fwd": round(sep_fwd / g_fwd, 3), "speedup_fwd_bwd": round(sep_fb / g_fb, 3)}


# GPU spin before each step of the per-kernel timing phase (~4 ms at 2 GHz):
# longer than the host takes to queue one step with its events.
KERNEL_TIMING_SPIN_CYCLES = 8_000_000

# Algorithmic bytes of the preprocess per Gaussian: read 44 B of parameters and
# 192 B of SH coefficients (degree 3), write mu^2D 8, conic+o 16, colour+depth
# 16, box 16, 3-sigma radius 4, meta 4, count 4, depth-sort key and index 8
# (76 B).  The QPass run records (16 to 64 B per visible Gaussian) are left
# out, which understates the kernel's fraction slightly.
PREPROCESS_BYTES = 236 + 76

# FP32 arithmetic of Eq. 2's per-pixel loop (an FMA counts 2, comparisons
# and min/max none).  Every evaluated (pixel, entry): d = mu - p (2 sub), the
# power a' dx^2 + b' dx dy + c' dy^2 as dx (a' dx) + dy (c' dy + b' dx)
# (3 mul + 2 FMA) = 9.  An entry whose power test passes also takes alpha =
# o exp(power) (exp 1 + its argument scaling 1 + mul 1), T' = T (1 - alpha)
# (sub 1 + mul 1), the weight alpha T (mul 1) and three colour FMAs (6) = 12.
RENDER_FLOPS_POWER_TEST = 9
RENDER_FLOPS_PASSED = 12


# --------------------------------------------------------------------------
# CPU oracle (cpu_baseline and the reference arm)
# --------------------------------------------------------------------------

def oracle_frame_seconds(scene_np, cam, row_stride=16):
    """One forward frame of the FP64 oracle: projection, binning and sort
    in full, compositing on every row_stride-th tile row (scaled up)."""
    import numpy as np

    from oracle import oracle as O
    W, H = cam["width"], cam["height"]
    t0 = time.time()
    s64 = {k: (v.astype(np.float64) if isinstance(v, np.ndarray) else v) for k, v in scene_np.items()}
    proj = O.project(s64, cam)
    L = O.own_lists(proj, W, H, O.QUADBOX, True)
    t1 = time.time()
    ty = (H + 15) // 16
    rows = list(range(0, ty, row_stride))
    tx = (W + 15) // 16
    pxs, pys = [], []
    for r in rows:
        ys = np.arange(r * 16, min(H, r * 16 + 16))
        xs = np.arange(W)
        yy, xx = np.meshgrid(ys, xs, indexing="ij")
        pxs.append(xx.ravel())
        pys.append(yy.ravel())
    pxs, pys = np.concatenate(pxs), np.concatenate(pys)
    t2 = time.time()
    O.render_pixels(W, H, pxs, pys, L["ranges"], L["vals"], proj)
    t3 = time.time()
    frac = len(pxs) / (W * H)
    return (t1 - t0) + (t3 - t2) / frac, len(L["vals"]), len(pxs)


def cpu_baseline(scene_np, cam):
    """The FP64 oracle on the host cores: the C2 frame on all cores (the
    reported value) and on one core, and the whole C1 frame on both."""
    from oracle import oracle as O
    from paper_2605_04844_gb300 import synth
    O.build()
    cores = O.max_threads()
    secs, P, npx = oracle_frame_seconds(scene_np, cam)
    O.set_threads(1)
    secs1, _, npx1 = oracle_frame_seconds(scene_np, cam, row_stride=64)
    c1_scene, c1_cam = synth.config1()
    c1_1 = oracle_frame_seconds(c1_scene, c1_cam, row_stride=1)[0]
    O.set_threads(cores)
    c1_all = oracle_frame_seconds(c1_scene, c1_cam, row_stride=1)[0]
    return {"value": round(1.0 / secs, 5), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"the C2 frame in FP64: projection, binning, sort in full; every 16th tile row "
                      f"composited ({npx} px), scaled",
            "seconds_per_frame": round(secs, 3),
            "one_core_seconds_per_frame": round(secs1, 3),
            "one_core_sample": f"the same frame with every 64th tile row composited ({npx1} pixels), scaled",
            "c1_10k_256x256_seconds": {"all_cores": round(c1_all, 4), "one_core": round(c1_1, 4)}}


def run_reference(args):
    from paper_2605_04844_gb300 import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    scene_np, cam = synth.config2(args.n, args.width, args.height)
    from oracle import oracle as O
    O.build()
    for _ in range(args.warmup):
        oracle_frame_seconds(scene_np, cam, row_stride=64)
    times = []
    for _ in range(args.steps):
        secs, P, npx = oracle_frame_seconds(scene_np, cam, row_stride=64)
        times.append(secs)
    sec = statistics.mean(times)
    cores = int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count())
    val = round(1.0 / sec, 5)
    return {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(sec * 1000, 2),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded 1M-Gaussian clustered scene)",
            "config": {"workload": "1M Gaussians, 1920x1080, SH degree 3, QuadBox binning; FP64 CPU oracle"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "per step: full FP64 projection, binning and sort of the frame, "
                                       "compositing of every 64th tile row, scaled to the frame"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


# Sections of the full result printed on their own lines before the headline
# (and kept whole in the --out file).
DETAIL_SECTIONS = ("kernels_fwd", "roofline_kernels", "render_work", "quadbox_other_sort_modes", "autotune",
                   "c4_fwd_bwd", "binning_modes", "c3_zoom", "batch64", "cpu_baseline")

HEADLINE_MAX_BYTES = 2000


def output_lines(res):
    """The lines the run prints: each detail section on its own line, then
    the compact headline last (the line a reader of the output tail parses)."""
    lines = [json.dumps({"section": name, name: res[name]}) for name in DETAIL_SECTIONS if name in res]
    lines.append(json.dumps(headline(res)))
    return lines


def headline(res):
    """The compact last line of the run: the headline metric, the QuadBox and
    3-sigma AABB forward and forward+backward times with their pairs per
    frame, the end-to-end rate, clocks, the dominant kernel's roofline row
    and the CPU oracle baseline; everything else is in the detail lines."""
    h = {k: res[k] for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                             "higher_is_better", "scaling", "vs_baseline", "dtype", "data") if k in res}
    cfg = res.get("config", {})
    h["config"] = {k: cfg[k] for k in ("workload", "n_gaussians", "width", "height", "sh_degree", "l2",
                                       "sort_digit_bits", "parallelism") if k in cfg}
    for side in ("quadbox", "aabb3s"):
        if side in res:
            h[side] = {k: res[side][k] for k in ("fwd_ms", "fwd_bwd_ms", "pairs_per_frame") if k in res[side]}
    if "stage_ms" in res.get("quadbox", {}):
        h["quadbox"]["stage_ms"] = res["quadbox"]["stage_ms"]
    for k in ("speedup_vs_aabb", "e2e", "gpu_launches"):
        if k in res:
            h[k] = res[k]
    clk = res.get("clocks") or {}
    h["clocks"] = {k: clk.get(k) for k in ("sm_mhz", "sm_max_mhz", "reasons")}
    rf = res.get("roofline") or {}
    h["roofline"] = {k: rf.get(k) for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "traffic")}
    if "peak_source" in rf:
        h["roofline"]["peak_source"] = rf["peak_source"]
    cb = res.get("cpu_baseline")
    if cb:
        h["cpu_baseline"] = {k: cb.get(k) for k in ("value", "unit", "cores", "kind", "sample")}
    b = res.get("batch64")
    if b:
        h["batch64"] = {k: b.get(k) for k in ("graph_fwd_ms", "graph_fwd_bwd_ms", "speedup_fwd", "speedup_fwd_bwd")}
    h["paper_context"] = "paper: 1.85x FPS over 3DGS on NVIDIA A100 (Table 1)"
    h["details"] = "sections on the preceding output lines"
    # optional keys go first when the line would grow past the bound
    for k in ("paper_context", "details", "batch64", ("roofline", "peak_source"), ("quadbox", "stage_ms")):
        if len(json.dumps(h)) <= HEADLINE_MAX_BYTES:
            break
        if isinstance(k, tuple):
            h.get(k[0], {}).pop(k[1], None)
        else:
            h.pop(k, None)
    if "cpu_baseline" in h and len(json.dumps(h)) > HEADLINE_MAX_BYTES:
        h["cpu_baseline"]["sample"] = h["cpu_baseline"]["sample"][:120]
    return h


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    import torch
    if world > 1:
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res = run_ours(args, rank, world, local_rank)
    if rank == 0:
        import torch
        dev = torch.device("cuda", local_rank)
        if not args.no_c4:
            res["c4_fwd_bwd"] = run_c4(args, dev)
            res["binning_modes"] = run_modes(args, dev)
        if not args.no_c3:
            res["c3_zoom"] = run_c3(args, dev)
        if not args.no_batch:
            res["batch64"] = run_batch(args, dev)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            from paper_2605_04844_gb300 import synth
            scene_np, cam = synth.config2(args.n, args.width, args.height)
            res["cpu_baseline"] = cpu_baseline(scene_np, cam)
        if args.out:
            with open(args.out, "w") as f:
                f.write(json.dumps(res) + "\n")
        for line in output_lines(res):
            print(line, flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
