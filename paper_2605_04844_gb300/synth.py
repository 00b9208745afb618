"""Seeded synthetic scenes and cameras (inputs only).

This module holds none of the rasteriser's arithmetic: it draws Gaussian
parameters and builds pinhole cameras, as plain numpy arrays, so that the
CUDA path and the CPU oracle receive identical inputs.  It stands in for the
paper's trained scenes (Mip-NeRF 360, Deep Blending, Tanks & Temples), which
are not available: the shapes, sizes and distributions follow the benchmark
configurations (10k / 256^2; 1M / 1080p SH3 with blobs; 3M / 1440p zoom
sweep; 500k / 1264x832 forward+backward; 1M scene with 64 cameras).

Scene dict: means [n,3], scales [n,3] (log-scales), quats [n,4] (w,x,y,z,
unnormalised), opacities [n] (logits), sh [n,K,3], sh_degree, raw=1.
Camera dict: viewmat [4,4] (row-major world->view, view looks down +z),
fx, fy, cx, cy, tan_fovx, tan_fovy, campos [3], width, height, znear.
"""
from __future__ import annotations

import math

import numpy as np

SH_C0 = 1.0 / (2.0 * math.sqrt(math.pi))  # degree-0 basis value: colour = C0 * DC + 0.5
RESOLUTIONS = [(800, 800), (1264, 832), (1600, 900), (1920, 1080)]


def look_at(campos, target, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->view matrix of a camera at campos looking at target (view +z)."""
    c = np.asarray(campos, dtype=np.float64)
    z = np.asarray(target, dtype=np.float64) - c
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(up, dtype=np.float64), z)
    if np.linalg.norm(x) < 1e-9:
        x = np.cross(np.array([1.0, 0.0, 0.0]), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    V = np.eye(4)
    V[0, :3], V[1, :3], V[2, :3] = x, y, z
    V[:3, 3] = -V[:3, :3] @ c
    return V


def pinhole(width, height, fov_x_deg=60.0, viewmat=None, znear=0.2):
    """Pinhole camera with square pixels and pixel centres at integers."""
    tanx = math.tan(math.radians(fov_x_deg) / 2.0)
    fx = width / (2.0 * tanx)
    fy = fx
    tany = height / (2.0 * fy)
    V = np.eye(4) if viewmat is None else np.asarray(viewmat, dtype=np.float64)
    R, t = V[:3, :3], V[:3, 3]
    campos = -R.T @ t
    return {"viewmat": V.astype(np.float32), "fx": fx, "fy": fy, "cx": (width - 1) / 2.0,
            "cy": (height - 1) / 2.0, "tan_fovx": tanx, "tan_fovy": tany,
            "campos": campos.astype(np.float32), "width": int(width), "height": int(height), "znear": znear}


def _quats(rng, n):
    return rng.standard_normal((n, 4)).astype(np.float32)


def _sh(rng, n, deg, higher_sigma=0.1):
    K = (deg + 1) ** 2
    sh = np.zeros((n, K, 3), dtype=np.float32)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    sh[:, 0, :] = (rgb - 0.5) / SH_C0
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, higher_sigma, (n, K - 1, 3))
    return sh


def _frustum_points(rng, n, depth_lo, depth_hi, tanx, tany):
    z = rng.uniform(depth_lo, depth_hi, n)
    x = rng.uniform(-1.0, 1.0, n) * z * tanx
    y = rng.uniform(-1.0, 1.0, n) * z * tany
    return np.stack([x, y, z], axis=1)


def scene_uniform(n, seed, cam, depth=(2.0, 6.0), logscale=(-3.5, 0.8), opac_sigma=1.5, deg=0):
    """Means uniform across the camera frustum at the given depth range
    (world = view space), log-scales N(mu, sigma), random unit quaternions,
    opacity logits N(0, opac_sigma), uniform RGB."""
    rng = np.random.default_rng(seed)
    means = _frustum_points(rng, n, depth[0], depth[1], cam["tan_fovx"], cam["tan_fovy"])
    return {
        "means": means.astype(np.float32),
        "scales": rng.normal(logscale[0], logscale[1], (n, 3)).astype(np.float32),
        "quats": _quats(rng, n),
        "opacities": rng.normal(0.0, opac_sigma, n).astype(np.float32),
        "sh": _sh(rng, n, deg),
        "sh_degree": deg, "raw": 1,
    }


def scene_blobs(n, seed, cam, depth=(1.0, 50.0), n_blobs=64, blob_frac=0.8, blob_sigma=0.05,
                logscale=(-4.0, 1.0), aniso_frac=0.1, aniso_boost=2.5, opac_sigma=2.0, deg=3):
    """Clustered scene in the camera frustum: blob_frac of the means in
    n_blobs Gaussian blobs (centres uniform in the frustum, sigma =
    blob_sigma * depth), the rest uniform in the frustum; log-scales
    N(mu, sigma) with aniso_frac Gaussians getting +aniso_boost on one random
    axis; opacity logits N(0, opac_sigma); SH of degree deg with uniform DC
    colour and N(0, 0.1) higher bands."""
    rng = np.random.default_rng(seed)
    tanx, tany = cam["tan_fovx"], cam["tan_fovy"]
    nb = int(round(n * blob_frac))
    centres = _frustum_points(rng, n_blobs, depth[0], depth[1], tanx, tany)
    which = rng.integers(0, n_blobs, nb)
    sig = blob_sigma * centres[which, 2:3]
    blob_pts = centres[which] + rng.standard_normal((nb, 3)) * sig
    bg_pts = _frustum_points(rng, n - nb, depth[0], depth[1], tanx, tany)
    means = np.concatenate([blob_pts, bg_pts], axis=0)
    means = means[rng.permutation(n)]
    # scene is given in the camera's view space; express it in world space
    V = np.asarray(cam["viewmat"], dtype=np.float64)
    means = (means - V[:3, 3]) @ V[:3, :3]
    scales = rng.normal(logscale[0], logscale[1], (n, 3))
    boost = rng.random(n) < aniso_frac
    axis = rng.integers(0, 3, n)
    scales[np.arange(n)[boost], axis[boost]] += aniso_boost
    return {
        "means": means.astype(np.float32),
        "scales": scales.astype(np.float32),
        "quats": _quats(rng, n),
        "opacities": rng.normal(0.0, opac_sigma, n).astype(np.float32),
        "sh": _sh(rng, n, deg),
        "sh_degree": deg, "raw": 1,
    }


def scene_ball(n, seed, radius=10.0, n_blobs=64, blob_frac=0.8, blob_sigma=0.5, logscale=(-4.0, 1.0),
               aniso_frac=0.1, aniso_boost=2.5, opac_sigma=2.0, deg=3):
    """Clustered scene centred at the origin: blob centres and background
    uniform in a ball of the given radius, otherwise as scene_blobs."""
    rng = np.random.default_rng(seed)

    def ball(m):
        d = rng.standard_normal((m, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        r = radius * rng.random(m) ** (1.0 / 3.0)
        return d * r[:, None]

    nb = int(round(n * blob_frac))
    centres = ball(n_blobs)
    which = rng.integers(0, n_blobs, nb)
    blob_pts = centres[which] + rng.standard_normal((nb, 3)) * blob_sigma
    means = np.concatenate([blob_pts, ball(n - nb)], axis=0)[rng.permutation(n)]
    scales = rng.normal(logscale[0], logscale[1], (n, 3))
    boost = rng.random(n) < aniso_frac
    axis = rng.integers(0, 3, n)
    scales[np.arange(n)[boost], axis[boost]] += aniso_boost
    return {
        "means": means.astype(np.float32),
        "scales": scales.astype(np.float32),
        "quats": _quats(rng, n),
        "opacities": rng.normal(0.0, opac_sigma, n).astype(np.float32),
        "sh": _sh(rng, n, deg),
        "sh_degree": deg, "raw": 1,
    }


def zoom_cameras(width, height, n_views=30, d_far=40.0, d_near=2.0):
    """Cameras on the -z axis at d_k = d_far (d_near/d_far)^(k/(n-1)), looking at the origin."""
    cams = []
    for k in range(n_views):
        d = d_far * (d_near / d_far) ** (k / max(1, n_views - 1))
        cams.append(pinhole(width, height, viewmat=look_at((0.0, 0.0, -d), (0.0, 0.0, 0.0))))
    return cams


def sphere_cameras(n_cams, radius, seed, resolutions=RESOLUTIONS):
    """n_cams cameras on a Fibonacci lattice of the sphere of the given radius,
    looking at the origin with +y up; resolutions drawn with the seed."""
    rng = np.random.default_rng(seed)
    golden = math.pi * (3.0 - math.sqrt(5.0))
    cams = []
    for k in range(n_cams):
        y = 1.0 - 2.0 * (k + 0.5) / n_cams
        r = math.sqrt(max(0.0, 1.0 - y * y))
        th = golden * k
        pos = radius * np.array([r * math.cos(th), y, r * math.sin(th)])
        W, H = resolutions[int(rng.integers(0, len(resolutions)))]
        cams.append(pinhole(W, H, viewmat=look_at(pos, (0.0, 0.0, 0.0))))
    return cams


# --------------------------------------------------------------------------
# Benchmark configurations (seed = 1000 + configuration number)
# --------------------------------------------------------------------------

def config1(n=10_000, width=256, height=256):
    """Plain forward, 10k Gaussians, 256x256, SH degree 0."""
    cam = pinhole(width, height)
    return scene_uniform(n, 1001, cam), cam


def config2(n=1_000_000, width=1920, height=1080):
    """Forward, 1M Gaussians, 1920x1080, SH degree 3, 64 blobs + 20% background."""
    cam = pinhole(width, height)
    return scene_blobs(n, 1002, cam), cam


def config3(n=3_000_000, width=2560, height=1440, n_views=30):
    """Zoom sweep, 3M Gaussians, 2560x1440, 30 views from distance 40 to 2."""
    return scene_ball(n, 1003), zoom_cameras(width, height, n_views)


def config4(n=500_000, width=1264, height=832):
    """Forward+backward, 500k Gaussians, 1264x832, SH degree 3, target U[0,1]."""
    cam = pinhole(width, height)
    scene = scene_blobs(n, 1004, cam)
    target = np.random.default_rng(2004).uniform(0.0, 1.0, (3, height, width)).astype(np.float32)
    return scene, cam, target


def config5(n=1_000_000, n_cams=64):
    """Batched: 1M-Gaussian scene at the origin, 64 cameras on a sphere of radius 8."""
    return scene_ball(n, 1005, radius=4.0), sphere_cameras(n_cams, 8.0, 1005)
