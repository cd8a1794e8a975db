"""Seeded synthetic scenes and cameras for the 3DGS rasterizer.

This module only *draws inputs*: Gaussian attribute arrays and pinhole cameras.
It holds none of the rendering arithmetic (no projection, no covariance, no
spherical-harmonics evaluation, no compositing), so both the CUDA path and the
FP64 oracle may consume what it produces without sharing method code.

Scene arrays (all float32, C-contiguous):
  means          [N, 3]     world-space centres
  log_scales     [N, 3]     per-axis log standard deviation
  quats          [N, 4]     rotation quaternion, (w, x, y, z), not necessarily unit
  opacity_logits [N]        pre-sigmoid opacity
  sh             [N, K, 3]  K = (deg+1)^2 coefficients per channel, index l*l+l+m

Cameras follow the pinhole model with OpenCV axes (x right, y down, z forward):
a world point X maps to camera space as R @ X + t; pixel (x, y) covers
[x, x+1) x [y, y+1) and the principal point is (W/2, H/2).

Random numbers: numpy PCG64 seeded per workload, fp64 draws cast to fp32, in the
order means, log_scales, quats, opacity_logits, sh, then workload extras.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Degree-0 real spherical harmonic Y_0^0 = 1 / (2 sqrt(pi)). The workloads specify
# the *rendered* DC colour c in [0, 1]; the stored coefficient is (c - 0.5) / Y_0^0
# under the renderer's "+0.5 offset" colour convention. This is the only place the
# generator touches SH, and only to express the workload's colour distribution.
_Y00 = 0.5 / math.sqrt(math.pi)


@dataclass
class Camera:
    R: np.ndarray      # [3, 3] float32 world->camera rotation, row-major
    t: np.ndarray      # [3] float32
    fx: float
    fy: float
    cx: float
    cy: float
    near: float
    W: int
    H: int

    def as_array(self) -> np.ndarray:
        """[R(9), t(3), fx, fy, cx, cy, near] as float32 (17 values)."""
        return np.concatenate([
            self.R.reshape(-1), self.t.reshape(-1),
            np.array([self.fx, self.fy, self.cx, self.cy, self.near], np.float32),
        ]).astype(np.float32)


def look_at(eye, target, W, H, fov_v_deg, near=0.2, up=(0.0, 1.0, 0.0)) -> Camera:
    """Pinhole camera at `eye` looking at `target`, world up +y, vertical FOV in degrees.

    fy = H / (2 tan(fov_v / 2)), fx = fy (square pixels), principal point at the
    image centre.
    """
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    f = target - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:  # looking straight along up: pick another up
        r = np.cross(f, np.array([0.0, 0.0, 1.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f]).astype(np.float32)
    t = (-(R.astype(np.float64) @ eye)).astype(np.float32)
    fy = H / (2.0 * math.tan(math.radians(fov_v_deg) / 2.0))
    return Camera(R=R, t=t, fx=float(np.float32(fy)), fy=float(np.float32(fy)),
                  cx=W / 2.0, cy=H / 2.0, near=near, W=W, H=H)


def orbit_cameras(n, radius, W, H, fov_v_deg, height=0.0, phase=0.0, near=0.2):
    """n cameras on a circle of `radius` in the y = height plane, looking at the origin."""
    cams = []
    for k in range(n):
        a = phase + 2.0 * math.pi * k / n
        eye = (radius * math.sin(a), height, radius * math.cos(a))
        cams.append(look_at(eye, (0.0, 0.0, 0.0), W, H, fov_v_deg, near=near))
    return cams


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _sh_coeffs(rng, n, deg, hi_std):
    K = (deg + 1) ** 2
    sh = np.zeros((n, K, 3), np.float64)
    dc = rng.uniform(0.0, 1.0, (n, 3))
    sh[:, 0, :] = (dc - 0.5) / _Y00
    if K > 1:
        sh[:, 1:, :] = rng.normal(0.0, hi_std, (n, K - 1, 3))
    return sh


def _pack(means, log_scales, quats, logits, sh, deg):
    return dict(
        means=np.ascontiguousarray(means, np.float32),
        log_scales=np.ascontiguousarray(log_scales, np.float32),
        quats=np.ascontiguousarray(quats, np.float32),
        opacity_logits=np.ascontiguousarray(logits, np.float32),
        sh=np.ascontiguousarray(sh, np.float32),
        sh_degree=int(deg),
    )


def uniform_cube_scene(n, seed, sh_degree=0, extent=1.0, log_scale_mean=-4.0,
                       log_scale_std=0.5, logit_mean=0.0, logit_std=1.0, hi_std=0.05):
    """Means uniform in [-extent, extent]^3; the 10k-Gaussian SH0 workload's recipe."""
    rng = np.random.Generator(np.random.PCG64(seed))
    means = rng.uniform(-extent, extent, (n, 3))
    log_scales = rng.normal(log_scale_mean, log_scale_std, (n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(logit_mean, logit_std, n)
    sh = _sh_coeffs(rng, n, sh_degree, hi_std)
    return _pack(means, log_scales, quats, logits, sh, sh_degree)


def mixture_scene(n, seed, sh_degree=3, components=64, ball_radius=10.0, comp_std=0.8,
                  log_scale_mean=-3.5, log_scale_std=0.7, logit_mean=0.5, logit_std=1.5,
                  hi_std=0.05, rng=None):
    """Means from an isotropic Gaussian mixture whose centres are uniform in a ball.

    This is the large-scene recipe (1M / 6M / 500k Gaussians, SH3): centres
    r = R U^(1/3) along a uniform direction, component picked uniformly, std 0.8.
    """
    if rng is None:
        rng = np.random.Generator(np.random.PCG64(seed))
    cdir = rng.standard_normal((components, 3))
    cdir /= np.linalg.norm(cdir, axis=1, keepdims=True)
    crad = ball_radius * rng.uniform(0.0, 1.0, components) ** (1.0 / 3.0)
    centres = cdir * crad[:, None]
    comp = rng.integers(0, components, n)
    means = centres[comp] + comp_std * rng.standard_normal((n, 3))
    log_scales = rng.normal(log_scale_mean, log_scale_std, (n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(logit_mean, logit_std, n)
    sh = _sh_coeffs(rng, n, sh_degree, hi_std)
    return _pack(means, log_scales, quats, logits, sh, sh_degree)


# --------------------------------------------------------------------------------------
# The five benchmark workloads (sizes and distributions as stated for each).
# --------------------------------------------------------------------------------------

def workload_small(seed=0):
    """10,000 Gaussians, SH0, 256x256, one camera at (0,0,4) with 60 deg vertical FOV."""
    scene = uniform_cube_scene(10_000, seed, sh_degree=0)
    cam = look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), 256, 256, 60.0)
    return scene, [cam]


def workload_1m(seed=1, n=1_000_000, views=32, W=1920, H=1080):
    """1M Gaussians, SH3, 32 orbit views (radius 15) at 1920x1080, 50 deg vertical FOV."""
    scene = mixture_scene(n, seed, sh_degree=3)
    cams = orbit_cameras(views, 15.0, W, H, 50.0)
    return scene, cams


def workload_dynamic(seed=2, n=6_000_000, frames=120, W=1920, H=1080):
    """6M Gaussians, SH3, moving means and pulsing opacity over 120 frames, one camera.

    Extras (drawn after the scene): velocity v ~ N(0, 0.02 I) (covariance 0.02 I);
    opacity pulse amplitude A ~ U[0,1], integer frequency f ~ U{1,2,3}, phase
    phi ~ U[0, 2 pi). Frame k uses normalised time t = k / frames:
      mu_t = mu_0 + t v,  logit_t = logit_0 + A sin(2 pi f t + phi).
    The camera orbits slowly: radius 15, azimuth 0.25 deg per frame.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    scene = mixture_scene(n, seed, sh_degree=3, rng=rng)
    extras = dict(
        velocity=(math.sqrt(0.02) * rng.standard_normal((n, 3))).astype(np.float32),
        amp=rng.uniform(0.0, 1.0, n).astype(np.float32),
        freq=rng.integers(1, 4, n).astype(np.float32),
        phase=rng.uniform(0.0, 2.0 * math.pi, n).astype(np.float32),
    )
    cams = [look_at((15.0 * math.sin(math.radians(0.25 * k)), 0.0,
                     15.0 * math.cos(math.radians(0.25 * k))), (0, 0, 0), W, H, 50.0)
            for k in range(frames)]
    return scene, extras, cams


def dynamic_frame_inputs(scene, extras, k, frames=120):
    """Means and opacity logits of frame k of the dynamic workload (host arrays)."""
    t = np.float32(k / frames)
    means = scene["means"] + t * extras["velocity"]
    logits = scene["opacity_logits"] + extras["amp"] * np.sin(
        np.float32(2 * math.pi) * extras["freq"] * t + extras["phase"]).astype(np.float32)
    return means.astype(np.float32), logits.astype(np.float32)


def workload_fwdbwd(seed=3, n=500_000, W=800, H=800, views=4):
    """500k Gaussians, SH3, 800x800; target = render of means/log-scales + N(0, 0.01)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    scene = mixture_scene(n, seed, sh_degree=3, rng=rng)
    target = dict(scene)
    target["means"] = (scene["means"] + 0.01 * rng.standard_normal((n, 3))).astype(np.float32)
    target["log_scales"] = (scene["log_scales"] + 0.01 * rng.standard_normal((n, 3))).astype(np.float32)
    cams = orbit_cameras(views, 15.0, W, H, 50.0)
    return scene, target, cams


def fd_scene(seed=3, n=64, W=64, H=64):
    """Finite-difference scene: 64 Gaussians, SH3, 64x64, camera at (0,0,4), 60 deg."""
    rng = np.random.Generator(np.random.PCG64(seed + 1000))
    means = rng.uniform(-0.5, 0.5, (n, 3))
    log_scales = rng.normal(-2.0, 0.3, (n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, n)
    sh = _sh_coeffs(rng, n, 3, 0.05)
    scene = _pack(means, log_scales, quats, logits, sh, 3)
    cam = look_at((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), W, H, 60.0)
    return scene, cam


def fd_branch_scene(seed=3):
    """The finite-difference scene plus three Gaussians that drive the definition's clamps:

    index 64  "clamp": isotropic, logit 8 (opacity 0.99966), world (-0.632, -0.470, 0.9),
              log-scale -1.785: about 3 px wide, centred 0.2 px right of and 0.1 px above
              the centre of pixel (20, 40), so that pixel takes alpha = min(0.99, o G) at
              the clamp while its neighbours stay near 0.95;
    index 65  "guard": world (3.4, -0.1, 0), i.e. camera-space x/z = 0.85, beyond the
              Jacobian guard 1.3 tan(30 deg) = 0.75 of the 60 deg view, with scales
              (0.7, 0.5, 0.6) so that its footprint still reaches the right image border;
    index 66  "black": SH3 with rendered DC colour (0.6, -0.4, 0.3), so that the green sum
              stays below zero (the higher bands are N(0, 0.05)) and the channel renders
              black under the colour clamp.
    The 64x64 camera at (0, 0, 4) maps world (X, Y, Z) to camera (X, -Y, 4 - Z)."""
    scene, cam = fd_scene(seed)
    rng = np.random.Generator(np.random.PCG64(seed + 2000))
    means = np.array([[-0.632, -0.470, 0.9], [3.4, -0.1, 0.0], [0.1, 0.15, -0.3]])
    log_scales = np.array([[-1.785] * 3, np.log([0.7, 0.5, 0.6]), [-1.9, -2.1, -2.0]])
    quats = np.array([[1.0, 0.0, 0.0, 0.0], [0.9, 0.2, -0.3, 0.25], [0.6, -0.3, 0.5, 0.4]])
    logits = np.array([8.0, 3.0, 1.5])
    sh = np.zeros((3, 16, 3))
    sh[:, 0, :] = (np.array([[0.8, 0.3, 0.6], [0.2, 0.7, 0.4], [0.6, -0.4, 0.3]]) - 0.5) / _Y00
    sh[:, 1:, :] = rng.normal(0.0, 0.05, (3, 15, 3))
    extra = _pack(means, log_scales, quats, logits, sh, 3)
    out = {k: np.concatenate([scene[k], extra[k]]) for k in
           ("means", "log_scales", "quats", "opacity_logits", "sh")}
    out["sh_degree"] = 3
    return out, cam


BATCH_RESOLUTIONS = ((512, 512), (1280, 720), (1920, 1080))


def workload_batch(seed=4, assets=16, cams_per_asset=8, n_min=20_000, n_max=2_000_000,
                   scale=1.0):
    """16 assets (N log-uniform in [2e4, 2e6], SH degree uniform in {0..3}), 8 orbit
    cameras each at a resolution drawn from {512^2, 1280x720, 1920x1080}: 128 images.

    `scale` shrinks every Gaussian count (for small parity cases); 1.0 is the full size.
    Returns (scenes, cams, cam_scene) with cam_scene[i] the asset index of camera i.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), assets))
    degs = rng.integers(0, 4, assets)
    res = rng.integers(0, len(BATCH_RESOLUTIONS), assets * cams_per_asset)
    scenes = []
    for a in range(assets):
        n = max(1, int(round(ns[a] * scale)))
        scenes.append(mixture_scene(n, seed * 1000 + a, sh_degree=int(degs[a])))
    cams, cam_scene = [], []
    for a in range(assets):
        for k in range(cams_per_asset):
            W, H = BATCH_RESOLUTIONS[int(res[a * cams_per_asset + k])]
            ang = 2.0 * math.pi * k / cams_per_asset
            cams.append(look_at((15.0 * math.sin(ang), 0.0, 15.0 * math.cos(ang)),
                                (0, 0, 0), W, H, 50.0))
            cam_scene.append(a)
    return scenes, cams, cam_scene


# --------------------------------------------------------------------------------------
# Per-model affine transforms (Algorithm 1's M_k) and the multi-asset workload.
# --------------------------------------------------------------------------------------

def _axis_rotation(axis, angle_rad):
    """Rotation matrix about a unit axis (Rodrigues)."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])
    return np.eye(3) + math.sin(angle_rad) * K + (1.0 - math.cos(angle_rad)) * (K @ K)


def rigid_model(angle_deg=0.0, axis=(0.0, 1.0, 0.0), translation=(0.0, 0.0, 0.0), scale=1.0):
    """[A | b] (3x4 float32) with A = scale * rotation(axis, angle), b = translation."""
    A = scale * _axis_rotation(axis, math.radians(angle_deg))
    return np.ascontiguousarray(np.concatenate([A, np.asarray(translation, np.float64)[:, None]], 1), np.float32)


def affine_model(rng, translation_std=0.3, log_scale_std=0.3, shear=0.3):
    """A general affine [A | b] (3x4 float32): rotation * shear * anisotropic scale * rotation,
    det(A) > 0."""
    def rot():
        return _axis_rotation(rng.standard_normal(3), rng.uniform(0.0, 2.0 * math.pi))
    Sh = np.eye(3)
    Sh[0, 1], Sh[0, 2], Sh[1, 2] = rng.uniform(-shear, shear, 3)
    A = rot() @ Sh @ np.diag(np.exp(rng.normal(0.0, log_scale_std, 3))) @ rot()
    b = rng.normal(0.0, translation_std, 3)
    return np.ascontiguousarray(np.concatenate([A, b[:, None]], 1), np.float32)


def workload_multi(seed=5, assets=4, n_min=100_000, n_max=1_000_000, W=1920, H=1080, scale=1.0):
    """Multi-asset frame (section 3.4, several models in one image): `assets` mixture-scene
    models (N log-uniform in [n_min, n_max], SH degree uniform in {0..3}, ball radius 2.5),
    each placed by a rigid transform (rotation about y, uniform scale in [0.7, 1.4]) on a
    ring of radius 2.5 around the origin, so that the models overlap on screen and
    interleave in depth; one camera at (0, 3, 14) looking at the origin, 50 deg.
    `scale` shrinks every Gaussian count (for small parity cases).
    Returns (scenes, models [K,3,4] float32, camera)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.exp(rng.uniform(math.log(n_min), math.log(n_max), assets))
    degs = rng.integers(0, 4, assets)
    scenes, models = [], []
    for a in range(assets):
        n = max(1, int(round(ns[a] * scale)))
        scenes.append(mixture_scene(n, seed * 1000 + a, sh_degree=int(degs[a]), ball_radius=2.5, comp_std=0.4,
                                    log_scale_mean=-4.0))
        ang = 2.0 * math.pi * a / assets + rng.uniform(-0.3, 0.3)
        models.append(rigid_model(rng.uniform(0.0, 360.0), (0.0, 1.0, 0.0),
                                  (2.5 * math.sin(ang), rng.uniform(-0.5, 0.5), 2.5 * math.cos(ang)),
                                  rng.uniform(0.7, 1.4)))
    cam = look_at((0.0, 3.0, 14.0), (0.0, 0.0, 0.0), W, H, 50.0)
    return scenes, np.stack(models), cam


def random_keys(m, seed, kind="random", tile_bits=13):
    """Synthetic (tile, depth) sort inputs for stage tests of the radix sort.

    kind: random | equal | sorted | reverse | high_only | few_tiles.
    Keys are (tile << 32) | depth_bits with depth_bits the float32 pattern of a
    positive depth; vals are 0..m-1 (the duplication order).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    tiles = rng.integers(0, 1 << tile_bits, m, dtype=np.uint64)
    depth = rng.uniform(0.2, 40.0, m).astype(np.float32).view(np.uint32).astype(np.uint64)
    if kind == "equal":
        tiles[:] = 5
        depth[:] = np.float32(3.0).view(np.uint32)
    elif kind == "few_tiles":
        tiles = rng.integers(0, 3, m, dtype=np.uint64)
        depth = rng.integers(0, 4, m, dtype=np.uint64) + np.uint64(np.float32(1.0).view(np.uint32))
    elif kind == "high_only":
        depth[:] = np.float32(2.0).view(np.uint32)
    keys = (tiles << np.uint64(32)) | depth
    if kind == "sorted":
        keys = np.sort(keys)
    elif kind == "reverse":
        keys = np.sort(keys)[::-1].copy()
    vals = np.arange(m, dtype=np.uint32)
    return np.ascontiguousarray(keys, np.uint64), vals
