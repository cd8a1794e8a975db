"""The oracle's FP64 adjoint against FP64 central finite differences of its forward.

Scene: 64 Gaussians, SH3, 64x64, camera at (0,0,4), 60 deg (the finite-difference
workload); step 1e-6. The loss is a fixed random linear functional of the image,
L = sum(gC * rgb) + sum(gA * alpha), so that dL/dimage = (gC, gA) exactly.
A parameter whose difference quotients at steps 1e-6 and 1e-5 disagree has moved a
decision (a 3-sigma cut, the 1/255 skip, the early stop, a clamp): it is reported
and excluded, since the adjoint holds decision sets fixed.
"""
import numpy as np
import pytest

import oracle
from paper_2512_08478_b300 import synth

FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def _loss(scene, cam, gC, gA, bg, depth=None):
    img, _ = oracle.render(scene, cam, bg, depth=depth)
    return float(np.sum(gC * img["rgb"]) + np.sum(gA * img["alpha"]))


def _fd(scene, cam, gC, gA, bg, field, idx, h, depth=None):
    vals = []
    for s in (+1, -1):
        sc = {k: (np.array(v, np.float64, copy=True) if k in FIELDS else v) for k, v in scene.items()}
        sc[field].reshape(-1)[idx] += s * h
        vals.append(_loss(sc, cam, gC, gA, bg, depth))
    return (vals[0] - vals[1]) / (2 * h)


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.3, 0.6, 0.9)])
def test_adjoint_matches_central_differences(bg):
    scene, cam = synth.fd_scene()
    scene = {k: (v.astype(np.float64) if k in FIELDS else v) for k, v in scene.items()}
    rng = np.random.default_rng(17)
    gC = rng.standard_normal((3, cam.H, cam.W))
    gA = rng.standard_normal((cam.H, cam.W))
    grads = oracle.adjoint(scene, cam, gC, gA, bg)
    checked = excluded = 0
    for field in FIELDS:
        g = grads[field].reshape(-1)
        n = g.shape[0]
        idxs = range(n) if field != "sh" else rng.choice(n, 400, replace=False)
        scale = np.max(np.abs(g)) + 1e-30
        for idx in idxs:
            f1 = _fd(scene, cam, gC, gA, bg, field, idx, 1e-6)
            f2 = _fd(scene, cam, gC, gA, bg, field, idx, 1e-5)
            if abs(f1 - f2) > 1e-4 * max(abs(f1), abs(f2)) + 1e-7 * scale:
                excluded += 1
                continue
            checked += 1
            assert abs(f1 - g[idx]) <= 1e-6 * abs(f1) + 1e-6 * scale, (field, idx, f1, g[idx])
    assert checked > 900
    assert excluded < 0.05 * (checked + excluded), (checked, excluded)


def test_adjoint_with_depth_buffer_matches_central_differences():
    """The same check with a slanted depth buffer through the scene (depth-buffer-aware
    compositing): splats behind a pixel's depth value take no part there, in the forward
    and in the adjoint alike."""
    scene, cam = synth.fd_scene()
    scene = {k: (v.astype(np.float64) if k in FIELDS else v) for k, v in scene.items()}
    rng = np.random.default_rng(23)
    gC = rng.standard_normal((3, cam.H, cam.W))
    gA = rng.standard_normal((cam.H, cam.W))
    xs = np.arange(cam.W)[None, :].repeat(cam.H, 0)
    depth = (3.75 + 0.5 * xs / cam.W).astype(np.float32)
    bg = (0.2, 0.4, 0.6)
    grads = oracle.adjoint(scene, cam, gC, gA, bg, depth=depth)
    free = oracle.adjoint(scene, cam, gC, gA, bg)
    assert not np.allclose(grads["means"], free["means"])   # the buffer does cut the scene
    checked = excluded = 0
    for field in FIELDS:
        g = grads[field].reshape(-1)
        n = g.shape[0]
        idxs = rng.choice(n, min(n, 120), replace=False)
        scale = np.max(np.abs(g)) + 1e-30
        for idx in idxs:
            f1 = _fd(scene, cam, gC, gA, bg, field, idx, 1e-6, depth)
            f2 = _fd(scene, cam, gC, gA, bg, field, idx, 1e-5, depth)
            if abs(f1 - f2) > 1e-4 * max(abs(f1), abs(f2)) + 1e-7 * scale:
                excluded += 1
                continue
            checked += 1
            assert abs(f1 - g[idx]) <= 1e-6 * abs(f1) + 1e-6 * scale, (field, idx, f1, g[idx])
    assert checked > 300
    assert excluded < 0.05 * (checked + excluded), (checked, excluded)


def _multi_loss(scenes, models, cam, gC, gA, bg):
    img, _ = oracle.render_multi(scenes, models, cam, bg)
    return float(np.sum(gC * img["rgb"]) + np.sum(gA * img["alpha"]))


def test_multi_model_adjoint_matches_central_differences():
    """Two models drawn together, one under a general affine map (rotation, shear,
    anisotropic scale, translation) and one translated: the gradients with respect to
    each model's own parameters (the compositing adjoint over the global order, then each
    model's preprocess adjoint through A Sigma A^T, A mu + b and the model-frame SH ray)
    against central differences of the joint image."""
    base, cam = synth.fd_scene()
    base = {k: (v.astype(np.float64) if k in FIELDS else v) for k, v in base.items()}
    s1 = {k: (v[:32].copy() if k in FIELDS else v) for k, v in base.items()}
    s2 = {k: (v[32:].copy() if k in FIELDS else v) for k, v in base.items()}
    rng = np.random.default_rng(31)
    M1 = synth.affine_model(rng, translation_std=0.1, log_scale_std=0.2, shear=0.3).astype(np.float64)
    M2 = np.concatenate([np.eye(3), np.array([[0.125], [-0.0625], [0.25]])], 1)
    gC = rng.standard_normal((3, cam.H, cam.W))
    gA = rng.standard_normal((cam.H, cam.W))
    bg = (0.1, 0.3, 0.5)
    grads = oracle.adjoint_multi([s1, s2], [M1, M2], cam, gC, gA, bg)
    # the single-model entry point agrees with the multi-model one for a lone model (up to
    # the order of the per-tile additions, which threads make in any order)
    lone = oracle.adjoint(s1, cam, gC, gA, bg, model=M1)
    lone_multi = oracle.adjoint_multi([s1], [M1], cam, gC, gA, bg)[0]
    for f in FIELDS:
        assert np.allclose(lone[f], lone_multi[f], rtol=1e-11, atol=1e-13 * np.abs(lone[f]).max()), f
    checked = excluded = 0
    for which, sc in enumerate((s1, s2)):
        for field in FIELDS:
            g = grads[which][field].reshape(-1)
            idxs = rng.choice(g.shape[0], min(g.shape[0], 60), replace=False)
            scale = np.max(np.abs(g)) + 1e-30
            for idx in idxs:
                fd = []
                for h in (1e-6, 1e-5):
                    vals = []
                    for sgn in (+1, -1):
                        moved = {k: (np.array(v, copy=True) if k in FIELDS else v) for k, v in sc.items()}
                        moved[field].reshape(-1)[idx] += sgn * h
                        pair = [moved, s2] if which == 0 else [s1, moved]
                        vals.append(_multi_loss(pair, [M1, M2], cam, gC, gA, bg))
                    fd.append((vals[0] - vals[1]) / (2 * h))
                f1, f2 = fd
                if abs(f1 - f2) > 1e-4 * max(abs(f1), abs(f2)) + 1e-7 * scale:
                    excluded += 1
                    continue
                checked += 1
                assert abs(f1 - g[idx]) <= 1e-6 * abs(f1) + 1e-6 * scale, (which, field, idx, f1, g[idx])
    assert checked > 350
    assert excluded < 0.05 * (checked + excluded), (checked, excluded)


def test_adjoint_clamp_branches_match_central_differences():
    """The three places where the definition passes no gradient, each pinned by central
    differences of the forward on a Gaussian built to sit in it (synth.fd_branch_scene):

    - alpha clamp (reading S11): Gaussian 64 reaches o G > 0.99 at one pixel, where
      alpha = 0.99 whatever its parameters are, so that pixel adds nothing to any of its
      derivatives;
    - Jacobian guard (reading S5): Gaussian 65 sits at x/z = 0.85, beyond 1.3 tan(half
      FOV), where J is taken at the clamped ratio and so does not move with x;
    - colour clamp (reading S2): Gaussian 66's green sum is negative, rendered as 0, so
      its green SH coefficients have zero derivative.
    Every parameter of the three Gaussians is checked (59 each)."""
    scene, cam = synth.fd_branch_scene()
    scene = {k: (v.astype(np.float64) if k in FIELDS else v) for k, v in scene.items()}
    prep = oracle.preprocess(scene, cam)
    # the scene is what it claims to be
    u, v = prep["uv"][64]
    d = np.array([20.5 - u, 40.5 - v])
    a, b, c = prep["conic"][64]
    q = a * d[0] ** 2 + 2 * b * d[0] * d[1] + c * d[1] ** 2
    assert prep["opacity"][64] * np.exp(-0.5 * q) > float(np.float32(0.99)) + 1e-3
    p_cam = cam.R.astype(np.float64) @ scene["means"][65] + cam.t.astype(np.float64)
    assert p_cam[0] / p_cam[2] > 1.3 * (cam.W / (2.0 * cam.fx)) + 0.05
    assert prep["valid"][65] == 1 and prep["rect"][65][0] < cam.W // 16
    assert prep["rgb"][66][1] == 0.0 and prep["valid"][66] == 1

    rng = np.random.default_rng(41)
    gC = rng.standard_normal((3, cam.H, cam.W))
    gA = rng.standard_normal((cam.H, cam.W))
    bg = (0.25, 0.5, 0.75)
    grads = oracle.adjoint(scene, cam, gC, gA, bg)
    K = 16
    checked = excluded = 0
    for field in FIELDS:
        g = grads[field].reshape(-1)
        per = g.shape[0] // scene["means"].shape[0]
        scale = np.max(np.abs(g)) + 1e-30
        for i in (64, 65, 66):
            for idx in range(i * per, (i + 1) * per):
                f1 = _fd(scene, cam, gC, gA, bg, field, idx, 1e-6)
                f2 = _fd(scene, cam, gC, gA, bg, field, idx, 1e-5)
                if abs(f1 - f2) > 1e-4 * max(abs(f1), abs(f2)) + 1e-7 * scale:
                    excluded += 1
                    continue
                checked += 1
                assert abs(f1 - g[idx]) <= 1e-6 * abs(f1) + 1e-6 * scale, (field, i, idx, f1, g[idx])
    assert checked >= 170 and excluded <= 7, (checked, excluded)
    # the clamped colour channel: exactly zero, from both sides
    sh_g = grads["sh"].reshape(-1, K, 3)
    assert np.all(sh_g[66, :, 1] == 0.0) and np.all(sh_g[66, :, 0] != 0.0)
