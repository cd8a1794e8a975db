"""Several scenes in one image (vis_render_multi / vis_render_backward_multi): every model
preprocessed under its own affine transform M_k into its own workspace slots, then one
global sort and one compositing pass (Algorithm 1). Parity with the oracle's multi-model
render and adjoint, and bit-identity with the single merged scene when the transforms
are identities."""
import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth
from gpu_helpers import image_parity

pytestmark = pytest.mark.gpu

BG = (0.1, 0.2, 0.3)


def _multi(scenes_np, models, cam, opts=None, depth=None, bg=BG):
    import torch
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    ws = vis.multi_workspace(scenes, cam.W, cam.H, opts=opts)
    d = None if depth is None else torch.from_numpy(np.ascontiguousarray(depth, np.float32)).cuda()
    rgb, alpha = vis._render_multi_checked(scenes, models, cam, cam.W, cam.H, bg, ws, opts, depth=d)
    return rgb.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64), scenes, ws, d


def _scenes(sizes, deg, seed=0):
    return [synth.mixture_scene(n, seed + k, sh_degree=deg, components=8, ball_radius=1.0, comp_std=0.35,
                                log_scale_mean=-3.2, hi_std=0.2) for k, n in enumerate(sizes)]


def _concat(scenes):
    return dict({k: np.ascontiguousarray(np.concatenate([s[k] for s in scenes])) for k in vis.FIELDS},
                sh_degree=scenes[0]["sh_degree"])


@pytest.mark.parametrize("opts", [dict(), dict(sort_mode=0), dict(tile=8),
                                  dict(pixels_per_thread=2)])
def test_identity_models_equal_the_concatenated_scene(opts):
    """Ragged scene sizes (padding slots between the scenes): the image is the single
    concatenated scene's, bit for bit (same splats, same global order)."""
    scs = _scenes([300, 1000, 2049, 1], 2, seed=3)
    cam = synth.look_at((0.4, 0.3, 4.0), (0, 0, 0), 200, 150, 50.0)
    o = vis.make_opts(**opts)
    a_rgb, a_alpha, *_ = _multi(scs, None, cam, o)
    eye = np.tile(np.concatenate([np.eye(3), np.zeros((3, 1))], 1)[None], (4, 1, 1))
    e_rgb, e_alpha, *_ = _multi(scs, eye, cam, o)
    sc = vis.Scene.from_numpy(_concat(scs))
    ws = vis.Workspace(sc.n, cam.W, cam.H, opts=o)
    b_rgb, b_alpha = vis._render_checked(sc, cam, cam.W, cam.H, BG, ws, o)
    assert np.array_equal(a_rgb, b_rgb.cpu().numpy()) and np.array_equal(a_alpha, b_alpha.cpu().numpy())
    assert np.array_equal(a_rgb, e_rgb) and np.array_equal(a_alpha, e_alpha)


@pytest.mark.parametrize("opts", [dict(), dict(sort_mode=0), dict(tile=8)])
def test_multi_asset_workload_parity(opts):
    """The multi-asset workload (rigidly placed models, SH degrees 0..3) at 1/50 of its size."""
    scs, models, cam = synth.workload_multi(scale=0.02, W=480, H=270)
    rgb, alpha, *_ = _multi(scs, models, cam, vis.make_opts(**opts))
    ref, prep = oracle.render_multi(scs, list(models), cam, BG)
    assert prep["valid"].sum() > 5000
    image_parity(rgb, alpha, ref)


@pytest.mark.parametrize("seed", [0, 1])
def test_general_affine_models_parity(seed):
    """Sheared, anisotropically scaled models with SH3 (model-frame SH rays)."""
    rng = np.random.default_rng(seed)
    scs = _scenes([1500, 2500, 700], 3, seed=10 + 5 * seed)
    models = [synth.affine_model(rng, translation_std=0.6, shear=0.4) for _ in scs]
    cam = synth.look_at((0.5, 1.0, 5.0), (0, 0, 0), 256, 192, 50.0)
    rgb, alpha, *_ = _multi(scs, models, cam)
    ref, _ = oracle.render_multi(scs, models, cam, BG)
    image_parity(rgb, alpha, ref)


def test_same_scene_instanced_twice():
    scs = _scenes([2000], 1, seed=20)
    models = [synth.rigid_model(30.0, (0, 1, 0), (-0.6, 0.0, 0.0)), synth.rigid_model(-50.0, (1, 0, 0), (0.6, 0.1, -0.3))]
    cam = synth.look_at((0.0, 0.5, 5.0), (0, 0, 0), 192, 128, 50.0)
    rgb, alpha, *_ = _multi([scs[0], scs[0]], models, cam)
    ref, _ = oracle.render_multi([scs[0], scs[0]], models, cam, BG)
    image_parity(rgb, alpha, ref)


def test_multi_with_depth_buffer():
    scs, models, cam = synth.workload_multi(scale=0.01, W=320, H=180, seed=6)
    xs = (np.arange(cam.W)[None, :] + 0.5) / cam.W
    depth = np.repeat(12.0 + 4.0 * xs, cam.H, axis=0).astype(np.float32)
    rgb, alpha, *_ = _multi(scs, models, cam, depth=depth)
    ref, _ = oracle.render_multi(scs, list(models), cam, BG, depth=depth)
    free, _ = oracle.render_multi(scs, list(models), cam, BG)
    assert np.abs(ref["rgb"] - free["rgb"]).max() > 0.05
    image_parity(rgb, alpha, ref)


def test_multi_culled_scene_and_one_gaussian():
    scs = _scenes([800, 1], 0, seed=30)
    behind = [synth.rigid_model(0.0, (0, 1, 0), (0.0, 0.0, 0.0)), synth.rigid_model(0.0, (0, 1, 0), (0.0, 0.0, 9.0))]
    cam = synth.look_at((0.0, 0.0, 4.0), (0, 0, 0), 96, 64, 50.0)
    dead = dict(scs[0], opacity_logits=np.full_like(scs[0]["opacity_logits"], -30.0))
    for sc_list, mdl in (([scs[0], scs[1]], behind), ([dead, scs[1]], None)):
        rgb, alpha, *_ = _multi(sc_list, mdl, cam)
        ref, _ = oracle.render_multi(sc_list, mdl, cam, BG)
        image_parity(rgb, alpha, ref)


def _grads_multi(scs, models, cam, gC, gA, bg, opts=None):
    import torch
    _, _, scenes, ws, _ = _multi(scs, models, cam, opts, bg=bg)
    grads = [{k: torch.empty_like(s.tensors[k]) for k in vis.FIELDS} for s in scenes]
    vis.vis_render_backward_multi([s.handle for s in scenes], models, cam, cam.W, cam.H, bg,
                                  torch.from_numpy(gC.astype(np.float32)).cuda(),
                                  torch.from_numpy(gA.astype(np.float32)).cuda(), ws.buf, grads, opts)
    return [{k: g[k].cpu().numpy().astype(np.float64) for k in vis.FIELDS} for g in grads]


@pytest.mark.parametrize("opts", [dict(), dict(sort_mode=0)])
def test_multi_gradients_match_oracle(opts):
    base, cam = synth.fd_scene()
    s1 = {k: (v[:40].copy() if k in vis.FIELDS else v) for k, v in base.items()}
    s2 = {k: (v[40:].copy() if k in vis.FIELDS else v) for k, v in base.items()}
    rng = np.random.default_rng(5)
    models = [synth.affine_model(rng, translation_std=0.1, log_scale_std=0.2, shear=0.3),
              synth.rigid_model(25.0, (0.3, 1.0, 0.2), (0.1, -0.05, 0.2))]
    gC = rng.standard_normal((3, cam.H, cam.W))
    gA = rng.standard_normal((cam.H, cam.W))
    bg = (0.2, 0.4, 0.6)
    got = _grads_multi([s1, s2], models, cam, gC, gA, bg, vis.make_opts(**opts))
    ref = oracle.adjoint_multi([s1, s2], models, cam, gC, gA, bg)
    for k_s in range(2):
        for f in vis.FIELDS:
            a, b = got[k_s][f].ravel(), ref[k_s][f].ravel()
            assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), (k_s, f)


def test_autograd_render_multi_instanced():
    """The autograd wrapper: one scene drawn twice under two transforms gets the sum of
    both instances' gradients."""
    import torch
    base, cam = synth.fd_scene()
    sc = vis.Scene.from_numpy(base)
    for k in vis.FIELDS:
        sc.tensors[k].requires_grad_(True)
    models = np.stack([synth.rigid_model(20.0, (0, 1, 0), (-0.3, 0.0, 0.0)),
                       synth.rigid_model(-35.0, (0, 1, 0), (0.35, 0.05, -0.2))])
    rng = np.random.default_rng(8)
    gC = rng.standard_normal((3, cam.H, cam.W))
    gA = rng.standard_normal((cam.H, cam.W))
    rgb, alpha = vis.render_multi([sc, sc], models, cam, cam.W, cam.H)
    ref, _ = oracle.render_multi([base, base], list(models), cam)
    image_parity(rgb.detach().cpu().numpy().astype(np.float64), alpha.detach().cpu().numpy().astype(np.float64),
                 ref)
    loss = (rgb * torch.from_numpy(gC.astype(np.float32)).cuda()).sum() + \
        (alpha * torch.from_numpy(gA.astype(np.float32)).cuda()).sum()
    loss.backward()
    r = oracle.adjoint_multi([base, base], list(models), cam, gC, gA)
    for f in vis.FIELDS:
        a = sc.tensors[f].grad.cpu().numpy().astype(np.float64).ravel()
        b = (r[0][f] + r[1][f]).ravel()
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), f


def test_multi_rejects_singular_model():
    scs = _scenes([100], 0)
    cam = synth.look_at((0.0, 0.0, 4.0), (0, 0, 0), 64, 64, 50.0)
    sing = np.zeros((1, 3, 4), np.float32)
    sing[0, 0, 0] = sing[0, 1, 1] = 1.0
    with pytest.raises(vis.VisError):
        _multi(scs, sing, cam)


def test_multi_gradients_with_depth_buffer_match_oracle():
    """The multi-model adjoint with a depth buffer (the depth test among the held decisions)."""
    import torch
    base, cam = synth.fd_scene()
    s1 = {k: (v[:40].copy() if k in vis.FIELDS else v) for k, v in base.items()}
    s2 = {k: (v[40:].copy() if k in vis.FIELDS else v) for k, v in base.items()}
    rng = np.random.default_rng(12)
    models = [synth.rigid_model(15.0, (0, 1, 0), (0.05, 0.0, 0.1)), synth.rigid_model(-20.0, (1, 0, 0), (0.0, 0.05, -0.1))]
    gC = rng.standard_normal((3, cam.H, cam.W))
    gA = rng.standard_normal((cam.H, cam.W))
    xs = (np.arange(cam.W)[None, :] + 0.5) / cam.W
    depth = np.repeat(3.75 + 0.5 * xs, cam.H, axis=0).astype(np.float32)
    bg = (0.2, 0.4, 0.6)
    _, _, scenes, ws, d = _multi([s1, s2], models, cam, None, depth=depth, bg=bg)
    grads = [{k: torch.empty_like(s.tensors[k]) for k in vis.FIELDS} for s in scenes]
    vis.vis_render_backward_multi([s.handle for s in scenes], models, cam, cam.W, cam.H, bg,
                                  torch.from_numpy(gC.astype(np.float32)).cuda(),
                                  torch.from_numpy(gA.astype(np.float32)).cuda(), ws.buf, grads, None, depth=d)
    ref = oracle.adjoint_multi([s1, s2], models, cam, gC, gA, bg, depth=depth)
    free = oracle.adjoint_multi([s1, s2], models, cam, gC, gA, bg)
    assert not np.allclose(ref[0]["means"], free[0]["means"])
    for k_s in range(2):
        for f in vis.FIELDS:
            a = grads[k_s][f].cpu().numpy().astype(np.float64).ravel()
            b = ref[k_s][f].ravel()
            assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), (k_s, f)
