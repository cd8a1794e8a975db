"""Depth-buffer-aware compositing on the GPU (vis_render_depth / vis_render_backward_depth):
a splat deeper than a pixel's depth-buffer value is not composited there. Parity with the
FP64 oracle's depth-tested definition, the +inf identity, and the adjoint."""
import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth
from gpu_helpers import image_parity

pytestmark = pytest.mark.gpu


def _render(sc_np, cam, depth, opts=None, bg=(0.1, 0.2, 0.3)):
    import torch
    sc = vis.Scene.from_numpy(sc_np)
    ws = vis.Workspace(sc.n, cam.W, cam.H, opts=opts)
    d = None if depth is None else torch.from_numpy(np.ascontiguousarray(depth, np.float32)).cuda()
    rgb, alpha = vis._render_checked(sc, cam, cam.W, cam.H, bg, ws, opts, depth=d)
    return rgb.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64), sc, ws, d


def _slanted(cam, z0, slope):
    """A plane of view depths z0 + slope * (x / W - 0.5) across the image."""
    xs = (np.arange(cam.W)[None, :] + 0.5) / cam.W - 0.5
    return np.repeat(z0 + slope * xs, cam.H, axis=0).astype(np.float32)


@pytest.mark.parametrize("opts", [dict(), dict(pixels_per_thread=2), dict(tile=8), dict(tile=32, sort_mode=0)])
def test_infinite_depth_buffer_is_the_plain_render(opts):
    sc, cams = synth.workload_small()
    cam = cams[0]
    o = vis.make_opts(**opts)
    a_rgb, a_alpha, *_ = _render(sc, cam, None, o)
    b_rgb, b_alpha, *_ = _render(sc, cam, np.full((cam.H, cam.W), np.inf, np.float32), o)
    assert np.array_equal(a_rgb, b_rgb) and np.array_equal(a_alpha, b_alpha)


@pytest.mark.parametrize("opts", [dict(), dict(pixels_per_thread=2), dict(tile=8)])
def test_depth_buffer_parity_with_oracle(opts):
    sc, cams = synth.workload_small()
    cam = cams[0]                                   # scene depths ~3..5 from (0, 0, 4)
    depth = _slanted(cam, 4.0, 1.5)
    rgb, alpha, *_ = _render(sc, cam, depth, vis.make_opts(**opts))
    ref, _ = oracle.render(sc, cam, (0.1, 0.2, 0.3), depth=depth)
    free, _ = oracle.render(sc, cam, (0.1, 0.2, 0.3))
    assert np.abs(ref["rgb"] - free["rgb"]).max() > 0.1      # the buffer hides part of the scene
    image_parity(rgb, alpha, ref)


def test_depth_wall_in_front_gives_background():
    sc, cams = synth.workload_small()
    cam = cams[0]
    rgb, alpha, *_ = _render(sc, cam, np.full((cam.H, cam.W), 0.5, np.float32))
    assert np.all(alpha == 0.0)
    assert np.all(rgb == np.asarray((0.1, 0.2, 0.3), np.float32)[:, None, None].astype(np.float64))


def test_depth_buffer_gradients_match_oracle():
    import torch
    sc, cam = synth.fd_scene()
    rng = np.random.default_rng(23)
    gC = rng.standard_normal((3, cam.H, cam.W))
    gA = rng.standard_normal((cam.H, cam.W))
    depth = _slanted(cam, 4.0, 0.5)
    opts = vis.make_opts()
    _, _, s, ws, d = _render(sc, cam, depth, opts, bg=(0.2, 0.4, 0.6))
    grads = {k: torch.empty_like(s.tensors[k]) for k in vis.FIELDS}
    vis.vis_render_backward(s.handle, cam, cam.W, cam.H, (0.2, 0.4, 0.6),
                            torch.from_numpy(gC.astype(np.float32)).cuda(),
                            torch.from_numpy(gA.astype(np.float32)).cuda(), ws.buf, grads, opts, depth=d)
    ref = oracle.adjoint(sc, cam, gC, gA, (0.2, 0.4, 0.6), depth=depth)
    free = oracle.adjoint(sc, cam, gC, gA, (0.2, 0.4, 0.6))
    assert not np.allclose(ref["means"], free["means"])
    for k in vis.FIELDS:
        a = grads[k].cpu().numpy().astype(np.float64).ravel()
        b = ref[k].ravel()
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), k


def test_autograd_render_with_depth():
    import torch
    sc_np, cam = synth.fd_scene()
    sc = vis.Scene.from_numpy(sc_np)
    for k in vis.FIELDS:
        sc.tensors[k].requires_grad_(True)
    depth = torch.from_numpy(_slanted(cam, 4.0, 0.5)).cuda()
    rgb, alpha = vis.render(sc, cam, cam.W, cam.H, depth=depth)
    ref, _ = oracle.render(sc_np, cam, depth=depth.cpu().numpy())
    image_parity(rgb.detach().cpu().numpy().astype(np.float64), alpha.detach().cpu().numpy().astype(np.float64),
                 ref)
    (rgb.sum() + alpha.sum()).backward()
    assert all(torch.isfinite(sc.tensors[k].grad).all() for k in vis.FIELDS)


def test_depth_buffer_special_values():
    """-inf rejects every splat, +inf and NaN none; mixed per pixel, with a wall region."""
    sc, cams = synth.workload_small()
    cam = cams[0]
    ys, xs = np.mgrid[0:cam.H, 0:cam.W]
    depth = np.full((cam.H, cam.W), np.inf, np.float32)
    depth[xs < 64] = -np.inf
    depth[(xs >= 64) & (xs < 128)] = np.nan
    depth[xs >= 192] = 3.9                                 # a wall through the scene
    rgb, alpha, *_ = _render(sc, cam, depth)
    ref, _ = oracle.render(sc, cam, (0.1, 0.2, 0.3), depth=depth)
    image_parity(rgb, alpha, ref)
    assert np.all(alpha[:, :64] == 0.0)
    free_rgb, free_alpha, *_ = _render(sc, cam, None)
    assert np.array_equal(rgb[:, :, 64:192], free_rgb[:, :, 64:192])


@pytest.mark.parametrize("z", [3.0, 4.0, 5.5])
def test_depth_wall_culling_matches_oracle(z):
    """A wall at several depths over a 30k mixture at 480x270 (the tile lists are cut at the
    first chunk beyond every limit in the tile); pixels are compared with the oracle."""
    sc = synth.mixture_scene(30_000, 5, sh_degree=2, components=16, ball_radius=1.5, comp_std=0.5,
                             log_scale_mean=-3.5)
    cam = synth.look_at((0.0, 0.0, 4.5), (0, 0, 0), 480, 270, 50.0)
    depth = _slanted(cam, z, 1.0)
    rgb, alpha, *_ = _render(sc, cam, depth)
    ref, _ = oracle.render(sc, cam, (0.1, 0.2, 0.3), depth=depth)
    image_parity(rgb, alpha, ref)
