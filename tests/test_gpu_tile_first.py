"""Tile-first ordering (sort_mode 3): copies placed in their tiles, each tile sorted in
shared memory by (depth bits, index). It must give the (tile, depth, index) order of the
64-bit key sort (sort_mode 0) bit for bit -- values, ranges and image -- including tiles
that go through the 1024 / 4096 / 16384-copy sorts and the merged runs above 16384."""
import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth
from gpu_helpers import image_parity, render_gpu, ws_view

pytestmark = pytest.mark.gpu


def _vals_ranges(ws):
    L = ws.layout()
    m = int(ws_view(ws, L.off_ctrl, 1, np.uint32)[0])
    vals = ws_view(ws, L.off_vals[L.sorted_buffer], m, np.uint32)
    nt = L.tiles_x * L.tiles_y
    ranges = ws_view(ws, L.off_ranges, 2 * nt, np.uint32).reshape(nt, 2)
    return vals, ranges, L


def _crowded_scene(n, seed, log_scale):
    """n Gaussians that all cover the whole (small) view: every tile lists ~n copies."""
    sc = synth.mixture_scene(n, seed, sh_degree=0, ball_radius=0.3, comp_std=0.2, log_scale_mean=log_scale,
                             log_scale_std=0.1)
    return sc


@pytest.mark.parametrize("case", [
    ("mixture 301x187 t8", None, 301, 187, 8),
    ("mixture 1080p t16", None, 1920, 1080, 16),
    ("crowded 3k", 3000, 96, 64, 16),       # tiles of ~3000 copies (the 4096 sort)
    ("crowded 12k", 12000, 64, 48, 16),     # tiles of ~12000 copies (the 16384 sort)
    ("crowded 40k", 40000, 48, 32, 16),     # tiles of ~40000 copies: three runs, two merge rounds
])
def test_tile_first_equals_tile_depth_sort(case):
    name, crowd, W, H, tile = case
    if crowd:
        sc = _crowded_scene(crowd, 41, -0.5)
        cam = synth.look_at((0.0, 0.0, 4.0), (0, 0, 0), W, H, 50.0)
    else:
        sc = synth.mixture_scene(30000, 17, sh_degree=1, ball_radius=3.0, comp_std=0.5, log_scale_mean=-3.2)
        cam = synth.look_at((1.0, 2.0, 9.0), (0, 0, 0), W, H, 55.0)
    a_rgb, a_alpha, _, wa = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, sort_mode=0))
    b_rgb, b_alpha, _, wb = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, sort_mode=3))
    va, ra, _ = _vals_ranges(wa)
    vb, rb, Lb = _vals_ranges(wb)
    assert Lb.sort_mode == 3 and Lb.key_bytes == 8
    cnt = ra[:, 1] - ra[:, 0]
    if crowd:
        assert cnt.max() > {3000: 1024, 12000: 4096, 40000: 16384}[crowd], (name, int(cnt.max()))
    assert len(va) == len(vb) > 0
    assert np.array_equal(ra, rb), name
    assert np.array_equal(va, vb), name
    assert np.array_equal(a_rgb, b_rgb) and np.array_equal(a_alpha, b_alpha)


def test_tile_first_small_workload_parity():
    sc, cams = synth.workload_small()
    rgb, alpha, _, _ = render_gpu(sc, cams[0], opts=vis.make_opts(sort_mode=3))
    ref, _ = oracle.render(sc, cams[0])
    image_parity(rgb, alpha, ref)


def test_tile_first_all_culled_and_single_tile():
    sc, cams = synth.workload_small()
    dead = dict(sc, opacity_logits=np.full_like(sc["opacity_logits"], -30.0))
    rgb, alpha, _, ws = render_gpu(dead, cams[0], (0.5, 0.5, 0.5), vis.make_opts(sort_mode=3))
    assert np.all(alpha == 0.0) and vis.vis_check(ws.buf) == 0
    cam = synth.look_at((0, 0, 4), (0, 0, 0), 12, 10, 60.0)   # one tile
    rgb, alpha, _, _ = render_gpu(sc, cam, opts=vis.make_opts(sort_mode=3))
    ref, _ = oracle.render(sc, cam)
    image_parity(rgb, alpha, ref)


def test_tile_first_gradients_match_oracle():
    import torch
    sc, cam = synth.fd_scene()
    rng = np.random.default_rng(9)
    gC = rng.standard_normal((3, cam.H, cam.W))
    gA = rng.standard_normal((cam.H, cam.W))
    opts = vis.make_opts(sort_mode=3)
    _, _, s, ws = render_gpu(sc, cam, (0, 0, 0), opts)
    grads = {k: torch.empty_like(s.tensors[k]) for k in vis.FIELDS}
    vis.vis_render_backward(s.handle, cam, cam.W, cam.H, (0, 0, 0),
                            torch.from_numpy(gC.astype(np.float32)).cuda(),
                            torch.from_numpy(gA.astype(np.float32)).cuda(), ws.buf, grads, opts)
    ref = oracle.adjoint(sc, cam, gC, gA)
    for k in vis.FIELDS:
        a = grads[k].cpu().numpy().astype(np.float64).ravel()
        b = ref[k].ravel()
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(b), k


def test_tile_first_capacity_error_then_retry():
    sc_np, cams = synth.workload_small()
    cam = cams[0]
    opts = vis.make_opts(sort_mode=3)
    s = vis.Scene.from_numpy(sc_np)
    ws = vis.Workspace(s.n, cam.W, cam.H, key_capacity=100, opts=opts)
    rgb, alpha = vis._render_checked(s, cam, cam.W, cam.H, (0, 0, 0), ws, opts)
    assert ws.key_capacity > 100
    ref, _ = oracle.render(sc_np, cam)
    image_parity(rgb.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64), ref)
