"""Depth-first sort mode (sort_mode = 1): depth sort of the surviving splats, then a
stable tile sort of their copies. It must give the same (tile, depth, index) order as
the 64-bit (tile, depth) key sort -- hence the same values, ranges and image, bit for
bit -- and pass the same oracle parity."""
import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth
from gpu_helpers import footprint_tiles, gpu_stage_outputs, image_parity, render_gpu, ws_view

pytestmark = pytest.mark.gpu


def _norm(ranges):
    """Empty tiles may be [s, s) for any s: compare them as [0, 0)."""
    r = ranges.copy()
    r[r[:, 0] == r[:, 1]] = 0
    return r


def _sorted_vals_and_ranges(sc, ws):
    L = ws.layout()
    m = int(ws_view(ws, L.off_ctrl, 1, np.uint32)[0])
    vals = ws_view(ws, L.off_vals[L.sorted_buffer], m, np.uint32)
    nt = L.tiles_x * L.tiles_y
    ranges = ws_view(ws, L.off_ranges, 2 * nt, np.uint32).reshape(nt, 2)
    return vals, ranges, L


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_depth_first_equals_tile_depth_sort(tile):
    sc = synth.mixture_scene(20000, 31, sh_degree=2, ball_radius=3.0, comp_std=0.5, log_scale_mean=-3.2)
    cam = synth.look_at((1.0, 2.0, 9.0), (0, 0, 0), 301, 187, 55.0)
    a_rgb, a_alpha, sa, wa = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, sort_mode=0))
    b_rgb, b_alpha, sb, wb = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, sort_mode=1))
    c_rgb, c_alpha, sc_, wc = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, sort_mode=1, tile_extent=0))
    d_rgb, d_alpha, sd, wd = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, sort_mode=1, tile_extent=1))
    # the tile extent only changes which tiles list a splat, never a pixel
    assert np.array_equal(c_rgb, b_rgb) and np.array_equal(c_alpha, b_alpha)
    assert np.array_equal(d_rgb, b_rgb) and np.array_equal(d_alpha, b_alpha)
    assert vis.vis_check(wb.buf) < vis.vis_check(wd.buf) < vis.vis_check(wc.buf)
    va, ra, La = _sorted_vals_and_ranges(sa, wa)
    vb, rb, Lb = _sorted_vals_and_ranges(sb, wb)
    assert La.key_bytes == 8 and Lb.key_bytes == 2 and Lb.sort_mode == 1
    assert np.array_equal(va, vb)
    assert np.array_equal(ra, rb)
    assert np.array_equal(a_rgb, b_rgb) and np.array_equal(a_alpha, b_alpha)


def _huge_splat_scene(n, seed):
    """A mixture scene whose first Gaussian covers the whole view (its copies span several
    4096-copy partitions of the tile binning)."""
    sc = synth.mixture_scene(n, seed, sh_degree=1, ball_radius=3.0, comp_std=0.5, log_scale_mean=-3.2)
    sc = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    sc["means"][0] = 0.0
    sc["log_scales"][0] = np.log(4.0)
    sc["opacity_logits"][0] = -2.0
    return sc


@pytest.mark.parametrize("shape", [
    ("one pass", 200, 150, 16, False),      # 130 tiles: the binning pass is the only pass
    ("two passes", 301, 187, 8, False),     # 912 tiles
    ("huge splat", 640, 480, 8, True),      # 4800 copies of one splat
    ("big grid", 1920, 1080, 8, False),     # 32400 tiles: 130 KB of per-tile counters
    ("unfused", 2048, 1632, 8, False),      # 52224 tiles: counters do not fit, 4-byte tile sort
])
def test_fused_binning_equals_tile_depth_sort(shape):
    name, W, H, tile, huge = shape
    sc = _huge_splat_scene(30000, 5) if huge else synth.mixture_scene(
        30000, 17, sh_degree=1, ball_radius=3.0, comp_std=0.5, log_scale_mean=-3.2)
    cam = synth.look_at((1.0, 2.0, 9.0), (0, 0, 0), W, H, 55.0)
    a_rgb, a_alpha, sa, wa = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, sort_mode=0))
    b_rgb, b_alpha, sb, wb = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, sort_mode=1))
    va, ra, La = _sorted_vals_and_ranges(sa, wa)
    vb, rb, Lb = _sorted_vals_and_ranges(sb, wb)
    nt = Lb.tiles_x * Lb.tiles_y
    assert Lb.key_bytes == (4 if nt > 51200 else 2), name
    assert Lb.sort_passes == (1 if nt <= 256 else (2 if nt <= 65536 else 3))
    if huge:
        assert int(ws_view(wb, Lb.off_touched, 1, np.uint32)[0]) == nt   # splat 0 lists every tile
    assert len(va) == len(vb) > 0
    assert np.array_equal(va, vb)
    assert np.array_equal(ra, rb)
    assert np.array_equal(a_rgb, b_rgb) and np.array_equal(a_alpha, b_alpha)


@pytest.mark.parametrize("tile", [8, 16])
def test_exact_row_footprint_covers_every_reachable_pixel(tile):
    """tile_extent 2: every tile holding a pixel centre where the FP64 oracle's splat
    passes q <= min(9, 2 ln(opacity / alpha_min)) is in the splat's footprint; the
    footprint's copies are as many as tiles touched; the image equals tile_extent 0's."""
    sc = synth.mixture_scene(4000, 23, sh_degree=0, ball_radius=2.0, comp_std=0.6, log_scale_mean=-2.6)
    cam = synth.look_at((0.5, 1.5, 6.0), (0, 0, 0), 197, 131, 55.0)
    a_rgb, a_alpha, sa, wa = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, tile_extent=2))
    b_rgb, b_alpha, _, _ = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, tile_extent=0))
    assert np.array_equal(a_rgb, b_rgb) and np.array_equal(a_alpha, b_alpha)
    g = gpu_stage_outputs(sa, wa)
    o = oracle.preprocess(sc, cam)
    L = g["layout"]
    tx = L.tiles_x
    px = np.arange(cam.W) + 0.5
    py = np.arange(cam.H) + 0.5
    trimmed = 0
    for i in np.nonzero((g["valid"] == 1) & (o["valid"] == 1))[0]:
        fp = footprint_tiles(g["rect"][i], g["trims"][i], tx)
        assert len(fp) == int(g["touched"][i])
        trimmed += g["trims"][i] != 0
        x0, y0, x1, y1 = g["rect"][i]
        u, v = o["uv"][i]
        a, b, c = o["conic"][i]
        thr = min(9.0, 2.0 * np.log(o["opacity"][i] * 255.0)) * (1.0 - 1e-5)
        xs = px[max(0, int(x0 * tile) - tile): min(cam.W, int(x1 * tile) + tile)]
        ys = py[max(0, int(y0 * tile) - tile): min(cam.H, int(y1 * tile) + tile)]
        dx = xs[None, :] - u
        dy = ys[:, None] - v
        q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
        yy, xx = np.nonzero(q <= thr)
        need = set(((ys[yy] // tile).astype(int) * tx + (xs[xx] // tile).astype(int)).tolist())
        assert need <= set(fp), (i, sorted(need - set(fp)))
    assert trimmed > 100


@pytest.mark.parametrize("mode", [0, 1])
def test_depth_first_small_workload_parity(mode):
    sc, cams = synth.workload_small()
    rgb, alpha, _, _ = render_gpu(sc, cams[0], opts=vis.make_opts(sort_mode=mode))
    ref, _ = oracle.render(sc, cams[0])
    image_parity(rgb, alpha, ref)


@pytest.mark.parametrize("mode", [0, 1])
def test_depth_first_all_culled_and_single_tile(mode):
    sc, cams = synth.workload_small()
    dead = dict(sc, opacity_logits=np.full_like(sc["opacity_logits"], -30.0))
    rgb, alpha, _, ws = render_gpu(dead, cams[0], (0.5, 0.5, 0.5), vis.make_opts(sort_mode=mode))
    assert np.all(alpha == 0.0) and vis.vis_check(ws.buf) == 0
    cam = synth.look_at((0, 0, 4), (0, 0, 0), 12, 10, 60.0)   # one tile
    rgb, alpha, _, _ = render_gpu(sc, cam, opts=vis.make_opts(sort_mode=mode))
    ref, _ = oracle.render(sc, cam)
    image_parity(rgb, alpha, ref)


@pytest.mark.parametrize("mode", [0, 1])
def test_depth_first_gradients_match_oracle(mode):
    import torch
    sc, cam = synth.fd_scene()
    rng = np.random.default_rng(8)
    gC = rng.standard_normal((3, cam.H, cam.W))
    gA = rng.standard_normal((cam.H, cam.W))
    opts = vis.make_opts(sort_mode=mode)
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


@pytest.mark.parametrize("mode", [0, 1])
def test_depth_first_capacity_error_then_retry(mode):
    sc_np, cams = synth.workload_small()
    cam = cams[0]
    opts = vis.make_opts(sort_mode=mode)
    s = vis.Scene.from_numpy(sc_np)
    ws = vis.Workspace(s.n, cam.W, cam.H, key_capacity=100, opts=opts)
    rgb, alpha = vis._render_checked(s, cam, cam.W, cam.H, (0, 0, 0), ws, opts)
    assert ws.key_capacity > 100
    ref, _ = oracle.render(sc_np, cam)
    image_parity(rgb.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64), ref)


@pytest.mark.parametrize("digit_bits", [10, 11])
@pytest.mark.parametrize("grid", [(1280, 720, 16), (2048, 1632, 8)])
def test_wide_radix_digits_equal_tile_depth_sort(digit_bits, grid):
    """The depth sort with 10- or 11-bit digits (32-bit keys in 4 or 3 passes, an odd count
    at 11 bits) and, on a grid beyond the 16-bit tile path, the 4-byte tile sort too: the
    same (tile, depth, index) order as the 64-bit key sort, bit for bit, over enough
    survivors to span hundreds of partitions."""
    W, H, tile = grid
    sc = synth.mixture_scene(300_000, 23, sh_degree=1, ball_radius=4.0, comp_std=0.6, log_scale_mean=-3.4)
    cam = synth.look_at((1.0, 2.0, 11.0), (0, 0, 0), W, H, 55.0)
    a_rgb, a_alpha, sa, wa = render_gpu(sc, cam, (0.1, 0.2, 0.3), vis.make_opts(tile=tile, sort_mode=0))
    b_rgb, b_alpha, sb, wb = render_gpu(sc, cam, (0.1, 0.2, 0.3),
                                        vis.make_opts(tile=tile, sort_mode=1, digit_bits=digit_bits))
    assert int(vis.read_ctrl(wb.buf)["num_visible"]) > 100_000
    va, ra, _ = _sorted_vals_and_ranges(sa, wa)
    vb, rb, Lb = _sorted_vals_and_ranges(sb, wb)
    assert np.array_equal(va, vb)
    assert np.array_equal(_norm(ra), _norm(rb))
    assert np.array_equal(a_rgb, b_rgb) and np.array_equal(a_alpha, b_alpha)
