"""Forward parity of the CUDA path (through the C ABI) against the FP64 oracle.

Bars: per-Gaussian preprocess within float32 rounding; (tile, depth, index) keys,
sort permutation and tile ranges bit-exact; images max-abs <= 2e-4 on pixels the
oracle does not flag as decided within float32 rounding of a threshold, mean-abs
<= 1e-5 per channel on all pixels.
"""
import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth
from gpu_helpers import gpu_stage_outputs, image_parity, render_gpu, ws_view

pytestmark = pytest.mark.gpu


def test_small_workload_image_parity():
    sc, cams = synth.workload_small()
    cam = cams[0]
    rgb, alpha, _, _ = render_gpu(sc, cam)
    ref, _ = oracle.render(sc, cam)
    image_parity(rgb, alpha, ref)


@pytest.mark.parametrize("ppt", [1, 2])
@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_ragged_image_all_tiles_and_degrees(tile, deg, ppt):
    sc = synth.mixture_scene(4000, 100 + deg, sh_degree=deg, ball_radius=2.0, comp_std=0.4,
                             log_scale_mean=-3.0)
    cam = synth.look_at((2.0, 1.0, 7.0), (0, 0, 0), 203, 117, 55.0)
    bg = (0.2, 0.45, 0.7)
    opts = dict(tile=tile)
    rgb, alpha, _, _ = render_gpu(sc, cam, bg, vis.make_opts(tile=tile, pixels_per_thread=ppt))
    ref, _ = oracle.render(sc, cam, bg, opts)
    image_parity(rgb, alpha, ref)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_two_pixels_per_thread_bit_identical(tile):
    """The packed two-pixel compositor rounds each pixel as the one-pixel compositor does:
    images, final transmittance and last composited positions are identical bit for bit."""
    sc = synth.mixture_scene(200_000, 17, sh_degree=3)
    cam = synth.look_at((0.0, 2.0, 14.0), (0, 0, 0), 1001, 603, 50.0)
    out = []
    for ppt in (1, 2):
        rgb, alpha, s, ws = render_gpu(sc, cam, (0.3, 0.2, 0.1), vis.make_opts(tile=tile, pixels_per_thread=ppt))
        L = ws.layout()
        npx = cam.W * cam.H
        out.append((rgb, alpha, ws_view(ws, L.off_tfinal, npx, np.float32), ws_view(ws, L.off_last, npx, np.int32)))
    assert (out[0][2] < 1.0).mean() > 0.3   # the view covers a good part of the image
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("ppt", [1, 2])
def test_tile_size_does_not_change_the_image(ppt):
    """Every pixel composites the same splats in the same depth order whatever the tile size,
    so 8-, 16- and 32-pixel tiles (the last composited by four 16 x 16 CTAs per tile, each
    walking the whole tile's list) agree up to rounding: a splat's centre is staged relative
    to its tile's centre, which rounds differently per tile size, and on a few pixels that
    last bit flips a cut or stop decision (the ambiguous pixels of the oracle parity). A square
    placed or masked wrongly would drop splats from whole warp blocks, far beyond these bounds."""
    sc = synth.mixture_scene(200_000, 29, sh_degree=3)
    cam = synth.look_at((1.0, 2.5, 13.0), (0, 0, 0), 1001, 603, 50.0)
    out = []
    for tile in (8, 16, 32):
        rgb, alpha, s, ws = render_gpu(sc, cam, (0.3, 0.2, 0.1), vis.make_opts(tile=tile, pixels_per_thread=ppt))
        L = ws.layout()
        out.append((rgb, alpha, ws_view(ws, L.off_tfinal, cam.W * cam.H, np.float32)))
    assert (out[0][2] < 1.0).mean() > 0.3
    for other in out[1:]:
        for a, b in zip(out[0], other):
            d = np.abs(a.astype(np.float64) - b.astype(np.float64))
            assert (d > 1e-5).mean() <= 1e-4 and d.mean() <= 1e-7 and d.max() <= 5e-3, \
                ((d > 1e-5).mean(), d.mean(), d.max())


def _stage_inputs():
    sc, cams = synth.workload_small()
    return sc, cams[0]


def test_preprocess_stage_matches_oracle():
    sc, cam = _stage_inputs()
    _, _, s, ws = render_gpu(sc, cam, opts=vis.make_opts(sort_mode=0, tile_extent=0))
    g = gpu_stage_outputs(s, ws)
    o = oracle.preprocess(sc, cam)
    both = (g["valid"] == 1) & (o["valid"] == 1)
    assert (g["valid"] != o["valid"]).sum() <= 2
    assert both.sum() > 1000
    np.testing.assert_allclose(g["uv"][both], o["uv"][both], atol=2e-5)
    scale = np.abs(o["conic"][both]).max(axis=1, keepdims=True)
    assert np.all(np.abs(g["conic"][both] - o["conic"][both]) <= 2e-5 * scale)
    np.testing.assert_allclose(g["opacity"][both], o["opacity"][both], rtol=1e-6)
    np.testing.assert_allclose(g["rgb"][both], o["rgb"][both], atol=2e-6)
    assert (g["zkey"][both] == o["zkey"][both]).mean() > 0.999
    assert (g["rect"][both] != o["rect"][both]).any(axis=1).sum() <= 2


def _expected_keys(o, tiles_x, keep):
    valid = np.where(keep, o["valid"], 0).astype(np.int32)
    k, v = oracle.duplicate_raw(valid, o["rect"], o["zkey"], tiles_x)
    return oracle.stable_sort_pairs(k, v)


def test_keys_sort_and_ranges_bitexact():
    sc, cam = _stage_inputs()
    _, _, s, ws = render_gpu(sc, cam, opts=vis.make_opts(sort_mode=0, tile_extent=0))
    g = gpu_stage_outputs(s, ws)
    o = oracle.preprocess(sc, cam)
    # Gaussians whose float32 decisions differ from FP64 (rect edge, cull) are set aside
    same = ((g["valid"] == o["valid"]) & (g["zkey"] == o["zkey"])
            & ((g["rect"] == o["rect"]).all(axis=1) | (o["valid"] == 0)))
    assert (~same).sum() <= 3
    L = g["layout"]
    ek, ev = _expected_keys(o, L.tiles_x, same)
    keep = same[g["vals"]]
    assert np.array_equal(g["keys"][keep], ek)
    assert np.array_equal(g["vals"][keep], ev)
    # every sorted run is one tile's range, and the ranges cover the keys exactly
    tiles = (g["keys"] >> np.uint64(32)).astype(np.int64)
    assert np.all(np.diff(g["keys"].astype(np.uint64)) >= 0) or np.all(g["keys"][1:] >= g["keys"][:-1])
    for t in np.unique(tiles):
        idx = np.nonzero(tiles == t)[0]
        assert (g["ranges"][t, 0], g["ranges"][t, 1]) == (idx[0], idx[-1] + 1)
    empty = np.setdiff1d(np.arange(L.tiles_x * L.tiles_y), np.unique(tiles))
    assert np.all(g["ranges"][empty, 0] == g["ranges"][empty, 1])
    if (~same).sum() == 0:
        assert np.array_equal(g["ranges"], oracle.tile_ranges(ek, L.tiles_x * L.tiles_y))


def test_all_culled_gives_background():
    sc, cams = synth.workload_small()
    sc = dict(sc)
    sc["opacity_logits"] = np.full_like(sc["opacity_logits"], -30.0)
    bg = (0.25, 0.5, 0.75)
    rgb, alpha, _, ws = render_gpu(sc, cams[0], bg)
    assert np.all(rgb == np.asarray(bg, np.float32)[:, None, None].astype(np.float64))
    assert np.all(alpha == 0.0)
    assert vis.vis_check(ws.buf) == 0


def test_camera_facing_away_gives_background():
    sc, _ = synth.workload_small()
    cam = synth.look_at((0, 0, 4), (0, 0, 8), 64, 48, 60.0)   # scene is behind the camera
    rgb, alpha, _, ws = render_gpu(sc, cam, (0.1, 0.2, 0.3))
    assert np.all(alpha == 0.0)
    assert vis.vis_check(ws.buf) == 0


def test_single_gaussian_and_tiny_image():
    sc = synth.uniform_cube_scene(1, 3, sh_degree=1, log_scale_mean=-1.5)
    sc["means"][:] = 0.0
    for W, H in ((1, 1), (5, 3), (17, 33)):
        cam = synth.look_at((0, 0, 4), (0, 0, 0), W, H, 60.0)
        rgb, alpha, _, _ = render_gpu(sc, cam, (0.3, 0.3, 0.3))
        ref, _ = oracle.render(sc, cam, (0.3, 0.3, 0.3))
        image_parity(rgb, alpha, ref)


def test_render_is_deterministic():
    sc, cams = synth.workload_small()
    a, aa, _, _ = render_gpu(sc, cams[0])
    b, bb, _, _ = render_gpu(sc, cams[0])
    assert np.array_equal(a, b) and np.array_equal(aa, bb)


def test_capacity_error_then_retry():
    torch = pytest.importorskip("torch")
    sc_np, cams = synth.workload_small()
    cam = cams[0]
    sc = vis.Scene.from_numpy(sc_np)
    ws = vis.Workspace(sc.n, cam.W, cam.H, key_capacity=64)
    rgb = torch.empty((3, cam.H, cam.W), device="cuda")
    alpha = torch.empty((cam.H, cam.W), device="cuda")
    vis.vis_render(sc.handle, cam, cam.W, cam.H, (0, 0, 0), rgb, alpha, ws.buf)
    with pytest.raises(vis.VisError) as e:
        vis.vis_check(ws.buf)
    assert e.value.status == vis.VIS_ERR_CAPACITY
    need = e.value.num_keys
    assert need > 64
    ws.grow(need)
    vis.vis_render(sc.handle, cam, cam.W, cam.H, (0, 0, 0), rgb, alpha, ws.buf)
    assert vis.vis_check(ws.buf) == need
    ref, _ = oracle.render(sc_np, cam)
    image_parity(rgb.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64), ref)


def test_host_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    sc_np, cams = synth.workload_small()
    sc = vis.Scene.from_numpy(sc_np)
    cam = cams[0]
    ws = vis.Workspace(sc.n, cam.W, cam.H)
    rgb = torch.empty((3, cam.H, cam.W), device="cuda")
    alpha = torch.empty((cam.H, cam.W), device="cuda")
    bad = vis.make_camera(cam)
    bad.fx = float("nan")
    with pytest.raises(vis.VisError) as e:
        vis.vis_render(sc.handle, bad, cam.W, cam.H, (0, 0, 0), rgb, alpha, ws.buf)
    assert e.value.status == vis.VIS_ERR_INVALID_ARG
    with pytest.raises(vis.VisError):
        vis.vis_render(sc.handle, cam, 0, cam.H, (0, 0, 0), rgb, alpha, ws.buf)
    with pytest.raises(vis.VisError):
        vis.vis_render(sc.handle, cam, cam.W, cam.H, (0, 0, 0), rgb, alpha, ws.buf, vis.make_opts(tile=12))
    misaligned = torch.empty(sc.n * 3 + 1, device="cuda")[1:]
    with pytest.raises(vis.VisError):
        vis.vis_scene_upload(misaligned, sc.tensors["log_scales"], sc.tensors["quats"],
                             sc.tensors["opacity_logits"], sc.tensors["sh"], 0)
    with pytest.raises(vis.VisError):
        vis.vis_scene_upload(*[sc.tensors[k] for k in vis.FIELDS], 4)


def _sampled_tile_parity(sc, cam, n_tiles=48, seed=0):
    """Parity at full size on a random sample of whole tiles (plus the four corners)."""
    rgb, alpha, _, _ = render_gpu(sc, cam)
    tiles_x, tiles_y = (cam.W + 15) // 16, (cam.H + 15) // 16
    rng = np.random.default_rng(seed)
    pick = set(rng.choice(tiles_x * tiles_y, n_tiles, replace=False).tolist())
    pick |= {0, tiles_x - 1, (tiles_y - 1) * tiles_x, tiles_x * tiles_y - 1}
    mask = np.zeros(tiles_x * tiles_y, np.uint8)
    mask[list(pick)] = 1
    ref, _ = oracle.render(sc, cam, tile_mask=mask)
    sel = ~np.isnan(ref["alpha"])
    sub = dict(rgb=ref["rgb"][:, sel], alpha=ref["alpha"][sel], ambiguous=ref["ambiguous"][sel])
    return image_parity(rgb[:, sel], alpha[sel], sub)


@pytest.mark.slow
def test_1m_sh3_1080p_sampled_tiles():
    sc, cams = synth.workload_1m(views=32)
    for k in (0, 11):
        _sampled_tile_parity(sc, cams[k], seed=k)


@pytest.mark.slow
def test_6m_dynamic_frame_sampled_tiles():
    sc, extras, cams = synth.workload_dynamic()
    k = 60
    means, logits = synth.dynamic_frame_inputs(sc, extras, k)
    frame = dict(sc, means=means, opacity_logits=logits)
    _sampled_tile_parity(frame, cams[k], n_tiles=32, seed=3)


def test_compositor_statistics_do_not_change_the_image():
    sc, cams = synth.workload_small()
    a_rgb, a_alpha, _, _ = render_gpu(sc, cams[0])
    b_rgb, b_alpha, _, ws = render_gpu(sc, cams[0], opts=vis.make_opts(collect_stats=1))
    assert np.array_equal(a_rgb, b_rgb) and np.array_equal(a_alpha, b_alpha)
    c = vis.read_ctrl(ws.buf)
    ref, _ = oracle.render(sc, cams[0])
    # every composited pair is one the oracle composites too (up to flagged pixels)
    assert 0 < c["hits"] <= c["pair_tests"]
    assert abs(c["hits"] - int(ref["n_contrib"].sum())) <= max(10, 1e-4 * c["hits"])


def test_tile_order_is_a_longest_first_permutation():
    """The compositor's tile order: every tile once, by non-increasing key count up to the
    width of a bucket (two per octave)."""
    sc = synth.mixture_scene(300_000, 23, sh_degree=1)
    cam = synth.look_at((0.0, 3.0, 15.0), (0, 0, 0), 1280, 720, 50.0)
    _, _, s, ws = render_gpu(sc, cam)
    L = ws.layout()
    nt = L.tiles_x * L.tiles_y
    assert L.key_bytes == 2 and L.off_order > 0
    order = ws_view(ws, L.off_order, nt, np.uint32)
    assert np.array_equal(np.sort(order), np.arange(nt, dtype=np.uint32))
    ranges = ws_view(ws, L.off_ranges, 2 * nt, np.uint32).reshape(nt, 2).astype(np.int64)
    c = (ranges[:, 1] - ranges[:, 0])[order]
    assert c.max() > 100 and (c == 0).any()

    def bucket(x):   # 2 log2(x) rounded down to half octaves; empty tiles last
        lg = np.floor(np.log2(np.maximum(x, 1))).astype(np.int64)
        half = np.where(lg >= 1, (x >> np.maximum(lg - 1, 0)) & 1, 0)
        return np.where(x == 0, -1, 2 * lg + half)
    b = bucket(c)
    assert np.all(np.diff(b) <= 0)

