"""Pre-packed FP16 scenes (Algorithm 1's pre-pack; section 3.4's FP16 layout): the renderer
reading fp16 planes against the FP64 oracle run on the values those planes decode to (the
planes are built on the host by the oracle's prepack, so no oracle input comes from the
GPU), and the GPU's own pack kernel against the host packing."""
import math

import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth
from gpu_helpers import image_parity

pytestmark = pytest.mark.gpu

BG = (0.1, 0.2, 0.3)


def _packed_render(sc_np, cam, opts=None, bg=BG):
    planes, dec = oracle.prepack(sc_np)
    ps = vis.PackedScene.from_planes(planes, sc_np["sh_degree"])
    ws = vis.Workspace(ps.n, cam.W, cam.H, opts=opts)
    rgb, alpha = vis._render_checked(ps, cam, cam.W, cam.H, bg, ws, opts)
    return rgb.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64), dec, ps, ws


@pytest.mark.parametrize("opts", [dict(), dict(sort_mode=0), dict(tile=8),
                                  dict(pixels_per_thread=2)])
def test_packed_small_workload_parity(opts):
    sc, cams = synth.workload_small()
    rgb, alpha, dec, *_ = _packed_render(sc, cams[0], vis.make_opts(**opts))
    ref, _ = oracle.render(dec, cams[0], BG)
    image_parity(rgb, alpha, ref)


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_packed_mixture_parity(deg):
    """A 60k-Gaussian mixture at 960x540 (the large-scene recipe at 1/16 of the 1M size)."""
    sc = synth.mixture_scene(60_000, 90 + deg, sh_degree=deg, hi_std=0.2)
    cam = synth.orbit_cameras(4, 15.0, 960, 540, 50.0)[deg]
    rgb, alpha, dec, *_ = _packed_render(sc, cam)
    ref, prep = oracle.render(dec, cam, BG)
    assert prep["valid"].sum() > 20_000
    image_parity(rgb, alpha, ref)


def test_packed_needles_parity():
    """Strongly anisotropic Gaussians (scale ratios up to ~e^3): the unfactored fp16
    covariance goes through the cofactor form of the projected determinant."""
    sc = synth.mixture_scene(20_000, 95, sh_degree=1, components=16, ball_radius=2.0, log_scale_mean=-3.0,
                             log_scale_std=1.2)
    cam = synth.look_at((0.5, 0.5, 6.0), (0, 0, 0), 512, 384, 50.0)
    rgb, alpha, dec, *_ = _packed_render(sc, cam)
    ref, _ = oracle.render(dec, cam, BG)
    image_parity(rgb, alpha, ref)


def test_packed_scenes_in_a_multi_render():
    scs, models, cam = synth.workload_multi(scale=0.01, W=480, H=270, seed=7)
    packed = [oracle.prepack(s) for s in scs]
    ps = [vis.PackedScene.from_planes(pl, s["sh_degree"]) for (pl, _), s in zip(packed, scs)]
    ws = vis.multi_workspace(ps, cam.W, cam.H)
    rgb, alpha = vis._render_multi_checked(ps, models, cam, cam.W, cam.H, BG, ws, None)
    ref, _ = oracle.render_multi([d for _, d in packed], list(models), cam, BG)
    image_parity(rgb.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64), ref)


def _halves(words):
    return np.ascontiguousarray(words).view(np.uint32).view(np.float16).astype(np.float64)


def test_gpu_pack_matches_host_packing():
    """vis_scene_pack: the SH planes and means bit for bit; alpha and the covariance (float
    arithmetic on the GPU, FP64 on the host) differ at most by one fp16 step, and only where
    the exact value lies within float rounding of the midpoint between two halves."""
    import torch
    sc = synth.mixture_scene(30_000, 99, sh_degree=3, log_scale_std=1.0)
    s = vis.Scene.from_numpy(sc)
    ps = vis.PackedScene.pack(s)
    torch.cuda.synchronize()
    planes, dec = oracle.prepack(sc)
    got = {k: ps.planes[k].cpu().numpy().view(np.uint32) for k in ("pos", "cov", "col")}
    assert np.array_equal(got["col"], planes["col"])
    gpos, hpos = _halves(got["pos"]), _halves(planes["pos"])
    assert np.array_equal(gpos[:, :3], hpos[:, :3])
    sig = oracle.covariance(sc["log_scales"], sc["quats"])
    exact = dict(alpha=1.0 / (1.0 + np.exp(-sc["opacity_logits"].astype(np.float64))),
                 cov=np.stack([sig[:, 0, 0], sig[:, 0, 1], sig[:, 0, 2], sig[:, 1, 1], sig[:, 1, 2], sig[:, 2, 2]], 1))
    scale = dict(alpha=np.ones(30_000), cov=np.max(np.abs(exact["cov"]), axis=1))
    for key, g, h in (("alpha", gpos[:, 3], hpos[:, 3]), ("cov", _halves(got["cov"]), _halves(planes["cov"]))):
        bad = g != h
        assert bad.mean() < 1e-3, key
        if not bad.any():
            continue
        e = exact[key][bad]
        tol = 2e-6 * (scale[key][bad] if key == "alpha" else np.broadcast_to(scale[key][:, None], bad.shape)[bad])
        g16, h16 = g[bad].astype(np.float16), h[bad].astype(np.float16)
        assert np.array_equal(np.nextafter(h16, g16), g16), key                 # adjacent halves
        assert np.all(np.abs(e - 0.5 * (g[bad] + h[bad])) <= tol + 1e-12), key   # a near tie
    # and the packed render of the GPU's planes matches the fp32 scene's to fp16 accuracy
    cam = synth.orbit_cameras(2, 15.0, 480, 270, 50.0)[0]
    ws = vis.Workspace(s.n, cam.W, cam.H)
    a, _ = vis._render_checked(ps, cam, cam.W, cam.H, BG, ws, None)
    b, _ = vis._render_checked(s, cam, cam.W, cam.H, BG, ws, None)
    assert float((a - b).abs().mean()) < 2e-3


def test_packed_scene_has_no_gradients():
    import torch
    sc, cams = synth.workload_small()
    rgb, alpha, dec, ps, ws = _packed_render(sc, cams[0])
    cam = cams[0]
    g = {k: torch.zeros(1, device="cuda").expand(16).contiguous() for k in vis.FIELDS}
    with pytest.raises(vis.VisError) as e:
        vis.vis_render_backward(ps.handle, cam, cam.W, cam.H, BG, torch.zeros((3, cam.H, cam.W), device="cuda"),
                                torch.zeros((cam.H, cam.W), device="cuda"), ws.buf, g)
    assert e.value.status == vis.VIS_ERR_UNSUPPORTED


def test_packed_scenes_through_the_python_renderers():
    """vis.render and vis.render_multi take packed scenes (forward only) and give the images of
    the plain calls."""
    import torch
    sc, cams = synth.workload_small()
    cam = cams[0]
    rgb, alpha, dec, ps, ws = _packed_render(sc, cam)
    r2, a2 = vis.render(ps, cam, cam.W, cam.H, BG)
    assert not r2.requires_grad
    assert np.array_equal(r2.cpu().numpy().astype(np.float64), rgb)
    assert np.array_equal(a2.cpu().numpy().astype(np.float64), alpha)
    plain = vis.Scene.from_numpy(sc)
    M = np.stack([synth.rigid_model(0.0, (0, 1, 0), (0.5, 0.0, 0.0)), synth.rigid_model(0.0, (0, 1, 0), (-0.5, 0.0, 0.0))])
    r3, a3 = vis.render_multi([ps, plain], M, cam, cam.W, cam.H, BG)
    ref, _ = oracle.render_multi([dec, sc], list(M), cam, BG)
    image_parity(r3.cpu().numpy().astype(np.float64), a3.cpu().numpy().astype(np.float64), ref)
    torch.cuda.synchronize()


def test_thresholds_at_equality_on_the_gpu():
    """The decisions at exact equality, as the oracle takes them: a splat whose alpha equals
    alpha_min is composited (a pre-packed opacity equal to the alpha_min option, on a pixel
    centre: q = 0), and a splat whose depth equals the depth-buffer value passes the test."""
    import torch
    W = H = 33
    cam = synth.look_at((0, 0, 4.0), (0, 0, 0), W, H, 60.0)
    amin = float(np.float16(1.0 / 255.0))
    sc = synth.uniform_cube_scene(1, 0, sh_degree=0, extent=0.0, log_scale_mean=math.log(0.05), log_scale_std=0.0)
    planes, dec = oracle.prepack(sc)
    dec = dict(dec, opacity=np.array([amin]))
    planes["pos"] = planes["pos"].copy()
    planes["pos"][0, 1] = (planes["pos"][0, 1] & 0xFFFF) | (int(np.array([amin], np.float16).view(np.uint16)[0]) << 16)
    ps = vis.PackedScene.from_planes(planes, 0)
    opts = vis.make_opts(alpha_min=amin)
    ws = vis.Workspace(1, W, H, opts=opts)
    rgb, alpha = vis._render_checked(ps, cam, W, H, BG, ws, opts)
    ref, prep = oracle.render(dec, cam, BG, opts=dict(alpha_min=amin))
    assert prep["uv"][0, 0] == W / 2 and ref["n_contrib"][H // 2, W // 2] == 1
    g = alpha.cpu().numpy().astype(np.float64)
    assert abs(g[H // 2, W // 2] - amin) <= 1e-7 and abs(ref["alpha"][H // 2, W // 2] - amin) <= 1e-12
    # depth equality: the buffer holds the splat's own float32 view depth
    s = vis.Scene.from_numpy(sc)
    free, fa = vis._render_checked(s, cam, W, H, BG, vis.Workspace(1, W, H), None)
    z = float(oracle.preprocess(sc, cam)["zkey"][0])
    d = torch.full((H, W), z, dtype=torch.float32, device="cuda")
    eq, ea = vis._render_checked(s, cam, W, H, BG, vis.Workspace(1, W, H), None, depth=d)
    assert torch.equal(eq, free) and torch.equal(ea, fa) and float(fa.max()) > 0.1


def test_packed_scenes_against_a_depth_buffer():
    """Pre-packed scenes behind a slanted depth wall, alone and as transformed models of one
    image (the packed, model-folded and occlusion-culled preprocess variants together)."""
    import torch
    sc = synth.mixture_scene(20_000, 97, sh_degree=2, components=16, ball_radius=1.5, comp_std=0.5,
                             log_scale_mean=-3.5)
    cam = synth.look_at((0.0, 0.0, 4.5), (0, 0, 0), 480, 270, 50.0)
    xs = (np.arange(cam.W)[None, :] + 0.5) / cam.W - 0.5
    depth = np.repeat(4.5 + 1.0 * xs, cam.H, axis=0).astype(np.float32)
    d = torch.from_numpy(depth).cuda()
    planes, dec = oracle.prepack(sc)
    ps = vis.PackedScene.from_planes(planes, 2)
    ws = vis.Workspace(ps.n, cam.W, cam.H)
    rgb, alpha = vis._render_checked(ps, cam, cam.W, cam.H, BG, ws, None, depth=d)
    ref, _ = oracle.render(dec, cam, BG, depth=depth)
    free, _ = oracle.render(dec, cam, BG)
    assert np.abs(ref["rgb"] - free["rgb"]).max() > 0.05
    image_parity(rgb.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64), ref)
    scs, models, mcam = synth.workload_multi(scale=0.01, W=480, H=270, seed=8)
    packed = [oracle.prepack(s) for s in scs]
    pss = [vis.PackedScene.from_planes(pl, s["sh_degree"]) for (pl, _), s in zip(packed, scs)]
    mdepth = np.repeat(12.0 + 4.0 * (xs + 0.5), mcam.H, axis=0).astype(np.float32)
    mws = vis.multi_workspace(pss, mcam.W, mcam.H)
    r2, a2 = vis._render_multi_checked(pss, models, mcam, mcam.W, mcam.H, BG, mws, None,
                                       depth=torch.from_numpy(mdepth).cuda())
    ref2, _ = oracle.render_multi([dd for _, dd in packed], list(models), mcam, BG, depth=mdepth)
    image_parity(r2.cpu().numpy().astype(np.float64), a2.cpu().numpy().astype(np.float64), ref2)
