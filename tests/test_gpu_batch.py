"""Batched render (vis_render_batch). The fused pipeline (lanes = 0: one preprocess over
the work list of (asset, camera) items; per group of images stacked on one tile canvas, one
depth sort of the group's survivors, one stable sort by canvas tile -- i.e. by (image, tile)
--, one compositor over the canvas) and the lane baseline (lanes >= 1: per-image renders on
concurrent streams) must both give every image bit-identical to vis_render of the same
(asset, camera, options), and so inherit its oracle parity; the fused images are also
checked against the oracle directly."""
import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth
from gpu_helpers import image_parity, render_gpu

pytestmark = pytest.mark.gpu


def _small_batch(assets=4, cams_per_asset=4, scale=0.01, seed=4):
    scenes_np, cams, cam_scene = synth.workload_batch(seed=seed, assets=assets, cams_per_asset=cams_per_asset,
                                                      scale=scale)
    return scenes_np, cams, cam_scene


def _equal_plain(b, scenes_np, cams, cam_scene, opts=None, bg=(0.1, 0.2, 0.3)):
    for i, cam in enumerate(cams):
        r, a, _, _ = render_gpu(scenes_np[cam_scene[i]], cam, bg, opts)
        assert np.array_equal(b.rgb[i].cpu().numpy().astype(np.float64), r), i
        assert np.array_equal(b.alpha[i].cpu().numpy().astype(np.float64), a), i


@pytest.mark.parametrize("lanes", [0, 1, 3, 8])
def test_batch_images_equal_plain_renders(lanes):
    scenes_np, cams, cam_scene = _small_batch()
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    b = vis.Batch(scenes, cams, cam_scene, lanes=lanes)
    b.render(bg=(0.1, 0.2, 0.3))
    for _ in range(2):              # graph replays give the same images
        b.launch(bg=(0.1, 0.2, 0.3))
    b.check()
    _equal_plain(b, scenes_np, cams, cam_scene)


@pytest.mark.parametrize("opts", [dict(tile=8), dict(tile=32, pixels_per_thread=2), dict(digit_bits=10),
                                  dict(digit_bits=11, tile=8), dict(pixels_per_thread=2, digit_bits=11)])
def test_fused_batch_options_equal_plain_renders(opts):
    """Every tile size, digit width and block shape the autotuner picks from: the same images."""
    scenes_np, cams, cam_scene = _small_batch(assets=3, cams_per_asset=3, scale=0.02, seed=7)
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    o = vis.make_opts(**opts)
    b = vis.Batch(scenes, cams, cam_scene, lanes=0, opts=o)
    b.render(bg=(0.1, 0.2, 0.3))
    _equal_plain(b, scenes_np, cams, cam_scene, opts=o)


def test_fused_batch_mixes_packed_and_plain_scenes():
    """Pre-packed (fp16) and fp32 assets in one fused batch: two preprocess work lists, one
    sort; each image equals the plain render of its own scene."""
    import torch
    scenes_np, cams, cam_scene = _small_batch(assets=4, cams_per_asset=2, scale=0.01, seed=9)
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    kinds = [vis.PackedScene.pack(s) if k % 2 else s for k, s in enumerate(scenes)]
    torch.cuda.synchronize()
    b = vis.Batch(kinds, cams, cam_scene, lanes=0)
    b.render(bg=(0.1, 0.2, 0.3))
    for i, cam in enumerate(cams):
        sc = kinds[cam_scene[i]]
        ws = vis.Workspace(scenes[cam_scene[i]].n, cam.W, cam.H)
        r, a = vis._render_checked(sc, cam, cam.W, cam.H, (0.1, 0.2, 0.3), ws, None)
        assert torch.equal(b.rgb[i], r) and torch.equal(b.alpha[i], a), i


def test_batch_oracle_parity_and_heterogeneous_degrees():
    scenes_np, cams, cam_scene = _small_batch(assets=3, cams_per_asset=2, scale=0.005)
    degs = {s["sh_degree"] for s in scenes_np}
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    b = vis.Batch(scenes, cams, cam_scene, lanes=0, opts=vis.make_opts(tile=8))
    b.render()
    for i in (0, len(cams) - 1):
        ref, _ = oracle.render(scenes_np[cam_scene[i]], cams[i], opts=dict(tile=8))
        image_parity(b.rgb[i].cpu().numpy().astype(np.float64), b.alpha[i].cpu().numpy().astype(np.float64), ref)
    assert len(degs) >= 1


@pytest.mark.parametrize("lanes", [0, 2])
def test_batch_capacity_error_is_reported_then_grown(lanes):
    scenes_np, cams, cam_scene = _small_batch(assets=2, cams_per_asset=2)
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    b = vis.Batch(scenes, cams, cam_scene, lanes=lanes, key_capacity=32)
    b.launch()
    with pytest.raises(vis.VisError) as e:
        b.check()
    assert e.value.status == vis.VIS_ERR_CAPACITY and e.value.num_keys > 32
    b.render()                       # grows the workspace and re-captures
    assert b.key_capacity > 32
    b.check()
    _equal_plain(b, scenes_np, cams, cam_scene, bg=(0.0, 0.0, 0.0))


def test_fused_batch_groups_and_oversized_image():
    """Many images fill several canvases (groups, on several streams), and an image of more
    tiles than a canvas holds (2048 x 1632 at 8-pixel tiles: 52224 tiles) is a group of its own
    with 32-bit tile ids: every image equals its plain render."""
    scenes_np, cams, cam_scene = _small_batch(assets=3, cams_per_asset=8, scale=0.01, seed=11)
    big = synth.look_at((0.0, 1.0, 6.0), (0, 0, 0), 2048, 1632, 55.0)
    cams = list(cams) + [big]
    cam_scene = list(cam_scene) + [1]
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    o = vis.make_opts(tile=8)
    b = vis.Batch(scenes, cams, cam_scene, lanes=0, opts=o)
    b.render(bg=(0.1, 0.2, 0.3))
    _equal_plain(b, scenes_np, cams, cam_scene, opts=o)

