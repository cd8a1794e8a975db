"""Batched render (vis_render_batch, one CUDA graph over lanes of images) against the
plain per-image path: every image must be bit-identical to vis_render of the same
(asset, camera, options), and so inherits its oracle parity."""
import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth
from gpu_helpers import image_parity, render_gpu

pytestmark = pytest.mark.gpu


def _small_batch(assets=4, cams_per_asset=4, scale=0.01):
    scenes_np, cams, cam_scene = synth.workload_batch(assets=assets, cams_per_asset=cams_per_asset, scale=scale)
    return scenes_np, cams, cam_scene


@pytest.mark.parametrize("lanes", [1, 3, 8])
def test_batch_images_equal_plain_renders(lanes):
    import torch
    scenes_np, cams, cam_scene = _small_batch()
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    b = vis.Batch(scenes, cams, cam_scene, lanes=lanes)
    rgb, alpha = b.render(bg=(0.1, 0.2, 0.3))
    for _ in range(2):              # graph replays give the same images
        b.launch(bg=(0.1, 0.2, 0.3))
    b.check()
    for i, cam in enumerate(cams):
        r, a, _, _ = render_gpu(scenes_np[cam_scene[i]], cam, (0.1, 0.2, 0.3))
        assert np.array_equal(b.rgb[i].cpu().numpy().astype(np.float64), r)
        assert np.array_equal(b.alpha[i].cpu().numpy().astype(np.float64), a)


def test_batch_oracle_parity_and_heterogeneous_degrees():
    scenes_np, cams, cam_scene = _small_batch(assets=3, cams_per_asset=2, scale=0.005)
    degs = {s["sh_degree"] for s in scenes_np}
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    b = vis.Batch(scenes, cams, cam_scene, lanes=4, opts=vis.make_opts(tile=8))
    b.render()
    for i in (0, len(cams) - 1):
        ref, _ = oracle.render(scenes_np[cam_scene[i]], cams[i], opts=dict(tile=8))
        image_parity(b.rgb[i].cpu().numpy().astype(np.float64), b.alpha[i].cpu().numpy().astype(np.float64), ref)
    assert len(degs) >= 1


def test_batch_capacity_error_is_reported_then_grown():
    scenes_np, cams, cam_scene = _small_batch(assets=2, cams_per_asset=2)
    scenes = [vis.Scene.from_numpy(s) for s in scenes_np]
    b = vis.Batch(scenes, cams, cam_scene, lanes=2, key_capacity=32)
    b.launch()
    with pytest.raises(vis.VisError) as e:
        b.check()
    assert e.value.status == vis.VIS_ERR_CAPACITY and e.value.num_keys > 32
    b.render()                       # grows the workspace and re-captures
    assert b.key_capacity > 32
    b.check()
