"""Failure detection on the GPU without a fault: the radix sort's bounded look-back wait.

A sort partition that polls a predecessor's unpublished look-back word more than
`spin_limit` times gives up, records VIS_ERR_TIMEOUT in the workspace's status block,
publishes its own counts so that nobody waits on it, and the render's later kernels skip
their work (the image comes out NaN). Here the limit is set to a single poll on a frame
whose sorts span hundreds of partitions, so some partition finds a predecessor that has
not yet published; the test checks the reported status, and that the same workspace then
renders the frame exactly as a fresh one does with the default limit.
"""
import numpy as np
import pytest

import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth
from gpu_helpers import render_gpu

pytestmark = pytest.mark.gpu


def test_lookback_timeout_is_reported_and_the_workspace_recovers():
    import torch
    sc_np = synth.mixture_scene(400_000, 9, sh_degree=1)
    cam = synth.orbit_cameras(1, 15.0, 1920, 1080, 50.0)[0]
    s = vis.Scene.from_numpy(sc_np)
    ws = vis.Workspace(s.n, cam.W, cam.H, key_capacity=8 * s.n)
    rgb = torch.empty((3, cam.H, cam.W), device="cuda")
    alpha = torch.empty((cam.H, cam.W), device="cuda")
    tight = vis.make_opts(spin_limit=1)
    timed_out = 0
    for _ in range(6):
        vis.vis_render(s.handle, cam, cam.W, cam.H, (0, 0, 0), rgb, alpha, ws.buf, tight)
        try:
            m = vis.vis_check(ws.buf)
            assert m > 100_000   # a sort of many partitions, even when no wait ran out
        except vis.VisError as e:
            assert e.status == vis.VIS_ERR_TIMEOUT, e
            assert torch.isnan(rgb).all() and torch.isnan(alpha).all()
            timed_out += 1
    assert timed_out > 0
    # the same workspace with the default limit: the frame of a fresh workspace, bit for bit
    vis.vis_render(s.handle, cam, cam.W, cam.H, (0, 0, 0), rgb, alpha, ws.buf)
    vis.vis_check(ws.buf)
    ref_rgb, ref_alpha, _, _ = render_gpu(sc_np, cam)
    assert np.array_equal(rgb.cpu().numpy().astype(np.float64), ref_rgb)
    assert np.array_equal(alpha.cpu().numpy().astype(np.float64), ref_alpha)


def test_spin_limit_is_validated_on_the_host():
    with pytest.raises(vis.VisError) as e:
        vis.vis_workspace_size(10, 8, 8, 10, vis.make_opts(spin_limit=-1))
    assert e.value.status == vis.VIS_ERR_INVALID_ARG
