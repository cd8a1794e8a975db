"""The per-frame update kernel of the dynamic workload against its FP64 reference, and the
dynamic frame that applies the same update inside the preprocess (vis_render_dynamic)."""
import numpy as np
import pytest

import oracle
import paper_2512_08478_b300 as vis
from paper_2512_08478_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n", [1, 1000, 100_003])
def test_dynamic_update_matches_reference(n):
    import torch
    sc, ex, _ = synth.workload_dynamic(n=n, frames=120)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    m_out = torch.empty((n, 3), device="cuda")
    l_out = torch.empty(n, device="cuda")
    for k in (0, 37, 119):
        t = k / 120
        vis.vis_dynamic_update(dev(sc["means"]), dev(ex["velocity"]), dev(sc["opacity_logits"]), dev(ex["amp"]),
                               dev(ex["freq"]), dev(ex["phase"]), t, m_out, l_out)
        torch.cuda.synchronize()
        rm, rl = oracle.dynamic_update(sc["means"], ex["velocity"], sc["opacity_logits"], ex["amp"], ex["freq"],
                                       ex["phase"], t)
        np.testing.assert_allclose(m_out.cpu().numpy(), rm, rtol=1e-6, atol=1e-6)
        np.testing.assert_allclose(l_out.cpu().numpy(), rl, atol=2e-6)


def test_dynamic_update_rejects_aliasing():
    import torch
    a = torch.zeros((16, 3), device="cuda")
    b = torch.zeros(16, device="cuda")
    with pytest.raises(vis.VisError):
        vis.vis_dynamic_update(a, a, b, b, b, b, 0.5, a, torch.zeros(16, device="cuda"))


def _dynamic_pair(n, k, W, H, opts=None):
    """Frame k of the dynamic workload (n Gaussians) rendered twice: vis_dynamic_update into
    a scene then vis_render, and vis_render_dynamic on the frame-0 scene."""
    import torch
    sc, ex, cams = synth.workload_dynamic(n=n, frames=120, W=W, H=H)
    base = vis.Scene.from_numpy(sc)
    dyn = {key: torch.from_numpy(np.ascontiguousarray(v)).cuda() for key, v in ex.items()}
    t = base.tensors
    m_t, l_t = torch.empty_like(t["means"]), torch.empty_like(t["opacity_logits"])
    frame = vis.Scene(m_t, t["log_scales"], t["quats"], l_t, t["sh"], sc["sh_degree"])
    vis.vis_dynamic_update(t["means"], dyn["velocity"], t["opacity_logits"], dyn["amp"], dyn["freq"], dyn["phase"],
                           k / 120, m_t, l_t)
    ws = vis.Workspace(n, W, H, key_capacity=16 * n + (1 << 20), opts=opts)
    out = []
    for dynamic in (False, True):
        rgb = torch.empty((3, H, W), device="cuda")
        alpha = torch.empty((H, W), device="cuda")
        if dynamic:
            vis.vis_render_dynamic(base.handle, dyn["velocity"], dyn["amp"], dyn["freq"], dyn["phase"], k / 120,
                                   cams[k], W, H, (0.1, 0.2, 0.3), rgb, alpha, ws.buf, opts)
        else:
            vis.vis_render(frame.handle, cams[k], W, H, (0.1, 0.2, 0.3), rgb, alpha, ws.buf, opts)
        vis.vis_check(ws.buf)
        out.append((rgb.cpu().numpy(), alpha.cpu().numpy()))
    return out, (base, frame, dyn, ws, cams[k])


@pytest.mark.parametrize("k", [0, 37, 119])
def test_dynamic_frame_equals_update_then_render(k):
    """vis_render_dynamic applies the update inside the preprocess with the update kernel's
    own arithmetic: the image is that of the update followed by a plain render, bit for bit."""
    (a, b), _ = _dynamic_pair(30_000, k, 640, 360)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[1].max() > 0.5   # the frame is not empty


def test_dynamic_frame_6m_equals_update_then_render():
    """The same at the full 6M dynamic workload, 1080p, in the bench's tuned options."""
    (a, b), _ = _dynamic_pair(6_000_000, 60, 1920, 1080, vis.make_opts(tile=32, pixels_per_thread=2))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_dynamic_frame_has_no_adjoint():
    """A backward on a dynamic frame's workspace computes nothing and vis_check reports
    VIS_ERR_UNSUPPORTED; the next plain render clears the mark."""
    import torch
    (_, _), (base, frame, dyn, ws, cam) = _dynamic_pair(20_000, 10, 320, 240)
    W, H = 320, 240
    rgb = torch.empty((3, H, W), device="cuda")
    alpha = torch.empty((H, W), device="cuda")
    vis.vis_render_dynamic(base.handle, dyn["velocity"], dyn["amp"], dyn["freq"], dyn["phase"], 10 / 120, cam, W, H,
                           (0.0, 0.0, 0.0), rgb, alpha, ws.buf)
    vis.vis_check(ws.buf)
    grads = {key: torch.full_like(base.tensors[key], 7.0) for key in vis.FIELDS}
    d_rgb = torch.ones((3, H, W), device="cuda")
    d_alpha = torch.zeros((H, W), device="cuda")
    vis.vis_render_backward(base.handle, cam, W, H, (0.0, 0.0, 0.0), d_rgb, d_alpha, ws.buf, grads)
    with pytest.raises(vis.VisError) as e:
        vis.vis_check(ws.buf)
    assert e.value.status == vis.VIS_ERR_UNSUPPORTED
    vis.vis_render(frame.handle, cam, W, H, (0.0, 0.0, 0.0), rgb, alpha, ws.buf)
    vis.vis_check(ws.buf)
    vis.vis_render_backward(frame.handle, cam, W, H, (0.0, 0.0, 0.0), d_rgb, d_alpha, ws.buf, grads)
    vis.vis_check(ws.buf)
    assert float(grads["means"].abs().sum()) > 0


def test_dynamic_render_rejects_packed_and_null():
    import torch
    sc, ex, cams = synth.workload_dynamic(n=1000, frames=120, W=64, H=64)
    base = vis.Scene.from_numpy(sc)
    v = torch.zeros((1000, 3), device="cuda")
    a = torch.zeros(1000, device="cuda")
    ws = vis.Workspace(1000, 64, 64)
    rgb = torch.empty((3, 64, 64), device="cuda")
    alpha = torch.empty((64, 64), device="cuda")
    with pytest.raises(vis.VisError) as e:
        vis.vis_render_dynamic(base.handle, None, a, a, a, 0.5, cams[0], 64, 64, (0, 0, 0), rgb, alpha, ws.buf)
    assert e.value.status == vis.VIS_ERR_INVALID_ARG
    packed = vis.PackedScene.pack(base)
    with pytest.raises(vis.VisError) as e:
        vis.vis_render_dynamic(packed.handle, v, a, a, a, 0.5, cams[0], 64, 64, (0, 0, 0), rgb, alpha, ws.buf)
    assert e.value.status == vis.VIS_ERR_UNSUPPORTED
