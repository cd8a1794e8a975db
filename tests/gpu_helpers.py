"""Shared helpers for the GPU tests (device buffers <-> numpy, workspace views)."""
import numpy as np

import paper_2512_08478_b300 as vis


def torch():
    import torch as t
    return t


def ws_view(ws, off, count, dtype):
    """numpy copy of `count` items of `dtype` at byte offset `off` of a workspace."""
    t = torch()
    itemsize = np.dtype(dtype).itemsize
    raw = ws.buf[off: off + count * itemsize].cpu().numpy()
    return raw.view(dtype).copy()


def render_gpu(scene_np, cam, bg=(0.0, 0.0, 0.0), opts=None, key_capacity=None):
    """Render through the C ABI; returns (rgb [3,H,W] np, alpha np, Scene, Workspace)."""
    sc = vis.Scene.from_numpy(scene_np)
    ws = vis.Workspace(sc.n, cam.W, cam.H, key_capacity=key_capacity, opts=opts)
    rgb, alpha = vis._render_checked(sc, cam, cam.W, cam.H, bg, ws, opts)
    return rgb.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64), sc, ws


def gpu_stage_outputs(sc, ws):
    """Preprocess and sort intermediates from the workspace of the last render."""
    L = ws.layout()
    n = sc.n
    rec = ws_view(ws, L.off_rec, 12 * n, np.float32).reshape(n, 3, 4)
    touched = ws_view(ws, L.off_touched, n, np.uint32)
    rect_p = ws_view(ws, L.off_rect, 4 * n, np.uint32).reshape(n, 4)
    depth = ws_view(ws, L.off_depth, n, np.float32)
    ctrl = ws_view(ws, L.off_ctrl, 64, np.uint32)
    m = int(ctrl[0])
    keys = ws_view(ws, L.off_keys[L.sorted_buffer], m, np.uint64)
    vals = ws_view(ws, L.off_vals[L.sorted_buffer], m, np.uint32)
    ntiles = L.tiles_x * L.tiles_y
    ranges = ws_view(ws, L.off_ranges, 2 * ntiles, np.uint32).reshape(ntiles, 2)
    rect = np.stack([rect_p[:, 0] & 0xFFFF, rect_p[:, 1] & 0xFFFF, rect_p[:, 0] >> 16, rect_p[:, 1] >> 16], 1)
    a, b, c = rec[:, 0], rec[:, 1], rec[:, 2]
    u = a[:, 0].astype(np.float64) + a[:, 2]
    v = a[:, 1].astype(np.float64) + a[:, 3]
    f1 = b[:, 0:2].astype(np.float64)
    f2 = b[:, 2:4].astype(np.float64)
    qscale = 0.5 / np.log(2.0)   # the record's whitening rows are scaled by sqrt(log2(e)/2)
    Q = (f1[:, :, None] * f1[:, None, :] + f2[:, :, None] * f2[:, None, :]) / qscale
    return dict(valid=(touched > 0).astype(np.int32), touched=touched, rect=rect.astype(np.int32), trims=rect_p[:, 2],
                zkey=depth, uv=np.stack([u, v], 1), conic=np.stack([Q[:, 0, 0], Q[:, 0, 1], Q[:, 1, 1]], 1),
                opacity=c[:, 0].astype(np.float64), rgb=c[:, 1:4].astype(np.float64), keys=keys, vals=vals,
                ranges=ranges, m=m, layout=L)


def image_parity(gpu_rgb, gpu_alpha, ref, max_abs=2e-4, mean_abs=1e-5, max_exempt_frac=1e-4):
    """The parity bar: max-abs on every pixel, mean-abs on all, per channel.

    A pixel may exceed max-abs only if the oracle flags it as ambiguous (a decision within
    FP32 rounding of its threshold, where both results are correct), and such exempt
    pixels may make up at most 1e-4 of the image."""
    amb = ref["ambiguous"] != 0
    d = np.abs(gpu_rgb - ref["rgb"])
    da = np.abs(gpu_alpha - ref["alpha"])
    per_pix = np.maximum(d.max(axis=0), da)
    over = per_pix > max_abs
    exempt = over & amb
    frac = exempt.mean()
    worst = per_pix[~exempt].max(initial=0.0)
    print(f"parity: max-abs {per_pix.max(initial=0.0):.3g} on all pixels, {worst:.3g} outside the exempt ones, "
          f"mean-abs {d.mean():.3g}, flagged {int(amb.sum())} ({amb.mean():.2e}), exempt {int(exempt.sum())}")
    assert frac <= max_exempt_frac, f"{int(exempt.sum())} flagged pixels beyond max-abs ({frac:.2e})"
    assert worst <= max_abs, f"max-abs {worst} on a pixel the oracle does not flag"
    for ch in range(3):
        assert d[ch].mean() <= mean_abs, f"channel {ch} mean-abs {d[ch].mean()}"
    assert da.mean() <= mean_abs, f"alpha mean-abs {da.mean()}"
    return dict(max_abs=float(per_pix.max(initial=0.0)), mean_abs=float(d.mean()), flagged=int(amb.sum()),
                exempt=int(exempt.sum()))


def footprint_tiles(rect, trims, tiles_x):
    """Tiles (row-major ids) of one footprint: the box [x0, x1) x [y0, y1) whose top and
    bottom rows drop Lt, Rt and Lb, Rb tiles at their ends (trims = Lt | Rt << 8 | Lb << 16
    | Rb << 24; a one-row box uses the top trims)."""
    x0, y0, x1, y1 = (int(v) for v in rect)
    t = int(trims)
    lt, rt, lb, rb = t & 255, (t >> 8) & 255, (t >> 16) & 255, (t >> 24) & 255
    out = []
    for y in range(y0, y1):
        a, b = x0, x1
        if y == y0:
            a, b = x0 + lt, x1 - rt
        elif y == y1 - 1:
            a, b = x0 + lb, x1 - rb
        out += [y * tiles_x + x for x in range(a, b)]
    return out
