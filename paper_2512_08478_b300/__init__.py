"""B300-native 3D Gaussian Splatting rasterizer (sm_103a CUDA behind a C ABI).

This module is a thin ctypes binding over ``libvis.so`` (see include/vis.h): it
marshals torch tensors to device pointers and the current CUDA stream; every step
of the render runs in the library's kernels. There is no CPU path: if the
library is missing or no CUDA device is present, calls raise.

Entry points with the C names: vis_scene_upload, vis_workspace_size,
vis_workspace_layout, vis_render, vis_check, vis_render_backward,
vis_sort_workspace_size, vis_sort_pairs, vis_default_opts, vis_last_error.
Convenience layer: ``Scene``, ``Workspace``, ``render`` (differentiable through
``torch.autograd``) and ``sort_pairs``.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "libvis.so"
_lib = None

VIS_OK, VIS_ERR_INVALID_ARG, VIS_ERR_CUDA, VIS_ERR_CAPACITY, VIS_ERR_TIMEOUT, VIS_ERR_UNSUPPORTED = range(6)
_STATUS = {0: "VIS_OK", 1: "VIS_ERR_INVALID_ARG", 2: "VIS_ERR_CUDA", 3: "VIS_ERR_CAPACITY",
           4: "VIS_ERR_TIMEOUT", 5: "VIS_ERR_UNSUPPORTED"}


class VisError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class vis_camera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("near_z", C.c_float)]


class vis_render_opts(C.Structure):
    _fields_ = [("tile", C.c_int), ("digit_bits", C.c_int), ("dilation", C.c_float),
                ("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_stop", C.c_float),
                ("sort_mode", C.c_int), ("pixels_per_thread", C.c_int), ("tile_extent", C.c_int),
                ("collect_stats", C.c_int), ("spin_limit", C.c_int)]


class vis_scene_grads(C.Structure):
    _fields_ = [("d_means", C.c_void_p), ("d_log_scales", C.c_void_p), ("d_quats", C.c_void_p),
                ("d_opacity_logits", C.c_void_p), ("d_sh", C.c_void_p)]


class vis_ws_layout(C.Structure):
    _fields_ = [("total_bytes", C.c_size_t), ("key_capacity", C.c_int64), ("tiles_x", C.c_int),
                ("tiles_y", C.c_int), ("sort_passes", C.c_int), ("sorted_buffer", C.c_int),
                ("off_ctrl", C.c_size_t), ("off_rec", C.c_size_t), ("off_depth", C.c_size_t),
                ("off_rect", C.c_size_t), ("off_touched", C.c_size_t), ("off_keys", C.c_size_t * 2),
                ("off_vals", C.c_size_t * 2), ("off_ranges", C.c_size_t), ("off_tfinal", C.c_size_t),
                ("off_last", C.c_size_t), ("off_g2", C.c_size_t), ("key_bytes", C.c_int),
                ("sort_mode", C.c_int), ("off_order", C.c_size_t)]


_P = C.c_void_p


def lib():
    """Load libvis.so (built in-tree by paper_2512_08478_b300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2512_08478_b300.build`")
        L = C.CDLL(str(LIB_PATH))
        sig = {
            "vis_default_opts": (None, [C.POINTER(vis_render_opts)]),
            "vis_last_error": (C.c_char_p, []),
            "vis_scene_upload": (C.c_int, [_P, _P, _P, _P, _P, C.c_int, C.c_int64, C.POINTER(_P)]),
            "vis_scene_destroy": (None, [_P]),
            "vis_workspace_size": (C.c_int, [C.c_int64, C.c_int, C.c_int, C.c_int64,
                                             C.POINTER(vis_render_opts), C.POINTER(C.c_size_t)]),
            "vis_workspace_layout": (C.c_int, [C.c_int64, C.c_int, C.c_int, C.c_size_t,
                                               C.POINTER(vis_render_opts), C.POINTER(vis_ws_layout)]),
            "vis_render": (C.c_int, [_P, C.POINTER(vis_camera), C.c_int, C.c_int, C.POINTER(C.c_float),
                                     _P, _P, _P, C.c_size_t, C.POINTER(vis_render_opts), _P]),
            "vis_render_depth": (C.c_int, [_P, C.POINTER(vis_camera), C.c_int, C.c_int, C.POINTER(C.c_float),
                                           _P, _P, _P, _P, C.c_size_t, C.POINTER(vis_render_opts), _P]),
            "vis_check": (C.c_int, [_P, _P, C.POINTER(C.c_int64)]),
            "vis_render_backward": (C.c_int, [_P, C.POINTER(vis_camera), C.c_int, C.c_int,
                                              C.POINTER(C.c_float), _P, _P, _P, C.c_size_t,
                                              C.POINTER(vis_render_opts), _P, _P, _P, _P, _P, _P]),
            "vis_render_backward_depth": (C.c_int, [_P, C.POINTER(vis_camera), C.c_int, C.c_int,
                                                    C.POINTER(C.c_float), _P, _P, _P, _P, C.c_size_t,
                                                    C.POINTER(vis_render_opts), _P, _P, _P, _P, _P, _P]),
            "vis_multi_slots": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int64)]),
            "vis_packed_size": (C.c_int, [C.c_int64, C.c_int, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                          C.POINTER(C.c_size_t)]),
            "vis_scene_pack": (C.c_int, [_P, _P, _P, _P, _P]),
            "vis_scene_upload_packed": (C.c_int, [_P, _P, _P, C.c_int, C.c_int64, C.POINTER(_P)]),
            "vis_render_multi": (C.c_int, [_P, _P, C.c_int, C.POINTER(vis_camera), C.c_int, C.c_int,
                                           C.POINTER(C.c_float), _P, _P, _P, _P, C.c_size_t,
                                           C.POINTER(vis_render_opts), _P]),
            "vis_render_backward_multi": (C.c_int, [_P, _P, C.c_int, C.POINTER(vis_camera), C.c_int, C.c_int,
                                                    C.POINTER(C.c_float), _P, _P, _P, _P, C.c_size_t,
                                                    C.POINTER(vis_render_opts), _P, _P]),
            "vis_sort_workspace_size": (C.c_int, [C.c_int64, C.c_int, C.POINTER(C.c_size_t)]),
            "vis_sort_pairs": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int, _P, C.c_size_t, _P]),
            "vis_sort_pairs_noalloc": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int, _P]),
            "vis_sort_noalloc_check": (C.c_int, [_P]),
            "vis_profile_begin": (C.c_int, []),
            "vis_batch_create": (C.c_int, [C.c_int, C.POINTER(_P)]),
            "vis_batch_destroy": (None, [_P]),
            "vis_batch_workspace_size": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int, C.c_int, C.c_int64,
                                                   C.POINTER(vis_render_opts), C.POINTER(C.c_size_t)]),
            "vis_render_batch": (C.c_int, [_P, _P, C.c_int, _P, _P, _P, _P, C.c_int, C.POINTER(C.c_float),
                                           _P, _P, _P, C.c_size_t, C.POINTER(vis_render_opts), _P]),
            "vis_batch_check": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_int64)]),
            "vis_dynamic_update": (C.c_int, [_P, _P, _P, _P, _P, _P, C.c_float, C.c_int64, _P, _P, _P]),
            "vis_render_dynamic": (C.c_int, [_P, _P, _P, _P, _P, C.c_float, C.POINTER(vis_camera), C.c_int, C.c_int,
                                             C.POINTER(C.c_float), _P, _P, _P, C.c_size_t, C.POINTER(vis_render_opts),
                                             _P]),
            "vis_profile_end": (C.c_int, [C.POINTER(C.c_double), C.c_int, C.POINTER(C.c_int),
                                          C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ok(status):
    if status != VIS_OK:
        raise VisError(status, lib().vis_last_error().decode())


def _torch():
    import torch
    return torch


def _ptr(t):
    return _P(t.data_ptr() if t is not None else None)


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return _P(s.cuda_stream)


def make_camera(cam) -> vis_camera:
    """From a synth.Camera (or anything with R, t, fx, fy, cx, cy, near)."""
    c = vis_camera()
    R = [float(v) for v in cam.R.reshape(-1)]
    t = [float(v) for v in cam.t.reshape(-1)]
    c.R[:] = R
    c.t[:] = t
    c.fx, c.fy, c.cx, c.cy, c.near_z = (float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy),
                                        float(cam.near))
    return c


def make_opts(**kw) -> vis_render_opts:
    o = vis_render_opts()
    lib().vis_default_opts(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _opts_ref(opts):
    if opts is None:
        return None
    if isinstance(opts, dict):
        opts = make_opts(**opts)
    return C.byref(opts)


def _bg(bg):
    return (C.c_float * 3)(*[float(v) for v in bg])


# ----------------------------------------------------------------------------------
# C-named entry points (argument marshalling only)
# ----------------------------------------------------------------------------------

def vis_scene_upload(means, log_scales, quats, opacity_logits, sh, sh_degree):
    h = _P()
    _ok(lib().vis_scene_upload(_ptr(means), _ptr(log_scales), _ptr(quats), _ptr(opacity_logits), _ptr(sh),
                               int(sh_degree), int(means.shape[0]), C.byref(h)))
    return h


def vis_workspace_size(n, W, H, key_capacity, opts=None):
    b = C.c_size_t()
    _ok(lib().vis_workspace_size(int(n), int(W), int(H), int(key_capacity), _opts_ref(opts), C.byref(b)))
    return b.value


def vis_workspace_layout(n, W, H, ws_bytes, opts=None) -> vis_ws_layout:
    L = vis_ws_layout()
    _ok(lib().vis_workspace_layout(int(n), int(W), int(H), int(ws_bytes), _opts_ref(opts), C.byref(L)))
    return L


def vis_render(scene_handle, cam, W, H, bg, out_rgb, out_alpha, ws, opts=None, stream=None, depth=None):
    """depth: optional float32 [H,W] CUDA tensor of per-pixel view depths (vis_render_depth)."""
    c = cam if isinstance(cam, vis_camera) else make_camera(cam)
    if depth is None:
        _ok(lib().vis_render(scene_handle, C.byref(c), int(W), int(H), _bg(bg), _ptr(out_rgb), _ptr(out_alpha),
                             _ptr(ws), ws.numel() * ws.element_size(), _opts_ref(opts), _stream(stream)))
    else:
        _ok(lib().vis_render_depth(scene_handle, C.byref(c), int(W), int(H), _bg(bg), _ptr(depth), _ptr(out_rgb),
                                   _ptr(out_alpha), _ptr(ws), ws.numel() * ws.element_size(), _opts_ref(opts),
                                   _stream(stream)))


def vis_check(ws, stream=None):
    """Synchronise the stream; return the key count, raise VisError on a device error."""
    m = C.c_int64()
    st = lib().vis_check(_ptr(ws), _stream(stream), C.byref(m))
    if st != VIS_OK:
        err = VisError(st, lib().vis_last_error().decode())
        err.num_keys = m.value
        raise err
    return m.value


def read_ctrl(ws):
    """The workspace's device-written status block as a dict (synchronises)."""
    import numpy as np
    raw = ws[:256].cpu().numpy()
    u32 = raw.view(np.uint32)
    u64 = raw[80:96].view(np.uint64)
    return dict(num_keys=int(u32[0]), error=int(u32[1]), num_visible=int(u32[18]), pair_tests=int(u64[0]),
                hits=int(u64[1]))


def vis_render_backward(scene_handle, cam, W, H, bg, d_rgb, d_alpha, ws, grads, opts=None, stream=None,
                        depth=None):
    c = cam if isinstance(cam, vis_camera) else make_camera(cam)
    g = [_ptr(grads[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    if depth is None:
        _ok(lib().vis_render_backward(scene_handle, C.byref(c), int(W), int(H), _bg(bg), _ptr(d_rgb),
                                      _ptr(d_alpha), _ptr(ws), ws.numel() * ws.element_size(), _opts_ref(opts),
                                      *g, _stream(stream)))
    else:
        _ok(lib().vis_render_backward_depth(scene_handle, C.byref(c), int(W), int(H), _bg(bg), _ptr(depth),
                                            _ptr(d_rgb), _ptr(d_alpha), _ptr(ws), ws.numel() * ws.element_size(),
                                            _opts_ref(opts), *g, _stream(stream)))


def vis_sort_workspace_size(m, key_bits):
    b = C.c_size_t()
    _ok(lib().vis_sort_workspace_size(int(m), int(key_bits), C.byref(b)))
    return b.value


def vis_sort_pairs(keys_in, vals_in, keys_out, vals_out, key_bits, ws, stream=None):
    _ok(lib().vis_sort_pairs(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out), int(keys_in.numel()),
                             int(key_bits), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def vis_sort_pairs_noalloc(keys_in, vals_in, keys_out, vals_out, key_bits, stream=None):
    """Same sort with the library's static device scratch (no workspace; m <= 2^20)."""
    _ok(lib().vis_sort_pairs_noalloc(_ptr(keys_in), _ptr(vals_in), _ptr(keys_out), _ptr(vals_out),
                                     int(keys_in.numel()), int(key_bits), _stream(stream)))


def vis_dynamic_update(means0, velocity, logits0, amp, freq, phase, t, means_out, logits_out, stream=None):
    """Frame-t update of a dynamic scene: means0 + t v, logits0 + A sin(2 pi f t + phi)."""
    _ok(lib().vis_dynamic_update(_ptr(means0), _ptr(velocity), _ptr(logits0), _ptr(amp), _ptr(freq), _ptr(phase),
                                 float(t), int(means0.shape[0]), _ptr(means_out), _ptr(logits_out),
                                 _stream(stream)))


def vis_render_dynamic(scene_handle, velocity, amp, freq, phase, t, cam, W, H, bg, out_rgb, out_alpha, ws, opts=None,
                       stream=None):
    """Frame t of a dynamic scene whose handle borrows the frame-0 means and logits: the
    update of vis_dynamic_update applied inside the preprocess (the same image, bit for bit)."""
    c = cam if isinstance(cam, vis_camera) else make_camera(cam)
    _ok(lib().vis_render_dynamic(scene_handle, _ptr(velocity), _ptr(amp), _ptr(freq), _ptr(phase), float(t),
                                 C.byref(c), int(W), int(H), _bg(bg), _ptr(out_rgb), _ptr(out_alpha), _ptr(ws),
                                 ws.numel() * ws.element_size(), _opts_ref(opts), _stream(stream)))


def vis_last_error():
    return lib().vis_last_error().decode()


# ----------------------------------------------------------------------------------
def _handles(handles):
    arr = (_P * len(handles))(*[h.value if isinstance(h, _P) else h for h in handles])
    return arr


def _models(models, k):
    """Host float32 [k][12] array (row-major [A | b] per scene) or None."""
    if models is None:
        return None, None
    import numpy as np
    m = np.ascontiguousarray(np.asarray(models, np.float32).reshape(k, 12))
    return m, m.ctypes.data_as(_P)


def vis_multi_slots(handles):
    n = C.c_int64()
    _ok(lib().vis_multi_slots(_handles(handles), len(handles), C.byref(n)))
    return n.value


def vis_render_multi(handles, models, cam, W, H, bg, out_rgb, out_alpha, ws, opts=None, stream=None, depth=None):
    """handles: scene handles; models: [k,3,4] float array-like or None (identities)."""
    c = cam if isinstance(cam, vis_camera) else make_camera(cam)
    hs = _handles(handles)
    m, mp = _models(models, len(handles))
    _ok(lib().vis_render_multi(hs, mp, len(handles), C.byref(c), int(W), int(H), _bg(bg),
                               None if depth is None else _ptr(depth), _ptr(out_rgb), _ptr(out_alpha), _ptr(ws),
                               ws.numel() * ws.element_size(), _opts_ref(opts), _stream(stream)))


def vis_render_backward_multi(handles, models, cam, W, H, bg, d_rgb, d_alpha, ws, grads, opts=None, stream=None,
                              depth=None):
    """grads: one dict of gradient tensors (FIELDS) per scene."""
    c = cam if isinstance(cam, vis_camera) else make_camera(cam)
    hs = _handles(handles)
    m, mp = _models(models, len(handles))
    gs = (vis_scene_grads * len(handles))(*[vis_scene_grads(*[g[k].data_ptr() for k in
                                                               ("means", "log_scales", "quats", "opacity_logits",
                                                                "sh")]) for g in grads])
    _ok(lib().vis_render_backward_multi(hs, mp, len(handles), C.byref(c), int(W), int(H), _bg(bg),
                                        None if depth is None else _ptr(depth), _ptr(d_rgb), _ptr(d_alpha),
                                        _ptr(ws), ws.numel() * ws.element_size(), _opts_ref(opts), gs,
                                        _stream(stream)))


# Convenience layer
# ----------------------------------------------------------------------------------

FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")


class Scene:
    """Borrowed device tensors of one Gaussian asset plus its C handle.

    The tensors must stay alive and unmoved while the Scene is used; they may be
    rewritten in place between frames.
    """

    def __init__(self, means, log_scales, quats, opacity_logits, sh, sh_degree):
        torch = _torch()
        t = dict(means=means, log_scales=log_scales, quats=quats, opacity_logits=opacity_logits, sh=sh)
        for k, v in t.items():
            if not (v.is_cuda and v.dtype == torch.float32 and v.is_contiguous()):
                raise ValueError(f"{k} must be a contiguous float32 CUDA tensor")
        self.tensors = t
        self.sh_degree = int(sh_degree)
        self.n = int(means.shape[0])
        self.handle = vis_scene_upload(means, log_scales, quats, opacity_logits, sh, sh_degree)

    @classmethod
    def from_numpy(cls, scene, device="cuda"):
        torch = _torch()
        ts = {k: torch.from_numpy(scene[k]).to(device).contiguous() for k in FIELDS}
        return cls(**ts, sh_degree=scene["sh_degree"])

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.vis_scene_destroy(h)
            self.handle = None


def vis_packed_size(n, sh_degree):
    """Bytes of the (pos, cov, col) planes of a pre-packed scene."""
    a, b, c = C.c_size_t(), C.c_size_t(), C.c_size_t()
    _ok(lib().vis_packed_size(int(n), int(sh_degree), C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


class PackedScene:
    """A pre-packed fp16 scene (vis_scene_upload_packed): device planes pos [n,2], cov [n,3],
    col [n,W] of uint32 words (stored as int32 tensors), borrowed by the C handle."""

    def __init__(self, pos, cov, col, sh_degree):
        torch = _torch()
        for name, t in (("pos", pos), ("cov", cov), ("col", col)):
            if not (t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()):
                raise ValueError(f"{name} must be a contiguous int32 CUDA tensor")
        self.planes = dict(pos=pos, cov=cov, col=col)
        self.sh_degree = int(sh_degree)
        self.n = int(pos.shape[0])
        h = _P()
        _ok(lib().vis_scene_upload_packed(_ptr(pos), _ptr(cov), _ptr(col), self.sh_degree, self.n, C.byref(h)))
        self.handle = h

    @classmethod
    def from_planes(cls, planes, sh_degree, device="cuda"):
        """From host uint32 planes (e.g. the oracle's prepack)."""
        import numpy as np
        torch = _torch()
        ts = {k: torch.from_numpy(np.ascontiguousarray(planes[k], np.uint32).view(np.int32)).to(device)
              for k in ("pos", "cov", "col")}
        return cls(ts["pos"], ts["cov"], ts["col"], sh_degree)

    @classmethod
    def pack(cls, scene, stream=None):
        """Pack an fp32 Scene on the device (vis_scene_pack)."""
        torch = _torch()
        a, b, c = vis_packed_size(scene.n, scene.sh_degree)
        dev = scene.tensors["means"].device
        pos = torch.empty(a // 4, dtype=torch.int32, device=dev).view(scene.n, 2)
        cov = torch.empty(b // 4, dtype=torch.int32, device=dev).view(scene.n, 3)
        col = torch.empty(c // 4, dtype=torch.int32, device=dev).view(scene.n, -1)
        _ok(lib().vis_scene_pack(scene.handle, _ptr(pos), _ptr(cov), _ptr(col), _stream(stream)))
        return cls(pos, cov, col, scene.sh_degree)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.vis_scene_destroy(h)
            self.handle = None


class Workspace:
    """A caller-owned device workspace, grown on a capacity error."""

    def __init__(self, n, W, H, key_capacity=None, opts=None, device="cuda"):
        self.n, self.W, self.H, self.opts = n, W, H, opts
        cap = key_capacity if key_capacity is not None else max(1 << 16, 4 * n)
        self._alloc(cap, device)

    def _alloc(self, cap, device="cuda"):
        torch = _torch()
        nbytes = vis_workspace_size(self.n, self.W, self.H, cap, self.opts)
        self.buf = torch.empty((nbytes + 15) // 16 * 16, dtype=torch.uint8, device=device)
        self.key_capacity = cap

    def grow(self, needed):
        self._alloc(int(needed * 1.25) + 1024, self.buf.device)

    def layout(self) -> vis_ws_layout:
        return vis_workspace_layout(self.n, self.W, self.H, self.buf.numel(), self.opts)


def _render_checked(scene, cam, W, H, bg, ws, opts, stream=None, depth=None):
    torch = _torch()
    out_rgb = torch.empty((3, H, W), dtype=torch.float32, device=ws.buf.device)
    out_alpha = torch.empty((H, W), dtype=torch.float32, device=ws.buf.device)
    for _ in range(2):
        vis_render(scene.handle, cam, W, H, bg, out_rgb, out_alpha, ws.buf, opts, stream, depth)
        try:
            vis_check(ws.buf, stream)
            return out_rgb, out_alpha
        except VisError as e:
            if e.status != VIS_ERR_CAPACITY:
                raise
            ws.grow(e.num_keys)
    raise VisError(VIS_ERR_CAPACITY, "workspace growth did not converge")


def _render_multi_checked(scenes, models, cam, W, H, bg, ws, opts, stream=None, depth=None):
    torch = _torch()
    out_rgb = torch.empty((3, H, W), dtype=torch.float32, device=ws.buf.device)
    out_alpha = torch.empty((H, W), dtype=torch.float32, device=ws.buf.device)
    handles = [s.handle for s in scenes]
    for _ in range(2):
        vis_render_multi(handles, models, cam, W, H, bg, out_rgb, out_alpha, ws.buf, opts, stream, depth)
        try:
            vis_check(ws.buf, stream)
            return out_rgb, out_alpha
        except VisError as e:
            if e.status != VIS_ERR_CAPACITY:
                raise
            ws.grow(e.num_keys)
    raise VisError(VIS_ERR_CAPACITY, "workspace growth did not converge")


def _make_autograd():
    torch = _torch()

    class RenderFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, scene, cam, W, H, bg, ws, opts, depth, means, log_scales, quats, opacity_logits, sh):
            rgb, alpha = _render_checked(scene, cam, W, H, bg, ws, opts, depth=depth)
            ctx.scene, ctx.cam, ctx.W, ctx.H, ctx.bg, ctx.ws, ctx.opts = scene, cam, W, H, bg, ws, opts
            ctx.depth = depth
            return rgb, alpha

        @staticmethod
        def backward(ctx, d_rgb, d_alpha):
            sc = ctx.scene
            d_rgb = (d_rgb if d_rgb is not None else torch.zeros((3, ctx.H, ctx.W), device=ctx.ws.buf.device))
            d_alpha = (d_alpha if d_alpha is not None else torch.zeros((ctx.H, ctx.W), device=ctx.ws.buf.device))
            d_rgb = d_rgb.contiguous().float()
            d_alpha = d_alpha.contiguous().float()
            grads = {k: torch.empty_like(sc.tensors[k]) for k in FIELDS}
            vis_render_backward(sc.handle, ctx.cam, ctx.W, ctx.H, ctx.bg, d_rgb, d_alpha, ctx.ws.buf, grads,
                                ctx.opts, depth=ctx.depth)
            return (None, None, None, None, None, None, None, None, grads["means"], grads["log_scales"],
                    grads["quats"], grads["opacity_logits"], grads["sh"])

    class RenderMultiFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, scenes, models, cam, W, H, bg, ws, opts, depth, *tensors):
            rgb, alpha = _render_multi_checked(scenes, models, cam, W, H, bg, ws, opts, depth=depth)
            ctx.args = (scenes, models, cam, W, H, bg, ws, opts, depth)
            return rgb, alpha

        @staticmethod
        def backward(ctx, d_rgb, d_alpha):
            scenes, models, cam, W, H, bg, ws, opts, depth = ctx.args
            dev = ws.buf.device
            d_rgb = (d_rgb if d_rgb is not None else torch.zeros((3, H, W), device=dev)).contiguous().float()
            d_alpha = (d_alpha if d_alpha is not None else torch.zeros((H, W), device=dev)).contiguous().float()
            grads = [{k: torch.empty_like(s.tensors[k]) for k in FIELDS} for s in scenes]
            vis_render_backward_multi([s.handle for s in scenes], models, cam, W, H, bg, d_rgb, d_alpha, ws.buf,
                                      grads, opts, depth=depth)
            flat = [g[k] for g in grads for k in FIELDS]
            return (None,) * 9 + tuple(flat)

    return RenderFn, RenderMultiFn


_RENDER_FN = None
_RENDER_MULTI_FN = None


def render(scene: Scene, cam, W, H, bg=(0.0, 0.0, 0.0), ws: Workspace | None = None, opts=None, depth=None):
    """Render one view; differentiable w.r.t. the scene tensors (if they require grad).

    depth: optional float32 [H,W] CUDA tensor: depth-buffer-aware compositing (a splat
    deeper than a pixel's value is not composited there). Returns (rgb [3,H,W],
    alpha [H,W]). The workspace keeps the forward's intermediates for the backward; do
    not reuse it for another render before calling backward. A PackedScene (fp16, for
    viewing) renders without autograd.
    """
    global _RENDER_FN, _RENDER_MULTI_FN
    if _RENDER_FN is None:
        _RENDER_FN, _RENDER_MULTI_FN = _make_autograd()
    if ws is None:
        ws = Workspace(scene.n, W, H, opts=opts)
    if depth is not None:
        depth = depth.contiguous().float()
    if isinstance(scene, PackedScene):
        return _render_checked(scene, cam, W, H, tuple(bg), ws, opts, depth=depth)
    t = scene.tensors
    return _RENDER_FN.apply(scene, cam, W, H, tuple(bg), ws, opts, depth, t["means"], t["log_scales"], t["quats"],
                            t["opacity_logits"], t["sh"])


def multi_workspace(scenes, W, H, key_capacity=None, opts=None):
    """A Workspace sized for render_multi over `scenes` (vis_multi_slots slots)."""
    return Workspace(vis_multi_slots([s.handle for s in scenes]), W, H, key_capacity, opts)


def render_multi(scenes, models, cam, W, H, bg=(0.0, 0.0, 0.0), ws: Workspace | None = None, opts=None,
                 depth=None):
    """Several scenes in one image, each under its own affine transform (models: [k,3,4]
    float array-like, row-major [A | b], or None for identities), composited in one global
    depth order (vis_render_multi). Differentiable w.r.t. every scene's tensors; the
    gradients are w.r.t. the untransformed parameters. If any scene is a PackedScene the
    render runs without autograd. Returns (rgb [3,H,W], alpha [H,W])."""
    global _RENDER_FN, _RENDER_MULTI_FN
    if _RENDER_FN is None:
        _RENDER_FN, _RENDER_MULTI_FN = _make_autograd()
    scenes = list(scenes)
    if ws is None:
        ws = multi_workspace(scenes, W, H, opts=opts)
    if models is not None:
        import numpy as np
        models = np.ascontiguousarray(np.asarray(models, np.float32).reshape(len(scenes), 12))
    if depth is not None:
        depth = depth.contiguous().float()
    if any(isinstance(s, PackedScene) for s in scenes):
        return _render_multi_checked(scenes, models, cam, W, H, tuple(bg), ws, opts, depth=depth)
    tensors = [s.tensors[k] for s in scenes for k in FIELDS]
    return _RENDER_MULTI_FN.apply(scenes, models, cam, W, H, tuple(bg), ws, opts, depth, *tensors)


def sort_pairs(keys, vals, key_bits=64):
    """Stable device sort of uint64 keys (int64 tensor) with uint32 values (int32 tensor)."""
    torch = _torch()
    m = keys.numel()
    ko = torch.empty_like(keys)
    vo = torch.empty_like(vals)
    ws = torch.empty(max(16, vis_sort_workspace_size(m, key_bits)), dtype=torch.uint8, device=keys.device)
    vis_sort_pairs(keys, vals, ko, vo, key_bits, ws)
    return ko, vo


class Batch:
    """Many (asset, camera) images rendered by one vis_render_batch call (a CUDA graph).

    scenes: list of Scene; cams: list of cameras; cam_scene: asset index per image.
    lanes = 0 (default): one fused pipeline (one preprocess over the work list of all images,
    then, per group of images stacked on one tile canvas, one depth sort, one counts-first sort
    by canvas tile and one compositor over the canvas); the workspace holds `key_capacity` tile
    copies per group (the default: all images' copies). lanes >= 1: per-image renders on that
    many concurrent lanes, each a workspace slice of `key_capacity` keys.
    Outputs are allocated here.
    """

    def __init__(self, scenes, cams, cam_scene, lanes=0, key_capacity=None, opts=None):
        torch = _torch()
        self.scenes, self.cams, self.cam_scene = list(scenes), list(cams), list(cam_scene)
        self.n = len(self.cams)
        self.opts = opts
        self.lanes = int(lanes)
        h = _P()
        _ok(lib().vis_batch_create(self.lanes, C.byref(h)))
        self.handle = h
        self._scene_arr = (_P * len(self.scenes))(*[s.handle.value for s in self.scenes])
        self._cams = (vis_camera * self.n)(*[make_camera(c) for c in self.cams])
        self._cs = (C.c_int * self.n)(*self.cam_scene)
        self._W = (C.c_int * self.n)(*[int(c.W) for c in self.cams])
        self._H = (C.c_int * self.n)(*[int(c.H) for c in self.cams])
        self.rgb = [torch.empty((3, c.H, c.W), device="cuda") for c in self.cams]
        self.alpha = [torch.empty((c.H, c.W), device="cuda") for c in self.cams]
        self._rgb_p = (_P * self.n)(*[t.data_ptr() for t in self.rgb])
        self._a_p = (_P * self.n)(*[t.data_ptr() for t in self.alpha])
        if key_capacity is None:
            if self.lanes == 0:   # all images' copies: about 5 per Gaussian seen, grown on demand
                slots = sum((self.scenes[a].n + 255) // 256 * 256 for a in self.cam_scene)
                key_capacity = min((1 << 30) - 1, 5 * slots + (1 << 20))
            else:
                key_capacity = max(1 << 16, 8 * max(s.n for s in self.scenes))
        self._alloc(key_capacity)

    def _alloc(self, key_capacity):
        torch = _torch()
        b = C.c_size_t()
        _ok(lib().vis_batch_workspace_size(self._scene_arr, len(self.scenes), self._cs, self._W, self._H, self.n,
                                           self.lanes, int(key_capacity), _opts_ref(self.opts), C.byref(b)))
        self.ws = torch.empty((b.value + 15) // 16 * 16, dtype=torch.uint8, device="cuda")
        self.key_capacity = key_capacity

    def launch(self, bg=(0.0, 0.0, 0.0), stream=None):
        _ok(lib().vis_render_batch(self.handle, self._scene_arr, len(self.scenes), self._cams, self._cs, self._W,
                                   self._H, self.n, _bg(bg), self._rgb_p, self._a_p, _ptr(self.ws),
                                   self.ws.numel(), _opts_ref(self.opts), _stream(stream)))

    def check(self, stream=None):
        m = C.c_int64()
        st = lib().vis_batch_check(_ptr(self.ws), self.n, _stream(stream), C.byref(m))
        if st != VIS_OK:
            err = VisError(st, lib().vis_last_error().decode())
            err.num_keys = m.value
            raise err
        return m.value

    def render(self, bg=(0.0, 0.0, 0.0)):
        """Launch, check, and grow the workspace once on a capacity error."""
        for _ in range(2):
            self.launch(bg)
            try:
                self.check()
                return self.rgb, self.alpha
            except VisError as e:
                if e.status != VIS_ERR_CAPACITY:
                    raise
                self._alloc(min((1 << 30) - 1, int(e.num_keys * 1.25) + 1024))
        raise VisError(VIS_ERR_CAPACITY, "batch workspace growth did not converge")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.vis_batch_destroy(h)
            self.handle = None
