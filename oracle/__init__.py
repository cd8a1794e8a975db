"""FP64 CPU oracle for the 3DGS rasterization hot path -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package. The CUDA library never does, and this package
never imports the CUDA library: the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, double precision, OpenMP over
independent outputs); this module compiles it with gcc on first use and marshals
numpy arrays. Every function follows the paper's section 3.2 (Eqs. 1-3) and
Algorithm 1 under the readings listed at the top of ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB_PATH = _HERE / "liboracle.so"
_lib = None

DEFAULT_OPTS = dict(tile=16, dilation=0.3, alpha_min=1.0 / 255.0, alpha_max=0.99,
                    t_stop=1e-4, q_max=9.0)


def _override():
    """ORACLE_LIB names another build of oracle.c to load instead of liboracle.so: the
    mutation tests point it at a copy with one planted mistake."""
    p = os.environ.get("ORACLE_LIB")
    return Path(p) if p else None


def build(force: bool = False) -> Path:
    """Compile oracle.c into liboracle.so beside it (gcc -O2 -fopenmp)."""
    if _override() is not None:
        return _override()
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_PATH.with_suffix(f".so.{os.getpid()}.tmp")
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    if _lib is None:
        _lib = C.CDLL(str(build()))
        _lib.orc_duplicate.restype = C.c_int64
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, np.float32)


def _f64(a):
    return np.ascontiguousarray(a, np.float64)


def opts_array(opts=None):
    """[tile, dilation, alpha_min, alpha_max, t_stop, q_max] as float64.

    The thresholds are rounded to float32 first, so that the oracle compares
    against exactly the values the CUDA library receives.
    """
    o = dict(DEFAULT_OPTS)
    if opts:
        o.update(opts)
    vals = [o["tile"], o["dilation"], o["alpha_min"], o["alpha_max"], o["t_stop"], o["q_max"]]
    return np.array([float(np.float32(v)) for v in vals], np.float64)


def cam_array(cam):
    """Camera -> 17 float64 values made from its float32 parameters."""
    return cam.as_array().astype(np.float64)


def model_array(model):
    """Per-model affine transform [A | b] (3x4, row-major) -> 12 float64 values made from its
    float32 rounding (the values the CUDA library receives); None stays None (identity)."""
    if model is None:
        return None
    m = np.asarray(model, np.float64).reshape(-1)
    if m.shape[0] != 12:
        raise ValueError("a model transform is 3x4 ([A | b])")
    return m.astype(np.float32).astype(np.float64)


def _mp(m):
    return None if m is None else _p(m)


def num_threads() -> int:
    return len(os.sched_getaffinity(0))


def preprocess(scene, cam, opts=None, model=None):
    """Per-Gaussian projection, conic, extent, tile rectangle and colour (Eq. 1).
    model: optional 3x4 [A | b]; the scene is drawn transformed by it (Algorithm 1's M_k).

    Returns a dict of numpy arrays: valid [N] int32, uv [N,2], conic [N,3]
    (a, b, c with q = a dx^2 + 2 b dx dy + c dy^2), S [N,3] (s00, s01, s11),
    opacity [N], rgb [N,3], z [N], zkey [N] float32, radius [N], rect [N,4]
    (x0, y0, x1, y1 in tiles, upper bounds exclusive).
    """
    n = scene["means"].shape[0]
    out = dict(valid=np.zeros(n, np.int32), uv=np.zeros((n, 2)), conic=np.zeros((n, 3)),
               S=np.zeros((n, 3)), opacity=np.zeros(n), rgb=np.zeros((n, 3)), z=np.zeros(n),
               zkey=np.zeros(n, np.float32), radius=np.zeros(n, np.int32),
               rect=np.zeros((n, 4), np.int32))
    m = model_array(model)
    if "cov6" in scene:   # pre-packed form: mean, covariance upper triangle, opacity, SH
        arrs = [_f64(scene[k]) for k in ("means", "cov6", "opacity", "sh")]
        rc = _L().orc_preprocess_cov(C.c_int64(n), *[_p(a) for a in arrs], C.c_int(scene["sh_degree"]), _mp(m),
                                     _p(cam_array(cam)), C.c_int(cam.W), C.c_int(cam.H), _p(opts_array(opts)),
                                     *[_p(out[k]) for k in ("valid", "uv", "conic", "S", "opacity", "rgb",
                                                            "z", "zkey", "radius", "rect")])
        if rc != 0:
            raise ValueError("oracle preprocess rejected its arguments")
        return out
    arrs = [_f64(scene[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    rc = _L().orc_preprocess(C.c_int64(n), *[_p(a) for a in arrs], C.c_int(scene["sh_degree"]), _mp(m),
                             _p(cam_array(cam)), C.c_int(cam.W), C.c_int(cam.H), _p(opts_array(opts)),
                             *[_p(out[k]) for k in ("valid", "uv", "conic", "S", "opacity", "rgb",
                                                    "z", "zkey", "radius", "rect")])
    if rc != 0:
        raise ValueError("oracle preprocess rejected its arguments")
    return out


def _zlim(depth, count):
    """float32 depth limits (or None): splats deeper than a pixel's limit are not composited."""
    if depth is None:
        return None, None
    z = np.ascontiguousarray(np.asarray(depth, np.float32).reshape(-1))
    if z.shape[0] != count:
        raise ValueError("depth buffer has the wrong size")
    return z, _p(z)


def render_pixels(prep, px, py, bg=(0.0, 0.0, 0.0), opts=None, depth=None):
    """Brute-force definition at the given pixels: every valid splat is a candidate.
    depth: optional float32 [P] depth limits (depth-buffer-aware compositing).

    Returns dict rgb [P,3], alpha [P], T [P], n_contrib [P], ambiguous [P].
    """
    n = prep["valid"].shape[0]
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    P = px.shape[0]
    out = dict(rgb=np.zeros((P, 3)), alpha=np.zeros(P), T=np.zeros(P),
               n_contrib=np.zeros(P, np.int32), ambiguous=np.zeros(P, np.int32))
    zl, zl_p = _zlim(depth, P)
    _L().orc_render_pixels(C.c_int64(n), _p(prep["valid"]), _p(prep["uv"]), _p(prep["conic"]),
                           _p(prep["opacity"]), _p(prep["rgb"]), _p(prep["zkey"]), C.c_int64(P),
                           _p(px), _p(py), _p(_f64(bg)), _p(opts_array(opts)), zl_p,
                           _p(out["rgb"]), _p(out["alpha"]), _p(out["T"]), _p(out["n_contrib"]),
                           _p(out["ambiguous"]))
    return out


def render_bruteforce(prep, W, H, bg=(0.0, 0.0, 0.0), opts=None, depth=None):
    """Whole image by the brute-force definition; rgb returned planar [3,H,W]."""
    ys, xs = np.mgrid[0:H, 0:W]
    r = render_pixels(prep, xs.ravel(), ys.ravel(), bg, opts, depth)
    return dict(rgb=r["rgb"].T.reshape(3, H, W).copy(), alpha=r["alpha"].reshape(H, W),
                T=r["T"].reshape(H, W), n_contrib=r["n_contrib"].reshape(H, W),
                ambiguous=r["ambiguous"].reshape(H, W))


def render_tiled(prep, W, H, bg=(0.0, 0.0, 0.0), opts=None, tile_mask=None, depth=None):
    """Tile-binned render (same result as the brute force; faster on big scenes).
    depth: optional float32 [H,W] depth buffer (view depth); a splat deeper than a
    pixel's value is not composited there (tested, never written).

    tile_mask: optional uint8 [tiles_y * tiles_x]; only those tiles are computed
    (other pixels are NaN in rgb/alpha/T and -1 in n_contrib/ambiguous).
    """
    n = prep["valid"].shape[0]
    out = dict(rgb=np.full((3, H, W), np.nan), alpha=np.full((H, W), np.nan),
               T=np.full((H, W), np.nan), n_contrib=np.full((H, W), -1, np.int32),
               ambiguous=np.full((H, W), -1, np.int32))
    mask_p = None
    if tile_mask is not None:
        tile_mask = np.ascontiguousarray(tile_mask, np.uint8)
        mask_p = _p(tile_mask)
    zl, zl_p = _zlim(depth, H * W)
    rc = _L().orc_render_tiled(C.c_int64(n), _p(prep["valid"]), _p(prep["uv"]), _p(prep["conic"]),
                               _p(prep["opacity"]), _p(prep["rgb"]), _p(prep["zkey"]), _p(prep["rect"]),
                               C.c_int(W), C.c_int(H), _p(_f64(bg)), _p(opts_array(opts)), mask_p, zl_p,
                               _p(out["rgb"]), _p(out["alpha"]), _p(out["T"]), _p(out["n_contrib"]),
                               _p(out["ambiguous"]))
    if rc != 0:
        raise MemoryError("oracle tile binning failed")
    return out


def render(scene, cam, bg=(0.0, 0.0, 0.0), opts=None, tile_mask=None, depth=None):
    """Preprocess + tile-binned render of one view (depth: optional [H,W] depth buffer)."""
    prep = preprocess(scene, cam, opts)
    return render_tiled(prep, cam.W, cam.H, bg, opts, tile_mask, depth), prep


def packed_words(sh_degree):
    """uint32 words per Gaussian of the colour plane: 3 (deg+1)^2 halves, rounded up to an
    even number of words (8-byte rows)."""
    halves = 3 * (sh_degree + 1) ** 2
    words = (halves + 1) // 2
    return words + (words & 1)


def prepack(scene):
    """The pre-pack step of Algorithm 1 (section 3.4, FP16 layout), once per scene:
    Sigma = CovFromScaleRot(s, r) in FP64, then mean, opacity alpha = sigmoid(logit),
    the covariance's upper triangle (xx, xy, xz, yy, yz, zz) and the SH coefficients are
    cast to fp16 (round to nearest even) and packed two halves per uint32, low half first:
      pos  [n,2]  (mu_x, mu_y), (mu_z, alpha)
      cov  [n,3]  (xx, xy), (xz, yy), (yz, zz)
      col  [n,W]  the SH coefficients in their [K,3] order, zero-padded (W = packed_words)
    Returns (planes, decoded): the uint32 planes and the scene they decode to (float64,
    the pre-packed form the oracle's preprocess takes: means, cov6, opacity, sh)."""
    n = scene["means"].shape[0]
    deg = scene["sh_degree"]
    K = (deg + 1) ** 2
    sig = covariance(scene["log_scales"], scene["quats"])
    cov6 = np.stack([sig[:, 0, 0], sig[:, 0, 1], sig[:, 0, 2], sig[:, 1, 1], sig[:, 1, 2], sig[:, 2, 2]], 1)
    alpha = 1.0 / (1.0 + np.exp(-_f64(scene["opacity_logits"])))
    mu_h = _f64(scene["means"]).astype(np.float16)
    a_h = alpha.astype(np.float16)
    cov_h = cov6.astype(np.float16)
    sh_h = _f64(scene["sh"]).reshape(n, 3 * K).astype(np.float16)

    def pack(halves):
        h = np.ascontiguousarray(halves, np.float16)
        if h.shape[1] % 2:
            h = np.concatenate([h, np.zeros((n, 1), np.float16)], 1)
        return np.ascontiguousarray(h).view(np.uint32)

    words = packed_words(deg)
    col_h = np.zeros((n, 2 * words), np.float16)
    col_h[:, : 3 * K] = sh_h
    planes = dict(pos=pack(np.concatenate([mu_h, a_h[:, None]], 1)), cov=pack(cov_h), col=pack(col_h))
    decoded = dict(means=mu_h.astype(np.float64), cov6=cov_h.astype(np.float64), opacity=a_h.astype(np.float64),
                   sh=sh_h.astype(np.float64).reshape(n, K, 3), sh_degree=deg)
    return planes, decoded


PREP_KEYS = ("valid", "uv", "conic", "S", "opacity", "rgb", "z", "zkey", "radius", "rect")


def concat_preps(preps):
    """One splat set from several models' preprocess outputs, in model order (the
    global index of model k's Gaussian i is the sum of the earlier models' sizes + i)."""
    return {k: np.ascontiguousarray(np.concatenate([p[k] for p in preps], axis=0)) for k in PREP_KEYS}


def render_multi(scenes, models, cam, bg=(0.0, 0.0, 0.0), opts=None, tile_mask=None, depth=None):
    """Several models drawn into one image (Algorithm 1): each model is preprocessed
    with its own transform M_k (None = identity), then all splats are sorted and
    composited together in one global (tile, depth, index) order."""
    models = [None] * len(scenes) if models is None else list(models)
    if len(models) != len(scenes):
        raise ValueError("one model transform per scene")
    prep = concat_preps([preprocess(s, cam, opts, m) for s, m in zip(scenes, models)])
    return render_tiled(prep, cam.W, cam.H, bg, opts, tile_mask, depth), prep


def duplicate(prep, tiles_x, cap=None):
    """Keys (tile << 32 | float bits of zkey) and vals (Gaussian index), index-major."""
    n = prep["valid"].shape[0]
    rect = prep["rect"]
    counts = np.where(prep["valid"] != 0, (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1]), 0)
    m_total = int(counts.sum())
    cap = m_total if cap is None else cap
    keys = np.zeros(max(cap, 1), np.uint64)
    vals = np.zeros(max(cap, 1), np.uint32)
    m = _L().orc_duplicate(C.c_int64(n), _p(prep["valid"]), _p(rect), _p(prep["zkey"]),
                           C.c_int(tiles_x), _p(keys), _p(vals), C.c_int64(cap))
    if m < 0:
        raise OverflowError("more keys than capacity")
    return keys[:m], vals[:m]


def duplicate_raw(valid, rect, zkey, tiles_x):
    """Same as duplicate() from explicit arrays (valid [N], rect [N,4], zkey [N])."""
    return duplicate(dict(valid=np.ascontiguousarray(valid, np.int32),
                          rect=np.ascontiguousarray(rect, np.int32),
                          zkey=np.ascontiguousarray(zkey, np.float32)), tiles_x)


def stable_sort_pairs(keys, vals):
    keys = np.ascontiguousarray(keys, np.uint64)
    vals = np.ascontiguousarray(vals, np.uint32)
    m = keys.shape[0]
    ok = np.zeros(max(m, 1), np.uint64)
    ov = np.zeros(max(m, 1), np.uint32)
    _L().orc_stable_sort_pairs(C.c_int64(m), _p(keys), _p(vals), _p(ok), _p(ov))
    return ok[:m], ov[:m]


def tile_ranges(sorted_keys, ntiles):
    sorted_keys = np.ascontiguousarray(sorted_keys, np.uint64)
    r = np.zeros((ntiles, 2), np.uint32)
    _L().orc_tile_ranges(C.c_int64(sorted_keys.shape[0]), _p(sorted_keys), C.c_int64(ntiles), _p(r))
    return r


def sh_eval(deg, direction):
    """Real SH basis values Y_k, k < (deg+1)^2, at a unit direction (x, y, z)."""
    Y = np.zeros(16)
    x, y, z = (float(v) for v in direction)
    _L().orc_sh_eval(C.c_int(deg), C.c_double(x), C.c_double(y), C.c_double(z), _p(Y))
    return Y[: (deg + 1) ** 2].copy()


def covariance(log_scales, quats):
    """Sigma = R diag(exp(log_s))^2 R^T per Gaussian, [N,3,3]."""
    ls = _f64(np.atleast_2d(log_scales))
    q = _f64(np.atleast_2d(quats))
    n = ls.shape[0]
    out = np.zeros((n, 9))
    _L().orc_covariance(C.c_int64(n), _p(ls), _p(q), _p(out))
    return out.reshape(n, 3, 3)


def _grad_dict(n, K):
    return dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                opacity_logits=np.zeros(n), sh=np.zeros((n, K, 3)))


def adjoint(scene, cam, gC, gA, bg=(0.0, 0.0, 0.0), opts=None, return_g2=False, depth=None, model=None):
    """FP64 gradient of L = sum(gC * rgb) + sum(gA * alpha) w.r.t. all Gaussian inputs.

    gC: [3,H,W], gA: [H,W]; depth: optional [H,W] depth buffer (as in render); model:
    optional 3x4 transform (as in preprocess; gradients are w.r.t. the untransformed
    parameters). Returns dict
    means [N,3], log_scales [N,3], quats [N,4], opacity_logits [N], sh [N,K,3] (and g2
    [N,9] screen-space gradients if asked).
    """
    n = scene["means"].shape[0]
    K = (scene["sh_degree"] + 1) ** 2
    out = _grad_dict(n, K)
    g2 = np.zeros((n, 9))
    arrs = [_f64(scene[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")]
    zl, zl_p = _zlim(depth, cam.W * cam.H)   # zl keeps the buffer alive through the call
    m = model_array(model)
    rc = _L().orc_adjoint(C.c_int64(n), *[_p(a) for a in arrs], C.c_int(scene["sh_degree"]), _mp(m),
                          _p(cam_array(cam)), C.c_int(cam.W), C.c_int(cam.H), _p(opts_array(opts)),
                          _p(_f64(bg)), _p(_f64(gC)), _p(_f64(gA)), zl_p,
                          *[_p(out[k]) for k in ("means", "log_scales", "quats", "opacity_logits", "sh")],
                          _p(g2))
    if rc != 0:
        raise ValueError("oracle adjoint failed")
    if return_g2:
        out["g2"] = g2
    return out


def adjoint_multi(scenes, models, cam, gC, gA, bg=(0.0, 0.0, 0.0), opts=None, depth=None):
    """FP64 gradients of a render_multi image's loss (as adjoint) w.r.t. every model's
    own (untransformed) parameters: the compositing adjoint over the global order,
    then each model's preprocess adjoint on its slice. Returns one dict per scene."""
    models = [None] * len(scenes) if models is None else list(models)
    _, prep = render_multi(scenes, models, cam, bg, opts, depth=depth)
    n = prep["valid"].shape[0]
    g2 = np.zeros((max(n, 1), 9))
    zl, zl_p = _zlim(depth, cam.W * cam.H)
    rc = _L().orc_composite_adjoint(C.c_int64(n), *[_p(prep[k]) for k in ("valid", "uv", "conic", "opacity",
                                                                           "rgb", "zkey", "rect")],
                                    C.c_int(cam.W), C.c_int(cam.H), _p(opts_array(opts)), _p(_f64(bg)),
                                    _p(_f64(gC)), _p(_f64(gA)), zl_p, _p(g2))
    if rc != 0:
        raise ValueError("oracle compositing adjoint failed")
    outs, off = [], 0
    for sc, mdl in zip(scenes, models):
        k = sc["means"].shape[0]
        out = _grad_dict(k, (sc["sh_degree"] + 1) ** 2)
        arrs = [_f64(sc[f]) for f in ("means", "log_scales", "quats", "opacity_logits", "sh")]
        g2k = np.ascontiguousarray(g2[off:off + k])
        m = model_array(mdl)
        rc = _L().orc_preprocess_adjoint(C.c_int64(k), *[_p(a) for a in arrs], C.c_int(sc["sh_degree"]), _mp(m),
                                         _p(cam_array(cam)), C.c_int(cam.W), C.c_int(cam.H),
                                         _p(opts_array(opts)), _p(g2k),
                                         *[_p(out[f]) for f in ("means", "log_scales", "quats",
                                                                "opacity_logits", "sh")])
        if rc != 0:
            raise ValueError("oracle preprocess adjoint failed")
        outs.append(out)
        off += k
    return outs


def dynamic_update(means0, velocity, logits0, amp, freq, phase, t):
    """FP64 frame-t update of the dynamic workload (stands in for the per-frame
    generator of section 3.3): mu_t = mu_0 + t v, logit_t = logit_0 + A sin(2 pi f t + phi).
    Computed from the float32 inputs and the float32 t."""
    t = float(np.float32(t))
    m = _f64(means0) + t * _f64(velocity)
    lg = _f64(logits0) + _f64(amp) * np.sin(2.0 * np.pi * _f64(freq) * t + _f64(phase))
    return m, lg
