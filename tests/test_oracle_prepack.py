"""Pins of the oracle's pre-packed input form (Algorithm 1's pre-pack; section 3.4's FP16
layout): a Gaussian given by mean, covariance upper triangle and opacity instead of
log-scales, quaternion and logit, and the fp16 packing itself.
  - with the exact covariance (numpy/scipy from scales and quaternions, an independent
    route) and the exact opacity, the image equals the scale/quaternion path's to 1e-12,
    also under a model transform;
  - the packed planes decode (numpy float16 views) to the decoded scene, every value is the
    nearest fp16 of the FP64 original, and the padding halves are zero.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2512_08478_b300 import synth


def _exact_cov_form(sc):
    q = sc["quats"].astype(np.float64)
    rot = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], 1)).as_matrix()
    s2 = np.exp(2.0 * sc["log_scales"].astype(np.float64))
    sig = np.einsum("nij,nj,nkj->nik", rot, s2, rot)
    cov6 = np.stack([sig[:, 0, 0], sig[:, 0, 1], sig[:, 0, 2], sig[:, 1, 1], sig[:, 1, 2], sig[:, 2, 2]], 1)
    return dict(means=sc["means"].astype(np.float64), cov6=cov6,
                opacity=1.0 / (1.0 + np.exp(-sc["opacity_logits"].astype(np.float64))),
                sh=sc["sh"].astype(np.float64), sh_degree=sc["sh_degree"])


def _same(a, b, tol):
    ok = (a["ambiguous"] == 0) & (b["ambiguous"] == 0)
    assert ok.mean() > 0.99
    assert np.abs(a["rgb"] - b["rgb"])[:, ok].max() <= tol
    assert np.abs(a["alpha"] - b["alpha"])[ok].max() <= tol


@pytest.mark.parametrize("deg", [0, 3])
def test_covariance_form_equals_scale_rotation_form(deg):
    sc = synth.mixture_scene(1500, 60 + deg, sh_degree=deg, components=8, ball_radius=1.0, comp_std=0.4,
                             log_scale_mean=-3.0, hi_std=0.2)
    cam = synth.look_at((0.3, 0.5, 4.0), (0, 0, 0), 128, 96, 50.0)
    a, pa = oracle.render(sc, cam, (0.1, 0.2, 0.3))
    b, pb = oracle.render(_exact_cov_form(sc), cam, (0.1, 0.2, 0.3))
    assert np.array_equal(pa["valid"], pb["valid"])
    assert np.abs(pa["conic"] - pb["conic"]).max() <= 1e-9 * np.abs(pa["conic"]).max()
    _same(a, b, 1e-12)
    M = synth.affine_model(np.random.default_rng(deg), shear=0.3)
    a, _ = oracle.render_multi([sc], [M], cam)
    b, _ = oracle.render_multi([_exact_cov_form(sc)], [M], cam)
    _same(a, b, 1e-12)


def test_covariance_entry_order_matters():
    """Swapping two entries of the upper triangle (xz <-> yy) changes the image."""
    sc = synth.mixture_scene(800, 70, sh_degree=0, components=4, ball_radius=0.8, comp_std=0.3,
                             log_scale_mean=-2.5)
    cam = synth.look_at((0.0, 0.0, 4.0), (0, 0, 0), 96, 96, 50.0)
    good = _exact_cov_form(sc)
    bad = dict(good, cov6=good["cov6"][:, [0, 1, 3, 2, 4, 5]].copy())
    a, _ = oracle.render(good, cam)
    b, _ = oracle.render(bad, cam)
    assert np.abs(a["alpha"] - b["alpha"]).max() > 1e-2


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_prepack_planes_decode_to_nearest_fp16(deg):
    sc = synth.mixture_scene(500, 80 + deg, sh_degree=deg, ball_radius=3.0)
    planes, dec = oracle.prepack(sc)
    n, K = 500, (deg + 1) ** 2
    assert planes["pos"].shape == (n, 2) and planes["cov"].shape == (n, 3)
    assert planes["col"].shape == (n, oracle.packed_words(deg))
    assert oracle.packed_words(deg) == {0: 2, 1: 6, 2: 14, 3: 24}[deg]
    pos = planes["pos"].view(np.float16).astype(np.float64)
    cov = planes["cov"].view(np.float16).astype(np.float64)
    col = planes["col"].view(np.float16).astype(np.float64)
    assert np.array_equal(pos[:, :3], dec["means"]) and np.array_equal(pos[:, 3], dec["opacity"])
    assert np.array_equal(cov, dec["cov6"])
    assert np.array_equal(col[:, : 3 * K], dec["sh"].reshape(n, 3 * K)) and not col[:, 3 * K:].any()
    ex = _exact_cov_form(sc)
    for got, want in ((dec["means"], ex["means"]), (dec["cov6"], ex["cov6"]), (dec["opacity"], ex["opacity"]),
                      (dec["sh"], ex["sh"])):
        g16 = got.astype(np.float16)
        up = np.nextafter(g16, np.float16(np.inf)).astype(np.float64)
        dn = np.nextafter(g16, np.float16(-np.inf)).astype(np.float64)
        err = np.abs(got - want)
        assert np.all(err <= np.abs(up - want) + 1e-300) and np.all(err <= np.abs(dn - want) + 1e-300)
