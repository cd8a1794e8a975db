"""Pins of the oracle's multi-model render (Algorithm 1: every model preprocessed with its
own affine transform M_k = [A | b], then one global sort and compositing over all
splats; section 3.4). Each check ties the transform path to something other than itself:
  - moving a model rigidly is the same as moving the camera the opposite way (this also
    fixes the frame of the SH evaluation: the model's own);
  - scaling the world about the camera centre leaves the image unchanged (perspective);
  - a general affine map of an SH0 model equals the plain scene whose Gaussians are the
    mapped ones, re-parametrised through numpy's eigendecomposition and scipy's rotations;
  - translated models drawn together equal the single merged scene bit for bit, and the
    global order differs from drawing one model over the other.
"""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle
from paper_2512_08478_b300 import synth


def _cam(R, t, like):
    return synth.Camera(R=np.asarray(R, np.float32), t=np.asarray(t, np.float32), fx=like.fx, fy=like.fy,
                        cx=like.cx, cy=like.cy, near=like.near, W=like.W, H=like.H)


def _scene(n, seed, deg, **kw):
    return synth.mixture_scene(n, seed, sh_degree=deg, components=8, ball_radius=0.8, comp_std=0.3,
                               log_scale_mean=-2.8, log_scale_std=0.4, hi_std=0.3, **kw)


def _close(a, b, tol):
    """Images a, b (render_tiled outputs) agree to tol outside either one's ambiguous pixels."""
    ok = (a["ambiguous"] == 0) & (b["ambiguous"] == 0)
    assert ok.mean() > 0.97
    assert np.abs(a["rgb"] - b["rgb"])[:, ok].max() <= tol
    assert np.abs(a["alpha"] - b["alpha"])[ok].max() <= tol


def test_identity_model_is_the_plain_render():
    sc = _scene(400, 1, 3)
    cam = synth.look_at((0.3, 0.4, 4.0), (0, 0, 0), 96, 80, 50.0)
    eye = np.concatenate([np.eye(3), np.zeros((3, 1))], 1)
    a, _ = oracle.render_multi([sc], [eye], cam, (0.1, 0.2, 0.3))
    b, _ = oracle.render(sc, cam, (0.1, 0.2, 0.3))
    for k in ("rgb", "alpha", "n_contrib"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rigid_model_equals_the_camera_moved_instead(seed):
    """Rendering M = [Q | b] from camera (R, t) is rendering the model itself from camera
    (R Q, R b + t): x_c = R (Q mu + b) + t, Sigma_c = R Q Sigma Q^T R^T, and the camera
    centre seen from the model is Q^T (c - b), the point the SH direction starts from."""
    rng = np.random.default_rng(seed)
    sc = _scene(500, 10 + seed, 3)
    cam = synth.look_at((0.5, 0.8, 4.5), (0, 0, 0), 96, 72, 50.0)
    Q = synth._axis_rotation(rng.standard_normal(3), rng.uniform(0.5, 2.5))
    b = rng.normal(0.0, 0.3, 3)
    M = np.concatenate([Q, b[:, None]], 1).astype(np.float32).astype(np.float64)
    Qf, bf = M[:, :3], M[:, 3]
    R, t = cam.R.astype(np.float64), cam.t.astype(np.float64)
    moved = _cam(R @ Qf, R @ bf + t, cam)
    a, _ = oracle.render_multi([sc], [M], cam)
    ref, _ = oracle.render(sc, moved)
    still, _ = oracle.render(sc, cam)
    assert np.abs(a["rgb"] - still["rgb"]).max() > 0.1        # the model did move
    _close(a, ref, 2e-5)     # the moved camera is rounded to float32 (~1e-7 relative)
    # the SH frame matters: colours evaluated along the world-space ray differ
    sh0 = dict(sc, sh=np.ascontiguousarray(sc["sh"][:, :1, :]), sh_degree=0)
    a0, _ = oracle.render_multi([sh0], [M], cam)
    assert np.abs(a["rgb"] - a0["rgb"]).max() > 1e-3          # SH3 terms are visible


@pytest.mark.parametrize("s", [0.5, 2.5])
def test_scaling_about_the_camera_centre_is_invisible(s):
    """x -> c + s (x - c) maps every Gaussian to one s times as far along the same ray and
    s times as large: the perspective image is unchanged."""
    sc = _scene(500, 20, 2)
    cam = synth.look_at((0.0, 0.0, 5.0), (0, 0, 0), 80, 64, 45.0)   # centre exact in float32
    R, t = cam.R.astype(np.float64), cam.t.astype(np.float64)
    c = -R.T @ t
    M = np.concatenate([s * np.eye(3), ((1.0 - s) * c)[:, None]], 1)
    assert np.array_equal(M.astype(np.float32).astype(np.float64), M)   # exact in float32
    a, _ = oracle.render_multi([sc], [M], cam)
    b, _ = oracle.render(sc, cam)
    _close(a, b, 1e-9)


def _merged_affine(sc, M):
    """The plain scene of the Gaussians mapped by M = [A | b]: means A mu + b, and the
    covariance A Sigma A^T re-parametrised as log-scales and a unit quaternion through
    numpy's symmetric eigendecomposition and scipy's rotation conversion."""
    A, b = M[:, :3], M[:, 3]
    q = sc["quats"].astype(np.float64)
    rot = Rotation.from_quat(np.stack([q[:, 1], q[:, 2], q[:, 3], q[:, 0]], 1)).as_matrix()
    s2 = np.exp(2.0 * sc["log_scales"].astype(np.float64))
    Sig = np.einsum("nij,nj,nkj->nik", rot, s2, rot)
    Sw = np.einsum("ij,njk,lk->nil", A, Sig, A)
    lam, V = np.linalg.eigh(Sw)
    V[np.linalg.det(V) < 0, :, 2] *= -1.0
    xyzw = Rotation.from_matrix(V).as_quat()
    return dict(means=sc["means"].astype(np.float64) @ A.T + b, log_scales=0.5 * np.log(lam),
                quats=np.stack([xyzw[:, 3], xyzw[:, 0], xyzw[:, 1], xyzw[:, 2]], 1),
                opacity_logits=sc["opacity_logits"].astype(np.float64), sh=sc["sh"].astype(np.float64),
                sh_degree=sc["sh_degree"])


@pytest.mark.parametrize("seed", [3, 4])
def test_general_affine_equals_the_mapped_scene(seed):
    rng = np.random.default_rng(seed)
    sc = _scene(600, 30 + seed, 0)
    cam = synth.look_at((0.4, 0.2, 4.5), (0, 0, 0), 96, 80, 50.0)
    M = synth.affine_model(rng, shear=0.5).astype(np.float64)
    a, _ = oracle.render_multi([sc], [M], cam)
    b, _ = oracle.render(_merged_affine(sc, M), cam)
    _close(a, b, 1e-9)
    # the covariance mapped the wrong way round (A^T Sigma A, same means) draws another image
    Mt = np.concatenate([M[:, :3].T, M[:, 3:]], 1)
    wrong = dict(_merged_affine(sc, Mt), means=_merged_affine(sc, M)["means"])
    c, _ = oracle.render(wrong, cam)
    assert np.abs(a["alpha"] - c["alpha"]).max() > 1e-2


def test_translated_models_equal_the_merged_scene_and_interleave():
    """Two models translated so that their depth ranges overlap: drawn together they are
    the single scene of both translated point sets (zero-padded to a common SH degree),
    bit for bit; drawing one whole model over the other gives a different image."""
    s1 = _scene(500, 40, 0)
    s2 = _scene(700, 41, 2)
    cam = synth.look_at((0.0, 0.0, 5.0), (0, 0, 0), 96, 96, 50.0)
    b1, b2 = np.array([0.25, 0.0, 0.125]), np.array([-0.25, 0.0625, -0.125])   # exact in float32
    M1 = np.concatenate([np.eye(3), b1[:, None]], 1)
    M2 = np.concatenate([np.eye(3), b2[:, None]], 1)
    multi, prep = oracle.render_multi([s1, s2], [M1, M2], cam, (0.0, 0.0, 0.0))
    K = 9
    sh1 = np.zeros((500, K, 3))
    sh1[:, :1] = s1["sh"]
    merged = dict(means=np.concatenate([s1["means"].astype(np.float64) + b1, s2["means"].astype(np.float64) + b2]),
                  log_scales=np.concatenate([s1["log_scales"], s2["log_scales"]]).astype(np.float64),
                  quats=np.concatenate([s1["quats"], s2["quats"]]).astype(np.float64),
                  opacity_logits=np.concatenate([s1["opacity_logits"], s2["opacity_logits"]]).astype(np.float64),
                  sh=np.concatenate([sh1, s2["sh"].astype(np.float64)]), sh_degree=2)
    ref, _ = oracle.render(merged, cam, (0.0, 0.0, 0.0))
    for k in ("rgb", "alpha", "n_contrib"):
        assert np.array_equal(multi[k], ref[k]), k
    # depth ranges overlap, so the global order interleaves the models
    z1, z2 = prep["z"][:500][prep["valid"][:500] == 1], prep["z"][500:][prep["valid"][500:] == 1]
    assert z1.min() < z2.max() and z2.min() < z1.max()
    i1, _ = oracle.render_multi([s1], [M1], cam)
    i2, _ = oracle.render_multi([s2], [M2], cam)
    over = i1["rgb"] + (1.0 - i1["alpha"])[None] * i2["rgb"]     # model 1 wholly in front
    assert np.abs(over - multi["rgb"]).max() > 0.05


def test_singular_model_is_rejected():
    sc = _scene(50, 50, 0)
    cam = synth.look_at((0.0, 0.0, 5.0), (0, 0, 0), 32, 32, 50.0)
    M = np.zeros((3, 4))
    M[0, 0] = M[1, 1] = 1.0
    with pytest.raises(ValueError):
        oracle.render_multi([sc], [M], cam)
    with pytest.raises(ValueError):
        oracle.render_multi([sc], [np.full((3, 4), np.nan)], cam)
