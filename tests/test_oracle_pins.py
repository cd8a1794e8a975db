"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test checks the oracle against a closed form, a textbook identity, an
invariant of the definition (section 3.2, Eqs. 1-3), brute force on tiny inputs,
or finite differences -- chosen so that a dropped term, a wrong sign or index or
a transposed operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2512_08478_b300 import synth

Y00 = 0.5 / math.sqrt(math.pi)   # textbook value of the degree-0 real SH
DIL = float(np.float32(0.3))      # the low-pass dilation as the library receives it (float32)


def _one_gaussian_scene(mu, sigma3, quat, logit, colour, deg=0):
    K = (deg + 1) ** 2
    sh = np.zeros((1, K, 3), np.float32)
    sh[0, 0, :] = (np.asarray(colour) - 0.5) / Y00
    return dict(means=np.array([mu], np.float32),
                log_scales=np.full((1, 3), math.log(sigma3), np.float32),
                quats=np.array([quat], np.float32),
                opacity_logits=np.array([logit], np.float32), sh=sh, sh_degree=deg)


def _stack(scenes):
    out = {k: np.concatenate([s[k] for s in scenes]) for k in
           ("means", "log_scales", "quats", "opacity_logits", "sh")}
    out["sh_degree"] = scenes[0]["sh_degree"]
    return out


def _dc_colour(scene, i):
    """Rendered colour of an SH0 Gaussian from its stored (float32) coefficient."""
    return scene["sh"][i, 0, :].astype(np.float64) * Y00 + 0.5


# ---------------------------------------------------------------------------------
# Closed forms (Eqs. 1-3)
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("quat", [(1, 0, 0, 0), (0.3, -0.5, 0.7, 0.2), (0, 0, 0, 1)])
@pytest.mark.parametrize("bg", [(0, 0, 0), (0.2, 0.5, 0.9)])
def test_single_isotropic_gaussian_closed_form(quat, bg):
    d, sig3, logit = 4.0, 0.05, 1.2
    W, H = 64, 48
    cam = synth.look_at((0, 0, d), (0, 0, 0), W, H, 60.0)
    sc = _one_gaussian_scene((0, 0, 0), sig3, quat, logit, (0.9, 0.4, 0.1))
    prep = oracle.preprocess(sc, cam)
    f = cam.fx
    s_true = math.exp(float(np.float32(math.log(sig3))))
    var = (f * s_true / d) ** 2 + DIL          # EWA on the optical axis + dilation
    assert prep["valid"][0] == 1
    np.testing.assert_allclose(prep["uv"][0], [W / 2, H / 2], atol=1e-12)
    np.testing.assert_allclose(prep["conic"][0], [1 / var, 0, 1 / var], rtol=1e-12, atol=1e-15)
    o = 1 / (1 + math.exp(-float(np.float32(logit))))
    c = _dc_colour(sc, 0)
    ys, xs = np.mgrid[0:H, 0:W]
    rho2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2
    a = np.minimum(float(np.float32(0.99)), o * np.exp(-rho2 / (2 * var)))
    a = np.where((rho2 / var <= 9.0) & (a >= np.float32(1 / 255)), a, 0.0)
    expect = c[:, None, None] * a + np.asarray(bg)[:, None, None] * (1 - a)
    for img in (oracle.render_bruteforce(prep, W, H, bg), oracle.render_tiled(prep, W, H, bg)):
        np.testing.assert_allclose(img["rgb"], expect, atol=1e-12)
        np.testing.assert_allclose(img["alpha"], a, atol=1e-12)


def test_two_coaxial_gaussians_closed_form_and_order():
    W, H, d = 40, 40, 5.0
    cam = synth.look_at((0, 0, d), (0, 0, 0), W, H, 60.0)
    g_front = _one_gaussian_scene((0, 0, 1.0), 0.06, (1, 0, 0, 0), 0.5, (1.0, 0.0, 0.2))
    g_back = _one_gaussian_scene((0, 0, -1.0), 0.12, (1, 0, 0, 0), 2.0, (0.1, 0.8, 0.3))
    bg = np.array([0.3, 0.3, 0.6])
    ys, xs = np.mgrid[0:H, 0:W]
    rho2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2

    def alpha(g, z):
        s = float(np.exp(np.float64(g["log_scales"][0, 0])))
        var = (cam.fx * s / z) ** 2 + DIL
        o = 1 / (1 + math.exp(-float(g["opacity_logits"][0])))
        a = np.minimum(float(np.float32(0.99)), o * np.exp(-rho2 / (2 * var)))
        return np.where((rho2 / var <= 9) & (a >= np.float32(1 / 255)), a, 0.0)

    a1, a2 = alpha(g_front, d - 1.0), alpha(g_back, d + 1.0)
    c1, c2 = _dc_colour(g_front, 0), _dc_colour(g_back, 0)
    assert np.all((1 - a1) * (1 - a2) >= 1e-4)   # no early stop in this scene
    expect = (c1[:, None, None] * a1 + c2[:, None, None] * a2 * (1 - a1)
              + bg[:, None, None] * (1 - a1) * (1 - a2))
    for order in ([g_front, g_back], [g_back, g_front]):   # input order must not matter
        sc = _stack(order)
        img, _ = oracle.render(sc, cam, bg)
        np.testing.assert_allclose(img["rgb"], expect, atol=1e-12)
        np.testing.assert_allclose(img["alpha"], 1 - (1 - a1) * (1 - a2), atol=1e-12)


def test_depth_buffer_closed_forms():
    """Depth-buffer-aware compositing (a splat deeper than the pixel's depth value is not
    composited there): a plane between two coaxial Gaussians leaves the front one's closed
    form over the background; +inf everywhere changes nothing; a plane in front of both
    leaves the background; a plane that covers half the image splits it accordingly."""
    W, H, d = 40, 40, 5.0
    cam = synth.look_at((0, 0, d), (0, 0, 0), W, H, 60.0)
    g_front = _one_gaussian_scene((0, 0, 1.0), 0.06, (1, 0, 0, 0), 0.5, (1.0, 0.0, 0.2))
    g_back = _one_gaussian_scene((0, 0, -1.0), 0.12, (1, 0, 0, 0), 2.0, (0.1, 0.8, 0.3))
    sc = _stack([g_back, g_front])
    bg = np.array([0.3, 0.3, 0.6])
    ys, xs = np.mgrid[0:H, 0:W]
    rho2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2
    s = float(np.exp(np.float64(g_front["log_scales"][0, 0])))
    var = (cam.fx * s / (d - 1.0)) ** 2 + DIL
    o = 1 / (1 + math.exp(-float(g_front["opacity_logits"][0])))
    a1 = np.minimum(float(np.float32(0.99)), o * np.exp(-rho2 / (2 * var)))
    a1 = np.where((rho2 / var <= 9) & (a1 >= np.float32(1 / 255)), a1, 0.0)
    c1 = _dc_colour(g_front, 0)
    front_only = c1[:, None, None] * a1 + bg[:, None, None] * (1 - a1)
    plane = np.full((H, W), d, np.float32)                    # between the two (depths 4 and 6)
    img, _ = oracle.render(sc, cam, bg, depth=plane)
    np.testing.assert_allclose(img["rgb"], front_only, atol=1e-12)
    np.testing.assert_allclose(img["alpha"], a1, atol=1e-12)
    bf = oracle.render_bruteforce(oracle.preprocess(sc, cam), W, H, bg, depth=plane)
    np.testing.assert_allclose(bf["rgb"], front_only, atol=1e-12)
    free, _ = oracle.render(sc, cam, bg)
    inf, _ = oracle.render(sc, cam, bg, depth=np.full((H, W), np.inf, np.float32))
    assert np.array_equal(inf["rgb"], free["rgb"]) and np.array_equal(inf["alpha"], free["alpha"])
    wall, _ = oracle.render(sc, cam, bg, depth=np.full((H, W), 1.0, np.float32))
    assert np.all(wall["rgb"] == bg[:, None, None]) and np.all(wall["alpha"] == 0.0)
    half = np.where(xs < W // 2, np.float32(1.0), np.float32(np.inf)).astype(np.float32)
    split, _ = oracle.render(sc, cam, bg, depth=half)
    assert np.all(split["rgb"][:, :, : W // 2] == bg[:, None, None])
    assert np.array_equal(split["rgb"][:, :, W // 2:], free["rgb"][:, :, W // 2:])
    # the test read literally (reject where z > limit): -inf rejects every splat, NaN none
    ninf, _ = oracle.render(sc, cam, bg, depth=np.full((H, W), -np.inf, np.float32))
    assert np.all(ninf["rgb"] == bg[:, None, None]) and np.all(ninf["alpha"] == 0.0)
    nan, _ = oracle.render(sc, cam, bg, depth=np.full((H, W), np.nan, np.float32))
    assert np.array_equal(nan["rgb"], free["rgb"]) and np.array_equal(nan["alpha"], free["alpha"])


def test_early_stop_excludes_the_stopping_splat():
    # Three Gaussians stacked on the optical axis, seen at the pixel whose centre is
    # the principal point (G = 1 there): alpha = 0.99 (clamped), then 0.95, 0.95.
    # T goes 1 -> 0.01 -> 5e-4 -> 2.5e-5 < 1e-4, so the third splat is excluded.
    W = H = 15
    cam = synth.look_at((0, 0, 5), (0, 0, 0), W, H, 60.0)
    l95 = math.log(0.95 / 0.05)
    gs = [_one_gaussian_scene((0, 0, z), 0.3, (1, 0, 0, 0), lg, (1, 1, 1))
          for z, lg in ((0.5, 20.0), (0.0, l95), (-0.5, l95))]
    img, _ = oracle.render(_stack(gs), cam)
    a1 = float(np.float32(0.99))
    o2 = 1 / (1 + math.exp(-float(np.float32(l95))))
    assert img["n_contrib"][7, 7] == 2
    np.testing.assert_allclose(img["T"][7, 7], (1 - a1) * (1 - o2), rtol=1e-12)
    c = _dc_colour(gs[0], 0)
    np.testing.assert_allclose(img["rgb"][:, 7, 7], c * (a1 + o2 * (1 - a1)), rtol=1e-12)


# ---------------------------------------------------------------------------------
# Invariants
# ---------------------------------------------------------------------------------

def test_zero_opacity_returns_background():
    sc, cams = synth.workload_small()
    sc = dict(sc)
    sc["opacity_logits"] = np.full_like(sc["opacity_logits"], -30.0)
    bg = (0.25, 0.5, 0.75)
    img, prep = oracle.render(sc, cams[0], bg)
    assert prep["valid"].sum() == 0
    assert np.all(img["rgb"] == np.asarray(bg)[:, None, None])
    assert np.all(img["alpha"] == 0.0)


def _small_random_scene(n=600, seed=5, deg=0):
    sc = synth.uniform_cube_scene(n, seed, sh_degree=deg, log_scale_mean=-3.0)
    cam = synth.look_at((0.3, -0.2, 3.5), (0, 0, 0), 72, 56, 60.0)
    return sc, cam


def test_background_linearity_and_bounds():
    sc, cam = _small_random_scene()
    bg = np.array([0.7, 0.2, 0.4])
    a, _ = oracle.render(sc, cam, (0, 0, 0))
    b, _ = oracle.render(sc, cam, bg)
    np.testing.assert_allclose(b["rgb"] - a["rgb"], a["T"][None] * bg[:, None, None], atol=1e-14)
    assert np.all(a["T"] >= np.float32(1e-4)) and np.all(a["T"] <= 1.0)
    assert np.all(b["rgb"] >= 0) and np.all(b["rgb"] <= 1 + 1e-12)   # SH0 colours, bg in [0,1]


def test_transmittance_monotone_when_adding_splats():
    sc, cam = _small_random_scene(n=300)
    prev = None
    for k in (50, 120, 300):   # a superset of splats can only lower T (cut decisions fixed per splat)
        sub = {key: (v[:k] if isinstance(v, np.ndarray) else v) for key, v in sc.items()}
        img, _ = oracle.render(sub, cam, opts=dict(t_stop=0.0))
        if prev is not None:
            assert np.all(img["T"] <= prev + 1e-15)
        prev = img["T"]


def test_tile_size_independence_equals_bruteforce():
    sc, cam = _small_random_scene(n=1500, seed=9, deg=2)
    prep = oracle.preprocess(sc, cam)
    ref = oracle.render_bruteforce(prep, cam.W, cam.H)
    for T in (8, 16, 32):
        o = dict(tile=T)
        p = oracle.preprocess(sc, cam, o)
        img = oracle.render_tiled(p, cam.W, cam.H, opts=o)
        assert np.array_equal(img["rgb"], ref["rgb"])
        assert np.array_equal(img["n_contrib"], ref["n_contrib"])


def test_shuffle_invariance():
    sc, cam = _small_random_scene(n=800, seed=11, deg=1)
    perm = np.random.default_rng(0).permutation(800)
    shuf = {k: (v[perm] if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
    a, pa = oracle.render(sc, cam)
    b, pb = oracle.render(shuf, cam)
    assert len(np.unique(pa["zkey"][pa["valid"] == 1])) == (pa["valid"] == 1).sum()  # distinct depths
    np.testing.assert_allclose(a["rgb"], b["rgb"], atol=1e-13)


def test_bruteforce_tiny_scene_matches_python_reference():
    """A from-scratch pure-Python per-pixel depth sort over precomputed splats."""
    sc, cam = _small_random_scene(n=40, seed=3)
    prep = oracle.preprocess(sc, cam)
    W, H = 24, 20
    img = oracle.render_bruteforce(prep, W, H, (0.1, 0.2, 0.3))
    valid = [i for i in range(40) if prep["valid"][i]]
    order = sorted(valid, key=lambda i: (float(prep["zkey"][i]), i))
    a_min, t_stop = float(np.float32(1 / 255)), float(np.float32(1e-4))
    a_max = float(np.float32(0.99))
    for y in range(0, H, 3):
        for x in range(0, W, 3):
            T, col = 1.0, [0.0, 0.0, 0.0]
            for i in order:
                dx, dy = x + 0.5 - prep["uv"][i, 0], y + 0.5 - prep["uv"][i, 1]
                a, b, c = prep["conic"][i]
                q = a * dx * dx + 2 * b * dx * dy + c * dy * dy
                if q > 9:
                    continue
                al = min(a_max, prep["opacity"][i] * math.exp(-q / 2))
                if al < a_min:
                    continue
                if T * (1 - al) < t_stop:
                    break
                for ch in range(3):
                    col[ch] += prep["rgb"][i, ch] * al * T
                T *= 1 - al
            exp = [col[ch] + T * (0.1, 0.2, 0.3)[ch] for ch in range(3)]
            np.testing.assert_allclose(img["rgb"][:, y, x], exp, atol=1e-13)


# ---------------------------------------------------------------------------------
# Spherical harmonics
# ---------------------------------------------------------------------------------

def test_sh_orthonormal_by_quadrature():
    zs, wz = np.polynomial.legendre.leggauss(12)
    nphi = 24
    phis = 2 * np.pi * np.arange(nphi) / nphi
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        r = math.sqrt(1 - z * z)
        for ph in phis:
            Y = oracle.sh_eval(3, (r * math.cos(ph), r * math.sin(ph), z))
            G += np.outer(Y, Y) * w * (2 * np.pi / nphi)
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)


def test_sh_textbook_low_orders():
    rng = np.random.default_rng(1)
    for _ in range(5):
        d = rng.standard_normal(3)
        x, y, z = d / np.linalg.norm(d)
        Y = oracle.sh_eval(2, (x, y, z))
        c1 = math.sqrt(3 / (4 * math.pi))
        np.testing.assert_allclose(Y[0], Y00, rtol=1e-14)
        # Condon-Shortley phase: Y_1^-1 = -c y, Y_1^0 = c z, Y_1^1 = -c x
        np.testing.assert_allclose(Y[1:4], [-c1 * y, c1 * z, -c1 * x], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(Y[6], math.sqrt(5 / (16 * math.pi)) * (3 * z * z - 1), rtol=1e-12,
                                   atol=1e-15)
        np.testing.assert_allclose(Y[8], math.sqrt(15 / (16 * math.pi)) * (x * x - y * y), rtol=1e-12,
                                   atol=1e-15)


def test_sh0_colour_is_view_independent():
    sc = synth.mixture_scene(2000, 7, sh_degree=0)
    cams = synth.orbit_cameras(32, 15.0, 320, 180, 50.0)
    cols = []
    for cam in cams:
        p = oracle.preprocess(sc, cam)
        cols.append(np.where(p["valid"][:, None] == 1, p["rgb"], np.nan))
    cols = np.stack(cols)
    ref = np.maximum(sc["sh"][:, 0, :].astype(np.float64) * Y00 + 0.5, 0)
    ok = ~np.isnan(cols)
    assert ok.sum() > 1000
    np.testing.assert_allclose(cols[ok], np.broadcast_to(ref, cols.shape)[ok], atol=1e-14)


# ---------------------------------------------------------------------------------
# Covariance and projection
# ---------------------------------------------------------------------------------

def test_covariance_invariants():
    rng = np.random.default_rng(2)
    ls = rng.normal(-2, 0.5, (20, 3))
    q = rng.standard_normal((20, 4))
    S = oracle.covariance(ls, q)
    S_neg = oracle.covariance(ls, -q)
    S_scaled = oracle.covariance(ls, 3.7 * q)
    np.testing.assert_allclose(S, np.transpose(S, (0, 2, 1)), atol=1e-16)
    np.testing.assert_allclose(S, S_neg, atol=1e-15)
    np.testing.assert_allclose(S, S_scaled, atol=1e-15)
    for i in range(20):
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(S[i])), np.sort(np.exp(2 * ls[i])), rtol=1e-10)
    # 90 degrees about z maps the x-axis onto the y-axis: Sigma = diag(sy^2, sx^2, sz^2)
    h = math.sqrt(0.5)
    S90 = oracle.covariance(np.log([[0.1, 0.2, 0.3]]), [[h, 0, 0, h]])[0]
    np.testing.assert_allclose(S90, np.diag([0.04, 0.01, 0.09]), atol=1e-15)
    # isotropic scales: independent of rotation
    Si = oracle.covariance(np.log([[0.2, 0.2, 0.2]] * 3), rng.standard_normal((3, 4)))
    np.testing.assert_allclose(Si, np.broadcast_to(0.04 * np.eye(3), Si.shape), atol=1e-15)


def _project(cam, X):
    """Pinhole camera model (the input convention): pixel coordinates of world points."""
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    p = X @ R.T + t
    return np.stack([cam.fx * p[:, 0] / p[:, 2] + cam.cx, cam.fy * p[:, 1] / p[:, 2] + cam.cy], 1)


def test_ewa_matches_projected_sample_covariance():
    """Eq. 1: S = J Sigma J^T is the linearised covariance of the projected Gaussian."""
    cam = synth.look_at((1.0, 0.5, 6.0), (0, 0, 0), 200, 150, 60.0)
    sc = dict(means=np.array([[0.6, -0.4, 0.3]], np.float32),
              log_scales=np.log(np.array([[0.004, 0.0015, 0.002]], np.float32)),
              quats=np.array([[0.8, 0.2, -0.3, 0.4]], np.float32),
              opacity_logits=np.array([3.0], np.float32), sh=np.zeros((1, 1, 3), np.float32), sh_degree=0)
    prep = oracle.preprocess(sc, cam, dict(dilation=0.0))
    Sig = oracle.covariance(sc["log_scales"].astype(np.float64), sc["quats"].astype(np.float64))[0]
    rng = np.random.default_rng(0)
    X = rng.multivariate_normal(sc["means"][0].astype(np.float64), Sig, 400_000)
    P = _project(cam, X)
    emp = np.cov(P.T)
    s00, s01, s11 = prep["S"][0]
    np.testing.assert_allclose([s00, s01, s11], [emp[0, 0], emp[0, 1], emp[1, 1]], rtol=0.02,
                               atol=0.02 * max(s00, s11))
    np.testing.assert_allclose(prep["uv"][0], _project(cam, sc["means"].astype(np.float64))[0], atol=1e-9)
    np.testing.assert_allclose(prep["z"][0], (cam.R.astype(np.float64) @ sc["means"][0] + cam.t)[2],
                               atol=1e-12)


def test_ewa_jacobian_matches_numerical_derivative_of_projection():
    cam = synth.look_at((0.5, 1.0, 5.0), (0, 0, 0), 160, 120, 60.0)
    mu = np.array([0.3, -0.2, 0.4])
    h = 1e-6
    Jn = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        Jn[:, k] = (_project(cam, (mu + e)[None])[0] - _project(cam, (mu - e)[None])[0]) / (2 * h)
    # an isotropic Sigma = s^2 I gives S = s^2 Jn Jn^T (+ dilation 0 here)
    s = 0.01
    sc = dict(means=mu[None].astype(np.float32), log_scales=np.full((1, 3), math.log(s)),
              quats=np.array([[1, 0, 0, 0]], np.float32), opacity_logits=np.array([3.0], np.float32),
              sh=np.zeros((1, 1, 3), np.float32), sh_degree=0)
    sc["means"] = mu[None]   # exact fp64 mean for this check
    prep = oracle.preprocess(sc, cam, dict(dilation=0.0))
    s_eff = math.exp(float(np.float64(sc["log_scales"][0, 0])))
    expect = s_eff ** 2 * (Jn @ Jn.T)
    np.testing.assert_allclose(prep["S"][0], [expect[0, 0], expect[0, 1], expect[1, 1]], rtol=1e-6)


def test_tilted_anisotropic_gaussian_alpha_closed_form():
    """Eqs. 1-2 for a splat whose screen ellipse is tilted: at every pixel the alpha is
    min(0.99, o exp(-d^T S^-1 d / 2)), S = J Sigma J^T + dilation I. Here J is the numerical
    Jacobian of the projection, Sigma = R diag(s^2) R^T with R from scipy's quaternion
    rotation, and S^-1 comes from numpy, so the conic's off-diagonal term and the factor 2 of
    its cross term both enter the comparison."""
    from scipy.spatial.transform import Rotation
    W, H = 96, 80
    cam = synth.look_at((0.7, -0.4, 5.0), (0, 0, 0), W, H, 50.0)
    mu = np.array([0.15, -0.1, 0.2])
    s = np.array([0.3, 0.06, 0.15])
    q = np.array([0.8, 0.2, -0.3, 0.4])            # (w, x, y, z)
    logit = 2.0
    sc = dict(means=mu[None], log_scales=np.log(s)[None], quats=q[None], opacity_logits=np.array([logit]),
              sh=np.zeros((1, 1, 3)), sh_degree=0)
    prep = oracle.preprocess(sc, cam)
    assert prep["valid"][0] == 1
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    s_eff = np.exp(np.log(s))
    Sig = R @ np.diag(s_eff ** 2) @ R.T
    h = 1e-6
    Jn = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        Jn[:, k] = (_project(cam, (mu + e)[None])[0] - _project(cam, (mu - e)[None])[0]) / (2 * h)
    S = Jn @ Sig @ Jn.T + DIL * np.eye(2)
    assert abs(S[0, 1]) > 0.2 * math.sqrt(S[0, 0] * S[1, 1])   # the ellipse is tilted
    Sinv = np.linalg.inv(S)
    uv = _project(cam, mu[None])[0]
    ys, xs = np.mgrid[0:H, 0:W]
    d = np.stack([xs + 0.5 - uv[0], ys + 0.5 - uv[1]], -1)
    qq = np.einsum("...i,ij,...j->...", d, Sinv, d)
    o = 1 / (1 + math.exp(-logit))
    raw = o * np.exp(-0.5 * qq)
    a = np.minimum(float(np.float32(0.99)), raw)
    amin = float(np.float32(1 / 255))
    a = np.where((qq <= 9.0) & (a >= amin), a, 0.0)
    # decisions within rounding of a threshold are left out (both outcomes are correct there)
    clear = (np.abs(qq - 9.0) > 1e-6) & (np.abs(raw - amin) > 1e-9)
    got = oracle.render_bruteforce(prep, W, H)["alpha"]
    assert (a > 0).sum() > 100
    np.testing.assert_allclose(got[clear], a[clear], atol=1e-8)


# ---------------------------------------------------------------------------------
# Sort-stage oracles (brute force)
# ---------------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["random", "equal", "few_tiles", "sorted", "reverse"])
def test_stable_sort_matches_python_sorted(kind):
    keys, vals = synth.random_keys(3000, 4, kind)
    vals = np.random.default_rng(1).permutation(3000).astype(np.uint32)
    ok, ov = oracle.stable_sort_pairs(keys, vals)
    order = sorted(range(3000), key=lambda j: (int(keys[j]), j))
    assert np.array_equal(ok, keys[order])
    assert np.array_equal(ov, vals[order])


def test_duplicate_and_ranges_match_naive_loops():
    rng = np.random.default_rng(3)
    n, tiles_x, tiles_y = 200, 7, 5
    x0 = rng.integers(0, tiles_x, n)
    y0 = rng.integers(0, tiles_y, n)
    rect = np.stack([x0, y0, np.minimum(tiles_x, x0 + rng.integers(0, 3, n)),
                     np.minimum(tiles_y, y0 + rng.integers(0, 3, n))], 1)
    valid = (rng.uniform(size=n) > 0.2).astype(np.int32)
    zkey = rng.uniform(0.5, 9, n).astype(np.float32)
    keys, vals = oracle.duplicate_raw(valid, rect, zkey, tiles_x)
    ek, ev = [], []
    for i in range(n):
        if not valid[i]:
            continue
        for ty in range(rect[i, 1], rect[i, 3]):
            for tx in range(rect[i, 0], rect[i, 2]):
                ek.append(((ty * tiles_x + tx) << 32) | int(zkey[i].view(np.uint32)))
                ev.append(i)
    assert keys.tolist() == ek and vals.tolist() == ev
    sk, sv = oracle.stable_sort_pairs(keys, vals)
    r = oracle.tile_ranges(sk, tiles_x * tiles_y)
    for t in range(tiles_x * tiles_y):
        idx = [j for j in range(len(sk)) if (int(sk[j]) >> 32) == t]
        if idx:
            assert (r[t, 0], r[t, 1]) == (idx[0], idx[-1] + 1)
        else:
            assert r[t, 0] == r[t, 1]


def test_dynamic_update_reference_pins():
    sc, ex, _ = synth.workload_dynamic(n=1000, frames=4)
    m0, l0 = oracle.dynamic_update(sc["means"], ex["velocity"], sc["opacity_logits"], ex["amp"], ex["freq"],
                                   ex["phase"], 0.0)
    assert np.array_equal(m0, sc["means"].astype(np.float64))                 # t = 0: unchanged means
    np.testing.assert_allclose(l0, sc["opacity_logits"] + ex["amp"] * np.sin(ex["phase"].astype(np.float64)),
                               atol=1e-12)
    ma, la = oracle.dynamic_update(sc["means"], ex["velocity"], sc["opacity_logits"], ex["amp"], ex["freq"],
                                   ex["phase"], 0.25)
    mb, lb = oracle.dynamic_update(sc["means"], ex["velocity"], sc["opacity_logits"], ex["amp"], ex["freq"],
                                   ex["phase"], 1.25)
    np.testing.assert_allclose(lb, la, atol=1e-9)                              # integer f: period 1 in t
    np.testing.assert_allclose(mb - ma, ex["velocity"].astype(np.float64), atol=1e-9)   # linear in t


# ---------------------------------------------------------------------------------
# Depth ties and the off-axis Jacobian guard (readings S9 and S5)
# ---------------------------------------------------------------------------------

def test_equal_depths_composite_in_index_order():
    """Two Gaussians at the same point (same depth to the bit) with different colours and
    opacities: the lower index is in front (ties go by index), so at the centre pixel
    C = c0 a0 + c1 a1 (1 - a0) + bg (1 - a0)(1 - a1), and listing them the other way round
    swaps the roles."""
    W, H, d = 32, 32, 4.0
    cam = synth.look_at((0, 0, d), (0, 0, 0), W, H, 60.0)
    g0 = _one_gaussian_scene((0, 0, 0), 0.08, (1, 0, 0, 0), 0.8, (0.9, 0.1, 0.1))
    g1 = _one_gaussian_scene((0, 0, 0), 0.08, (1, 0, 0, 0), -0.4, (0.1, 0.1, 0.9))
    bg = np.array([0.0, 0.5, 0.0])
    px, py = W // 2, H // 2                      # pixel centre 0.5 px off the splat centre
    for order in ((g0, g1), (g1, g0)):
        sc = _stack(list(order))
        img, prep = oracle.render(sc, cam, bg)
        assert prep["zkey"][0] == prep["zkey"][1]
        s = math.exp(float(np.float32(math.log(0.08))))
        var = (cam.fx * s / d) ** 2 + DIL
        G = math.exp(-0.5 * (0.5 ** 2 + 0.5 ** 2) / var)
        a = [1 / (1 + math.exp(-float(g["opacity_logits"][0]))) * G for g in order]
        c = [_dc_colour(g, 0) for g in order]
        want = c[0] * a[0] + c[1] * a[1] * (1 - a[0]) + bg * (1 - a[0]) * (1 - a[1])
        np.testing.assert_allclose(img["rgb"][:, py, px], want, atol=1e-12)


def test_jacobian_guard_freezes_the_footprint_beyond_it():
    """J is taken at x/z clamped to 1.3 tan(half FOV): beyond the guard, moving a Gaussian
    further sideways at the same depth leaves its projected covariance unchanged (only the
    centre moves), while inside the guard the covariance does change."""
    W, H, d = 64, 48, 5.0
    cam = synth.look_at((0, 0, d), (0, 0, 0), W, H, 60.0)
    limx = 1.3 * (W / (2.0 * cam.fx))
    sig = 0.6                                     # large: reaches the image from outside it
    outs = []
    for k in (1.6, 2.4):                          # x/z beyond the guard, both sides
        for sgn in (1.0, -1.0):
            x = sgn * k * limx * d                # camera at z = d looking at the origin
            sc = _one_gaussian_scene((x, 0.0, 0.0), sig, (1, 0, 0, 0), 2.0, (0.5, 0.5, 0.5))
            outs.append(oracle.preprocess(sc, cam)["S"][0])
    assert min(np.abs(o).max() for o in outs) > 0
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[3])
    inside = [oracle.preprocess(_one_gaussian_scene((f * limx * d, 0, 0), sig, (1, 0, 0, 0), 2.0,
                                                     (0.5, 0.5, 0.5)), cam)["S"][0] for f in (0.2, 0.6)]
    assert np.abs(inside[0] - inside[1]).max() > 1e-3 * np.abs(inside[0]).max()


def test_thresholds_at_equality():
    """The readings at exact equality: a splat whose alpha equals alpha_min is composited (only
    alpha < 1/255 is skipped), and a splat whose depth equals the depth-buffer value passes
    the depth test (only deeper splats are rejected). Built exactly: the pre-packed form gives
    the opacity directly (the float32 alpha_min itself), the splat sits on a pixel centre (odd
    image size, q = 0, so alpha = opacity), and the buffer holds the splat's own float32 depth."""
    W = H = 33
    cam = synth.look_at((0, 0, 4.0), (0, 0, 0), W, H, 60.0)
    amin = float(np.float32(1.0 / 255.0))
    bg = np.array([0.2, 0.3, 0.4])
    sc = dict(means=np.zeros((1, 3)), cov6=np.array([[0.01, 0, 0, 0.01, 0, 0.01]]), opacity=np.array([amin]),
              sh=((np.array([[[0.9, 0.1, 0.5]]]) - 0.5) / Y00), sh_degree=0)
    img, prep = oracle.render(sc, cam, bg)
    assert prep["valid"][0] == 1 and prep["uv"][0, 0] == W / 2 and prep["uv"][0, 1] == H / 2
    c = np.array([0.9, 0.1, 0.5])
    np.testing.assert_allclose(img["rgb"][:, H // 2, W // 2], c * amin + bg * (1 - amin), atol=1e-15)
    assert img["n_contrib"][H // 2, W // 2] == 1
    # depth test at equality
    sc2 = _one_gaussian_scene((0, 0, 0), 0.05, (1, 0, 0, 0), 2.0, (0.9, 0.1, 0.5))
    free, p2 = oracle.render(sc2, cam, bg)
    z = p2["zkey"][0]
    eq, _ = oracle.render(sc2, cam, bg, depth=np.full((H, W), z, np.float32))
    assert np.array_equal(eq["rgb"], free["rgb"]) and free["alpha"].max() > 0.5
    below = np.nextafter(np.float32(z), np.float32(-np.inf))
    wall, _ = oracle.render(sc2, cam, bg, depth=np.full((H, W), below, np.float32))
    assert np.all(wall["alpha"] == 0.0)


def _axis_splats(opacities, depths_world, screen_var, cam):
    """Pre-packed isotropic splats on the optical axis (world z given), each with the given
    screen-space variance before dilation (Sigma = var z^2 / fx^2 I at view depth z = 4 - z_w)."""
    n = len(opacities)
    cov6 = np.zeros((n, 6))
    for j, zw in enumerate(depths_world):
        s2 = screen_var * (4.0 - zw) ** 2 / float(cam.fx) ** 2
        cov6[j] = [s2, 0, 0, s2, 0, s2]
    return dict(means=np.array([[0.0, 0.0, zw] for zw in depths_world]), cov6=cov6,
                opacity=np.asarray(opacities, np.float64), sh=np.zeros((n, 1, 3)), sh_degree=0)


def test_ambiguity_flags_mark_decisions_at_their_thresholds():
    """A pixel is flagged ambiguous when one of its decisions lies within float32 rounding of
    its threshold: the early stop (T (1 - alpha) against 1e-4), the alpha_min skip, the 3-sigma
    cut (q against 9, for a splat that would pass alpha_min) and the depth test. Each decision is
    placed here 1e-6 (relative) from its threshold, where the pixel must be flagged, and then
    far from it, where it must not be. The camera looks down the axis from (0, 0, 4) onto an
    odd-sized image, so the centre pixel sees q = 0 and alpha = opacity."""
    W = H = 33
    cam = synth.look_at((0, 0, 4.0), (0, 0, 0), W, H, 60.0)
    f32 = lambda v: float(np.float32(v))
    t_stop, amin, amax = f32(1e-4), f32(1 / 255), f32(0.99)
    cx, cy = np.array([W // 2]), np.array([H // 2])

    def flag(scene, px=cx, py=cy, depth=None):
        prep = oracle.preprocess(scene, cam)
        assert prep["valid"].all()
        return int(oracle.render_pixels(prep, px, py, depth=depth)["ambiguous"][0])

    # early stop: alpha 0.99 (clamped), then a2 with 0.01 (1 - a2) = t_stop (1 + e)
    for e, want in ((1e-6, 1), (0.3, 0)):
        a2 = 1.0 - t_stop * (1.0 + e) / (1.0 - amax)
        assert flag(_axis_splats([1.0, a2], [0.5, 0.0], 1.0, cam)) == want, ("stop", e)
    # alpha_min skip: opacity alpha_min (1 + e) at q = 0
    for e, want in ((1e-6, 1), (30.0, 0)):
        assert flag(_axis_splats([amin * (1.0 + e)], [0.0], 1.0, cam)) == want, ("alpha_min", e)
    # 3-sigma cut: the pixel 3 px right of the centre sees q = 9 / var (dilation added to var)
    for qv, want in ((9.0 * (1.0 + 1e-6), 1), (4.0, 0)):
        var = 9.0 / qv - DIL
        assert flag(_axis_splats([0.9], [0.0], var, cam), px=cx + 3) == want, ("cut", qv)
    # depth test: a buffer value 1e-7 (relative) beyond the splat's float32 view depth
    sc = _axis_splats([0.5], [0.0], 1.0, cam)
    z = float(oracle.preprocess(sc, cam)["zkey"][0])
    for lim, want in ((z * (1.0 + 1e-7), 1), (z + 1.0, 0)):
        assert flag(sc, depth=np.array([lim], np.float32)) == want, ("depth", lim)


def test_near_plane_at_equality():
    """Reading S6 at equality: a Gaussian whose view depth equals the near plane is culled
    (z <= near), and one a double-precision step beyond it is kept. The camera looks down the
    axis from (0, 0, 4) with an exact rotation (entries 0 and +-1), so a mean on the axis at
    world z = 4 - near has view depth near exactly."""
    cam = synth.look_at((0, 0, 4.0), (0, 0, 0), 33, 33, 60.0)
    assert np.array_equal(cam.R[2], [0, 0, -1]) and cam.t[2] == 4.0
    near = float(np.float32(cam.near))   # the near plane as the library receives it
    on = 4.0 - near
    beyond = np.nextafter(on, -np.inf)
    for zw, depth_ok in ((on, False), (beyond, True)):
        sc = dict(means=np.array([[0.0, 0.0, zw]]), log_scales=np.log(np.full((1, 3), 0.01)),
                  quats=np.array([[1.0, 0, 0, 0]]), opacity_logits=np.array([2.0]), sh=np.zeros((1, 1, 3)),
                  sh_degree=0)
        prep = oracle.preprocess(sc, cam)
        assert (prep["z"][0] > near) == depth_ok and (prep["z"][0] == near) != depth_ok
        assert prep["valid"][0] == (1 if depth_ok else 0)


def test_negative_colour_sum_renders_black_closed_form():
    """Reading S2's clamp rgb = max(0, sum + 0.5): an SH0 Gaussian whose stored DC gives a
    negative sum in one channel draws that channel as a black splat, bg (1 - alpha), with the
    other channels at their closed form; the adjoint passes no gradient to the clamped
    channel's coefficient and the textbook c alpha to the others (dC/dc = alpha per pixel)."""
    d, sig3, logit = 4.0, 0.05, 1.2
    W, H = 48, 40
    cam = synth.look_at((0, 0, d), (0, 0, 0), W, H, 60.0)
    colour = (0.7, -0.35, 0.2)
    sc = _one_gaussian_scene((0, 0, 0), sig3, (1, 0, 0, 0), logit, colour)
    prep = oracle.preprocess(sc, cam)
    s_true = math.exp(float(np.float32(math.log(sig3))))
    var = (cam.fx * s_true / d) ** 2 + DIL
    o = 1 / (1 + math.exp(-float(np.float32(logit))))
    ys, xs = np.mgrid[0:H, 0:W]
    rho2 = (xs + 0.5 - W / 2) ** 2 + (ys + 0.5 - H / 2) ** 2
    a = np.minimum(float(np.float32(0.99)), o * np.exp(-rho2 / (2 * var)))
    a = np.where((rho2 / var <= 9.0) & (a >= np.float32(1 / 255)), a, 0.0)
    c = np.maximum(_dc_colour(sc, 0), 0.0)
    assert c[1] == 0.0 and c[0] > 0 and c[2] > 0
    bg = np.array([0.3, 0.6, 0.9])
    expect = c[:, None, None] * a + bg[:, None, None] * (1 - a)
    np.testing.assert_allclose(prep["rgb"][0], c, atol=1e-15)
    for img in (oracle.render_bruteforce(prep, W, H, bg), oracle.render_tiled(prep, W, H, bg)):
        np.testing.assert_allclose(img["rgb"], expect, atol=1e-12)
        np.testing.assert_allclose(img["rgb"][1], bg[1] * (1 - a), atol=1e-12)
    # L = sum over the image of channel ch: dL/dsh_ch = Y00 * sum alpha, or 0 where clamped
    for ch in range(3):
        gC = np.zeros((3, H, W))
        gC[ch] = 1.0
        g = oracle.adjoint(sc, cam, gC, np.zeros((H, W)), bg)
        want = 0.0 if ch == 1 else Y00 * a.sum()
        assert abs(g["sh"][0, 0, ch] - want) <= 1e-12 * max(1.0, abs(want)), (ch, g["sh"][0, 0, ch], want)
