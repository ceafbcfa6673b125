"""Pins of the oracle's compositing, depth output and conic against values computed here by hand.

The expected values below come from the paper's definitions written out in this file for
special cases with a closed form, never from the oracle:
  * the front-to-back composite of Eq. "volume_desc" (Sec. 2.1): C = sum_i c_i alpha_i T_i with
    T_1 = 1, T_{i+1} = T_i (1 - alpha_i), alpha_i = min(0.99, opacity_i G2_i(x)), and the image
    value C + T_N * bg;
  * the 3DGS early-out the paper keeps: the Gaussian that would take T below 1e-4 is not
    blended and the ray stops;
  * the volumetric depth of Sec. 4.1 "Depth Evaluation" with phi = t_opt, unnormalised:
    zeta = sum_i t_opt,i alpha_i T_i;
  * t_opt for an isotropic Gaussian (Sec. 3.2, Eq. "dopt"): the distance along the unit ray to
    the foot of the perpendicular from the mean, d . (mu - o);
  * the EWA splat of an isotropic Gaussian on the optical axis: Sigma2 = (s f / z)^2 I + 0.3 I.
The conic (Sigma2^-1) is pinned against numpy.linalg.inv of the projected covariance, which the
projection pin (finite-difference Jacobian) fixes independently.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2402_00525_gb300 import inputs as I

Y00 = 0.5 / math.sqrt(math.pi)           # real SH basis, l = 0
F = 64.0                                 # focal length in pixels (exact in float32)
W = H = 16


def _f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def _camera():
    return I.Camera(R=np.eye(3), t=np.zeros(3), fx=F, fy=F, cx=W / 2, cy=H / 2, width=W, height=H)


def _scene(means, scales, opac, colours, quats=None):
    n = len(means)
    q = np.tile([1.0, 0.0, 0.0, 0.0], (n, 1)) if quats is None else np.asarray(quats)
    sh = np.zeros((n, 1, 3))
    sh[:, 0, :] = (np.asarray(colours, np.float64) - 0.5) / Y00
    logit = np.log(np.asarray(opac)) - np.log1p(-np.asarray(opac))
    ls = np.log(np.asarray(scales, np.float64))
    if ls.ndim == 1:
        ls = np.repeat(ls[:, None], 3, 1)
    return I.Scene(np.asarray(means, np.float32), ls.astype(np.float32), q.astype(np.float32),
                   logit.astype(np.float32), sh.astype(np.float32), 0)


def _decoded(sc):
    """Opacity and colour as the renderer sees them: from the float32 inputs, in float64."""
    op = 1.0 / (1.0 + np.exp(-_f32(sc.opacity_logits)))
    col = np.maximum(0.0, _f32(sc.sh[:, 0, :]) * Y00 + 0.5)
    return op, col


def _composite(alphas, ts, cols, bg, t_min=1e-4):
    """Eq. "volume_desc" front to back with the early-out, and Sec. 4.1's zeta."""
    T, C, Z, nb = 1.0, np.zeros(3), 0.0, 0
    for a, t, c in zip(alphas, ts, cols):
        if T * (1.0 - a) < t_min:
            break
        C = C + c * a * T
        Z += t * a * T
        T *= 1.0 - a
        nb += 1
    return C + T * np.asarray(bg), Z, T, nb


MODES = [dict(), dict(head=16), dict(mode=I.MODE_FULL), dict(mode=I.MODE_GLOBAL),
         dict(mode=I.MODE_WINDOW, window_k=4), dict(flags=I.FLAG_HEAD_EVICT_FIRST)]


@pytest.mark.parametrize("kw", MODES, ids=["hier", "hier16", "full", "global", "window4", "evict"])
def test_single_isotropic_gaussian_every_pixel(oracle, kw):
    """One isotropic Gaussian on the optical axis: at every pixel rgb = c alpha + (1 - alpha) bg,
    zeta = t_opt alpha and T = 1 - alpha, with alpha from the closed-form EWA splat."""
    z, s = 3.0, 0.05
    sc = _scene([[0.0, 0.0, z]], [s], [0.8], [[0.9, 0.3, 0.6]])
    prm = dataclasses.replace(I.RenderParams(bg=(0.2, 0.4, 0.6)), **kw)
    out = oracle.render(sc, _camera(), prm)
    op, col = _decoded(sc)
    sz = math.exp(_f32(sc.log_scales)[0, 0]) * F / z
    var2 = sz * sz + prm.dilation
    xs = np.arange(W) + 0.5 - W / 2
    dx, dy = np.meshgrid(xs, xs)              # [y, x]
    a = np.minimum(0.99, op[0] * np.exp(-0.5 * (dx * dx + dy * dy) / var2))
    # unit ray through the pixel centre; the mean is on the axis at depth z, camera at 0
    t = z / np.sqrt(1.0 + (dx / F) ** 2 + (dy / F) ** 2)
    keep = a >= prm.eps_o
    away = np.abs(a / prm.eps_o - 1.0) > 1e-6
    assert keep.sum() > 30 and (~keep).sum() > 30
    bg = np.array(prm.bg)
    exp_rgb = np.where(keep[..., None], col[0] * a[..., None] + (1 - a[..., None]) * bg, bg)
    np.testing.assert_allclose(out["rgb"][away], exp_rgb[away], rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["depth"][away], np.where(keep, t * a, 0.0)[away], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(out["tfinal"][away], np.where(keep, 1 - a, 1.0)[away], rtol=0, atol=1e-12)
    assert np.array_equal(out["nblend"][away], keep[away].astype(np.int32))


def _stack(zs, opac, colours):
    """Isotropic Gaussians whose means lie on the ray through the centre of pixel (8, 8)."""
    u = 0.5 / F                               # (8.5 - cx) / fx
    means = [[z * u, z * u, z] for z in zs]   # exact in float32 for z in halves
    return _scene(means, [0.02] * len(zs), opac, colours)


@pytest.mark.parametrize("kw", MODES, ids=["hier", "hier16", "full", "global", "window4", "evict"])
@pytest.mark.parametrize("shuffle", [False, True])
def test_stack_on_one_ray_composites_front_to_back(oracle, kw, shuffle):
    """Five Gaussians on one pixel's ray at different depths and in any input order: the pixel
    composites them by depth with Eq. "volume_desc", alpha = min(0.99, opacity) since G2 = 1 at
    the projected mean, t_opt = |mu| (the camera is at the origin), and bg weighted by T_N."""
    zs = [2.0, 2.5, 3.0, 4.0, 5.5]
    op = [0.5, 0.3, 0.995, 0.6, 0.4]
    cols = [[0.9, 0.1, 0.2], [0.2, 0.8, 0.3], [0.3, 0.3, 0.9], [0.7, 0.7, 0.1], [0.5, 0.2, 0.6]]
    order = [3, 0, 4, 2, 1] if shuffle else list(range(5))
    sc = _stack([zs[i] for i in order], [op[i] for i in order], [cols[i] for i in order])
    prm = dataclasses.replace(I.RenderParams(bg=(0.25, 0.5, 0.75)), **kw)
    out = oracle.render(sc, _camera(), prm)
    o, c = _decoded(sc)
    m = _f32(sc.means)
    depth_order = np.argsort(m[:, 2])
    alphas = np.minimum(0.99, o[depth_order])
    ts = np.linalg.norm(m[depth_order], axis=1)
    rgb, Z, T, nb = _composite(alphas, ts, c[depth_order], prm.bg)
    assert nb == 5                             # the 0.995 Gaussian is clamped to 0.99
    assert out["decided"][8, 8]
    np.testing.assert_allclose(out["rgb"][8, 8], rgb, rtol=0, atol=1e-12)
    assert out["depth"][8, 8] == pytest.approx(Z, rel=1e-12)
    assert out["tfinal"][8, 8] == pytest.approx(T, rel=1e-12)
    assert out["nblend"][8, 8] == nb


@pytest.mark.parametrize("kw", MODES, ids=["hier", "hier16", "full", "global", "window4", "evict"])
def test_termination_gaussian_is_not_blended(oracle, kw):
    """A stack of opacity-0.95 Gaussians: T runs 1, 0.05, 0.0025, 1.25e-4, and the fourth would
    take it to 6.25e-6 < 1e-4, so exactly three are blended, T_final = 0.05^3 and the image
    is their composite plus 0.05^3 * bg."""
    zs = [2.0, 2.5, 3.0, 3.5, 4.0]
    cols = [[0.9, 0.1, 0.2], [0.2, 0.8, 0.3], [0.3, 0.3, 0.9], [1.0, 1.0, 1.0], [1.0, 1.0, 1.0]]
    sc = _stack(zs, [0.95] * 5, cols)
    prm = dataclasses.replace(I.RenderParams(bg=(0.3, 0.6, 0.9)), **kw)
    out = oracle.render(sc, _camera(), prm)
    o, c = _decoded(sc)
    ts = np.linalg.norm(_f32(sc.means), axis=1)
    rgb, Z, T, nb = _composite(np.minimum(0.99, o), ts, c, prm.bg)
    assert nb == 3 and 1e-4 < T < 2e-4
    assert out["nblend"][8, 8] == 3
    np.testing.assert_allclose(out["rgb"][8, 8], rgb, rtol=0, atol=1e-12)
    assert out["depth"][8, 8] == pytest.approx(Z, rel=1e-12)
    assert out["tfinal"][8, 8] == pytest.approx(T, rel=1e-12)


def _rot_wxyz(q):
    q = np.asarray(q, np.float64)
    return Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy: scalar last


def test_single_anisotropic_gaussian_every_pixel(oracle):
    """One rotated anisotropic Gaussian near the axis: alpha at every pixel centre from
    numpy.linalg.inv of J Sigma J^T + 0.3 I (J the pinhole Jacobian at the mean, Sigma from
    scipy's rotation of the quaternion), t_opt from Eq. "dopt" with numpy's Sigma^-1."""
    mu = np.array([0.05, -0.03, 3.0])
    q = np.array([0.8, 0.3, -0.4, 0.33])
    s = np.array([0.09, 0.03, 0.05])
    sc = _scene([mu], [s], [0.9], [[0.4, 0.7, 0.2]], quats=[q])
    prm = I.RenderParams(bg=(0.1, 0.2, 0.3))
    out = oracle.render(sc, _camera(), prm)
    m = _f32(sc.means)[0]
    Rq = _rot_wxyz(_f32(sc.quats)[0])
    sig = Rq @ np.diag(np.exp(2 * _f32(sc.log_scales)[0])) @ Rq.T
    x, y, z = m
    J = np.array([[F / z, 0, -F * x / z ** 2], [0, F / z, -F * y / z ** 2]])
    cov2 = J @ sig @ J.T + prm.dilation * np.eye(2)
    A = np.linalg.inv(cov2)
    mean2 = np.array([F * x / z + W / 2, F * y / z + H / 2])
    op, col = _decoded(sc)
    sinv = np.linalg.inv(sig)
    xs = np.arange(W) + 0.5
    exp_rgb = np.zeros((H, W, 3))
    exp_z = np.zeros((H, W))
    nblend = np.zeros((H, W), np.int32)
    away = np.ones((H, W), bool)
    for py in range(H):
        for px in range(W):
            d2 = np.array([xs[px], xs[py]]) - mean2
            a = min(0.99, op[0] * math.exp(-0.5 * d2 @ A @ d2))
            away[py, px] = abs(a / prm.eps_o - 1) > 1e-6
            ray = np.array([(xs[px] - W / 2) / F, (xs[py] - H / 2) / F, 1.0])
            ray /= np.linalg.norm(ray)
            t = (ray @ sinv @ m) / (ray @ sinv @ ray)
            if a >= prm.eps_o:
                exp_rgb[py, px] = col[0] * a + (1 - a) * np.array(prm.bg)
                exp_z[py, px] = t * a
                nblend[py, px] = 1
            else:
                exp_rgb[py, px] = prm.bg
    assert nblend.sum() > 20 and (nblend == 0).sum() > 20
    np.testing.assert_allclose(out["rgb"][away], exp_rgb[away], rtol=0, atol=1e-11)
    np.testing.assert_allclose(out["depth"][away], exp_z[away], rtol=1e-10, atol=1e-12)
    assert np.array_equal(out["nblend"][away], nblend[away])


def test_conic_is_the_inverse_of_the_projected_covariance(oracle):
    """Preprocess's conic A = Sigma2^-1 (Sec. 2.1) against numpy.linalg.inv of the projected
    covariance, on random anisotropic Gaussians in front of the camera."""
    sc = I.uniform_scene(300, 91, scale_range=(0.005, 0.2), extent=0.8)
    cam = I.look_at((0.2, -0.1, -3), (0, 0, 0), (0, 1, 0), 128, 96, 60.0)
    prm = I.RenderParams()
    with oracle.OracleRun(sc, cam, prm) as r:
        pp = r.preprocess()
    vis = np.flatnonzero(pp["visible"])
    assert len(vis) > 200
    camf = oracle.cam_struct(cam)
    Rc = np.array(camf.R[:]).reshape(3, 3)
    for i in vis[:120]:
        sig = oracle.sigma(_f32(sc.quats[i]), _f32(sc.log_scales[i]))
        _, cov, _ = oracle.project(cam, prm, _f32(sc.means[i]), sig)
        C2 = np.array([[cov[0], cov[1]], [cov[1], cov[2]]])
        a, b, c = pp["conic"][i]
        A = np.array([[a, b], [b, c]])
        np.testing.assert_allclose(A @ C2, np.eye(2), atol=1e-9)
        np.testing.assert_allclose(A, np.linalg.inv(C2), rtol=1e-9, atol=1e-12)
        # the projected mean of the same Gaussian from the camera model alone
        p = Rc @ _f32(sc.means[i]) + np.array(camf.t[:])
        mean2 = np.array([camf.fx * p[0] / p[2] + camf.cx, camf.fy * p[1] / p[2] + camf.cy])
        np.testing.assert_allclose(pp["mean2"][i], mean2, rtol=1e-12, atol=1e-9)


# ------------------------------------------------------------ inputs outside the domain
def invalid_variant(sc):
    """Copy of `sc` with twelve Gaussians made invalid in different ways, the indices, and a
    reference copy where the same Gaussians are merely invisible (opacity logit -30, so
    opacity < eps_O)."""
    bad = np.array([3, 17, 29, 41, 55, 68, 80, 97, 110, 123, 140, 151])
    s1 = I.Scene(sc.means.copy(), sc.log_scales.copy(), sc.quats.copy(), sc.opacity_logits.copy(),
                 sc.sh.copy(), sc.sh_degree)
    s1.means[bad[0], 0] = np.nan
    s1.means[bad[1], 2] = np.inf
    s1.log_scales[bad[2], 1] = -np.inf          # zero scale
    s1.log_scales[bad[3], 0] = np.inf
    s1.quats[bad[4]] = 0.0                       # no rotation defined
    s1.quats[bad[5], 3] = np.nan
    s1.opacity_logits[bad[6]] = np.nan
    s1.opacity_logits[bad[7]] = np.inf
    s1.sh[bad[8], 0, 1] = np.nan
    s1.sh[bad[9], -1, 2] = np.inf               # highest band: its basis value may be 0
    s1.sh[bad[10], 1, 0] = -np.inf
    s1.means[bad[11], 1] = -np.inf
    s2 = I.Scene(sc.means.copy(), sc.log_scales.copy(), sc.quats.copy(), sc.opacity_logits.copy(),
                 sc.sh.copy(), sc.sh_degree)
    s2.opacity_logits[bad] = -30.0
    return s1, s2, bad


def test_invalid_gaussians_are_dropped_and_counted(oracle):
    """A Gaussian with a non-finite parameter or a zero-length quaternion covers no pixel: the
    image equals that of the same scene with those Gaussians made invisible, bit for bit, the
    oracle counts them, and their adjoint is zero while every other gradient is unchanged."""
    sc = I.uniform_scene(160, 93, scale_range=(0.02, 0.12), sh_degree=2)
    cam = I.look_at((0.2, 0.1, -3), (0, 0, 0), (0, 1, 0), 64, 48, 60.0)
    prm = I.RenderParams()
    s1, s2, bad = invalid_variant(sc)
    rng = np.random.default_rng(5)
    w = rng.normal(size=(cam.height, cam.width, 3))
    with oracle.OracleRun(s1, cam, prm, record=True) as r1, oracle.OracleRun(s2, cam, prm, record=True) as r2:
        assert r1.num_invalid == len(bad) and r2.num_invalid == 0
        a, b = r1.render(), r2.render()
        for k in ("rgb", "depth", "tfinal", "nblend", "hash"):
            assert np.array_equal(a[k], b[k]), k
        assert a["nblend"].sum() > 0
        g1, g2 = r1.backward(w), r2.backward(w)
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        assert np.all(g1[k][bad] == 0) and np.all(np.isfinite(g1[k])), k
        keep = np.setdiff1d(np.arange(sc.n), bad)
        assert np.array_equal(g1[k][keep], g2[k][keep]), k


def test_quaternion_length_threshold(oracle):
    """Reading for invalid inputs: a quaternion whose squared length is below 1e-20 defines no
    rotation, so the Gaussian is dropped and counted; just above it the quaternion is
    normalised and the Gaussian renders like its unit-length twin."""
    sc = I.uniform_scene(40, 94, scale_range=(0.05, 0.2))
    cam = I.look_at((0.2, 0.1, -3), (0, 0, 0), (0, 1, 0), 48, 48, 60.0)
    prm = I.RenderParams()
    q = sc.quats.astype(np.float64)
    tiny = I.Scene(sc.means, sc.log_scales, (q * 1e-11).astype(np.float32), sc.opacity_logits, sc.sh, 0)
    small = I.Scene(sc.means, sc.log_scales, (q * 1e-9).astype(np.float32), sc.opacity_logits, sc.sh, 0)
    with oracle.OracleRun(tiny, cam, prm) as r:
        assert r.num_invalid == sc.n
        assert r.render()["nblend"].sum() == 0
    with oracle.OracleRun(small, cam, prm) as r1, oracle.OracleRun(sc, cam, prm) as r2:
        assert r1.num_invalid == 0
        a, b = r1.render(), r2.render()
        assert a["nblend"].sum() > 0
        assert np.array_equal(a["nblend"], b["nblend"]) and np.array_equal(a["hash"], b["hash"])
        # the scaled quaternion rounds to float32 on its own, so its direction differs from the
        # unit one by a few 1e-8; the colours by as much
        assert np.allclose(a["rgb"], b["rgb"], rtol=0, atol=1e-6)
