"""Pins of the FP64 CPU oracle against things other than itself: values the paper prints,
closed forms, brute force on small inputs, textbook routines and invariants of the method.

Each test names the passage of StopThePop (arXiv 2402.00525) it pins.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

from paper_2402_00525_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _paper_values():
    vals = {}
    for line in open(os.path.join(GOLD, "paper_values.txt")):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()
            vals[k] = float(v)
    return vals


def _rand_rot(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    # independent of the oracle's formula: build from an axis-angle with Rodrigues' formula
    ang = 2 * math.acos(min(1.0, abs(w)))
    ax = np.array([x, y, z])
    ax = ax / (np.linalg.norm(ax) + 1e-300)
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


# --------------------------------------------------------------------- Appendix B.2: t_O
def test_t_o_bound_printed_value(oracle):
    pv = _paper_values()
    assert oracle.t_o(1.0, pv["eps_o"]) == pytest.approx(pv["t_o_max"], abs=5e-5)
    assert oracle.t_o(pv["eps_o"], pv["eps_o"]) == 0.0
    # the bound is monotone in alpha and never above t_O(1)
    a = np.linspace(pv["eps_o"], 1.0, 200)
    t = np.array([oracle.t_o(x, pv["eps_o"]) for x in a])
    assert np.all(np.diff(t) > 0) and t.max() <= pv["t_o_max"] + 5e-5
    # the paper's conclusion: 3DGS's t_O = 3 is too small for eps_O = 1/255 (opacity 1)
    assert math.exp(-0.5 * 3.0 ** 2) > pv["eps_o"]


def test_paper_defaults_match_render_params():
    pv = _paper_values()
    p = I.RenderParams()
    assert (p.tail, p.mid, p.head, p.lb_threshold) == (pv["tail_queue"], pv["mid_queue"],
                                                       pv["head_queue"], pv["lb_threshold"])
    assert p.eps_o == pytest.approx(pv["eps_o"], rel=1e-15)
    assert p.inv_scale_max == pv["inv_scale_max"]
    # window bounds implied by the queue sizes (Sec. 3.4): 17 + 4 + 4 and 64 + 4 + 4
    assert pv["tail_drain_min"] + (p.mid - 4) + p.head == pv["window_min"]
    assert p.tail + (p.mid - 4) + p.head == pv["window_max"]


# --------------------------------------------------------------------- Eq. dopt, Sec. 3.2
def test_isotropic_worked_example(oracle):
    rows = np.loadtxt(os.path.join(GOLD, "isotropic_depth.txt"))
    for th, muy, t in rows:
        d = np.array([math.sin(math.radians(th)), math.cos(math.radians(th)), 0.0])
        got = oracle.t_opt(d, np.zeros(3), np.array([0.0, muy, 0.0]), np.eye(3))
        assert got == pytest.approx(t, rel=1e-12, abs=1e-12)


def _golden_min(f, a, b, it=200):
    g = (math.sqrt(5) - 1) / 2
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(it):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
    return 0.5 * (a + b)


def test_t_opt_maximises_gaussian_along_ray(oracle):
    """t_opt is the argmax of G(o + t d): dense sampling then golden-section search."""
    rng = np.random.default_rng(11)
    for _ in range(150):
        R = _rand_rot(rng)
        s = np.exp(rng.uniform(math.log(0.01), math.log(1.0), 3))
        sinv = R @ np.diag(1 / s ** 2) @ R.T
        mu = rng.uniform(-3, 3, 3) + np.array([0, 0, 8.0])
        o = rng.uniform(-1, 1, 3)
        d = mu - o + rng.normal(0, 0.3, 3)
        d /= np.linalg.norm(d)
        f = lambda t: float((o + t * d - mu) @ sinv @ (o + t * d - mu))
        ts = np.linspace(-40, 60, 20001)
        vals = np.array([f(t) for t in ts])
        k = int(np.argmin(vals))
        tb = _golden_min(f, ts[max(k - 1, 0)], ts[min(k + 1, len(ts) - 1)])
        got = oracle.t_opt(d, o, mu, sinv)
        assert got == pytest.approx(tb, rel=2e-7, abs=2e-7)


# --------------------------------------------------------------------- Appendix A, Sec. 3.2
def test_sigma_inverse_and_clamp(oracle):
    rng = np.random.default_rng(12)
    for _ in range(100):
        q = rng.normal(size=4)
        ls = rng.uniform(math.log(2e-3), 0.0, 3)
        S = oracle.sigma(q, ls)
        Si = oracle.sigma_inv(q, ls, 1e3)
        assert np.allclose(Si @ S, np.eye(3), atol=1e-9)
        # eigen-decomposition check against the textbook routine
        ev = np.sort(np.linalg.eigvalsh(S))
        assert np.allclose(ev, np.sort(np.exp(2 * ls)), rtol=1e-9)
    # clamp: S^-1 entries bounded by 1e3, so the thin axis of s = 1e-4 has Sigma^-1 eigenvalue
    # 1e6 while the other axes are untouched
    q = rng.normal(size=4)
    ls = np.log([1e-4, 0.05, 0.2])
    ev = np.sort(np.linalg.eigvalsh(oracle.sigma_inv(q, ls, 1e3)))
    assert np.allclose(ev, np.sort([1e6, 1 / 0.05 ** 2, 1 / 0.2 ** 2]), rtol=1e-9)


# --------------------------------------------------------------------- Algorithm 1
def test_alg1_matches_grid_search(oracle):
    rng = np.random.default_rng(13)
    boxes = [(0.5, 15.5, 0.5, 15.5), (16.5, 19.5, 32.5, 35.5), (0.5, 1.5, 0.5, 1.5),
             (4.5, 4.5, 0.5, 15.5), (0.5, 15.5, 7.5, 7.5)]
    for trial in range(250):
        box = boxes[trial % len(boxes)]
        th = rng.uniform(0, math.pi)
        c, s = math.cos(th), math.sin(th)
        Rr = np.array([[c, -s], [s, c]])
        lam = np.exp(rng.uniform(math.log(0.3), math.log(400.0), 2))
        cov = Rr @ np.diag(lam) @ Rr.T
        A = np.linalg.inv(cov)
        conic = np.array([A[0, 0], A[0, 1], A[1, 1]])
        ctr = np.array([(box[0] + box[1]) / 2, (box[2] + box[3]) / 2])
        mu = ctr + rng.uniform(-30, 30, 2)
        if trial % 7 == 0:
            mu = ctr + rng.uniform(-1, 1, 2)
        xh = oracle.alg1(mu, conic, np.array(box))
        assert box[0] - 1e-12 <= xh[0] <= box[1] + 1e-12 and box[2] - 1e-12 <= xh[1] <= box[3] + 1e-12
        gx = np.linspace(box[0], box[1], 601)
        gy = np.linspace(box[2], box[3], 601)
        X, Y = np.meshgrid(gx, gy, indexing="ij")
        dx, dy = X - mu[0], Y - mu[1]
        Q = A[0, 0] * dx * dx + 2 * A[0, 1] * dx * dy + A[1, 1] * dy * dy
        dxh = xh - mu
        qh = dxh @ A @ dxh
        assert qh <= Q.min() + 1e-9 * (1 + abs(Q.min()))
        inside = box[0] <= mu[0] <= box[1] and box[2] <= mu[1] <= box[3]
        if not inside:   # then x_hat lies on the boundary (Sec. 3.4: on an edge nearest mu2)
            on_edge = (min(abs(xh[0] - box[0]), abs(xh[0] - box[1])) < 1e-9 or
                       min(abs(xh[1] - box[2]), abs(xh[1] - box[3])) < 1e-9)
            assert on_edge


# --------------------------------------------------------------------- SH colour
def test_sh_basis_orthonormal_and_matches_textbook(oracle):
    sp = pytest.importorskip("scipy.special")
    # Gauss-Legendre in cos(theta) x uniform phi: exact for these polynomial degrees
    xs, ws = np.polynomial.legendre.leggauss(24)
    phis = np.arange(48) * 2 * math.pi / 48
    Gm = np.zeros((16, 16))
    for ct, w in zip(xs, ws):
        st = math.sqrt(1 - ct * ct)
        for ph in phis:
            d = np.array([st * math.cos(ph), st * math.sin(ph), ct])
            y = oracle.sh_basis(d)
            Gm += np.outer(y, y) * w * (2 * math.pi / 48)
    assert np.allclose(Gm, np.eye(16), atol=1e-12)
    # against scipy's complex harmonics, which carry the Condon-Shortley phase: the real basis
    # is sqrt(2) Re Y_l^m for m > 0, Y_l^0, and sqrt(2) Im Y_l^|m| for m < 0, signs included;
    # index (l, m)
    rng = np.random.default_rng(14)
    lm = [(l, m) for l in range(4) for m in range(-l, l + 1)]
    for _ in range(20):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        y = oracle.sh_basis(d)
        for k, (l, m) in enumerate(lm):
            Yc = sp.sph_harm_y(l, abs(m), theta, phi)
            ref = Yc.real if m == 0 else math.sqrt(2) * (Yc.real if m > 0 else Yc.imag)
            assert abs(y[k] - ref) < 1e-12, (l, m)


def test_sh_degree0_colour_is_view_independent(oracle):
    sc = I.uniform_scene(64, 5, sh_degree=0)
    cams = I.orbit_cameras(3, 4.0, 0.5, [(64, 64)], 60.0)
    cols = []
    for cam in cams:
        with oracle.OracleRun(sc, cam, I.RenderParams()) as r:
            pp = r.preprocess()
        cols.append(pp["color"])
    y00 = 1.0 / math.sqrt(4 * math.pi)   # textbook constant
    expect = np.maximum(0.0, 0.5 + y00 * sc.sh[:, 0, :].astype(np.float64))
    for c in cols:
        assert np.allclose(c, expect, atol=1e-12)


# --------------------------------------------------------------------- EWA splat (Sec. 2.1)
def test_projection_jacobian_is_finite_difference(oracle):
    rng = np.random.default_rng(15)
    cam = I.look_at((0.3, -0.2, -4), (0, 0, 0), (0, 1, 0), 320, 240, 55.0)
    # the oracle receives the camera as the renderer does, rounded to float32
    cam = I.Camera(cam.R.astype(np.float32).astype(np.float64), cam.t.astype(np.float32).astype(np.float64),
                   float(np.float32(cam.fx)), float(np.float32(cam.fy)), float(np.float32(cam.cx)),
                   float(np.float32(cam.cy)), cam.width, cam.height)
    prm = I.RenderParams()

    def proj(mu):
        p = cam.R @ mu + cam.t
        return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])

    for _ in range(50):
        mu = rng.uniform(-1, 1, 3)
        q = rng.normal(size=4)
        ls = rng.uniform(-4, -1, 3)
        S = oracle.sigma(q, ls)
        m2, cov, J = oracle.project(cam, prm, mu, S)
        assert np.allclose(m2, proj(mu), rtol=1e-13)
        h = 1e-6
        Jfd = np.stack([(proj(mu + h * e) - proj(mu - h * e)) / (2 * h) for e in np.eye(3)], 1)
        assert np.allclose(J @ cam.R, Jfd, rtol=1e-7, atol=1e-6)
        C2 = Jfd @ S @ Jfd.T
        assert np.allclose([cov[0] - 0.3, cov[1], cov[2] - 0.3], [C2[0, 0], C2[0, 1], C2[1, 1]],
                           rtol=1e-6, atol=1e-8)


def test_splat_shape_stops_changing_beyond_the_jacobian_clamp(oracle):
    """The EWA Jacobian of the preprocess kept from 3DGS takes the view-space x/z and y/z
    clamped to 1.3 times the half field of view (reading: kept). So beyond that limit the 2D
    covariance no longer changes as the mean moves outward at a fixed depth; inside it does."""
    cam = I.Camera(R=np.eye(3), t=np.zeros(3), fx=64.0, fy=64.0, cx=32.0, cy=24.0, width=64, height=48)
    prm = I.RenderParams()
    lim = (1.3 * 0.5 * 64 / 64, 1.3 * 0.5 * 48 / 64)
    S = oracle.sigma(np.array([0.9, 0.2, -0.3, 0.25]), np.log([0.05, 0.2, 0.1]))
    z = 2.0
    for axis in (0, 1):
        def cov(u):
            mu = np.zeros(3)
            mu[axis], mu[2] = u * z, z
            return oracle.project(cam, prm, mu, S)[1]
        outside = [cov(f * lim[axis]) for f in (1.2, 2.0, 5.0)]
        for c in outside[1:]:
            assert np.allclose(c, outside[0], rtol=1e-12, atol=0)
        assert not np.allclose(cov(0.2 * lim[axis]), cov(0.8 * lim[axis]), rtol=1e-6, atol=0)
        assert not np.allclose(cov(0.8 * lim[axis]), outside[0], rtol=1e-6, atol=0)


def test_near_plane_culls_gaussians_in_front_of_znear(oracle):
    """The preprocess kept from 3DGS culls Gaussians whose view-space depth is not above
    znear = 0.2 (reading: kept as a parameter)."""
    zs = [0.04, 0.1, 0.15, 0.199, 0.201, 0.3, 1.0, 5.0]
    n = len(zs)
    sh = np.zeros((n, 1, 3), np.float32)
    sc = I.Scene(np.array([[0.0, 0.0, z] for z in zs], np.float32), np.full((n, 3), math.log(0.01), np.float32),
                 np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)), np.full(n, 2.0, np.float32), sh, 0)
    cam = I.Camera(R=np.eye(3), t=np.zeros(3), fx=16.0, fy=16.0, cx=8.0, cy=8.0, width=16, height=16)
    with oracle.OracleRun(sc, cam, I.RenderParams()) as r:
        vis = r.preprocess()["visible"]
    assert list(vis) == [int(z > 0.2) for z in zs]


def test_sh_colour_uses_the_direction_from_the_camera_to_the_mean(oracle):
    """App. B.4: each Gaussian's colour is 0.5 + sum_lm Y_lm(d) c_lm, clamped at 0, with d the
    unit vector from the camera centre to the mean. Y here from scipy's complex harmonics
    (Condon-Shortley phase, real combinations), d from the float32 camera the renderer gets."""
    sp = pytest.importorskip("scipy.special")
    sc = I.uniform_scene(60, 41, extent=0.8, sh_degree=3)
    sc.sh[:, 1:, :] *= 5.0                        # strong view dependence; some colours clamp
    cam = I.look_at((1.0, -0.5, -3.0), (0, 0, 0), (0, 1, 0), 64, 64, 60.0)
    with oracle.OracleRun(sc, cam, I.RenderParams()) as r:
        pp = r.preprocess()
    R = cam.R.astype(np.float32).astype(np.float64)
    o = -R.T @ cam.t.astype(np.float32).astype(np.float64)
    lm = [(l, m) for l in range(4) for m in range(-l, l + 1)]
    checked = clamped = 0
    for i in np.nonzero(pp["visible"])[0]:
        d = sc.means[i].astype(np.float64) - o
        d /= np.linalg.norm(d)
        theta, phi = math.acos(d[2]), math.atan2(d[1], d[0])
        Y = np.empty(16)
        for k, (l, m) in enumerate(lm):
            Yc = sp.sph_harm_y(l, abs(m), theta, phi)
            Y[k] = Yc.real if m == 0 else math.sqrt(2) * (Yc.real if m > 0 else Yc.imag)
        col = 0.5 + Y @ sc.sh[i].astype(np.float64)
        assert np.allclose(pp["color"][i], np.maximum(col, 0.0), rtol=0, atol=1e-12), i
        checked += 1
        clamped += int((col < 0).any())
    assert checked >= 40 and clamped >= 1


# --------------------------------------------------------------------- culling exactness
def _alpha_all_pixels(pp, cam):
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    px, py = xs.ravel() + 0.5, ys.ravel() + 0.5
    vis = np.nonzero(pp["visible"])[0]
    out = {}
    for i in vis:
        dx, dy = px - pp["mean2"][i, 0], py - pp["mean2"][i, 1]
        a, b, c = pp["conic"][i]
        al = np.minimum(0.99, pp["opacity"][i] * np.exp(-0.5 * (a * dx * dx + 2 * b * dx * dy + c * dy * dy)))
        out[i] = al.reshape(cam.height, cam.width)
    return out


@pytest.mark.parametrize("which", ["fd", "plain"])
def test_tile_culling_never_drops_a_contributor(oracle, which):
    """Sec. 3.4: culling is exact; brute force over every pixel finds no pixel with
    alpha >= eps_O whose tile list lacks the Gaussian (rectangle bound of App. B.2 included)."""
    if which == "fd":
        sc, _, cam, prm = I.fd_subcase()
    else:
        sc = I.uniform_scene(600, 21, scale_range=(0.01, 0.2))
        cam = I.look_at((0, 0, -3), (0, 0, 0), (0, 1, 0), 96, 80, 60.0)
        prm = I.RenderParams()
    with oracle.OracleRun(sc, cam, prm) as r:
        pp = r.preprocess()
        start, ids, _ = r.tile_lists()
    alphas = _alpha_all_pixels(pp, cam)
    lists = [set(ids[start[t]:start[t + 1]].tolist()) for t in range(cam.num_tiles)]
    kept_somewhere = 0
    for i, al in alphas.items():
        ys, xs = np.nonzero(al >= prm.eps_o)
        for t in set((ys // 16 * cam.tiles_x + xs // 16).tolist()):
            assert i in lists[t]
            kept_somewhere += 1
    assert kept_somewhere > 100
    # entries counted by the preprocess equal the entries written (one key per kept tile)
    assert int(pp["ntiles"].sum()) == len(ids)


def test_hier_blends_the_same_set_as_full_sort(oracle):
    """Culling at the 4x4, 2x2 and pixel levels (Sec. 3.4) drops no contributor: without early
    termination every pixel blends exactly the Gaussians a full per-ray sort blends."""
    sc, cams, prm = I.plain_forward_workload()
    prm = dataclasses.replace(prm, t_min=1e-30)
    h = oracle.render(sc, cams[0], prm, max_seq=96)
    f = oracle.render(sc, cams[0], dataclasses.replace(prm, mode=I.MODE_FULL), max_seq=96)
    assert h["nblend"].max() < 96
    assert np.array_equal(h["nblend"], f["nblend"])
    hs = np.sort(np.where(h["seq"] < 0, 1 << 30, h["seq"]), axis=2)
    fs = np.sort(np.where(f["seq"] < 0, 1 << 30, f["seq"]), axis=2)
    assert np.array_equal(hs, fs)


@pytest.mark.parametrize("flags", [0, I.FLAG_HEAD_EVICT_FIRST, I.FLAG_LEVEL_CENTRE_RAYS],
                         ids=["default", "evict_first", "level_centre_rays"])
def test_readings_change_the_order_never_the_set(oracle, flags):
    """The two alternative readings (evict before insert in the per-pixel queue; 4x4 / 2x2 keys
    from the level-centre ray) change only the order in which a pixel blends: culling does not
    depend on keys, so without early termination every pixel still blends exactly the set the
    full per-ray sort blends. On a clustered scene each reading reorders some pixels."""
    sc = I.cluster_scene(3000, 33, nclusters=4, centre_range=0.5, scale_range=(0.01, 0.15))
    cam = I.look_at((0, 0.5, -5), (0, 0, 0), (0, 1, 0), 64, 64, 50.0)
    prm = I.RenderParams(t_min=1e-30)
    f = oracle.render(sc, cam, dataclasses.replace(prm, mode=I.MODE_FULL), max_seq=600)
    h = oracle.render(sc, cam, dataclasses.replace(prm, flags=flags), max_seq=600)
    assert f["nblend"].max() < 600
    assert np.array_equal(h["nblend"], f["nblend"])
    hs = np.sort(np.where(h["seq"] < 0, 1 << 30, h["seq"]), axis=2)
    fs = np.sort(np.where(f["seq"] < 0, 1 << 30, f["seq"]), axis=2)
    assert np.array_equal(hs, fs)
    if flags:
        base = oracle.render(sc, cam, prm)
        assert (h["hash"] != base["hash"]).mean() > 0.05


# --------------------------------------------------------------------- Sec. 3.4 schedule
def _late(n, src, D):
    order = list(range(n))
    x = order.pop(src)
    order.insert(src + D, x)
    return np.array(order, float)


def test_hier_window_is_25_in_the_worst_case(oracle):
    """Sec. 3.4: the effective window is at least 25 (tail drained to 17 plus 4 in mid and 4 in
    head). Worst case: 32 survivors, then 17 survivors (15 culled) drain the tail to 17; an entry
    arriving 25 survivor positions late is still sorted, 26 is not."""
    def case(disp):
        xr = 49 - disp
        loaded = [r for r in range(50) if r != xr]
        t = loaded[:32] + loaded[32:49] + [1000 + k for k in range(15)] + [xr]
        keep = [1] * 49 + [0] * 15 + [1]
        t = np.array(t, float)
        out = oracle.schedule_synthetic(t, np.array(keep))
        assert len(out) == 50
        return bool(np.all(np.diff(t[out]) >= 0))
    assert all(case(d) for d in range(0, 26))
    assert not case(26)


def test_hier_sorts_any_list_displaced_by_at_most_25(oracle):
    rng = np.random.default_rng(16)
    for trial in range(200):
        n = int(rng.integers(1, 300))
        keep = (rng.random(n) < rng.uniform(0.3, 1.0)).astype(np.int32)
        surv = np.nonzero(keep)[0]
        # survivor ranks displaced by at most 25 positions (late or early)
        keys = np.arange(len(surv)) + rng.uniform(0, 25.999, len(surv))
        rank_at = np.empty(len(surv))
        rank_at[np.argsort(keys, kind="stable")] = np.arange(len(surv))
        t = np.full(n, 1e6) + np.arange(n)
        t[surv] = np.argsort(np.argsort(keys, kind="stable"), kind="stable")
        ranks_in_list = t[surv]
        disp = np.abs(np.argsort(np.argsort(ranks_in_list)) - np.arange(len(surv)))
        assert disp.max(initial=0) <= 25
        out = oracle.schedule_synthetic(t, keep)
        assert len(out) == len(surv)
        assert np.all(np.diff(t[out]) >= 0)


@pytest.mark.parametrize("k", [4, 8, 16, 24])
def test_resort_window_k(oracle, k):
    """Sec. 3.3: a k-buffer of size k blends the smallest on overflow, so an entry arriving
    up to k positions late is placed correctly and k+1 is not."""
    n = 80
    ok = [bool(np.all(np.diff(t[oracle.schedule_synthetic(t, None, mode=I.MODE_WINDOW, head=k)]) >= 0))
          for t in (_late(n, 30, d) for d in (k, k + 1))]
    assert ok == [True, False]


def test_equal_depths_keep_their_list_order(oracle):
    """Reading of the queue merges (Sec. 3.4) and the per-pixel insertion (Sec. 3.3): entries of
    equal depth leave every queue in list order (existing entries first, a new one after its
    equals), so within the sorting window the blend order is the STABLE sort of the list; the
    full per-ray sort (Sec. 3.2) breaks ties by list position too. Lists with many exact ties,
    each entry displaced by at most 21 positions."""
    rng = np.random.default_rng(31)
    # a sorted list of runs of 6 equal depths: the order must stay the list order
    t = np.arange(200) // 6 * 1.0
    keep = (rng.random(200) < 0.7).astype(np.int32)
    assert np.array_equal(oracle.schedule_synthetic(t, keep), np.nonzero(keep)[0])
    for trial in range(120):
        n = int(rng.integers(1, 300))
        keep = (rng.random(n) < rng.uniform(0.3, 1.0)).astype(np.int32)
        s = np.sort(rng.integers(0, max(1, n // 6), n)).astype(float)
        t = s[np.argsort(np.arange(n) + rng.uniform(0, 20.999, n), kind="stable")]
        surv = np.nonzero(keep)[0]
        assert np.array_equal(oracle.schedule_synthetic(t, keep), surv[np.argsort(t[surv], kind="stable")])
        stable = np.argsort(t, kind="stable")
        assert np.array_equal(oracle.schedule_synthetic(t, None, mode=I.MODE_FULL), stable)
        assert np.array_equal(oracle.schedule_synthetic(t, None, mode=I.MODE_WINDOW, head=24), stable)


def test_evict_first_reading_shrinks_every_window_by_one(oracle):
    """Under the other reading of the full per-pixel queue (Sec. 3.4: blend the front before
    inserting), a k-buffer handles an entry k - 1 positions late but not k, and the hierarchy's
    worst-case window is 24 instead of 25."""
    for k in (1, 2, 4, 8, 16, 24):
        ok = [bool(np.all(np.diff(t[oracle.schedule_synthetic(t, None, mode=I.MODE_WINDOW, head=k,
                                                               flags=I.FLAG_HEAD_EVICT_FIRST)]) >= 0))
              for t in (_late(80, 30, d) for d in (k - 1, k))]
        assert ok == [True, False], k

    def case(disp):
        xr = 49 - disp
        loaded = [r for r in range(50) if r != xr]
        t = np.array(loaded[:32] + loaded[32:49] + [1000 + k for k in range(15)] + [xr], float)
        keep = np.array([1] * 49 + [0] * 15 + [1])
        out = oracle.schedule_synthetic(t, keep, flags=I.FLAG_HEAD_EVICT_FIRST)
        return bool(np.all(np.diff(t[out]) >= 0))
    assert all(case(d) for d in range(0, 25)) and not case(25)


def test_layered_scene_all_orderings_agree(oracle):
    sc = I.layered_scene(6, 10, 7)
    cam = I.look_at((0.2, 0.1, -3), (0, 0, 0), (0, 1, 0), 160, 144, 60.0)
    outs = {m: oracle.render(sc, cam, I.RenderParams(mode=m)) for m in
            (I.MODE_HIER, I.MODE_FULL, I.MODE_GLOBAL)}
    d = outs[0]["decided"] & outs[1]["decided"] & outs[2]["decided"]
    assert d.mean() > 0.99 and outs[0]["nblend"].max() >= 3
    for m in (I.MODE_FULL, I.MODE_GLOBAL):
        assert np.array_equal(outs[m]["hash"][d], outs[0]["hash"][d])
        assert np.allclose(outs[m]["rgb"][d], outs[0]["rgb"][d], atol=1e-12)


def test_sort_error_full_is_zero_and_hier_beats_small_windows(oracle):
    """Sec. 3.3 / Tab. sortcost: full per-ray sort has delta = 0; the hierarchical order has a
    smaller sort error than a resort window of 4 (trend of the table, on a synthetic scene)."""
    sc = I.cluster_scene(20000, 31, nclusters=8, centre_range=1.0, scale_range=(0.005, 0.1))
    cam = I.look_at((0, 0.5, -6), (0, 0, 0), (0, 1, 0), 128, 128, 50.0)
    full = oracle.render(sc, cam, I.RenderParams(mode=I.MODE_FULL))
    hier = oracle.render(sc, cam, I.RenderParams())
    win4 = oracle.render(sc, cam, I.RenderParams(mode=I.MODE_WINDOW, window_k=4))
    glob = oracle.render(sc, cam, I.RenderParams(mode=I.MODE_GLOBAL))
    assert full["delta"].max() == 0.0
    assert hier["delta"].mean() < win4["delta"].mean() < glob["delta"].mean()
    assert hier["nblend"].mean() > 5


def test_tile_depth_adjustment_reduces_sort_error(oracle):
    """Sec. 3.4 "Tile-depth adjustment": a tile key from t_opt on the ray through x_hat sorts
    better than the key from the tile-centre ray (the paper: (1.553, 0.006) -> (0.575, 0.003))
    and better than 3DGS's view-space depth of the mean (ablation B)."""
    sc = I.cluster_scene(20000, 32, nclusters=8, centre_range=1.0, scale_range=(0.005, 0.15))
    cam = I.look_at((0, 0.5, -6), (0, 0, 0), (0, 1, 0), 128, 128, 50.0)
    a = oracle.render(sc, cam, I.RenderParams(mode=I.MODE_GLOBAL))
    b = oracle.render(sc, cam, I.RenderParams(mode=I.MODE_GLOBAL, flags=I.FLAG_TILE_CENTRE_KEY))
    c = oracle.render(sc, cam, I.RenderParams(mode=I.MODE_GLOBAL, flags=I.FLAG_VIEW_DEPTH_KEY))
    assert a["delta"].mean() < b["delta"].mean() and a["delta"].mean() < c["delta"].mean()
    ha = oracle.render(sc, cam, I.RenderParams())
    hb = oracle.render(sc, cam, I.RenderParams(flags=I.FLAG_TILE_CENTRE_KEY))
    assert ha["delta"].mean() < hb["delta"].mean() and ha["delta"].max() < hb["delta"].max()


def test_input_order_does_not_matter(oracle):
    sc, cams, prm = I.plain_forward_workload()
    perm = np.random.default_rng(17).permutation(sc.n)
    a = oracle.render(sc, cams[0], prm, max_seq=64)
    b = oracle.render(sc.permuted(perm), cams[0], prm, max_seq=64)
    d = a["decided"] & b["decided"]
    assert d.mean() > 0.98
    assert np.allclose(a["rgb"][d], b["rgb"][d], atol=1e-12)
    sa = a["seq"][d]
    sb = np.where(b["seq"][d] >= 0, perm[np.maximum(b["seq"][d], 0)], -1)
    assert np.array_equal(sa, sb)


# --------------------------------------------------------------------- Sec. 3.5 adjoint
def _scene64(sc):
    return I.Scene(sc.means.astype(np.float64), sc.log_scales.astype(np.float64),
                   sc.quats.astype(np.float64), sc.opacity_logits.astype(np.float64),
                   sc.sh.astype(np.float64), sc.sh_degree)


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.2, 0.5, 0.9)], ids=["black", "coloured"])
def test_adjoint_matches_central_differences(oracle, bg):
    """Front-to-back adjoint with C - C_i and T_N / T_i (Sec. 3.5) chained through the
    preprocess, against FP64 central differences of L = <w, rgb> + <wz, depth>; parameters
    whose +-h perturbation changes any blend decision are skipped. A coloured background
    brings in the T_N bg term of the colour gradient."""
    sc, _, cam, prm = I.fd_subcase()
    prm = dataclasses.replace(prm, bg=bg)
    sc = _scene64(sc)
    rng = np.random.default_rng(18)
    H, W = cam.height, cam.width
    w = rng.normal(size=(H, W, 3)) / (H * W)
    wz = rng.normal(size=(H, W)) / (H * W) * 0.1
    with oracle.OracleRun(sc, cam, prm, record=True) as r:
        base = r.render()
        adj = r.backward(w, wz)

    def loss_and_hash(s):
        o = oracle.render(s, cam, prm)
        return float((w * o["rgb"]).sum() + (wz * o["depth"]).sum()), o["hash"], o["nblend"]

    contrib = np.nonzero(np.abs(adj["opacity"]) > 1e-6)[0]
    assert len(contrib) > 50
    fields = [("means", 3), ("log_scales", 3), ("quats", 4), ("opacity_logits", 1), ("sh", 48)]
    checked = 0
    for trial in range(90):
        i = int(rng.choice(contrib))
        name, k = fields[trial % len(fields)]
        j = int(rng.integers(k))
        arr = getattr(sc, name)
        val = arr.reshape(sc.n, -1)[i, j]
        h = 1e-6 * max(1.0, abs(val))
        res = []
        for sgn in (1, -1):
            s2 = I.Scene(*(a.copy() for a in (sc.means, sc.log_scales, sc.quats, sc.opacity_logits, sc.sh)),
                         sc.sh_degree)
            getattr(s2, name).reshape(sc.n, -1)[i, j] = val + sgn * h
            res.append(loss_and_hash(s2))
        if not all(np.array_equal(rr[1], base["hash"]) and np.array_equal(rr[2], base["nblend"])
                   for rr in res):
            continue
        fd = (res[0][0] - res[1][0]) / (2 * h)
        g = adj[name].reshape(sc.n, -1)[i, j]
        assert abs(fd - g) <= 1e-6 * max(abs(g), abs(fd)) + 1e-9, (name, i, j, fd, g)
        checked += 1
    assert checked >= 60


def test_adjoint_suffix_terms_equal_a_back_to_front_pass(oracle):
    """Sec. 3.5: the adjoint walks the blend order front to back with the suffix colour C - C_i
    (plus T_N bg) and the suffix transmittance T_N / T_i. A back-to-front pass, written here in
    numpy from the blend order alone (3DGS's order of accumulation), must give the same
    colour and opacity gradients, to rounding, with a coloured background and a depth term."""
    sc, _, cam, prm = I.fd_subcase()
    sc = _scene64(sc)
    bg = np.array([0.2, 0.5, 0.9])
    prm = dataclasses.replace(prm, bg=tuple(bg))
    rng = np.random.default_rng(19)
    H, W = cam.height, cam.width
    w = rng.normal(size=(H, W, 3))
    wz = rng.normal(size=(H, W)) * 0.1
    with oracle.OracleRun(sc, cam, prm, record=True) as r:
        pp = r.preprocess()
        out = r.render(max_seq=512)
        adj = r.backward(w, wz)
    assert out["nblend"].max() < 512
    Rc = cam.R.astype(np.float32).astype(np.float64)
    f32 = lambda v: float(np.float32(v))  # noqa: E731
    fx, fy, cx, cy = f32(cam.fx), f32(cam.fy), f32(cam.cx), f32(cam.cy)
    s6 = pp["sinv6"]
    sinv = np.stack([s6[:, [0, 1, 2]], s6[:, [1, 3, 4]], s6[:, [2, 4, 5]]], 1)
    gcol, gop = np.zeros((sc.n, 3)), np.zeros(sc.n)
    for y in range(H):
        for x in range(W):
            ids = out["seq"][y, x, :out["nblend"][y, x]]
            if len(ids) == 0:
                continue
            px, py = x + 0.5, y + 0.5
            d = Rc.T @ np.array([(px - cx) / fx, (py - cy) / fy, 1.0])
            d /= np.linalg.norm(d)
            dx, dy = px - pp["mean2"][ids, 0], py - pp["mean2"][ids, 1]
            cn = pp["conic"][ids]
            G2 = np.exp(-0.5 * (cn[:, 0] * dx * dx + 2 * cn[:, 1] * dx * dy + cn[:, 2] * dy * dy))
            raw = pp["opacity"][ids] * G2
            a = np.minimum(0.99, raw)
            t = (pp["v"][ids] @ d) / np.einsum("i,kij,j->k", d, sinv[ids], d)
            T = np.concatenate([[1.0], np.cumprod(1.0 - a)])
            assert T[-1] == pytest.approx(out["tfinal"][y, x], rel=1e-12)
            col = pp["color"][ids]
            acc_c, acc_z = bg * T[-1], 0.0            # what lies behind: the background first
            for k in range(len(ids) - 1, -1, -1):
                i = ids[k]
                gcol[i] += w[y, x] * a[k] * T[k]
                da = w[y, x] @ (col[k] * T[k] - acc_c / (1.0 - a[k])) + wz[y, x] * (t[k] * T[k] - acc_z / (1.0 - a[k]))
                if raw[k] < 0.99:
                    gop[i] += da * G2[k]
                acc_c = acc_c + col[k] * a[k] * T[k]
                acc_z += t[k] * a[k] * T[k]
    assert np.abs(gop).max() > 1e-3
    assert np.allclose(adj["color"], gcol, rtol=1e-9, atol=1e-12 * np.abs(gcol).max())
    assert np.allclose(adj["opacity"], gop, rtol=1e-9, atol=1e-12 * np.abs(gop).max())


# --------------------------------------------------------------------- ablations D and E
def test_without_tile_culling_lists_grow_but_per_pixel_orders_do_not_change(oracle):
    """Ablation D (Tab. performance_ablation): keeping every tile of a Gaussian's rectangle
    adds exactly the rectangle tiles Algorithm 1 culls. Each added entry is below eps_O at every
    pixel of its tile, so the orders that test alpha per pixel over the whole list (FULL,
    GLOBAL) give the same images, and the hierarchy culls the additions at its 4x4 level."""
    sc = I.uniform_scene(600, 21, scale_range=(0.01, 0.2))
    cam = I.look_at((0, 0, -3), (0, 0, 0), (0, 1, 0), 96, 80, 60.0)
    base = I.RenderParams()
    with oracle.OracleRun(sc, cam, base) as r:
        pp = r.preprocess()
    vis = pp["visible"] > 0
    rc = pp["rect"][vis]
    area = int(((rc[:, 2] - rc[:, 0] + 1) * (rc[:, 3] - rc[:, 1] + 1)).sum())
    for mode in (I.MODE_FULL, I.MODE_GLOBAL, I.MODE_HIER):
        a = oracle.render(sc, cam, dataclasses.replace(base, mode=mode))
        b = oracle.render(sc, cam, dataclasses.replace(base, mode=mode, flags=I.FLAG_NO_TILE_CULL))
        assert b["num_entries"] == area > a["num_entries"] == int(pp["ntiles"].sum())
        d = a["decided"] & b["decided"]
        if mode != I.MODE_HIER:
            assert d.mean() > 0.97
            assert np.array_equal(a["hash"][d], b["hash"][d]) and np.array_equal(a["rgb"][d], b["rgb"][d])
        else:
            # same 4x4 survivors; only the batch boundaries of the longer lists move
            assert a["counters"]["surv_subtile"] == b["counters"]["surv_subtile"]
            assert b["counters"]["eval_subtile"] > a["counters"]["eval_subtile"]


def test_without_hierarchical_culling_every_entry_reaches_the_pixels(oracle):
    """Ablation E: without the 4x4 / 2x2 culls every list entry survives both levels, the
    per-pixel alpha test still drops the non-contributors, so well separated layers blend in
    the exact order, as with culling."""
    sc = I.layered_scene(6, 10, 7)
    cam = I.look_at((0.2, 0.1, -3), (0, 0, 0), (0, 1, 0), 160, 144, 60.0)
    full = oracle.render(sc, cam, I.RenderParams(mode=I.MODE_FULL))
    e = oracle.render(sc, cam, I.RenderParams(flags=I.FLAG_NO_HIER_CULL))
    h = oracle.render(sc, cam, I.RenderParams())
    d = full["decided"] & e["decided"]
    assert d.mean() > 0.97
    assert np.array_equal(e["hash"][d], full["hash"][d])
    assert e["counters"]["surv_subtile"] == e["counters"]["eval_subtile"] > h["counters"]["surv_subtile"]
    assert e["counters"]["eval_quad"] > h["counters"]["eval_quad"]


def test_global_order_decided_pixels_have_a_clear_termination_order(oracle):
    """Reading R9 for the list orders: a pixel counts as decided only if the entry that ends its
    ray and the next contributing entry of the tile list are more than the depth-gap threshold
    apart (swapped, the other one would be taken first). Recomputed here from the oracle's own
    tile lists and preprocess: GLOBAL blending per pixel in numpy."""
    base = I.cluster_scene(3000, 41, nclusters=4, centre_range=1.0, scale_range=(0.01, 0.1))
    base.opacity_logits[:] = 4.0                     # opaque: rays end after a few blends
    cam = I.look_at((0.2, -0.1, -4), (0, 0, 0), (0, 1, 0), 128, 96, 50.0)
    # a tenth of the Gaussians get a twin 1e-7 of their depth further along their view ray, so
    # some rays end on an entry whose twin follows it in the list at a near-equal key
    eye = -cam.R.T @ cam.t
    pick = np.random.default_rng(5).random(base.n) < 0.1
    d = base.means[pick] - eye
    twin = I.Scene(base.means[pick] + 1e-7 * d, base.log_scales[pick], base.quats[pick],
                   base.opacity_logits[pick], base.sh[pick], base.sh_degree)
    sc = I.Scene(*[np.concatenate([getattr(base, f), getattr(twin, f)]) for f in
                   ("means", "log_scales", "quats", "opacity_logits", "sh")], base.sh_degree)
    prm = I.RenderParams(mode=I.MODE_GLOBAL)
    with oracle.OracleRun(sc, cam, prm) as r:
        pp = r.preprocess()
        start, ids, ts = r.tile_lists()
        out = r.render()
    checked = tied = 0
    for y in range(cam.height):
        for x in range(cam.width):
            t = (y // 16) * cam.tiles_x + x // 16
            L, K = ids[start[t]:start[t + 1]], ts[start[t]:start[t + 1]]
            m = pp["mean2"][L]
            a_, b_, c_ = pp["conic"][L].T
            dx, dy = x + 0.5 - m[:, 0], y + 0.5 - m[:, 1]
            al = np.minimum(prm.alpha_max, pp["opacity"][L] * np.exp(-0.5 * (a_ * dx * dx + 2 * b_ * dx * dy + c_ * dy * dy)))
            contrib = np.nonzero(al >= prm.eps_o)[0]
            T, stop = 1.0, None
            for k, j in enumerate(contrib):
                if T * (1 - al[j]) < prm.t_min:
                    stop = k
                    break
                T *= 1 - al[j]
            if stop is None or stop + 1 >= len(contrib):
                continue
            k0, k1 = K[contrib[stop]], K[contrib[stop + 1]]
            gap = abs(k0 - k1) / max(abs(k0), abs(k1), 1e-30)
            if out["decided"][y, x]:
                assert gap > oracle.GAP_THR, (x, y, gap)
            checked += 1
            tied += gap <= oracle.GAP_THR
    assert checked > 200 and tied > 20


def test_key_prefix_keeps_pixels_finished_inside_its_complete_batches(oracle):
    """A render of each tile's list truncated to the entries below a depth cut (a prefix of
    the sorted list, Sec. 3.4 consumes lists in batches of 32) blends, at every pixel whose
    ray terminated while a batch the prefix holds completely was being processed, exactly
    the sequence the full list gives: up to that batch both runs take identical batches,
    pops and blends. This is the exactness condition of building the lists in depth slices
    (render a prefix, redo only the tiles it cannot finish). The condition is sharp: pixels
    that terminated inside the prefix's last, incomplete batch can differ."""
    sc = I.cluster_scene(20000, 91, nclusters=4, centre_range=0.8, scale_range=(0.01, 0.15))
    cam = I.orbit_cameras(1, 4.0, 0.5, [(128, 96)], 50.0)[0]
    with oracle.OracleRun(sc, cam, I.RenderParams()) as r:
        full = r.render()
        start, ids, ts = r.tile_lists()
        cut = float(np.quantile(ts, 0.4))
        pre = r.render(key_cut=cut)
    m = np.array([np.count_nonzero(ts[start[t]:start[t + 1]] < cut) for t in range(cam.num_tiles)])
    yy, xx = np.mgrid[0:cam.height, 0:cam.width]
    tile = (yy // 16) * cam.tiles_x + xx // 16
    b = full["sat_batch"]
    inside = (b >= 0) & (32 * (b + 1) <= m[tile])           # finished within complete batches
    partial = (b >= 0) & (32 * b < m[tile]) & ~inside       # finished in the last, partial batch
    same = (full["hash"] == pre["hash"]) & (full["nblend"] == pre["nblend"])
    assert inside.mean() > 0.1
    assert same[inside].all()
    assert (~same[partial]).any()                           # the complete-batch condition matters
    assert (~same).sum() > 1000                              # the cut removed entries others need
