"""The seeded input generators (no GPU): each draws the distribution its recipe states, the same
seed gives the same scene, and the workload helpers build the sizes and cameras they name."""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2402_00525_gb300 import inputs as I

Y00 = 0.5 / math.sqrt(math.pi)          # degree-0 real SH basis value


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, np.float64)))


def _same(a: I.Scene, b: I.Scene) -> bool:
    return all(np.array_equal(getattr(a, f), getattr(b, f))
               for f in ("means", "log_scales", "quats", "opacity_logits", "sh")) and a.sh_degree == b.sh_degree


def test_same_seed_same_scene_other_seed_other_scene():
    assert _same(I.uniform_scene(500, 7), I.uniform_scene(500, 7))
    assert _same(I.cluster_scene(700, 7, nclusters=5), I.cluster_scene(700, 7, nclusters=5))
    assert not np.array_equal(I.cluster_scene(700, 7, nclusters=5).means, I.cluster_scene(700, 8, nclusters=5).means)
    s = I.cluster_scene(300, 3, nclusters=4)
    for arr in (s.means, s.log_scales, s.quats, s.opacity_logits, s.sh):
        assert arr.dtype == np.float32 and np.isfinite(arr).all()


def test_quaternions_are_unit_and_uniform_on_the_sphere():
    q = I._uniform_quats(np.random.default_rng(1), 200_000)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-12)
    # Haar-uniform rotations: E[q q^T] = I/4 and every coordinate has mean 0
    assert np.abs(q.T @ q / len(q) - 0.25 * np.eye(4)).max() < 4e-3
    assert np.abs(q.mean(0)).max() < 4e-3
    # ... and each coordinate of a uniform point on S^3 follows the semicircle law on [-1, 1],
    # which second moments alone do not fix
    def semicircle_cdf(x):
        x = np.clip(x, -1.0, 1.0)
        return 0.5 + (x * np.sqrt(1.0 - x * x) + np.arcsin(x)) / np.pi
    for j in range(4):
        assert stats.kstest(q[:50_000, j], semicircle_cdf).pvalue > 1e-3


def test_cluster_rotations_are_proper():
    R = I._random_rotations(np.random.default_rng(2), 500)
    assert np.allclose(R @ np.transpose(R, (0, 2, 1)), np.eye(3), atol=1e-12)
    assert np.allclose(np.linalg.det(R), 1.0, atol=1e-12)


def test_uniform_scene_ranges_and_distributions():
    n = 20_000
    s = I.uniform_scene(n, 11, sh_degree=1)
    assert s.means.shape == (n, 3) and s.sh.shape == (n, 4, 3)
    assert np.abs(s.means).max() <= 1.0
    sc = np.exp(s.log_scales.astype(np.float64))
    assert sc.min() >= 0.005 * (1 - 1e-6) and sc.max() <= 0.05 * (1 + 1e-6)
    op = _sigmoid(s.opacity_logits)
    assert op.min() >= 0.1 - 1e-5 and op.max() <= 0.99 + 1e-5
    rgb = Y00 * s.sh[:, 0, :].astype(np.float64) + 0.5          # decoded DC colour
    assert stats.kstest(rgb.ravel()[:n], "uniform").pvalue > 1e-3
    assert stats.kstest(s.log_scales[:, 0], "uniform",
                        args=(math.log(0.005), math.log(0.05) - math.log(0.005))).pvalue > 1e-3
    assert abs(s.sh[:, 1:, :].std() - 0.1) < 5e-3


def test_cluster_scene_recipe():
    n, k = 40_000, 16
    s = I.cluster_scene(n, 12, nclusters=k)
    ls = s.log_scales.astype(np.float64)
    assert ls.min() >= math.log(1e-3) - 1e-5 and ls.max() <= math.log(0.3) + 1e-5
    assert (ls.max(1) - ls.min(1)).max() <= math.log(100.0) + 1e-5     # max/min scale <= 100
    op = _sigmoid(s.opacity_logits)
    assert stats.kstest(op, stats.beta(0.5, 0.5).cdf).pvalue > 1e-3
    assert stats.kstest(Y00 * s.sh[:, 0, 1].astype(np.float64) + 0.5, "uniform").pvalue > 1e-3
    assert abs(s.sh[:, 1:, :].std() - 0.1) < 3e-3 and s.sh.shape[1] == 16
    # members come in k equal consecutive runs; each run's spread lies within [0.2, 1] per axis
    # along its own principal axes (up to sampling error)
    for c in range(k):
        m = s.means[c * (n // k):(c + 1) * (n // k)].astype(np.float64)
        ev = np.linalg.eigvalsh(np.cov(m.T))
        assert np.sqrt(ev).min() > 0.2 * 0.9 and np.sqrt(ev).max() < 1.0 * 1.1
        assert np.abs(m.mean(0)).max() < 5.0 + 0.1


def test_cluster_scene_with_fixed_centre():
    s = I.cluster_scene(2000, 13, centres=np.zeros((1, 3)), spread_range=(0.3, 0.3))
    assert np.abs(s.means.mean(0)).max() < 0.03
    assert np.allclose(np.sqrt(np.linalg.eigvalsh(np.cov(s.means.T.astype(np.float64)))), 0.3, rtol=0.1)


def _project(cam: I.Camera, x):
    p = np.asarray(cam.R) @ np.asarray(x, np.float64) + np.asarray(cam.t)
    return cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy, p[2]


def test_look_at_geometry():
    cam = I.look_at((1.0, -2.0, -3.0), (0.5, 0.5, 0.0), (0.0, 1.0, 0.0), 320, 200, 60.0)
    R = np.asarray(cam.R)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and math.isclose(np.linalg.det(R), 1.0, abs_tol=1e-12)
    u, v, z = _project(cam, (0.5, 0.5, 0.0))
    assert math.isclose(u, 160.0, abs_tol=1e-9) and math.isclose(v, 100.0, abs_tol=1e-9) and z > 0
    assert math.isclose(z, math.dist((1.0, -2.0, -3.0), (0.5, 0.5, 0.0)), rel_tol=1e-12)
    # the world `down` vector points down the image (v grows)
    assert _project(cam, (0.5, 0.5 + 0.1, 0.0))[1] > 100.0
    # a ray at half the vertical fov above the axis meets the top image edge
    fwd, dn = R[2], R[1]
    top = np.asarray((1.0, -2.0, -3.0)) + fwd - math.tan(math.radians(30.0)) * dn
    assert math.isclose(_project(cam, top)[1], 0.0, abs_tol=1e-9)
    assert cam.fx == cam.fy and cam.num_pixels == 64_000 and cam.num_tiles == 20 * 13


def test_orbit_cameras():
    sizes = [(64, 48), (32, 32), (80, 16)]
    cams = I.orbit_cameras(7, 15.0, 2.0, sizes, 50.0)
    assert len(cams) == 7
    for v, cam in enumerate(cams):
        assert (cam.width, cam.height) == sizes[v % 3]
        eye = -np.asarray(cam.R).T @ np.asarray(cam.t)
        assert math.isclose(math.hypot(eye[0], eye[2]), 15.0, rel_tol=1e-12)
        assert math.isclose(eye[1], 2.0, abs_tol=1e-12)
        assert math.isclose(math.atan2(eye[2], eye[0]) % (2 * math.pi), 2 * math.pi * v / 7, abs_tol=1e-9)
        u, w, _ = _project(cam, (0.0, 0.0, 0.0))
        assert math.isclose(u, cam.width / 2, abs_tol=1e-9) and math.isclose(w, cam.height / 2, abs_tol=1e-9)
        assert math.isclose(cam.fy, 0.5 * cam.height / math.tan(math.radians(25.0)), rel_tol=1e-12)


def test_perturbed_targets():
    s = I.cluster_scene(20_000, 14, nclusters=8)
    t = I.perturbed(s, 15)
    assert np.array_equal(t.quats, s.quats) and np.array_equal(t.sh[:, 1:], s.sh[:, 1:])
    for a, b, sd in ((t.means, s.means, 0.01), (t.log_scales, s.log_scales, 0.05),
                     (t.sh[:, 0], s.sh[:, 0], 0.05), (t.opacity_logits, s.opacity_logits, 0.1)):
        d = (a.astype(np.float64) - b).ravel()
        assert abs(d.std() - sd) < 0.05 * sd and abs(d.mean()) < 0.05 * sd


def test_layered_scene_footprints_do_not_overlap_within_a_layer():
    grid, nl = 6, 3
    s = I.layered_scene(nl, grid, 16)
    assert s.n == nl * grid * grid and s.sh_degree == 0
    cell = 2.0 / grid
    sigma = float(np.exp(s.log_scales.astype(np.float64)).max())
    assert math.isclose(sigma, 0.06 * cell, rel_tol=1e-6)
    z = s.means[:, 2].astype(np.float64)
    assert sorted(set(np.round(z, 5))) == pytest.approx([2.0, 3.0, 4.0])
    for zk in (2.0, 3.0, 4.0):
        p = s.means[np.isclose(z, zk)][:, :2].astype(np.float64)
        d = np.sqrt(((p[:, None] - p[None]) ** 2).sum(-1)) + np.eye(len(p)) * 1e9
        assert d.min() >= 0.8 * cell - 1e-6                    # >= 13 sigma between centres


def test_workload_sizes():
    scene, cams, prm = I.plain_forward_workload()
    assert scene.n == 4096 and scene.sh_degree == 0 and len(cams) == 1
    assert (cams[0].width, cams[0].height) == (256, 256) and prm.head == 16
    scene, cams, _ = I.full_hd_workload(n=2000)
    assert scene.n == 2000 and scene.sh_degree == 3 and len(cams) == 16
    assert all((c.width, c.height) == (1920, 1080) for c in cams)
    _, cams, _ = I.batching_workload(n=1000)
    assert len(cams) == 64 and sum(c.num_pixels for c in cams) == 88_166_400
    sizes = [(c.width, c.height) for c in cams]
    assert [sizes.count(s) for s in I.C4_SIZES] == [13, 13, 13, 13, 12]
    scenes, cams, _ = I.batched_training_workload(scale=1e-4)
    assert len(scenes) == 8 and all(len(c) == 4 for c in cams)
    assert sum(c.num_pixels for cs in cams for c in cs) == 37_939_200
    assert [s.n for s in scenes] == [max(64, int(x * 1e-4)) for x in I.C5_SCENE_SIZES]
    scene, target, cam, _ = I.fd_subcase()
    assert scene.n == 512 and (cam.width, cam.height) == (64, 64) and target.n == 512
    scene, target, cam, _ = I.differentiation_workload(n=3000)
    assert (cam.width, cam.height) == (1280, 720) and target.n == scene.n == 3000
