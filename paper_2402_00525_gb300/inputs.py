"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the bench.

This module holds input construction only: random scenes, pinhole cameras and the render
parameter record. It contains none of the renderer's arithmetic (no projection, no culling,
no depth, no blending), so both implementations can consume it without sharing method code.

Scene shapes follow the workloads of StopThePop (Radl et al. 2024): the paper renders
trained 3DGS scenes of about 1-6 M anisotropic Gaussians with SH degree 3 at Full HD
(Sec. 4.3, Tab. "performance_ablation"). Those scenes are not available here, so seeded
generators with the same sizes and a heavy-tailed screen-size distribution stand in for
them.

Conventions (shared by both sides):
  * Gaussians are SoA float32: means [N,3], log_scales [N,3], quats [N,4] in (w, x, y, z)
    order (not necessarily normalised), opacity_logits [N], sh [N, (deg+1)^2, 3].
  * Cameras map world to camera space with p = R @ x + t, OpenCV axes (x right, y down,
    z forward), pinhole intrinsics fx, fy, cx, cy in pixels; pixel (u, v) has its centre
    at (u + 0.5, v + 0.5).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence

import numpy as np

# Paper constants (Sec. 3.4 "Tile-based culling": eps_O = 1/255; Sec. 3.2: S^-1 entries
# bounded by 1e3; Sec. 3.4: queue sizes 64/8/4; load-balance threshold 32).
EPS_O = 1.0 / 255.0

MODE_HIER = 0     # the paper's hierarchical 4x4 / 2x2 / per-pixel queues (Sec. 3.4)
MODE_FULL = 1     # full per-ray sort (Sec. 3.2, "naive sorting")
MODE_GLOBAL = 2   # blend in tile-list order (3DGS order, with per-tile t_opt keys)
MODE_WINDOW = 3   # per-ray resort window of K entries (Sec. 3.3, k-buffer)

# flag bits of RenderParams.flags
FLAG_HEAD_EVICT_FIRST = 1      # head queue: blend the front before inserting (alternative reading)
FLAG_LEVEL_CENTRE_RAYS = 2     # 4x4 / 2x2 depth from the level-centre ray instead of its x_hat
FLAG_TILE_CENTRE_KEY = 4       # tile sort key from the tile-centre ray (no tile-depth adjustment)
FLAG_VIEW_DEPTH_KEY = 8        # tile sort key = view-space depth of the mean (3DGS global depth)
FLAG_NO_LOAD_BALANCE = 16      # every Gaussian's tiles handled by its own thread
FLAG_GLOBAL_SORT = 256         # one global radix sort of (tile, depth) keys (same order)
FLAG_NO_TILE_CULL = 512        # ablation D: Duplicate keeps every tile of the rectangle
FLAG_NO_HIER_CULL = 1024       # ablation E: no culling at the 4x4 / 2x2 levels of Render


@dataclasses.dataclass
class RenderParams:
    """Knobs of the renderer. Defaults are the paper's (64/8/4 queues, eps_O = 1/255). The
    library checks every value on the host (include/stp.h states the ranges) and rejects a bad
    one before any launch."""
    tail: int = 64            # 4x4 tile-queue size, 32n+32 (Sec. 3.4)
    mid: int = 8              # 2x2 tile-queue size, 4m+4 (Sec. 3.4)
    head: int = 4             # per-pixel queue size (Sec. 3.4)
    lb_threshold: int = 32    # load-balancing tile threshold (Sec. 3.4 "Load Balancing")
    eps_o: float = EPS_O
    t_min: float = 1e-4       # transmittance early-out
    alpha_max: float = 0.99
    inv_scale_max: float = 1e3
    dilation: float = 0.3     # EWA low-pass kept from 3DGS
    frustum_clamp: float = 1.3
    znear: float = 0.2
    bg: tuple = (0.0, 0.0, 0.0)
    mode: int = MODE_HIER
    window_k: int = 16
    flags: int = 0
    # ids stored per pixel by a forward that a backward follows (the backward walks them instead
    # of replaying the queues; pixels that blend more are replayed): 4 * blend_cap bytes a pixel
    blend_cap: int = 192
    # FULL order only: bound on the peeling passes over a tile's list (0 = enough for any list)
    full_max_passes: int = 0
    # HIER with the partitioned sort: lists built in depth slices, about the slice_k nearest
    # entries of each tile first (0 = whole lists in one pass); the images are the same
    slice_k: int = 2048


@dataclasses.dataclass
class Camera:
    R: np.ndarray          # [3,3] float64, world -> camera rotation
    t: np.ndarray          # [3]   float64
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int

    @property
    def tiles_x(self) -> int:
        return (self.width + 15) // 16

    @property
    def tiles_y(self) -> int:
        return (self.height + 15) // 16

    @property
    def num_tiles(self) -> int:
        return self.tiles_x * self.tiles_y

    @property
    def num_pixels(self) -> int:
        return self.width * self.height


@dataclasses.dataclass
class Scene:
    means: np.ndarray          # [N,3] float32
    log_scales: np.ndarray     # [N,3] float32
    quats: np.ndarray          # [N,4] float32 (w, x, y, z)
    opacity_logits: np.ndarray # [N]   float32
    sh: np.ndarray             # [N,K,3] float32, K = (deg+1)^2
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def permuted(self, perm: np.ndarray) -> "Scene":
        return Scene(self.means[perm].copy(), self.log_scales[perm].copy(),
                     self.quats[perm].copy(), self.opacity_logits[perm].copy(),
                     self.sh[perm].copy(), self.sh_degree)


# ----------------------------------------------------------------------------- cameras
def look_at(eye: Sequence[float], target: Sequence[float], down: Sequence[float],
            width: int, height: int, fov_y_deg: float, fov_x_deg: float | None = None) -> Camera:
    """OpenCV-axes pinhole camera at `eye` looking at `target`; `down` is the world vector
    that should appear pointing down in the image."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(down, fwd)
    right /= np.linalg.norm(right)
    dn = np.cross(fwd, right)
    R = np.stack([right, dn, fwd])          # rows = camera axes in world coordinates
    t = -R @ eye
    fy = 0.5 * height / math.tan(math.radians(fov_y_deg) * 0.5)
    fx = fy if fov_x_deg is None else 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return Camera(R=R, t=t, fx=float(fx), fy=float(fy), cx=0.5 * width, cy=0.5 * height,
                  width=int(width), height=int(height))


def orbit_cameras(nviews: int, radius: float, height: float, sizes: Sequence[tuple],
                  fov_y_deg: float) -> List[Camera]:
    """`nviews` cameras on a 360 degree orbit around the world y axis, looking at the origin.
    `sizes` is cycled round-robin over the views."""
    cams = []
    for v in range(nviews):
        phi = 2.0 * math.pi * v / nviews
        eye = (radius * math.cos(phi), height, radius * math.sin(phi))
        w, h = sizes[v % len(sizes)]
        cams.append(look_at(eye, (0.0, 0.0, 0.0), (0.0, -1.0, 0.0), w, h, fov_y_deg))
    return cams


# ----------------------------------------------------------------------------- scenes
# Decoded DC colour rgb = Y00 * dc + 0.5 with Y00 = 1/(2 sqrt(pi)); a DC coefficient drawn
# uniformly from [-sqrt(pi), sqrt(pi)] therefore decodes to a colour uniform in [0, 1].
_DC_HALF_RANGE = math.sqrt(math.pi)


def _uniform_quats(rng: np.random.Generator, n: int) -> np.ndarray:
    """Uniformly distributed unit quaternions (Shoemake's subgroup algorithm)."""
    u = rng.random((n, 3))
    a = np.sqrt(1.0 - u[:, 0])
    b = np.sqrt(u[:, 0])
    q = np.stack([a * np.sin(2 * np.pi * u[:, 1]), a * np.cos(2 * np.pi * u[:, 1]),
                  b * np.sin(2 * np.pi * u[:, 2]), b * np.cos(2 * np.pi * u[:, 2])], axis=1)
    return q


def _logit(p: np.ndarray) -> np.ndarray:
    p = np.clip(p, 1e-6, 1 - 1e-6)
    return np.log(p) - np.log1p(-p)


def _random_rotations(rng: np.random.Generator, n: int) -> np.ndarray:
    """Random rotation matrices (QR of Gaussian matrices, sign-fixed, det +1) for the
    cluster shapes of the generator."""
    A = rng.standard_normal((n, 3, 3))
    Q, Rr = np.linalg.qr(A)
    Q = Q * np.sign(np.diagonal(Rr, axis1=1, axis2=2))[:, None, :]
    Q[np.linalg.det(Q) < 0, :, 0] *= -1.0
    return Q


def uniform_scene(n: int, seed: int, scale_range=(0.005, 0.05), opacity_range=(0.1, 0.99),
                  extent: float = 1.0, sh_degree: int = 0) -> Scene:
    """Means uniform in [-extent, extent]^3, per-axis scales log-uniform, uniform rotations,
    opacity uniform, DC colour uniform in [0,1] (higher SH bands N(0, 0.1) if sh_degree > 0)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-extent, extent, (n, 3))
    ls = rng.uniform(math.log(scale_range[0]), math.log(scale_range[1]), (n, 3))
    quats = _uniform_quats(rng, n)
    op = rng.uniform(opacity_range[0], opacity_range[1], n)
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, (n, k - 1, 3))
    return Scene(means.astype(np.float32), ls.astype(np.float32), quats.astype(np.float32),
                 _logit(op).astype(np.float32), sh.astype(np.float32), sh_degree)


def cluster_scene(n: int, seed: int, nclusters: int = 64, centre_range: float = 5.0,
                  spread_range=(0.2, 1.0), scale_range=(1e-3, 0.3), max_aniso: float = 100.0,
                  sh_degree: int = 3, centres: np.ndarray | None = None) -> Scene:
    """Mixture of anisotropic Gaussian clusters.

    Cluster centres uniform in [-c, c]^3; member offsets ~ N(0, R_k diag(sigma_k^2) R_k^T)
    with per-axis sigma_k log-uniform in `spread_range`; per-axis scales log-uniform in
    `scale_range`, resampled until max/min <= `max_aniso`; opacity Beta(0.5, 0.5) drawn by the
    exact inverse CDF sin^2(pi U / 2); SH DC decoded colour uniform in [0,1], higher bands
    N(0, 0.1).
    """
    rng = np.random.default_rng(seed)
    if centres is None:
        centres = rng.uniform(-centre_range, centre_range, (nclusters, 3))
    else:
        centres = np.asarray(centres, np.float64).reshape(-1, 3)
        nclusters = centres.shape[0]
    sig = np.exp(rng.uniform(math.log(spread_range[0]), math.log(spread_range[1]), (nclusters, 3)))
    rk = _random_rotations(rng, nclusters)
    counts = np.full(nclusters, n // nclusters)
    counts[: n - counts.sum()] += 1
    means = np.empty((n, 3))
    o = 0
    for k in range(nclusters):
        z = rng.standard_normal((counts[k], 3)) * sig[k]
        means[o:o + counts[k]] = centres[k] + z @ rk[k].T
        o += counts[k]
    lo, hi = math.log(scale_range[0]), math.log(scale_range[1])
    ls = rng.uniform(lo, hi, (n, 3))
    bad = (ls.max(1) - ls.min(1)) > math.log(max_aniso)
    while bad.any():
        ls[bad] = rng.uniform(lo, hi, (int(bad.sum()), 3))
        bad = (ls.max(1) - ls.min(1)) > math.log(max_aniso)
    quats = _uniform_quats(rng, n)
    op = np.sin(0.5 * np.pi * rng.random(n)) ** 2
    k = (sh_degree + 1) ** 2
    sh = np.empty((n, k, 3), np.float32)
    sh[:, 0, :] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, 0.1, (n, k - 1, 3))
    return Scene(means.astype(np.float32), ls.astype(np.float32), quats.astype(np.float32),
                 _logit(op).astype(np.float32), sh, sh_degree)


def perturbed(scene: Scene, seed: int, mean_sd=0.01, log_scale_sd=0.05, dc_sd=0.05,
              logit_sd=0.1) -> Scene:
    """Copy of `scene` with Gaussian noise on means, log-scales, SH DC and opacity logits
    (the differentiation workload's target parameters)."""
    rng = np.random.default_rng(seed)
    sh = scene.sh.copy()
    sh[:, 0, :] += rng.normal(0, dc_sd, sh[:, 0, :].shape).astype(np.float32)
    return Scene((scene.means + rng.normal(0, mean_sd, scene.means.shape)).astype(np.float32),
                 (scene.log_scales + rng.normal(0, log_scale_sd, scene.log_scales.shape)).astype(np.float32),
                 scene.quats.copy(),
                 (scene.opacity_logits + rng.normal(0, logit_sd, scene.n)).astype(np.float32),
                 sh, scene.sh_degree)


def layered_scene(nlayers: int, grid: int, seed: int, spacing: float = 1.0, z0: float = 2.0,
                  extent: float = 1.0) -> Scene:
    """Gaussians on planes z = z0 + k*spacing: each layer is a jittered grid x grid lattice
    over [-extent, extent]^2 of small isotropic Gaussians whose footprints do not overlap
    within a layer. Every ordering (global, per-tile, per-ray) then agrees at every pixel,
    which pins the hierarchical schedule against the full per-ray sort."""
    rng = np.random.default_rng(seed)
    cell = 2.0 * extent / grid
    pts = []
    for k in range(nlayers):
        gx, gy = np.meshgrid(np.arange(grid), np.arange(grid), indexing="ij")
        c = np.stack([gx.ravel(), gy.ravel()], 1) * cell - extent + 0.5 * cell
        c = c + rng.uniform(-0.1 * cell, 0.1 * cell, c.shape)
        z = np.full((c.shape[0], 1), z0 + spacing * k)
        pts.append(np.concatenate([c, z], 1))
    means = np.concatenate(pts, 0)
    n = means.shape[0]
    ls = np.full((n, 3), math.log(0.06 * cell))
    quats = _uniform_quats(rng, n)
    op = rng.uniform(0.3, 0.9, n)
    sh = np.zeros((n, 1, 3))
    sh[:, 0, :] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (n, 3))
    perm = rng.permutation(n)   # input order must not matter
    return Scene(means[perm].astype(np.float32), ls[perm].astype(np.float32),
                 quats[perm].astype(np.float32), _logit(op[perm]).astype(np.float32),
                 sh[perm].astype(np.float32), 0)


# ----------------------------------------------------------------------------- workloads
SEED_BASE = 0x57090000

C2_SIZES = [(1920, 1080)]
C4_SIZES = [(320, 240), (640, 480), (1280, 720), (1920, 1080), (2560, 1440)]
C5_SIZES = [(640, 480), (1280, 720), (1600, 900), (1920, 1080)]
C5_SCENE_SIZES = [100_000, 250_000, 500_000, 750_000, 1_000_000, 1_500_000, 2_000_000, 3_000_000]


def plain_forward_workload():
    """4096 Gaussians, means U[-1,1]^3, scales log-U[0.005,0.05], opacity U[0.1,0.99], SH0;
    camera at distance 3 looking at the origin, fov 60 deg, 256x256; k-buffer window 16."""
    scene = uniform_scene(4096, SEED_BASE + 1)
    cam = look_at((0, 0, -3), (0, 0, 0), (0, 1, 0), 256, 256, 60.0)
    return scene, [cam], RenderParams(head=16)


def full_hd_workload(n: int = 3_000_000, nviews: int = 16):
    """3M Gaussians in 64 anisotropic clusters, SH3; 16 orbit views at 1920x1080, fov 50."""
    scene = cluster_scene(n, SEED_BASE + 2)
    cams = orbit_cameras(nviews, 15.0, 2.0, C2_SIZES, 50.0)
    return scene, cams, RenderParams()


def differentiation_workload(n: int = 500_000):
    """500k Gaussians (cluster generator, SH3), one 1280x720 view; target rendered from
    perturbed parameters."""
    scene = cluster_scene(n, SEED_BASE + 3)
    cam = orbit_cameras(1, 15.0, 2.0, [(1280, 720)], 50.0)[0]
    target = perturbed(scene, SEED_BASE + 4)
    return scene, target, cam, RenderParams()


def fd_subcase():
    """512 Gaussians in one cluster at the origin (sigma 0.3, scales [0.01, 0.1]), SH3,
    64x64 view from radius 3: the finite-difference check case."""
    scene = cluster_scene(512, SEED_BASE + 5, centres=np.zeros((1, 3)), spread_range=(0.3, 0.3),
                          scale_range=(0.01, 0.1))
    cam = orbit_cameras(1, 3.0, 0.4, [(64, 64)], 50.0)[0]
    target = perturbed(scene, SEED_BASE + 6)
    return scene, target, cam, RenderParams()


def batching_workload(n: int = 3_000_000, nviews: int = 64):
    scene = cluster_scene(n, SEED_BASE + 2)
    cams = orbit_cameras(nviews, 15.0, 2.0, C4_SIZES, 50.0)
    return scene, cams, RenderParams()


def batched_training_workload(scale: float = 1.0):
    scenes = [cluster_scene(max(64, int(s * scale)), SEED_BASE + 10 + i)
              for i, s in enumerate(C5_SCENE_SIZES)]
    cams = [orbit_cameras(4, 15.0, 2.0, C5_SIZES, 50.0) for _ in scenes]
    return scenes, cams, RenderParams()
