"""Depth-slice list building (RenderParams.slice_k) against whole lists (slice_k = 0).

The per-tile sort orders each tile's list only up to the first boundary of its depth buckets
that holds at least slice_k entries. A Render warp whose pixels all terminate within the
complete 32-entry batches of that prefix has consumed exactly what it would consume from the
whole list; the others are queued, their tiles' lists are sorted whole, and the warps are
rendered again. So every output -- image, depth, final T, blend count, blend-order
hash, sort error, the stored blend order and the gradients -- must equal the whole-list run.
slice_k = 1 sends nearly every warp of every covered tile through the second pass.
"""
import dataclasses

import numpy as np
import pytest
import torch

from gpu_helpers import gpu_render
from paper_2402_00525_gb300 import inputs as I
from paper_2402_00525_gb300 import renderer as R

pytestmark = pytest.mark.gpu

OUTPUTS = ("rgb", "depth", "tfinal", "nblend", "hash", "delta")


def _scene():
    sc = I.cluster_scene(60000, 80, nclusters=8, centre_range=1.5, scale_range=(0.003, 0.3))
    cams = I.orbit_cameras(3, 6.0, 1.0, [(320, 240), (256, 256), (200, 120)], 50.0)
    return sc, cams


def _same(a, b, label):
    for k in OUTPUTS:
        for v in range(len(a[k])):
            assert np.array_equal(a[k][v], b[k][v]), (label, k, v)


@pytest.mark.parametrize("k", [1, 32, 256, 1024])
def test_slices_equal_whole_lists(k):
    sc, cams = _scene()
    prm = I.RenderParams(slice_k=0)
    whole = gpu_render(sc, cams, prm)
    part = gpu_render(sc, cams, dataclasses.replace(prm, slice_k=k))
    _same(part, whole, "slice_k %d" % k)
    sw, sp = whole["renderer"].status(), part["renderer"].status()
    assert sw.error_bits == 0 and sp.error_bits == 0 and sp.mismatched == 0
    assert sw.redo_warps == 0
    # the work counters count each warp once: the second pass replaces, not adds
    assert list(sp.counters) == list(sw.counters)
    if k == 1:
        # most warps of the three images went through the second pass
        assert sp.redo_warps > 0.4 * 8 * sum(c.num_tiles for c in cams)
    print("slice_k", k, "warps rendered twice:", sp.redo_warps)


def test_slice_lists_are_prefixes_or_whole():
    """With slices the tile ranges start where the whole lists start; a tile the second pass
    completed holds its whole list, every other tile a prefix of it."""
    sc, cams = _scene()
    prm = I.RenderParams(slice_k=0)
    whole = gpu_render(sc, cams, prm)
    part = gpu_render(sc, cams, dataclasses.replace(prm, slice_k=1024))
    rw, _, vw = [x.cpu().numpy() for x in whole["renderer"].sorted_lists()]
    rp, _, vp = [x.cpu().numpy() for x in part["renderer"].sorted_lists()]
    nw, np_ = rw[:, 1] - rw[:, 0], rp[:, 1] - rp[:, 0]
    live = nw > 0
    assert np.array_equal(rw[live, 0], rp[live, 0])
    assert np.all(np_ <= nw)
    assert (np_ < nw).any() and (np_[live] == nw[live]).any()
    for t in np.nonzero(live)[0]:
        a, n = int(rp[t, 0]), int(np_[t])
        assert np.array_equal(vp[a:a + n], vw[a:a + n]), t


@pytest.mark.parametrize("cap", [0, 192])
def test_slices_backward_equals_whole_lists(cap):
    """Stored blend order (cap 192) and pure replay (cap 0) after a sliced forward: the same
    gradients as after a whole-list forward (up to the order of the float atomics)."""
    sc, cams = _scene()
    g = R.scene_to_device(sc)
    res = {}
    for k in (0, 1):
        prm = I.RenderParams(slice_k=k, blend_cap=cap)
        r = R.Renderer(sc.n, cams, prm, backward=True)
        rgb, depth, _ = r.forward(g)
        gen = torch.Generator(device="cuda").manual_seed(11)
        d_rgb = torch.randn(rgb.shape, device="cuda", generator=gen)
        d_z = torch.randn(depth.shape, device="cuda", generator=gen)
        grads = {f: torch.zeros_like(g[f]) for f in R.FIELDS}
        r.backward(g, d_rgb, d_z, grads)
        torch.cuda.synchronize()
        st = r.status()
        assert st.error_bits == 0, (k, st.error_bits)
        if k:
            assert st.redo_warps > 0
        res[k] = {f: v.cpu().numpy().astype(np.float64) for f, v in grads.items()}
        res[k]["rgb"] = rgb.cpu().numpy()
    assert np.array_equal(res[0]["rgb"], res[1]["rgb"])
    for f in R.FIELDS:
        a, b = res[1][f], res[0][f]
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), f


def test_slices_in_a_multi_scene_batch():
    sc1, cams = _scene()
    sc2 = I.cluster_scene(20000, 81, nclusters=4, centre_range=1.0, scale_range=(0.003, 0.2))
    outs = {}
    for k in (0, 1, 512):
        r = R.Renderer([sc1.n, sc2.n], [cams[0], cams[1], cams[2], cams[0]], I.RenderParams(slice_k=k),
                       views_per_scene=[3, 1], debug=True)
        rgb, depth, tf = r.forward([R.scene_to_device(sc1), R.scene_to_device(sc2)])
        nb, h = r.debug_stats()
        torch.cuda.synchronize()
        assert r.status().error_bits == 0
        outs[k] = [x.cpu().numpy() for x in (rgb, depth, tf, nb, h)]
    for k in (1, 512):
        for a, b in zip(outs[k], outs[0]):
            assert np.array_equal(a, b), k


def test_slices_under_graph_replay():
    """The second pass is launched unconditionally (its kernels return at once when nothing is
    queued), so a captured forward replays it; graph and eager agree bit for bit."""
    sc, cams = _scene()
    g = R.scene_to_device(sc)
    r = R.Renderer(sc.n, cams, I.RenderParams(slice_k=1))
    eager = [x.clone() for x in r.forward(g)]
    torch.cuda.synchronize()
    out = tuple(torch.full_like(x, -1.0) for x in eager)
    graph = r.capture(g, out)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert r.status().error_bits == 0 and r.status().redo_warps > 0
    for a, b in zip(eager, out):
        assert torch.equal(a, b)


def test_slices_keep_the_blend_traces():
    """The per-pixel traces of the first blended ids: a warp rendered again over its whole list
    rewrites its trace from the start, so nothing of the first pass's partial trace remains."""
    sc, cams = _scene()
    g = R.scene_to_device(sc)
    out = {}
    for k in (0, 1):
        r = R.Renderer(sc.n, cams, I.RenderParams(slice_k=k), trace=True)
        r.forward(g)
        torch.cuda.synchronize()
        assert r.status().error_bits == 0
        out[k] = r.debug_trace().cpu().numpy()
    assert (out[0] >= 0).any() and np.array_equal(out[1], out[0])
