"""Failure handling on the GPU path, made on the host: invalid inputs and a bounded loop that
runs out. Nothing here faults or hangs the device; every condition is reported through the
workspace's status block.

  * Invalid Gaussians (non-finite parameters, a zero-length quaternion) are dropped and
    counted once per scene, exactly as the oracle drops and counts them.
  * The FULL comparison order peels a tile's list in passes; a caller-set bound on the passes
    that runs out ends the tile, sets error bit 4 and surfaces as STP_ERR_TIMEOUT.
"""
import dataclasses

import numpy as np
import pytest
import torch

from gpu_helpers import compare_view, gpu_render
from test_oracle_composite import invalid_variant
from paper_2402_00525_gb300 import _native as N
from paper_2402_00525_gb300 import inputs as I
from paper_2402_00525_gb300 import renderer as R

pytestmark = pytest.mark.gpu


def _case():
    sc = I.uniform_scene(160, 93, scale_range=(0.02, 0.12), sh_degree=2)
    cams = [I.look_at((0.2, 0.1, -3), (0, 0, 0), (0, 1, 0), 64, 48, 60.0),
            I.look_at((-0.4, 0.2, -2.8), (0, 0, 0), (0, 1, 0), 80, 40, 55.0)]
    return sc, cams


def test_invalid_gaussians_dropped_and_counted_like_the_oracle(oracle):
    sc, cams = _case()
    prm = I.RenderParams()
    s1, s2, bad = invalid_variant(sc)
    a = gpu_render(s1, cams, prm)
    b = gpu_render(s2, cams, prm)
    st = a["renderer"].status()
    assert st.error_bits == 0
    assert st.invalid_gaussians == len(bad)               # once per scene, not per view
    assert b["renderer"].status().invalid_gaussians == 0
    for k in ("rgb", "depth", "tfinal", "nblend", "hash"):
        for v in range(len(cams)):
            assert np.array_equal(a[k][v], b[k][v]), (k, v)
    for v, cam in enumerate(cams):
        with oracle.OracleRun(s1, cam, prm) as r:
            assert r.num_invalid == len(bad)
            compare_view(a, v, r.render(), label="invalid inputs, view %d" % v)


def test_invalid_gaussians_receive_zero_gradient():
    sc, cams = _case()
    prm = I.RenderParams()
    s1, s2, bad = invalid_variant(sc)
    out = {}
    for name, s in (("invalid", s1), ("invisible", s2)):
        g = R.scene_to_device(s)
        r = R.Renderer(s.n, cams, prm, backward=True)
        rgb, depth, _ = r.forward(g)
        grads = {k: torch.zeros_like(g[k]) for k in R.FIELDS}
        gen = torch.Generator(device="cuda").manual_seed(3)
        r.backward(g, torch.randn(rgb.shape, device="cuda", generator=gen),
                   torch.randn(depth.shape, device="cuda", generator=gen), grads)
        torch.cuda.synchronize()
        assert r.status().error_bits == 0
        out[name] = {k: v.cpu().numpy() for k, v in grads.items()}
    keep = np.setdiff1d(np.arange(sc.n), bad)
    for k in R.FIELDS:
        assert np.all(np.isfinite(out["invalid"][k])), k
        assert np.all(out["invalid"][k][bad] == 0), k
        # the same blends; only the order of the float reductions differs between the runs
        a, b = out["invalid"][k][keep].astype(np.float64), out["invisible"][k][keep].astype(np.float64)
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b), k


def test_invalid_gaussians_counted_per_scene_in_a_batch():
    sc, cams = _case()
    s1, s2, bad = invalid_variant(sc)
    gs = [R.scene_to_device(s1), R.scene_to_device(s2), R.scene_to_device(s1)]
    r = R.Renderer([sc.n] * 3, [cams[0], cams[1], cams[0], cams[1]], I.RenderParams(),
                   views_per_scene=[2, 1, 1])
    r.forward(gs)
    assert r.status().invalid_gaussians == 2 * len(bad)


def test_full_order_pass_bound_runs_out_and_reports_timeout():
    """FULL peels 16 entries per pass; a bound of one pass cannot finish the dense tiles of the
    4096-Gaussian view, so the render stops those tiles and reports STP_ERR_TIMEOUT. A bound
    large enough gives the image of the default bound."""
    sc, cams, prm = I.plain_forward_workload()
    full = dataclasses.replace(prm, mode=I.MODE_FULL)
    ref = gpu_render(sc, cams, full)
    assert ref["renderer"].status().error_bits == 0
    loose = gpu_render(sc, cams, dataclasses.replace(full, full_max_passes=100000))
    assert np.array_equal(loose["rgb"][0], ref["rgb"][0]) and np.array_equal(loose["hash"][0], ref["hash"][0])
    g = R.scene_to_device(sc)
    r = R.Renderer(sc.n, cams, dataclasses.replace(full, full_max_passes=1), debug=True)
    with pytest.raises(N.StpError) as e:
        r.forward(g)
    assert e.value.code == N.STP_ERR_TIMEOUT
    assert r.status().error_bits & 4
    # the pixels of tiles that needed more passes blended fewer Gaussians than the full order
    nb = r.debug_stats()[0].cpu().numpy()
    assert nb.sum() < ref["nblend"][0].sum()
