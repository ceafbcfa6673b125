"""The torch.autograd.Function path (Sec. 3.5 behind autograd): render() -> loss -> backward().

Gradients reach the leaf tensors through libstp's backward and are compared with the FP64
adjoint of the oracle at the parity bar (rel-L2 <= 1e-4, cosine >= 0.9999 per parameter block).
The upstream gradient is fixed by the loss, so the oracle is given the same loss weights: they
are zero on pixels the oracle marks undecided and, for the L1 term, on pixels whose oracle
colour lies within 1e-3 of the target (there the sign of rgb - target is not fixed by parity).
"""
import dataclasses

import numpy as np
import pytest
import torch

from paper_2402_00525_gb300 import _native as N
from paper_2402_00525_gb300 import inputs as I
from paper_2402_00525_gb300 import renderer as R

pytestmark = pytest.mark.gpu


def _leaves(g):
    return {k: (g[k].clone().requires_grad_(True) if k in R.FIELDS else g[k]) for k in g}


def _compare(grads, adj, label):
    for k in R.FIELDS:
        a = grads[k].detach().cpu().numpy().astype(np.float64).ravel()
        b = adj[k].ravel()
        if not b.any():              # a block the loss does not reach (SH under a depth loss)
            assert not a.any(), (label, k)
            continue
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
        print(label, k, "rel-L2 %.3g cos %.8f" % (rel, cos))
        assert rel <= 1e-4 and cos >= 0.9999, (label, k, rel, cos)


@pytest.mark.parametrize("cap", [0, 192])
def test_l1_and_depth_loss_through_autograd_matches_adjoint(oracle, cap):
    sc, target, cam, prm = I.fd_subcase()
    prm = dataclasses.replace(prm, blend_cap=cap)
    HW = cam.num_pixels
    tgt = oracle.render(target, cam, prm)["rgb"]
    rng = np.random.default_rng(17)
    wz = rng.normal(size=(cam.height, cam.width)) / HW * 0.1
    with oracle.OracleRun(sc, cam, prm, record=True) as r:
        ora = r.render()
        dec = ora["decided"]
        assert dec.mean() >= 0.99
        diff = ora["rgb"] - tgt
        m = dec[..., None] & (np.abs(diff) > 1e-3)
        w_rgb = np.where(m, np.sign(diff), 0.0) / (3 * HW)
        w_z = np.where(dec, wz, 0.0)
        adj = r.backward(w_rgb, w_z)
    g = _leaves(R.scene_to_device(sc))
    rr = R.Renderer(sc.n, [cam], prm, backward=True)
    rgb, depth = R.render(rr, g)
    mask = torch.from_numpy(m.reshape(-1, 3)).cuda()
    tg = torch.from_numpy(tgt.reshape(-1, 3).astype(np.float32)).cuda()
    wzt = torch.from_numpy(w_z.reshape(-1).astype(np.float32)).cuda()
    loss = (mask * (rgb - tg).abs()).sum() / (3 * HW) + (wzt * depth).sum()
    loss.backward()
    torch.cuda.synchronize()
    # the GPU image agrees in sign with the oracle's wherever the L1 weight is non-zero
    s_gpu = torch.sign(rgb - tg).detach().cpu().numpy().reshape(cam.height, cam.width, 3)
    assert np.array_equal(s_gpu[m], np.sign(diff)[m])
    _compare({k: g[k].grad for k in R.FIELDS}, adj, "L1+depth cap %d" % cap)


def test_depth_only_loss_through_autograd_matches_adjoint(oracle):
    """Only depth reaches the loss, so autograd hands the backward d_rgb = None."""
    sc, _, cam, prm = I.fd_subcase()
    rng = np.random.default_rng(23)
    with oracle.OracleRun(sc, cam, prm, record=True) as r:
        ora = r.render()
        w_z = np.where(ora["decided"], rng.normal(size=(cam.height, cam.width)), 0.0) / cam.num_pixels
        adj = r.backward(np.zeros((cam.height, cam.width, 3)), w_z)
    g = _leaves(R.scene_to_device(sc))
    rr = R.Renderer(sc.n, [cam], prm, backward=True)
    _, depth = R.render(rr, g)
    (torch.from_numpy(w_z.reshape(-1).astype(np.float32)).cuda() * depth).sum().backward()
    torch.cuda.synchronize()
    _compare({k: g[k].grad for k in R.FIELDS}, adj, "depth only")


def test_backward_after_another_forward_raises():
    """Two forwards on one renderer, then the backward of the first: its blend order is gone
    from the workspace, so the backward refuses; the second output still differentiates."""
    sc, _, cam, prm = I.fd_subcase()
    g = _leaves(R.scene_to_device(sc))
    rr = R.Renderer(sc.n, [cam], prm, backward=True)
    rgb1, _ = R.render(rr, g)
    rgb2, _ = R.render(rr, g)
    with pytest.raises(R.StaleForwardError):
        rgb1.sum().backward()
    for k in R.FIELDS:
        g[k].grad = None
    rgb2.sum().backward()
    assert all(torch.isfinite(g[k].grad).all() for k in R.FIELDS)
    assert sum(float(g[k].grad.abs().sum()) for k in R.FIELDS) > 0


def test_backward_reports_a_changed_workspace():
    """The stored-order backward recomputes every alpha and must end on the forward's final T
    bit for bit. Halving the opacities in the workspace's records between forward and backward
    breaks that; the autograd backward reads the status block and raises STP_ERR_INCONSISTENT."""
    sc, _, cam, prm = I.fd_subcase()
    g = _leaves(R.scene_to_device(sc))
    rr = R.Renderer(sc.n, [cam], prm, backward=True)
    rgb, _ = R.render(rr, g)
    geom = rr.records()[0]
    with torch.no_grad():
        geom[..., 8] *= 0.5                     # record float 8 is the opacity
    with pytest.raises(N.StpError) as e:
        rgb.sum().backward()
    assert e.value.code == N.STP_ERR_INCONSISTENT


def test_forward_raises_when_capacity_cannot_be_reached():
    """The forward grows the workspace to the entry count it learns times `headroom`; with a
    headroom below one it never fits, and after three attempts it raises instead of returning
    a truncated image."""
    sc, cams, prm = I.plain_forward_workload()
    g = R.scene_to_device(sc)
    rr = R.Renderer(sc.n, cams, prm, capacity=2048, headroom=0.5)
    with pytest.raises(N.CapacityError):
        rr.forward(g)
