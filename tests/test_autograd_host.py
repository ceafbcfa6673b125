"""Host logic of the autograd path (no GPU): render() with a stand-in renderer, so that what is
checked is the torch.autograd.Function wiring, not the kernels: which gradient reaches which
input, the zero colour adjoint of a depth-only loss, the stale-forward refusal and the status
check after the backward."""
import types

import pytest
import torch

from paper_2402_00525_gb300 import _native as N
from paper_2402_00525_gb300 import renderer as R


class _FakeRenderer:
    flags = N.FLAG_BACKWARD

    def __init__(self, pixels):
        self.total_pixels = pixels
        self.device = torch.device("cpu")
        self.generation = 0
        self.ws = None
        self.seen = []

    def forward(self, g):
        self.generation += 1
        P = self.total_pixels
        return torch.full((P, 3), 0.5), torch.full((P,), 2.0), torch.ones(P)

    def backward(self, g, d_rgb, d_depth, grads):
        self.seen.append((d_rgb.clone(), None if d_depth is None else d_depth.clone()))
        s = float(d_rgb.sum()) + (0.0 if d_depth is None else 10.0 * float(d_depth.sum()))
        for i, k in enumerate(R.FIELDS):          # a distinct value per input field
            grads[k] += (i + 1) * s


def _scene(n=5, k=16):
    g = dict(means=torch.randn(n, 3), log_scales=torch.randn(n, 3), quats=torch.randn(n, 4),
             opacity_logits=torch.randn(n), sh=torch.randn(n, k, 3), sh_degree=3)
    for f in R.FIELDS:
        g[f].requires_grad_(True)
    return g


def test_gradients_reach_their_inputs():
    r, g = _FakeRenderer(6), _scene()
    rgb, depth = R.render(r, g, check_status=False)
    assert rgb.shape == (6, 3) and depth.shape == (6,)
    (rgb.sum() + 0.5 * depth.sum()).backward()
    d_rgb, d_depth = r.seen[0]
    assert torch.equal(d_rgb, torch.ones(6, 3)) and torch.equal(d_depth, torch.full((6,), 0.5))
    s = 18.0 + 10.0 * 3.0
    for i, k in enumerate(R.FIELDS):
        assert g[k].grad.shape == g[k].shape
        assert torch.all(g[k].grad == (i + 1) * s), k


def test_depth_only_loss_passes_a_zero_colour_adjoint():
    r, g = _FakeRenderer(4), _scene()
    _, depth = R.render(r, g, check_status=False)
    depth.sum().backward()
    d_rgb, d_depth = r.seen[0]
    assert torch.equal(d_rgb, torch.zeros(4, 3)) and torch.equal(d_depth, torch.ones(4))


def test_backward_after_another_forward_raises():
    r, g = _FakeRenderer(4), _scene()
    rgb1, _ = R.render(r, g, check_status=False)
    rgb2, _ = R.render(r, g, check_status=False)
    with pytest.raises(R.StaleForwardError, match="1 more forward"):
        rgb1.sum().backward()
    rgb2.sum().backward()                         # the latest output is still differentiable
    assert len(r.seen) == 1


def test_status_error_after_the_backward_surfaces(monkeypatch):
    monkeypatch.setattr(torch.cuda, "current_stream", lambda device=None: types.SimpleNamespace(cuda_stream=0))
    calls = []

    def read_status(ws, stream, raise_on_error=True):
        calls.append(raise_on_error)
        raise N.StpError(N.STP_ERR_INCONSISTENT, "blend sequence differs")
    monkeypatch.setattr(N, "read_status", read_status)
    r, g = _FakeRenderer(4), _scene()
    rgb, _ = R.render(r, g)
    with pytest.raises(N.StpError, match="blend sequence"):
        rgb.sum().backward()
    assert calls == [True]


def test_render_needs_a_backward_renderer():
    r = _FakeRenderer(4)
    r.flags = 0
    with pytest.raises(RuntimeError, match="backward=True"):
        R.render(r, _scene())
