"""Host logic of the Python front end (no GPU): the capacity retry loop of Renderer.forward.

The library's sizing calls are the real host-only ones; the render call, the status read and
the stream are stand-ins, so the loop's decisions (grow the workspace, retry, give up loudly)
are checked without a device."""
import types

import pytest

from paper_2402_00525_gb300 import _native as N
from paper_2402_00525_gb300 import inputs as I
from paper_2402_00525_gb300 import renderer as R


class _Lib:
    """Delegates to the real library except for the render call, which it counts."""

    def __init__(self, real):
        self._real = real
        self.renders = 0

    def __getattr__(self, name):
        return getattr(self._real, name)

    def stp_render(self, *args):
        self.renders += 1
        return N.STP_OK


@pytest.fixture
def rig(monkeypatch):
    real = N.lib()
    fake = _Lib(real)
    cams = I.orbit_cameras(2, 3.0, 0.5, [(64, 48)], 50.0)
    r = R.Renderer(1000, cams, I.RenderParams(), device="cpu", capacity=2048, backward=True)
    monkeypatch.setattr(N, "lib", lambda: fake)
    monkeypatch.setattr(R, "gaussians_struct", lambda g: N.Gaussians(n=1000, sh_degree=0))
    statuses = []

    def read_status(ws, stream, raise_on_error=True):
        return statuses.pop(0)
    monkeypatch.setattr(N, "read_status", read_status)
    stream = types.SimpleNamespace(cuda_stream=0)
    return r, fake, statuses, stream


def _st(bits, entries):
    return types.SimpleNamespace(error_bits=bits, num_entries=entries)


def test_overflow_grows_the_workspace_and_retries(rig):
    r, fake, statuses, stream = rig
    cap0 = r.capacity
    need = 10 * cap0
    statuses += [_st(1, need), _st(0, need)]
    gen = r.generation
    r.forward({}, stream=stream)
    assert fake.renders == 2 and not statuses
    assert r.capacity >= int(need * r.headroom) + 1024 > cap0
    assert r.workspace_bytes == r.ws.numel() and r._fwd_ready and r.generation == gen + 1
    assert r.last_status.num_entries == need


def test_overflow_on_every_attempt_raises_and_leaves_no_forward(rig):
    r, fake, statuses, stream = rig
    statuses += [_st(1, 5000), _st(1, 50_000), _st(1, 500_000)]
    gen = r.generation
    with pytest.raises(N.CapacityError, match="three attempts"):
        r.forward({}, stream=stream)
    assert fake.renders == 3 and not statuses
    # nothing truncated is handed on: no forward state, the generation unchanged
    assert not r._fwd_ready and r.generation == gen
    with pytest.raises(RuntimeError, match="needs a forward"):
        R.Renderer.backward(r, {}, None, None, {}, stream=stream)


def test_unchecked_forward_reads_no_status(rig):
    r, fake, statuses, stream = rig
    r.forward({}, check=False, stream=stream)         # an empty status list would raise if read
    assert fake.renders == 1 and r._fwd_ready
