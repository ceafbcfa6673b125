"""stp_sort_pairs_noalloc: the radix sort for callers that cannot allocate device memory
(stream-capture recorders, plugins inside a framework that owns the memory pool, loops that
must not allocate after start-up). It uses a fixed scratch array inside the library instead
of a caller buffer. Checked through the C ABI against stp_sort_pairs on two calls in a row;
both are integer sorts, so the results must be identical.

Kept in a file of its own, collected last, so that a run stopping at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2402_00525_gb300 import _native as N  # noqa: E402


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _reference_sort(lib, kd, vd, n, bits, stream):
    ko, vo = torch.empty_like(kd), torch.empty_like(vd)
    tb = lib.stp_sort_temp_bytes(n)
    tmp = torch.empty(max(tb, 1), dtype=torch.uint8, device="cuda")
    N.check(lib.stp_sort_pairs(_ptr(kd), _ptr(vd), _ptr(ko), _ptr(vo), n, None, bits, _ptr(tmp), tb, stream))
    return ko, vo


def test_sort_without_allocation_matches_sort_with_workspace():
    from paper_2402_00525_gb300 import build
    build.build()
    lib = N.lib()
    rng = np.random.default_rng(2024)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two calls in a row: the second must not see anything left from the first
    for n, bits in [(N.SORT_STATIC_MAX_N, 45), (300_001, 41)]:
        keys = rng.integers(0, 1 << min(bits, 62), n, dtype=np.int64).astype(np.uint64)
        keys[rng.random(n) < 0.25] = keys[1]              # many equal keys: stability matters
        vals = rng.permutation(n).astype(np.uint32)
        kd = torch.from_numpy(keys.view(np.int64)).cuda()
        vd = torch.from_numpy(vals.view(np.int32)).cuda()
        ko_ref, vo_ref = _reference_sort(lib, kd, vd, n, bits, stream)
        ko, vo = torch.empty_like(kd), torch.empty_like(vd)
        N.check(lib.stp_sort_pairs_noalloc(_ptr(kd), _ptr(vd), _ptr(ko), _ptr(vo), n, None, bits, stream))
        torch.cuda.synchronize()
        assert torch.equal(ko, ko_ref) and torch.equal(vo, vo_ref)
        order = np.argsort(keys & np.uint64((1 << bits) - 1), kind="stable")
        assert np.array_equal(vo.cpu().numpy().view(np.uint32), vals[order])
        assert np.array_equal(kd.cpu().numpy().view(np.uint64), keys)     # input preserved


def test_sort_without_allocation_rejects_oversized_input():
    lib = N.lib()
    rc = lib.stp_sort_pairs_noalloc(None, None, None, None, N.SORT_STATIC_MAX_N + 1, None, 32, None)
    assert rc == N.STP_ERR_ARG
    assert "exceeds the fixed scratch" in N.last_error()
