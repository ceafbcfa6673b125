"""C-ABI checks that need no GPU: the library loads, exports every function include/stp.h
declares, sizes workspaces and rejects bad arguments on the host before any launch."""
import ctypes as C
import os
import re

import pytest

from paper_2402_00525_gb300 import _native as N
from paper_2402_00525_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_00525_gb300 import build
    build.build()
    return N.lib()


def _declared_functions():
    txt = open(os.path.join(ROOT, "include", "stp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(stp_[a-z_]+)\s*\(", txt)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert len(declared) >= 9
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(N.EXPORTS) == declared
    assert lib.stp_version() == 0x000100


def test_workspace_layout_is_consistent(lib):
    sc, cams, prm = I.plain_forward_workload()
    p = N.params_struct(prm, N.FLAG_DEBUG_STATS | N.FLAG_BACKWARD, max_entries=123456)
    L = N.layout(sc.n, cams, p)
    d = L.as_dict()
    assert d["capacity"] == 123456
    assert d["total_tiles"] == 256 and d["total_pixels"] == 256 * 256
    assert d["key_bits"] == 32 + 9          # 256 tiles need 9 bits (all-ones reserved)
    offs = sorted((v, k) for k, v in d.items() if k in N._LAYOUT_SIZE_FIELDS and k != "total" and v)
    assert all(v % 256 == 0 for v, _ in offs)
    assert d["total"] > d["grad_geom"] >= d["dbg_hash"] > d["dbg_nblend"]
    assert d["sorted_keys"] in (d["keys"], d["keys_alt"])
    size = lib.stp_workspace_size(sc.n, C.cast(N.cameras_array(cams), C.c_void_p), 1, C.byref(p))
    assert size == d["total"]
    # several views of mixed sizes: tiles and pixels add up, key bits grow with the tile count
    cams4 = I.orbit_cameras(5, 15.0, 2.0, I.C4_SIZES, 50.0)
    L4 = N.layout(1000, cams4, N.params_struct(I.RenderParams()))
    assert L4.total_tiles == sum(c.num_tiles for c in cams4)
    assert L4.total_pixels == sum(c.num_pixels for c in cams4)


@pytest.mark.parametrize("field,value,code", [
    ("tail", 48, N.STP_ERR_ARG), ("tail", 80, N.STP_ERR_ARG), ("mid", 6, N.STP_ERR_ARG),
    ("mid", 10, N.STP_ERR_ARG), ("head", 5, N.STP_ERR_NOT_SUPPORTED), ("lb_threshold", 0, N.STP_ERR_ARG),
    ("eps_o", 0.0, N.STP_ERR_ARG), ("mode", 7, N.STP_ERR_NOT_SUPPORTED), ("max_entries", -1, N.STP_ERR_ARG),
])
def test_bad_parameters_rejected_on_host(lib, field, value, code):
    sc, cams, prm = I.plain_forward_workload()
    p = N.params_struct(prm)
    setattr(p, field, value)
    L = N.Layout()
    rc = lib.stp_workspace_layout_get(sc.n, C.cast(N.cameras_array(cams), C.c_void_p), 1, C.byref(p),
                                      C.byref(L))
    assert rc == code
    assert N.last_error()


def test_render_rejects_bad_arguments_before_launch(lib):
    sc, cams, prm = I.plain_forward_workload()
    p = N.params_struct(prm)
    g = N.Gaussians()
    g.n = sc.n
    g.sh_degree = 0
    arr = N.cameras_array(cams)
    # null Gaussian arrays, then too-small workspace: both are host-side errors (no CUDA call)
    rc = lib.stp_render(C.byref(g), C.cast(arr, C.c_void_p), 1, C.byref(p), None, 0, None, None, None, None)
    assert rc == N.STP_ERR_ARG and "null" in N.last_error()
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        setattr(g, k, 256)
    rc = lib.stp_render(C.byref(g), C.cast(arr, C.c_void_p), 1, C.byref(p), None, 0, None, None, None, None)
    assert rc == N.STP_ERR_ARG and "workspace" in N.last_error()
    bad = N.cameras_array([I.look_at((0, 0, -3), (0, 0, 0), (0, 1, 0), 0, 64, 60.0)])
    rc = lib.stp_render(C.byref(g), C.cast(bad, C.c_void_p), 1, C.byref(p), None, 0, None, None, None, None)
    assert rc == N.STP_ERR_ARG
    # backward without the backward reservation flag
    rc = lib.stp_render_backward(C.byref(g), C.cast(arr, C.c_void_p), 1, C.byref(p), None, 0, None, None,
                                 None, None)
    assert rc == N.STP_ERR_ARG and "flag 64" in N.last_error()
    # sort primitive argument checks
    assert lib.stp_sort_pairs(None, None, None, None, 10, None, 0, None, 0, None) == N.STP_ERR_ARG
    assert lib.stp_sort_pairs(None, None, None, None, 10, None, 40, None, 0, None) == N.STP_ERR_ARG
    assert lib.stp_sort_temp_bytes(1000) > 12000
