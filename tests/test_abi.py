"""C-ABI checks that need no GPU: the library loads, exports every function include/stp.h
declares, sizes workspaces and rejects bad arguments on the host before any launch."""
import ctypes as C
import dataclasses
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
    assert lib.stp_version() == 0x000300


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
    # stored blend order: blend_cap ids for each of the 256 lanes of every tile, one count a pixel
    assert d["blend_count"] >= d["blend_ids"] + 256 * 256 * prm.blend_cap * 4
    assert d["replay_warps"] >= d["blend_count"] + 256 * 256 * 4
    assert d["total"] >= d["replay_warps"] + 256 * 8 * 4
    size = lib.stp_workspace_size(sc.n, C.cast(N.cameras_array(cams), C.c_void_p), 1, C.byref(p))
    assert size == d["total"]
    # no stored order without the backward flag, with blend_cap 0 or outside the HIER order
    for flags, cap, mode in ((0, 192, I.MODE_HIER), (N.FLAG_BACKWARD, 0, I.MODE_HIER),
                             (N.FLAG_BACKWARD, 192, I.MODE_GLOBAL)):
        q = N.params_struct(prm, flags)
        q.blend_cap, q.mode = cap, mode
        Lq = N.layout(sc.n, cams, q)
        assert Lq.blend_ids == 0 and Lq.blend_count == 0 and Lq.replay_warps == 0
    # depth slices: the prefix lengths, second-pass flags and warp queue exist only for the HIER
    # order over the partitioned sort with slice_k > 0, one word per tile (eight for the queue)
    assert prm.slice_k > 0 and d["tile_front"] and d["tile_redo"] and d["redo_warps"]
    assert d["tile_redo"] >= d["tile_front"] + 256 * 4 and d["redo_warps"] >= d["tile_redo"] + 256 * 4
    assert d["total"] >= d["redo_warps"] + 256 * 8 * 4
    for flags, k, mode in ((0, 0, I.MODE_HIER), (N.FLAG_GLOBAL_SORT, 2048, I.MODE_HIER),
                           (0, 2048, I.MODE_FULL), (0, 2048, I.MODE_WINDOW)):
        q = N.params_struct(prm, flags)
        q.slice_k, q.mode = k, mode
        Lq = N.layout(sc.n, cams, q)
        assert Lq.tile_front == 0 and Lq.tile_redo == 0 and Lq.redo_warps == 0, (flags, k, mode)
    # several views of mixed sizes: tiles and pixels add up, key bits grow with the tile count
    cams4 = I.orbit_cameras(5, 15.0, 2.0, I.C4_SIZES, 50.0)
    L4 = N.layout(1000, cams4, N.params_struct(I.RenderParams()))
    assert L4.total_tiles == sum(c.num_tiles for c in cams4)
    assert L4.total_pixels == sum(c.num_pixels for c in cams4)


@pytest.mark.parametrize("field,value,code", [
    ("tail", 48, N.STP_ERR_ARG), ("tail", 80, N.STP_ERR_ARG), ("mid", 6, N.STP_ERR_ARG),
    ("mid", 10, N.STP_ERR_ARG), ("head", 5, N.STP_ERR_NOT_SUPPORTED), ("lb_threshold", 0, N.STP_ERR_ARG),
    ("eps_o", 0.0, N.STP_ERR_ARG), ("mode", 7, N.STP_ERR_ARG), ("mode", -1, N.STP_ERR_ARG), ("max_entries", -1, N.STP_ERR_ARG),
    ("blend_cap", -1, N.STP_ERR_ARG), ("blend_cap", 4097, N.STP_ERR_ARG), ("slice_k", -1, N.STP_ERR_ARG),
    ("full_max_passes", -1, N.STP_ERR_ARG),
    ("head", 0, N.STP_ERR_NOT_SUPPORTED), ("head", 17, N.STP_ERR_NOT_SUPPORTED), ("tail", 288, N.STP_ERR_ARG),
    ("mid", 24, N.STP_ERR_ARG), ("eps_o", 1.0, N.STP_ERR_ARG), ("eps_o", float("nan"), N.STP_ERR_ARG),
    ("t_min", 1.0, N.STP_ERR_ARG), ("t_min", -0.1, N.STP_ERR_ARG), ("alpha_max", 1.0, N.STP_ERR_ARG),
    ("alpha_max", 1.0 / 512, N.STP_ERR_ARG), ("inv_scale_max", 0.0, N.STP_ERR_ARG),
    ("dilation", -0.1, N.STP_ERR_ARG), ("frustum_clamp", 0.0, N.STP_ERR_ARG), ("znear", 0.0, N.STP_ERR_ARG),
    ("max_entries", 0xFFFFFFFF, N.STP_ERR_ARG),
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


def _layout_rc(lib, n, cams, p):
    L = N.Layout()
    return lib.stp_workspace_layout_get(n, C.cast(N.cameras_array(cams), C.c_void_p), len(cams), C.byref(p),
                                        C.byref(L))


def test_window_k_is_checked_only_for_the_window_order(lib):
    sc, cams, prm = I.plain_forward_workload()
    p = N.params_struct(prm)
    p.window_k = 5
    assert _layout_rc(lib, sc.n, cams, p) == N.STP_OK
    p.mode = I.MODE_WINDOW
    assert _layout_rc(lib, sc.n, cams, p) == N.STP_ERR_NOT_SUPPORTED
    p.window_k = 8
    assert _layout_rc(lib, sc.n, cams, p) == N.STP_OK


@pytest.mark.parametrize("field,value", [("width", 0), ("height", 0), ("width", 16385), ("height", 16385),
                                         ("fx", 0.0), ("fy", -1.0), ("cx", float("inf")), ("cy", float("nan"))])
def test_bad_cameras_rejected_on_host(lib, field, value):
    sc, cams, prm = I.plain_forward_workload()
    p = N.params_struct(prm)
    cams = cams + [dataclasses.replace(cams[0], **{field: value})]
    assert _layout_rc(lib, sc.n, cams, p) == N.STP_ERR_ARG
    assert "view 1" in N.last_error()
    ok = [dataclasses.replace(cams[0], width=16384, height=1)]
    assert _layout_rc(lib, sc.n, ok, p) == N.STP_OK


def test_view_count_range(lib):
    sc, cams, prm = I.plain_forward_workload()
    p = N.params_struct(prm)
    assert _layout_rc(lib, sc.n, cams * 64, p) == N.STP_OK
    assert _layout_rc(lib, sc.n, cams * 65, p) == N.STP_ERR_ARG
    L = N.Layout()
    rc = lib.stp_workspace_layout_get(sc.n, C.cast(N.cameras_array(cams), C.c_void_p), 0, C.byref(p), C.byref(L))
    assert rc == N.STP_ERR_ARG


def test_window_sizes_are_the_compiled_ones(lib):
    sc, cams, prm = I.plain_forward_workload()
    L = N.Layout()
    for k, code in ((3, N.STP_ERR_NOT_SUPPORTED), (8, N.STP_OK), (32, N.STP_ERR_NOT_SUPPORTED)):
        p = N.params_struct(prm)
        p.mode, p.window_k = I.MODE_WINDOW, k
        rc = lib.stp_workspace_layout_get(sc.n, C.cast(N.cameras_array(cams), C.c_void_p), 1, C.byref(p),
                                          C.byref(L))
        assert rc == code, k


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


def test_sort_entry_points_reject_bad_arguments_on_host(lib):
    """Every case fails a host check before any device call (the dummy addresses are never
    dereferenced)."""
    fake = [C.c_void_p(256 * (k + 1)) for k in range(4)]
    tmp = C.c_void_p(4096)
    ok_temp = lib.stp_sort_temp_bytes(10)
    cases = [
        (-1, 40, fake, tmp, ok_temp, "n out of range"),
        (0xFFFFFFFF, 40, fake, tmp, ok_temp, "n out of range"),
        (10, 0, fake, tmp, ok_temp, "key_bits"),
        (10, 65, fake, tmp, ok_temp, "key_bits"),
        (10, 40, [None] + fake[1:], tmp, ok_temp, "null array"),
        (10, 40, fake[:3] + [None], tmp, ok_temp, "null array"),
        (10, 40, fake, None, ok_temp, "temp"),
        (10, 40, fake, tmp, ok_temp - 1, "temp"),
    ]
    for n, bits, arrs, temp, tb, msg in cases:
        assert lib.stp_sort_pairs(*arrs, n, None, bits, temp, tb, None) == N.STP_ERR_ARG, (n, bits, msg)
        assert msg in N.last_error()
    assert lib.stp_sort_temp_bytes(-1) == 0
    assert lib.stp_sort_temp_bytes(2_000_000) > lib.stp_sort_temp_bytes(1000)
    for n, bits, arrs, msg in [(-1, 40, fake, "exceeds"), ((1 << 20) + 1, 40, fake, "exceeds"), (10, 0, fake, "key_bits"),
                               (10, 65, fake, "key_bits"), (10, 40, [None] + fake[1:], "null array")]:
        assert lib.stp_sort_pairs_noalloc(*arrs, n, None, bits, None) == N.STP_ERR_ARG, (n, bits, msg)
        assert msg in N.last_error()


def test_batched_layout_adds_up_over_scenes(lib):
    cams = I.orbit_cameras(6, 15.0, 2.0, I.C4_SIZES, 50.0)
    p = N.params_struct(I.RenderParams(), N.FLAG_BACKWARD, max_entries=1 << 20)
    ns, vps = [1000, 0, 70001], [2, 1, 3]
    L = N.layout(ns, cams, p, vps)
    # one scene through the batched call equals the single-scene layout
    L1 = N.layout(5000, cams, p, [6])
    assert L1.as_dict() == N.layout(5000, cams, p).as_dict()
    m = sum(n * v for n, v in zip(ns, vps))
    assert L.total_tiles == sum(c.num_tiles for c in cams)
    assert L.total_pixels == sum(c.num_pixels for c in cams)
    assert L.view_z + m * 4 <= L.rect                  # one camera-space depth per (view, Gaussian)
    assert L.grad_geom and L.total >= L.grad_geom + m * 24 * 4
    arr_n = (C.c_int64 * 3)(*ns)
    arr_v = (C.c_int32 * 3)(*vps)
    size = lib.stp_workspace_size_batched(C.cast(arr_n, C.c_void_p), C.cast(arr_v, C.c_void_p), 3,
                                          C.cast(N.cameras_array(cams), C.c_void_p), 6, C.byref(p))
    assert size == L.total


@pytest.mark.parametrize("ns,vps,nviews,msg", [
    ([10, 10], [3, 2], 6, "sum to"),
    ([10], [-1], 6, "negative"),
    ([-5], [6], 6, "out of range"),
    ([1] * 65, [0] * 64 + [6], 6, "nscenes"),
])
def test_batched_layout_rejects_bad_scene_tables(lib, ns, vps, nviews, msg):
    cams = I.orbit_cameras(nviews, 15.0, 2.0, I.C4_SIZES, 50.0)
    p = N.params_struct(I.RenderParams())
    arr_n = (C.c_int64 * len(ns))(*ns)
    arr_v = (C.c_int32 * len(vps))(*vps)
    out = N.Layout()
    rc = lib.stp_workspace_layout_batched(C.cast(arr_n, C.c_void_p), C.cast(arr_v, C.c_void_p), len(ns),
                                          C.cast(N.cameras_array(cams), C.c_void_p), nviews, C.byref(p),
                                          C.byref(out))
    assert rc == N.STP_ERR_ARG and msg in N.last_error()


def test_batched_render_checks_scene_pointers_before_launch(lib):
    cams = I.orbit_cameras(2, 15.0, 2.0, I.C4_SIZES, 50.0)
    p = N.params_struct(I.RenderParams())
    scenes = (N.Gaussians * 2)()
    scenes[0].n, scenes[0].sh_degree = 10, 0
    scenes[0].means = scenes[0].log_scales = scenes[0].quats = scenes[0].opacity_logits = scenes[0].sh = 256
    scenes[1].n, scenes[1].sh_degree = 10, 0          # null arrays in scene 1
    vps = (C.c_int32 * 2)(1, 1)
    rc = lib.stp_render_batched(C.cast(scenes, C.c_void_p), 2, C.cast(vps, C.c_void_p),
                                C.cast(N.cameras_array(cams), C.c_void_p), 2, C.byref(p), C.c_void_p(256),
                                1 << 40, C.c_void_p(256), C.c_void_p(256), None, None)
    assert rc == N.STP_ERR_ARG and "scene 1" in N.last_error()
    scenes[1].sh_degree = 4
    rc = lib.stp_render_batched(C.cast(scenes, C.c_void_p), 2, C.cast(vps, C.c_void_p),
                                C.cast(N.cameras_array(cams), C.c_void_p), 2, C.byref(p), C.c_void_p(256),
                                1 << 40, C.c_void_p(256), C.c_void_p(256), None, None)
    assert rc == N.STP_ERR_ARG and "sh_degree" in N.last_error()


def test_backward_before_forward_is_refused_on_the_host(lib):
    """The backward reads the forward's state from the workspace; the front end refuses it on
    a workspace no forward has filled (fresh, regrown, or after new image sizes) before any
    library call. A CPU workspace suffices: nothing is launched."""
    torch = pytest.importorskip("torch")
    from paper_2402_00525_gb300 import renderer as R
    sc, cams, prm = I.plain_forward_workload()
    r = R.Renderer(sc.n, cams, prm, device="cpu", backward=True)
    with pytest.raises(RuntimeError, match="forward"):
        r.backward({}, torch.zeros(1), None, {})
    r2 = R.Renderer(sc.n, cams, prm, device="cpu")
    with pytest.raises(RuntimeError, match="backward=True"):
        r2.backward({}, torch.zeros(1), None, {})


def test_binding_matches_the_header_layouts_and_constants(tmp_path):
    """The ctypes structs of the binding have the C header's size and field offsets (a plain C
    program built against include/stp.h prints them), and every constant the binding mirrors
    has the header's value."""
    import shutil
    import subprocess
    if not shutil.which("gcc"):
        pytest.skip("needs gcc")
    pairs = [(N.Gaussians, "stp_gaussians"), (N.GaussiansGrad, "stp_gaussians_grad"), (N.CameraS, "stp_camera"),
             (N.Params, "stp_params"), (N.RunStatus, "stp_run_status"), (N.Layout, "stp_workspace_layout")]
    consts = {"STP_OK": N.STP_OK, "STP_ERR_ARG": N.STP_ERR_ARG, "STP_ERR_CAPACITY": N.STP_ERR_CAPACITY,
              "STP_ERR_TIMEOUT": N.STP_ERR_TIMEOUT, "STP_ERR_CUDA": N.STP_ERR_CUDA,
              "STP_ERR_NOT_SUPPORTED": N.STP_ERR_NOT_SUPPORTED, "STP_ERR_INCONSISTENT": N.STP_ERR_INCONSISTENT,
              "STP_MODE_HIER": I.MODE_HIER, "STP_MODE_FULL": I.MODE_FULL, "STP_MODE_GLOBAL": I.MODE_GLOBAL,
              "STP_MODE_WINDOW": I.MODE_WINDOW, "STP_FLAG_HEAD_EVICT_FIRST": I.FLAG_HEAD_EVICT_FIRST,
              "STP_FLAG_LEVEL_CENTRE_RAYS": I.FLAG_LEVEL_CENTRE_RAYS, "STP_FLAG_TILE_CENTRE_KEY": I.FLAG_TILE_CENTRE_KEY,
              "STP_FLAG_VIEW_DEPTH_KEY": I.FLAG_VIEW_DEPTH_KEY, "STP_FLAG_NO_LOAD_BALANCE": I.FLAG_NO_LOAD_BALANCE,
              "STP_FLAG_DEBUG_STATS": N.FLAG_DEBUG_STATS, "STP_FLAG_BACKWARD": N.FLAG_BACKWARD,
              "STP_FLAG_DEBUG_TRACE": N.FLAG_DEBUG_TRACE, "STP_FLAG_GLOBAL_SORT": N.FLAG_GLOBAL_SORT,
              "STP_FLAG_NO_TILE_CULL": N.FLAG_NO_TILE_CULL, "STP_FLAG_NO_HIER_CULL": N.FLAG_NO_HIER_CULL,
              "STP_TRACE_LEN": N.TRACE_LEN, "STP_MAX_SCENES": N.MAX_SCENES, "STP_MAX_VIEWS": N.MAX_VIEWS,
              "STP_SORT_STATIC_MAX_N": N.SORT_STATIC_MAX_N, "STP_NUM_STAGES": N.NUM_STAGES}
    assert I.FLAG_GLOBAL_SORT == N.FLAG_GLOBAL_SORT and I.FLAG_NO_TILE_CULL == N.FLAG_NO_TILE_CULL
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "stp.h"', "int main(void) {"]
    expect = {}
    for cls, cname in pairs:
        lines.append('printf("%%s %%zu\\n", "%s", sizeof(%s));' % (cname, cname))
        expect[cname] = C.sizeof(cls)
        for f, _ in cls._fields_:
            key = "%s.%s" % (cname, f)
            lines.append('printf("%%s %%zu\\n", "%s", offsetof(%s, %s));' % (key, cname, f))
            expect[key] = getattr(cls, f).offset
    for k, v in consts.items():
        lines.append('printf("%%s %%lld\\n", "%s", (long long)(%s));' % (k, k))
        expect[k] = v
    lines += ["return 0;", "}"]
    src = tmp_path / "layouts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layouts"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                          text=True).stdout.splitlines())
    assert {k: int(v) for k, v in got.items()} == expect
