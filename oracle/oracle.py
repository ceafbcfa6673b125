"""ctypes front end of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg use this module. It
loads oracle/_build/libstp_oracle.so (built by oracle/build.py) and converts between numpy
arrays and the oracle's C structs. It never touches the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(_HERE)) if os.path.dirname(_HERE) not in sys.path else None

from paper_2402_00525_gb300.inputs import Camera, RenderParams, Scene  # noqa: E402

# counter indices of orc_render
COUNTERS = ["visible", "entries", "eval_subtile", "surv_subtile", "eval_quad", "surv_quad",
            "eval_pixel", "head_inserts", "blends", "candidate_tiles", "done_pixels"]

GAP_THR = 1e-6     # relative depth gap below which an ordering is not decided
CULL_THR = 1e-5    # relative distance of a cull / alpha / T test to its threshold


class _Cam(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32)]


class _Prm(C.Structure):
    _fields_ = [("tail", C.c_int32), ("mid", C.c_int32), ("head", C.c_int32),
                ("mode", C.c_int32), ("window_k", C.c_int32), ("flags", C.c_int32),
                ("sh_degree", C.c_int32), ("record_blends", C.c_int32),
                ("eps_o", C.c_double), ("t_min", C.c_double), ("alpha_max", C.c_double),
                ("inv_scale_max", C.c_double), ("dilation", C.c_double),
                ("frustum_clamp", C.c_double), ("znear", C.c_double), ("bg", C.c_double * 3),
                ("gap_thr", C.c_double), ("cull_thr", C.c_double)]


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                ("quats", C.c_void_p), ("logits", C.c_void_p), ("sh", C.c_void_p)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        from oracle import build as _b  # noqa
        # STP_ORACLE_LIB: load another build of the oracle (the tests that plant a mistake in
        # a copy of its source run the pins against that build)
        path = os.environ.get("STP_ORACLE_LIB") or _b.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        vp = C.c_void_p
        L.orc_t_opt.restype = C.c_double
        L.orc_t_opt.argtypes = [dp, dp, dp, dp]
        L.orc_alg1.argtypes = [dp, dp, dp, dp]
        L.orc_sigma_inv.argtypes = [dp, dp, C.c_double, dp]
        L.orc_sigma.argtypes = [dp, dp, dp]
        L.orc_sh_basis.argtypes = [dp, dp]
        L.orc_t_o.restype = C.c_double
        L.orc_t_o.argtypes = [C.c_double, C.c_double]
        L.orc_project.argtypes = [C.POINTER(_Cam), C.POINTER(_Prm), dp, dp, dp, dp, dp]
        L.orc_create.restype = vp
        L.orc_create.argtypes = [C.POINTER(_Scene), C.POINTER(_Cam), C.POINTER(_Prm), vp, C.c_int32]
        L.orc_destroy.argtypes = [vp]
        L.orc_num_entries.restype = C.c_int64
        L.orc_num_entries.argtypes = [vp]
        L.orc_num_invalid.restype = C.c_int64
        L.orc_num_invalid.argtypes = [vp]
        L.orc_get_preprocess.argtypes = [vp] + [vp] * 11
        L.orc_get_tile_lists.argtypes = [vp, vp, vp, vp]
        L.orc_render.argtypes = [vp] + [vp] * 9 + [C.c_int32, vp]
        L.orc_render_ex.argtypes = [vp] + [vp] * 9 + [C.c_int32, vp, vp, C.c_double]
        L.orc_backward.argtypes = [vp, C.POINTER(_Scene)] + [vp] * 11
        L.orc_schedule_synthetic.restype = C.c_int32
        L.orc_schedule_synthetic.argtypes = [C.c_int32, vp, vp, C.c_double, C.c_int32, C.c_int32,
                                             C.c_int32, C.c_int32, C.c_int32, vp]
        _lib = L
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def cam_struct(cam: Camera) -> _Cam:
    """The camera as the renderer receives it: every value rounded to float32 (the C ABI's
    camera is float32), then widened exactly to FP64, so both sides see the same camera."""
    f32 = lambda v: float(np.float32(v))  # noqa: E731
    c = _Cam()
    c.R[:] = [f32(v) for v in np.asarray(cam.R, np.float64).reshape(9)]
    c.t[:] = [f32(v) for v in np.asarray(cam.t, np.float64).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = f32(cam.fx), f32(cam.fy), f32(cam.cx), f32(cam.cy)
    c.width, c.height = cam.width, cam.height
    return c


def prm_struct(prm: RenderParams, sh_degree: int = 0, record: bool = False,
               gap_thr: float = GAP_THR, cull_thr: float = CULL_THR) -> _Prm:
    p = _Prm()
    p.tail, p.mid, p.head, p.mode, p.window_k, p.flags = (prm.tail, prm.mid, prm.head, prm.mode,
                                                          prm.window_k, prm.flags)
    p.sh_degree = sh_degree
    p.record_blends = int(record)
    p.eps_o, p.t_min, p.alpha_max = prm.eps_o, prm.t_min, prm.alpha_max
    p.inv_scale_max, p.dilation, p.frustum_clamp, p.znear = (prm.inv_scale_max, prm.dilation,
                                                             prm.frustum_clamp, prm.znear)
    p.bg[:] = [float(b) for b in prm.bg]
    p.gap_thr, p.cull_thr = gap_thr, cull_thr
    return p


# ----------------------------------------------------------------------------- blocks
def t_opt(d, o, mu, sinv) -> float:
    _, pd = _d(d); _, po = _d(o); _, pm = _d(mu); _, ps = _d(np.asarray(sinv).reshape(9))
    return lib().orc_t_opt(pd, po, pm, ps)


def alg1(mu2, conic, box) -> np.ndarray:
    out = np.zeros(2)
    _, a = _d(mu2); _, b = _d(conic); _, c = _d(box)
    lib().orc_alg1(a, b, c, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def sigma_inv(q, ls, inv_scale_max=1e3) -> np.ndarray:
    out = np.zeros(9)
    _, a = _d(q); _, b = _d(ls)
    lib().orc_sigma_inv(a, b, inv_scale_max, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out.reshape(3, 3)


def sigma(q, ls) -> np.ndarray:
    out = np.zeros(9)
    _, a = _d(q); _, b = _d(ls)
    lib().orc_sigma(a, b, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out.reshape(3, 3)


def sh_basis(direction) -> np.ndarray:
    out = np.zeros(16)
    _, a = _d(direction)
    lib().orc_sh_basis(a, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def t_o(opacity, eps_o=1.0 / 255.0) -> float:
    return lib().orc_t_o(opacity, eps_o)


def project(cam: Camera, prm: RenderParams, mu, sig):
    c, p = cam_struct(cam), prm_struct(prm)
    m2, cov, jac = np.zeros(2), np.zeros(3), np.zeros(6)
    _, a = _d(mu); _, b = _d(np.asarray(sig).reshape(9))
    dp = C.POINTER(C.c_double)
    lib().orc_project(C.byref(c), C.byref(p), a, b, m2.ctypes.data_as(dp), cov.ctypes.data_as(dp),
                      jac.ctypes.data_as(dp))
    return m2, cov, jac.reshape(2, 3)


def schedule_synthetic(t, keep=None, alpha=0.01, mode=0, tail=64, mid=8, head=4,
                       flags=0) -> np.ndarray:
    """Blend order (list indices) of one pixel for a synthetic tile list: depth t[k] at every
    level, alpha everywhere, keep[k] = 0 culls entry k at the 4x4 level."""
    t = np.ascontiguousarray(t, np.float64)
    kp = None if keep is None else np.ascontiguousarray(keep, np.int32)
    order = np.zeros(len(t) + 1, np.int32)
    m = lib().orc_schedule_synthetic(len(t), _ptr(t), _ptr(kp), alpha, mode, tail, mid, head,
                                     flags, _ptr(order))
    return order[:m]


# ----------------------------------------------------------------------------- pipeline
class OracleRun:
    """One (scene, camera, params) oracle evaluation; tiles=None renders every tile."""

    def __init__(self, scene: Scene, cam: Camera, prm: RenderParams, tiles=None,
                 record: bool = False, gap_thr: float = GAP_THR, cull_thr: float = CULL_THR):
        self.scene, self.cam, self.prm = scene, cam, prm
        self._arrs = [np.ascontiguousarray(a, np.float64) for a in
                      (scene.means, scene.log_scales, scene.quats, scene.opacity_logits, scene.sh)]
        self._sc = _Scene(scene.n, *[_ptr(a) for a in self._arrs])
        self._cam = cam_struct(cam)
        self._prm = prm_struct(prm, scene.sh_degree, record, gap_thr, cull_thr)
        self._tiles = None if tiles is None else np.ascontiguousarray(tiles, np.int32)
        self.h = lib().orc_create(C.byref(self._sc), C.byref(self._cam), C.byref(self._prm),
                                  _ptr(self._tiles), 0 if tiles is None else len(self._tiles))

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def num_entries(self) -> int:
        return int(lib().orc_num_entries(self.h))

    @property
    def num_invalid(self) -> int:
        """Gaussians dropped as invalid (non-finite inputs or a zero-length quaternion)."""
        return int(lib().orc_num_invalid(self.h))

    def preprocess(self) -> dict:
        n = self.scene.n
        out = dict(visible=np.zeros(n, np.int32), mean2=np.zeros((n, 2)), conic=np.zeros((n, 3)),
                   opacity=np.zeros(n), color=np.zeros((n, 3)), sinv6=np.zeros((n, 6)),
                   v=np.zeros((n, 3)), pcam=np.zeros((n, 3)), rect=np.zeros((n, 4), np.int32),
                   ntiles=np.zeros(n, np.int32), margin=np.zeros(n))
        lib().orc_get_preprocess(self.h, *[_ptr(out[k]) for k in
                                           ("visible", "mean2", "conic", "opacity", "color", "sinv6",
                                            "v", "pcam", "rect", "ntiles", "margin")])
        return out

    def tile_lists(self):
        T = self.cam.num_tiles
        E = self.num_entries
        start = np.zeros(T + 1, np.int64)
        ids = np.zeros(max(E, 1), np.int32)
        ts = np.zeros(max(E, 1))
        lib().orc_get_tile_lists(self.h, _ptr(start), _ptr(ids), _ptr(ts))
        return start, ids[:E], ts[:E]

    def render(self, max_seq: int = 0, key_cut: float = np.inf) -> dict:
        """Render the selected tiles. sat_batch[y, x] is the HIER batch during which the
        pixel's ray terminated (-1: in the final drain or a flat order, -2: never); with a
        finite key_cut every tile list is truncated to its entries with key t < key_cut."""
        H, W = self.cam.height, self.cam.width
        out = dict(rgb=np.zeros((H, W, 3)), depth=np.zeros((H, W)), tfinal=np.ones((H, W)),
                   nblend=np.zeros((H, W), np.int32), hash=np.zeros((H, W), np.uint64),
                   dmargin=np.full((H, W), np.inf), cmargin=np.full((H, W), np.inf),
                   delta=np.zeros((H, W)), sat_batch=np.full((H, W), -2, np.int32))
        seq = np.full((H, W, max(max_seq, 1)), -1, np.int32)
        cnt = np.zeros(16, np.int64)
        lib().orc_render_ex(self.h, *[_ptr(out[k]) for k in ("rgb", "depth", "tfinal", "nblend", "hash",
                                                             "dmargin", "cmargin", "delta")],
                            _ptr(seq), max_seq, _ptr(cnt), _ptr(out["sat_batch"]), float(key_cut))
        if max_seq:
            out["seq"] = seq
        out["counters"] = {k: int(cnt[i]) for i, k in enumerate(COUNTERS)}
        out["decided"] = (out["dmargin"] > self._prm.gap_thr) & (out["cmargin"] > self._prm.cull_thr)
        return out

    def backward(self, dl_drgb, dl_ddepth=None) -> dict:
        n, K = self.scene.n, (self.scene.sh_degree + 1) ** 2
        g = np.ascontiguousarray(dl_drgb, np.float64)
        gz = None if dl_ddepth is None else np.ascontiguousarray(dl_ddepth, np.float64)
        out = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
                   opacity_logits=np.zeros(n), sh=np.zeros((n, K, 3)), mean2=np.zeros((n, 2)),
                   conic=np.zeros((n, 3)), opacity=np.zeros(n), color=np.zeros((n, 3)))
        lib().orc_backward(self.h, C.byref(self._sc), _ptr(g), _ptr(gz),
                           *[_ptr(out[k]) for k in ("means", "log_scales", "quats", "opacity_logits",
                                                    "sh", "mean2", "conic", "opacity", "color")])
        return out


def render(scene, cam, prm, tiles=None, max_seq=0, **kw) -> dict:
    with OracleRun(scene, cam, prm, tiles, **kw) as r:
        out = r.render(max_seq)
        out["num_entries"] = r.num_entries
        return out
