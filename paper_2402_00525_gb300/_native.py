"""ctypes binding of libstp.so (include/stp.h): struct mirrors and argument marshalling.

Nothing here computes any part of the renderer; every step runs in the CUDA library. If the
library has not been built the import of a function fails loudly -- there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .inputs import Camera, RenderParams

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libstp.so")

(STP_OK, STP_ERR_ARG, STP_ERR_CAPACITY, STP_ERR_TIMEOUT, STP_ERR_CUDA, STP_ERR_NOT_SUPPORTED,
 STP_ERR_INCONSISTENT) = range(7)
FLAG_DEBUG_STATS = 32
FLAG_BACKWARD = 64
FLAG_DEBUG_TRACE = 128
FLAG_GLOBAL_SORT = 256
FLAG_NO_TILE_CULL = 512
FLAG_NO_HIER_CULL = 1024
SORT_STATIC_MAX_N = 1 << 20
TRACE_LEN = 64
MAX_SCENES = 64
MAX_VIEWS = 64


class StpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("stp error %d: %s" % (code, msg))
        self.code = code


class CapacityError(StpError):
    pass


class Gaussians(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int32), ("reserved", C.c_int32)]


class GaussiansGrad(C.Structure):
    _fields_ = [("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logits", C.c_void_p), ("sh", C.c_void_p)]


class CameraS(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("tail", C.c_int32), ("mid", C.c_int32), ("head", C.c_int32),
                ("lb_threshold", C.c_int32), ("eps_o", C.c_float), ("t_min", C.c_float),
                ("alpha_max", C.c_float), ("inv_scale_max", C.c_float), ("dilation", C.c_float),
                ("frustum_clamp", C.c_float), ("znear", C.c_float), ("bg", C.c_float * 3),
                ("mode", C.c_int32), ("window_k", C.c_int32), ("flags", C.c_int32),
                ("blend_cap", C.c_int32), ("max_entries", C.c_int64), ("full_max_passes", C.c_int32),
                ("slice_k", C.c_int32)]


class RunStatus(C.Structure):
    _fields_ = [("error_bits", C.c_uint32), ("mismatched", C.c_uint32),
                ("num_entries", C.c_uint64), ("capacity", C.c_uint64),
                ("counters", C.c_uint64 * 5), ("invalid_gaussians", C.c_uint64), ("redo_warps", C.c_uint64)]


_LAYOUT_SIZE_FIELDS = ["status", "views", "scenes", "geom", "view_z", "rect", "counts", "offsets", "keep_mask",
                       "scan_partials", "keys", "vals", "keys_alt", "vals_alt", "sorted_keys",
                       "sorted_vals", "ranges", "tfinal", "pix_state", "scratch", "dbg_nblend",
                       "dbg_hash", "dbg_delta", "grad_geom", "dbg_trace", "tile_counts", "tile_offsets",
                       "tile_cursor", "tile_partials", "blend_ids", "blend_count", "replay_warps", "tile_front",
                       "tile_redo", "redo_warps", "total"]


class Layout(C.Structure):
    _fields_ = [(f, C.c_size_t) for f in _LAYOUT_SIZE_FIELDS] + [
        ("capacity", C.c_int64), ("total_tiles", C.c_int64), ("total_pixels", C.c_int64),
        ("key_bits", C.c_int32), ("reserved", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


# every symbol include/stp.h declares (the CPU tests check the library exports them)
EXPORTS = ["stp_workspace_size", "stp_workspace_layout_get", "stp_render", "stp_render_backward",
           "stp_workspace_size_batched", "stp_workspace_layout_batched", "stp_render_batched",
           "stp_render_backward_batched", "stp_read_status", "stp_sort_temp_bytes", "stp_sort_pairs", "stp_sort_pairs_noalloc",
           "stp_profile_enable",
           "stp_profile_read", "stp_last_error", "stp_version", "stp_kernel_launches"]

NUM_STAGES = 8
STAGE_NAMES = ["setup", "preprocess", "scan", "duplicate", "sort", "ranges", "render", "bwd_preprocess"]
# the forward's stage 7 is the second depth-slice pass (its kernels return at once when the
# first pass finished every tile); the backward's is the backward Preprocess
FWD_STAGE_NAMES = STAGE_NAMES[:7] + ["second_pass"]

_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libstp.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, sz = C.c_void_p, C.c_size_t
        L.stp_workspace_size.restype = sz
        L.stp_workspace_size.argtypes = [C.c_int64, vp, C.c_int32, vp]
        L.stp_workspace_layout_get.restype = C.c_int
        L.stp_workspace_layout_get.argtypes = [C.c_int64, vp, C.c_int32, vp, vp]
        L.stp_render.restype = C.c_int
        L.stp_render.argtypes = [vp, vp, C.c_int32, vp, vp, sz, vp, vp, vp, vp]
        L.stp_render_backward.restype = C.c_int
        L.stp_render_backward.argtypes = [vp, vp, C.c_int32, vp, vp, sz, vp, vp, vp, vp]
        L.stp_workspace_size_batched.restype = sz
        L.stp_workspace_size_batched.argtypes = [vp, vp, C.c_int32, vp, C.c_int32, vp]
        L.stp_workspace_layout_batched.restype = C.c_int
        L.stp_workspace_layout_batched.argtypes = [vp, vp, C.c_int32, vp, C.c_int32, vp, vp]
        L.stp_render_batched.restype = C.c_int
        L.stp_render_batched.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, vp, vp, sz, vp, vp, vp, vp]
        L.stp_render_backward_batched.restype = C.c_int
        L.stp_render_backward_batched.argtypes = [vp, C.c_int32, vp, vp, C.c_int32, vp, vp, sz, vp, vp, vp, vp]
        L.stp_read_status.restype = C.c_int
        L.stp_read_status.argtypes = [vp, vp, vp]
        L.stp_sort_temp_bytes.restype = sz
        L.stp_sort_temp_bytes.argtypes = [C.c_int64]
        L.stp_sort_pairs.restype = C.c_int
        L.stp_sort_pairs.argtypes = [vp, vp, vp, vp, C.c_int64, vp, C.c_int32, vp, sz, vp]
        L.stp_sort_pairs_noalloc.restype = C.c_int
        L.stp_sort_pairs_noalloc.argtypes = [vp, vp, vp, vp, C.c_int64, vp, C.c_int32, vp]
        L.stp_profile_enable.restype = C.c_int
        L.stp_profile_enable.argtypes = [C.c_int32]
        L.stp_profile_read.restype = C.c_int
        L.stp_profile_read.argtypes = [vp, C.c_int32, vp]
        L.stp_last_error.restype = C.c_char_p
        L.stp_last_error.argtypes = []
        L.stp_version.restype = C.c_int32
        L.stp_kernel_launches.restype = C.c_uint64
        L.stp_kernel_launches.argtypes = []
        L.stp_version.argtypes = []
        _lib = L
    return _lib


def kernel_launches() -> int:
    return int(lib().stp_kernel_launches())


def last_error() -> str:
    return lib().stp_last_error().decode()


def check(code: int) -> None:
    if code != STP_OK:
        msg = last_error()
        if code == STP_ERR_CAPACITY:
            raise CapacityError(code, msg)
        raise StpError(code, msg)


def camera_struct(cam: Camera) -> CameraS:
    c = CameraS()
    c.R[:] = [float(v) for v in np.asarray(cam.R, np.float64).reshape(9)]
    c.t[:] = [float(v) for v in np.asarray(cam.t, np.float64).reshape(3)]
    c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
    c.width, c.height = cam.width, cam.height
    return c


def cameras_array(cams):
    arr = (CameraS * len(cams))()
    for k, cam in enumerate(cams):
        arr[k] = camera_struct(cam)
    return arr


def params_struct(prm: RenderParams, extra_flags: int = 0, max_entries: int = 0) -> Params:
    p = Params()
    p.tail, p.mid, p.head, p.lb_threshold = prm.tail, prm.mid, prm.head, prm.lb_threshold
    p.eps_o, p.t_min, p.alpha_max = prm.eps_o, prm.t_min, prm.alpha_max
    p.inv_scale_max, p.dilation, p.frustum_clamp, p.znear = (prm.inv_scale_max, prm.dilation,
                                                             prm.frustum_clamp, prm.znear)
    p.bg[:] = [float(b) for b in prm.bg]
    p.mode, p.window_k, p.flags = prm.mode, prm.window_k, prm.flags | extra_flags
    p.blend_cap = int(prm.blend_cap)
    p.max_entries = int(max_entries)
    p.full_max_passes = int(prm.full_max_passes)
    p.slice_k = int(prm.slice_k)
    return p


def layout(n, cams, prm: Params, views_per_scene=None) -> Layout:
    """Workspace layout for one scene of n Gaussians, or for several scenes (n a sequence of
    sizes, views_per_scene the number of consecutive cameras of each)."""
    arr = cameras_array(cams)
    L = Layout()
    if views_per_scene is None:
        check(lib().stp_workspace_layout_get(int(n), C.cast(arr, C.c_void_p), len(cams), C.byref(prm),
                                             C.byref(L)))
    else:
        n = [n] if np.isscalar(n) else list(n)
        ns = (C.c_int64 * len(n))(*[int(x) for x in n])
        vps = (C.c_int32 * len(views_per_scene))(*[int(x) for x in views_per_scene])
        check(lib().stp_workspace_layout_batched(C.cast(ns, C.c_void_p), C.cast(vps, C.c_void_p), len(n),
                                                 C.cast(arr, C.c_void_p), len(cams), C.byref(prm), C.byref(L)))
    return L


def read_status(ws_ptr: int, stream: int, raise_on_error: bool = True) -> RunStatus:
    st = RunStatus()
    code = lib().stp_read_status(C.c_void_p(ws_ptr), C.byref(st), C.c_void_p(stream))
    if raise_on_error:
        check(code)
    return st


def profile_enable(max_calls: int) -> None:
    check(lib().stp_profile_enable(int(max_calls)))


def profile_read(max_calls: int) -> np.ndarray:
    """[ncalls, NUM_STAGES] milliseconds of the calls recorded since the last read."""
    out = np.zeros(max(1, max_calls) * NUM_STAGES, np.float32)
    n = C.c_int32(0)
    check(lib().stp_profile_read(out.ctypes.data_as(C.c_void_p), int(max_calls), C.byref(n)))
    return out[: n.value * NUM_STAGES].reshape(n.value, NUM_STAGES)
