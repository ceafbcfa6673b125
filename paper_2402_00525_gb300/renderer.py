"""PyTorch front end of libstp: device memory, streams and autograd plumbing only.

Every step of the renderer runs in libstp.so (include/stp.h). This module allocates the
caller-owned workspace with torch, passes raw device pointers through the C ABI, and wraps
forward + backward in a torch.autograd.Function.
"""
from __future__ import annotations

import ctypes as C
from typing import List, Sequence

import numpy as np
import torch

from . import _native as N
from .inputs import Camera, RenderParams, Scene

FIELDS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def scene_to_device(scene: Scene, device="cuda") -> dict:
    """Copy a numpy Scene to contiguous float32 device tensors."""
    out = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)).to(device)
           for k in FIELDS}
    out["sh_degree"] = scene.sh_degree
    return out


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


def gaussians_struct(g: dict) -> N.Gaussians:
    s = N.Gaussians()
    for k in FIELDS:
        t = g[k]
        if t.dtype != torch.float32 or not t.is_contiguous() or not t.is_cuda:
            raise ValueError("%s must be a contiguous float32 CUDA tensor" % k)
        setattr(s, k, _ptr(t))
    s.n = int(g["means"].shape[0])
    s.sh_degree = int(g["sh_degree"])
    return s


def _grads_struct(grads: dict) -> N.GaussiansGrad:
    gs = N.GaussiansGrad()
    for k in FIELDS:
        t = grads[k]
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError("gradient %s must be contiguous float32" % k)
        setattr(gs, k, _ptr(t))
    return gs


class Renderer:
    """Renders one scene size (or, with views_per_scene, several scenes) from a fixed list of
    cameras with fixed parameters, in one launch per stage.

    With views_per_scene, n is the list of scene sizes and scene s owns views_per_scene[s]
    consecutive cameras; forward / backward then take lists of scene dicts (one per scene).
    The workspace is sized for the configuration and grown on demand when the sort-entry
    capacity turns out too small (this needs one host synchronisation; pass check=False in
    a steady-state loop once the capacity is known). A backward pass reuses the workspace of
    the preceding forward pass, so do not interleave forward calls between the two.

    With backward=True the forward also stores each pixel's blend order for the backward:
    4 * prm.blend_cap bytes a pixel (768 B at the default 192, 1.6 GB per 1920x1080 view).
    Pixels that blend more Gaussians than that are handled by replaying the queues.
    prm.blend_cap = 0 stores nothing and replays every pixel; it is slower, with the same
    gradients up to float rounding.
    """

    def __init__(self, n, cams: Sequence[Camera], prm: RenderParams, device="cuda",
                 backward: bool = False, debug: bool = False, capacity: int | None = None,
                 headroom: float = 1.15, trace: bool = False, views_per_scene: Sequence[int] | None = None):
        self.batched = views_per_scene is not None
        if self.batched:
            self.scene_sizes = [int(x) for x in n]
            self.views_per_scene = [int(x) for x in views_per_scene]
            if len(self.scene_sizes) != len(self.views_per_scene):
                raise ValueError("one view count per scene expected")
            self.n = sum(self.scene_sizes)
        else:
            self.scene_sizes = [int(n)]
            self.views_per_scene = [len(cams)]
            self.n = int(n)
        self._vps_arr = (C.c_int32 * len(self.views_per_scene))(*self.views_per_scene)
        self.cams = list(cams)
        self.prm = prm
        self.device = torch.device(device)
        self.flags = ((N.FLAG_BACKWARD if backward else 0) | (N.FLAG_DEBUG_STATS if debug else 0) |
                      (N.FLAG_DEBUG_TRACE if trace else 0))
        self.headroom = headroom
        self._cams_arr = N.cameras_array(self.cams)
        self.total_pixels = sum(c.width * c.height for c in self.cams)
        self.pixel_offsets = np.cumsum([0] + [c.width * c.height for c in self.cams])
        self.ws = None
        self._graphs = 0
        self.generation = 0              # forwards run so far (the autograd path checks it)
        self._alloc(capacity or 0)

    # ------------------------------------------------------------------ workspace
    def _params(self) -> N.Params:
        return N.params_struct(self.prm, self.flags, self.capacity_req)

    def _alloc(self, capacity: int) -> None:
        if self._graphs:
            raise N.CapacityError(N.STP_ERR_CAPACITY, "the workspace is bound to a captured CUDA graph and "
                                  "cannot grow; build the Renderer with a larger capacity")
        self.capacity_req = int(capacity)
        self.p = self._params()
        if self.batched:
            self.layout = N.layout(self.scene_sizes, self.cams, self.p, self.views_per_scene)
        else:
            self.layout = N.layout(self.n, self.cams, self.p)
        self.capacity = int(self.layout.capacity)
        self._fwd_ready = False          # the workspace holds no forward state yet
        self.ws = None
        torch.cuda.empty_cache() if self.device.type == "cuda" else None
        self.ws = torch.empty(int(self.layout.total), dtype=torch.uint8, device=self.device)

    def _region(self, off: int, count: int, dtype) -> torch.Tensor:
        nbytes = count * torch.empty((), dtype=dtype).element_size()
        return self.ws[off:off + nbytes].view(dtype)

    def set_cameras(self, cams: Sequence[Camera]) -> None:
        """Replace the cameras (same count per scene). The workspace is kept when the image
        sizes are unchanged, so a captured graph stays valid only in that case: it keeps the
        camera poses it was recorded with."""
        cams = list(cams)
        if len(cams) != len(self.cams):
            raise ValueError("expected %d cameras, got %d" % (len(self.cams), len(cams)))
        same = all(a.width == b.width and a.height == b.height for a, b in zip(cams, self.cams))
        self.cams = cams
        self._cams_arr = N.cameras_array(self.cams)
        self._fwd_ready = False
        if not same:
            self.total_pixels = sum(c.width * c.height for c in self.cams)
            self.pixel_offsets = np.cumsum([0] + [c.width * c.height for c in self.cams])
            self._alloc(self.capacity_req)

    @property
    def workspace_bytes(self) -> int:
        return int(self.layout.total)

    # ------------------------------------------------------------------ forward
    def forward(self, g: dict, out=None, check: bool = True, stream=None):
        """Render every camera. Returns (rgb [P,3], depth [P], tfinal [P]) packed view after
        view (see split())."""
        P = self.total_pixels
        if out is None:
            out = (torch.empty((P, 3), dtype=torch.float32, device=self.device),
                   torch.empty((P,), dtype=torch.float32, device=self.device),
                   torch.empty((P,), dtype=torch.float32, device=self.device))
        rgb, depth, tfin = out
        sc = self._scenes(g)
        strm = stream if stream is not None else torch.cuda.current_stream(self.device)
        for attempt in range(3):
            N.check(N.lib().stp_render_batched(C.cast(sc, C.c_void_p), len(sc), C.cast(self._vps_arr, C.c_void_p),
                                               C.cast(self._cams_arr, C.c_void_p), len(self.cams),
                                               C.byref(self.p), C.c_void_p(_ptr(self.ws)), self.layout.total,
                                               C.c_void_p(_ptr(rgb)), C.c_void_p(_ptr(depth)),
                                               C.c_void_p(_ptr(tfin)), C.c_void_p(strm.cuda_stream))
                    if self.batched else
                    N.lib().stp_render(C.byref(sc[0]), C.cast(self._cams_arr, C.c_void_p), len(self.cams),
                                       C.byref(self.p), C.c_void_p(_ptr(self.ws)), self.layout.total,
                                       C.c_void_p(_ptr(rgb)), C.c_void_p(_ptr(depth)),
                                       C.c_void_p(_ptr(tfin)), C.c_void_p(strm.cuda_stream)))
            if not check:
                break
            st = N.read_status(_ptr(self.ws), strm.cuda_stream, raise_on_error=False)
            if st.error_bits & 1:
                if attempt == 2:
                    raise N.CapacityError(N.STP_ERR_CAPACITY, "%d sort entries needed, capacity %d after "
                                          "three attempts" % (st.num_entries, self.capacity))
                self._alloc(int(st.num_entries * self.headroom) + 1024)
                continue
            if st.error_bits & ~2:
                N.check(N.lib().stp_read_status(C.c_void_p(_ptr(self.ws)), C.byref(N.RunStatus()),
                                                C.c_void_p(strm.cuda_stream)))
            self.last_status = st
            break
        self._fwd_ready = True
        self.generation += 1
        return rgb, depth, tfin

    def _scenes(self, g):
        gl = list(g) if self.batched else [g]
        if len(gl) != len(self.scene_sizes):
            raise ValueError("expected %d scenes, got %d" % (len(self.scene_sizes), len(gl)))
        arr = (N.Gaussians * len(gl))()
        for k, (gk, nk) in enumerate(zip(gl, self.scene_sizes)):
            arr[k] = gaussians_struct(gk)
            if arr[k].n != nk:
                raise ValueError("scene %d: renderer was built for n = %d, got %d" % (k, nk, arr[k].n))
        return arr

    def status(self, stream=None) -> N.RunStatus:
        strm = stream if stream is not None else torch.cuda.current_stream(self.device)
        return N.read_status(_ptr(self.ws), strm.cuda_stream, raise_on_error=False)

    # ------------------------------------------------------------------ backward
    def backward(self, g: dict, d_rgb: torch.Tensor, d_depth: torch.Tensor | None, grads: dict,
                 stream=None) -> None:
        """Accumulate (+=) the gradients of <d_rgb, rgb> + <d_depth, depth> of the last forward
        into grads (dict of tensors shaped like the inputs)."""
        if not (self.flags & N.FLAG_BACKWARD):
            raise RuntimeError("construct the Renderer with backward=True")
        if not self._fwd_ready:
            # the backward reads the forward's blend order, lists and records from the workspace
            raise RuntimeError("backward needs a forward with the current workspace and cameras first")
        sc = self._scenes(g)
        gl = list(grads) if self.batched else [grads]
        if len(gl) != len(sc):
            raise ValueError("one gradient dict per scene expected")
        gs = (N.GaussiansGrad * len(gl))()
        for k, gk in enumerate(gl):
            gs[k] = _grads_struct(gk)
        d_rgb = d_rgb.contiguous()
        d_depth = None if d_depth is None else d_depth.contiguous()
        strm = stream if stream is not None else torch.cuda.current_stream(self.device)
        if self.batched:
            N.check(N.lib().stp_render_backward_batched(
                C.cast(sc, C.c_void_p), len(sc), C.cast(self._vps_arr, C.c_void_p),
                C.cast(self._cams_arr, C.c_void_p), len(self.cams), C.byref(self.p), C.c_void_p(_ptr(self.ws)),
                self.layout.total, C.c_void_p(_ptr(d_rgb)), C.c_void_p(_ptr(d_depth)), C.cast(gs, C.c_void_p),
                C.c_void_p(strm.cuda_stream)))
        else:
            N.check(N.lib().stp_render_backward(C.byref(sc[0]), C.cast(self._cams_arr, C.c_void_p), len(self.cams),
                                                C.byref(self.p), C.c_void_p(_ptr(self.ws)), self.layout.total,
                                                C.c_void_p(_ptr(d_rgb)), C.c_void_p(_ptr(d_depth)),
                                                C.byref(gs[0]), C.c_void_p(strm.cuda_stream)))

    # ------------------------------------------------------------------ inspection
    def split(self, packed: torch.Tensor) -> List[torch.Tensor]:
        """Per-view images [H, W, ...] from a packed [P, ...] tensor."""
        out = []
        for k, c in enumerate(self.cams):
            a, b = int(self.pixel_offsets[k]), int(self.pixel_offsets[k + 1])
            out.append(packed[a:b].reshape((c.height, c.width) + tuple(packed.shape[1:])))
        return out

    def debug_stats(self):
        """Per-pixel blend counts and blend-order hashes (needs debug=True)."""
        L = self.layout
        P = int(L.total_pixels)
        nbl = self._region(L.dbg_nblend, P, torch.int32)
        h = self._region(L.dbg_hash, P, torch.int64)
        return nbl, h

    def debug_delta(self) -> torch.Tensor:
        """Per-pixel sort error delta of the last forward (needs debug=True)."""
        return self._region(self.layout.dbg_delta, int(self.layout.total_pixels), torch.float32)

    def capture(self, g, out, d_rgb=None, d_depth=None, grads=None):
        """Record forward (and, with d_rgb, backward) into a CUDA graph. The workspace must
        already be large enough (run forward once with check=True first); from now on it
        cannot grow (a later overflow raises instead of reallocating). Returns the graph;
        graph.replay() re-renders with the current contents of the bound tensors, and
        status() after a replay tells whether the capacity sufficed."""
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.forward(g, out=out, check=False, stream=side)
            if d_rgb is not None:
                self.backward(g, d_rgb, d_depth, grads, stream=side)
        torch.cuda.current_stream(self.device).wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        self._graphs += 1
        with torch.cuda.graph(graph):
            strm = torch.cuda.current_stream(self.device)
            self.forward(g, out=out, check=False, stream=strm)
            if d_rgb is not None:
                self.backward(g, d_rgb, d_depth, grads, stream=strm)
        return graph

    def debug_trace(self) -> torch.Tensor:
        """[P, TRACE_LEN] ids of the first blended Gaussians per pixel (needs trace=True)."""
        P = int(self.layout.total_pixels)
        return self._region(self.layout.dbg_trace, P * N.TRACE_LEN, torch.int32).view(P, N.TRACE_LEN)

    def sorted_lists(self):
        """(ranges [T,2] int32, sorted keys int64, sorted ids int32) of the last forward. With
        the per-tile sort (the default) the keys are written only by a debug renderer."""
        L = self.layout
        st = self.status()
        E = min(int(st.num_entries), self.capacity)
        ranges = self._region(L.ranges, int(L.total_tiles) * 2, torch.int32).view(-1, 2)
        keys = self._region(L.sorted_keys, E, torch.int64)
        vals = self._region(L.sorted_vals, E, torch.int32)
        return ranges, keys, vals

    def records(self):
        """(geom [V, N, 24], view_z [V, N], rect [V, N, 4], counts [V, N]) of one scene. A record's
        24 floats: projected mean as hi, lo pairs (0-3), conic in eigen form (4-7), opacity (8),
        colour (9-11), depth factors m_0, m_1, m_2 (12-20) and c_0..c_2 (21-23); view_z is the
        camera-space depth of the mean."""
        if self.batched:
            raise RuntimeError("records() reads single-scene workspaces")
        L = self.layout
        m = self.n * len(self.cams)
        geom = self._region(L.geom, m * 24, torch.float32).view(len(self.cams), self.n, 24)
        view_z = self._region(L.view_z, m, torch.float32).view(len(self.cams), self.n)
        rect = self._region(L.rect, m * 4, torch.int16).view(len(self.cams), self.n, 4)
        counts = self._region(L.counts, m, torch.int32).view(len(self.cams), self.n)
        return geom, view_z, rect, counts


class StaleForwardError(RuntimeError):
    """The renderer ran another forward between an output's forward and its backward."""


class _RenderFn(torch.autograd.Function):
    """Forward and backward of one Renderer call (Sec. 3.5). The backward state (sorted lists,
    records, the stored blend order) lives in the renderer's one workspace, so an output can
    be differentiated only while that workspace still holds its forward: ctx keeps the
    renderer's forward generation, and the backward raises if another forward ran since."""

    @staticmethod
    def forward(ctx, renderer: Renderer, sh_degree: int, check_status: bool, means, log_scales, quats,
                opacity_logits, sh):
        g = dict(means=means.contiguous(), log_scales=log_scales.contiguous(), quats=quats.contiguous(),
                 opacity_logits=opacity_logits.contiguous(), sh=sh.contiguous(), sh_degree=sh_degree)
        rgb, depth, _ = renderer.forward(g)
        ctx.renderer = renderer
        ctx.generation = renderer.generation
        ctx.check_status = check_status
        ctx.g = g
        return rgb, depth

    @staticmethod
    def backward(ctx, d_rgb, d_depth):
        r = ctx.renderer
        if r.generation != ctx.generation:
            raise StaleForwardError("the renderer ran %d more forward pass(es) after this output was "
                                    "rendered; its workspace no longer holds this output's blend order"
                                    % (r.generation - ctx.generation))
        g = ctx.g
        if d_rgb is None:            # only depth reaches the loss
            d_rgb = torch.zeros((r.total_pixels, 3), dtype=torch.float32, device=r.device)
        grads = {k: torch.zeros_like(g[k]) for k in FIELDS}
        r.backward(g, d_rgb.float(), None if d_depth is None else d_depth.float(), grads)
        if ctx.check_status:
            # synchronises; raises on error bit 8 (the backward did not reproduce the forward's
            # blend sequence) and on any other recorded condition
            N.read_status(_ptr(r.ws), torch.cuda.current_stream(r.device).cuda_stream)
        return (None, None, None) + tuple(grads[k] for k in FIELDS)


def render(renderer: Renderer, g: dict, check_status: bool = True):
    """Differentiable render: returns (rgb [P,3], depth [P]); backward via libstp.

    Each output must be differentiated before the same renderer renders again (the backward
    raises StaleForwardError otherwise). With check_status the backward reads the device
    status block (one host synchronisation) and raises if it recorded an error."""
    if not (renderer.flags & N.FLAG_BACKWARD):
        raise RuntimeError("construct the Renderer with backward=True")
    return _RenderFn.apply(renderer, int(g["sh_degree"]), bool(check_status), g["means"], g["log_scales"],
                           g["quats"], g["opacity_logits"], g["sh"])
