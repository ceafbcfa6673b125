"""Measurement-driven choice of the renderer's size parameters for a workload.

The paper fixes its queue sizes (tail 64, mid 8, head 4) and Duplicate's load-balancing
threshold (32) by an ablation on its own GPU and scenes (appendix C); this module runs that
ablation on the GPU at hand and for the caller's workload, and picks a table from it.

Two kinds of knobs are swept:

* knobs that never change the image: Duplicate's load-balancing threshold (which Gaussians
  are expanded by a warp instead of their own thread, Sec. 3.4), the sort path (per-tile
  partitioned sort or one global radix sort, appendix B.3) and, for the per-tile sort, the
  depth-slice size slice_k (how much of each tile's list it orders before the Render asks for
  more). For these the fastest setting is taken, after checking that its image is
  bit-identical to the base parameters';
* the queue sizes (tail = 32n+32, mid = 4m+4, head window k), which set how far the
  hierarchical resort can move a Gaussian (Sec. 3.3) and so change the sort error delta and
  the image. A setting is admissible under policy "same-result" only if it equals the base
  queue sizes, under "no-worse" if its mean and maximum delta over the covered pixels do not
  exceed the base's, and under "fastest" always. The fastest admissible setting is taken.

Every setting is timed with CUDA events over `reps` forward calls after `warmup` calls; the
sort error of a setting comes from one extra forward with per-pixel debug statistics.
"""
from __future__ import annotations

import argparse
import dataclasses
import itertools
import json
import os
import sys
from typing import List, Sequence

import numpy as np
import torch

from . import _native as N
from . import inputs as I
from . import renderer as R

SPACE = dict(tail=(64, 96, 128), mid=(8, 12, 16, 20), head=(4, 8, 16), lb_threshold=(16, 32, 64),
             slice_k=(0, 1024, 2048, 4096))
POLICIES = ("same-result", "no-worse", "fastest")
TABLE_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned.json")
_TABLE_KEYS = ("tail", "mid", "head", "lb_threshold", "flags", "slice_k")


def table(workload: str) -> dict | None:
    """The stored tuned setting of a workload (written by `--save-table`), or None."""
    if not os.path.exists(TABLE_PATH):
        return None
    with open(TABLE_PATH) as f:
        return json.load(f).get(workload)


def tuned_params(workload: str, base: I.RenderParams) -> I.RenderParams:
    """base with the stored tuned setting of `workload` applied (base itself if none)."""
    t = table(workload)
    if not t:
        return base
    return dataclasses.replace(base, **{k: int(t[k]) for k in _TABLE_KEYS if k in t})


def save_table(workload: str, prm: I.RenderParams, note: str) -> None:
    data = {}
    if os.path.exists(TABLE_PATH):
        with open(TABLE_PATH) as f:
            data = json.load(f)
    data[workload] = dict({k: int(getattr(prm, k)) for k in _TABLE_KEYS}, note=note)
    with open(TABLE_PATH, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
        f.write("\n")


@dataclasses.dataclass
class Trial:
    tail: int
    mid: int
    head: int
    lb_threshold: int
    global_sort: bool
    ms: float                    # median forward time
    delta_avg: float             # sort error over pixels that blend at least one Gaussian
    delta_max: float
    same_image: bool             # bit-identical rgb/depth/T and blend order to the base setting
    slice_k: int = -1            # depth-slice size of the per-tile sort (-1: the base's)

    def params(self, base: I.RenderParams) -> I.RenderParams:
        flags = (base.flags & ~N.FLAG_GLOBAL_SORT) | (N.FLAG_GLOBAL_SORT if self.global_sort else 0)
        return dataclasses.replace(base, tail=self.tail, mid=self.mid, head=self.head,
                                   lb_threshold=self.lb_threshold, flags=flags,
                                   slice_k=self.slice_k if self.slice_k >= 0 else base.slice_k)


class _Workload:
    """Scene(s) on the device plus one renderer per parameter setting (created on demand)."""

    def __init__(self, scenes, cams, views_per_scene=None):
        self.batched = views_per_scene is not None
        self.scenes = list(scenes) if self.batched else [scenes]
        self.cams = list(cams)
        self.vps = views_per_scene
        self.g = [R.scene_to_device(s) for s in self.scenes]
        self.capacity = 0

    def renderer(self, prm, debug):
        n = [s.n for s in self.scenes] if self.batched else self.scenes[0].n
        return R.Renderer(n, self.cams, prm, debug=debug, capacity=self.capacity or None,
                          views_per_scene=self.vps)

    def arg(self):
        return self.g if self.batched else self.g[0]


def _time_forward(r: R.Renderer, g, reps: int, warmup: int) -> float:
    r.forward(g)                                  # sizes the workspace
    strm = torch.cuda.current_stream()
    for _ in range(warmup):
        r.forward(g, check=False)
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(strm)
        r.forward(g, check=False)
        b.record(strm)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    st = r.status()
    if st.error_bits & 1:
        raise N.CapacityError(N.STP_ERR_CAPACITY, "capacity exceeded while timing")
    return float(np.median(ts))


def _debug_run(w: _Workload, prm):
    r = w.renderer(prm, debug=True)
    rgb, depth, tf = r.forward(w.arg())
    nbl, h = r.debug_stats()
    d = r.debug_delta()
    cov = nbl > 0
    dv = d[cov].double()
    stats = (float(dv.mean()) if dv.numel() else 0.0, float(dv.max()) if dv.numel() else 0.0)
    img = (rgb.clone(), depth.clone(), tf.clone(), nbl.clone(), h.clone())
    w.capacity = max(w.capacity, int(r.capacity))
    del r
    return stats, img


def _same(a, b) -> bool:
    return all(torch.equal(x, y) for x, y in zip(a, b))


def tune(scenes, cams: Sequence[I.Camera], base: I.RenderParams | None = None,
         views_per_scene: Sequence[int] | None = None, policy: str = "same-result",
         space: dict | None = None, reps: int = 5, warmup: int = 2, log=None):
    """Sweep `space` on the workload; returns (chosen RenderParams, list of Trial, the base
    setting's sort error {delta_avg, delta_max}).

    scenes is one Scene (views_per_scene None) or a list of scenes with the number of
    consecutive cameras of each."""
    if policy not in POLICIES:
        raise ValueError("policy must be one of %s" % (POLICIES,))
    base = base or I.RenderParams()
    space = dict(SPACE if space is None else space)
    w = _Workload(scenes, cams, views_per_scene)
    say = log or (lambda *a: None)
    (b_avg, b_max), b_img = _debug_run(w, base)
    trials: List[Trial] = []

    def run(tail, mid, head, lb, gsort, img_ref, slice_k=-1):
        t = Trial(tail, mid, head, lb, gsort, 0.0, 0.0, 0.0, False, slice_k)
        prm = t.params(base)
        (t.delta_avg, t.delta_max), img = _debug_run(w, prm)
        t.same_image = _same(img, img_ref)
        r = w.renderer(prm, debug=False)
        t.ms = _time_forward(r, w.arg(), reps, warmup)
        del r
        torch.cuda.empty_cache()
        trials.append(t)
        say("tail %3d mid %2d head %2d lb %2d %s slice %4d: %8.3f ms  delta avg %.5f max %.4f %s" % (
            tail, mid, head, lb, "global" if gsort else "tiles ", prm.slice_k, t.ms, t.delta_avg,
            t.delta_max, "same image" if t.same_image else ""))
        return t

    # 1. knobs that keep the image: load-balancing threshold, sort path and (per-tile sort only)
    # depth-slice size, at the base queues
    inv = []
    for lb, gsort in itertools.product(space.get("lb_threshold", (base.lb_threshold,)), (False, True)):
        for k in ((base.slice_k,) if gsort else space.get("slice_k", (base.slice_k,))):
            inv.append(run(base.tail, base.mid, base.head, lb, gsort, b_img, k))
    bad = [t for t in inv if not t.same_image]
    if bad:
        raise RuntimeError("result-invariant knob changed the image: %s" % bad[0])
    best_inv = min(inv, key=lambda t: t.ms)
    # 2. queue sizes, with the best invariant knobs
    queues = [q for q in itertools.product(space.get("tail", (base.tail,)), space.get("mid", (base.mid,)),
                                           space.get("head", (base.head,)))
              if q != (base.tail, base.mid, base.head)]
    for tail, mid, head in queues:
        run(tail, mid, head, best_inv.lb_threshold, best_inv.global_sort, b_img, best_inv.slice_k)

    def admissible(t: Trial) -> bool:
        if policy == "same-result":
            return (t.tail, t.mid, t.head) == (base.tail, base.mid, base.head)
        if policy == "no-worse":
            return t.delta_avg <= b_avg * (1 + 1e-6) and t.delta_max <= b_max * (1 + 1e-6)
        return True

    best = min((t for t in trials if admissible(t)), key=lambda t: t.ms)
    return best.params(base), trials, dict(delta_avg=b_avg, delta_max=b_max)


def report(trials: Sequence[Trial], chosen: I.RenderParams, base_delta: dict, title: str, policy: str) -> str:
    lines = ["# %s" % title, "",
             "Policy `%s`. Base sort error: delta avg %.5f, max %.4f." % (policy, base_delta["delta_avg"],
                                                                          base_delta["delta_max"]),
             "Chosen: tail %d, mid %d, head %d, lb_threshold %d, %s sort, slice_k %d." % (
                 chosen.tail, chosen.mid, chosen.head, chosen.lb_threshold,
                 "global radix" if chosen.flags & N.FLAG_GLOBAL_SORT else "per-tile", chosen.slice_k), "",
             "| tail | mid | head | LB | sort | fwd ms | delta avg | delta max | same image | slice_k |",
             "|---:|---:|---:|---:|---|---:|---:|---:|---|---:|"]
    for t in sorted(trials, key=lambda t: t.ms):
        lines.append("| %d | %d | %d | %d | %s | %.3f | %.5f | %.4f | %s | %s |" % (
            t.tail, t.mid, t.head, t.lb_threshold, "global" if t.global_sort else "tiles", t.ms,
            t.delta_avg, t.delta_max, "yes" if t.same_image else "no",
            "-" if t.global_sort else ("base" if t.slice_k < 0 else str(t.slice_k))))
    return "\n".join(lines) + "\n"


WORKLOADS = {
    "batching": "3M Gaussians, 64 orbit views at 320x240 .. 2560x1440",
    "full_hd": "3M Gaussians, 16 orbit views at 1920x1080",
    "plain": "4096 uniform Gaussians, one 256x256 view",
    "training": "8 scenes of 100k .. 3M Gaussians, 4 views each at 640x480 .. 1920x1080",
}


def _load(name: str):
    if name == "batching":
        sc, cams, prm = I.batching_workload()
        return sc, cams, prm, None
    if name == "full_hd":
        sc, cams, prm = I.full_hd_workload()
        return sc, cams, prm, None
    if name == "plain":
        sc, cams, prm = I.plain_forward_workload()
        return sc, cams, prm, None
    scenes, cams, prm = I.batched_training_workload()
    return scenes, [c for cs in cams for c in cs], prm, [len(cs) for cs in cams]


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="batching")
    ap.add_argument("--policy", choices=POLICIES, default="same-result")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--out", default=None, help="write the markdown report here")
    ap.add_argument("--json", default=None, help="write the chosen parameters here")
    ap.add_argument("--save-table", action="store_true", help="store the choice in the package's tuned table")
    a = ap.parse_args(argv)
    scenes, cams, prm, vps = _load(a.workload)
    chosen, trials, bd = tune(scenes, cams, prm, vps, policy=a.policy, reps=a.reps, warmup=a.warmup,
                              log=lambda s: print(s, flush=True))
    txt = report(trials, chosen, bd, "Autotuner sweep: %s" % WORKLOADS[a.workload], a.policy)
    print(txt)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    if a.json:
        with open(a.json, "w") as f:
            json.dump(dict(tail=chosen.tail, mid=chosen.mid, head=chosen.head, lb_threshold=chosen.lb_threshold,
                           flags=chosen.flags, slice_k=chosen.slice_k), f)
    if a.save_table:
        best = min(trials, key=lambda t: t.ms if t.params(prm) == chosen else float("inf"))
        save_table(a.workload, chosen, "policy %s, %.3f ms forward (%s)" % (a.policy, best.ms,
                                                                           torch.cuda.get_device_name()))
    return 0


if __name__ == "__main__":
    sys.exit(main())
