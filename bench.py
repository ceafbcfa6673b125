"""Benchmark of the hierarchical sorted splatting path on GB300.

Workload: 3,000,000 Gaussians (64 anisotropic clusters, SH degree 3), 16 views on a 360 degree
orbit at 1920x1080, fov 50 (synthetic, seeded; stands in for the paper's trained scenes).
One step = one batched forward over the 16 views (Preprocess -> Duplicate -> sort -> hierarchical
Render, one launch sequence for all views) followed by the backward pass of those views
(backward Render replay + backward Preprocess) for a fixed synthetic dL/drgb.

  value         forward Mpix/s = 16 x 1920 x 1080 / forward time of a step (CUDA events)
  ms_per_step   forward + backward of the 16 views
  per_view      the same forward as 16 separate single-view launch sequences
  e2e           forward through the public API with the scene copied in from pinned host
                memory and rgb + depth copied back inside the timed region
  roofline      the dominant kernel (forward Render), ALU bound: algorithmic FP32 work from
                its counted work units / its event-timed duration
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload

--impl reference runs that oracle as the reference arm. Multi-GPU (torchrun): views are
independent, so every rank renders its own 16 views of the scene (weak scaling); only the
timing uses a collective (barrier + max).
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2402_00525_gb300 import inputs as I  # noqa: E402

WORKLOAD = "3M Gaussians (64 clusters, SH3), 16 orbit views 1920x1080, fov 50"
METRIC = "Mpix/s fwd and fwd+bwd ms/view, 3M Gaussians @1080p; batched vs per-view"
FP32_LANES_PER_SM = 128
# algorithmic FP32 operations per work unit of the forward Render (cull by Algorithm 1 + G2 +
# t_opt at a 4x4 or 2x2 box; alpha + t_opt at a pixel)
FLOP_PER_SUBTILE_EVAL, FLOP_PER_QUAD_EVAL, FLOP_PER_PIXEL_EVAL = 80, 80, 45
FLOP_PER_BLEND_GRAD = 40
# backward over the stored blend order, per blend: alpha recomputed at the pixel (G2, exp,
# opacity) with the colour and transmittance updates; then the gradient terms above
FLOP_PER_BLEND_EVAL = 28


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "render_traffic_fullhd_3m_16views.md")
RENDER_SOURCES = ["stp_render.cu", "stp_common.cuh", "stp_kernels.cuh"]


def render_source_hash() -> str:
    """SHA-256 of the Render sources with comments and whitespace removed (code changes only)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in RENDER_SOURCES:
        with open(os.path.join(ROOT, "paper_2402_00525_gb300", "csrc", f)) as fh:
            txt = fh.read()
        txt = re.sub(r"/\*.*?\*/", " ", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", " ", txt)
        h.update(" ".join(txt.split()).encode())
    return h.hexdigest()


def measured_traffic(kernel: str, n: int, views: int):
    """DRAM bytes per launch of a Render kernel from the committed ncu capture of this workload,
    or None when the capture is of other kernel sources or another workload size."""
    if n != 3_000_000 or views != 16 or not os.path.exists(TRAFFIC_FILE):
        return None
    vals = {}
    for line in open(TRAFFIC_FILE):
        if ":" in line and line.startswith("- `"):
            k, v = line[3:].split("`", 1)[0], line.split(":", 1)[1].strip()
            vals[k] = v
    if vals.get("render source sha256") != render_source_hash():
        return None
    v = vals.get(kernel + " DRAM bytes per launch")
    return int(v) if v else None


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def shard_views(all_cams, rank: int, world: int):
    """Views are independent: rank r renders views r, r + world, ... (no forward collective)."""
    from paper_2402_00525_gb300 import distributed as D
    return D.shard_views(all_cams, rank, world)


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings (the job is as slow as its slowest rank)."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def job_mpix_per_s(pixels_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the pixels of all ranks over the slowest rank's time."""
    return pixels_per_rank * world / (ms * 1e-3) / 1e6


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [ln.strip().split(", ") for ln in self.f.read().splitlines() if ln.strip()]
        os.unlink(self.f.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1].split()[0]))
                smax.append(float(r[2].split()[0]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
            except (IndexError, ValueError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(scene, cam, prm, ntiles, seed):
    """Time the FP64 oracle (as it stands) on `ntiles` random tiles of one view."""
    from oracle import oracle as O
    tiles = np.random.default_rng(seed).choice(cam.num_tiles, ntiles, replace=False)
    t0 = time.perf_counter()
    with O.OracleRun(scene, cam, prm, tiles=tiles) as r:
        r.render()
    dt = time.perf_counter() - t0
    return ntiles * 256, dt


def single_thread_oracle(n: int, ntiles: int = 64):
    """The same oracle sample on one host thread (OpenMP fixed at load, so a child process)."""
    code = ("import json, sys; sys.path.insert(0, %r); import bench; from paper_2402_00525_gb300 import inputs as I; "
            "sc, cams, prm = I.full_hd_workload(n=%d, nviews=1); px, t = bench.oracle_sample(sc, cams[0], prm, %d, 7); "
            "print(json.dumps([px, t]))" % (ROOT, n, ntiles))
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300,
                           env=dict(os.environ, OMP_NUM_THREADS="1"))
        px, t = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as e:                      # reported, never fatal for the benchmark
        return {"value": None, "error": str(e)[:200]}
    return {"value": px / t / 1e6, "unit": "Mpix/s", "cores": 1,
            "sample": "%d random tiles of view 0, incl. the preprocess of all Gaussians, %.1f s" % (ntiles, t)}


def oracle_threads() -> int:
    return int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))


def cpu_model() -> str:
    """The host CPU's model name (lscpu on Arm hosts, /proc/cpuinfo otherwise)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def oracle_legs() -> dict:
    """The FP64 oracle on the other workloads of the measurement plan, all host cores: the
    4096-Gaussian 256x256 forward in full, the 512-Gaussian 64x64 forward + adjoint (the
    finite-difference case), and one full 1280x720 forward of the 500k-Gaussian scene."""
    from oracle import oracle as O
    legs = {}
    sc, cams, prm = I.plain_forward_workload()
    t0 = time.perf_counter()
    O.render(sc, cams[0], prm)
    dt = time.perf_counter() - t0
    legs["plain_4096_256x256_fwd"] = {"value": cams[0].num_pixels / dt / 1e6, "unit": "Mpix/s", "seconds": dt}
    sc, _, cam, prm = I.fd_subcase()
    t0 = time.perf_counter()
    with O.OracleRun(sc, cam, prm, record=True) as r:
        r.render()
        r.backward(np.full((cam.height, cam.width, 3), 1.0 / (3 * cam.num_pixels)))
    dt = time.perf_counter() - t0
    legs["fd_512_64x64_fwd_bwd"] = {"value": 1e3 * dt, "unit": "ms per forward + adjoint", "seconds": dt}
    sc, _, cam, prm = I.differentiation_workload()
    t0 = time.perf_counter()
    O.render(sc, cam, prm)
    dt = time.perf_counter() - t0
    legs["diff_500k_1280x720_fwd"] = {"value": cam.num_pixels / dt / 1e6, "unit": "Mpix/s", "seconds": dt}
    return legs


def run_reference(args, rank, world):
    if rank != 0:
        return
    from oracle import build as OB
    OB.build()
    scene, cams, prm = I.full_hd_workload(n=args.n)
    ntiles = 96
    for w in range(args.warmup):
        oracle_sample(scene, cams[w % len(cams)], prm, ntiles, 100 + w)
    px, secs = 0, 0.0
    for k in range(args.steps):
        p, dt = oracle_sample(scene, cams[k % len(cams)], prm, ntiles, 200 + k)
        px += p
        secs += dt
    val = px / secs / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": "%d random tiles of one view per step" % ntiles},
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": oracle_threads(), "cpu_model": cpu_model(),
                             "kind": "oracle",
                             "sample": "%d random 16x16 tiles of view (step mod 16) per step, full preprocess of the 3M Gaussians" % ntiles},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def batching_leg(torch, R, N, g, n):
    """64 views of the 3M scene at 320x240 .. 2560x1440: the batched forward recorded in one
    CUDA graph with the autotuned setting, against 64 single-view launch sequences at the
    default setting (outputs compared bit for bit)."""
    from paper_2402_00525_gb300 import autotune as A
    cams = I.orbit_cameras(64, 15.0, 2.0, I.C4_SIZES, 50.0)
    base = I.RenderParams()
    prm_t = A.tuned_params("batching", base)
    P = sum(c.num_pixels for c in cams)
    rb = R.Renderer(n, cams, prm_t, headroom=1.1)
    out = tuple(torch.empty(sh, device="cuda") for sh in ((P, 3), (P,), (P,)))
    rb.forward(g, out=out)
    graph = rb.capture(g, out)
    for _ in range(2):
        graph.replay()
    ms = []
    for _ in range(3):
        a, b = _events(torch)
        a.record()
        graph.replay()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    assert rb.status().error_bits == 0
    g_ms = float(np.median(ms))
    per = {}
    for c in cams:
        key = (c.width, c.height)
        if key not in per:
            per[key] = R.Renderer(n, [c], base)
    outs = [tuple(torch.empty(sh, device="cuda") for sh in ((c.num_pixels, 3), (c.num_pixels,), (c.num_pixels,)))
            for c in cams]
    for c, o in zip(cams, outs):
        r1 = per[(c.width, c.height)]
        r1.set_cameras([c])
        r1.forward(g, out=o)
    torch.cuda.synchronize()
    pv = []
    l0 = N.kernel_launches()
    for it in range(3):
        a, b = _events(torch)
        a.record()
        for c, o in zip(cams, outs):
            r1 = per[(c.width, c.height)]
            r1.set_cameras([c])
            r1.forward(g, out=o, check=False)
        b.record()
        torch.cuda.synchronize()
        if it:
            pv.append(a.elapsed_time(b))
    pv_ms = float(np.mean(pv))
    same = all(torch.equal(out[0][int(rb.pixel_offsets[k]):int(rb.pixel_offsets[k + 1])], outs[k][0])
               for k in range(len(cams)))
    kernels = N.kernel_launches() - l0
    res = {"workload": "3M Gaussians, 64 orbit views, 13/13/13/13/12 at 320x240/640x480/1280x720/1920x1080/2560x1440",
           "pixels": P, "graph_fwd_ms": g_ms, "graph_mpix_s": P / (g_ms * 1e-3) / 1e6,
           "per_view_fwd_ms": pv_ms, "per_view_mpix_s": P / (pv_ms * 1e-3) / 1e6, "batched_speedup": pv_ms / g_ms,
           "identical_to_per_view": bool(same),
           "tuned": {k: getattr(prm_t, k) for k in ("tail", "mid", "head", "lb_threshold", "flags")},
           "per_view_launch_kernels": kernels // 3}
    del rb, out, graph, per, outs
    torch.cuda.empty_cache()
    return res


def training_leg(torch, R, N):
    """8 scenes (100k .. 3M Gaussians, SH3), 4 views each at 640x480 .. 1920x1080: one training
    step (forward + backward, gradients per scene) recorded in one CUDA graph, against the same
    step as one eager launch sequence per scene."""
    scenes, cams, prm = I.batched_training_workload()
    gs = [R.scene_to_device(sc) for sc in scenes]
    allc = [c for cs in cams for c in cs]
    P = sum(c.num_pixels for c in allc)
    gen = torch.Generator(device="cuda").manual_seed(99)
    d_rgb = (torch.randint(0, 2, (P, 3), device="cuda", generator=gen).float() * 2 - 1) / (3 * P)
    rb = R.Renderer([sc.n for sc in scenes], allc, prm, backward=True, views_per_scene=[len(cs) for cs in cams],
                    headroom=1.1)
    out = tuple(torch.empty(sh, device="cuda") for sh in ((P, 3), (P,), (P,)))
    grads = [{k: torch.zeros_like(g[k]) for k in R.FIELDS} for g in gs]
    rb.forward(gs, out=out)
    graph = rb.capture(gs, out, d_rgb=d_rgb, grads=grads)
    for _ in range(2):
        graph.replay()
    ms = []
    for _ in range(3):
        a, b = _events(torch)
        a.record()
        graph.replay()
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    assert rb.status().error_bits == 0
    g_ms = float(np.median(ms))
    del rb, graph
    torch.cuda.empty_cache()
    singles, offs, o = [], [], 0
    for sc, cs in zip(scenes, cams):
        r1 = R.Renderer(sc.n, cs, prm, backward=True)
        n1 = sum(c.num_pixels for c in cs)
        singles.append((r1, slice(o, o + n1)))
        o += n1
    for (r1, sl), g, gr in zip(singles, gs, grads):
        r1.forward(g)
        r1.backward(g, d_rgb[sl], None, gr)
    torch.cuda.synchronize()
    pv = []
    for _ in range(2):
        a, b = _events(torch)
        a.record()
        for (r1, sl), g, gr in zip(singles, gs, grads):
            r1.forward(g, check=False)
            r1.backward(g, d_rgb[sl], None, gr)
        b.record()
        torch.cuda.synchronize()
        pv.append(a.elapsed_time(b))
    pv_ms = float(np.mean(pv))
    del singles, gs, grads, out
    torch.cuda.empty_cache()
    return {"workload": "8 scenes of 100k/250k/500k/750k/1M/1.5M/2M/3M Gaussians (SH3), 4 views each at "
                        "640x480/1280x720/1600x900/1920x1080",
            "pixels": P, "graph_step_ms": g_ms, "per_scene_step_ms": pv_ms, "batched_speedup": pv_ms / g_ms,
            "fwd_bwd_ms_per_view": g_ms / len(allc)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="stp", choices=["stp", "reference"])
    ap.add_argument("--gaussians", dest="n", type=int, default=3_000_000, help="Gaussians (default: the workload's 3M)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--per-view-rounds", type=int, default=2)
    ap.add_argument("--no-extra", action="store_true", help="skip the 64-view and 8-scene legs")
    ap.add_argument("--views", type=int, default=16, help="views per GPU (default: the workload's 16)")
    ap.add_argument("--profile", choices=["forward", "step"], default=None,
                    help="only run warm-up + steps of the batched forward (no backward flag: a small "
                         "workspace) or of the forward + backward step, for profiler captures")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        return
    args.warmup = max(3, args.warmup)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2402_00525_gb300 import build as B
    B.build()
    from paper_2402_00525_gb300 import _native as N
    from paper_2402_00525_gb300 import renderer as R

    scene, _, prm = I.full_hd_workload(n=args.n, nviews=1)
    all_cams = I.orbit_cameras(args.views * world, 15.0, 2.0, I.C2_SIZES, 50.0)
    cams = shard_views(all_cams, rank, world)
    V = len(cams)
    P = sum(c.num_pixels for c in cams)
    g = R.scene_to_device(scene)
    if args.profile:
        step_too = args.profile == "step"
        fr = R.Renderer(scene.n, cams, prm, backward=step_too)
        fr.forward(g)                                        # sizes the capacity (may render twice)
        d = torch.full((P, 3), 1.0 / (3 * P), device="cuda")
        gr = {k: torch.zeros_like(g[k]) for k in R.FIELDS}
        for _ in range(args.warmup + args.steps):
            fr.forward(g, check=False)
            if step_too:
                fr.backward(g, d, None, gr)
        torch.cuda.synchronize()
        assert fr.status().error_bits == 0
        print(json.dumps({"profile": args.profile, "gaussians": scene.n, "views": V,
                          "workspace_gb": fr.workspace_bytes / 1e9}), flush=True)
        return
    rnd = R.Renderer(scene.n, cams, prm, backward=True)
    out = (torch.empty((P, 3), device="cuda"), torch.empty((P,), device="cuda"), torch.empty((P,), device="cuda"))
    rnd.forward(g, out=out)                                   # sizes the sort-entry capacity
    gen = torch.Generator(device="cuda").manual_seed(1234)
    d_rgb = (torch.randint(0, 2, (P, 3), device="cuda", generator=gen).float() * 2 - 1) / (3 * P)
    # the gradient lives in one flat buffer: with several ranks on one scene the step ends with
    # its sum over the ranks (the one exchange of the path), reduced in place
    from paper_2402_00525_gb300 import distributed as D
    gflat, grads = D.gradient_buffers(g)

    def step():
        rnd.forward(g, out=out, check=False)
        rnd.backward(g, d_rgb, None, grads)
        if dist:
            D.allreduce_buffer(gflat)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    st = rnd.status()
    assert st.error_bits == 0, "status %d after warm-up" % st.error_bits
    entries = int(st.num_entries)

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    clocks = ClockSampler(torch.cuda.current_device())
    N.profile_enable(2 * K)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = N.kernel_launches()
    for k in range(K):
        ev[k][0].record()
        rnd.forward(g, out=out, check=False)
        ev[k][1].record()
        rnd.backward(g, d_rgb, None, grads)
        if dist:
            D.allreduce_buffer(gflat)            # NCCL: the per-scene gradient summed over ranks
        ev[k][2].record()
    torch.cuda.synchronize()
    launches = N.kernel_launches() - launches0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    stages = N.profile_read(2 * K)
    N.profile_enable(0)
    fwd_ms = float(np.mean([e[0].elapsed_time(e[1]) for e in ev]))
    step_ms = float(np.mean([e[0].elapsed_time(e[2]) for e in ev]))
    st = rnd.status()
    assert st.error_bits == 0, "status %d after the timed region" % st.error_bits
    fwd_stage = stages[0::2].mean(0)
    bwd_stage = stages[1::2].mean(0)
    fwd_ms, step_ms = max_over_ranks([fwd_ms, step_ms], dist, "cuda")
    total_px = P * world
    value = job_mpix_per_s(P, world, fwd_ms)

    # ---------------------------------------------------------------- per-view launches
    single = [R.Renderer(scene.n, [c], prm) for c in cams]
    souts = [(torch.empty((c.num_pixels, 3), device="cuda"), torch.empty((c.num_pixels,), device="cuda"),
              torch.empty((c.num_pixels,), device="cuda")) for c in cams]
    for r_, o_ in zip(single, souts):
        r_.forward(g, out=o_)
    torch.cuda.synchronize()
    pv_ms = []
    for _ in range(args.per_view_rounds + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for r_, o_ in zip(single, souts):
            r_.forward(g, out=o_, check=False)
        e1.record()
        torch.cuda.synchronize()
        pv_ms.append(e0.elapsed_time(e1))
    pv_ms = float(np.mean(pv_ms[1:]))
    same = all(torch.equal(out[0][int(rnd.pixel_offsets[k]):int(rnd.pixel_offsets[k + 1])], souts[k][0])
               for k in range(V))
    del single, souts
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- forward only (serving)
    # The training forward above also stores each pixel's blend order for the backward; a
    # renderer without the backward flag stores nothing beyond the images.
    rnd_ws_gb = rnd.workspace_bytes / 1e9
    fo = R.Renderer(scene.n, cams, prm, capacity=rnd.capacity)
    fout = (torch.empty_like(out[0]), torch.empty_like(out[1]), torch.empty_like(out[2]))
    for _ in range(max(args.warmup, 1)):
        fo.forward(g, out=fout, check=False)
    torch.cuda.synchronize()
    fo_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    for e0, e1 in fo_ev:
        e0.record()
        fo.forward(g, out=fout, check=False)
        e1.record()
    torch.cuda.synchronize()
    assert fo.status().error_bits == 0
    fo_ms = max_over_ranks([float(np.mean([e0.elapsed_time(e1) for e0, e1 in fo_ev]))], dist, "cuda")[0]
    fo_same = bool(torch.equal(fout[0], out[0]) and torch.equal(fout[1], out[1]))
    del fo, fout
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- backward by replay
    # The backward of Sec. 3.5 as the paper runs it: no per-pixel lists are stored, every warp
    # recomputes the forward's queues (blend_cap 0). Same step, same gradients up to the order
    # of float atomics; the headline step above walks the stored blend order instead.
    rp = R.Renderer(scene.n, cams, dataclasses.replace(prm, blend_cap=0), backward=True, capacity=rnd.capacity)
    rgrads = {k: torch.zeros_like(g[k]) for k in R.FIELDS}
    rout = (torch.empty_like(out[0]), torch.empty_like(out[1]), torch.empty_like(out[2]))
    for _ in range(max(args.warmup, 1)):
        rp.forward(g, out=rout, check=False)
        rp.backward(g, d_rgb, None, rgrads)
    torch.cuda.synchronize()
    rp_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(K)]
    N.profile_enable(2 * K)
    for e in rp_ev:
        e[0].record()
        rp.forward(g, out=rout, check=False)
        e[1].record()
        rp.backward(g, d_rgb, None, rgrads)
        e[2].record()
    torch.cuda.synchronize()
    rp_stages = N.profile_read(2 * K)
    N.profile_enable(0)
    assert rp.status().error_bits == 0
    rp_fwd, rp_step = max_over_ranks([float(np.mean([e[0].elapsed_time(e[1]) for e in rp_ev])),
                                      float(np.mean([e[0].elapsed_time(e[2]) for e in rp_ev]))], dist, "cuda")
    # gradients of one step of each backward agree (same blend order, other reduction order)
    one = {k: torch.zeros_like(g[k]) for k in R.FIELDS}
    two = {k: torch.zeros_like(g[k]) for k in R.FIELDS}
    rp.forward(g, out=rout, check=False)
    rp.backward(g, d_rgb, None, one)
    rnd.forward(g, out=out, check=False)
    rnd.backward(g, d_rgb, None, two)
    torch.cuda.synchronize()
    rp_rel = max(float((one[k] - two[k]).double().norm() / max(two[k].double().norm().item(), 1e-30)) for k in R.FIELDS)
    replay = {"fwd_bwd_ms_per_view": rp_step / V, "ms_per_step": rp_step, "fwd_ms": rp_fwd,
              "stage_ms": {"forward": {n: round(float(x), 4) for n, x in zip(N.FWD_STAGE_NAMES, rp_stages[0::2].mean(0))},
                           "backward": {n: round(float(x), 4) for n, x in zip(N.STAGE_NAMES, rp_stages[1::2].mean(0))}},
              "grad_rel_l2_vs_stored_order": rp_rel,
              "note": "blend_cap 0: the backward replays the hierarchical queues (recomputed k-buffers, no "
                      "per-pixel lists stored), as Sec. 3.5 specifies"}
    del rp, rgrads, rout, one, two
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- end to end (host buffers)
    # A serving loop through the public API: every step copies its scene in from pinned host
    # memory and its rgb + depth out to pinned host memory. Two buffer sets and two copy
    # streams let step k's upload and step k-1's download overlap step k-1's / k's render.
    host = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)).pin_memory() for k in R.FIELDS}
    h2d = sum(t.numel() * 4 for t in host.values())
    d2h = (P * 3 + P) * 4
    comp = torch.cuda.current_stream()
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    gbuf = [g, dict({k: torch.empty_like(g[k]) for k in R.FIELDS}, sh_degree=g["sh_degree"])]
    obuf = [out, tuple(torch.empty_like(t) for t in out)]
    hout = [(torch.empty((P, 3), pin_memory=True), torch.empty((P,), pin_memory=True)) for _ in range(2)]
    ev = lambda: torch.cuda.Event(enable_timing=False)
    loaded, rendered, drained, consumed = [ev(), ev()], [ev(), ev()], [ev(), ev()], [ev(), ev()]
    for e_ in drained + consumed:
        e_.record(comp)

    def e2e_step(k):
        b = k % 2
        with torch.cuda.stream(up):
            up.wait_event(consumed[b])                   # the render of step k-2 has read gbuf[b]
            for f in R.FIELDS:
                gbuf[b][f].copy_(host[f], non_blocking=True)
            loaded[b].record(up)
        comp.wait_event(loaded[b])
        comp.wait_event(drained[b])                      # step k-2's images have left obuf[b]
        rnd.forward(gbuf[b], out=obuf[b], check=False, stream=comp)
        consumed[b].record(comp)
        rendered[b].record(comp)
        with torch.cuda.stream(down):
            down.wait_event(rendered[b])
            hout[b][0].copy_(obuf[b][0], non_blocking=True)
            hout[b][1].copy_(obuf[b][1], non_blocking=True)
            drained[b].record(down)

    for k in range(2):
        e2e_step(k)
    torch.cuda.synchronize()
    n_e2e = K
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(up)
    for k in range(n_e2e):
        e2e_step(k)
    t1.record(down)
    torch.cuda.synchronize()
    assert rnd.status().error_bits == 0
    same_e2e = torch.equal(hout[0][0], hout[1][0]) and torch.equal(hout[1][0].cuda(), obuf[0][0])
    e2e_ms = max_over_ranks([t0.elapsed_time(t1) / n_e2e], dist, "cuda")[0]
    e2e_val = job_mpix_per_s(P, world, e2e_ms)
    del gbuf, obuf, hout

    # ---------------------------------------------------------------- work counters (untimed)
    dbg = R.Renderer(scene.n, cams, prm, debug=True, capacity=rnd.capacity)
    dbg.forward(g)
    cst = dbg.status()
    cnt = [int(x) for x in cst.counters]
    del dbg
    torch.cuda.empty_cache()
    flops = FLOP_PER_SUBTILE_EVAL * cnt[0] + FLOP_PER_QUAD_EVAL * cnt[2] + FLOP_PER_PIXEL_EVAL * cnt[4]
    render_ms = float(fwd_stage[6])
    props = torch.cuda.get_device_properties(0)
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (render_ms * 1e-3) / 1e12
    bwd_render_ms = float(bwd_stage[6])
    # backward Render: per blend of the stored order, alpha again plus the gradient terms (the
    # few warps with a pixel past blend_cap replay the queues inside the same stage time)
    bflops = (FLOP_PER_BLEND_EVAL + FLOP_PER_BLEND_GRAD) * cnt[3]
    bachieved = bflops / (bwd_render_ms * 1e-3) / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n_gaussians": scene.n, "views_per_gpu": V, "resolution": "1920x1080",
                   "queues": "%d/%d/%d" % (prm.tail, prm.mid, prm.head), "l2": "inputs larger than L2 (708 MB scene, 3.8 GB records)",
                   "parallelism": ("views sharded over ranks, gradients all-reduced (sum) each step"
                                   if world > 1 else "single GPU")},
        "fwd_ms_per_step": fwd_ms, "fwd_bwd_ms_per_view": step_ms / V,
        "backward_modes": {"headline": "stored blend order (blend_cap %d): ms_per_step and fwd_bwd_ms_per_view"
                                       % prm.blend_cap,
                           "stored_order": {"fwd_bwd_ms_per_view": step_ms / V, "ms_per_step": step_ms,
                                            "workspace_gb": rnd_ws_gb},
                           "replay": replay},
        "stage_ms": {"forward": {n: round(float(x), 4) for n, x in zip(N.FWD_STAGE_NAMES, fwd_stage)},
                     "backward": {n: round(float(x), 4) for n, x in zip(N.STAGE_NAMES, bwd_stage)}},
        "per_view": {"fwd_mpix_s": total_px / world / (pv_ms * 1e-3) / 1e6, "fwd_ms_16_views": pv_ms,
                     "batched_speedup": pv_ms / fwd_ms, "identical_to_batched": bool(same)},
        "forward_only": {"mpix_s": job_mpix_per_s(P, world, fo_ms), "fwd_ms": fo_ms,
                         "batched_speedup_vs_per_view": pv_ms / fo_ms, "identical_to_training_forward": fo_same,
                         "note": "batched forward without the backward flag (no stored blend order)"},
        "entries_per_step": entries,
        "e2e": {"value": e2e_val, "unit": "Mpix/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms, "steps": n_e2e, "images_match_device": bool(same_e2e),
                "pipeline": "double-buffered: step k's upload and step k-1's download overlap the renders"},
        "gpu_launches": launches,
        "clocks": clk,
        "roofline": {"bound": "alu", "kernel": "k_render (forward)", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": measured_traffic("k_render<4,0>", scene.n, V),
                     "work_units": {"subtile_evals": cnt[0], "subtile_survivors": cnt[1], "quad_evals": cnt[2],
                                    "blends": cnt[3], "pixel_evals": cnt[4]},
                     "peak_basis": "FP32 FMA issue: %d SMs x 128 lanes x 2 x %.0f MHz" % (props.multi_processor_count, sm_max)},
        "roofline_backward": {"bound": "alu", "kernel": "k_render_bwd_list (stored blend order)", "achieved": bachieved,
                              "peak": peak, "unit": "TFLOP/s", "frac": bachieved / peak,
                              "traffic": measured_traffic("k_render_bwd_list", scene.n, V),
                              "note": "%d FLOP per blend (alpha again, %d; gradient terms, %d); the kernel is "
                                      "limited by its L2 float reductions, not by FP32 issue"
                                      % (FLOP_PER_BLEND_EVAL + FLOP_PER_BLEND_GRAD, FLOP_PER_BLEND_EVAL,
                                         FLOP_PER_BLEND_GRAD)},
    }
    # the paper's own figure, for context only (other GPU, other scenes: not a baseline)
    line["paper_context"] = {
        "fwd_mpix_s": 2073600 / 4.986e-3 / 1e6, "ms_per_1080p_view": 4.986,
        "hardware": "NVIDIA RTX 4090, CUDA 11.8",
        "workload": "13 trained scenes (Mip-NeRF 360, Tanks & Temples, Deep Blending), avg 2.98M Gaussians, "
                    "1.7-2.9M sort entries per view",
        "entries_per_view_here": entries / V,
    }
    if world == 1 and not args.no_extra:
        del rnd, out, grads, gflat
        torch.cuda.empty_cache()
        line["batching"] = batching_leg(torch, R, N, g, scene.n)
        del g
        torch.cuda.empty_cache()
        line["training"] = training_leg(torch, R, N)
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import build as OB
        OB.build()
        ntiles = 6000         # about 10-20 s of FP64 work on 16 host cores
        px, secs = oracle_sample(scene, cams[0], prm, ntiles, 7)
        line["cpu_baseline"] = {"value": px / secs / 1e6, "unit": "Mpix/s", "cores": oracle_threads(),
                                "cpu_model": cpu_model(), "kind": "oracle",
                                "sample": "%d random 16x16 tiles of view 0 (%d px), FP64, incl. the preprocess of all 3M Gaussians, %.1f s" % (ntiles, px, secs),
                                "single_thread": single_thread_oracle(args.n),
                                "legs": oracle_legs()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
