"""The multi-rank path of bench.py on CPU: two gloo ranks (views shard with no data-path
collective; only the timings are reduced, by maximum), and the reference arm launched with
torchrun on two ranks (rank 0 alone runs the oracle and prints; the other exits 0)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2402_00525_gb300 import inputs as I  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_views_shard_over_ranks_exactly_once():
    cams = I.orbit_cameras(16 * 3, 15.0, 2.0, I.C2_SIZES, 50.0)
    parts = [bench.shard_views(cams, r, 3) for r in range(3)]
    assert [len(p) for p in parts] == [16, 16, 16]
    seen = sorted(id(c) for p in parts for c in p)
    assert seen == sorted(id(c) for c in cams)
    assert bench.job_mpix_per_s(1000, 4, 2.0) == pytest.approx(2.0)


def test_view_sharding_edge_cases():
    from paper_2402_00525_gb300 import distributed as D
    cams = list(range(5))
    assert [D.shard_views(cams, r, 3) for r in range(3)] == [[0, 3], [1, 4], [2]]
    assert [D.shard_views(cams[:2], r, 4) for r in range(4)] == [[0], [1], [], []]
    assert D.shard_views(cams, 0, 1) == cams
    for rank, world in ((0, 0), (3, 3), (-1, 2)):
        with pytest.raises(ValueError):
            D.shard_views(cams, rank, world)


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = bench.max_over_ranks([10.0 + rank, 5.0 - rank], dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(out % rank, "w") as f:
        json.dump(got, f)


def test_timings_reduce_by_maximum_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    out = str(tmp_path / "r%d.json")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        assert json.load(open(out % r)) == [11.0, 5.0]


@pytest.mark.slow
def test_reference_arm_prints_once_under_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % port, os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--gaussians", "20000"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="2"))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


# ------------------------------------------------------------- one scene, views over ranks
def _scene_case():
    sc = I.cluster_scene(300, 61, nclusters=2, centre_range=0.3, spread_range=(0.2, 0.3),
                         scale_range=(0.01, 0.06), sh_degree=1)
    cams = I.orbit_cameras(4, 3.0, 0.3, [(48, 40), (40, 32)], 50.0)
    return sc, cams


def _view_adjoint(sc, cam, seed):
    """The oracle's adjoint of one view for a seeded dL/drgb (FP64, CPU)."""
    import numpy as np
    from oracle import oracle as O
    rng = np.random.default_rng(seed)
    with O.OracleRun(sc, cam, I.RenderParams(), record=True) as r:
        r.render()
        adj = r.backward(rng.normal(size=(cam.height, cam.width, 3)) / cam.num_pixels)
    return {k: adj[k] for k in ("means", "log_scales", "quats", "opacity_logits", "sh")}


def _train_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2402_00525_gb300 import distributed as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc, cams = _scene_case()
    mine = D.shard_views(list(enumerate(cams)), rank, world)
    # this rank's backward: accumulate (+=) the gradients of its own views
    grads = {k: torch.zeros(v.shape, dtype=torch.float64) for k, v in _view_adjoint(sc, cams[0], 0).items()}
    for v, cam in mine:
        for k, a in _view_adjoint(sc, cam, 100 + v).items():
            grads[k] += torch.from_numpy(a)
    D.allreduce_gradients(grads)
    dist.barrier()
    dist.destroy_process_group()
    np.savez(out % rank, **{k: t.numpy() for k, t in grads.items()})


def test_views_of_one_scene_over_two_gloo_ranks_sum_to_the_single_rank_gradient(tmp_path):
    """Two ranks each differentiate their half of four views (the oracle's adjoint stands in for
    the per-rank backward) and all-reduce: both end with the gradient one rank computes over all
    four views."""
    import numpy as np
    import torch.multiprocessing as mp
    out = str(tmp_path / "g%d.npz")
    mp.start_processes(_train_rank, args=(2, _free_port(), out), nprocs=2, start_method="spawn", join=True)
    sc, cams = _scene_case()
    total = None
    for v, cam in enumerate(cams):
        a = _view_adjoint(sc, cam, 100 + v)
        total = a if total is None else {k: total[k] + a[k] for k in a}
    assert any(np.abs(total[k]).max() > 0 for k in total)
    for r in range(2):
        got = np.load(out % r)
        for k in total:
            np.testing.assert_allclose(got[k], total[k], rtol=1e-12, atol=1e-15)


def test_allreduce_of_several_scenes_and_average(tmp_path):
    """Several scenes' buffers (mixed dtypes) go in one call; each is summed separately, and
    average=True divides by the number of ranks."""
    import torch.multiprocessing as mp
    out = str(tmp_path / "s%d.json")
    mp.start_processes(_multi_scene_rank, args=(3, _free_port(), out), nprocs=3, start_method="spawn", join=True)
    for r in range(3):
        got = json.load(open(out % r))
        assert got["sum"] == [[0 + 1 + 2] * 3, [10 * (0 + 1 + 2)] * 2]
        assert got["avg"] == [2.0, 2.0]           # ranks hold 1, 2, 3
        assert got["flat"] == [3.0 * j + 3.0 for j in range(5)] and got["flat_n"] == 4 * (3 + 3 + 4 + 1 + 48)


def _multi_scene_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch
    import torch.distributed as dist
    from paper_2402_00525_gb300 import distributed as D
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mk = lambda n, v, dt: {k: torch.full((n,), float(v), dtype=dt) for k in D.FIELDS}  # noqa: E731
    scenes = [mk(3, rank, torch.float32), mk(2, 10 * rank, torch.float64)]
    D.allreduce_gradients(scenes)
    avg = mk(1, 1 + rank, torch.float32)
    D.allreduce_gradients(avg, average=True)
    # the flat-buffer form the bench uses: parameter-shaped views of one buffer, reduced in place
    shapes = {"means": (4, 3), "log_scales": (4, 3), "quats": (4, 4), "opacity_logits": (4,), "sh": (4, 16, 3)}
    flat, views = D.gradient_buffers({k: torch.empty(s) for k, s in shapes.items()})
    for j, k in enumerate(D.FIELDS):
        views[k] += rank + j
    D.allreduce_buffer(flat)
    dist.destroy_process_group()
    with open(out % rank, "w") as f:
        json.dump({"sum": [scenes[0]["sh"].tolist(), scenes[1]["means"].tolist()],
                   "avg": [avg["means"].item(), avg["sh"].item()],
                   "flat": [float(views[k].mean()) for k in D.FIELDS], "flat_n": flat.numel()}, f)
