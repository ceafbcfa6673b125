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
