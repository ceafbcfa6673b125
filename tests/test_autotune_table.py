"""Host logic of the autotuner (no GPU): stored tables apply only to their workload, and the
report lists every trial with its sort error and the chosen setting."""
import dataclasses
import json

import pytest

torch = pytest.importorskip("torch")

from paper_2402_00525_gb300 import autotune as A  # noqa: E402
from paper_2402_00525_gb300 import inputs as I  # noqa: E402


def test_tuned_table_applies_only_to_its_workload(tmp_path, monkeypatch):
    path = tmp_path / "tuned.json"
    monkeypatch.setattr(A, "TABLE_PATH", str(path))
    base = I.RenderParams()
    assert A.table("batching") is None and A.tuned_params("batching", base) == base
    chosen = dataclasses.replace(base, tail=96, mid=12, head=8, lb_threshold=16, slice_k=4096)
    A.save_table("batching", chosen, "test")
    data = json.loads(path.read_text())
    assert data["batching"]["tail"] == 96 and data["batching"]["note"] == "test"
    got = A.tuned_params("batching", base)
    assert (got.tail, got.mid, got.head, got.lb_threshold, got.slice_k) == (96, 12, 8, 16, 4096)
    # a table written before a knob existed leaves that knob at the base value
    data["batching"].pop("slice_k")
    path.write_text(json.dumps(data))
    assert A.tuned_params("batching", base).slice_k == base.slice_k
    assert got.eps_o == base.eps_o and got.t_min == base.t_min      # only the tuned knobs move
    assert A.tuned_params("full_hd", base) == base


def test_committed_table_keeps_the_paper_queues_for_the_batching_workload():
    t = A.table("batching")
    assert t is not None
    assert (t["tail"], t["mid"], t["head"]) == (64, 8, 4)       # policy same-result


def test_report_lists_trials_and_choice():
    base = I.RenderParams()
    trials = [A.Trial(64, 8, 4, 16, False, 10.0, 0.1, 2.0, True, 1024),
              A.Trial(96, 12, 4, 16, False, 11.0, 0.05, 1.5, False),
              A.Trial(64, 8, 4, 32, True, 20.0, 0.1, 2.0, True)]
    chosen = trials[0].params(base)
    assert chosen.slice_k == 1024 and trials[1].params(base).slice_k == base.slice_k
    txt = A.report(trials, chosen, dict(delta_avg=0.1, delta_max=2.0), "t", "same-result")
    rows = [ln for ln in txt.splitlines() if ln.startswith("| ") and ln[2].isdigit()]
    assert len(rows) == 3 and rows[0].split("|")[6].strip() == "10.000"       # sorted by time
    assert rows[0].split("|")[10].strip() == "1024" and rows[2].split("|")[10].strip() == "-"
    assert "global" in rows[2]
    assert "Chosen: tail 64, mid 8, head 4, lb_threshold 16, per-tile sort, slice_k 1024." in txt
    assert trials[2].params(base).flags & A.N.FLAG_GLOBAL_SORT
