"""Host-side parts of the benchmark: the CPU oracle's timing on one thread and
on several spawned processes (the `cpu_baseline` leg and the reference arm)."""

import bench
from paper_2606_15622_gb300 import populations as P


def test_cpu_baseline_single_and_all_cores():
    pop = P.couette(seed=4)
    out = bench.cpu_baseline(pop, budget_s=0.5, workers=2)
    assert out["kind"] == "oracle" and out["cores"] == 2 and out["unit"] == "cells/s"
    assert out["value"] > 0 and out["single_thread"]["value"] > 0 and out["single_thread"]["cores"] == 1
    assert "2 processes" in out["sample"]
    one = bench.cpu_baseline(pop, budget_s=0.3, workers=1)
    assert one["cores"] == 1 and one["value"] > 0 and "single_thread" not in one
    assert out["host"]["nproc"] >= 1 and one["host"]["model"]


def test_worker_shares_cover_every_block_once():
    for n_blocks in (1, 4, 32):
        for workers in (1, 2, 3, 16, 40):
            shares = [bench.oracle_share(w, workers, n_blocks) for w in range(workers)]
            assert all(shares)
            flat = [b for sh in shares for b in sh]
            assert set(flat) == set(range(n_blocks))
            if workers <= n_blocks:
                assert len(flat) == n_blocks


def test_host_record_and_step_statistics():
    h = bench.host_cpu()
    assert isinstance(h["model"], str) and h["model"] and h["nproc"] >= 1
    st = bench.step_stats([0.7, 0.6, 0.65, 0.9])
    assert st == {"median": 0.675, "best": 0.6}
