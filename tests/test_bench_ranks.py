"""The multi-rank plumbing of bench.py on the host: two gloo ranks on 127.0.0.1.

bench.py runs one process per GPU (replicas of the product; no collective on the data
path).  What the ranks share is the timing: a barrier on both sides of the timed
region, the slowest rank's time, and the whole-job throughput from it.  This test runs
that code with the gloo backend on the CPU; the reference arm's non-zero ranks exit
without work.
"""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, local = bench.dist_setup()
    ranks = bench.Ranks(w, backend="gloo", device="cpu")
    ranks.barrier()
    ms = 10.0 + 5.0 * r  # rank 1 is the slow one
    slowest = ranks.max(ms)
    ranks.barrier()
    value = bench.job_throughput(w, 1, slowest)
    ranks.close()
    with open(os.path.join(out_dir, "rank%d.json" % r), "w") as f:
        json.dump({"world": w, "rank": r, "local": local, "slowest": slowest, "value": value}, f)


def test_two_gloo_ranks_share_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(world)]
    for r, d in enumerate(res):
        assert d["world"] == world and d["rank"] == r and d["local"] == r
        assert d["slowest"] == 15.0  # max over ranks
        assert d["value"] == pytest.approx(world * 1e3 / 15.0)


def test_job_throughput_is_whole_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(1, 1, 2.0) == pytest.approx(500.0)
    assert bench.job_throughput(4, 64, 100.0) == pytest.approx(4 * 64 * 10.0)


def test_reference_arm_nonzero_rank_exits_without_work():
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=0)
    assert bench.run_reference(args, world=2, rank=1) == 0


def test_all_core_oracle_timing_runs_on_a_spawned_pool():
    """The CPU baseline's all-core leg: two spawned workers, each with its own oracle,
    run one task per worker for every sampled stage of the product."""
    sys.path.insert(0, ROOT)
    import bench
    from workloads import get_config
    pool = bench.OraclePool("tiny", 2)
    try:
        o = bench.build_oracle(get_config("tiny"))
        sec, parts, desc = pool.sampled_product(o, n_leaves=2, n_boxes=2, n_rows=4, seed=5)
    finally:
        pool.close()
    assert sec > 0 and "2 worker processes" in desc
    assert set(parts) == {"sources", "near", "radiation", "source_transfer", "translation", "reception", "testing"}
    assert all(v >= 0 for v in parts.values())
