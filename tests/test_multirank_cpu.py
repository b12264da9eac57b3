"""Multi-rank host logic of the benchmark, on CPU with world_size-2 `gloo` ranks.

The coalescence step shards by independent boxes (replicas): each rank steps its own box and the
only collective is the one all_gather that forms the whole-job figures (slowest rank's time, sum
of SD-steps).  These tests run that host logic in two processes without a GPU: the combination
rule, per-rank independent workloads, and that the reference arm does its work on rank 0 only.
"""
import io
import json
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        # rank r reports its own span, SD-steps and end-to-end step time
        tot_ms, sd, e2e = bench.combine_ranks(10.0 + rank, 1000.0 * (rank + 1), 0.5 + 0.25 * rank, dist, world,
                                              "cpu")
        # replicas draw different boxes
        box = bench.workload("gravitational_box", rank)
        # the reference arm prints on rank 0 only
        args = type("A", (), {"workload": "golovin_box", "steps": 1, "warmup": 3})()
        buf = io.StringIO()
        with redirect_stdout(buf):
            bench.run_reference(args, rank, world)
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"tot_ms": tot_ms, "sd": sd, "e2e": e2e, "v_head": box["v"][:8].tolist(),
                       "printed": buf.getvalue()}, f)
    finally:
        dist.destroy_process_group()


@pytest.fixture(scope="module")
def two_ranks(tmp_path_factory):
    out = tmp_path_factory.mktemp("ranks")
    mp.start_processes(_worker, args=(2, _free_port(), str(out)), nprocs=2, join=True, start_method="spawn")
    res = []
    for r in range(2):
        with open(out / f"r{r}.json") as f:
            res.append(json.load(f))
    return res


def test_whole_job_figures_are_max_time_and_summed_work(two_ranks):
    for r in two_ranks:
        assert r["tot_ms"] == 11.0            # slowest rank's timed span
        assert r["sd"] == 3000.0              # SD-steps of both ranks
        assert r["e2e"] == 0.75               # slowest end-to-end step


def test_replicas_are_independent_boxes(two_ranks):
    assert not np.array_equal(two_ranks[0]["v_head"], two_ranks[1]["v_head"])


def test_reference_arm_runs_on_rank_zero_only(two_ranks):
    line = json.loads(two_ranks[0]["printed"].strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
    assert two_ranks[1]["printed"] == ""


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(5.0, 7.0, 0.1, None, 1, "cpu") == (5.0, 7.0, 0.1)
