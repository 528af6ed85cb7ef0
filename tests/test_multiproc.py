"""The multi-replica timing of bench.py on CPU: two gloo ranks (127.0.0.1), each with its
own local time; the job rate uses the slowest rank's time and the total points of all
replicas, the same on every rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        value, ms = bench.job_rate(local_ms[rank], 1000, 5, world, dist)
        out[rank] = (value, ms)
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank():
    world, port = 2, _free_port()
    local_ms = [40.0, 50.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, local_ms, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        value, ms = res[r]
        assert ms == pytest.approx(50.0)
        assert value == pytest.approx(world * 1000 * 5 / 0.050)


def test_job_rate_single_process():
    import bench

    value, ms = bench.job_rate(20.0, 100, 4, 1)
    assert ms == 20.0 and value == pytest.approx(100 * 4 / 0.020)


def _shard_rank(rank, world, port, out):
    import numpy as np
    import torch.distributed as dist

    import paper_2204_08988_gb300 as P

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # a statistics table of this rank's shard: counts and FP64 sums of very different sizes
        rng = np.random.default_rng(100 + rank)
        table = rng.standard_normal((6, 45)) * 10.0 ** rng.integers(-8, 8, (6, 45))
        out[rank] = P.shard_allreduce(table).tobytes()
    finally:
        dist.destroy_process_group()


def test_shard_statistics_sum_in_rank_order():
    """The cross-process exchange of a point-sharded chain: every rank receives the same
    bits, the sum rank 0 + rank 1 + rank 2 in that order (FP64 addition is not associative,
    so a fixed order is what makes the shards agree)."""
    import numpy as np

    world, port = 3, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_shard_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    tables = []
    for r in range(world):
        rng = np.random.default_rng(100 + r)
        tables.append(rng.standard_normal((6, 45)) * 10.0 ** rng.integers(-8, 8, (6, 45)))
    want = (tables[0] + tables[1]) + tables[2]
    for r in range(world):
        got = np.frombuffer(res[r], dtype=np.float64).reshape(6, 45)
        assert np.array_equal(got, want)


def test_reference_arm_runs_one_oracle_chain_per_core():
    """`bench.py --impl reference` on a small sample: the oracle as it stands, one chain per
    host core in spawned processes started together; the JSON line carries its rate and the
    cores it used."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--workload", "gauss_d2", "--n", "3000"], cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
