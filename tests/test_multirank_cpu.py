"""The multi-GPU (N > 1) logic of bench.py on CPU, world size 2 over gloo.

Chains are independent (Sec. III: samples need no communication), so ranks
own disjoint chain ids (disjoint Philox streams) and the only cross-rank
traffic is the timing reduction.  This runs the same helpers bench.py uses,
as two gloo processes on 127.0.0.1.
"""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ids = bench.rank_chain_ids(rank, 5)
        t = bench.max_over_ranks(10.0 + rank, dist)          # rank 1 is the slowest
        gathered = [None] * world
        dist.all_gather_object(gathered, ids)
        out[rank] = (ids, t, gathered)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_chains_and_take_the_slowest_time():
    world, port = 2, _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    ids0, t0, g = out[0]
    ids1, t1, _ = out[1]
    assert ids0 == [0, 1, 2, 3, 4] and ids1 == [5, 6, 7, 8, 9]
    assert not set(g[0]) & set(g[1])                          # disjoint Philox streams
    assert t0 == t1 == 11.0                                  # max over ranks, on every rank


def test_single_rank_helpers_without_a_process_group():
    import bench
    assert bench.max_over_ranks(3.5, dist) == 3.5
    assert bench.rank_chain_ids(0, 3) == [0, 1, 2]


def test_reference_arm_is_silent_on_other_ranks(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")

    class A:
        warmup, steps, gpus, chains = 3, 1, 2, 256
        Lx = two_W = beta = chi_max = None
        precision = "mixed"
    bench.run_reference(A())
    assert capsys.readouterr().out == ""


pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def test_oracle_baseline_pool_uses_every_requested_core():
    """bench.oracle_parallel: one oracle chain per spawned process, 1 BLAS thread each."""
    import bench
    cfg = dict(Lx=2, two_W=2, J_leg=1.0, J_rung=1.0, beta=0.2, tau=0.1, chi_max=8, cutoff=1e-10)
    rate, per_step, procs, wall = bench.oracle_parallel(2, procs=2, cfg=cfg)
    assert procs == 2 and len(per_step) == 2 and rate > 0 and wall > 0
    assert abs(rate - 4 / sum(per_step)) < 1e-12


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference on a tiny ladder: one JSON line with the
    contract's keys (the oracle on host cores, steps bounded)."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--Lx", "2", "--two-W", "2", "--chi-max", "8", "--beta", "0.2"],
                       capture_output=True, text=True, timeout=300, cwd=root,
                       env=dict(os.environ, RANK="0", WORLD_SIZE="1"))
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["config"]["Lx"] == 2 and line["config"]["schedule"] == "plain"
