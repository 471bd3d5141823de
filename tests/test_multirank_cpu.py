"""Replicas on several ranks (CPU, gloo, world size 2).

Proofs are independent, so N GPUs run N replicas: each rank proves its own
step (its own seed), there is no data-path collective, and the job's time is
the slowest rank's.  This checks that host logic in two processes: the rank
seeds give different, individually valid proofs; the max over ranks and the
whole-job value are what bench.py reports.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2508_21393_gb300 import workload as W
    seed = bench.rank_seed(rank)
    t = W.lora_projection(seed, 0, "q", 8, 16, 16, 4)
    jobs = W.projection_products(t, seed)
    j = jobs[0]
    pf = oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"])
    C = W.exact_matmul(j["P"].T if j["tp"] else j["P"], j["Q"].T if j["tq"] else j["Q"])
    ok, _ = oracle.verify_matmul(j["P"], j["Q"], C, pf, j["tp"], j["tq"], seed=j["seed"])
    macs = sum(W.macs(x) for x in jobs)
    local_ms = 2.0 + rank  # rank 1 is the slower one
    ms_max = bench.max_over_ranks(local_ms, world, "cpu")
    value = bench.job_value(macs, world, ms_max / 1e3)
    q.put((rank, ok, pf.to_bytes(), ms_max, value, macs))
    dist.destroy_process_group()


def test_two_rank_replicas_and_max_timing():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ok0, pf0, mx0, v0, macs0), (r1, ok1, pf1, mx1, v1, macs1) = res
    assert ok0 and ok1
    assert pf0 != pf1                 # each rank proves its own, different step
    assert mx0 == mx1 == 3.0          # both see the slowest rank's time
    assert macs0 == macs1
    assert v0 == v1 == pytest.approx(2 * macs0 / 3e-3)
