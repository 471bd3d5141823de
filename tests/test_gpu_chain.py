"""GPU parity of the chained projection proof (Sec. IV sequential
composition; vl_prove_chain): every proof equals the oracle's byte for byte
through the C ABI, and the library's host verifier accepts it.

Cases: ragged shapes (odd dimensions, rank 1, one token) on both fold paths
(dimensions TMA can and cannot address), a batch of mixed chains equal to
each chain proved alone, binds, and one full 7B-shaped projection (seq 512,
hidden 4096, rank 16) at the benchmark's scale.
"""
import numpy as np
import pytest

import oracle
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)

BINDS = tuple(bytes([i + 7]) * 32 for i in range(7))


def _proj(n, d, k, r, seed=3, layer=0):
    return W.chain_tensors(W.lora_projection(seed, layer, "q", n, d, k, r))


def _dev_job(t, seed, binds=None):
    dev = {k: torch.from_numpy(np.ascontiguousarray(t[k])).cuda() for k in B.CHAIN_MATS}
    return B.chain_job(dev, seed=seed, binds=binds)


def _prove(ts, seeds, binds=None):
    jobs = [_dev_job(t, s, binds) for t, s in zip(ts, seeds)]
    n = B.vl_chain_workspace_bytes(jobs)
    assert n > 0
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    out = B.vl_prove_chain(jobs, ws.data_ptr(), n)
    torch.cuda.synchronize()
    return out


def _host_job(t, seed, binds=None):
    return B.chain_job({k: np.ascontiguousarray(t[k]) for k in B.CHAIN_MATS}, seed=seed, binds=binds)


@pytest.mark.parametrize("shape", [(6, 10, 12, 3), (8, 16, 8, 4), (5, 7, 9, 2), (1, 4, 4, 1),
                                   (64, 256, 128, 16), (100, 200, 72, 8), (256, 512, 512, 64)])
def test_chain_matches_oracle(shape):
    t = _proj(*shape)
    pf = _prove([t], [11], BINDS)[0]
    assert pf.status == 0
    assert B.chain_proof_bytes(pf) == oracle.prove_chain(t, seed=11, binds=BINDS).to_bytes()
    assert B.vl_verify_chain(_host_job(t, 11, BINDS), W.chain_outputs(t), pf)


def test_batch_of_chains_equals_each_alone():
    ts = [_proj(6, 10, 12, 3, layer=1), _proj(64, 256, 128, 16, layer=2), _proj(8, 16, 8, 4, layer=3)]
    seeds = [21, 22, 23]
    batch = _prove(ts, seeds)
    for t, s, pf in zip(ts, seeds, batch):
        alone = _prove([t], [s])[0]
        assert B.chain_proof_bytes(pf) == B.chain_proof_bytes(alone)
        assert B.chain_proof_bytes(pf) == oracle.prove_chain(t, seed=s).to_bytes()


def test_chain_7b_projection_full_size():
    t = W.chain_tensors(W.lora_projection(W.GLOBAL_SEED, 0, "q", 512, 4096, 4096, 16))
    seed = W.proof_seed(W.GLOBAL_SEED, 0, "q", "chain")
    pf = _prove([t], [seed])[0]
    assert pf.status == 0
    assert B.chain_proof_bytes(pf) == oracle.prove_chain(t, seed=seed).to_bytes()
    assert B.vl_verify_chain(_host_job(t, seed), W.chain_outputs(t), pf)


def test_chain_plan_reruns_and_rebinds():
    ts = [_proj(64, 256, 128, 16, layer=4), _proj(6, 10, 12, 3, layer=5)]
    jobs = [_dev_job(t, 30 + i) for i, t in enumerate(ts)]
    plan = B.ChainPlan(jobs)
    try:
        n = plan.workspace_bytes()
        assert n == B.vl_chain_workspace_bytes(jobs)
        ws1 = torch.empty(n, dtype=torch.uint8, device="cuda")
        ws2 = torch.empty(n + 4096, dtype=torch.uint8, device="cuda")
        want = [oracle.prove_chain(t, seed=30 + i).to_bytes() for i, t in enumerate(ts)]
        for ws in (ws1, ws1, ws2, ws1):  # rerun, then another workspace, then back
            out = plan.run(ws.data_ptr(), n)
            assert [B.chain_proof_bytes(p) for p in out] == want
    finally:
        plan.destroy()
