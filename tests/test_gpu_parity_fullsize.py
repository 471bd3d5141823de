"""Full-size parity at the benchmark's configuration: the batched 7B-shaped
LoRA step (32 layers x {q,k,v,o}, hidden 4096, seq 512, ranks {8,16,64};
1024 proofs) proved with one plan and CUDA-graph replay, exactly as bench.py
runs it.

* Sampled outputs: all eight proofs of two projections (one of rank 64 when
  the draw has one) are recomputed by the oracle and compared byte for byte.
* Properties on every proof: dims, status, the transcript replayed from the
  public statement (u, v, every r_i and the final state), g_i(0) + g_i(1)
  equal to the running claim, and the final claim equal to a_r . b_r.
"""
import ctypes

import numpy as np
import pytest

import oracle
from oracle.field import R_MOD
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)


def _fr(x):
    return x.to_int()


def _replay(job, pf):
    m, k, n = W.op_shape(job)
    d0, d1, d2 = (m - 1).bit_length(), (k - 1).bit_length(), (n - 1).bit_length()
    assert (pf.m, pf.k, pf.n, pf.d0, pf.d1, pf.d2, pf.status) == (m, k, n, d0, d1, d2, 0)
    T = oracle.Transcript(job["seed"], m, k, n, job["tp"], job["tq"])
    T.squeeze(b"u", d0)
    T.squeeze(b"v", d2)
    claim = _fr(pf.c)
    T.absorb_fr(b"c", [claim])
    for i in range(d1):
        g = [_fr(pf.g[i][q]) for q in range(3)]
        assert (g[0] + g[1]) % R_MOD == claim, f"round {i}"
        T.absorb_fr(b"g", [g[0], g[2]])  # g(1) is fixed by the running claim
        r = T.squeeze(b"r", 1)[0]
        claim = oracle.round_poly_eval(*g, r)
    assert claim == _fr(pf.a_r) * _fr(pf.b_r) % R_MOD
    T.absorb_fr(b"f", [_fr(pf.a_r), _fr(pf.b_r)])
    assert T.state == bytes(pf.state)


def test_7b_step_batched_graph():
    projs = W.make_step("7b")
    jobs = [j for t in projs for j in W.projection_products(t)]
    dev = {}
    for t in projs:
        for key in ("X", "W", "A", "B", "dY", "H", "dH"):
            dev[id(t[key])] = torch.from_numpy(t[key]).cuda()
    djobs = [B.job(dev[id(j["P"])], dev[id(j["Q"])], j["tp"], j["tq"], j["seed"]) for j in jobs]
    plan = B.vl_plan_create(djobs)
    try:
        nws = B.vl_plan_workspace_bytes(plan)
        ws = torch.empty(nws, dtype=torch.uint8, device="cuda")
        out = torch.empty(len(djobs) * ctypes.sizeof(B.vl_proof), dtype=torch.uint8, device="cuda")
        for _ in range(2):  # capture, then replay
            B.vl_plan_run(plan, ws.data_ptr(), nws, out.data_ptr(), B.VL_DEVICE)
        torch.cuda.synchronize()
        proofs = (B.vl_proof * len(djobs)).from_buffer_copy(out.cpu().numpy().tobytes())
    finally:
        B.vl_plan_destroy(plan)
    for j, pf in zip(jobs, proofs):
        _replay(j, pf)
    ranks = [t["r"] for t in projs]
    other = next((i for i, r in enumerate(ranks) if r == 64 and i > 0), len(projs) - 1)
    sample = [0, other]
    for pi in sample:
        for q in range(8):
            idx = pi * 8 + q
            j = jobs[idx]
            ref = oracle.prove_matmul(j["P"], j["Q"], j["tp"], j["tq"], seed=j["seed"]).to_bytes()
            assert B.proof_bytes(proofs[idx]) == ref, j["name"]
