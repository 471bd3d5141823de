"""GPU parity of the batched-claim sumcheck: every batched proof from the
CUDA path (claims, rounds, final values, state) equals the oracle's byte for
byte, through the C ABI; and the library verifier accepts it.

Cases: k = 1 (no rounds) and 2 (one round), ragged k, a batch of one,
transposed operands, host operands, the products of a LoRA projection grouped
by inner dimension, and a batch of 64 products."""
import numpy as np
import pytest

from oracle import batch as OB
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no GPU", allow_module_level=True)


def _rand(rng, shape):
    return rng.integers(-(1 << 15), 1 << 15, size=shape).astype(np.int16)


def _jobs(rng, K, k, host=False):
    out = []
    for i in range(K):
        m, n, tp, tq = 5 + 3 * i, 4 + 7 * i, i % 2, (i // 2) % 2
        A, Bm = _rand(rng, (m, k)), _rand(rng, (k, n))
        P = np.ascontiguousarray(A.T) if tp else A
        Q = np.ascontiguousarray(Bm.T) if tq else Bm
        out.append({"P": P, "Q": Q, "tp": tp, "tq": tq, "binds": (bytes([i + 1]) * 32, bytes(32), bytes(32)),
                    "C": A.astype(np.int64) @ Bm.astype(np.int64)})
    return out


def gpu_batch(jobs, seed, host=False):
    keep = []
    cj = []
    for j in jobs:
        P = j["P"] if host else torch.from_numpy(np.ascontiguousarray(j["P"])).cuda()
        Q = j["Q"] if host else torch.from_numpy(np.ascontiguousarray(j["Q"])).cuda()
        keep += [P, Q]
        cj.append(B.job(P, Q, j["tp"], j["tq"], 0, j.get("binds")))
    n = B.vl_batch_workspace_bytes(cj)
    assert n > 0
    ws = torch.empty(n, dtype=torch.uint8, device="cuda")
    res = B.vl_prove_matmul_batched(cj, seed, ws.data_ptr(), n)
    assert res.proof.status == 0
    return res


@pytest.mark.parametrize("K,k", [(1, 1), (3, 2), (1, 37), (4, 33), (3, 300), (2, 4096)])
def test_batch_parity(K, k):
    rng = np.random.default_rng(K * 1000 + k)
    jobs = _jobs(rng, K, k)
    res = gpu_batch(jobs, seed=K + k)
    assert res.to_bytes() == OB.prove_matmul_batch(jobs, seed=K + k).to_bytes()


def test_batch_host_operands_and_verifier():
    rng = np.random.default_rng(5)
    jobs = _jobs(rng, 3, 64)
    res = gpu_batch(jobs, seed=9, host=True)
    assert res.to_bytes() == OB.prove_matmul_batch(jobs, seed=9).to_bytes()
    cj = [B.job(j["P"], j["Q"], j["tp"], j["tq"], 0, j["binds"]) for j in jobs]
    assert B.vl_verify_matmul_batched(cj, [B.mat(j["C"]) for j in jobs], 9, res)
    bad = [j["C"].copy() for j in jobs]
    bad[1][0, 0] += 1
    assert not B.vl_verify_matmul_batched(cj, [B.mat(C) for C in bad], 9, res)


def test_batch_lora_projection_grouped_by_inner_dimension():
    """A projection's eight products in three batches (inner d = k, n and r)."""
    t = W.lora_projection(W.GLOBAL_SEED, 0, "q", 32, 64, 64, 8)
    prods = W.projection_products(t)
    groups = {}
    for j in prods:
        groups.setdefault(W.op_shape(j)[1], []).append(j)
    assert sorted(groups) == [8, 32, 64]
    for kk, jobs in groups.items():
        res = gpu_batch(jobs, seed=kk)
        assert res.to_bytes() == OB.prove_matmul_batch(jobs, seed=kk).to_bytes()


def test_batch_of_64():
    rng = np.random.default_rng(6)
    jobs = []
    for i in range(64):
        A, Bm = _rand(rng, (8 + i % 5, 96)), _rand(rng, (96, 3 + i % 7))
        jobs.append({"P": A, "Q": Bm, "tp": 0, "tq": 0})
    res = gpu_batch(jobs, seed=1)
    assert res.to_bytes() == OB.prove_matmul_batch(jobs, seed=1).to_bytes()


def test_claims_plan_reruns_rebinds_device_output():
    import ctypes
    rng = np.random.default_rng(7)
    jobs = _jobs(rng, 3, 40)
    keep, cj = [], []
    for i, j in enumerate(jobs):
        P = j["P"] if i == 0 else torch.from_numpy(np.ascontiguousarray(j["P"])).cuda()  # one host operand
        Q = torch.from_numpy(np.ascontiguousarray(j["Q"])).cuda()
        keep += [P, Q]
        cj.append(B.job(P, Q, j["tp"], j["tq"], 0, j["binds"]))
    want = OB.prove_matmul_batch(jobs, seed=11).to_bytes()
    plan = B.ClaimsPlan(cj, 11)
    n = plan.workspace_bytes()
    ws1 = torch.empty(n, dtype=torch.uint8, device="cuda")
    ws2 = torch.empty(n, dtype=torch.uint8, device="cuda")
    for ws in (ws1, ws1, ws2, ws1):
        assert plan.run(ws.data_ptr(), n).to_bytes() == want
    K = len(jobs)
    dproof = torch.empty(ctypes.sizeof(B.vl_batch_proof), dtype=torch.uint8, device="cuda")
    dvals = torch.empty(3 * K * 32, dtype=torch.uint8, device="cuda")
    base = dvals.data_ptr()
    plan.run(ws2.data_ptr(), n, device_out=(dproof.data_ptr(), base, base + K * 32, base + 2 * K * 32))
    torch.cuda.synchronize()
    res = B.BatchedProof(K)
    ctypes.memmove(ctypes.addressof(res.proof), dproof.cpu().numpy().tobytes(), ctypes.sizeof(B.vl_batch_proof))
    raw = dvals.cpu().numpy().tobytes()
    ctypes.memmove(ctypes.addressof(res.claims), raw[:K * 32], K * 32)
    ctypes.memmove(ctypes.addressof(res.a), raw[K * 32:2 * K * 32], K * 32)
    ctypes.memmove(ctypes.addressof(res.b), raw[2 * K * 32:], K * 32)
    assert res.to_bytes() == want
    plan.destroy()


def test_batch_long_inner_dimension():
    """k = 2^16 + 8: 17 rounds, folds over 65544 lines, a ragged last round."""
    rng = np.random.default_rng(8)
    k = (1 << 16) + 8
    jobs = []
    for i in range(2):
        A, Bm = _rand(rng, (3 + i, k)), _rand(rng, (k, 2 + i))
        jobs.append({"P": A, "Q": Bm, "tp": 0, "tq": 0})
    res = gpu_batch(jobs, seed=3)
    assert res.proof.d1 == 17
    assert res.to_bytes() == OB.prove_matmul_batch(jobs, seed=3).to_bytes()
