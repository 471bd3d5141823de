"""CPU tests of the batched-claim boundary: workspace sizing and argument
checks, and the library's host verifier against proofs made by the oracle.
No GPU is touched."""
import os

import numpy as np
import pytest

from oracle import batch as OB
from paper_2508_21393_gb300 import binding as B


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(B.LIB_PATH):
        from paper_2508_21393_gb300 import build
        build.build(quiet=True)
    return B.lib()


def _rand(rng, shape):
    return rng.integers(-(1 << 15), 1 << 15, size=shape).astype(np.int16)


def _jobs(rng, K, k):
    out = []
    for i in range(K):
        m, n, tp, tq = 3 + i, 2 + 2 * i, i % 2, (i // 2) % 2
        A, Bm = _rand(rng, (m, k)), _rand(rng, (k, n))
        P = np.ascontiguousarray(A.T) if tp else A
        Q = np.ascontiguousarray(Bm.T) if tq else Bm
        binds = (bytes([i]) * 32, bytes(32), bytes([7]) * 32)
        out.append({"P": P, "Q": Q, "tp": tp, "tq": tq, "binds": binds, "C": A.astype(np.int64) @ Bm})
    return out


def _c_jobs(jobs):
    return [B.job(j["P"], j["Q"], j["tp"], j["tq"], 0, j["binds"]) for j in jobs]


def to_c(p):
    r = B.BatchedProof(p.K)
    r.proof.K, r.proof.k, r.proof.d1, r.proof.status = p.K, p.k, p.d1, 0
    for t, g in enumerate(p.rounds):
        for q in range(3):
            r.proof.g[t][q] = B.fr(g[q])
    for i in range(p.K):
        r.claims[i], r.a[i], r.b[i] = B.fr(p.claims[i]), B.fr(p.a[i]), B.fr(p.b[i])
    for i, x in enumerate(p.state):
        r.proof.state[i] = x
    return r


def test_workspace_sizing(L):
    rng = np.random.default_rng(0)
    jobs = _jobs(rng, 3, 9)
    assert B.vl_batch_workspace_bytes(_c_jobs(jobs)) > 0
    # inner dimensions differ
    other = _jobs(rng, 1, 10)
    assert B.vl_batch_workspace_bytes(_c_jobs(jobs + other)) == 0
    assert B.vl_batch_workspace_bytes([]) == 0


@pytest.mark.parametrize("K,k", [(1, 1), (1, 6), (3, 9), (5, 16)])
def test_host_verifier_accepts_oracle_proofs(L, K, k):
    rng = np.random.default_rng(K * 100 + k)
    jobs = _jobs(rng, K, k)
    p = OB.prove_matmul_batch(jobs, seed=7)
    r = to_c(p)
    assert r.to_bytes() == p.to_bytes()
    Cs = [B.mat(j["C"]) for j in jobs]
    assert B.vl_verify_matmul_batched(_c_jobs(jobs), Cs, 7, r)


def test_host_verifier_rejections(L):
    rng = np.random.default_rng(3)
    jobs = _jobs(rng, 4, 12)
    p = OB.prove_matmul_batch(jobs, seed=2)
    cj = _c_jobs(jobs)
    Cs = [B.mat(j["C"]) for j in jobs]
    assert B.vl_verify_matmul_batched(cj, Cs, 2, to_c(p))
    for name in ("claims", "a", "b"):
        for i in range(4):
            r = to_c(p)
            getattr(r, name)[i] = B.fr(getattr(p, name)[i] + 1)
            assert not B.vl_verify_matmul_batched(cj, Cs, 2, r)
    for t in range(p.d1):
        for q in range(3):
            r = to_c(p)
            r.proof.g[t][q] = B.fr(p.rounds[t][q] + 1)
            assert not B.vl_verify_matmul_batched(cj, Cs, 2, r)
    r = to_c(p)
    r.proof.state[3] ^= 1
    assert not B.vl_verify_matmul_batched(cj, Cs, 2, r)
    assert not B.vl_verify_matmul_batched(cj, Cs, 3, to_c(p))
    bad = [j["C"].copy() for j in jobs]
    bad[2][1, 1] += 1
    assert not B.vl_verify_matmul_batched(cj, [B.mat(C) for C in bad], 2, to_c(p))


def test_host_verifier_argument_errors(L):
    rng = np.random.default_rng(4)
    jobs = _jobs(rng, 2, 6)
    Cs = [B.mat(j["C"]) for j in jobs]
    r = B.BatchedProof(2)
    # inner dimensions differ
    other = _jobs(rng, 1, 7)
    with pytest.raises(B.VLError):
        B.vl_verify_matmul_batched(_c_jobs(jobs[:1] + other), Cs[:1] + [B.mat(other[0]["C"])], 0, r)
    # a claimed product of the wrong shape
    with pytest.raises(B.VLError):
        B.vl_verify_matmul_batched(_c_jobs(jobs), [Cs[1], Cs[0]], 0, r)
    # a zeroed proof of a valid statement is simply rejected
    assert not B.vl_verify_matmul_batched(_c_jobs(jobs), Cs, 0, r)
