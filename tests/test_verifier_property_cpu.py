"""Property tests (hypothesis) of the library's host verifiers against the
oracle over random small statements: every oracle proof of a true statement
is accepted, and the same proof is rejected for a statement that differs in
one entry (a false product, a broken relation, a value outside the table)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")
settings = hyp.settings(max_examples=25, deadline=None, derandomize=True)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_2508_21393_gb300 import build
        build.build(quiet=True)
    return B.lib()


def _vl_proof(pf):
    out = B.vl_proof()
    out.m, out.k, out.n, out.d0, out.d1, out.d2, out.status = pf.m, pf.k, pf.n, pf.d0, pf.d1, pf.d2, 0
    out.c, out.a_r, out.b_r = B.fr(pf.c), B.fr(pf.a_r), B.fr(pf.b_r)
    for t, g in enumerate(pf.g):
        for q in range(3):
            out.g[t][q] = B.fr(g[q])
    for i in range(32):
        out.state[i] = pf.state[i]
    return out


@settings
@hyp.given(m=st.integers(1, 9), k=st.integers(1, 17), n=st.integers(1, 9), tp=st.integers(0, 1),
           tq=st.integers(0, 1), seed=st.integers(0, 2**64 - 1), data=st.integers(0, 2**32 - 1))
def test_matmul(m, k, n, tp, tq, seed, data):
    rng = np.random.default_rng(data)
    A = rng.integers(-(1 << 15), 1 << 15, size=(m, k)).astype(np.int16)
    Bm = rng.integers(-(1 << 15), 1 << 15, size=(k, n)).astype(np.int16)
    P = np.ascontiguousarray(A.T) if tp else A
    Q = np.ascontiguousarray(Bm.T) if tq else Bm
    C = W.exact_matmul(A, Bm).astype(np.int64)
    vp = _vl_proof(oracle.prove_matmul(P, Q, tp, tq, seed=seed))
    assert B.vl_verify_matmul(B.mat(P, tp), B.mat(Q, tq), B.mat(C), B.fs_init(seed), vp)
    C2 = C.copy()
    C2[rng.integers(m), rng.integers(n)] += 1
    assert not B.vl_verify_matmul(B.mat(P, tp), B.mat(Q, tq), B.mat(C2), B.fs_init(seed), vp)


@settings
@hyp.given(rows=st.integers(1, 9), cols=st.integers(1, 9), q=st.integers(1, 5), seed=st.integers(0, 2**64 - 1),
           data=st.integers(0, 2**32 - 1))
def test_linear(rows, cols, q, seed, data):
    """sum_i c_i M_i = 0 with the last matrix chosen to make it hold (c_q = 1)."""
    rng = np.random.default_rng(data)
    coeffs = [int(c) for c in rng.integers(-3, 4, size=q - 1)] + [1]
    mats = [rng.integers(-100, 100, size=(rows, cols)).astype(np.int16) for _ in range(q - 1)]
    last = -sum((c * m.astype(np.int64) for c, m in zip(coeffs, mats)), np.zeros((rows, cols), np.int64))
    mats.append(last.astype(np.int16))
    pf = oracle.prove_linear(mats, coeffs, seed=seed)
    lp = B.vl_lin_proof()
    lp.rows, lp.cols, lp.d0, lp.d1, lp.nmats, lp.status = pf.rows, pf.cols, pf.d0, pf.d1, q, 0
    for i, e in enumerate(pf.evals):
        lp.evals[i] = B.fr(e)
    for i in range(32):
        lp.state[i] = pf.state[i]
    assert B.vl_verify_linear(B.lin_job([B.mat(m) for m in mats], coeffs, seed), lp)
    bad = [m.copy() for m in mats]
    bad[-1][rng.integers(rows), rng.integers(cols)] += 1
    assert not B.vl_verify_linear(B.lin_job([B.mat(m) for m in bad], coeffs, seed), lp)


@settings
@hyp.given(n=st.integers(1, 70), ln=st.integers(0, 7), t0=st.integers(-300, 300), seed=st.integers(0, 2**64 - 1),
           data=st.integers(0, 2**32 - 1))
def test_lookup(n, ln, t0, seed, data):
    rng = np.random.default_rng(data)
    S = rng.integers(t0, t0 + (1 << ln), size=(1, n)).astype(np.int16)
    pf = oracle.prove_lookup(S, t0, ln, seed=seed)
    kp = B.vl_lookup_proof()
    kp.n, kp.log2_d, kp.log2_n, kp.t0, kp.status = pf.n, pf.log2_d, pf.log2_n, pf.t0, 0
    for t, g in enumerate(pf.rounds):
        for i in range(4):
            kp.g[t][i] = B.fr(g[i])
    kp.a_r, kp.s_r, kp.b_r, kp.m_r = B.fr(pf.a_r), B.fr(pf.s_r), B.fr(pf.b_r), B.fr(pf.m_r)
    for i in range(32):
        kp.state[i] = pf.state[i]
    assert B.vl_verify_lookup(B.lookup_job(B.mat(S), t0, ln, seed), kp)
    bad = S.copy()
    bad[0, rng.integers(n)] = t0 + (1 << ln)  # one past the table's end
    assert not B.vl_verify_lookup(B.lookup_job(B.mat(bad), t0, ln, seed), kp)


@settings
@hyp.given(K=st.integers(1, 5), k=st.integers(1, 12), seed=st.integers(0, 2**64 - 1), data=st.integers(0, 2**32 - 1))
def test_batched(K, k, seed, data):
    rng = np.random.default_rng(data)
    ops = [(rng.integers(-(1 << 15), 1 << 15, size=(int(rng.integers(1, 6)), k)).astype(np.int16),
            rng.integers(-(1 << 15), 1 << 15, size=(k, int(rng.integers(1, 6)))).astype(np.int16)) for _ in range(K)]
    pf = oracle.prove_matmul_batch([{"P": P, "Q": Q, "tp": 0, "tq": 0} for P, Q in ops], seed=seed)
    res = B.BatchedProof(K)
    res.proof.K, res.proof.k, res.proof.d1, res.proof.status = pf.K, pf.k, pf.d1, 0
    for t, g in enumerate(pf.rounds):
        for i in range(3):
            res.proof.g[t][i] = B.fr(g[i])
    for i in range(32):
        res.proof.state[i] = pf.state[i]
    for i in range(K):
        res.claims[i], res.a[i], res.b[i] = B.fr(pf.claims[i]), B.fr(pf.a[i]), B.fr(pf.b[i])
    jobs = [B.job(P, Q, 0, 0, 0) for P, Q in ops]
    prods = [W.exact_matmul(P, Q).astype(np.int64) for P, Q in ops]
    assert B.vl_verify_matmul_batched(jobs, [B.mat(C) for C in prods], seed, res)
    j = int(rng.integers(K))
    prods[j][0, 0] += 1
    assert not B.vl_verify_matmul_batched(jobs, [B.mat(C) for C in prods], seed, res)
