"""The host verifiers take proofs from untrusted provers.  Fed an honest
proof (made by the oracle) with one random bit flipped anywhere in the C
structures -- header fields, unused round slots, padding, the batch's claim
arrays -- or a structure of random bytes, each verifier returns VL_OK or
VL_REJECT and never crashes; it accepts exactly when every field it reads
(the proof's canonical bytes and its status) is unchanged."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

FLIPS = 300


@pytest.fixture(scope="module")
def L():
    import os
    if not os.path.exists(B.LIB_PATH):
        from paper_2508_21393_gb300 import build
        build.build(quiet=True)
    return B.lib()


def _flip(struct, rng):
    """A copy of a ctypes structure with one random bit flipped."""
    raw = bytearray(bytes(struct))
    i = int(rng.integers(len(raw)))
    raw[i] ^= 1 << int(rng.integers(8))
    return type(struct).from_buffer_copy(bytes(raw))


def _random(cls, rng):
    return cls.from_buffer_copy(rng.integers(0, 256, size=ctypes.sizeof(cls), dtype=np.uint8).tobytes())


def _rand16(rng, shape):
    return rng.integers(-(1 << 15), 1 << 15, size=shape).astype(np.int16)


def test_matmul_verifier(L):
    rng = np.random.default_rng(101)
    P, Q = _rand16(rng, (5, 13)), _rand16(rng, (13, 6))
    C = W.exact_matmul(P, Q).astype(np.int64)
    pf = oracle.prove_matmul(P, Q, 0, 0, seed=11)
    H = B.vl_proof()
    H.m, H.k, H.n, H.d0, H.d1, H.d2, H.status = pf.m, pf.k, pf.n, pf.d0, pf.d1, pf.d2, 0
    H.c, H.a_r, H.b_r = B.fr(pf.c), B.fr(pf.a_r), B.fr(pf.b_r)
    for t, g in enumerate(pf.g):
        for q in range(3):
            H.g[t][q] = B.fr(g[q])
    for i in range(32):
        H.state[i] = pf.state[i]
    want = pf.to_bytes()
    args = (B.mat(P), B.mat(Q), B.mat(C), B.fs_init(11))
    assert L.vl_verify_matmul(*(ctypes.byref(a) for a in args), ctypes.byref(H)) == B.VL_OK
    header = lambda p: (p.m, p.k, p.n, p.d0, p.d1, p.d2)
    accepted = 0
    for _ in range(FLIPS):
        M = _flip(H, rng)
        code = L.vl_verify_matmul(*(ctypes.byref(a) for a in args), ctypes.byref(M))
        same = header(M) == header(H) and M.status == 0 and B.proof_bytes(M) == want
        assert code == (B.VL_OK if same else B.VL_REJECT)
        accepted += same
    assert 0 < accepted < FLIPS  # flips land in unused round slots and in read fields
    for _ in range(50):
        assert L.vl_verify_matmul(*(ctypes.byref(a) for a in args), ctypes.byref(_random(B.vl_proof, rng))) \
            == B.VL_REJECT


def test_linear_verifier(L):
    rng = np.random.default_rng(102)
    A = rng.integers(-(1 << 14), 1 << 14, size=(6, 9)).astype(np.int16)
    G = rng.integers(-(1 << 13), 1 << 13, size=(6, 9)).astype(np.int16)
    A2 = (A.astype(np.int32) - G).astype(np.int16)  # no wrap-around: |A - G| < 2^15
    mats = [A2, A, G]
    pf = oracle.prove_linear(mats, [1, -1, 1], seed=12)
    H = B.vl_lin_proof()
    H.rows, H.cols, H.d0, H.d1, H.nmats, H.status = pf.rows, pf.cols, pf.d0, pf.d1, len(pf.evals), 0
    for q, e in enumerate(pf.evals):
        H.evals[q] = B.fr(e)
    for i in range(32):
        H.state[i] = pf.state[i]
    want = pf.to_bytes()
    job = B.lin_job([B.mat(m) for m in mats], [1, -1, 1], 12)
    assert L.vl_verify_linear(ctypes.byref(job), ctypes.byref(H)) == B.VL_OK
    header = lambda p: (p.rows, p.cols, p.d0, p.d1, p.nmats)
    for _ in range(FLIPS):
        M = _flip(H, rng)
        code = L.vl_verify_linear(ctypes.byref(job), ctypes.byref(M))
        same = header(M) == header(H) and M.status == 0 and B.lin_proof_bytes(M) == want
        assert code == (B.VL_OK if same else B.VL_REJECT)
    for _ in range(50):
        assert L.vl_verify_linear(ctypes.byref(job), ctypes.byref(_random(B.vl_lin_proof, rng))) == B.VL_REJECT


def test_lookup_verifier(L):
    rng = np.random.default_rng(103)
    S = rng.integers(-8, 24, size=(5, 7)).astype(np.int16)
    pf = oracle.prove_lookup(S, -8, 5, seed=13)
    H = B.vl_lookup_proof()
    H.n, H.log2_d, H.log2_n, H.t0, H.status = pf.n, pf.log2_d, pf.log2_n, pf.t0, 0
    for t, g in enumerate(pf.rounds):
        for q in range(4):
            H.g[t][q] = B.fr(g[q])
    H.a_r, H.s_r, H.b_r, H.m_r = B.fr(pf.a_r), B.fr(pf.s_r), B.fr(pf.b_r), B.fr(pf.m_r)
    for i in range(32):
        H.state[i] = pf.state[i]
    want = pf.to_bytes()
    job = B.lookup_job(B.mat(S), -8, 5, 13)
    assert L.vl_verify_lookup(ctypes.byref(job), ctypes.byref(H)) == B.VL_OK
    header = lambda p: (p.n, p.log2_d, p.log2_n, p.t0)
    for _ in range(FLIPS):
        M = _flip(H, rng)
        code = L.vl_verify_lookup(ctypes.byref(job), ctypes.byref(M))
        same = header(M) == header(H) and M.status == 0 and B.lookup_proof_bytes(M) == want
        assert code == (B.VL_OK if same else B.VL_REJECT)
    for _ in range(50):
        assert L.vl_verify_lookup(ctypes.byref(job), ctypes.byref(_random(B.vl_lookup_proof, rng))) == B.VL_REJECT


def test_batched_verifier(L):
    rng = np.random.default_rng(104)
    ops = [(_rand16(rng, (3 + i, 8)), _rand16(rng, (8, 2 + i))) for i in range(3)]
    pf = oracle.prove_matmul_batch([{"P": P, "Q": Q, "tp": 0, "tq": 0} for P, Q in ops], seed=14)
    K = len(ops)
    H = B.BatchedProof(K)
    H.proof.K, H.proof.k, H.proof.d1, H.proof.status = pf.K, pf.k, pf.d1, 0
    for t, g in enumerate(pf.rounds):
        for q in range(3):
            H.proof.g[t][q] = B.fr(g[q])
    for i in range(32):
        H.proof.state[i] = pf.state[i]
    for i in range(K):
        H.claims[i], H.a[i], H.b[i] = B.fr(pf.claims[i]), B.fr(pf.a[i]), B.fr(pf.b[i])
    want = pf.to_bytes()
    assert H.to_bytes() == want
    prods = [W.exact_matmul(P, Q).astype(np.int64) for P, Q in ops]
    jobs = [B.job(P, Q, 0, 0, 0) for P, Q in ops]
    Cs = [B.mat(C) for C in prods]
    assert B.vl_verify_matmul_batched(jobs, Cs, 14, H)
    parts = ("proof", "claims", "a", "b")
    for _ in range(FLIPS):
        M = B.BatchedProof(K)
        for name in parts:
            setattr(M, name, type(getattr(H, name)).from_buffer_copy(bytes(getattr(H, name))))
        name = parts[int(rng.integers(4))] if rng.random() < 0.5 else "proof"
        setattr(M, name, _flip(getattr(M, name), rng))
        same = (M.proof.K, M.proof.k, M.proof.d1) == (K, pf.k, pf.d1) and M.proof.status == 0 and \
            M.to_bytes() == want
        assert B.vl_verify_matmul_batched(jobs, Cs, 14, M) == same
    for _ in range(50):
        M = B.BatchedProof(K)
        M.proof = _random(B.vl_batch_proof, rng)
        assert not B.vl_verify_matmul_batched(jobs, Cs, 14, M)
