"""Golden proofs (tests/golden/proofs_small.json, written by
tests/golden/make_golden.py from the oracle): the oracle still produces the
stored bytes for every proof kind, and the library's host verifiers accept
the stored proofs and reject a flipped byte.  This freezes the project's own
transcript formats."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2508_21393_gb300 import binding as B

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def golden():
    with open(os.path.join(HERE, "golden", "proofs_small.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(B.LIB_PATH):
        from paper_2508_21393_gb300 import build
        build.build(quiet=True)
    return B.lib()


def _a(x):
    return np.ascontiguousarray(np.array(x, dtype=np.int16))


def _fr_list(raw, n):
    return [int.from_bytes(raw[32 * i:32 * i + 32], "little") for i in range(n)]


def test_oracle_reproduces_the_golden_bytes(golden):
    g = golden["matmul"]
    assert oracle.prove_matmul(_a(g["P"]), _a(g["Q"]), g["tp"], g["tq"], seed=g["seed"]).to_bytes().hex() == g["proof"]
    g = golden["linear"]
    assert oracle.prove_linear([_a(m) for m in g["mats"]], g["coeffs"], seed=g["seed"]).to_bytes().hex() == g["proof"]
    g = golden["lookup"]
    assert oracle.prove_lookup(_a(g["S"]), g["t0"], g["log2_n"], seed=g["seed"]).to_bytes().hex() == g["proof"]
    g = golden["batch"]
    jobs = [{"P": _a(j["P"]), "Q": _a(j["Q"]), "tp": 0, "tq": 0} for j in g["jobs"]]
    assert oracle.prove_matmul_batch(jobs, seed=g["seed"]).to_bytes().hex() == g["proof"]


def _matmul_proof(raw):
    p = B.vl_proof()
    p.m, p.k, p.n, p.d0, p.d1, p.d2 = (int.from_bytes(raw[4 * i:4 * i + 4], "little") for i in range(6))
    off = 24
    p.c = B.fr(int.from_bytes(raw[off:off + 32], "little"))
    off += 32
    for t in range(p.d1):
        for q in range(3):
            p.g[t][q] = B.fr(int.from_bytes(raw[off:off + 32], "little"))
            off += 32
    p.a_r = B.fr(int.from_bytes(raw[off:off + 32], "little"))
    p.b_r = B.fr(int.from_bytes(raw[off + 32:off + 64], "little"))
    for i in range(32):
        p.state[i] = raw[off + 64 + i]
    return p


def test_host_verifiers_accept_golden_proofs(L, golden):
    # matmul
    g = golden["matmul"]
    P, Q = _a(g["P"]), _a(g["Q"])
    C = np.ascontiguousarray(P.T.astype(np.int64) @ Q.astype(np.int64))  # kept alive: B.mat holds its pointer
    raw = bytes.fromhex(g["proof"])
    fs = B.fs_init(g["seed"])
    assert B.vl_verify_matmul(B.mat(P, 1), B.mat(Q), B.mat(C), fs, _matmul_proof(raw))
    bad = bytearray(raw)
    bad[-1] ^= 1
    assert not B.vl_verify_matmul(B.mat(P, 1), B.mat(Q), B.mat(C), fs, _matmul_proof(bytes(bad)))
    # linear
    g = golden["linear"]
    mats = [_a(m) for m in g["mats"]]
    raw = bytes.fromhex(g["proof"])
    lp = B.vl_lin_proof()
    lp.rows, lp.cols, lp.d0, lp.d1, lp.nmats = (int.from_bytes(raw[4 * i:4 * i + 4], "little") for i in range(5))
    for q, e in enumerate(_fr_list(raw[20:], lp.nmats)):
        lp.evals[q] = B.fr(e)
    for i in range(32):
        lp.state[i] = raw[20 + 32 * lp.nmats + i]
    assert B.lin_proof_bytes(lp) == raw
    job = B.lin_job([B.mat(m) for m in mats], g["coeffs"], g["seed"])
    assert B.vl_verify_linear(job, lp)
    lp.state[0] ^= 1
    assert not B.vl_verify_linear(job, lp)
    # lookup
    g = golden["lookup"]
    raw = bytes.fromhex(g["proof"])
    kp = B.vl_lookup_proof()
    kp.n, kp.log2_d, kp.log2_n = (int.from_bytes(raw[4 * i:4 * i + 4], "little") for i in range(3))
    kp.t0 = int.from_bytes(raw[12:20], "little", signed=True)
    off = 20
    for t in range(kp.log2_d):
        for q, v in enumerate(_fr_list(raw[off:], 4)):
            kp.g[t][q] = B.fr(v)
        off += 128
    kp.a_r, kp.s_r, kp.b_r, kp.m_r = (B.fr(v) for v in _fr_list(raw[off:], 4))
    for i in range(32):
        kp.state[i] = raw[off + 128 + i]
    assert B.lookup_proof_bytes(kp) == raw
    S = _a(g["S"]).reshape(1, -1)
    kj = B.lookup_job(B.mat(S), g["t0"], g["log2_n"], g["seed"])
    assert B.vl_verify_lookup(kj, kp)
    kp.state[0] ^= 1
    assert not B.vl_verify_lookup(kj, kp)
    # batch
    g = golden["batch"]
    raw = bytes.fromhex(g["proof"])
    K, k, d1 = (int.from_bytes(raw[4 * i:4 * i + 4], "little") for i in range(3))
    res = B.BatchedProof(K)
    res.proof.K, res.proof.k, res.proof.d1 = K, k, d1
    off = 12
    for i, v in enumerate(_fr_list(raw[off:], K)):
        res.claims[i] = B.fr(v)
    off += 32 * K
    for t in range(d1):
        for q, v in enumerate(_fr_list(raw[off:], 3)):
            res.proof.g[t][q] = B.fr(v)
        off += 96
    for i in range(K):
        res.a[i] = B.fr(int.from_bytes(raw[off:off + 32], "little"))
        res.b[i] = B.fr(int.from_bytes(raw[off + 32:off + 64], "little"))
        off += 64
    for i in range(32):
        res.proof.state[i] = raw[off + i]
    assert res.to_bytes() == raw
    ops = [(_a(j["P"]), _a(j["Q"])) for j in g["jobs"]]  # kept alive: the descriptors hold their pointers
    prods = [np.ascontiguousarray(P.astype(np.int64) @ Q.astype(np.int64)) for P, Q in ops]
    jobs = [B.job(P, Q, 0, 0, 0) for P, Q in ops]
    Cs = [B.mat(C) for C in prods]
    assert B.vl_verify_matmul_batched(jobs, Cs, g["seed"], res)
    res.proof.state[0] ^= 1
    assert not B.vl_verify_matmul_batched(jobs, Cs, g["seed"], res)
