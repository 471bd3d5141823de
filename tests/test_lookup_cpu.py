"""CPU tests of the lookup-argument boundary (Protocol 1): workspace sizing
and argument checks that fail before any CUDA call, and the library's host
verifier against proofs made by the oracle.  No GPU is touched."""
import copy
import os

import numpy as np
import pytest

from oracle import lookup as OL
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(B.LIB_PATH):
        from paper_2508_21393_gb300 import build
        build.build(quiet=True)
    return B.lib()


def _job(S, t0, ln, seed=0, bind=None):
    S2 = np.ascontiguousarray(S.reshape(S.shape[0], -1) if S.ndim == 2 else S.reshape(1, -1))
    return B.lookup_job(B.mat(S2), t0, ln, seed, bind)


def to_c(p):
    c = B.vl_lookup_proof()
    c.n, c.log2_d, c.log2_n, c.t0, c.status = p.n, p.log2_d, p.log2_n, p.t0, 0
    for t, g in enumerate(p.rounds):
        for q in range(4):
            c.g[t][q] = B.fr(g[q])
    c.a_r, c.s_r, c.b_r, c.m_r = B.fr(p.a_r), B.fr(p.s_r), B.fr(p.b_r), B.fr(p.m_r)
    for i, b in enumerate(p.state):
        c.state[i] = b
    return c


def test_workspace_sizing_and_argument_errors(L):
    S = np.zeros((40, 30), np.int16)
    assert B.vl_lookup_workspace_bytes([_job(S, 0, 8)]) > 0
    assert B.vl_lookup_workspace_bytes([_job(S, 0, 8)] * 3) > B.vl_lookup_workspace_bytes([_job(S, 0, 8)])
    assert B.vl_lookup_workspace_bytes([_job(S, 0, B.VL_LOOKUP_MAX_LOG_N + 1)]) == 0
    assert B.vl_lookup_workspace_bytes([_job(S, 0, -1)]) == 0
    j = _job(S, 0, 8)
    j.reserved = 1
    assert B.vl_lookup_workspace_bytes([j]) == 0
    j = _job(S, 0, 8)
    j.S.trans = 1
    assert B.vl_lookup_workspace_bytes([j]) == 0
    assert B.vl_lookup_workspace_bytes([_job(S.astype(np.int64), 0, 8)]) == 0  # int16 only on the GPU
    big = B.vl_mat()
    big.data, big.rows, big.cols, big.ld, big.dtype, big.space = 256, 1 << 13, (1 << 11) + 1, (1 << 11) + 1, 1, 0
    assert B.vl_lookup_workspace_bytes([B.lookup_job(big, 0, 8)]) == 0  # more than 2^24 entries
    big.rows = big.cols = big.ld = 1 << 40  # rows * cols would overflow int64
    assert B.vl_lookup_workspace_bytes([B.lookup_job(big, 0, 8)]) == 0
    assert B.vl_lookup_workspace_bytes([_job(S, (1 << 40) + 1, 8)]) == 0
    assert B.vl_lookup_workspace_bytes([_job(S, -(1 << 40) - 1, 8)]) == 0
    assert B.vl_lookup_workspace_bytes([_job(S, -(1 << 40), 8)]) > 0
    assert B.vl_lookup_workspace_bytes([]) == 0
    with pytest.raises(B.VLError):
        B.LookupPlan([_job(S, 0, 17)])
    arr = B.lookup_jobs_array([_job(S, 0, 8)])
    out = (B.vl_lookup_proof * 1)()
    n = B.vl_lookup_workspace_bytes([_job(S, 0, 8)])
    assert L.vl_prove_lookup(arr, 1, None, n, out, None) == B.VL_EINVAL
    assert L.vl_prove_lookup(arr, 1, 256 + 8, n, out, None) == B.VL_EINVAL
    assert L.vl_prove_lookup(arr, 1, 256, n - 1, out, None) == B.VL_ENOMEM
    assert B.vl_strerror(B.VL_ELOOKUP) == "a lookup value lies outside its table"


CASES = [((7, 9), 4, 0), ((1,), 0, 3), ((33,), 5, -16), ((4, 64), 8, 0), ((3, 3), 4, 0), ((2, 2), 1, 5),
         ((100,), 2, 0)]


@pytest.mark.parametrize("shape,ln,t0", CASES)
def test_host_verifier_accepts_oracle_proofs(L, shape, ln, t0):
    rng = np.random.default_rng(sum(shape) * 7 + ln)
    S = rng.integers(t0, t0 + (1 << ln), size=shape).astype(np.int16)
    bind = bytes([ln]) * 32
    p = OL.prove_lookup(S, t0, ln, seed=5, bind=bind)
    c = to_c(p)
    assert B.lookup_proof_bytes(c) == p.to_bytes()
    assert B.vl_verify_lookup(_job(S, t0, ln, 5, bind), c)
    # the same values as int64 give the same verdict
    S64 = np.ascontiguousarray(S.reshape(S.shape[0], -1) if S.ndim == 2 else S.reshape(1, -1)).astype(np.int64)
    assert B.vl_verify_lookup(B.lookup_job(B.mat(S64), t0, ln, 5, bind), c)


def test_host_verifier_rejections(L):
    rng = np.random.default_rng(4)
    S = rng.integers(0, 64, size=(5, 40)).astype(np.int16)
    p = OL.prove_lookup(S, 0, 6, seed=3)
    job = _job(S, 0, 6, 3)
    assert B.vl_verify_lookup(job, to_c(p))
    for t in range(p.log2_d):
        for q in range(4):
            c = to_c(p)
            c.g[t][q] = B.fr(p.rounds[t][q] + 1)
            assert not B.vl_verify_lookup(job, c)
    for name in ("a_r", "s_r", "b_r", "m_r"):
        c = to_c(p)
        setattr(c, name, B.fr(getattr(p, name) + 1))
        assert not B.vl_verify_lookup(job, c)
    c = to_c(p)
    c.state[0] ^= 1
    assert not B.vl_verify_lookup(job, c)
    c = to_c(p)
    c.status = B.VL_ELOOKUP
    assert not B.vl_verify_lookup(job, c)
    assert not B.vl_verify_lookup(_job(S, 0, 6, 4), to_c(p))
    assert not B.vl_verify_lookup(_job(S, 0, 6, 3, b"\x01" * 32), to_c(p))
    assert not B.vl_verify_lookup(_job(S, 0, 7, 3), to_c(p))
    S2 = S.copy()
    S2[1, 1] = (S2[1, 1] + 1) % 64
    assert not B.vl_verify_lookup(_job(S2, 0, 6, 3), to_c(p))
    S3 = S.copy()
    S3[0, 0] = 64  # outside the table
    assert not B.vl_verify_lookup(_job(S3, 0, 6, 3), to_c(p))


def test_rescale_lookup_statements_hold():
    """The workload's remainders satisfy z + 2^(s-1) = 2^s z' + rho with rho
    in the table (so their lookups must verify)."""
    t = W.lora_projection(W.GLOBAL_SEED, 0, "q", 32, 64, 48, 8)
    looks = W.rescale_lookups(t)
    assert [x["log2_n"] for x in looks] == [8, 8, 12, 12]
    Z = W.exact_matmul(t["X"], t["A"])
    rho = looks[0]["S"].astype(np.int64)
    assert np.array_equal(Z + 128, ((Z + 128) >> 8) * 256 + rho)
    for x in looks:
        assert x["S"].min() >= 0 and x["S"].max() < (1 << x["log2_n"])


def test_host_verifier_argument_errors(L):
    S = np.zeros((3, 4), np.int16)
    p = B.vl_lookup_proof()
    j = _job(S, 0, 4)
    j.S.trans = 1
    with pytest.raises(B.VLError):
        B.vl_verify_lookup(j, p)
    j = _job(S, 0, 4)
    j.log2_n = 17
    with pytest.raises(B.VLError):
        B.vl_verify_lookup(j, p)
    j = _job(S, 0, 4)
    j.reserved = 2
    with pytest.raises(B.VLError):
        B.vl_verify_lookup(j, p)
    for t0 in ((1 << 40) + 1, -(1 << 40) - 1):  # the prover's bound on the table's offset
        with pytest.raises(B.VLError) as ei:
            B.vl_verify_lookup(_job(S, t0, 4), p)
        assert ei.value.code == B.VL_EINVAL
    big = B.vl_mat()
    big.data, big.rows, big.cols, big.ld, big.dtype, big.space = 256, 1 << 40, 1 << 40, 1 << 40, B.VL_I16, B.VL_HOST
    with pytest.raises(B.VLError) as ei:  # more than 2^24 entries; rows * cols would overflow int64
        B.vl_verify_lookup(B.lookup_job(big, 0, 4), p)
    assert ei.value.code == B.VL_ESHAPE
    # a zeroed proof of a valid statement is simply rejected
    assert not B.vl_verify_lookup(_job(S, 0, 4), p)
