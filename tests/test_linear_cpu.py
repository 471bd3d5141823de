"""CPU tests of the linear zkMat boundary (sum_q c_q op(M_q) = 0, Sec. IV):
workspace sizing and argument checks that fail before any CUDA call, and the
library's host verifier against proofs made by the oracle.

No GPU is touched.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(B.LIB_PATH):
        from paper_2508_21393_gb300 import build
        build.build(quiet=True)
    return B.lib()


def _rand(rng, shape, lo=-(1 << 15), hi=1 << 15):
    return rng.integers(lo, hi, size=shape).astype(np.int16)


def _host_job(mats, coeffs, seed=0, trans=None, binds=None):
    trans = trans or [0] * len(mats)
    return B.lin_job([B.mat(np.ascontiguousarray(m), t) for m, t in zip(mats, trans)], coeffs, seed, binds)


def _to_c(proof):
    """The oracle's LinearProof as a vl_lin_proof."""
    p = B.vl_lin_proof()
    p.rows, p.cols, p.d0, p.d1, p.nmats = proof.rows, proof.cols, proof.d0, proof.d1, len(proof.evals)
    for q, e in enumerate(proof.evals):
        p.evals[q] = B.fr(e)
    for i, b in enumerate(proof.state):
        p.state[i] = b
    return p


def test_workspace_sizing_and_argument_errors(L):
    rng = np.random.default_rng(0)
    M = [_rand(rng, (40, 24)) for _ in range(3)]
    assert B.vl_linear_workspace_bytes([_host_job(M, [1, -1, 1])]) > 0
    # batch: sizes add up (every proof has its own buffers)
    one = B.vl_linear_workspace_bytes([_host_job(M, [1, -1, 1])])
    assert B.vl_linear_workspace_bytes([_host_job(M, [1, -1, 1])] * 3) > one
    # shapes differ
    assert B.vl_linear_workspace_bytes([_host_job([M[0], _rand(rng, (40, 23))], [1, 1])]) == 0
    # a transpose flag fixes a transposed operand
    assert B.vl_linear_workspace_bytes([_host_job([M[0], np.ascontiguousarray(M[1].T)], [1, 1], trans=[0, 1])]) > 0
    # no matrices, too many matrices
    assert B.vl_linear_workspace_bytes([_host_job([], [])]) == 0
    assert B.vl_linear_workspace_bytes([_host_job([M[0]] * (B.VL_LIN_MAX + 1), [1] * (B.VL_LIN_MAX + 1))]) == 0
    # int64 operands are verifier-only
    assert B.vl_linear_workspace_bytes([_host_job([M[0].astype(np.int64)], [1])]) == 0
    # logical dimension above VL_MAX_REDUCE
    big = np.zeros((1, B.VL_MAX_REDUCE + 1), np.int16)
    assert B.vl_linear_workspace_bytes([_host_job([big], [1])]) == 0
    # reserved field, bad leading dimension
    j = _host_job(M, [1, -1, 1])
    j.reserved = 1
    assert B.vl_linear_workspace_bytes([j]) == 0
    j = _host_job(M, [1, -1, 1])
    j._mats[1].ld = 3
    assert B.vl_linear_workspace_bytes([j]) == 0


def test_prove_rejects_before_any_cuda_call(L):
    rng = np.random.default_rng(1)
    M = [_rand(rng, (9, 33)) for _ in range(2)]
    j = _host_job(M, [1, 1])
    arr = B.lin_jobs_array([j])
    out = (B.vl_lin_proof * 1)()
    n = B.vl_linear_workspace_bytes([j])
    # no workspace, misaligned workspace, workspace too small
    assert L.vl_prove_linear(arr, 1, None, n, out, None) == B.VL_EINVAL
    assert L.vl_prove_linear(arr, 1, 256 + 16, n, out, None) == B.VL_EINVAL
    assert L.vl_prove_linear(arr, 1, 256, n - 1, out, None) == B.VL_ENOMEM
    # a coefficient that is not canonical (>= r)
    j._coeffs[0].limb[7] = 0xFFFFFFFF
    arr = B.lin_jobs_array([j])
    assert L.vl_prove_linear(arr, 1, 256, n, out, None) == B.VL_EINVAL
    # no jobs
    assert L.vl_prove_linear(arr, 0, 256, n, out, None) == B.VL_EINVAL


CASES = [
    # (rows, cols, nmats, transposes)
    (1, 1, 1, [0]),
    (1, 300, 2, [0, 1]),
    (300, 1, 2, [1, 0]),
    (5, 7, 3, [0, 0, 1]),
    (129, 65, 3, [1, 0, 0]),
]


@pytest.mark.parametrize("rows,cols,q,trans", CASES)
def test_host_verifier_accepts_oracle_proofs(L, rows, cols, q, trans):
    """A true relation: M_{q-1} = -(c_0 M_0 + ... ) with small entries so the
    last matrix is int16; the oracle's proof must verify in the library."""
    rng = np.random.default_rng(rows * 1000 + cols)
    mats = [_rand(rng, (rows, cols), -1000, 1000) for _ in range(q - 1)]
    coeffs = [int(c) for c in rng.integers(-5, 6, size=q - 1)]
    last = -sum(c * m.astype(np.int64) for c, m in zip(coeffs, mats)) if mats else np.zeros((rows, cols), np.int64)
    mats.append(last.astype(np.int16))
    coeffs.append(1)
    seed = 77 + rows
    binds = [bytes([q, i]) * 16 for i in range(q)]
    proof = oracle.prove_linear(mats, coeffs, seed=seed, binds=binds)
    assert oracle.verify_linear(mats, coeffs, proof, seed=seed, binds=binds)[0]
    stored = [np.ascontiguousarray(m.T) if t else m for m, t in zip(mats, trans)]
    job = _host_job(stored, coeffs, seed, trans, binds)
    p = _to_c(proof)
    assert B.lin_proof_bytes(p) == proof.to_bytes()
    assert B.vl_verify_linear(job, p)


def test_host_verifier_rejections(L):
    rng = np.random.default_rng(5)
    A = _rand(rng, (6, 10), -2000, 2000)
    G = _rand(rng, (6, 10), -2000, 2000)
    A2 = (A - G).astype(np.int16)
    mats, coeffs, seed = [A2, A, G], [1, -1, 1], 31
    proof = oracle.prove_linear(mats, coeffs, seed=seed)
    job = _host_job(mats, coeffs, seed)
    assert B.vl_verify_linear(job, _to_c(proof))
    # every evaluation perturbed
    for q in range(3):
        p = _to_c(proof)
        p.evals[q] = B.fr(proof.evals[q] + 1)
        assert not B.vl_verify_linear(job, p)
    # non-canonical evaluation (e + r)
    p = _to_c(proof)
    v = proof.evals[0] + B.R_MOD
    if v < 1 << 256:
        for i in range(8):
            p.evals[0].limb[i] = (v >> (32 * i)) & 0xFFFFFFFF
        assert not B.vl_verify_linear(job, p)
    # final state, dimensions, matrix count
    p = _to_c(proof)
    p.state[5] ^= 1
    assert not B.vl_verify_linear(job, p)
    p = _to_c(proof)
    p.d1 += 1
    assert not B.vl_verify_linear(job, p)
    p = _to_c(proof)
    p.status = B.VL_ETIMEOUT
    assert not B.vl_verify_linear(job, p)
    # another statement: seed, coefficient, bind, matrix order
    assert not B.vl_verify_linear(_host_job(mats, coeffs, seed + 1), _to_c(proof))
    assert not B.vl_verify_linear(_host_job(mats, [1, -1, 2], seed), _to_c(proof))
    assert not B.vl_verify_linear(_host_job(mats, coeffs, seed, binds=[b"\x01" * 32] * 3), _to_c(proof))
    assert not B.vl_verify_linear(_host_job([A, A2, G], coeffs, seed), _to_c(proof))
    # a false relation: its honest proof carries sum c_q e_q != 0
    bad = [A2.copy(), A, G]
    bad[0][2, 3] += 1
    pb = oracle.prove_linear(bad, coeffs, seed=seed)
    assert not B.vl_verify_linear(_host_job(bad, coeffs, seed), _to_c(pb))


def test_host_verifier_other_dtypes(L):
    """Operands the verifier reads as int64 or Montgomery field elements give
    the same verdict as int16."""
    rng = np.random.default_rng(6)
    A = _rand(rng, (4, 12), -100, 100)
    G = _rand(rng, (4, 12), -100, 100)
    A2 = (A - G).astype(np.int16)
    mats, coeffs = [A2, A, G], [1, -1, 1]
    proof = oracle.prove_linear(mats, coeffs, seed=2)
    j64 = _host_job([m.astype(np.int64) for m in mats], coeffs, 2)
    assert B.vl_verify_linear(j64, _to_c(proof))


def test_update_statements_are_true_relations():
    """The workload's parameter-update relations hold entrywise (so their
    proofs must verify)."""
    t = W.lora_projection(W.GLOBAL_SEED, 0, "q", 64, 256, 256, 8)
    for st in W.update_statements(t):
        F2, F, G = (m.astype(np.int64) for m in st["mats"])
        assert np.array_equal(F2 - F + G, np.zeros_like(F))
        assert st["coeffs"] == (1, -1, 1)


def test_plan_create_validation(L):
    rng = np.random.default_rng(7)
    M = [_rand(rng, (20, 30)) for _ in range(2)]
    j = _host_job(M, [1, 2])
    plan = B.LinPlan([j])
    assert plan.workspace_bytes() == B.vl_linear_workspace_bytes([j])
    plan.destroy()
    j._coeffs[1].limb[7] = 0xFFFFFFFF
    with pytest.raises(B.VLError):
        B.LinPlan([j])
    with pytest.raises(B.VLError):
        B.LinPlan([_host_job([M[0], _rand(rng, (20, 31))], [1, 1])])


def test_paper_route_products_shapes_and_claims():
    """The paper's backward route: R1 is the full weight gradient X^T.dY
    (d x k), R2 and R3 take its rescaled form to the LoRA gradients
    (d x r and r x k), the same shapes as B3 (dA) and B2 (dB) of the
    eight-product set; a tiny claimed product is checked entry by entry."""
    t = W.lora_projection(W.GLOBAL_SEED, 0, "q", 8, 12, 10, 4)
    jobs, dWr = W.paper_route_products(t)
    shapes = {j["name"].rsplit(".", 1)[1]: W.op_shape(j) for j in jobs}
    assert shapes["R1"] == (12, 8, 10) and shapes["R2"] == (12, 10, 4) and shapes["R3"] == (4, 12, 10)
    base = {j["name"].rsplit(".", 1)[1]: W.op_shape(j) for j in W.projection_products(t)}
    assert (shapes["R2"][0], shapes["R2"][2]) == (base["B3"][0], base["B3"][2])  # dA: d x r
    assert (shapes["R3"][0], shapes["R3"][2]) == (base["B2"][0], base["B2"][2])  # dB: r x k
    X, dY = t["X"].astype(np.int64), t["dY"].astype(np.int64)
    R1 = W.claimed_product(jobs[6])
    for i in range(12):
        for j in range(10):
            assert R1[i, j] == sum(X[s, i] * dY[s, j] for s in range(8))
    assert np.array_equal(dWr, W.rescale(R1))
