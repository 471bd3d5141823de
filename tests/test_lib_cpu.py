"""CPU tests of the C-ABI library: it loads, exports every declared symbol,
validates inputs on the host, and its host verifier agrees with the oracle.

No GPU is touched: only host-side entry points are called (input checks that
fail before any CUDA call, workspace sizing, and the host verifier).
"""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(B.LIB_PATH):
        from paper_2508_21393_gb300 import build
        build.build(quiet=True)
    return B.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "verilora.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(vl_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol(L):
    declared = _declared()
    assert declared == sorted(B.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name


def test_workspace_forget_without_a_record(L):
    # no plan ran on this address: nothing to forget; no CUDA call is made
    assert B.vl_workspace_forget(4096) is False
    assert L.vl_workspace_forget(None) == -B.VL_EINVAL
    with pytest.raises(B.VLError):
        B.vl_workspace_forget(None)


def test_version_and_strerror(L):
    assert B.vl_version() == 100
    assert B.vl_strerror(B.VL_OK) == "ok"
    assert B.vl_strerror(B.VL_REJECT) == "proof rejected"
    assert B.vl_strerror(99) == "unknown status"


def _host_job(P, Q, tp=0, tq=0, seed=0):
    return B.job(np.ascontiguousarray(P), np.ascontiguousarray(Q), tp, tq, seed)


def test_workspace_sizing_and_shape_errors(L):
    P = np.zeros((8, 16), np.int16)
    Q = np.zeros((16, 4), np.int16)
    assert B.vl_workspace_bytes([_host_job(P, Q)]) > 0
    # inner dimensions differ -> invalid plan (0 bytes)
    assert B.vl_workspace_bytes([_host_job(P, np.zeros((15, 4), np.int16))]) == 0
    # transposed Q fixes it
    assert B.vl_workspace_bytes([_host_job(P, np.zeros((4, 16), np.int16), 0, 1)]) > 0
    # a reduced dimension above 2^16 is refused
    big = np.zeros((1, (1 << 16) + 1), np.int16)
    assert B.vl_workspace_bytes([_host_job(big, np.zeros(((1 << 16) + 1, 1), np.int16), 1, 0)]) == 0


def test_prove_rejects_bad_input_before_any_cuda_call(L):
    P = np.zeros((8, 16), np.int16)
    Q = np.zeros((15, 4), np.int16)
    j = _host_job(P, Q)
    with pytest.raises(B.VLError) as e:
        B.vl_prove_matmul(j.P, j.Q, j.fs, 256, 1 << 20, stream=0)
    assert e.value.code == B.VL_ESHAPE
    j = _host_job(P, np.zeros((16, 4), np.int16))
    with pytest.raises(B.VLError) as e:
        B.vl_prove_matmul(j.P, j.Q, j.fs, 256, 16, stream=0)  # workspace too small
    assert e.value.code == B.VL_ENOMEM
    bad = _host_job(P, np.zeros((16, 4), np.int16))
    bad.P.ld = 3  # ld < cols
    with pytest.raises(B.VLError) as e:
        B.vl_prove_matmul(bad.P, bad.Q, bad.fs, 256, 1 << 20, stream=0)
    assert e.value.code == B.VL_EINVAL
    empty = _host_job(P, np.zeros((16, 4), np.int16))
    empty.P.rows = 0
    with pytest.raises(B.VLError) as e:
        B.vl_prove_matmul(empty.P, empty.Q, empty.fs, 256, 1 << 20, stream=0)
    assert e.value.code in (B.VL_ESHAPE, B.VL_EINVAL)


def _to_vl_proof(pf):
    out = B.vl_proof()
    out.m, out.k, out.n, out.d0, out.d1, out.d2 = pf.m, pf.k, pf.n, pf.d0, pf.d1, pf.d2
    out.status = 0

    def setfr(dst, v):
        for i, l in enumerate(oracle.limbs_le32(v)):
            dst.limb[i] = l
    setfr(out.c, pf.c)
    for i, tri in enumerate(pf.g):
        for q in range(3):
            setfr(out.g[i][q], tri[q])
    setfr(out.a_r, pf.a_r)
    setfr(out.b_r, pf.b_r)
    for i in range(32):
        out.state[i] = pf.state[i]
    return out


@pytest.mark.parametrize("m,k,n,tp,tq", [(4, 8, 4, 0, 0), (5, 7, 3, 1, 0), (6, 9, 2, 0, 1), (1, 1, 1, 1, 1),
                                         (1, 37, 1, 0, 0), (9, 1, 5, 0, 0)])
def test_host_verifier_accepts_oracle_proofs(L, m, k, n, tp, tq):
    rng = np.random.default_rng(m * 100 + k * 10 + n + tp + 2 * tq)
    A = rng.integers(-(1 << 15), 1 << 15, size=(m, k)).astype(np.int16)
    Bm = rng.integers(-(1 << 15), 1 << 15, size=(k, n)).astype(np.int16)
    C = W.exact_matmul(A, Bm)
    P = np.ascontiguousarray(A.T) if tp else A
    Q = np.ascontiguousarray(Bm.T) if tq else Bm
    pf = oracle.prove_matmul(P, Q, tp, tq, seed=1234)
    vp = _to_vl_proof(pf)
    assert B.proof_bytes(vp) == pf.to_bytes()
    ok = B.vl_verify_matmul(B.mat(P, tp), B.mat(Q, tq), B.mat(C), B.fs_init(1234), vp)
    assert ok


def test_host_verifier_rejects_perturbations(L):
    rng = np.random.default_rng(7)
    A = rng.integers(-(1 << 15), 1 << 15, size=(8, 16)).astype(np.int16)
    Bm = rng.integers(-(1 << 15), 1 << 15, size=(16, 4)).astype(np.int16)
    C = W.exact_matmul(A, Bm)
    pf = oracle.prove_matmul(A, Bm, seed=9)
    fs = B.fs_init(9)
    assert B.vl_verify_matmul(B.mat(A), B.mat(Bm), B.mat(C), fs, _to_vl_proof(pf))

    def bumped(field, i=None, q=None):
        vp = _to_vl_proof(pf)
        f = getattr(vp, field) if i is None else vp.g[i][q]
        f.limb[0] = (f.limb[0] + 1) & 0xFFFFFFFF
        return vp
    cases = [bumped("c"), bumped("a_r"), bumped("b_r")]
    cases += [bumped("g", i, q) for i in range(pf.d1) for q in range(3)]
    st = _to_vl_proof(pf)
    st.state[5] ^= 0x40
    cases.append(st)
    for vp in cases:
        assert not B.vl_verify_matmul(B.mat(A), B.mat(Bm), B.mat(C), fs, vp)
    C2 = C.copy()
    C2[3, 1] += 1
    assert not B.vl_verify_matmul(B.mat(A), B.mat(Bm), B.mat(C2), fs, _to_vl_proof(pf))
    A2 = A.copy()
    A2[0, 0] ^= 1
    assert not B.vl_verify_matmul(B.mat(A2), B.mat(Bm), B.mat(C), fs, _to_vl_proof(pf))
    assert not B.vl_verify_matmul(B.mat(A), B.mat(Bm), B.mat(C), B.fs_init(10), _to_vl_proof(pf))


def test_server_rejects_bad_options_before_cuda():
    L = B.lib()
    s = ctypes.c_void_p()
    o = B.vl_server_opts()
    assert L.vl_server_create(ctypes.byref(o), ctypes.byref(s)) == B.VL_EINVAL  # no arena
    o.arena = 4096
    o.arena_bytes = 1 << 20
    o.reserved[1] = 1
    assert L.vl_server_create(ctypes.byref(o), ctypes.byref(s)) == B.VL_EINVAL  # reserved field set
    assert L.vl_server_submit(None, None, 0, None, None) == B.VL_EINVAL
    assert L.vl_server_destroy(None) == B.VL_EINVAL


def test_autotune_rejects_bad_arguments_before_cuda():
    L = B.lib()
    best = B.vl_batch_opts()
    assert L.vl_autotune(None, 1, None, 4096, 1 << 20, None, 0, ctypes.byref(best), None) == B.VL_EINVAL
    jb = (B.vl_job * 1)()
    assert L.vl_autotune(jb, 1, None, 4096 + 8, 1 << 20, None, 0, ctypes.byref(best), None) == B.VL_EINVAL  # unaligned
    assert L.vl_autotune(jb, 0, None, 4096, 1 << 20, None, 0, ctypes.byref(best), None) == B.VL_EINVAL
