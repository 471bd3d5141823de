"""The library's host verifier of chained projection proofs (vl_verify_chain)
against oracle proofs, on CPU: it accepts every honest oracle proof, rejects
each single perturbed value (every member's claim, round values, final
values and state, the remainder evaluations, the final state), false
outputs, a false H or remainder (the proof the oracle makes from it), another
seed or bind, and refuses malformed statements."""
import copy

import numpy as np
import pytest

from oracle import chain as C
from paper_2508_21393_gb300 import binding as B
from paper_2508_21393_gb300 import workload as W

SHAPES = [(6, 10, 12, 3), (8, 16, 8, 4), (5, 7, 9, 2), (1, 4, 4, 1), (16, 32, 24, 8)]
BINDS = tuple(bytes([i + 1]) * 32 for i in range(7))


def _proj(n, d, k, r, seed=3):
    return W.chain_tensors(W.lora_projection(seed, 0, "q", n, d, k, r))


def to_c(pf):
    """An oracle ChainProof as a vl_chain_proof."""
    P = B.vl_chain_proof()
    P.n, P.d, P.k, P.r = pf.n, pf.d, pf.k, pf.r
    for i, (sp, (m, k, n)) in enumerate(zip(pf.subs, pf.shapes)):
        q = P.sub[i]
        q.m, q.k, q.n = m, k, n
        q.d0, q.d1, q.d2 = (m - 1).bit_length(), (k - 1).bit_length(), (n - 1).bit_length()
        q.c, q.a_r, q.b_r = B.fr(sp.c), B.fr(sp.a_r), B.fr(sp.b_r)
        for a, tri in enumerate(sp.g):
            for b in range(3):
                q.g[a][b] = B.fr(tri[b])
        for z in range(32):
            q.state[z] = sp.state[z]
    for i in range(4):
        P.e[i] = B.fr(pf.e[i])
    for z in range(32):
        P.state[z] = pf.state[z]
    return P


def _job(t, seed=5, binds=BINDS):
    return B.chain_job({k: np.ascontiguousarray(t[k]) for k in B.CHAIN_MATS}, seed=seed, binds=binds)


@pytest.mark.parametrize("shape", SHAPES)
def test_library_verifier_accepts_oracle_proofs(shape):
    t = _proj(*shape)
    pf = C.prove_chain(t, seed=5, binds=BINDS)
    P = to_c(pf)
    assert B.chain_proof_bytes(P) == pf.to_bytes()
    assert B.vl_verify_chain(_job(t), W.chain_outputs(t), P)


def test_library_verifier_rejects_every_perturbation():
    t = _proj(5, 7, 9, 2)
    outs = W.chain_outputs(t)
    job = _job(t)
    P = to_c(C.prove_chain(t, seed=5, binds=BINDS))
    assert B.vl_verify_chain(job, outs, P)

    def bump(v):
        return B.fr(v.to_int() + 1)

    for p in range(B.VL_CHAIN_MEMBERS):
        for field in ("c", "a_r", "b_r"):
            Q = copy.deepcopy(P)
            setattr(Q.sub[p], field, bump(getattr(Q.sub[p], field)))
            assert not B.vl_verify_chain(job, outs, Q), (p, field)
        for i in range(P.sub[p].d1):
            for q in range(3):
                Q = copy.deepcopy(P)
                Q.sub[p].g[i][q] = bump(Q.sub[p].g[i][q])
                assert not B.vl_verify_chain(job, outs, Q), (p, i, q)
        Q = copy.deepcopy(P)
        Q.sub[p].state[3] ^= 1
        assert not B.vl_verify_chain(job, outs, Q), (p, "state")
    for i in range(4):
        Q = copy.deepcopy(P)
        Q.e[i] = bump(Q.e[i])
        assert not B.vl_verify_chain(job, outs, Q), ("e", i)
    Q = copy.deepcopy(P)
    Q.state[0] ^= 1
    assert not B.vl_verify_chain(job, outs, Q)
    assert not B.vl_verify_chain(_job(t, seed=6), outs, P)
    assert not B.vl_verify_chain(_job(t, binds=(bytes(32),) + BINDS[1:]), outs, P)
    for key in ("Y", "dX", "dA", "dB"):
        o2 = {k: v.copy() for k, v in outs.items()}
        o2[key][0, 0] += 1
        assert not B.vl_verify_chain(job, o2, P), key


@pytest.mark.parametrize("key", ["H", "dH", "rhoH", "rhodH"])
def test_false_witness_is_rejected(key):
    t = _proj(6, 10, 12, 3)
    t2 = dict(t)
    t2[key] = t[key].copy()
    t2[key][1, 2] += 1
    P = to_c(C.prove_chain(t2, seed=5, binds=BINDS))
    assert not B.vl_verify_chain(_job(t2), W.chain_outputs(t2), P)


def test_malformed_statements_are_refused():
    t = _proj(6, 10, 12, 3)
    outs = W.chain_outputs(t)
    P = to_c(C.prove_chain(t, seed=5, binds=BINDS))
    bad = dict(t)
    bad["rhoH"] = t["rhoH"][:, :2].copy()  # wrong shape
    with pytest.raises(B.VLError) as e:
        B.vl_verify_chain(_job(bad), outs, P)
    assert e.value.code == B.VL_ESHAPE
    o2 = dict(outs)
    o2["dA"] = outs["dA"][:, :1].copy()
    with pytest.raises(B.VLError) as e:
        B.vl_verify_chain(_job(t), o2, P)
    assert e.value.code == B.VL_ESHAPE
