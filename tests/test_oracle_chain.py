"""Pins for oracle/chain.py (the chained proof of one LoRA projection).

What fixes the chain independently of the oracle's own code:
* the rescale identity (X.A)~(p) = 2^8 H~(p) + rho~(p) - 2^7 J~(p) at random
  points, with the left side the MLE of the integer product computed with
  NumPy int64 and J~ against a brute-force eq:MLE sum of the all-ones matrix;
* every member's claim equals the MLE of its integer product (NumPy int64)
  at the member's point, and its rounds satisfy g(0) + g(1) = claim;
* the stage-3 points are the stage-1 members' final points (F3's and B2's
  claims on H, B5's and B3's on dH): the H~ / dH~ values the stage-1 proofs
  end on equal the MLEs of H, dH computed by definition there;
* completeness on ragged and power-of-two shapes; rejection of a false H,
  dH or remainder, of false outputs, and of every perturbed proof value;
* planted mistakes in the oracle (a wrong sign of the 2^7 term, swapped
  stage-3 points) are caught.
"""
import copy
import random

import numpy as np
import pytest

from oracle import chain as C
from oracle.field import R_MOD
from oracle.mle import eq_table, mle_eval_bruteforce, mle_eval_matrix
from paper_2508_21393_gb300 import workload as W

SHAPES = [(6, 10, 12, 3), (8, 16, 8, 4), (5, 7, 9, 2), (1, 4, 4, 1)]


def _proj(n, d, k, r, seed=3):
    return W.chain_tensors(W.lora_projection(seed, 0, "q", n, d, k, r))


def _pad_flat(M, rows2, cols2):
    out = np.zeros((rows2, cols2), dtype=np.int64)
    out[:M.shape[0], :M.shape[1]] = M
    return out.reshape(-1).tolist()


@pytest.mark.parametrize("n,d,k,r", SHAPES)
def test_rescale_identity_against_integer_product(n, d, k, r):
    t = _proj(n, d, k, r)
    rng = random.Random(n * 100 + r)
    XA = W.exact_matmul(t["X"], t["A"])
    ln, lr = (n - 1).bit_length(), (r - 1).bit_length()
    for _ in range(3):
        x = [rng.randrange(R_MOD) for _ in range(ln)]
        y = [rng.randrange(R_MOD) for _ in range(lr)]
        J = C.ones_mle(x, y, n, r)
        assert J == mle_eval_bruteforce(_pad_flat(np.ones((n, r), np.int64), 1 << ln, 1 << lr), x + y)
        rhs = (256 * mle_eval_matrix(t["H"], x, y) + mle_eval_matrix(t["rhoH"], x, y) - 128 * J) % R_MOD
        assert mle_eval_matrix(XA, x, y) == rhs


@pytest.mark.parametrize("n,d,k,r", SHAPES)
def test_member_claims_are_mles_of_the_integer_products(n, d, k, r):
    t = _proj(n, d, k, r)
    pf = C.prove_chain(t, seed=11)
    T = C._start(11, n, d, k, r, (bytes(32),) * 7)
    P = C._points(T, n, d, k, r)
    ops = C._operands(t)
    pts = C._stage1_points(P) + C._stage3_points(P, [sp.r for sp in pf.subs])
    for p, ((A, B), (u, v), sp) in enumerate(zip(ops, pts, pf.subs)):
        prod = W.exact_matmul(A, B)
        assert sp.c == mle_eval_matrix(prod, u, v), p
        if sp.g:  # later rounds follow from the challenges (the verifier replays them)
            assert (sp.g[0][0] + sp.g[0][1]) % R_MOD == sp.c
    # the stage-1 proofs end on H and dH at the stage-3 points
    p1, p2, q1, q2 = C._stage3_points(P, [sp.r for sp in pf.subs])
    assert pf.subs[1].a_r == mle_eval_matrix(t["H"], *p1)
    assert pf.subs[5].a_r == mle_eval_matrix(t["H"], *p2)
    assert pf.subs[3].a_r == mle_eval_matrix(t["dH"], *q1)
    assert pf.subs[4].b_r == mle_eval_matrix(t["dH"], *q2)
    # and the stage-3 claims are what the rescale relation derives
    assert [sp.c for sp in pf.subs[6:]] == C.derived_claims(pf.subs, pf.e, [p1, p2, q1, q2], n, r)


@pytest.mark.parametrize("n,d,k,r", SHAPES)
def test_completeness(n, d, k, r):
    t = _proj(n, d, k, r, seed=n + d)
    binds = tuple(bytes([i]) * 32 for i in range(7))
    pf = C.prove_chain(t, seed=5, binds=binds)
    assert C.verify_chain(t, W.chain_outputs(t), pf, seed=5, binds=binds) == (True, "accept")
    assert len(pf.to_bytes()) == 16 + sum(24 + 32 * (3 * (kk - 1).bit_length() + 3) + 32
                                          for (_, kk, _) in pf.shapes) + 4 * 32 + 32


def _false_rescale(t, key, rho_key, i, j):
    """H (or dH) one larger at (i, j), remainder unchanged: the rescale
    relation no longer holds (the prover proves with the false tensor)."""
    t2 = dict(t)
    M = t[key].copy()
    M[i, j] += 1
    t2[key] = M
    return t2


@pytest.mark.parametrize("key,rho", [("H", "rhoH"), ("dH", "rhodH")])
def test_false_intermediate_is_rejected(key, rho):
    t = _proj(6, 10, 12, 3)
    t2 = _false_rescale(t, key, rho, 2, 1)
    pf = C.prove_chain(t2, seed=5)
    # outputs recomputed from the false tensor, so every output claim holds
    ok, why = C.verify_chain(t2, W.chain_outputs(t2), pf, seed=5)
    assert not ok and "rescale-derived" in why


def test_false_remainder_is_rejected():
    t = _proj(6, 10, 12, 3)
    t2 = dict(t)
    t2["rhoH"] = t["rhoH"].copy()
    t2["rhoH"][0, 0] += 1
    pf = C.prove_chain(t2, seed=5)
    ok, why = C.verify_chain(t2, W.chain_outputs(t2), pf, seed=5)
    assert not ok and "rescale-derived" in why
    # a remainder shifted by 2^8 with H one smaller keeps the linear relation:
    # only the range lookup (Protocol 1) rejects that; the chain accepts it
    t3 = dict(t)
    t3["rhoH"] = t["rhoH"].astype(np.int32).copy()
    t3["rhoH"][0, 0] += 256
    t3["H"] = t["H"].copy()
    t3["H"][0, 0] -= 1
    pf = C.prove_chain(t3, seed=5)
    assert C.verify_chain(t3, W.chain_outputs(t3), pf, seed=5)[0]
    assert t3["rhoH"].max() >= 256  # out of the lookup's table [0, 2^8)


@pytest.mark.parametrize("out", ["Y", "dX", "dA", "dB"])
def test_false_output_is_rejected(out):
    t = _proj(6, 10, 12, 3)
    pf = C.prove_chain(t, seed=5)
    outs = W.chain_outputs(t)
    outs[out] = outs[out].copy()
    outs[out][0, 0] += 1
    ok, why = C.verify_chain(t, outs, pf, seed=5)
    assert not ok and "!=" in why


def test_every_perturbed_value_is_rejected():
    t = _proj(5, 7, 9, 2)
    outs = W.chain_outputs(t)
    pf = C.prove_chain(t, seed=9)
    assert C.verify_chain(t, outs, pf, seed=9)[0]
    cases = []
    for p in range(10):
        cases.append(("c", p, None))
        cases.append(("a_r", p, None))
        cases.append(("b_r", p, None))
        cases.append(("state", p, None))
        for i in range(len(pf.subs[p].g)):
            for q in range(3):
                cases.append(("g", p, (i, q)))
    for field, p, iq in cases:
        bad = copy.deepcopy(pf)
        sp = bad.subs[p]
        if field == "g":
            i, q = iq
            tri = list(sp.g[i])
            tri[q] = (tri[q] + 1) % R_MOD
            sp.g[i] = tuple(tri)
        elif field == "state":
            sp.state = bytes([sp.state[0] ^ 1]) + sp.state[1:]
        else:
            setattr(sp, field, (getattr(sp, field) + 1) % R_MOD)
        assert not C.verify_chain(t, outs, bad, seed=9)[0], (field, p, iq)
    for i in range(4):
        bad = copy.deepcopy(pf)
        bad.e[i] = (bad.e[i] + 1) % R_MOD
        assert not C.verify_chain(t, outs, bad, seed=9)[0], ("e", i)
    bad = copy.deepcopy(pf)
    bad.state = bytes(32)
    assert not C.verify_chain(t, outs, bad, seed=9)[0]
    assert not C.verify_chain(t, outs, pf, seed=10)[0]
    assert not C.verify_chain(t, outs, pf, seed=9, binds=(bytes([1]) * 32,) + (bytes(32),) * 6)[0]


def test_planted_sign_of_the_offset_is_caught(monkeypatch):
    t = _proj(6, 10, 12, 3)
    real = C.derived_claims

    def wrong(subs, e, pts, n, r):
        z = 256
        onH = [subs[1].a_r, subs[5].a_r, subs[3].a_r, subs[4].b_r]
        return [(z * onH[i] + e[i] + 128 * C.ones_mle(pts[i][0], pts[i][1], n, r)) % R_MOD for i in range(4)]

    monkeypatch.setattr(C, "derived_claims", wrong)
    pf = C.prove_chain(t, seed=5)
    assert not C.verify_chain(t, W.chain_outputs(t), pf, seed=5)[0]
    monkeypatch.setattr(C, "derived_claims", real)
    assert C.verify_chain(t, W.chain_outputs(t), pf, seed=5)[0]


def test_planted_swapped_points_are_caught(monkeypatch):
    t = _proj(6, 10, 12, 3)
    real = C._stage3_points

    def swapped(P, rs):
        p1, p2, q1, q2 = real(P, rs)
        return [p2, p1, q1, q2]

    monkeypatch.setattr(C, "_stage3_points", swapped)
    pf = C.prove_chain(t, seed=5)
    monkeypatch.setattr(C, "_stage3_points", real)
    assert not C.verify_chain(t, W.chain_outputs(t), pf, seed=5)[0]


def test_eq_sums_in_ones_mle():
    rng = random.Random(4)
    for rows in (1, 3, 4, 5, 8):
        ell = (rows - 1).bit_length()
        x = [rng.randrange(R_MOD) for _ in range(ell)]
        assert sum(eq_table(x, rows)) % R_MOD == mle_eval_bruteforce([1] * rows, x)
        if rows == 1 << ell:
            assert sum(eq_table(x, rows)) % R_MOD == 1
