"""Pins of the batched-claim matmul sumcheck oracle: round polynomials as
rho-weighted sums of per-product brute-force hypercube sums (eq:MLE written
out), the final combination, the Merkle tree, completeness and rejections."""
import copy
import hashlib

import numpy as np
import pytest

from oracle import batch as OB
from oracle.field import R_MOD
from oracle.mle import mle_eval_matrix
from oracle.sumcheck import _op


def _rand(rng, shape, lo=-(1 << 15), hi=1 << 15):
    return rng.integers(lo, hi, size=shape).astype(np.int16)


def _jobs(rng, K, k, shapes=None, trans=None):
    jobs = []
    for i in range(K):
        m, n = shapes[i] if shapes else (3 + i, 2 + 2 * i)
        tp, tq = trans[i] if trans else (i % 2, (i // 2) % 2)
        A, B = _rand(rng, (m, k)), _rand(rng, (k, n))
        jobs.append({"P": np.ascontiguousarray(A.T) if tp else A, "Q": np.ascontiguousarray(B.T) if tq else B,
                     "tp": tp, "tq": tq, "A": A, "B": B})
    return jobs


def _claimed(j):
    return j["A"].astype(np.int64) @ j["B"].astype(np.int64)


def test_merkle_root_by_hand():
    h = lambda b: hashlib.sha256(b).digest()
    l = [bytes([i]) * 32 for i in range(3)]
    assert OB.merkle_root(l[:1]) == l[0]
    assert OB.merkle_root(l[:2]) == h(b"\x01" + l[0] + l[1])
    assert OB.merkle_root(l) == h(b"\x01" + h(b"\x01" + l[0] + l[1]) + h(b"\x01" + l[2] + bytes(32)))


@pytest.mark.parametrize("K,k", [(1, 4), (3, 5), (4, 8), (2, 1)])
def test_rounds_are_rho_weighted_brute_force_sums(K, k):
    rng = np.random.default_rng(K * 10 + k)
    jobs = _jobs(rng, K, k)
    p = OB.prove_matmul_batch(jobs, seed=4)
    rho, rs = p.point["rho"], p.point["r"]
    d1 = p.d1
    for t in range(1, d1 + 1):
        rest = d1 - t
        g = [0, 0, 0]
        for i, j in enumerate(jobs):
            A, B = _op(j["P"], j["tp"]), _op(j["Q"], j["tq"])
            u, v = p.point["u"][i], p.point["v"][i]
            for X in range(3):
                tot = 0
                for b in range(1 << rest):
                    w = rs[:t - 1] + [X] + [(b >> (rest - 1 - q)) & 1 for q in range(rest)]
                    tot += mle_eval_matrix(A, u, w) * mle_eval_matrix(B, w, v)
                g[X] += pow(rho, i, R_MOD) * tot
        assert tuple(x % R_MOD for x in g) == p.rounds[t - 1]
    # the claims are the products' MLEs at (u_i, v_i)
    for i, j in enumerate(jobs):
        assert p.claims[i] == mle_eval_matrix(_claimed(j), p.point["u"][i], p.point["v"][i])
    # k = 1: no rounds, the final values are the claims' factors
    if k == 1:
        assert p.d1 == 0 and all(p.claims[i] == p.a[i] * p.b[i] % R_MOD for i in range(K))


@pytest.mark.parametrize("k,tp,tq", [(1, 0, 0), (6, 1, 0), (16, 0, 1), (21, 1, 1)])
def test_one_product_is_the_single_sumcheck_at_the_same_point(k, tp, tq):
    """K = 1 (rho^0 = 1): the batch's claim, rounds and final values are the
    single-product sumcheck's, run with the batch's challenges u, v, r."""
    rng = np.random.default_rng(50 + k)
    jobs = _jobs(rng, 1, k, shapes=[(5, 3)], trans=[(tp, tq)])
    p = OB.prove_matmul_batch(jobs, seed=8)
    pt = p.point
    from oracle.sumcheck import prove_matmul
    s = prove_matmul(jobs[0]["P"], jobs[0]["Q"], tp, tq, override={"u": pt["u"][0], "v": pt["v"][0], "r": pt["r"]})
    assert s.c == p.claims[0]
    assert [tuple(g) for g in s.g] == p.rounds
    assert (s.a_r, s.b_r) == (p.a[0], p.b[0])


@pytest.mark.parametrize("K,k", [(1, 7), (5, 16), (3, 33)])
def test_completeness(K, k):
    rng = np.random.default_rng(K + k)
    jobs = _jobs(rng, K, k)
    p = OB.prove_matmul_batch(jobs, seed=1)
    assert OB.verify_matmul_batch(jobs, [_claimed(j) for j in jobs], p, seed=1)[0]
    assert len(p.to_bytes()) == 12 + 32 * K + 96 * p.d1 + 64 * K + 32


def test_rejections():
    rng = np.random.default_rng(9)
    jobs = _jobs(rng, 4, 12)
    Cs = [_claimed(j) for j in jobs]
    p = OB.prove_matmul_batch(jobs, seed=2)
    assert OB.verify_matmul_batch(jobs, Cs, p, seed=2)[0]
    for j in range(4):  # a false product in any position
        bad = [C.copy() for C in Cs]
        bad[j][0, 0] += 1
        assert not OB.verify_matmul_batch(jobs, bad, p, seed=2)[0]
    for name in ("claims", "a", "b"):
        for i in range(4):
            q = copy.deepcopy(p)
            getattr(q, name)[i] = (getattr(q, name)[i] + 1) % R_MOD
            assert not OB.verify_matmul_batch(jobs, Cs, q, seed=2)[0]
    for t in range(p.d1):
        for x in range(3):
            q = copy.deepcopy(p)
            g = list(q.rounds[t])
            g[x] = (g[x] + 1) % R_MOD
            q.rounds[t] = tuple(g)
            assert not OB.verify_matmul_batch(jobs, Cs, q, seed=2)[0]
    q = copy.deepcopy(p)
    q.state = bytes([q.state[0] ^ 1]) + q.state[1:]
    assert not OB.verify_matmul_batch(jobs, Cs, q, seed=2)[0]
    assert not OB.verify_matmul_batch(jobs, Cs, p, seed=3)[0]
    # products in another order are another statement
    assert not OB.verify_matmul_batch(jobs[::-1], Cs[::-1], p, seed=2)[0]
    with pytest.raises(ValueError):
        OB.prove_matmul_batch(jobs + _jobs(rng, 1, 13), seed=2)


def test_planted_mistakes_are_caught(monkeypatch):
    """Mistakes planted in the batch oracle (rho^(i+1) weights, the round
    message's g(1) and g(2) swapped in the interpolation) each fail the
    rho-weighted brute-force pin or completeness."""
    rng = np.random.default_rng(12)
    jobs = _jobs(rng, 3, 4)
    Cs = [_claimed(j) for j in jobs]

    def ok():
        try:
            p = OB.prove_matmul_batch(jobs, seed=6)
        except AssertionError:
            return False
        return OB.verify_matmul_batch(jobs, Cs, p, seed=6)[0]

    assert ok()
    real_pow = pow
    monkeypatch.setattr(OB, "pow", lambda b, e, m=None: real_pow(b, e + 1, m) if m else real_pow(b, e), raising=False)
    p = OB.prove_matmul_batch(jobs, seed=6)
    # the shifted weights still give a self-consistent proof, but not the rho^i-weighted polynomial
    rho = p.point["rho"]
    monkeypatch.setattr(OB, "pow", real_pow, raising=False)
    g0 = 0
    for i, j in enumerate(jobs):
        A, B_ = _op(j["P"], j["tp"]), _op(j["Q"], j["tq"])
        u, v = p.point["u"][i], p.point["v"][i]
        tot = 0
        for b in range(1 << (p.d1 - 1)):
            w = [0] + [(b >> (p.d1 - 2 - q)) & 1 for q in range(p.d1 - 1)]
            tot += mle_eval_matrix(A, u, w) * mle_eval_matrix(B_, w, v)
        g0 += real_pow(rho, i, R_MOD) * tot
    assert g0 % R_MOD != p.rounds[0][0]
    orig = OB.round_poly_eval
    monkeypatch.setattr(OB, "round_poly_eval", lambda g0_, g1, g2, x: orig(g0_, g2, g1, x))
    assert not ok()
    monkeypatch.setattr(OB, "round_poly_eval", orig)
    assert ok()
