"""Pins for oracle/sumcheck.py (Sec. II-B sumcheck, Sec. II-C matmul identity).

Every check recomputes from definitions that do not share the prover's
round/fold code: brute-force hypercube sums of the MLEs, the integer matmul
(NumPy int64), closed forms of the special cases, and the verifier's
acceptance/rejection behaviour (perfect completeness, Sec. V-B; soundness by
perturbation, Sec. V-A).
"""
import itertools
import random

import numpy as np
import pytest

from oracle.field import R_MOD
from oracle.mle import mle_eval_bruteforce, eq_table
from oracle.sumcheck import prove_matmul, verify_matmul, round_poly_eval, ceil_log2, Proof


def _mats(rng, m, k, n, lo=-(1 << 15), hi=(1 << 15)):
    P = np.array([[rng.randrange(lo, hi) for _ in range(k)] for _ in range(m)], dtype=np.int64)
    Q = np.array([[rng.randrange(lo, hi) for _ in range(n)] for _ in range(k)], dtype=np.int64)
    return P, Q


def _flat(M, d_rows, d_cols):
    flat = [0] * (1 << (d_rows + d_cols))
    for i in range(M.shape[0]):
        for j in range(M.shape[1]):
            flat[(i << d_cols) + j] = int(M[i, j]) % R_MOD
    return flat


def _bruteforce_round(A, B, u, v, rs, X, d1):
    """g_i(X) = sum over the free w' of A~(u, rs, X, w') * B~(rs, X, w', v), by eq:MLE."""
    d0 = ceil_log2(A.shape[0])
    d2 = ceil_log2(B.shape[1])
    fa = _flat(A, d0, d1)
    fb = _flat(B, d1, d2)
    free = d1 - len(rs) - 1
    total = 0
    for tail in itertools.product((0, 1), repeat=free):
        w = list(rs) + [X] + list(tail)
        total += mle_eval_bruteforce(fa, list(u) + w) * mle_eval_bruteforce(fb, w + list(v))
    return total % R_MOD


@pytest.mark.parametrize("m,k,n", [(4, 8, 4), (3, 5, 2), (2, 16, 3), (1, 4, 1), (5, 1, 3), (8, 2, 8)])
def test_rounds_match_bruteforce(m, k, n):
    rng = random.Random(m * 100 + k * 10 + n)
    P, Q = _mats(rng, m, k, n)
    pf = prove_matmul(P, Q, seed=m + k + n)
    u, v, rs = pf.challenges["u"], pf.challenges["v"], pf.challenges["r"]
    d1 = ceil_log2(k)
    assert len(pf.g) == d1 == len(rs)
    claim = pf.c
    for i in range(d1):
        g0, g1, g2 = pf.g[i]
        assert (g0 + g1) % R_MOD == claim
        for X, gx in ((0, g0), (1, g1), (2, g2)):
            assert gx == _bruteforce_round(P, Q, u, v, rs[:i], X, d1)
        # Degree <= 2: the value at a 4th point equals the interpolation.
        assert round_poly_eval(g0, g1, g2, 3) == _bruteforce_round(P, Q, u, v, rs[:i], 3, d1)
        claim = round_poly_eval(g0, g1, g2, rs[i])
    assert claim == pf.a_r * pf.b_r % R_MOD


@pytest.mark.parametrize("m,k,n", [(4, 8, 4), (3, 5, 7), (6, 3, 2)])
def test_claim_and_final_by_definition(m, k, n):
    rng = random.Random(17 * m + k + n)
    P, Q = _mats(rng, m, k, n)
    pf = prove_matmul(P, Q, seed=99)
    u, v, rs = pf.challenges["u"], pf.challenges["v"], pf.challenges["r"]
    d0, d1, d2 = ceil_log2(m), ceil_log2(k), ceil_log2(n)
    C = P @ Q  # integer matmul, int64 exact at these sizes
    assert pf.c == mle_eval_bruteforce(_flat(C, d0, d2), list(u) + list(v))
    assert pf.a_r == mle_eval_bruteforce(_flat(P, d0, d1), list(u) + list(rs))
    assert pf.b_r == mle_eval_bruteforce(_flat(Q, d1, d2), list(rs) + list(v))


def test_boolean_challenges_give_integer_entries():
    rng = random.Random(21)
    m, k, n = 8, 16, 4
    P, Q = _mats(rng, m, k, n)
    C = P @ Q
    for _ in range(6):
        i, j = rng.randrange(m), rng.randrange(n)
        ub = [(i >> (2 - t)) & 1 for t in range(3)]
        vb = [(j >> (1 - t)) & 1 for t in range(2)]
        pf = prove_matmul(P, Q, seed=1, override={"u": ub, "v": vb})
        assert pf.c == int(C[i, j]) % R_MOD
    # Boolean round challenges too: a_r, b_r become entries of P and Q.
    wb = [1, 0, 1, 1]
    pf = prove_matmul(P, Q, seed=1, override={"u": [0, 1, 1], "v": [1, 0], "r": wb})
    assert pf.a_r == int(P[3, 11]) % R_MOD and pf.b_r == int(Q[11, 2]) % R_MOD


def test_k_equals_one():
    rng = random.Random(23)
    P, Q = _mats(rng, 4, 1, 4)
    pf = prove_matmul(P, Q, seed=3)
    assert pf.d1 == 0 and pf.g == []
    assert pf.c == pf.a_r * pf.b_r % R_MOD


def test_dot_product_case():
    rng = random.Random(29)
    P, Q = _mats(rng, 1, 37, 1)
    pf = prove_matmul(P, Q, seed=4)
    assert pf.d0 == 0 and pf.d2 == 0 and pf.d1 == 6
    assert pf.c == int((P @ Q)[0, 0]) % R_MOD


def test_transposes_are_variable_reorders():
    rng = random.Random(31)
    P, Q = _mats(rng, 5, 6, 3)
    a = prove_matmul(P, Q, 0, 0, seed=8)
    b = prove_matmul(np.ascontiguousarray(P.T), np.ascontiguousarray(Q.T), 1, 1, seed=8)
    # Different statements (trans flags) give different transcripts but the same
    # polynomial identities: both verify against the same C.
    C = P @ Q
    assert verify_matmul(P, Q, C, a, 0, 0, seed=8)[0]
    assert verify_matmul(np.ascontiguousarray(P.T), np.ascontiguousarray(Q.T), C, b, 1, 1, seed=8)[0]
    assert a.state != b.state


@pytest.mark.parametrize("m,k,n,tp,tq", [(4, 8, 4, 0, 0), (3, 5, 7, 1, 0), (6, 9, 2, 0, 1), (1, 1, 1, 1, 1), (7, 2, 1, 0, 0)])
def test_verifier_completeness(m, k, n, tp, tq):
    rng = random.Random(m + 3 * k + 5 * n + tp + 2 * tq)
    A, B = _mats(rng, m, k, n)
    C = A @ B
    P = np.ascontiguousarray(A.T) if tp else A
    Q = np.ascontiguousarray(B.T) if tq else B
    pf = prove_matmul(P, Q, tp, tq, seed=77)
    ok, why = verify_matmul(P, Q, C, pf, tp, tq, seed=77)
    assert ok, why


def _copy(pf, **kw):
    d = dict(m=pf.m, k=pf.k, n=pf.n, d0=pf.d0, d1=pf.d1, d2=pf.d2, c=pf.c,
             g=[tuple(t) for t in pf.g], a_r=pf.a_r, b_r=pf.b_r, state=pf.state)
    d.update(kw)
    return Proof(**d)


def test_verifier_rejects_every_single_field_perturbation():
    rng = random.Random(41)
    m, k, n = 4, 8, 4
    P, Q = _mats(rng, m, k, n)
    C = P @ Q
    pf = prove_matmul(P, Q, seed=5)
    assert verify_matmul(P, Q, C, pf, seed=5)[0]
    bad = [_copy(pf, c=(pf.c + 1) % R_MOD), _copy(pf, a_r=(pf.a_r + 1) % R_MOD),
           _copy(pf, b_r=(pf.b_r + 1) % R_MOD),
           _copy(pf, state=bytes([pf.state[0] ^ 1]) + pf.state[1:])]
    for i in range(len(pf.g)):
        for t in range(3):
            g = [list(x) for x in pf.g]
            g[i][t] = (g[i][t] + 1) % R_MOD
            bad.append(_copy(pf, g=[tuple(x) for x in g]))
    for b in bad:
        assert not verify_matmul(P, Q, C, b, seed=5)[0]
    # Perturbed statement: one entry of C, P or Q off by one; wrong seed; wrong flags.
    for M, which in ((C, "C"), (P, "P"), (Q, "Q")):
        M2 = M.copy()
        M2[rng.randrange(M.shape[0]), rng.randrange(M.shape[1])] += rng.choice((-1, 1))
        args = {"C": (P, Q, M2), "P": (M2, Q, C), "Q": (P, M2, C)}[which]
        assert not verify_matmul(*args, pf, seed=5)[0], which
    assert not verify_matmul(P, Q, C, pf, seed=6)[0]
    assert not verify_matmul(P, np.ascontiguousarray(Q), C, pf, 0, 0, seed=5, binds=(bytes([1]) + bytes(31), bytes(32), bytes(32)))[0]


def test_wrong_product_has_no_honest_proof():
    rng = random.Random(43)
    P, Q = _mats(rng, 4, 4, 4)
    C = P @ Q
    C[1, 2] += 1
    pf = prove_matmul(P, Q, seed=9)
    assert not verify_matmul(P, Q, C, pf, seed=9)[0]


def test_padding_is_zero_extension():
    """A ragged product proves the same identities as its explicit zero-padding."""
    rng = random.Random(47)
    P, Q = _mats(rng, 3, 5, 6)
    pf = prove_matmul(P, Q, seed=10)
    u, v, rs = pf.challenges["u"], pf.challenges["v"], pf.challenges["r"]
    Pp = np.zeros((4, 8), dtype=np.int64)
    Pp[:3, :5] = P
    Qp = np.zeros((8, 8), dtype=np.int64)
    Qp[:5, :6] = Q
    assert pf.a_r == mle_eval_bruteforce(_flat(Pp, 2, 3), list(u) + list(rs))
    assert pf.b_r == mle_eval_bruteforce(_flat(Qp, 3, 3), list(rs) + list(v))


def test_eq_table_size_and_padding_rows():
    x = [3, 5, 7]
    assert len(eq_table(x, 5)) == 5 and eq_table(x, 5) == eq_table(x)[:5]
