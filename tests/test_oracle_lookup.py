"""Pins of the lookup-argument oracle (Protocol 1, Eq. eq:lookup-sumcheck)
against what the mathematics fixes: inverses, multiplicities, the rational
identity, the cube sum alpha + alpha^2, brute-force round polynomials built
from eq:MLE, the degree bound, completeness and rejections; plus planted
mistakes that a pin must catch."""
import random

import numpy as np
import pytest

import oracle
from oracle import lookup as L
from oracle.field import R_MOD
from oracle.mle import eq_value, mle_eval_bruteforce


def _rand_fr(rng):
    return rng.randrange(R_MOD)


def test_cubic_eval_is_lagrange_through_four_points():
    rng = random.Random(1)
    for _ in range(20):
        c = [_rand_fr(rng) for _ in range(4)]
        poly = lambda x: (c[0] + c[1] * x + c[2] * x * x + c[3] * x ** 3) % R_MOD
        g = [poly(x) for x in range(4)]
        x = _rand_fr(rng)
        assert L.cubic_eval(g, x) == poly(x)
    # a degree-4 polynomial is not reproduced off the nodes
    q = lambda x: x ** 4 % R_MOD
    assert L.cubic_eval([q(x) for x in range(4)], 4) != q(4)


def test_inverses_and_multiplicities():
    rng = random.Random(2)
    beta = _rand_fr(rng)
    s = [3, 0, 7, 7, 2, -1 % 16]
    s = [v % 16 for v in s]
    for v in s:
        a = oracle.fr_inv((beta + v) % R_MOD)
        assert a * (beta + v) % R_MOD == 1
        assert a == pow((beta + v) % R_MOD, -1, R_MOD)  # Python's extended-Euclid inverse
    m = L.multiplicities(s, 0, 16)
    assert sum(m) == len(s)
    for j in range(16):
        assert m[j] == s.count(j)
    with pytest.raises(ValueError):
        L.multiplicities([0, 16], 0, 16)
    with pytest.raises(ValueError):
        L.multiplicities([-1], 0, 16)


@pytest.mark.parametrize("n,log2_n,t0", [(5, 2, 0), (16, 4, -8), (40, 3, 100), (1, 0, 7), (3, 3, 0)])
def test_rational_identity_and_cube_sum(n, log2_n, t0):
    rng = random.Random(n * 31 + log2_n)
    N = 1 << log2_n
    S = [t0 + rng.randrange(N) for _ in range(n)]
    D, log2_d = L.lookup_dims(n, log2_n)
    assert D >= N and D >= n and D % N == 0
    s_pad = L.padded(S, t0, D)
    beta, alpha = _rand_fr(rng), _rand_fr(rng)
    u = [_rand_fr(rng) for _ in range(log2_d)]
    vec, c = L.term_vectors(s_pad, t0, N, beta, alpha, u)
    # sum_i A_i = sum_j m_j B_j
    m = L.multiplicities(s_pad, t0, N)
    B = [oracle.fr_inv((beta + t0 + j) % R_MOD) for j in range(N)]
    assert sum(vec["A"]) % R_MOD == sum(mj * bj for mj, bj in zip(m, B)) % R_MOD
    # the cube sum of P is alpha + alpha^2
    total = sum(L.p_value({k: f[i] for k, f in vec.items()}, alpha, c) for i in range(D)) % R_MOD
    assert total == (alpha + alpha * alpha) % R_MOD
    # a wrong multiplicity vector (one count moved) breaks it
    if N > 1:
        bad = dict(vec)
        mm = list(m)
        j = next(i for i in range(N) if mm[i] > 0)
        mm[j] -= 1
        mm[(j + 1) % N] += 1
        bad["m"] = [mm[k % N] for k in range(D)]
        total = sum(L.p_value({k: f[i] for k, f in bad.items()}, alpha, c) for i in range(D)) % R_MOD
        assert total != (alpha + alpha * alpha) % R_MOD


def _mle_point(f, point):
    return mle_eval_bruteforce(f, point) if point else f[0] % R_MOD


@pytest.mark.parametrize("n,log2_n,t0", [(8, 2, 0), (5, 1, -3), (16, 4, 0), (3, 2, 5)])
def test_round_polynomials_match_brute_force(n, log2_n, t0):
    """g_t(X) = sum over b of P with every vector replaced by its MLE at
    (r_1 .. r_{t-1}, X, b), evaluated literally from eq:MLE; X = 4 checks the
    degree bound."""
    rng = random.Random(n + 100 * log2_n)
    N = 1 << log2_n
    S = [t0 + rng.randrange(N) for _ in range(n)]
    proof = L.prove_lookup(S, t0, log2_n, seed=9)
    D, log2_d = L.lookup_dims(n, log2_n)
    pt = proof.point
    vec, c = L.term_vectors(L.padded(S, t0, D), t0, N, pt["beta"], pt["alpha"], pt["u"])
    claim = (pt["alpha"] + pt["alpha"] ** 2) % R_MOD
    for t in range(1, log2_d + 1):
        prefix = pt["r"][:t - 1]
        rest = log2_d - t
        g = []
        for X in range(5):
            tot = 0
            for b in range(1 << rest):
                bits = [(b >> (rest - 1 - i)) & 1 for i in range(rest)]
                point = prefix + [X] + bits
                tot += L.p_value({k: _mle_point(f, point) for k, f in vec.items()}, pt["alpha"], c)
            g.append(tot % R_MOD)
        assert tuple(g[:4]) == proof.rounds[t - 1]
        assert (g[0] + g[1]) % R_MOD == claim
        assert L.cubic_eval(g[:4], 4) == g[4]
        claim = L.cubic_eval(g[:4], pt["r"][t - 1])
    # the final evaluations are the vectors' MLEs at r
    r = pt["r"]
    assert proof.a_r == _mle_point(vec["A"], r)
    assert proof.s_r == (_mle_point(vec["S"], r) - pt["beta"]) % R_MOD


@pytest.mark.parametrize("shape,log2_n,t0", [((7, 9), 4, 0), ((128,), 7, -64), ((1,), 0, 3), ((33,), 5, 0),
                                              ((2, 2), 4, 0)])
def test_completeness(shape, log2_n, t0):
    rng = np.random.default_rng(sum(shape) + log2_n)
    S = rng.integers(t0, t0 + (1 << log2_n), size=shape)
    bind = bytes(range(32))
    proof = L.prove_lookup(S, t0, log2_n, seed=11, bind=bind)
    assert L.verify_lookup(S, t0, log2_n, proof, seed=11, bind=bind)[0]
    assert len(proof.to_bytes()) == 12 + 8 + 128 * proof.log2_d + 128 + 32


def test_special_case_single_entry_table_of_one():
    """D = N = 1: no rounds; P(0) = alpha + alpha^2 with A = B and m = 1."""
    proof = L.prove_lookup([5], 5, 0, seed=4)
    assert proof.log2_d == 0 and proof.rounds == []
    assert proof.a_r == proof.b_r and proof.m_r == 1 and proof.s_r == 5
    assert L.verify_lookup([5], 5, 0, proof, seed=4)[0]


def test_rejections():
    rng = np.random.default_rng(3)
    S = rng.integers(0, 32, size=50)
    proof = L.prove_lookup(S, 0, 5, seed=2)
    assert L.verify_lookup(S, 0, 5, proof, seed=2)[0]
    import copy
    for t in range(proof.log2_d):
        for q in range(4):
            bad = copy.deepcopy(proof)
            g = list(bad.rounds[t])
            g[q] = (g[q] + 1) % R_MOD
            bad.rounds[t] = tuple(g)
            assert not L.verify_lookup(S, 0, 5, bad, seed=2)[0]
    for name in ("a_r", "s_r", "b_r", "m_r"):
        bad = copy.deepcopy(proof)
        setattr(bad, name, (getattr(bad, name) + 1) % R_MOD)
        assert not L.verify_lookup(S, 0, 5, bad, seed=2)[0]
    bad = copy.deepcopy(proof)
    bad.state = bytes([bad.state[0] ^ 1]) + bad.state[1:]
    assert not L.verify_lookup(S, 0, 5, bad, seed=2)[0]
    assert not L.verify_lookup(S, 0, 5, proof, seed=3)[0]
    assert not L.verify_lookup(S, 0, 5, proof, seed=2, bind=b"\x01" * 32)[0]
    S2 = S.copy()
    S2[7] = (S2[7] + 1) % 32
    assert not L.verify_lookup(S2, 0, 5, proof, seed=2)[0]
    # values outside the table: the prover refuses, the verifier rejects
    S3 = S.copy()
    S3[0] = 32
    with pytest.raises(ValueError):
        L.prove_lookup(S3, 0, 5, seed=2)
    assert not L.verify_lookup(S3, 0, 5, proof, seed=2)[0]


def test_planted_mistakes_are_caught(monkeypatch):
    """Mistakes planted in the oracle (a wrong u_low block, a wrong N/D
    scalar, a degree-2 interpolation) each break a pin above."""
    S, t0, log2_n = [1, 2, 3, 0, 1, 1, 2, 0, 3, 3, 1], 0, 2

    def proves_and_verifies():
        try:
            p = L.prove_lookup(S, t0, log2_n, seed=5)
        except AssertionError:
            return False
        return L.verify_lookup(S, t0, log2_n, p, seed=5)[0]

    assert proves_and_verifies()
    orig_tv = L.term_vectors

    def first_coords(s_pad, t0_, N, beta, alpha, u):
        vec, c = orig_tv(s_pad, t0_, N, beta, alpha, u)
        ej = oracle.eq_table(u[:2])
        vec["Ej"] = [ej[k % N] for k in range(len(s_pad))]
        return vec, c

    monkeypatch.setattr(L, "term_vectors", first_coords)
    assert not proves_and_verifies()
    monkeypatch.setattr(L, "term_vectors", orig_tv)

    def inverted_scalar(s_pad, t0_, N, beta, alpha, u):
        vec, c = orig_tv(s_pad, t0_, N, beta, alpha, u)
        return vec, len(s_pad) * oracle.fr_inv(N) % R_MOD

    monkeypatch.setattr(L, "term_vectors", inverted_scalar)
    assert not proves_and_verifies()
    monkeypatch.setattr(L, "term_vectors", orig_tv)

    orig_cubic = L.cubic_eval
    monkeypatch.setattr(L, "cubic_eval", lambda g, x: oracle.round_poly_eval(g[0], g[1], g[2], x))
    assert not proves_and_verifies()
    monkeypatch.setattr(L, "cubic_eval", orig_cubic)
    assert proves_and_verifies()


def test_eq_value_low_block_is_the_last_coordinates():
    """eq(u, k) factors as eq(u_high, i) . eq(u_low, j) for k = i N + j, which
    is why the table side uses the last log2 N coordinates of u."""
    rng = random.Random(8)
    u = [_rand_fr(rng) for _ in range(5)]
    for k in range(32):
        i, j = k >> 2, k & 3
        assert eq_value(u, k) == eq_value(u[:3], i) * eq_value(u[3:], j) % R_MOD
