"""Pins of the linear zkMat oracle (matrix additions by MLE linearity)."""
import itertools
import random

import numpy as np
import pytest

import oracle
from oracle.field import R_MOD
from oracle.mle import mle_eval_bruteforce, mle_eval_matrix


def _rand(rng, shape, lo=-(1 << 15), hi=1 << 15):
    return rng.integers(lo, hi, size=shape).astype(np.int64)


def _update_instance(rng, rows, cols, eta):
    """A' = A - eta dA with small entries so that A' stays an integer matrix."""
    A = _rand(rng, (rows, cols), -1000, 1000)
    dA = _rand(rng, (rows, cols), -100, 100)
    return [A - eta * dA, A, dA], [1, -1, eta]


def test_evaluations_are_hypercube_sums():
    rng = np.random.default_rng(1)
    M = _rand(rng, (3, 5))
    pf = oracle.prove_linear([M, -M], [1, 1], seed=3)
    x, y = pf.point["x"], pf.point["y"]
    # eq:MLE as a sum over the padded 4 x 8 cube, rows first
    table = [int(M[i][j]) if i < 3 and j < 5 else 0 for i in range(4) for j in range(8)]
    assert pf.evals[0] == mle_eval_bruteforce(table, list(x) + list(y))
    assert (pf.evals[0] + pf.evals[1]) % R_MOD == 0


def test_linearity_matches_the_mle_of_the_combination():
    rng = np.random.default_rng(2)
    mats = [_rand(rng, (6, 7)) for _ in range(3)]
    coeffs = [5, -3, 11]
    combo = sum(c * M for c, M in zip(coeffs, mats))  # exact int64 entrywise combination
    pf = oracle.prove_linear(mats + [combo], coeffs + [-1], seed=9)
    x, y = pf.point["x"], pf.point["y"]
    assert pf.evals[3] == mle_eval_matrix(combo, x, y)
    assert sum(c * e for c, e in zip(coeffs, pf.evals[:3])) % R_MOD == pf.evals[3]
    assert oracle.verify_linear(mats + [combo], coeffs + [-1], pf, seed=9)[0]


def test_boolean_points_recover_entries():
    rng = np.random.default_rng(3)
    M = _rand(rng, (4, 4))
    for i, j in itertools.product(range(4), range(4)):
        x = [(i >> 1) & 1, i & 1]
        y = [(j >> 1) & 1, j & 1]
        assert mle_eval_matrix(M, x, y) == int(M[i][j]) % R_MOD


@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (7, 1), (5, 6), (16, 16), (33, 20)])
def test_parameter_update_is_accepted(shape):
    rng = np.random.default_rng(sum(shape))
    mats, coeffs = _update_instance(rng, *shape, eta=3)
    pf = oracle.prove_linear(mats, coeffs, seed=shape[0] * 100 + shape[1])
    assert oracle.verify_linear(mats, coeffs, pf, seed=shape[0] * 100 + shape[1]) == (True, "accept")


def test_every_single_entry_perturbation_is_rejected():
    rng = np.random.default_rng(4)
    mats, coeffs = _update_instance(rng, 3, 5, eta=2)
    for q in range(3):
        for i in range(3):
            for j in range(5):
                bad = [M.copy() for M in mats]
                bad[q][i, j] += 1
                pf = oracle.prove_linear(bad, coeffs, seed=1)
                ok, why = oracle.verify_linear(bad, coeffs, pf, seed=1)
                assert not ok and why == "sum_q c_q e_q != 0"


def test_tampered_proofs_are_rejected():
    rng = np.random.default_rng(5)
    mats, coeffs = _update_instance(rng, 4, 4, eta=5)
    pf = oracle.prove_linear(mats, coeffs, seed=7)
    pf2 = oracle.LinearProof(pf.rows, pf.cols, pf.d0, pf.d1, list(pf.evals), pf.state)
    # shift two evaluations so the sum still vanishes: caught by the openings
    pf2.evals[1] = (pf2.evals[1] + 1) % R_MOD
    pf2.evals[0] = (pf2.evals[0] + 1) % R_MOD
    ok, why = oracle.verify_linear(mats, coeffs, pf2, seed=7)
    assert not ok
    assert not oracle.verify_linear(mats, coeffs, pf, seed=8)[0]  # another seed, another point
    assert not oracle.verify_linear(mats, [1, -1, 4], pf, seed=7)[0]  # another coefficient


def test_row_and_column_variables_are_not_swapped():
    """A planted mistake (the row point used for the columns and vice versa)
    changes the evaluation of a non-symmetric matrix, and the verifier that
    evaluates correctly rejects a proof built with it."""
    rng = np.random.default_rng(6)
    M = _rand(rng, (4, 4))
    assert not np.array_equal(M, M.T)
    pf = oracle.prove_linear([M, -M], [1, 1], seed=2)
    x, y = pf.point["x"], pf.point["y"]
    swapped = mle_eval_matrix(M, y, x)
    assert swapped != pf.evals[0]
    bad = oracle.LinearProof(pf.rows, pf.cols, pf.d0, pf.d1, [swapped, (-swapped) % R_MOD], pf.state)
    assert not oracle.verify_linear([M, -M], [1, 1], bad, seed=2)[0]


def test_planted_mistakes_are_caught(monkeypatch):
    """Mistakes planted in the oracle's evaluation (the row and column points
    swapped, the point's variables in reverse order) each fail the
    hypercube-sum pin or completeness."""
    from oracle import linear as OLin
    rng = np.random.default_rng(7)
    M = _rand(rng, (4, 4))
    mats, coeffs = [M, -M], [1, 1]

    def pinned():
        pf = oracle.prove_linear(mats, coeffs, seed=4)
        x, y = pf.point["x"], pf.point["y"]
        table = [int(M[i][j]) for i in range(4) for j in range(4)]
        ok_eval = pf.evals[0] == mle_eval_bruteforce(table, list(x) + list(y))
        return ok_eval and oracle.verify_linear(mats, coeffs, pf, seed=4)[0]

    assert pinned()
    orig = OLin.mle_eval_matrix
    monkeypatch.setattr(OLin, "mle_eval_matrix", lambda A, x, y: orig(A, y, x))
    assert not pinned()
    monkeypatch.setattr(OLin, "mle_eval_matrix", lambda A, x, y: orig(A, list(x)[::-1], list(y)[::-1]))
    assert not pinned()
    monkeypatch.setattr(OLin, "mle_eval_matrix", orig)
    assert pinned()
