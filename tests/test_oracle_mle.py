"""Pins for oracle/mle.py against Eq. eq:MLE written out by brute force."""
import itertools
import random

import numpy as np

from oracle.field import R_MOD
from oracle.mle import (eq_table, eq_value, mle_eval_bruteforce, mle_eval_matrix,
                        fold_rows, fold_cols)


def _rand_point(rng, ell):
    return [rng.randrange(R_MOD) for _ in range(ell)]


def _eq_literal(x, b):
    """prod_i (b_i x_i + (1 - b_i)(1 - x_i)) with b given as a bit tuple."""
    acc = 1
    for xi, bi in zip(x, b):
        acc = acc * (bi * xi + (1 - bi) * (1 - xi)) % R_MOD
    return acc


def test_eq_boolean_is_indicator():
    for ell in range(0, 5):
        for a in range(1 << ell):
            xa = [(a >> (ell - 1 - t)) & 1 for t in range(ell)]  # MSB first
            tab = eq_table(xa)
            assert tab == [1 if i == a else 0 for i in range(1 << ell)]


def test_eq_table_matches_literal_product_msb_first():
    rng = random.Random(1)
    for ell in range(1, 7):
        x = _rand_point(rng, ell)
        tab = eq_table(x)
        for i, bits in enumerate(itertools.product((0, 1), repeat=ell)):  # MSB varies slowest
            assert tab[i] == _eq_literal(x, bits)


def test_eq_table_sums_to_one():
    rng = random.Random(2)
    for ell in range(0, 9):
        assert sum(eq_table(_rand_point(rng, ell))) % R_MOD == 1


def test_eq_one_variable():
    x = 12345
    assert eq_table([x]) == [(1 - x) % R_MOD, x]


def test_mle_agrees_on_cube_and_is_multilinear():
    rng = random.Random(3)
    ell = 5
    f = [rng.randrange(-(1 << 15), 1 << 15) % R_MOD for _ in range(1 << ell)]
    for i in range(1 << ell):
        bits = [(i >> (ell - 1 - t)) & 1 for t in range(ell)]
        assert mle_eval_bruteforce(f, bits) == f[i]
    x = _rand_point(rng, ell)
    for t in range(ell):
        pts = []
        for val in (0, 1, 2, 3):
            y = list(x)
            y[t] = val
            pts.append(mle_eval_bruteforce(f, y))
        # Degree <= 1 in each variable: equally spaced values have constant difference.
        assert (pts[1] - pts[0]) % R_MOD == (pts[2] - pts[1]) % R_MOD == (pts[3] - pts[2]) % R_MOD


def test_matrix_mle_equals_bruteforce_on_flattened_index():
    rng = random.Random(4)
    for (rows, cols) in [(4, 8), (3, 5), (8, 2), (1, 4), (5, 1)]:
        M = np.array([[rng.randrange(-(1 << 15), 1 << 15) for _ in range(cols)] for _ in range(rows)])
        d0 = (rows - 1).bit_length()
        d1 = (cols - 1).bit_length()
        x = _rand_point(rng, d0)
        y = _rand_point(rng, d1)
        # Row-major padded matrix flattened: index = row * 2^d1 + col, row bits first.
        flat = [0] * (1 << (d0 + d1))
        for i in range(rows):
            for j in range(cols):
                flat[(i << d1) + j] = int(M[i, j]) % R_MOD
        assert mle_eval_matrix(M, x, y) == mle_eval_bruteforce(flat, x + y)


def test_folds_are_the_definition():
    rng = random.Random(5)
    M = np.array([[rng.randrange(-(1 << 15), 1 << 15) for _ in range(6)] for _ in range(5)])
    E = [rng.randrange(R_MOD) for _ in range(8)]
    fr_ = fold_rows(M, E)
    fc = fold_cols(M, E)
    for w in range(6):
        assert fr_[w] == sum(E[i] * int(M[i, w]) for i in range(5)) % R_MOD
    for w in range(5):
        assert fc[w] == sum(int(M[w, j]) * E[j] for j in range(6)) % R_MOD


def test_eq_value_consistent():
    rng = random.Random(6)
    x = _rand_point(rng, 4)
    assert [eq_value(x, i) for i in range(16)] == eq_table(x)


def test_mle_eval_bind_equals_bruteforce():
    from oracle.mle import mle_eval_bind
    rng = random.Random(11)
    for ell in range(0, 8):
        for n in {1, max(1, (1 << ell) - 3), 1 << ell}:
            f = [rng.randrange(R_MOD) if rng.random() < 0.7 else rng.randrange(-(1 << 15), 1 << 15)
                 for _ in range(n)]
            x = _rand_point(rng, ell)
            assert mle_eval_bind(f, x) == mle_eval_bruteforce([v % R_MOD for v in f], x)


def test_mle_eval_bind_on_cube_and_matrix():
    from oracle.mle import mle_eval_bind
    rng = np.random.default_rng(12)
    M = rng.integers(-(1 << 15), 1 << 15, size=(8, 16))
    r = random.Random(13)
    x, y = _rand_point(r, 3), _rand_point(r, 4)
    # row bits are the high variables: the flat row-major vector at (x, y)
    assert mle_eval_bind(M.reshape(-1).tolist(), x + y) == mle_eval_matrix(M, x, y)
    for i in range(16):
        bits = [(i >> (3 - t)) & 1 for t in range(4)]
        assert mle_eval_bind(M[0].tolist(), bits) == int(M[0, i]) % R_MOD


def test_mle_eval_bind_lsb_first_would_be_caught():
    from oracle.mle import mle_eval_bind
    rng = random.Random(14)
    f = [rng.randrange(R_MOD) for _ in range(16)]
    x = _rand_point(rng, 4)
    assert mle_eval_bind(f, x) != mle_eval_bind(f, x[::-1])  # the order matters ...
    assert mle_eval_bind(f, x) == mle_eval_bruteforce(f, x)  # ... and MSB first is eq:MLE's


def test_eq_eval_closed_form():
    from oracle.mle import eq_eval
    rng = random.Random(15)
    for ell in range(0, 7):
        x, y = _rand_point(rng, ell), _rand_point(rng, ell)
        assert eq_eval(x, y) == mle_eval_bruteforce(eq_table(x), y)
        assert eq_eval(x, y) == eq_eval(y, x)
        for i in range(1 << ell):
            bits = [(i >> (ell - 1 - t)) & 1 for t in range(ell)]
            assert eq_eval(x, bits) == eq_value(x, i)
