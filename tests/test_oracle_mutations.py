"""Plant plausible mistakes in the oracle (on the CPU) and check a pin catches each.

Each mutation is applied with monkeypatch to the oracle module only; the pin
functions from the other test files are then called and must fail.
"""
import numpy as np
import pytest

import oracle.mle as mle
import oracle.sumcheck as sc
from oracle.field import R_MOD

import test_oracle_mle as tm
import test_oracle_sumcheck as ts


def _fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_lsb_first_bit_order_is_caught(monkeypatch):
    monkeypatch.setattr(mle, "_bit", lambda i, t, ell: (i >> (t - 1)) & 1)
    _fails(tm.test_eq_table_matches_literal_product_msb_first)


def test_swapped_eq_factor_is_caught(monkeypatch):
    def bad(x, i):
        ell = len(x)
        acc = 1
        for t in range(1, ell + 1):
            b = (i >> (ell - t)) & 1
            acc = acc * ((1 - x[t - 1]) if b else x[t - 1]) % R_MOD
        return acc
    monkeypatch.setattr(mle, "eq_value", bad)
    _fails(tm.test_eq_table_matches_literal_product_msb_first)


def test_wrong_sign_in_round_message_is_caught(monkeypatch):
    real = sc.prove_matmul

    def patched(*a, **k):
        pf = real(*a, **k)
        pf.g = [(g0, g1, (g2 + 2 * g0) % R_MOD) for (g0, g1, g2) in pf.g]
        return pf
    monkeypatch.setattr(ts, "prove_matmul", patched)
    _fails(ts.test_rounds_match_bruteforce, 4, 8, 4)


def test_transposed_operand_in_fold_is_caught(monkeypatch):
    def bad(M, E):
        # Reads the stored matrix in the wrong orientation (M[w, i] for M[i, w]).
        M = np.asarray(M)
        rows, cols = M.shape
        return [sum(int(E[i]) * int(M[w % rows, i % cols]) for i in range(rows)) % R_MOD
                for w in range(cols)]
    monkeypatch.setattr(sc, "fold_rows", bad)
    _fails(ts.test_claim_and_final_by_definition, 4, 8, 4)


def test_dropped_term_in_round_is_caught():
    A = np.arange(32).reshape(4, 8) - 16
    B = np.arange(32).reshape(8, 4) - 9
    pf = sc.prove_matmul(A, B, seed=1)
    g = [list(t) for t in pf.g]
    g[0][0] = (g[0][0] - int(A[0, 0]) * int(B[0, 0])) % R_MOD  # one product left out
    pf.g = [tuple(t) for t in g]
    assert not sc.verify_matmul(A, B, A @ B, pf, seed=1)[0]


def test_missing_padding_zeros_is_caught(monkeypatch):
    real = sc.fold_cols

    def bad(M, E):
        out = real(M, E)
        return [(x + 1) % R_MOD for x in out]  # a stray constant term in every entry
    monkeypatch.setattr(sc, "fold_cols", bad)
    _fails(ts.test_claim_and_final_by_definition, 3, 5, 7)
