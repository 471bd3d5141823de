"""Multilinear extensions and eq tables (oracle; test infrastructure).

Eq. eq:MLE (Sec. II-B) defines the MLE of f: {0,1}^l -> F as
    f~(x) = sum_b f(b) * prod_i (b_i x_i + (1 - b_i)(1 - x_i)).
The product is the Lagrange basis polynomial eq(x, b).

Bit order (the paper is silent): index i in [0, 2^l) is the bit vector
(b_1, ..., b_l) with b_1 the most significant bit, so b_t = (i >> (l - t)) & 1.
A row-major matrix M (D0 x D1, dims padded to powers of two with zeros,
Sec. II-C) has MLE M~(x, y) with x the row bits and y the column bits.

The fold of a matrix against an eq table is the restriction of its MLE to a
fixed first (or last) block of variables, evaluated on the Boolean cube of the
other block:
    fold_rows(M, E_u)[w] = sum_i E_u[i] M[i, w] = M~(u, w)
    fold_cols(M, E_v)[w] = sum_j M[w, j] E_v[j] = M~(w, v)
The vector-matrix product is a NumPy object-dtype matmul over Python ints
(a library matmul serving as one step), reduced mod r afterwards.

Pins (tests/test_oracle_mle.py): eq at Boolean points is the indicator; the
eq table sums to 1; the MLE agrees with the function on the cube; brute-force
eq:MLE equals the fold-based evaluation; multilinearity along each variable;
the variable-binding evaluation (mle_eval_bind) and eq at two field points
(eq_eval) equal the brute-force sums, and a binding order reversed to LSB
first is caught.
"""

import numpy as np

from .field import R_MOD


def _bit(i: int, t: int, ell: int) -> int:
    """b_t of index i (t = 1..ell, b_1 the MSB)."""
    return (i >> (ell - t)) & 1


def eq_value(x, i: int) -> int:
    """eq(x, bits(i)) = prod_t (b_t x_t + (1-b_t)(1-x_t)) mod r."""
    ell = len(x)
    acc = 1
    for t in range(1, ell + 1):
        b = _bit(i, t, ell)
        acc = acc * (x[t - 1] if b else (1 - x[t - 1])) % R_MOD
    return acc


def eq_table(x, size=None):
    """[eq(x, bits(i)) for i < size], size defaulting to 2^len(x).

    Written entry by entry from the product definition (no doubling trick).
    """
    ell = len(x)
    full = 1 << ell
    if size is None:
        size = full
    assert 0 <= size <= full
    return [eq_value(x, i) for i in range(size)]


def mle_eval_bruteforce(f, x) -> int:
    """Eq. eq:MLE summed literally over the whole hypercube (small l only)."""
    ell = len(x)
    assert len(f) <= (1 << ell)
    total = 0
    for i in range(1 << ell):
        fi = f[i] if i < len(f) else 0
        if fi % R_MOD == 0:
            continue
        total = (total + fi * eq_value(x, i)) % R_MOD
    return total


def _obj(a):
    return np.asarray(a).astype(object)


def fold_rows(M, E):
    """f[w] = sum_{i < rows} E[i] * M[i, w] mod r, for w < cols."""
    M = np.asarray(M)
    rows = M.shape[0]
    e = np.array([int(v) for v in E[:rows]], dtype=object)
    out = e.dot(_obj(M)) if rows else np.zeros(M.shape[1], dtype=object)
    return [int(v) % R_MOD for v in out]


def fold_cols(M, E):
    """f[w] = sum_{j < cols} M[w, j] * E[j] mod r, for w < rows."""
    M = np.asarray(M)
    cols = M.shape[1]
    e = np.array([int(v) for v in E[:cols]], dtype=object)
    out = _obj(M).dot(e) if cols else np.zeros(M.shape[0], dtype=object)
    return [int(v) % R_MOD for v in out]


def mle_eval_matrix(M, x, y) -> int:
    """M~(x, y) for a row-major integer matrix, x over row bits, y over column bits.

    Equals sum_{i,j} M[i, j] eq(x, i) eq(y, j) (eq:MLE with the row bits first).
    """
    M = np.asarray(M)
    Ex = eq_table(x, M.shape[0])
    Ey = eq_table(y, M.shape[1])
    f = fold_rows(M, Ex)
    return sum(a * b for a, b in zip(f, Ey)) % R_MOD


def mle_eval_bind(f, x) -> int:
    """f~(x) for a vector f of at most 2^len(x) entries (zero-padded), by
    binding the variables one at a time, most significant first.

    eq:MLE is linear in each variable; in x_1 (the MSB) its two values are
    the MLEs of the halves f[0:h] and f[h:2h], so
        f~(x_1, x_2, ..) = g~(x_2, ..),  g[j] = f[j] + x_1 (f[j + h] - f[j]).
    Repeating this l times leaves one entry.  Same value as
    mle_eval_bruteforce with O(2^l) products instead of O(l 2^l); NumPy
    object arrays of Python ints hold the vectors.
    """
    ell = len(x)
    n = len(f)
    assert n <= (1 << ell)
    v = np.zeros(1 << ell, dtype=object)
    v[:] = 0
    v[:n] = [int(a) % R_MOD for a in f]
    for t in range(ell):
        h = len(v) // 2
        v = (v[:h] + int(x[t]) * (v[h:] - v[:h])) % R_MOD
    return int(v[0]) % R_MOD


def eq_eval(x, y) -> int:
    """eq(x, y) = prod_t (x_t y_t + (1 - x_t)(1 - y_t)) for two points of
    F^l: the Lagrange basis product of eq:MLE with the Boolean b replaced by
    a second field point (the MLE of eq_table(x) evaluated at y)."""
    assert len(x) == len(y)
    acc = 1
    for a, b in zip(x, y):
        acc = acc * ((a * b + (1 - a) * (1 - b)) % R_MOD) % R_MOD
    return acc
