"""Sumcheck proof of a matrix product (oracle; test infrastructure).

What is proved (Sec. II-C, Eq. eq:matmul and eq:zk-mle-matmul; zkMat in
Sec. IV-B): for A = op(P) (m x k), B = op(Q) (k x n) and C = A.B, all padded
with zeros to D0 = 2^d0, D1 = 2^d1, D2 = 2^d2,
    sum_{w in {0,1}^d1} A~(u, w) B~(w, v) = C~(u, v).

Readings of the paper taken here (it is silent or garbled on these points):
* u in F^d0 and v in F^d2 are transcript challenges and the sumcheck runs over
  w only (d1 = log2 D1 rounds).  Summing over u, v and w as the text of
  Sec. II-C suggests would only prove sum(C) = sum(AB).
* The D1^-1 C~(u, v) term of eq:zk-mle-matmul is handled in the equivalent
  claim form sum_w A~(u,w) B~(w,v) = c.
* Each round message is the evaluations g_i(0), g_i(1), g_i(2) of the degree-2
  univariate round polynomial; variables are bound most-significant bit first,
  so round i pairs entries j and j + h with h = 2^(d1 - i) (Sec. II-B describes
  the rounds: one univariate polynomial per variable, a random challenge each).
* Commitments are out of scope: the verifier evaluates A~, B~, C~ directly
  from the matrices in place of polynomial-commitment openings.

Transcript order: squeeze u (d0), squeeze v (d2), absorb c, then per round
absorb (g0, g2) and squeeze r_i, then absorb (a_r, b_r).  A round absorbs
g(0) and g(2) only: g(1) is fixed by the running claim (the verifier checks
g(0) + g(1) = claim), so it would bind nothing new.

Pins (tests/test_oracle_sumcheck.py): brute-force round polynomials on the
hypercube, g_i(0) + g_i(1) = claim_{i-1}, degree <= 2, the final claim equal to
A~(u, r) B~(r, v) evaluated by definition, Boolean challenges giving the
integer matmul entry, k = 1 and m = n = 1 special cases, verifier completeness
and rejection of every single-field perturbation.
"""

from dataclasses import dataclass, field as dc_field

import numpy as np

from .field import R_MOD, fr_inv, fr_to_bytes
from .mle import eq_table, fold_rows, fold_cols, mle_eval_matrix
from .transcript import Transcript

INV2 = fr_inv(2)


def ceil_log2(x: int) -> int:
    if x < 1:
        raise ValueError("dimension must be >= 1")
    return (x - 1).bit_length()


def round_poly_eval(g0: int, g1: int, g2: int, x: int) -> int:
    """g(x) for the degree-2 polynomial through (0, g0), (1, g1), (2, g2) (Lagrange)."""
    x %= R_MOD
    l0 = (x - 1) * (x - 2) % R_MOD * INV2 % R_MOD
    l1 = (R_MOD - x * (x - 2) % R_MOD) % R_MOD
    l2 = x * (x - 1) % R_MOD * INV2 % R_MOD
    return (g0 * l0 + g1 * l1 + g2 * l2) % R_MOD


@dataclass
class Proof:
    m: int
    k: int
    n: int
    d0: int
    d1: int
    d2: int
    c: int
    g: list            # d1 triples (g(0), g(1), g(2))
    a_r: int
    b_r: int
    state: bytes       # final transcript state
    challenges: dict = dc_field(default_factory=dict, compare=False, repr=False)

    def to_bytes(self) -> bytes:
        """Canonical serialisation: six u32le dims, c, g triples, a_r, b_r, state."""
        out = b"".join(int(x).to_bytes(4, "little")
                       for x in (self.m, self.k, self.n, self.d0, self.d1, self.d2))
        out += fr_to_bytes(self.c)
        for tri in self.g:
            out += b"".join(fr_to_bytes(x) for x in tri)
        out += fr_to_bytes(self.a_r) + fr_to_bytes(self.b_r) + bytes(self.state)
        return out


def _op(M, trans):
    M = np.asarray(M)
    return M.T if trans else M


def prove_matmul(P, Q, trans_p=0, trans_q=0, seed=0, binds=(bytes(32),) * 3, override=None):
    """Prover: proof that op(P) . op(Q) = C, without reading C.

    ``override`` (tests only) replaces squeezed challenges after each squeeze,
    e.g. {'u': [...], 'v': [...], 'r': [...]} with Boolean values; the
    transcript still advances exactly as without it.
    """
    A = _op(P, trans_p)
    B = _op(Q, trans_q)
    m, k = A.shape
    k2, n = B.shape
    if k != k2:
        raise ValueError("inner dimensions differ")
    d0, d1, d2 = ceil_log2(m), ceil_log2(k), ceil_log2(n)
    ov = override or {}

    T = Transcript(seed, m, k, n, trans_p, trans_q, binds)
    u = T.squeeze(b"u", d0)
    v = T.squeeze(b"v", d2)
    if "u" in ov:
        u = [x % R_MOD for x in ov["u"]]
    if "v" in ov:
        v = [x % R_MOD for x in ov["v"]]

    c, g_all, rs, a_r, b_r = sumcheck_at(A, B, u, v, T, ov.get("r"))
    return Proof(m, k, n, d0, d1, d2, c, g_all, a_r, b_r, T.state,
                 challenges={"u": u, "v": v, "r": rs})


def sumcheck_at(A, B, u, v, T, r_override=None):
    """The claim, rounds and final values for A (m x k) . B (k x n) at the
    point (u, v), continuing transcript T (after its u, v squeezes):
    absorb c, per round absorb (g0, g2) and squeeze r, absorb (a_r, b_r).
    Returns (c, rounds, challenges, a_r, b_r)."""
    m, k = A.shape
    n = B.shape[1]
    d1 = ceil_log2(k)
    # Restrictions A~(u, .) and B~(., v) on the Boolean cube of w.
    fa = fold_rows(A, eq_table(u, m)) + [0] * ((1 << d1) - k)
    fb = fold_cols(B, eq_table(v, n)) + [0] * ((1 << d1) - k)

    c = sum(a * b for a, b in zip(fa, fb)) % R_MOD
    T.absorb_fr(b"c", [c])

    g_all, rs = [], []
    for i in range(d1):
        h = len(fa) // 2
        g0 = sum(fa[j] * fb[j] for j in range(h)) % R_MOD
        g1 = sum(fa[j + h] * fb[j + h] for j in range(h)) % R_MOD
        g2 = sum((2 * fa[j + h] - fa[j]) * (2 * fb[j + h] - fb[j]) for j in range(h)) % R_MOD
        g_all.append((g0, g1, g2))
        T.absorb_fr(b"g", [g0, g2])
        r = T.squeeze(b"r", 1)[0]
        if r_override is not None:
            r = r_override[i] % R_MOD
        rs.append(r)
        fa = [(fa[j] + r * (fa[j + h] - fa[j])) % R_MOD for j in range(h)]
        fb = [(fb[j] + r * (fb[j + h] - fb[j])) % R_MOD for j in range(h)]

    a_r, b_r = fa[0], fb[0]
    T.absorb_fr(b"f", [a_r, b_r])
    return c, g_all, rs, a_r, b_r


def verify_matmul(P, Q, C, proof, trans_p=0, trans_q=0, seed=0, binds=(bytes(32),) * 3):
    """Verifier.  Returns (accept: bool, reason: str).

    Replays the transcript, checks each round against the running claim, and
    evaluates A~(u, r), B~(r, v), C~(u, v) directly from the matrices (the
    stand-in for commitment openings).
    """
    A = _op(P, trans_p)
    B = _op(Q, trans_q)
    C = np.asarray(C)
    m, k = A.shape
    n = B.shape[1]
    if B.shape[0] != k or C.shape != (m, n):
        return False, "shape"
    d0, d1, d2 = ceil_log2(m), ceil_log2(k), ceil_log2(n)
    if (proof.m, proof.k, proof.n, proof.d0, proof.d1, proof.d2) != (m, k, n, d0, d1, d2):
        return False, "dims"
    if len(proof.g) != d1:
        return False, "round count"
    vals = [proof.c, proof.a_r, proof.b_r] + [x for tri in proof.g for x in tri]
    if any(not (0 <= x < R_MOD) for x in vals):
        return False, "non-canonical element"

    T = Transcript(seed, m, k, n, trans_p, trans_q, binds)
    u = T.squeeze(b"u", d0)
    v = T.squeeze(b"v", d2)
    if proof.c != mle_eval_matrix(C, u, v):
        return False, "claim c != C~(u, v)"
    T.absorb_fr(b"c", [proof.c])
    claim = proof.c
    rs = []
    for i, (g0, g1, g2) in enumerate(proof.g):
        if (g0 + g1) % R_MOD != claim:
            return False, f"round {i + 1}: g(0) + g(1) != claim"
        T.absorb_fr(b"g", [g0, g2])
        r = T.squeeze(b"r", 1)[0]
        rs.append(r)
        claim = round_poly_eval(g0, g1, g2, r)
    if claim != proof.a_r * proof.b_r % R_MOD:
        return False, "final claim != a_r * b_r"
    T.absorb_fr(b"f", [proof.a_r, proof.b_r])
    if T.state != bytes(proof.state):
        return False, "transcript state"
    if proof.a_r != mle_eval_matrix(A, u, rs):
        return False, "a_r != A~(u, r)"
    if proof.b_r != mle_eval_matrix(B, rs, v):
        return False, "b_r != B~(r, v)"
    return True, "accept"
