"""Lookup-argument sumcheck (oracle; test infrastructure).

The lookup argument of Sec. II ("Lookup Arguments for Non-arithmetic
Operations"), Protocol 1 and Eq. eq:lookup-sumcheck, for a secret vector S
of D entries and a public table T of N entries (N, D powers of two, N | D):

* S is contained in T iff multiplicities m_j = |{i : S_i = T_j}| satisfy the
  rational-function identity (Eq. rational-function), i.e. at a random beta
      sum_i A_i = sum_j m_j B_j,   A_i = 1 / (beta + S_i),  B_j = 1 / (beta + T_j).
* With further randomness alpha and u in F^(log2 D), Eq. eq:lookup-sumcheck
  states that the polynomial over k = (i, j) in {0,1}^(log2 D) (i the high
  log2(D/N) bits, j the low log2 N bits)
      P(k) = alpha A(k) eq(u, k) (S(k) + beta) + A(k)
             + (N/D) alpha^2 B(j) eq(u_low, j) (T(j) + beta)
             - (N/D) B(j) m(j)
  sums to alpha + alpha^2 (u_low = the last log2 N coordinates of u).  A
  sumcheck over its log2 D variables (degree 3 in each: the product A.eq.S)
  reduces that to one evaluation of each vector at the final point.

Readings (the paper prints the identity only):
* the table is an integer range T_j = t0 + j, j < N (the range checks of
  rescale remainders, Sec. IV-A); S is an integer vector of n entries,
  padded with t0 to D = max(N, 2^ceil(log2 n)) entries (the padding is
  counted in m);
* "u, a binary vector" is a random point of F^(log2 D); the sum over
  "i (+) j" runs over the index i * N + j;
* commitments to S, m, A, B are out of scope: the verifier recomputes them
  from S and T and checks the final evaluations directly (the stand-in for
  opening proofs, as for the matmul sumcheck).

Protocol (Fiat-Shamir; byte format is this project's convention, so parity
unpinned for the format):
  S0 = SHA256(DOMAIN || seed u64le || n, log2 D, log2 N u32le || t0 i64le || bind)
  beta = squeeze('b', 1); alpha = squeeze('a', 1); u = squeeze('u', log2 D)
  claim_0 = alpha + alpha^2
  round t = 1 .. log2 D (variables bound from the most significant bit):
      g_t(X) at X = 0, 1, 2, 3 (degree 3); absorb('g', g0 || g2 || g3)
      (g1 = claim - g0 is implied); r_t = squeeze('r', 1); claim = g_t(r_t)
  finish: a_r = A~(r), s_r = S~(r), b_r = B~(r_low), m_r = m~(r_low);
      absorb('f', a_r || s_r || b_r || m_r)
  proof = (n, log2 D, log2 N, t0, rounds, a_r, s_r, b_r, m_r, final state)

Pins (tests/test_oracle_lookup.py): A and B against the inverse definition
(x . x^-1 = 1) and Python's modular inverse; m against np.bincount; the
rational identity; the cube sum of P equal to alpha + alpha^2 (closed form);
every round polynomial against a brute-force sum over the cube of P's
multilinear extension (eq:MLE written out) at small sizes, and degree <= 3
(a fifth point off the Lagrange curve through 0..3); g0 + g1 = claim; the
final claim against P's terms evaluated by definition; completeness;
rejection of perturbed proofs, of out-of-table values, and of a wrong
multiplicity vector (the first round check fails).
"""

import hashlib
from dataclasses import dataclass, field as dc_field

import numpy as np

from .field import R_MOD, fr_inv, fr_to_bytes
from .mle import eq_table, mle_eval_bruteforce
from .sumcheck import ceil_log2
from .transcript import Transcript

DOMAIN = b"verilora-gb300/zklookup/v1"


def cubic_eval(g, x: int) -> int:
    """g(x) for the polynomial of degree <= 3 through (0, g0) .. (3, g3) (Lagrange)."""
    x %= R_MOD
    total = 0
    for i in range(4):
        num, den = 1, 1
        for j in range(4):
            if j != i:
                num = num * (x - j) % R_MOD
                den = den * (i - j) % R_MOD
        total = (total + g[i] * num % R_MOD * fr_inv(den)) % R_MOD
    return total


@dataclass
class LookupProof:
    n: int
    log2_d: int
    log2_n: int
    t0: int
    rounds: list            # [(g0, g1, g2, g3)] per round
    a_r: int
    s_r: int
    b_r: int
    m_r: int
    state: bytes
    point: dict = dc_field(default_factory=dict, compare=False, repr=False)

    def to_bytes(self) -> bytes:
        """n, log2 D, log2 N as u32le, t0 as i64le, the rounds' four values,
        the four final evaluations, the final state."""
        out = b"".join(int(v).to_bytes(4, "little") for v in (self.n, self.log2_d, self.log2_n))
        out += int(self.t0).to_bytes(8, "little", signed=True)
        for g in self.rounds:
            out += b"".join(fr_to_bytes(v) for v in g)
        out += b"".join(fr_to_bytes(v) for v in (self.a_r, self.s_r, self.b_r, self.m_r))
        return out + bytes(self.state)


def lookup_dims(n: int, log2_n: int):
    """(D, log2 D) for n entries and a table of 2^log2_n entries."""
    log2_d = max(log2_n, ceil_log2(n))
    return 1 << log2_d, log2_d


def _start(seed, n, log2_d, log2_n, t0, bind):
    if len(bind) != 32:
        raise ValueError("the bind is 32 bytes")
    T = Transcript.__new__(Transcript)  # same absorb / squeeze rules, its own start message
    msg = (DOMAIN + int(seed).to_bytes(8, "little") + int(n).to_bytes(4, "little")
           + int(log2_d).to_bytes(4, "little") + int(log2_n).to_bytes(4, "little")
           + int(t0).to_bytes(8, "little", signed=True) + bytes(bind))
    T.state = hashlib.sha256(msg).digest()
    return T


def padded(S, t0, D):
    """S flattened (row-major) and padded with t0 to D entries (Python ints)."""
    s = [int(v) for v in np.asarray(S).reshape(-1)]
    return s + [int(t0)] * (D - len(s))


def multiplicities(s_pad, t0, N):
    """m_j = |{i : S_i = t0 + j}|; raises if a value lies outside the table."""
    idx = np.asarray(s_pad, dtype=np.int64) - int(t0)
    if idx.size and (idx.min() < 0 or idx.max() >= N):
        raise ValueError("a lookup value lies outside the table")
    return [int(c) for c in np.bincount(idx, minlength=N)]


def term_vectors(s_pad, t0, N, beta, alpha, u):
    """The seven vectors of P over the D-cube (Python ints mod r), each of
    length D: A, eq(u, .), S + beta, and the table-side B, eq(u_low, .),
    T + beta, m at j = k mod N; plus the scalar N / D."""
    D = len(s_pad)
    log2_n = ceil_log2(N) if N > 1 else 0
    A = [fr_inv((beta + s) % R_MOD) for s in s_pad]
    B = [fr_inv((beta + t0 + j) % R_MOD) for j in range(N)]
    m = multiplicities(s_pad, t0, N)
    E = eq_table(u)
    u_low = u[len(u) - log2_n:] if log2_n else []
    Ej = eq_table(u_low)
    vec = {
        "A": A, "E": E, "S": [(s + beta) % R_MOD for s in s_pad],
        "B": [B[k % N] for k in range(D)], "Ej": [Ej[k % N] for k in range(D)],
        "T": [(t0 + k % N + beta) % R_MOD for k in range(D)], "m": [m[k % N] for k in range(D)],
    }
    c = N * fr_inv(D) % R_MOD
    return vec, c


def p_value(v, alpha, c):
    """P at one point, from the values of the seven vectors there."""
    a2 = alpha * alpha % R_MOD
    return (alpha * v["A"] % R_MOD * v["E"] % R_MOD * v["S"] + v["A"]
            + c * (a2 * v["B"] % R_MOD * v["Ej"] % R_MOD * v["T"] - v["B"] * v["m"])) % R_MOD


def prove_lookup(S, t0, log2_n, seed=0, bind=bytes(32)):
    """Proof that every entry of S lies in T = [t0, t0 + 2^log2_n)."""
    N = 1 << log2_n
    n = int(np.asarray(S).size)
    if n < 1:
        raise ValueError("S is empty")
    D, log2_d = lookup_dims(n, log2_n)
    s_pad = padded(S, t0, D)
    multiplicities(s_pad, t0, N)  # refuses values outside the table before any transcript work
    T = _start(seed, n, log2_d, log2_n, t0, bind)
    beta = T.squeeze(b"b", 1)[0]
    if any((beta + t0 + j) % R_MOD == 0 for j in range(N)):
        raise ArithmeticError("beta + T_j = 0: no inverse (probability ~2^-239)")
    alpha = T.squeeze(b"a", 1)[0]
    u = T.squeeze(b"u", log2_d)
    vec, c = term_vectors(s_pad, t0, N, beta, alpha, u)
    claim = (alpha + alpha * alpha) % R_MOD
    rounds, rs = [], []
    for _ in range(log2_d):
        h = len(vec["A"]) // 2
        g = []
        for X in range(4):
            tot = 0
            for k in range(h):
                point = {name: (f[k] + X * (f[k + h] - f[k])) % R_MOD for name, f in vec.items()}
                tot += p_value(point, alpha, c)
            g.append(tot % R_MOD)
        assert (g[0] + g[1]) % R_MOD == claim, "round sum does not match the claim"
        T.absorb_fr(b"g", [g[0], g[2], g[3]])
        r = T.squeeze(b"r", 1)[0]
        rounds.append(tuple(g))
        rs.append(r)
        claim = cubic_eval(g, r)
        for name, f in vec.items():
            vec[name] = [(f[k] + r * (f[k + h] - f[k])) % R_MOD for k in range(h)]
    a_r, s_r, b_r, m_r = vec["A"][0], (vec["S"][0] - beta) % R_MOD, vec["B"][0], vec["m"][0]
    assert p_value({name: f[0] for name, f in vec.items()}, alpha, c) == claim
    T.absorb_fr(b"f", [a_r, s_r, b_r, m_r])
    return LookupProof(n, log2_d, log2_n, int(t0), rounds, a_r, s_r, b_r, m_r, T.state,
                       point={"beta": beta, "alpha": alpha, "u": u, "r": rs})


def verify_lookup(S, t0, log2_n, proof, seed=0, bind=bytes(32)):
    """(accept, reason).  Replays the transcript, checks every round against
    the running claim and the final claim against the sent evaluations, then
    checks those evaluations against S and T (the opening stand-in)."""
    N = 1 << log2_n
    n = int(np.asarray(S).size)
    if n < 1:
        return False, "empty"
    D, log2_d = lookup_dims(n, log2_n)
    if (proof.n, proof.log2_d, proof.log2_n, proof.t0, len(proof.rounds)) != (n, log2_d, log2_n, int(t0), log2_d):
        return False, "dims"
    vals = [v for g in proof.rounds for v in g] + [proof.a_r, proof.s_r, proof.b_r, proof.m_r]
    if any(not (0 <= v < R_MOD) for v in vals):
        return False, "non-canonical element"
    s_pad = padded(S, t0, D)
    try:
        m = multiplicities(s_pad, t0, N)
    except ValueError:
        return False, "a value lies outside the table"
    T = _start(seed, n, log2_d, log2_n, t0, bind)
    beta = T.squeeze(b"b", 1)[0]
    alpha = T.squeeze(b"a", 1)[0]
    u = T.squeeze(b"u", log2_d)
    claim = (alpha + alpha * alpha) % R_MOD
    rs = []
    for g in proof.rounds:
        if (g[0] + g[1]) % R_MOD != claim:
            return False, f"round {len(rs) + 1}: g(0) + g(1) != claim"
        T.absorb_fr(b"g", [g[0], g[2], g[3]])
        r = T.squeeze(b"r", 1)[0]
        rs.append(r)
        claim = cubic_eval(g, r)
    r_low = rs[log2_d - log2_n:] if log2_n else []
    u_low = u[log2_d - log2_n:] if log2_n else []
    e_r = mle_eval_bruteforce(eq_table(u), rs) if log2_d else 1
    ej_r = mle_eval_bruteforce(eq_table(u_low), r_low) if log2_n else 1
    t_r = mle_eval_bruteforce([t0 + j for j in range(N)], r_low) if log2_n else t0 % R_MOD
    c = N * fr_inv(D) % R_MOD
    final = p_value({"A": proof.a_r, "E": e_r, "S": (proof.s_r + beta) % R_MOD, "B": proof.b_r, "Ej": ej_r,
                     "T": (t_r + beta) % R_MOD, "m": proof.m_r}, alpha, c)
    if final != claim:
        return False, "final claim"
    T.absorb_fr(b"f", [proof.a_r, proof.s_r, proof.b_r, proof.m_r])
    if T.state != bytes(proof.state):
        return False, "transcript state"
    # Opening stand-in: the evaluations against the vectors recomputed from S and T.
    A = [fr_inv((beta + s) % R_MOD) for s in s_pad]
    B = [fr_inv((beta + t0 + j) % R_MOD) for j in range(N)]
    if proof.a_r != (mle_eval_bruteforce(A, rs) if log2_d else A[0]):
        return False, "a_r != A~(r)"
    if proof.s_r != (mle_eval_bruteforce([s % R_MOD for s in s_pad], rs) if log2_d else s_pad[0] % R_MOD):
        return False, "s_r != S~(r)"
    if proof.b_r != (mle_eval_bruteforce(B, r_low) if log2_n else B[0]):
        return False, "b_r != B~(r_low)"
    if proof.m_r != (mle_eval_bruteforce(m, r_low) if log2_n else m[0] % R_MOD):
        return False, "m_r != m~(r_low)"
    return True, "accept"
