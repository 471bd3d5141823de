"""Batched-claim matmul sumcheck (oracle; test infrastructure).

Sec. IV ("putting everything together") composes the proofs of a LoRA step
by random aggregation of point-value claims under one Fiat-Shamir
transcript.  Here K products C_i = op(P_i) . op(Q_i) with a common inner
dimension k are proved by ONE sumcheck over w in {0,1}^(log2 k):

  each product i draws its own u_i, v_i (from a member transcript bound to
  the batch), and c_i = sum_w A_i~(u_i, w) B_i~(w, v_i) (= C_i~(u_i, v_i) for
  the honest C_i, as in Eq. eq:zk-mle-matmul);  the batch transcript binds
  every member state and claim, then draws rho, and the sumcheck proves
      sum_w sum_i rho^i A_i~(u_i, w) B_i~(w, v_i) = sum_i rho^i c_i
  (degree 2 in each variable; one round message and one challenge per
  variable for the whole batch).  At the end the prover sends
  a_i = A_i~(u_i, r), b_i = B_i~(r, v_i) and the verifier checks
  sum_i rho^i a_i b_i against the final claim.  A false c_i survives only if
  the random combination cancels (probability <= K/|F|).

Protocol (this project's byte convention; parity unpinned for the format):
  member start  M_i = SHA256("verilora-gb300/zkbatch/v1/member" || seed u64le
                  || K, i u32le || m_i, k, n_i u32le || transP, transQ u8
                  || bindP || bindQ || bindC)
  u_i = squeeze(M_i, 'u', d0_i), v_i = squeeze('v', d2_i)   (member state S_i)
  leaves        l_i = SHA256(0x00 || S_i || c_i)
  tree          node = SHA256(0x01 || left || right), leaves padded with
                32 zero bytes to a power of two; root R_c
  batch start   B = SHA256("verilora-gb300/zkbatch/v1" || seed u64le || K u32le || R_c)
  rho = squeeze(B, 'p', 1); claim = sum_i rho^i c_i
  rounds        g(0), g(1), g(2) of sum_i rho^i a_i(X, .) b_i(X, .);
                absorb('g', g0 || g2); r = squeeze('r', 1)
  final         leaves f_i = SHA256(0x00 || i u32le || a_i || b_i), root R_f;
                absorb('f', R_f)

Pins (tests/test_oracle_batch.py): each round polynomial equals
sum_i rho^i times that product's brute-force round polynomial (eq:MLE over
the cube) at the batch's challenges; K = 1 with rho^0 = 1 gives the
single-product sumcheck's polynomials at the same point; the final claim
against sum_i rho^i A_i~(u_i, r) B_i~(r, v_i) evaluated from the matrices;
the Merkle root against a hand-built two- and three-leaf tree; completeness;
rejection of a false C_j in any position and of perturbed proof values.
"""

import hashlib
from dataclasses import dataclass, field as dc_field

import numpy as np

from .field import R_MOD, fr_to_bytes
from .mle import eq_table, fold_cols, fold_rows, mle_eval_matrix
from .sumcheck import _op, ceil_log2, round_poly_eval
from .transcript import Transcript

DOMAIN = b"verilora-gb300/zkbatch/v1"
MEMBER = b"verilora-gb300/zkbatch/v1/member"


def _h(b: bytes) -> bytes:
    return hashlib.sha256(b).digest()


def merkle_root(leaves):
    """Root of the binary tree over 32-byte leaves (zero-padded to 2^t)."""
    if not leaves:
        raise ValueError("no leaves")
    level = list(leaves)
    size = 1
    while size < len(level):
        size *= 2
    level += [bytes(32)] * (size - len(level))
    while len(level) > 1:
        level = [_h(b"\x01" + level[2 * i] + level[2 * i + 1]) for i in range(len(level) // 2)]
    return level[0]


def member_state(seed, K, i, m, k, n, tp, tq, binds):
    msg = (MEMBER + int(seed).to_bytes(8, "little") + int(K).to_bytes(4, "little") + int(i).to_bytes(4, "little")
           + int(m).to_bytes(4, "little") + int(k).to_bytes(4, "little") + int(n).to_bytes(4, "little")
           + bytes([int(tp) & 1, int(tq) & 1]) + b"".join(bytes(b) for b in binds))
    T = Transcript.__new__(Transcript)
    T.state = _h(msg)
    return T


@dataclass
class BatchProof:
    K: int
    k: int
    d1: int
    dims: list            # (m_i, n_i, d0_i, d2_i)
    claims: list          # c_i
    rounds: list          # (g0, g1, g2)
    a: list
    b: list
    state: bytes
    point: dict = dc_field(default_factory=dict, compare=False, repr=False)

    def to_bytes(self) -> bytes:
        """K, k, d1 as u32le; the claims; the rounds' three values; a_i, b_i
        interleaved; the final state."""
        out = b"".join(int(v).to_bytes(4, "little") for v in (self.K, self.k, self.d1))
        out += b"".join(fr_to_bytes(c) for c in self.claims)
        for g in self.rounds:
            out += b"".join(fr_to_bytes(v) for v in g)
        for a, b in zip(self.a, self.b):
            out += fr_to_bytes(a) + fr_to_bytes(b)
        return out + bytes(self.state)


def _members(jobs, seed):
    """Per product: A, B (logical), dims, u, v, member state."""
    K = len(jobs)
    out = []
    k = None
    for i, j in enumerate(jobs):
        A, B = _op(j["P"], j.get("tp", 0)), _op(j["Q"], j.get("tq", 0))
        m, ki = A.shape
        k2, n = B.shape
        if ki != k2:
            raise ValueError("inner dimensions differ")
        if k is None:
            k = ki
        elif ki != k:
            raise ValueError("the products of a batch share the inner dimension")
        d0, d2 = ceil_log2(m), ceil_log2(n)
        T = member_state(seed, K, i, m, ki, n, j.get("tp", 0), j.get("tq", 0), j.get("binds", (bytes(32),) * 3))
        u = T.squeeze(b"u", d0)
        v = T.squeeze(b"v", d2)
        out.append({"A": A, "B": B, "m": m, "n": n, "d0": d0, "d2": d2, "u": u, "v": v, "S": T.state})
    return out, k


def _batch_start(seed, K, root):
    T = Transcript.__new__(Transcript)
    T.state = _h(DOMAIN + int(seed).to_bytes(8, "little") + int(K).to_bytes(4, "little") + root)
    return T


def prove_matmul_batch(jobs, seed=0):
    """One batched proof for jobs = [{"P", "Q", "tp", "tq", "binds"?}, ...]."""
    if not jobs:
        raise ValueError("empty batch")
    mem, k = _members(jobs, seed)
    K, d1 = len(jobs), ceil_log2(k)
    fa, fb, claims = [], [], []
    for x in mem:
        a = fold_rows(x["A"], eq_table(x["u"], x["m"])) + [0] * ((1 << d1) - k)
        b = fold_cols(x["B"], eq_table(x["v"], x["n"])) + [0] * ((1 << d1) - k)
        fa.append(a)
        fb.append(b)
        claims.append(sum(p * q for p, q in zip(a, b)) % R_MOD)
    root = merkle_root([_h(b"\x00" + x["S"] + fr_to_bytes(c)) for x, c in zip(mem, claims)])
    T = _batch_start(seed, K, root)
    rho = T.squeeze(b"p", 1)[0]
    w = [pow(rho, i, R_MOD) for i in range(K)]
    claim = sum(wi * c for wi, c in zip(w, claims)) % R_MOD
    rounds, rs = [], []
    for _ in range(d1):
        h = len(fa[0]) // 2
        g = [0, 0, 0]
        for i in range(K):
            a, b = fa[i], fb[i]
            g[0] += w[i] * sum(a[j] * b[j] for j in range(h))
            g[1] += w[i] * sum(a[j + h] * b[j + h] for j in range(h))
            g[2] += w[i] * sum((2 * a[j + h] - a[j]) * (2 * b[j + h] - b[j]) for j in range(h))
        g = [x % R_MOD for x in g]
        assert (g[0] + g[1]) % R_MOD == claim
        T.absorb_fr(b"g", [g[0], g[2]])
        r = T.squeeze(b"r", 1)[0]
        rounds.append(tuple(g))
        rs.append(r)
        claim = round_poly_eval(g[0], g[1], g[2], r)
        fa = [[(a[j] + r * (a[j + h] - a[j])) % R_MOD for j in range(h)] for a in fa]
        fb = [[(b[j] + r * (b[j + h] - b[j])) % R_MOD for j in range(h)] for b in fb]
    a_r = [a[0] for a in fa]
    b_r = [b[0] for b in fb]
    assert sum(wi * x * y for wi, x, y in zip(w, a_r, b_r)) % R_MOD == claim
    root_f = merkle_root([_h(b"\x00" + i.to_bytes(4, "little") + fr_to_bytes(x) + fr_to_bytes(y))
                          for i, (x, y) in enumerate(zip(a_r, b_r))])
    T.absorb(b"f", root_f)
    dims = [(x["m"], x["n"], x["d0"], x["d2"]) for x in mem]
    return BatchProof(K, k, d1, dims, claims, rounds, a_r, b_r, T.state,
                      point={"rho": rho, "r": rs, "u": [x["u"] for x in mem], "v": [x["v"] for x in mem]})


def verify_matmul_batch(jobs, Cs, proof, seed=0):
    """(accept, reason): the batch's claims against the claimed products Cs
    (evaluated from the matrices), the rounds, the final combination, and the
    final evaluations against the operands (the opening stand-in)."""
    try:
        mem, k = _members(jobs, seed)
    except ValueError as e:
        return False, str(e)
    K, d1 = len(jobs), ceil_log2(k)
    if (proof.K, proof.k, proof.d1, len(proof.claims), len(proof.rounds), len(proof.a), len(proof.b)) != \
            (K, k, d1, K, d1, K, K):
        return False, "dims"
    vals = list(proof.claims) + [v for g in proof.rounds for v in g] + list(proof.a) + list(proof.b)
    if any(not (0 <= v < R_MOD) for v in vals):
        return False, "non-canonical element"
    for i, (x, C) in enumerate(zip(mem, Cs)):
        if proof.claims[i] != mle_eval_matrix(np.asarray(C), x["u"], x["v"]):
            return False, f"c_{i} != C_{i}~(u_{i}, v_{i})"
    root = merkle_root([_h(b"\x00" + x["S"] + fr_to_bytes(c)) for x, c in zip(mem, proof.claims)])
    T = _batch_start(seed, K, root)
    rho = T.squeeze(b"p", 1)[0]
    w = [pow(rho, i, R_MOD) for i in range(K)]
    claim = sum(wi * c for wi, c in zip(w, proof.claims)) % R_MOD
    rs = []
    for t, g in enumerate(proof.rounds):
        if (g[0] + g[1]) % R_MOD != claim:
            return False, f"round {t + 1}: g(0) + g(1) != claim"
        T.absorb_fr(b"g", [g[0], g[2]])
        r = T.squeeze(b"r", 1)[0]
        rs.append(r)
        claim = round_poly_eval(g[0], g[1], g[2], r)
    if sum(wi * x * y for wi, x, y in zip(w, proof.a, proof.b)) % R_MOD != claim:
        return False, "final claim"
    root_f = merkle_root([_h(b"\x00" + i.to_bytes(4, "little") + fr_to_bytes(x) + fr_to_bytes(y))
                          for i, (x, y) in enumerate(zip(proof.a, proof.b))])
    T.absorb(b"f", root_f)
    if T.state != bytes(proof.state):
        return False, "transcript state"
    for i, x in enumerate(mem):
        if proof.a[i] != mle_eval_matrix(x["A"], x["u"], rs) or proof.b[i] != mle_eval_matrix(x["B"], rs, x["v"]):
            return False, f"final evaluations of product {i}"
    return True, "accept"
