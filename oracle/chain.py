"""Chained proof of one LoRA projection (oracle; test infrastructure).

Sec. IV ("putting everything together") composes the proofs of a LoRA step
sequentially: the claim a sub-proof leaves on an intermediate tensor is not
opened, it is reduced to claims on the tensors that produced it, until only
claims on committed inputs, witnesses and outputs remain (zkLLM-style
sequential composition).  This module does that inside one projection of the
step (X.A.B convention, Y = X.W + H.B with H = rescale(X.A)):

  outputs    Y = X.W + H.B,  dX = dY.W^T + dH.A^T,  dA = X^T.dH,  dB = H^T.dY
  rescales   X.A + 2^7 = 2^8 H + rho_H,   dY.B^T + 2^7 = 2^8 dH + rho_dH
             (Sec. IV-A, zkSwiGLU's quantisation z = zeta z' + r with
             zeta = 2^8; the remainders rho are committed witnesses whose
             range the lookup argument proves, Protocol 1)

The intermediates H, dH, X.A and dY.B^T are never opened.  Each claim on H
(or dH) that a sumcheck leaves becomes, through the rescale relation (linear
in the MLEs, Eq. eq:MLE),
    (X.A)~(p) = 2^8 H~(p) + rho_H~(p) - 2^7 J~(p)
with J the all-ones n x r matrix, and the sumcheck of X.A at the point p
(Eq. eq:zk-mle-matmul with (u, v) = p) reduces it to claims on X and A.

Protocol (this project's byte convention; parity unpinned for the format):
  S0 = SHA256("verilora-gb300/zkchain/v1" || seed u64le || n, d, k, r u32le
              || bind_X, bind_W, bind_A, bind_B, bind_dY, bind_rhoH, bind_rhodH)
  squeeze('p', ...) gives, in order, u_Y, v_Y (log n, log k), u_dX, v_dX
  (log n, log d), u_dA, v_dA (log d, log r), u_dB, v_dB (log r, log k): S1
  stage 1, member p from M_p = SHA256(S1 || 'M' || p u32le), each the
  sumcheck of Eq. eq:zk-mle-matmul at the given point (absorb c, rounds,
  absorb a_r || b_r; final member state F_p):
      0 F1 X.W at (u_Y, v_Y)       1 F3 H.B at (u_Y, v_Y)
      2 B4 dY.W^T at (u_dX, v_dX)  3 B5 dH.A^T at (u_dX, v_dX)
      4 B3 X^T.dH at (u_dA, v_dA)  5 B2 H^T.dY at (u_dB, v_dB)
  S2 = SHA256(S1 || 'L' || F_0 .. F_5)
  the claims on the intermediates (r^p: member p's round challenges):
      p1 = (u_Y, r^1)   H~ from F3's a_r      p2 = (r^5, u_dB)  H~ from B2's a_r
      q1 = (u_dX, r^3)  dH~ from B5's a_r     q2 = (r^4, v_dA)  dH~ from B3's b_r
  e = (rho_H~(p1), rho_H~(p2), rho_dH~(q1), rho_dH~(q2)); S3 = absorb(S2, 'e', e)
  stage 3, members from M_p = SHA256(S3 || 'M' || p):
      6 F2 X.A at p1   7 F2 X.A at p2   8 B1 dY.B^T at q1   9 B1 dY.B^T at q2
  final state SHA256(S3 || 'Z' || F_6 .. F_9)

Verifier: replays everything; checks the output claims c_0 + c_1 = Y~(u_Y,
v_Y), c_2 + c_3 = dX~(u_dX, v_dX), c_4 = dA~(u_dA, v_dA), c_5 = dB~(u_dB,
v_dB) against the claimed outputs; each stage-3 claim against the value the
rescale relation derives (c_6 = 2^8 a_r^1 + e_0 - 2^7 J~(p1), and so on);
and opens only X, W, A, B, dY, rho_H, rho_dH (directly from the matrices:
the stand-in for commitment openings).

Pins (tests/test_oracle_chain.py): the derived-claim identity against the
MLE of the integer product X.A at random points (brute force), J~ against a
brute-force sum, every member claim against the MLE of its integer product,
completeness on ragged shapes, and rejection of a wrong H, dH, rho, output,
and of every perturbed proof value.
"""

import hashlib
from dataclasses import dataclass, field as dc_field

import numpy as np

from .field import R_MOD, fr_to_bytes
from .mle import eq_table, mle_eval_matrix
from .sumcheck import ceil_log2, round_poly_eval, sumcheck_at
from .transcript import Transcript

DOMAIN = b"verilora-gb300/zkchain/v1"
SHIFT = 8  # rescale zeta = 2^8
STAGE1 = ("F1", "F3", "B4", "B5", "B3", "B2")
STAGE3 = ("F2@p1", "F2@p2", "B1@q1", "B1@q2")


def _h(b: bytes) -> bytes:
    return hashlib.sha256(b).digest()


def _state(s: bytes) -> Transcript:
    T = Transcript.__new__(Transcript)
    T.state = s
    return T


def member_start(S: bytes, p: int) -> bytes:
    return _h(S + b"M" + int(p).to_bytes(4, "little"))


def ones_mle(x, y, rows, cols) -> int:
    """J~(x, y) for the all-ones rows x cols matrix (zero-padded):
    (sum_{i < rows} eq(x, i)) (sum_{j < cols} eq(y, j))."""
    return sum(eq_table(x, rows)) % R_MOD * (sum(eq_table(y, cols)) % R_MOD) % R_MOD


@dataclass
class SubProof:
    c: int
    g: list
    a_r: int
    b_r: int
    state: bytes
    r: list = dc_field(default_factory=list, compare=False, repr=False)

    def to_bytes(self, m, k, n) -> bytes:
        d0, d1, d2 = ceil_log2(m), ceil_log2(k), ceil_log2(n)
        out = b"".join(int(x).to_bytes(4, "little") for x in (m, k, n, d0, d1, d2))
        out += fr_to_bytes(self.c) + b"".join(fr_to_bytes(x) for tri in self.g for x in tri)
        return out + fr_to_bytes(self.a_r) + fr_to_bytes(self.b_r) + bytes(self.state)


@dataclass
class ChainProof:
    n: int
    d: int
    k: int
    r: int
    subs: list      # 10 SubProof, members 0..9
    e: list         # 4 remainder evaluations
    state: bytes
    shapes: list = dc_field(default_factory=list, compare=False, repr=False)

    def to_bytes(self) -> bytes:
        out = b"".join(int(x).to_bytes(4, "little") for x in (self.n, self.d, self.k, self.r))
        for sp, (m, k, n) in zip(self.subs, self.shapes):
            out += sp.to_bytes(m, k, n)
        return out + b"".join(fr_to_bytes(x) for x in self.e) + bytes(self.state)


def _dims(X, W, A):
    n, d = X.shape
    k = W.shape[1]
    r = A.shape[1]
    return n, d, k, r


def _start(seed, n, d, k, r, binds):
    if len(binds) != 7 or any(len(b) != 32 for b in binds):
        raise ValueError("seven 32-byte binds")
    msg = DOMAIN + int(seed).to_bytes(8, "little") + b"".join(int(x).to_bytes(4, "little") for x in (n, d, k, r))
    return _state(_h(msg + b"".join(bytes(b) for b in binds)))


def _points(T, n, d, k, r):
    ln, ld, lk, lr = (ceil_log2(x) for x in (n, d, k, r))
    sizes = (ln, lk, ln, ld, ld, lr, lr, lk)
    xs = T.squeeze(b"p", sum(sizes))
    out, o = [], 0
    for s in sizes:
        out.append(xs[o:o + s])
        o += s
    uY, vY, udX, vdX, udA, vdA, udB, vdB = out
    return {"Y": (uY, vY), "dX": (udX, vdX), "dA": (udA, vdA), "dB": (udB, vdB)}


def _operands(t):
    """(A, B) = (op(P), op(Q)) of the ten members, as int arrays."""
    X, W, A, B, dY, H, dH = (np.asarray(t[x]) for x in ("X", "W", "A", "B", "dY", "H", "dH"))
    return [(X, W), (H, B), (dY, W.T), (dH, A.T), (X.T, dH), (H.T, dY),
            (X, A), (X, A), (dY, B.T), (dY, B.T)]


def _stage1_points(P):
    return [P["Y"], P["Y"], P["dX"], P["dX"], P["dA"], P["dB"]]


def _stage3_points(P, rs):
    """p1, p2 (on H) and q1, q2 (on dH) from the stage-1 points and the
    stage-1 members' round challenges rs[p]."""
    p1 = (P["Y"][0], rs[1])
    p2 = (rs[5], P["dB"][0])
    q1 = (P["dX"][0], rs[3])
    q2 = (rs[4], P["dA"][1])
    return [p1, p2, q1, q2]


def _member(Aop, Bop, S, p, u, v):
    T = _state(member_start(S, p))
    c, g, rs, a_r, b_r = sumcheck_at(Aop, Bop, u, v, T)
    return SubProof(c, g, a_r, b_r, T.state, rs)


def prove_chain(t, seed=0, binds=(bytes(32),) * 7):
    """Chained proof of one projection.  t: the projection's tensors X, W, A,
    B, dY, H, dH, rhoH, rhodH (int16 arrays)."""
    X, W, A = (np.asarray(t[x]) for x in ("X", "W", "A"))
    n, d, k, r = _dims(X, W, A)
    T = _start(seed, n, d, k, r, binds)
    P = _points(T, n, d, k, r)
    S1 = T.state
    ops = _operands(t)
    subs = [_member(*ops[p], S1, p, *pt) for p, pt in enumerate(_stage1_points(P))]
    T.absorb(b"L", b"".join(sp.state for sp in subs))
    pts = _stage3_points(P, [sp.r for sp in subs])
    rhoH, rhodH = np.asarray(t["rhoH"]), np.asarray(t["rhodH"])
    e = [mle_eval_matrix(rhoH, *pts[0]), mle_eval_matrix(rhoH, *pts[1]),
         mle_eval_matrix(rhodH, *pts[2]), mle_eval_matrix(rhodH, *pts[3])]
    T.absorb_fr(b"e", e)
    S3 = T.state
    subs += [_member(*ops[6 + i], S3, 6 + i, *pts[i]) for i in range(4)]
    T.absorb(b"Z", b"".join(sp.state for sp in subs[6:]))
    shapes = [(a.shape[0], a.shape[1], b.shape[1]) for a, b in ops]
    return ChainProof(n, d, k, r, subs, e, T.state, shapes)


def derived_claims(subs, e, pts, n, r):
    """The stage-3 claims the rescale relations give: (X.A)~ at p1, p2 and
    (dY.B^T)~ at q1, q2 from the claims on H and dH and the remainders."""
    z, half = 1 << SHIFT, 1 << (SHIFT - 1)
    onH = [subs[1].a_r, subs[5].a_r, subs[3].a_r, subs[4].b_r]
    return [(z * onH[i] + e[i] - half * ones_mle(pts[i][0], pts[i][1], n, r)) % R_MOD for i in range(4)]


def _replay_member(sp, S, p, k):
    """Member p's rounds from its start state; returns (ok, reason, challenges)."""
    T = _state(member_start(S, p))
    T.absorb_fr(b"c", [sp.c])
    claim, rs = sp.c, []
    if len(sp.g) != ceil_log2(k):
        return False, "round count", rs
    for i, (g0, g1, g2) in enumerate(sp.g):
        if (g0 + g1) % R_MOD != claim:
            return False, f"round {i + 1}: g(0) + g(1) != claim", rs
        T.absorb_fr(b"g", [g0, g2])
        x = T.squeeze(b"r", 1)[0]
        rs.append(x)
        claim = round_poly_eval(g0, g1, g2, x)
    if claim != sp.a_r * sp.b_r % R_MOD:
        return False, "final claim != a_r * b_r", rs
    T.absorb_fr(b"f", [sp.a_r, sp.b_r])
    if T.state != bytes(sp.state):
        return False, "member transcript state", rs
    return True, "", rs


def verify_chain(t, outputs, proof, seed=0, binds=(bytes(32),) * 7):
    """(accept, reason).  t: X, W, A, B, dY, rhoH, rhodH (H and dH are not
    read); outputs: the claimed Y, dX, dA, dB (int64)."""
    X, W, A, B, dY = (np.asarray(t[x]) for x in ("X", "W", "A", "B", "dY"))
    rhoH, rhodH = np.asarray(t["rhoH"]), np.asarray(t["rhodH"])
    n, d, k, r = _dims(X, W, A)
    if (proof.n, proof.d, proof.k, proof.r) != (n, d, k, r) or len(proof.subs) != 10 or len(proof.e) != 4:
        return False, "dims"
    vals = list(proof.e) + [x for sp in proof.subs for x in [sp.c, sp.a_r, sp.b_r] + [y for g in sp.g for y in g]]
    if any(not (0 <= x < R_MOD) for x in vals):
        return False, "non-canonical element"
    inner = [d, r, k, r, n, n, d, d, k, k]
    T = _start(seed, n, d, k, r, binds)
    P = _points(T, n, d, k, r)
    S1 = T.state
    subs = proof.subs
    rs = []
    for p in range(6):
        ok, why, ch = _replay_member(subs[p], S1, p, inner[p])
        if not ok:
            return False, f"member {STAGE1[p]}: {why}"
        rs.append(ch)
    # output claims against the claimed outputs
    Y, dX, dA, dB = (np.asarray(outputs[x]) for x in ("Y", "dX", "dA", "dB"))
    if (subs[0].c + subs[1].c) % R_MOD != mle_eval_matrix(Y, *P["Y"]):
        return False, "c(F1) + c(F3) != Y~(u, v)"
    if (subs[2].c + subs[3].c) % R_MOD != mle_eval_matrix(dX, *P["dX"]):
        return False, "c(B4) + c(B5) != dX~(u, v)"
    if subs[4].c != mle_eval_matrix(dA, *P["dA"]):
        return False, "c(B3) != dA~(u, v)"
    if subs[5].c != mle_eval_matrix(dB, *P["dB"]):
        return False, "c(B2) != dB~(u, v)"
    # openings of the inputs at the stage-1 final points
    (uY, vY), (udX, vdX), (udA, vdA), (udB, vdB) = P["Y"], P["dX"], P["dA"], P["dB"]
    checks = [
        (subs[0].a_r, X, uY, rs[0], "F1 a_r"), (subs[0].b_r, W, rs[0], vY, "F1 b_r"),
        (subs[1].b_r, B, rs[1], vY, "F3 b_r"),
        (subs[2].a_r, dY, udX, rs[2], "B4 a_r"), (subs[2].b_r, W, vdX, rs[2], "B4 b_r"),
        (subs[3].b_r, A, vdX, rs[3], "B5 b_r"),
        (subs[4].a_r, X, rs[4], udA, "B3 a_r"),
        (subs[5].b_r, dY, rs[5], vdB, "B2 b_r"),
    ]
    for val, M, x, y, what in checks:
        if val != mle_eval_matrix(M, x, y):
            return False, f"{what} != opening"
    T.absorb(b"L", b"".join(bytes(sp.state) for sp in subs[:6]))
    pts = _stage3_points(P, rs)
    e = proof.e
    if e != [mle_eval_matrix(rhoH, *pts[0]), mle_eval_matrix(rhoH, *pts[1]),
             mle_eval_matrix(rhodH, *pts[2]), mle_eval_matrix(rhodH, *pts[3])]:
        return False, "remainder evaluations"
    T.absorb_fr(b"e", e)
    S3 = T.state
    want = derived_claims(subs, e, pts, n, r)
    for i in range(4):
        sp = subs[6 + i]
        if sp.c != want[i]:
            return False, f"member {STAGE3[i]}: claim != rescale-derived claim"
        ok, why, ch = _replay_member(sp, S3, 6 + i, inner[6 + i])
        if not ok:
            return False, f"member {STAGE3[i]}: {why}"
        x, y = pts[i]
        if i < 2:
            if sp.a_r != mle_eval_matrix(X, x, ch) or sp.b_r != mle_eval_matrix(A, ch, y):
                return False, f"member {STAGE3[i]}: final values != openings"
        else:
            if sp.a_r != mle_eval_matrix(dY, x, ch) or sp.b_r != mle_eval_matrix(B, y, ch):
                return False, f"member {STAGE3[i]}: final values != openings"
    T.absorb(b"Z", b"".join(bytes(sp.state) for sp in subs[6:]))
    if T.state != bytes(proof.state):
        return False, "transcript state"
    return True, "accept"
