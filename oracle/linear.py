"""Linear zkMat: proof that sum_q c_q M_q = 0 by MLE linearity (oracle;
test infrastructure).

zkMat proves matrix additions as well as products (Sec. IV, putting
everything together).  Additions need no sumcheck: the MLE is linear in the
table (Eq. eq:MLE), so if sum_q c_q M_q = 0 entrywise then
sum_q c_q M_q~(x, y) = 0 at every point, and for a false relation the
left-hand side is a nonzero multilinear polynomial that vanishes at a random
point with probability at most (d0 + d1)/|F| (Schwartz-Zippel).  The LoRA
parameter update A' = A - eta dA (Eq. eq:grad_update_ab) is the instance
M = (A', A, dA), c = (1, -1, eta) over F.

Protocol (Fiat-Shamir; the byte format is this project's convention, so
parity unpinned for the format):
  S0 = SHA256(DOMAIN || seed u64le || rows, cols, q u32le
              || c_1 .. c_q (32 B each) || bind_1 .. bind_q (32 B each))
  x = squeeze('x', d0), y = squeeze('y', d1)    (d0 = ceil log2 rows, d1 for cols)
  e_q = M_q~(x, y);  absorb('e', e_1 .. e_q)
Proof: rows, cols, d0, d1, e_1 .. e_q, final state.  The verifier replays
the transcript, checks sum_q c_q e_q = 0, and evaluates M_q~(x, y) from the
matrices (the stand-in for commitment openings).

Pins (tests/test_oracle_linear.py): e_q against brute-force hypercube sums of
eq:MLE on tiny matrices; sum_q c_q M_q~ equal to the MLE of the entrywise
combination (linearity, checked against the combination computed with NumPy
int64); Boolean points recover entries; completeness; rejection of any
single-entry perturbation and of a proof with a wrong evaluation.
"""

from dataclasses import dataclass, field as dc_field

import numpy as np

from .field import R_MOD, fr_to_bytes
from .mle import mle_eval_matrix
from .sumcheck import ceil_log2
from .transcript import Transcript

DOMAIN = b"verilora-gb300/zklin/v1"


@dataclass
class LinearProof:
    rows: int
    cols: int
    d0: int
    d1: int
    evals: list
    state: bytes
    point: dict = dc_field(default_factory=dict, compare=False, repr=False)

    def to_bytes(self) -> bytes:
        """rows, cols, d0, d1, q as u32le, the evaluations, the final state."""
        out = b"".join(int(v).to_bytes(4, "little") for v in (self.rows, self.cols, self.d0, self.d1, len(self.evals)))
        return out + b"".join(fr_to_bytes(e) for e in self.evals) + bytes(self.state)


def _start(seed, rows, cols, coeffs, binds):
    T = Transcript.__new__(Transcript)  # same absorb / squeeze rules, its own start message
    msg = (DOMAIN + int(seed).to_bytes(8, "little") + int(rows).to_bytes(4, "little")
           + int(cols).to_bytes(4, "little") + len(coeffs).to_bytes(4, "little")
           + b"".join(fr_to_bytes(c % R_MOD) for c in coeffs) + b"".join(bytes(b) for b in binds))
    import hashlib
    T.state = hashlib.sha256(msg).digest()
    return T


def _binds(binds, q):
    if binds is None:
        return [bytes(32)] * q
    if len(binds) != q or any(len(b) != 32 for b in binds):
        raise ValueError("one 32-byte bind per matrix")
    return list(binds)


def prove_linear(mats, coeffs, seed=0, binds=None):
    """Proof that sum_q coeffs[q] * mats[q] = 0 (entrywise, mod r)."""
    mats = [np.asarray(M) for M in mats]
    if not mats or len(coeffs) != len(mats):
        raise ValueError("one coefficient per matrix")
    rows, cols = mats[0].shape
    if any(M.shape != (rows, cols) for M in mats):
        raise ValueError("matrices differ in shape")
    d0, d1 = ceil_log2(rows), ceil_log2(cols)
    T = _start(seed, rows, cols, coeffs, _binds(binds, len(mats)))
    x = T.squeeze(b"x", d0)
    y = T.squeeze(b"y", d1)
    evals = [mle_eval_matrix(M, x, y) for M in mats]
    T.absorb_fr(b"e", evals)
    return LinearProof(rows, cols, d0, d1, evals, T.state, point={"x": x, "y": y})


def verify_linear(mats, coeffs, proof, seed=0, binds=None):
    """(accept, reason)."""
    mats = [np.asarray(M) for M in mats]
    rows, cols = mats[0].shape
    if any(M.shape != (rows, cols) for M in mats) or len(coeffs) != len(mats):
        return False, "shape"
    d0, d1 = ceil_log2(rows), ceil_log2(cols)
    if (proof.rows, proof.cols, proof.d0, proof.d1, len(proof.evals)) != (rows, cols, d0, d1, len(mats)):
        return False, "dims"
    if any(not (0 <= e < R_MOD) for e in proof.evals):
        return False, "non-canonical element"
    T = _start(seed, rows, cols, coeffs, _binds(binds, len(mats)))
    x = T.squeeze(b"x", d0)
    y = T.squeeze(b"y", d1)
    if sum(c * e for c, e in zip(coeffs, proof.evals)) % R_MOD != 0:
        return False, "sum_q c_q e_q != 0"
    T.absorb_fr(b"e", proof.evals)
    if T.state != bytes(proof.state):
        return False, "transcript state"
    for q, M in enumerate(mats):
        if proof.evals[q] != mle_eval_matrix(M, x, y):
            return False, f"e_{q} != M_{q}~(x, y)"
    return True, "accept"
