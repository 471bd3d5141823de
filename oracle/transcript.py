"""SHA-256 Fiat-Shamir transcript (oracle; test infrastructure).

The paper makes its protocol non-interactive with the Fiat-Shamir heuristic:
each verifier challenge is a hash of every commitment and prover message sent
before it (Sec. IV-A, footnote to zkSwiGLU; Sec. V, random-oracle model).  It
fixes no hash, byte layout or sampling rule; this project's convention is:

* state      S is 32 bytes.
* start      S0 = SHA256(DOMAIN || seed:u64le || m:u32le || k:u32le || n:u32le
                         || transP:u8 || transQ:u8 || bindP || bindQ || bindC)
             where each bind is 32 bytes (a commitment stand-in; zeros by
             default).
* absorb     S <- SHA256(S || label:1 byte || data)
* squeeze    count challenges from one state, in counter mode:
             x_t = LE512(SHA256(S || label || t:u32le || 0x00) ||
                         SHA256(S || label || t:u32le || 0x01)) mod r,
             for t = 0..count-1, then S <- SHA256(S || label || count:u32le).
             (The 512-bit reduction leaves a bias below 2^-256.)

Labels: squeeze 'u' (d0 row challenges), 'v' (d2 column challenges),
'r' (one per sumcheck round); absorb 'c' (the claim), 'g' (a round message
g(0)||g(2); g(1) is implied by the running claim), 'f' (the final
evaluations a_r||b_r).

Parity status: SHA-256 is ``hashlib`` (pinned by the FIPS 180-4 vectors in the
tests); the byte format above is our own convention: parity unpinned.
"""

import hashlib

from .field import R_MOD, fr_to_bytes

DOMAIN = b"verilora-gb300/zkmat/v1"


def _h(data: bytes) -> bytes:
    return hashlib.sha256(data).digest()


class Transcript:
    def __init__(self, seed: int, m: int, k: int, n: int, trans_p: int, trans_q: int,
                 binds=(bytes(32), bytes(32), bytes(32))):
        if any(len(b) != 32 for b in binds):
            raise ValueError("each bind is 32 bytes")
        msg = (DOMAIN + int(seed).to_bytes(8, "little")
               + int(m).to_bytes(4, "little") + int(k).to_bytes(4, "little")
               + int(n).to_bytes(4, "little")
               + bytes([int(trans_p) & 1, int(trans_q) & 1])
               + bytes(binds[0]) + bytes(binds[1]) + bytes(binds[2]))
        self.state = _h(msg)

    def absorb(self, label: bytes, data: bytes) -> None:
        assert len(label) == 1
        self.state = _h(self.state + label + data)

    def absorb_fr(self, label: bytes, values) -> None:
        self.absorb(label, b"".join(fr_to_bytes(v) for v in values))

    def squeeze(self, label: bytes, count: int):
        assert len(label) == 1
        out = []
        for t in range(count):
            tb = t.to_bytes(4, "little")
            wide = _h(self.state + label + tb + b"\x00") + _h(self.state + label + tb + b"\x01")
            out.append(int.from_bytes(wide, "little") % R_MOD)
        self.state = _h(self.state + label + count.to_bytes(4, "little"))
        return out
