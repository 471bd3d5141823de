"""Fixed-point to field encoding (oracle; test infrastructure).

Sec. II-C embeds integer (fixed-point) tensors into the field: x -> x mod r,
negative x -> r - |x|.  The device keeps field elements in Montgomery form,
x.2^256 mod r; this module states that map by its definition.

Pins (tests/test_oracle_encode.py): encode(1) = 2^256 mod r, additivity
mod r, and the sign rule.
"""

from .field import R_MOD

MONT_R = (1 << 256) % R_MOD


def encode_montgomery(x: int) -> int:
    """(x mod r) . 2^256 mod r."""
    return (int(x) % R_MOD) * (1 << 256) % R_MOD


def limbs_le32(v: int):
    """Eight 32-bit little-endian limbs of a field element."""
    return [(v >> (32 * i)) & 0xFFFFFFFF for i in range(8)]
