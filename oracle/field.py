"""BLS12-381 scalar field F_r in plain Python integers (oracle; test infrastructure).

Sec. V (Security Analysis) fixes the field: the scalar field of the BLS12-381
curve, |F| about 2^254.  Its order is r = z^4 - z^2 + 1 with the curve
parameter z = -0xd201000000010000 (255 bits, 2-adicity 32).

Fixed-point values enter the field as x mod r (Sec. II-C pads and embeds
integer tensors; negative x maps to r - |x|).

Elements are serialised as 32 bytes, little-endian, canonical (< r).

Pins (tests/test_oracle_field.py): the closed form of r, Miller-Rabin,
2-adicity, inverses, and the NIST-style round trips of the byte encoding.
"""

R_MOD = 0x73EDA753299D7D483339D80809A1D80553BDA402FFFE5BFEFFFFFFFF00000001


def fr(x: int) -> int:
    """Embed an integer (fixed-point value, possibly negative) into F_r."""
    return int(x) % R_MOD


def fr_add(a: int, b: int) -> int:
    return (a + b) % R_MOD


def fr_sub(a: int, b: int) -> int:
    return (a - b) % R_MOD


def fr_mul(a: int, b: int) -> int:
    return (a * b) % R_MOD


def fr_inv(a: int) -> int:
    if a % R_MOD == 0:
        raise ZeroDivisionError("0 has no inverse in F_r")
    return pow(a, R_MOD - 2, R_MOD)


def fr_to_bytes(a: int) -> bytes:
    """Canonical 32-byte little-endian encoding."""
    a %= R_MOD
    return a.to_bytes(32, "little")


def fr_from_bytes(b: bytes) -> int:
    """Inverse of fr_to_bytes; rejects non-canonical encodings."""
    if len(b) != 32:
        raise ValueError("an F_r element is 32 bytes")
    x = int.from_bytes(b, "little")
    if x >= R_MOD:
        raise ValueError("non-canonical F_r encoding")
    return x
