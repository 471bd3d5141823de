"""Pins for oracle/field.py: the field order and the arithmetic helpers."""
import random

import pytest

from oracle.field import R_MOD, fr, fr_add, fr_sub, fr_mul, fr_inv, fr_to_bytes, fr_from_bytes


def _miller_rabin(n, bases):
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in bases:
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = pow(x, 2, n)
            if x == n - 1:
                break
        else:
            return False
    return True


def test_order_closed_form():
    # BLS12 family: r = z^4 - z^2 + 1 with z = -0xd201000000010000 (BLS12-381).
    z = -0xD201000000010000
    assert R_MOD == z ** 4 - z ** 2 + 1
    assert R_MOD.bit_length() == 255


def test_order_prime_and_two_adicity():
    rng = random.Random(7)
    assert _miller_rabin(R_MOD, [2, 3, 5, 7, 11, 13] + [rng.randrange(2, R_MOD - 1) for _ in range(24)])
    assert (R_MOD - 1) % (1 << 32) == 0 and ((R_MOD - 1) >> 32) % 2 == 1
    # Miller-Rabin must reject a composite of the same size.
    assert not _miller_rabin(R_MOD + 2 * 3, [2, 3, 5, 7])


def test_embedding_of_fixed_point():
    assert fr(-1) == R_MOD - 1
    assert fr(-(1 << 15)) == R_MOD - (1 << 15)
    assert fr((1 << 15) - 1) == (1 << 15) - 1
    assert fr_add(fr(-5), fr(5)) == 0
    assert fr_sub(0, 1) == R_MOD - 1


def test_inverse_and_mul():
    rng = random.Random(11)
    for _ in range(50):
        a = rng.randrange(1, R_MOD)
        assert fr_mul(a, fr_inv(a)) == 1
    with pytest.raises(ZeroDivisionError):
        fr_inv(0)
    # Fermat: a^(r-1) = 1; the inverse of 2 is (r + 1) / 2.
    assert fr_inv(2) == (R_MOD + 1) // 2


def test_bytes_roundtrip():
    rng = random.Random(3)
    for a in [0, 1, R_MOD - 1] + [rng.randrange(R_MOD) for _ in range(20)]:
        b = fr_to_bytes(a)
        assert len(b) == 32 and fr_from_bytes(b) == a
    assert fr_to_bytes(1) == b"\x01" + bytes(31)
    with pytest.raises(ValueError):
        fr_from_bytes(R_MOD.to_bytes(32, "little"))
