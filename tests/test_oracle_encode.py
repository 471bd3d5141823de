"""Pins for oracle/encode.py (fixed-point embedding, Sec. II-C)."""
import random

from oracle.encode import encode_montgomery, limbs_le32, MONT_R
from oracle.field import R_MOD


def test_one_and_zero():
    assert encode_montgomery(0) == 0
    assert encode_montgomery(1) == pow(2, 256, R_MOD) == MONT_R


def test_sign_rule_and_additivity():
    rng = random.Random(5)
    for _ in range(100):
        a = rng.randrange(-(1 << 15), 1 << 15)
        b = rng.randrange(-(1 << 15), 1 << 15)
        assert (encode_montgomery(a) + encode_montgomery(b)) % R_MOD == encode_montgomery(a + b)
        assert (encode_montgomery(a) + encode_montgomery(-a)) % R_MOD == 0
    assert encode_montgomery(-1) == R_MOD - MONT_R


def test_limbs():
    v = (5 << 224) | 7
    assert limbs_le32(v) == [7, 0, 0, 0, 0, 0, 0, 5]
