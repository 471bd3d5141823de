"""Pins for oracle/transcript.py.

SHA-256 is pinned by FIPS 180-4 example vectors.  The transcript byte format
is this project's own convention (parity unpinned): the tests check its
determinism, domain separation and output range only.
"""
import hashlib

from oracle.field import R_MOD
from oracle.transcript import Transcript, DOMAIN


def test_sha256_fips_vectors():
    assert hashlib.sha256(b"abc").hexdigest() == \
        "ba7816bf8f01cfea414140de5dae2223b00361a396177a9cb410ff61f20015ad"
    assert hashlib.sha256(b"").hexdigest() == \
        "e3b0c44298fc1c149afbf4c8996fb92427ae41e4649b934ca495991b7852b855"
    assert hashlib.sha256(b"abcdbcdecdefdefgefghfghighijhijkijkljklmklmnlmnomnopnopq").hexdigest() == \
        "248d6a61d20638b8e5c026930c3e6039a33ce45964ff2167f6ecedd419db06c1"


def test_start_state_layout():
    t = Transcript(5, 64, 128, 32, 1, 0)
    msg = (DOMAIN + (5).to_bytes(8, "little") + (64).to_bytes(4, "little")
           + (128).to_bytes(4, "little") + (32).to_bytes(4, "little") + b"\x01\x00" + bytes(96))
    assert t.state == hashlib.sha256(msg).digest()


def test_squeeze_counter_mode_and_update():
    t = Transcript(1, 2, 2, 2, 0, 0)
    s = t.state
    xs = t.squeeze(b"u", 3)
    for i, x in enumerate(xs):
        tb = i.to_bytes(4, "little")
        wide = hashlib.sha256(s + b"u" + tb + b"\x00").digest() + hashlib.sha256(s + b"u" + tb + b"\x01").digest()
        assert x == int.from_bytes(wide, "little") % R_MOD
    assert t.state == hashlib.sha256(s + b"u" + (3).to_bytes(4, "little")).digest()
    assert len(set(xs)) == 3 and all(0 <= x < R_MOD for x in xs)


def test_domain_separation():
    a = Transcript(1, 2, 2, 2, 0, 0)
    b = Transcript(1, 2, 2, 2, 0, 1)
    c = Transcript(2, 2, 2, 2, 0, 0)
    assert len({a.state, b.state, c.state}) == 3
    x = Transcript(1, 2, 2, 2, 0, 0)
    y = Transcript(1, 2, 2, 2, 0, 0)
    assert x.squeeze(b"u", 1) != y.squeeze(b"v", 1)
