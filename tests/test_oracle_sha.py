"""Pins for the oracle's SHA-2, HMAC and MGF1 (FIPS 180-4, RFC 2104, RFC 8017).

The reference values come from Python's hashlib/hmac (OpenSSL), an
implementation independent of the oracle's C code; the round constants are
re-derived from their definition (fractional parts of cube / square roots of
the first primes) with exact integer arithmetic.
"""
import hashlib
import hmac
import os
import random
from math import isqrt

import pytest

LENGTHS = sorted(set(list(range(0, 300, 7)) + [55, 56, 63, 64, 65, 111, 112, 119, 120,
                                                 127, 128, 129, 191, 192, 255, 256, 65536]))


def test_sha256_sha512_match_hashlib(O):
    rng = random.Random(1)
    for L in LENGTHS:
        m = bytes(rng.getrandbits(8) for _ in range(L)) if L < 1000 else os.urandom(L)
        assert O.sha256(m) == hashlib.sha256(m).digest(), L
        assert O.sha512(m) == hashlib.sha512(m).digest(), L


def test_fips_abc_examples(O):
    # FIPS 180-4 appendix one-block and two-block examples, values from hashlib
    for m in (b"abc", b"abcdbcdecdefdefgefghfghighijhijkijkljklmklmnlmnomnopnopq"):
        assert O.sha256(m) == hashlib.sha256(m).digest()
        assert O.sha512(m) == hashlib.sha512(m).digest()


@pytest.mark.parametrize("big", [0, 1])
def test_hmac_matches_stdlib(O, big):
    rng = random.Random(2 + big)
    for keylen in (16, 24, 32):
        for L in (0, 1, 31, 32, 33, 64, 100, 128, 129, 1000, 4096):
            k = bytes(rng.getrandbits(8) for _ in range(keylen))
            m = bytes(rng.getrandbits(8) for _ in range(L))
            ref = hmac.new(k, m, hashlib.sha512 if big else hashlib.sha256).digest()
            assert O.hmac(big, k, m) == ref


@pytest.mark.parametrize("big", [0, 1])
def test_mgf1_matches_hashlib_composition(O, big):
    H = hashlib.sha512 if big else hashlib.sha256
    rng = random.Random(5)
    for seedlen in (0, 48, 96, 160):
        seed = bytes(rng.getrandbits(8) for _ in range(seedlen))
        for outlen in (1, 34, 42, 49, 64, 65, 130):
            ref = b"".join(H(seed + c.to_bytes(4, "big")).digest() for c in range(8))[:outlen]
            assert O.mgf1(big, seed, outlen) == ref


def _primes(n):
    ps, c = [], 2
    while len(ps) < n:
        if all(c % p for p in ps):
            ps.append(c)
        c += 1
    return ps


def _icbrt(x):
    lo, hi = 0, 1 << ((x.bit_length() + 2) // 3 + 1)
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if mid ** 3 <= x:
            lo = mid
        else:
            hi = mid - 1
    return lo


def sha_constants_from_definition():
    """K = first 32/64 fractional bits of cube roots of the first 64/80 primes;
    IV = same of the square roots of the first 8 primes (FIPS 180-4 4.2, 5.3)."""
    P = _primes(80)
    k256 = [_icbrt(p << 96) & 0xFFFFFFFF for p in P[:64]]
    iv256 = [isqrt(p << 64) & 0xFFFFFFFF for p in P[:8]]
    k512 = [_icbrt(p << 192) & (2 ** 64 - 1) for p in P]
    iv512 = [isqrt(p << 128) & (2 ** 64 - 1) for p in P[:8]]
    return k256, iv256, k512, iv512


def test_oracle_sha_tables_from_definition(O):
    assert tuple(O.sha_tables()) == tuple(sha_constants_from_definition())
