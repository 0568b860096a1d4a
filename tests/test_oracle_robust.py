"""Pins for the oracle's robust SHA2 instantiation (SPHINCS+ round 3.1; a
variant beside the paper's simple one).

Robust F, H and T_l hash M xor MGF1-SHA-x(PK.seed || ADRSc, |M|) instead of
M, with SHA-x the tweakable hash's own hash (SHA-256 for F; SHA-512 for H and
T_l at n = 24 / 32) and PK.seed unpadded in the mask seed; PRF, PRF_msg and
H_msg are unchanged.  Each composition is rebuilt here from hashlib with an
address builder and an MGF1 of this file's own; the full scheme is pinned by
verify / tamper / determinism at the three f sets, and by the independent
toy-parameter construction in test_oracle_toy_bruteforce.py.
"""
import hashlib
import random

import pytest

SETS = ("128f", "192f", "256f")


def _adrsc(w):
    """Compressed address: layer byte, 8 tree bytes, type byte, 3 words."""
    return (bytes([w[0] & 0xFF]) + w[2].to_bytes(4, "big") + w[3].to_bytes(4, "big")
            + bytes([w[4] & 0xFF]) + b"".join(x.to_bytes(4, "big") for x in w[5:8]))


def _mask(H, seed, n):
    out = b""
    c = 0
    while len(out) < n:
        out += H(seed + c.to_bytes(4, "big")).digest()
        c += 1
    return out[:n]


def _xor(a, b):
    return bytes(x ^ y for x, y in zip(a, b))


@pytest.mark.parametrize("ps", SETS + ("toy",))
def test_robust_thash_compositions_vs_hashlib(O, ps):
    P = O.params(ps)
    rps = "robust-" + ps
    rng = random.Random(29)
    pk_seed = bytes(rng.getrandbits(8) for _ in range(P.n))
    sk_seed = bytes(rng.getrandbits(8) for _ in range(P.n))
    words = [5, 0, 0x0A0B0C0D, 0x11223344, 3, 7, 2, 201]
    ad = _adrsc(words)
    s256, s512 = hashlib.sha256, hashlib.sha512
    big = s512 if P.n > 16 else s256
    pad256 = pk_seed + bytes(64 - P.n)
    padbig = pk_seed + bytes((128 if P.n > 16 else 64) - P.n)
    x = bytes(rng.getrandbits(8) for _ in range(P.n))
    want_f = s256(pad256 + ad + _xor(x, _mask(s256, pk_seed + ad, P.n))).digest()[:P.n]
    assert O.thash(rps, O.THASH_F, pk_seed, words, x) == want_f
    xy = bytes(rng.getrandbits(8) for _ in range(2 * P.n))
    want_h = big(padbig + ad + _xor(xy, _mask(big, pk_seed + ad, 2 * P.n))).digest()[:P.n]
    assert O.thash(rps, O.THASH_H, pk_seed, words, xy) == want_h
    for l in (P.k, P.len):               # masks of several MGF1 blocks
        v = bytes(rng.getrandbits(8) for _ in range(l * P.n))
        want_t = big(padbig + ad + _xor(v, _mask(big, pk_seed + ad, l * P.n))).digest()[:P.n]
        assert O.thash(rps, O.THASH_T, pk_seed, words, v, l=l) == want_t
    # PRF is not masked: the same value as the simple instantiation's
    prf = O.thash(rps, O.THASH_PRF, pk_seed, words, sk_seed=sk_seed)
    assert prf == s256(pad256 + ad + sk_seed).digest()[:P.n]
    assert prf == O.thash(ps, O.THASH_PRF, pk_seed, words, sk_seed=sk_seed)
    # and the masked hashes differ from the simple ones
    assert want_f != O.thash(ps, O.THASH_F, pk_seed, words, x)


@pytest.mark.parametrize("ps", SETS)
def test_robust_sign_verify_tamper(O, ps):
    P = O.params(ps)
    rps = "robust-" + ps
    rng = random.Random(31)
    seed = bytes(rng.getrandbits(8) for _ in range(3 * P.n))
    pk, sk = O.keygen(rps, seed)
    pk_s, sk_s = O.keygen(ps, seed)
    assert pk[:P.n] == pk_s[:P.n] and pk != pk_s          # same PK.seed, another PK.root
    assert sk[:2 * P.n] == sk_s[:2 * P.n]
    m = b"robust " + ps.encode()
    sig = O.sign(rps, sk, m)
    assert len(sig) == P.sig_bytes and O.sign(rps, sk, m) == sig
    assert O.verify(rps, pk, m, sig)
    assert not O.verify(ps, pk, m, sig)                   # the simple verifier rejects it
    sig_s = O.sign(ps, sk_s, m)
    assert sig_s[:P.n] == sig[:P.n]                       # R: PRF_msg is unchanged
    for pos in (P.n + 3, P.n + P.fors_bytes // 2, P.n + P.fors_bytes + 5, len(sig) - 7):
        bad = bytearray(sig)
        bad[pos] ^= 0x10
        assert not O.verify(rps, pk, m, bytes(bad)), pos
    assert not O.verify(rps, pk, m + b"!", sig)
