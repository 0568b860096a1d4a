"""Pins of the oracle's FIPS 205 (SLH-DSA) mode against its definition.

FIPS 205 departs from the round-3.1 scheme in two places at these sets: the
FORS indices are the base-2^a digits of md taken most significant bit first
(its base_2b), and pure signing signs M' = 0x00 || len(ctx) || ctx || M.
Everything is recomputed here from Python's hashlib/hmac and a big-integer
reading of md, independent of the oracle's code."""
import hashlib
import hmac
import random

import pytest

from test_oracle_toy_bruteforce import Toy

SETS = ("128f", "192f", "256f", "toy")


def base_2b(md, a, k):
    """Digit i = bits [i a, (i + 1) a) of md as one big-endian integer."""
    v, L = int.from_bytes(md, "big"), 8 * len(md)
    return [(v >> (L - (i + 1) * a)) & ((1 << a) - 1) for i in range(k)]


def fields(P, sk, mprime):
    """R, FORS indices, idx_tree, idx_leaf of M' from the standard library."""
    H = hashlib.sha512 if P.n > 16 else hashlib.sha256
    sk_prf, pk_seed, pk_root = sk[P.n:2 * P.n], sk[2 * P.n:3 * P.n], sk[3 * P.n:]
    R = hmac.new(sk_prf, pk_seed + mprime, H).digest()[:P.n]
    seed = R + pk_seed + H(R + pk_seed + pk_root + mprime).digest()
    dg = b"".join(H(seed + c.to_bytes(4, "big")).digest() for c in range(2))[:P.m]
    f = base_2b(dg[:P.md_bytes], P.a, P.k)
    it = int.from_bytes(dg[P.md_bytes:P.md_bytes + P.tree_bytes], "big") & ((1 << (P.h - P.hp)) - 1)
    il = int.from_bytes(dg[P.md_bytes + P.tree_bytes:P.m], "big") & ((1 << P.hp) - 1)
    return R, f, it, il


@pytest.mark.parametrize("ps", SETS)
def test_fips_index_order_is_msb_first(O, ps):
    P = O.params("slh-" + ps)
    rng = random.Random(205)
    for _ in range(50):
        dg = bytes(rng.getrandbits(8) for _ in range(P.m))
        f, it, il = O.split_digest("slh-" + ps, dg)
        assert f == base_2b(dg[:P.md_bytes], P.a, P.k)
        assert (it, il) == tuple(O.split_digest(ps, dg))[1:]        # the tree / leaf split is unchanged
    # a single set bit lands in the index and bit position the MSB-first reading says
    for q in (0, 1, 7, 8, P.a - 1, P.a, P.k * P.a - 1):
        md = bytearray(P.m)
        md[q // 8] = 0x80 >> (q % 8)
        f = O.split_digest("slh-" + ps, bytes(md))[0]
        want = [0] * P.k
        want[q // P.a] = 1 << (P.a - 1 - q % P.a)
        assert f == want, q


def test_fips_sets_keep_sizes_and_keys(O):
    for ps in SETS:
        a, b = O.params(ps), O.params("slh-" + ps)
        assert (a.n, a.h, a.d, a.a, a.k, a.len, a.m, a.sig_bytes) == (b.n, b.h, b.d, b.a, b.k, b.len, b.m,
                                                                      b.sig_bytes)
        seed = bytes(range(3 * a.n))
        assert O.keygen(ps, seed) == O.keygen("slh-" + ps, seed)


@pytest.mark.parametrize("ctx", [b"", b"\x01", bytes(range(255))])
def test_pure_sign_toy_against_bruteforce(O, ctx):
    seed = bytes(range(48))
    toy = Toy(seed)
    pk, sk = O.keygen("toy", seed)
    P = O.params("toy")
    for m in (b"", b"abc", bytes(range(200))):
        mprime = b"\x00" + bytes([len(ctx)]) + ctx + m
        R, f, it, il = fields(P, sk, mprime)
        sig = O.slh_sign("toy", sk, ctx, m)
        assert sig == toy.sign_fields(R, f, it, il)
        assert O.slh_verify("toy", pk, ctx, m, sig)
        assert O.sign("slh-toy", sk, mprime) == sig                 # the internal function on M'


@pytest.mark.parametrize("ps", ("128f", "192f", "256f"))
def test_pure_sign_composition_and_verify(O, ps):
    rng = random.Random({"128f": 1, "192f": 2, "256f": 3}[ps])
    P = O.params(ps)
    seed = bytes(rng.getrandbits(8) for _ in range(3 * P.n))
    pk, sk = O.keygen(ps, seed)
    ctx, m = b"ctx-string", bytes(rng.getrandbits(8) for _ in range(77))
    R, f, it, il = fields(P, sk, b"\x00" + bytes([len(ctx)]) + ctx + m)
    sig = O.slh_sign(ps, sk, ctx, m)
    assert sig == O.sign_fields(ps, sk, R, f, it, il)
    assert O.slh_verify(ps, pk, ctx, m, sig)
    assert not O.slh_verify(ps, pk, b"ctx-strinG", m, sig)          # another context
    assert not O.slh_verify(ps, pk, ctx, m[:-1], sig)
    assert not O.verify(ps, pk, m, sig)                              # not a round-3.1 signature of m
    bad = bytearray(sig)
    bad[P.n + 3] ^= 1                                                # a FORS secret byte
    assert not O.slh_verify(ps, pk, ctx, m, bytes(bad))


def test_context_length_limit(O):
    pk, sk = O.keygen("toy", bytes(48))
    O.slh_sign("toy", sk, bytes(255), b"m")
    with pytest.raises(ValueError):
        O.slh_sign("toy", sk, bytes(256), b"m")
