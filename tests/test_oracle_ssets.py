"""Pins of the oracle at the small-signature sets (128s / 192s / 256s, a
variant beside the paper's f sets): parameters and sizes against the
standard's table, the digest split with a two-byte leaf index, and the
sign / verify / tamper invariants on one signature per set."""
import hashlib
import json
import os
import random

import pytest

from test_oracle_fips205 import base_2b, fields

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sset_params.json")))["sets"]
SETS = ("128s", "192s", "256s")


@pytest.mark.parametrize("ps", SETS)
def test_parameters_and_sizes(O, ps):
    P, g = O.params(ps), GOLD[ps]
    assert (P.n, P.h, P.d, P.hp, P.a, P.k, P.m, P.sig_bytes) == (g["n"], g["h"], g["d"], g["hp"], g["a"], g["k"],
                                                                 g["m"], g["sig_bytes"])
    # closed forms: len = 2n + 3 at w = 16; SIG = n + k (a + 1) n + (h + d len) n
    assert P.len == 2 * P.n + 3
    assert P.sig_bytes == P.n + P.k * (P.a + 1) * P.n + (P.h + P.d * P.len) * P.n
    assert P.m == (P.k * P.a + 7) // 8 + (P.h - P.hp + 7) // 8 + (P.hp + 7) // 8
    pk, sk = O.keygen(ps, bytes(3 * P.n))
    assert len(pk) == g["pk_bytes"] and len(sk) == 2 * g["pk_bytes"]


@pytest.mark.parametrize("ps", SETS)
def test_digest_split(O, ps):
    P = O.params(ps)
    rng = random.Random(9)
    for _ in range(40):
        dg = bytes(rng.getrandbits(8) for _ in range(P.m))
        f, it, il = O.split_digest(ps, dg)
        md = dg[:P.md_bytes]
        bits = int.from_bytes(md, "little")          # stream bit q = bit q % 8 of byte q // 8
        assert f == [(bits >> (i * P.a)) & ((1 << P.a) - 1) for i in range(P.k)]
        assert it == int.from_bytes(dg[P.md_bytes:P.md_bytes + P.tree_bytes], "big") & ((1 << (P.h - P.hp)) - 1)
        assert il == int.from_bytes(dg[P.md_bytes + P.tree_bytes:], "big") & ((1 << P.hp) - 1)
        assert O.split_digest("slh-" + ps, dg)[0] == base_2b(md, P.a, P.k)


@pytest.mark.parametrize("ps", SETS)
def test_sign_verify_tamper(O, ps):
    P = O.params(ps)
    rng = random.Random(P.n)
    pk, sk = O.keygen(ps, bytes(rng.getrandbits(8) for _ in range(3 * P.n)))
    m = bytes(rng.getrandbits(8) for _ in range(50))
    sig = O.sign(ps, sk, m)
    assert len(sig) == P.sig_bytes and O.verify(ps, pk, m, sig)
    fors_end = P.n + P.fors_bytes
    spots = (0, P.n + 1, P.n + P.n * P.a, fors_end + 5, fors_end + P.len * P.n + 3,
             fors_end + (P.d - 1) * P.layer_bytes + P.len * P.n + P.n * P.hp - 1)
    for pos in spots:
        bad = bytearray(sig)
        bad[pos] ^= 0x10
        assert not O.verify(ps, pk, m, bytes(bad)), pos
    assert not O.verify(ps, pk, m + b"x", sig)
    if ps == "128s":          # the FIPS 205 mode through the same pipeline
        ctx = b"s-set"
        R, f, it, il = fields(P, sk, b"\x00" + bytes([len(ctx)]) + ctx + m)
        assert O.slh_sign(ps, sk, ctx, m) == O.sign_fields(ps, sk, R, f, it, il)
