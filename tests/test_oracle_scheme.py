"""Structural pins for the oracle's SPHINCS+ (paper Sec. II-A, Fig. 2).

* Call counts: one hypertree leaf costs len x w = 560 / 816 / 1072 F+PRF calls
  (Sec. III-C-2 of the paper), checked with the oracle's instrumentation.
* Invariants of the definition: verify(sign) accepts; single-bit tampering of
  the signature, the message or PK.root rejects; FORS and XMSS roots rebuilt
  from auth paths equal the full-tree roots; the top layer's root is PK.root
  for every message; chain(chain(x,0,s),s,t) = chain(x,0,s+t); the WOTS key
  recovered from a signature equals the generated one; determinism.
"""
import json
import os
import random

import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PAPER = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
SETS = ("128f", "192f", "256f")


def _seed(P, s):
    rng = random.Random(s)
    return bytes(rng.getrandbits(8) for _ in range(3 * P.n))


@pytest.fixture(scope="module")
def keys(O):
    out = {}
    for i, ps in enumerate(SETS + ("toy",)):
        P = O.params(ps)
        pk, sk = O.keygen(ps, _seed(P, 100 + i))
        out[ps] = (P, pk, sk)
    return out


@pytest.fixture(scope="module")
def signed(O, keys):
    out = {}
    for ps in SETS:
        P, pk, sk = keys[ps]
        m = b"HERO-Sign oracle test message " + ps.encode()
        out[ps] = (m, O.sign(ps, sk, m))
    return out


@pytest.mark.parametrize("ps", SETS)
def test_hash_calls_per_hypertree_leaf(O, keys, ps):
    P, pk, sk = keys[ps]
    O.counters(reset=True)
    O.wots_pkgen(ps, sk, 3, 12345, 5)
    c = O.counters(reset=True)
    f, prf, t = c[2], c[3], c[5]
    assert f + prf == PAPER["sha2_calls_per_hypertree_leaf_sec3c"][ps] == P.len * P.w
    assert prf == P.len and t == 1
    # SHA blocks: every F/PRF is 2 SHA-256 blocks (pad block + 1), T_len is
    # ceil((B + 22 + len n + pad) / B) blocks of SHA-x
    blocks_t = -(-(((128 if P.big else 64) + 22 + P.len * P.n) + (17 if P.big else 9)) // (128 if P.big else 64))
    if P.big:
        assert c[0] == 2 * (f + prf) and c[1] == blocks_t
    else:
        assert c[0] == 2 * (f + prf) + blocks_t


@pytest.mark.parametrize("ps", SETS)
def test_sign_verify_and_tamper(O, keys, signed, ps):
    P, pk, sk = keys[ps]
    m, sig = signed[ps]
    assert len(sig) == P.sig_bytes
    assert O.verify(ps, pk, m, sig)
    rng = random.Random(3)
    fors0 = P.n
    ht0 = P.n + P.fors_bytes
    regions = [
        (0, P.n),                                          # R
        (fors0, fors0 + P.n),                              # first FORS secret
        (fors0 + P.n, fors0 + (P.a + 1) * P.n),            # first FORS auth path
        (P.n + P.fors_bytes - P.n, P.n + P.fors_bytes),    # last FORS auth node
        (ht0, ht0 + P.len * P.n),                          # layer-0 WOTS signature
        (ht0 + P.len * P.n, ht0 + P.layer_bytes),          # layer-0 auth path
        (P.sig_bytes - P.layer_bytes, P.sig_bytes - P.hp * P.n),   # top WOTS
        (P.sig_bytes - P.hp * P.n, P.sig_bytes),           # top auth path
    ]
    for lo, hi in regions:
        for _ in range(3):
            pos = rng.randrange(lo, hi)
            bad = bytearray(sig)
            bad[pos] ^= 1 << rng.randrange(8)
            assert not O.verify(ps, pk, m, bytes(bad)), (lo, hi, pos)
    bad_m = bytearray(m)
    bad_m[0] ^= 0x80
    assert not O.verify(ps, pk, bytes(bad_m), sig)
    bad_pk = bytearray(pk)
    bad_pk[-1] ^= 1
    assert not O.verify(ps, bytes(bad_pk), m, sig)
    assert not O.verify(ps, pk, m + b"x", sig)


@pytest.mark.parametrize("ps", SETS)
def test_determinism(O, keys, signed, ps):
    P, pk, sk = keys[ps]
    m, sig = signed[ps]
    assert O.sign(ps, sk, m) == sig


@pytest.mark.parametrize("ps", SETS)
def test_roots_from_auth_equal_full_tree_roots(O, keys, signed, ps):
    P, pk, sk = keys[ps]
    m, sig = signed[ps]
    R, digest, fidx, it, il = O.hash_message(ps, sk, m)
    assert sig[:P.n] == R
    sig_fors = sig[P.n:P.n + P.fors_bytes]
    # FORS: sk entries are PRF outputs at the selected leaves, roots by definition
    for i in (0, P.k - 1):
        g = (i << P.a) + fidx[i]
        assert sig_fors[i * (P.a + 1) * P.n:][:P.n] == O.fors_sk(ps, sk, it, il, g)
    roots = b"".join(O.fors_node(ps, sk, it, il, i, P.a) for i in range(P.k))
    words_roots = [0, 0, it >> 32, it & 0xFFFFFFFF, 4, il, 0, 0]
    pk_fors = O.thash(ps, O.THASH_T, sk[2 * P.n:3 * P.n], words_roots, roots, l=P.k)
    assert O.fors_pk_from_sig(ps, sk, sig_fors, fidx, it, il) == pk_fors
    # Hypertree: each layer's root from (WOTS sig, auth) equals node(0, h'),
    # and that root is what the next layer signs.
    off = P.n + P.fors_bytes
    msg, tree, leaf = pk_fors, it, il
    layers = list(range(P.d)) if ps != "256f" else [0, 1, 7, P.d - 2, P.d - 1]
    for j in range(P.d):
        layer_sig = sig[off + j * P.layer_bytes: off + (j + 1) * P.layer_bytes]
        r = O.xmss_root_from_sig(ps, sk, layer_sig, msg, j, tree, leaf)
        if j in layers:
            assert r == O.xmss_node(ps, sk, j, tree, 0, P.hp)
            assert layer_sig[:P.len * P.n] == O.wots_sign(ps, sk, msg, j, tree, leaf)
        msg, leaf, tree = r, tree & (2 ** P.hp - 1), tree >> P.hp
    assert tree == 0
    assert msg == pk[P.n:]          # top-layer root is PK.root


def test_top_root_is_pk_root_for_many_messages(O, keys):
    """Climbing every layer of any signature ends at tree 0 of layer d-1 and at
    PK.root (closed form: idx_tree has exactly h - h' bits)."""
    ps = "128f"
    P, pk, sk = keys[ps]
    off = P.n + P.fors_bytes
    for i in range(3):
        m = bytes([i]) * (i * 13)
        sig = O.sign(ps, sk, m)
        R, digest, fidx, it, il = O.hash_message(ps, sk, m)
        msg = O.fors_pk_from_sig(ps, sk, sig[P.n:off], fidx, it, il)
        tree, leaf = it, il
        for j in range(P.d):
            layer_sig = sig[off + j * P.layer_bytes: off + (j + 1) * P.layer_bytes]
            msg = O.xmss_root_from_sig(ps, sk, layer_sig, msg, j, tree, leaf)
            leaf, tree = tree & (2 ** P.hp - 1), tree >> P.hp
        assert tree == 0
        assert msg == pk[P.n:]


def test_chain_composition_and_pk_from_sig(O, keys):
    rng = random.Random(9)
    for ps in SETS:
        P, pk, sk = keys[ps]
        x = bytes(rng.getrandbits(8) for _ in range(P.n))
        for s, t in ((0, 15), (3, 4), (7, 8), (14, 1), (5, 0)):
            a = O.wots_chain(ps, sk, 1, 99, 2, 4, x, 0, s)
            b = O.wots_chain(ps, sk, 1, 99, 2, 4, a, s, t)
            assert b == O.wots_chain(ps, sk, 1, 99, 2, 4, x, 0, s + t)
        msg = bytes(rng.getrandbits(8) for _ in range(P.n))
        wsig = O.wots_sign(ps, sk, msg, 2, 777, 3)
        assert O.wots_pk_from_sig(ps, sk, wsig, msg, 2, 777, 3) == O.wots_pkgen(ps, sk, 2, 777, 3)
        digits = O.wots_digits(ps, msg)
        for i in (0, P.len1 - 1, P.len - 1):
            start = O.wots_sk(ps, sk, 2, 777, 3, i)
            assert wsig[i * P.n:(i + 1) * P.n] == O.wots_chain(ps, sk, 2, 777, 3, i, start, 0, digits[i])
