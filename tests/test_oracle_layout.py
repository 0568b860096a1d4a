"""Pins for the oracle's parameter derivation, byte layouts and hash compositions.

* Parameters: the paper's Table 1 values and the 17,088-byte 128f signature
  (Sec. I) are read from tests/golden/paper_numbers.json.
* Address layout, base-16 digits with checksum, digest split: hand-derived
  fixtures in tests/golden/scheme_layout.json.
* Tweakable hashes F/H/T_l/PRF and PRF_msg/H_msg: each is rebuilt from hashlib
  and hmac (an independent SHA-2) over the byte string the definition names,
  which pins the block padding of PK.seed, the hash choice per set (SHA-512
  for H/T/H_msg/PRF_msg at n = 24, 32) and the truncation to n bytes.
"""
import hashlib
import hmac
import json
import os
import random

import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden")
PAPER = json.load(open(os.path.join(GOLD, "paper_numbers.json")))
LAYOUT = json.load(open(os.path.join(GOLD, "scheme_layout.json")))
SETS = ("128f", "192f", "256f")


@pytest.mark.parametrize("ps", SETS)
def test_params_match_table1(O, ps):
    P = O.params(ps)
    t = PAPER["table1"][ps]
    assert (P.n, P.h, P.d, P.a, P.k, P.w) == (t["n"], t["h"], t["d"], t["log_t"], t["k"], t["w"])
    assert P.hp * P.d == P.h
    assert P.big == (1 if P.n > 16 else 0)


def test_signature_sizes(O):
    assert O.params("128f").sig_bytes == PAPER["sig_bytes_128f_sec1"]
    # closed form n + k(a+1)n + (h + d len) n with len = 2n + 3 (w = 16)
    for ps, want_len, want_m, want_sig in (("128f", 35, 34, 17088), ("192f", 51, 42, 35664),
                                           ("256f", 67, 49, 49856), ("toy", 35, 4, 1456)):
        P = O.params(ps)
        assert P.len == want_len == 2 * P.n + 3
        assert P.m == want_m
        assert P.sig_bytes == want_sig == P.n + P.k * (P.a + 1) * P.n + (P.h + P.d * P.len) * P.n


def test_structure_counts_from_paper(O):
    for ps in SETS:
        P = O.params(ps)
        assert P.d * 2 ** P.hp == PAPER["hypertree_leaves_per_signature_sec3b"][ps]
        assert P.k * 2 ** P.a == PAPER["fors_leaves_per_signature_sec3b"][ps]


@pytest.mark.parametrize("case", LAYOUT["adrs"])
def test_adrs_compressed_layout(O, case):
    assert O.adrs_compress(case["words"]).hex() == case["adrsc_hex"]


@pytest.mark.parametrize("case", LAYOUT["wots_digits"])
def test_wots_digits_golden(O, case):
    d = O.wots_digits(case["params"], bytes.fromhex(case["msg_hex"]))
    if "digits" in case:
        assert d == case["digits"]
    else:
        assert d[-3:] == case["checksum_digits"]


def test_wots_digits_checksum_property(O):
    rng = random.Random(7)
    for ps in SETS:
        P = O.params(ps)
        for _ in range(50):
            m = bytes(rng.getrandbits(8) for _ in range(P.n))
            d = O.wots_digits(ps, m)
            assert len(d) == P.len and all(0 <= x < 16 for x in d)
            csum = sum(15 - x for x in d[:P.len1])
            assert (d[-3] << 8 | d[-2] << 4 | d[-1]) == csum


@pytest.mark.parametrize("case", LAYOUT["digest_split"])
def test_digest_split_golden(O, case):
    fidx, it, il = O.split_digest(case["params"], bytes.fromhex(case["digest_hex"]))
    if "fors" in case:
        assert fidx == case["fors"]
    else:
        assert fidx[:len(case["fors_prefix"])] == case["fors_prefix"]
    assert it == case["idx_tree"]
    assert il == case["idx_leaf"]


def test_digest_split_ranges(O):
    rng = random.Random(11)
    for ps in SETS + ("toy",):
        P = O.params(ps)
        for _ in range(100):
            dg = bytes(rng.getrandbits(8) for _ in range(P.m))
            fidx, it, il = O.split_digest(ps, dg)
            assert all(0 <= x < 2 ** P.a for x in fidx)
            assert 0 <= it < 2 ** (P.h - P.hp) and 0 <= il < 2 ** P.hp


def _adrsc_bytes(words):
    w = words
    return (bytes([w[0] & 0xFF]) + w[2].to_bytes(4, "big") + w[3].to_bytes(4, "big")
            + bytes([w[4] & 0xFF]) + b"".join(x.to_bytes(4, "big") for x in w[5:8]))


@pytest.mark.parametrize("ps", SETS + ("toy",))
def test_thash_compositions_vs_hashlib(O, ps):
    P = O.params(ps)
    rng = random.Random(13)
    pk_seed = bytes(rng.getrandbits(8) for _ in range(P.n))
    sk_seed = bytes(rng.getrandbits(8) for _ in range(P.n))
    words = [3, 0, 0x01020304, 0x05060708, 2, 9, 4, 77]
    ad = _adrsc_bytes(words)
    s256 = lambda b: hashlib.sha256(b).digest()
    s512 = lambda b: hashlib.sha512(b).digest()
    big = s512 if P.n > 16 else s256
    pad256 = pk_seed + bytes(64 - P.n)
    padbig = pk_seed + bytes((128 if P.n > 16 else 64) - P.n)
    x = bytes(rng.getrandbits(8) for _ in range(P.n))
    assert O.thash(ps, O.THASH_F, pk_seed, words, x) == s256(pad256 + ad + x)[:P.n]
    xy = bytes(rng.getrandbits(8) for _ in range(2 * P.n))
    assert O.thash(ps, O.THASH_H, pk_seed, words, xy) == big(padbig + ad + xy)[:P.n]
    for l in (P.k, P.len):
        v = bytes(rng.getrandbits(8) for _ in range(l * P.n))
        assert O.thash(ps, O.THASH_T, pk_seed, words, v, l=l) == big(padbig + ad + v)[:P.n]
    assert O.thash(ps, O.THASH_PRF, pk_seed, words, sk_seed=sk_seed) == s256(pad256 + ad + sk_seed)[:P.n]


@pytest.mark.parametrize("ps", SETS + ("toy",))
def test_prf_msg_and_h_msg_vs_stdlib(O, ps):
    P = O.params(ps)
    rng = random.Random(17)
    H = hashlib.sha512 if P.n > 16 else hashlib.sha256
    sk = bytes(rng.getrandbits(8) for _ in range(4 * P.n))
    sk_prf, pk_seed, pk_root = sk[P.n:2 * P.n], sk[2 * P.n:3 * P.n], sk[3 * P.n:]
    for L in (0, 1, 32, 200, 1024):
        m = bytes(rng.getrandbits(8) for _ in range(L))
        R, digest, fidx, it, il = O.hash_message(ps, sk, m)
        assert R == hmac.new(sk_prf, pk_seed + m, H).digest()[:P.n]
        seed = R + pk_seed + H(R + pk_seed + pk_root + m).digest()
        mgf = b"".join(H(seed + c.to_bytes(4, "big")).digest() for c in range(2))
        assert digest == mgf[:P.m]
        assert (fidx, it, il) == tuple(O.split_digest(ps, digest))
