"""The oracle's pins catch plausible mistakes.

Each case below plants one mistake -- a wrong rotation, a dropped term, a
swapped operand, a wrong index, bit or byte order -- into a copy of
oracle/spx_oracle.c (on the CPU; the real source is untouched), builds it,
and runs the pins of test_oracle_* against it.  Every mutant must fail at
least one pin; a mutant that survives would mean a mistake of that kind in
the oracle could go unnoticed.
"""
import ctypes
import hashlib
import hmac
import json
import os
import random
import subprocess
import tempfile

import pytest

from test_oracle_toy_bruteforce import Toy

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "spx_oracle.c")
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "scheme_layout.json")))
PAPER = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_numbers.json")))

# (name, original text, replacement, replace all occurrences)
MUTANTS = [
    ("sha256 Sigma1 rotation", "ror32(e, 25)", "ror32(e, 26)", False),
    ("sha256 schedule drops W[t-16]", "W[t] = s1 + W[t - 7] + s0 + W[t - 16];\n    }\n    a = H[0]; b = H[1]; c = H[2]; d = H[3]; e = H[4]; f = H[5]; g = H[6]; h = H[7];\n    for (t = 0; t < 64; t++)",
     "W[t] = s1 + W[t - 7] + s0;\n    }\n    a = H[0]; b = H[1]; c = H[2]; d = H[3]; e = H[4]; f = H[5]; g = H[6]; h = H[7];\n    for (t = 0; t < 64; t++)", False),
    ("sha512 sigma0 shift", "(W[t - 15] >> 7)", "(W[t - 15] >> 6)", False),
    ("sha512 short length field", "tl = (rem + 1 + 16 <= 128)", "tl = (rem + 1 + 8 <= 128)", False),
    ("hmac opad", "kpad[i] ^ 0x5c", "kpad[i] ^ 0x36", False),
    ("mgf1 counter byte order", "buf[seedlen] = (uint8_t)(c >> 24);", "buf[seedlen] = (uint8_t)c; buf[seedlen + 3] = (uint8_t)(c >> 24); (void)0;", False),
    ("adrs tree words swapped", "put_be32(out + 1, A->w[2]);\n    put_be32(out + 5, A->w[3]);",
     "put_be32(out + 1, A->w[3]);\n    put_be32(out + 5, A->w[2]);", False),
    ("T_len drops the last chain", "hash_T(c, &A, ends, c->p.len, pk);", "hash_T(c, &A, ends, c->p.len - 1, pk);", False),
    ("blockpad always 64 bytes", "size_t B = big ? 128 : 64;\n    if (c->p.shake) {",
     "size_t B = 64;\n    if (c->p.shake) {", False),
    ("H always SHA-256", "thash_masked(c, c->p.big, A, buf, 2 * (size_t)c->p.n, out);",
     "thash_masked(c, 0, A, buf, 2 * (size_t)c->p.n, out);", False),
    ("PRF uses SHA-512 when big", "g_calls_prf++; thash(c, 0, A,", "g_calls_prf++; thash(c, c->p.big, A,", False),
    ("checksum not shifted", "csum <<= (8 - (p->len2 * 4) % 8) % 8;", "", False),
    ("base_w nibble order", "digits[i] = (i % 2 == 0) ? (x[i / 2] >> 4) : (x[i / 2] & 15);",
     "digits[i] = (i % 2 == 1) ? (x[i / 2] >> 4) : (x[i / 2] & 15);", False),
    ("FORS index bit order", "(md[q / 8] >> (q % 8))", "(md[q / 8] >> (7 - q % 8))", False),
    ("FORS leaf index not global", "uint32_t g = ((uint32_t)i << a) + fidx[i];", "uint32_t g = fidx[i];", True),
    ("XMSS auth sibling", "xmss_node(c, layer, tree, (leaf >> z) ^ 1u, z,", "xmss_node(c, layer, tree, (leaf >> z) | 1u, z,", False),
    ("hypertree leaf taken after shift", "leaf = (uint32_t)(tree & (((uint64_t)1 << c->p.hp) - 1));\n        tree >>= c->p.hp;",
     "tree >>= c->p.hp;\n        leaf = (uint32_t)(tree & (((uint64_t)1 << c->p.hp) - 1));", True),
    ("verify chain starts at 0", "wots_chain(c, &A, sig + (size_t)i * n, digits[i], c->p.w - 1 - digits[i]",
     "wots_chain(c, &A, sig + (size_t)i * n, 0, c->p.w - 1 - digits[i]", False),
    ("FORS roots address type", "ADDR_FORS_ROOTS);\n    hash_T(c, &A, roots, c->p.k, pk_fors);", "ADDR_FORS_TREE);\n    hash_T(c, &A, roots, c->p.k, pk_fors);", True),
    ("keygen uses layer 0", "xmss_node(&c, (uint32_t)(c.p.d - 1), 0, 0, c.p.hp, c.pk_root);", "xmss_node(&c, 0, 0, 0, c.p.hp, c.pk_root);", False),
    ("H_msg drops PK.root", "R, n, c->pk_seed, n, c->pk_root, n, m, mlen);", "R, n, c->pk_seed, n, m, mlen, NULL, 0);", False),
    ("idx_leaf mask one bit wide", "l &= ((uint64_t)1 << p->leaf_bits) - 1;", "l &= ((uint64_t)1 << (p->leaf_bits + 1)) - 1;", False),
    ("tree bytes little-endian", "for (i = 0; i < nbytes; i++) v = (v << 8) | b[i];", "for (i = nbytes - 1; i >= 0; i--) v = (v << 8) | b[i];", False),
    ("XMSS children swapped", "hash_H(c, &A, l, r, out);\n}\n\n/* XMSS signature", "hash_H(c, &A, r, l, out);\n}\n\n/* XMSS signature", False),
    ("chain hash index off by one", "adrs_set_hash(A, (uint32_t)q);", "adrs_set_hash(A, (uint32_t)q + 1);", False),
    ("FORS PRF height 1", "adrs_set_height(&A, 0);\n    adrs_set_index(&A, g);\n    prf_addr(c, &A, out);", "adrs_set_height(&A, 1);\n    adrs_set_index(&A, g);\n    prf_addr(c, &A, out);", False),
    ("WOTS pk keypair dropped", "adrs_set_type(&A, ADDR_WOTS_PK);\n    adrs_set_keypair(&A, kp);", "adrs_set_type(&A, ADDR_WOTS_PK);", False),
    ("FIPS base_2b bytes enter from the right", "acc = (acc << 8) | md[in++];",
     "acc |= (uint64_t)md[in] << (8 * in); in++;", False),
    ("FIPS digit from the low bits", "idx[i] = (uint32_t)((acc >> have) & (((uint64_t)1 << p->a) - 1));",
     "idx[i] = (uint32_t)(acc & (((uint64_t)1 << p->a) - 1)); acc >>= p->a;", False),
    ("FIPS prefix domain byte", "w[0] = 0;", "w[0] = 1;", False),
    ("FIPS context length byte dropped", "w[1] = (uint8_t)ctxlen;", "w[1] = 0;", False),
    ("hmac ipad", "buf[i] = kpad[i] ^ 0x36;", "buf[i] = kpad[i] ^ 0x5c;", False),
    ("mgf1 counter starts at 1", "uint32_t c = 0;\n    uint8_t buf[256], dig[64];",
     "uint32_t c = 1;\n    uint8_t buf[256], dig[64];", False),
    ("WOTS and FORS PRF address types swapped", "ADDR_WOTS_PRF = 5, ADDR_FORS_PRF = 6",
     "ADDR_WOTS_PRF = 6, ADDR_FORS_PRF = 5", False),
    ("FORS roots in reverse order", "fors_node(c, idx_tree, idx_leaf, (uint32_t)i, a, roots + (size_t)i * n);",
     "fors_node(c, idx_tree, idx_leaf, (uint32_t)i, a, roots + (size_t)(c->p.k - 1 - i) * n);", False),
    ("FORS auth path in reverse height order",
     "fors_node(c, idx_tree, idx_leaf, (g >> z) ^ 1u, z, s + (size_t)(z + 1) * n);",
     "fors_node(c, idx_tree, idx_leaf, (g >> z) ^ 1u, z, s + (size_t)(a - z) * n);", False),
    ("checksum sums the digits", "csum += (uint32_t)(p->w - 1 - digits[i]);", "csum += (uint32_t)digits[i];", False),
    ("WOTS secret without the chain index", "adrs_set_keypair(&A, kp);\n    adrs_set_chain(&A, (uint32_t)i);\n    adrs_set_hash(&A, 0);",
     "adrs_set_keypair(&A, kp);\n    adrs_set_chain(&A, 0);\n    adrs_set_hash(&A, 0);", False),
    ("WOTS chain address off by one", "adrs_set_keypair(A, kp);\n    adrs_set_chain(A, (uint32_t)i);",
     "adrs_set_keypair(A, kp);\n    adrs_set_chain(A, (uint32_t)i + 1);", False),
    ("XMSS node height off by one", "adrs_set_height(&A, (uint32_t)z);\n    adrs_set_index(&A, i);\n    hash_H(c, &A, l, r, out);",
     "adrs_set_height(&A, (uint32_t)z - 1);\n    adrs_set_index(&A, i);\n    hash_H(c, &A, l, r, out);", False),
    ("verify FORS climb children swapped", "if ((gz & 1) == 0) hash_H(c, &A, node, au, node);",
     "if ((gz & 1) == 1) hash_H(c, &A, node, au, node);", False),
    ("Keccak rho offset walk", "int nx = y, ny = (2 * x + 3 * y) % 5;", "int nx = y, ny = (3 * x + 2 * y) % 5;", False),
    ("Keccak pi source lane", "int sx = (x + 3 * y) % 5, sy = x;", "int sx = (3 * x + y) % 5, sy = x;", False),
    ("Keccak chi operand order", "B[x + 5 * y] ^ (~B[(x + 1) % 5 + 5 * y] & B[(x + 2) % 5 + 5 * y])",
     "B[x + 5 * y] ^ (B[(x + 1) % 5 + 5 * y] & ~B[(x + 2) % 5 + 5 * y])", False),
    ("Keccak iota bit position", "g_keccak_rc[ir] |= (uint64_t)1 << ((1 << j) - 1);",
     "g_keccak_rc[ir] |= (uint64_t)1 << (1 << j);", False),
    ("SHAKE domain padding", "A[take / 8] ^= (uint64_t)0x1F << (8 * (take % 8));",
     "A[take / 8] ^= (uint64_t)0x06 << (8 * (take % 8));", False),
    ("SHAKE full ADRS word order", "for (i = 0; i < 8; i++) put_be32(out + 4 * i, A->w[i]);",
     "for (i = 0; i < 8; i++) put_be32(out + 4 * i, A->w[7 - i]);", False),
    ("robust mask always SHA-256", "mgf1_shax(big, seed, n + 22, x, inlen);", "mgf1_shax(0, seed, n + 22, x, inlen);", False),
    ("robust mask seed without PK.seed", "mgf1_shax(big, seed, n + 22, x, inlen);", "mgf1_shax(big, seed + n, 22, x, inlen);", False),
    ("robust mask seed one byte short", "mgf1_shax(big, seed, n + 22, x, inlen);", "mgf1_shax(big, seed, n + 21, x, inlen);", False),
    ("robust PRF masked", "g_calls_prf++; thash(c, 0, A,", "g_calls_prf++; thash_masked(c, 0, A,", False),
    ("robust T_l unmasked", "g_calls_t++; thash_masked(c, c->p.big, A,", "g_calls_t++; thash(c, c->p.big, A,", False),
    ("robust F unmasked", "g_calls_f++; thash_masked(c, 0, A,", "g_calls_f++; thash(c, 0, A,", False),
    ("SHAKE PRF_msg operand order", "memcpy(sb, c->sk_prf, n);\n        memcpy(sb + n, opt, n);",
     "memcpy(sb, opt, n);\n        memcpy(sb + n, c->sk_prf, n);", False),
]


def _build(src_text, out):
    with open(out + ".c", "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-w", "-fPIC", "-shared", "-o", out, out + ".c"], check=True)


def _pins_fail(O):
    """Run the pins; return the name of the first one that fails (None if all pass)."""
    rng = random.Random(1)
    try:
        for L in (0, 3, 55, 56, 64, 111, 112, 200):
            m = bytes(rng.getrandbits(8) for _ in range(L))
            if O.sha256(m) != hashlib.sha256(m).digest() or O.sha512(m) != hashlib.sha512(m).digest():
                return "sha2 vs hashlib"
            k = bytes(range(24))
            if O.hmac(0, k, m) != hmac.new(k, m, hashlib.sha256).digest() or \
               O.hmac(1, k, m) != hmac.new(k, m, hashlib.sha512).digest():
                return "hmac vs stdlib"
        seed = bytes(range(40))
        for big, H in ((0, hashlib.sha256), (1, hashlib.sha512)):
            ref = b"".join(H(seed + c.to_bytes(4, "big")).digest() for c in range(3))[:70]
            if O.mgf1(big, seed, 70) != ref:
                return "mgf1"
        for case in GOLD["adrs"]:
            if O.adrs_compress(case["words"]).hex() != case["adrsc_hex"]:
                return "adrs golden"
        for case in GOLD["wots_digits"]:
            d = O.wots_digits(case["params"], bytes.fromhex(case["msg_hex"]))
            if ("digits" in case and d != case["digits"]) or \
               ("checksum_digits" in case and d[-3:] != case["checksum_digits"]):
                return "digits golden"
        for case in GOLD["digest_split"]:
            f, it, il = O.split_digest(case["params"], bytes.fromhex(case["digest_hex"]))
            want_f = case.get("fors", case.get("fors_prefix"))
            if f[:len(want_f)] != want_f or it != case["idx_tree"] or il != case["idx_leaf"]:
                return "digest split golden"
        for ps in ("128f", "192f"):
            P = O.params(ps)
            pk_seed, words = bytes(range(P.n)), [3, 0, 1, 2, 2, 9, 4, 77]
            ad = bytes([3]) + (1).to_bytes(4, "big") + (2).to_bytes(4, "big") + bytes([2]) + \
                b"".join(x.to_bytes(4, "big") for x in (9, 4, 77))
            Hb = hashlib.sha512 if P.n > 16 else hashlib.sha256
            pad = pk_seed + bytes((128 if P.n > 16 else 64) - P.n)
            x2 = bytes(range(2 * P.n))
            if O.thash(ps, O.THASH_H, pk_seed, words, x2) != Hb(pad + ad + x2).digest()[:P.n]:
                return "H composition"
            x1 = bytes(range(P.n))
            if O.thash(ps, O.THASH_F, pk_seed, words, x1) != \
               hashlib.sha256(pk_seed + bytes(64 - P.n) + ad + x1).digest()[:P.n]:
                return "F composition"
            skseed = bytes(range(7, 7 + P.n))
            if O.thash(ps, O.THASH_PRF, pk_seed, words, sk_seed=skseed) != \
               hashlib.sha256(pk_seed + bytes(64 - P.n) + ad + skseed).digest()[:P.n]:
                return "PRF composition"
            sk = bytes(range(4 * P.n))
            R, dg, fidx, it, il = O.hash_message(ps, sk, b"msg")
            if R != hmac.new(sk[P.n:2 * P.n], sk[2 * P.n:3 * P.n] + b"msg", Hb).digest()[:P.n]:
                return "PRF_msg"
            sd = R + sk[2 * P.n:3 * P.n] + Hb(R + sk[2 * P.n:] + b"msg").digest()
            if dg != b"".join(Hb(sd + c.to_bytes(4, "big")).digest() for c in range(2))[:P.m]:
                return "H_msg"
        for ps in ("128f", "192f"):                 # robust instantiation
            P = O.params(ps)
            pk_seed, words = bytes(range(3, 3 + P.n)), [3, 0, 1, 2, 2, 9, 4, 77]
            ad = bytes([3]) + (1).to_bytes(4, "big") + (2).to_bytes(4, "big") + bytes([2]) + \
                b"".join(x.to_bytes(4, "big") for x in (9, 4, 77))
            Hb = hashlib.sha512 if P.n > 16 else hashlib.sha256

            def masked(H, data):
                mk = b"".join(H(pk_seed + ad + c.to_bytes(4, "big")).digest() for c in range(40))
                return bytes(a ^ b for a, b in zip(data, mk))
            pad256, padb = pk_seed + bytes(64 - P.n), pk_seed + bytes((128 if P.n > 16 else 64) - P.n)
            x1, x2, xl = bytes(range(P.n)), bytes(range(2 * P.n)), bytes(i & 0xFF for i in range(P.len * P.n))
            if O.thash("robust-" + ps, O.THASH_F, pk_seed, words, x1) != \
               hashlib.sha256(pad256 + ad + masked(hashlib.sha256, x1)).digest()[:P.n]:
                return "robust F composition"
            if O.thash("robust-" + ps, O.THASH_H, pk_seed, words, x2) != Hb(padb + ad + masked(Hb, x2)).digest()[:P.n]:
                return "robust H composition"
            if O.thash("robust-" + ps, O.THASH_T, pk_seed, words, xl, l=P.len) != \
               Hb(padb + ad + masked(Hb, xl)).digest()[:P.n]:
                return "robust T composition"
            skseed = bytes(range(7, 7 + P.n))
            if O.thash("robust-" + ps, O.THASH_PRF, pk_seed, words, sk_seed=skseed) != \
               hashlib.sha256(pad256 + ad + skseed).digest()[:P.n]:
                return "robust PRF composition"
        rtoy = Toy(bytes(range(48)), robust=True)
        rpk, rsk = O.keygen("robust-toy", bytes(range(48)))
        if rpk != rtoy.pk_seed + rtoy.pk_root() or O.sign("robust-toy", rsk, b"rm") != rtoy.sign(b"rm"):
            return "robust toy"
        P = O.params("128f")
        O.counters(reset=True)
        O.wots_pkgen("128f", bytes(64), 1, 2, 3)
        c = O.counters(reset=True)
        if c[2] + c[3] != PAPER["sha2_calls_per_hypertree_leaf_sec3c"]["128f"]:
            return "calls per leaf"
        toy = Toy(bytes(range(48)))
        pk, skt = O.keygen("toy", bytes(range(48)))
        if pk != toy.pk_seed + toy.pk_root():
            return "toy pk_root"
        R = bytes(16)
        for it, il in ((0, 0), (3, 1), (2, 3)):
            f = [1, 6, 3, 5]
            if O.sign_fields("toy", skt, R, f, it, il) != toy.sign_fields(R, f, it, il):
                return "toy sign_fields"
        for m in (b"", b"hello world"):
            s = O.sign("toy", skt, m)
            if s != toy.sign(m) or not O.verify("toy", pk, m, s):
                return "toy sign/verify"
        from test_oracle_fips205 import base_2b, fields
        for ps in ("slh-toy", "slh-128f"):
            P = O.params(ps)
            for t in range(6):
                dg = bytes(rng.getrandbits(8) for _ in range(P.m))
                if O.split_digest(ps, dg)[0] != base_2b(dg[:P.md_bytes], P.a, P.k):
                    return "FIPS base_2b"
        P = O.params("toy")
        for ctx in (b"", b"c1"):
            mp = b"\x00" + bytes([len(ctx)]) + ctx + b"m"
            if O.slh_sign("toy", skt, ctx, b"m") != toy.sign_fields(*fields(P, skt, mp)):
                return "FIPS pure sign"
        from test_oracle_shake import ToyShake
        for L in (0, 135, 136, 300):
            m = bytes(rng.getrandbits(8) for _ in range(L))
            if O.shake256(m, 200) != hashlib.shake_256(m).digest(200):
                return "shake256 vs hashlib"
        ts = ToyShake(bytes(range(48)))
        pks, sks = O.keygen("shake-toy", bytes(range(48)))
        if pks != ts.pk_seed + ts.pk_root() or O.sign("shake-toy", sks, b"mm") != ts.sign(b"mm"):
            return "shake toy"
        pk1, sk1 = O.keygen("128f", bytes(range(48)))
        s = O.sign("128f", sk1, b"x")
        if not O.verify("128f", pk1, b"x", s):
            return "128f verify"
        bad = bytearray(s)
        bad[5000] ^= 4
        if O.verify("128f", pk1, b"x", bytes(bad)):
            return "128f tamper"
    except Exception as exc:                     # a crash also counts as caught
        return "exception: %r" % (exc,)
    return None


def test_unmutated_source_passes_every_pin(O, tmp_path):
    out = str(tmp_path / "liborig.so")
    _build(open(SRC).read(), out)
    with O.library(out):
        assert _pins_fail(O) is None


@pytest.mark.parametrize("name,old,new,all_", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(O, tmp_path, name, old, new, all_):
    src = open(SRC).read()
    assert old in src, "mutation site not found: " + name
    mutated = src.replace(old, new) if all_ else src.replace(old, new, 1)
    out = str(tmp_path / "libmut.so")
    _build(mutated, out)
    with O.library(out):
        failed = _pins_fail(O)
    assert failed is not None, "planted mistake survived every pin: " + name
