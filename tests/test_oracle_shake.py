"""Pins of the oracle's SHAKE instantiation (a variant beside the paper's
SHA2 sets): its SHAKE256 against hashlib across the 136-byte rate boundary
(so Keccak-f[1600], its round constants and rotation offsets are pinned),
every tweakable hash, PRF_msg and H_msg against hashlib compositions with
an independently built 32-byte ADRS, the whole toy hypertree against a
SHAKE version of the independent Python construction, and sign / verify /
tamper at the f sets."""
import hashlib
import random

import pytest

from test_oracle_toy_bruteforce import A, HP, K, N, Toy


def adrs32(words):
    return b"".join(w.to_bytes(4, "big") for w in words)


class ToyShake(Toy):
    """The toy construction with SHAKE256 and the full 32-byte address."""

    @staticmethod
    def adrs(layer, tree, typ, kp=0, w6=0, w7=0):
        return adrs32([layer, 0, tree >> 32, tree & 0xFFFFFFFF, typ, kp, w6, w7])

    def th(self, ad, data, prf=False):
        return hashlib.shake_256(self.pk_seed + ad + data).digest(N)

    def sign(self, m):
        R = hashlib.shake_256(self.sk_prf + self.pk_seed + m).digest(N)
        digest = hashlib.shake_256(R + self.pk_seed + self.pk_root() + m).digest(4)
        q = [(digest[b // 8] >> (b % 8)) & 1 for b in range(16)]
        fidx = [sum(q[i * A + j] << j for j in range(A)) for i in range(K)]
        return self.sign_fields(R, fidx, digest[2] & 3, digest[3] & 3)


def test_shake256_vs_hashlib(O):
    rng = random.Random(202)
    for L in (0, 1, 31, 135, 136, 137, 271, 272, 273, 1000):
        m = bytes(rng.getrandbits(8) for _ in range(L))
        for outlen in (1, 16, 24, 32, 47, 135, 136, 137, 300):
            assert O.shake256(m, outlen) == hashlib.shake_256(m).digest(outlen), (L, outlen)


def test_keccak_permutation_is_the_one_shake_uses(O):
    # SHAKE256 of the empty message is the first permutation of the padded
    # all-zero state: byte 0 = 0x1F, byte 135 = 0x80.
    lanes = [0] * 25
    lanes[0] = 0x1F
    lanes[16] = 0x80 << 56
    out = O.keccak_f1600(lanes)
    got = b"".join(x.to_bytes(8, "little") for x in out[:17])
    assert got == hashlib.shake_256(b"").digest(136)


@pytest.mark.parametrize("ps", ("128f", "192f", "256f"))
def test_thash_compositions(O, ps):
    P = O.params("shake-" + ps)
    rng = random.Random(P.n)
    pk_seed = bytes(rng.getrandbits(8) for _ in range(P.n))
    sk_seed = bytes(rng.getrandbits(8) for _ in range(P.n))
    words = [5, 0, 0x01020304, 0x05060708, 2, 0x0a0b0c0d, 3, 0x77]
    ad = adrs32(words)
    sh = lambda data: hashlib.shake_256(pk_seed + ad + data).digest(P.n)
    x1 = bytes(rng.getrandbits(8) for _ in range(P.n))
    x2 = bytes(rng.getrandbits(8) for _ in range(2 * P.n))
    xl = bytes(rng.getrandbits(8) for _ in range(P.len * P.n))
    assert O.thash("shake-" + ps, O.THASH_F, pk_seed, words, x1) == sh(x1)
    assert O.thash("shake-" + ps, O.THASH_H, pk_seed, words, x2) == sh(x2)
    assert O.thash("shake-" + ps, O.THASH_T, pk_seed, words, xl, l=P.len) == sh(xl)
    assert O.thash("shake-" + ps, O.THASH_PRF, pk_seed, words, sk_seed=sk_seed) == sh(sk_seed)


@pytest.mark.parametrize("ps", ("128f", "192f", "256f", "128s"))
def test_prf_msg_and_h_msg(O, ps):
    P = O.params("shake-" + ps)
    rng = random.Random(3)
    sk = bytes(rng.getrandbits(8) for _ in range(4 * P.n))
    sk_prf, pk_seed, pk_root = sk[P.n:2 * P.n], sk[2 * P.n:3 * P.n], sk[3 * P.n:]
    for L in (0, 5, 200):
        m = bytes(rng.getrandbits(8) for _ in range(L))
        R, digest, fidx, it, il = O.hash_message("shake-" + ps, sk, m)
        assert R == hashlib.shake_256(sk_prf + pk_seed + m).digest(P.n)
        assert digest == hashlib.shake_256(R + pk_seed + pk_root + m).digest(P.m)
        assert (fidx, it, il) == tuple(O.split_digest(ps, digest))


def test_toy_hypertree_against_independent_construction(O):
    rng = random.Random(55)
    seed = bytes(rng.getrandbits(8) for _ in range(3 * N))
    toy = ToyShake(seed)
    pk, sk = O.keygen("shake-toy", seed)
    assert pk == toy.pk_seed + toy.pk_root()
    for layer, trees in ((0, range(4)), (1, [0])):
        for t in trees:
            lv = toy.xmss_levels(layer, t)
            for z in range(HP + 1):
                for i in range(2 ** (HP - z)):
                    assert O.xmss_node("shake-toy", sk, layer, t, i, z) == lv[z][i]
    R = bytes(rng.getrandbits(8) for _ in range(N))
    for idx_tree, idx_leaf in ((0, 0), (3, 1), (2, 3)):
        f = [rng.randrange(2 ** A) for _ in range(K)]
        assert O.sign_fields("shake-toy", sk, R, f, idx_tree, idx_leaf) == toy.sign_fields(R, f, idx_tree, idx_leaf)
    for m in (b"", b"shake", bytes(range(150))):
        sig = O.sign("shake-toy", sk, m)
        assert sig == toy.sign(m)
        assert O.verify("shake-toy", pk, m, sig)


@pytest.mark.parametrize("ps", ("128f", "192f", "256f"))
def test_sign_verify_tamper(O, ps):
    P = O.params("shake-" + ps)
    rng = random.Random(P.n + 1)
    seed = bytes(rng.getrandbits(8) for _ in range(3 * P.n))
    pk, sk = O.keygen("shake-" + ps, seed)
    assert pk[:P.n] == seed[2 * P.n:] and pk[P.n:] != O.keygen(ps, seed)[0][P.n:]   # another PK.root
    m = b"shake message"
    sig = O.sign("shake-" + ps, sk, m)
    assert O.verify("shake-" + ps, pk, m, sig)
    assert not O.verify(ps, pk, m, sig)                     # not a SHA2 signature
    for pos in (1, P.n + 2, P.n + P.fors_bytes + 3, P.sig_bytes - 1):
        bad = bytearray(sig)
        bad[pos] ^= 0x40
        assert not O.verify("shake-" + ps, pk, m, bytes(bad)), pos
