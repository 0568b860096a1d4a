"""Brute-force pin of the oracle at toy parameters (n=16, h=4, d=2, h'=2,
a=3, k=4, w=16; SHA-256 throughout), in the simple and the robust
instantiation.

A second, independent construction written here in Python straight from the
definition (hashlib for SHA-256, its own address builder, explicit iterative
full-tree construction level by level, no recursion) builds every WOTS key,
every node of every XMSS tree of both layers and every FORS tree, then signs
for ALL 2^h (idx_tree, idx_leaf) pairs.  The oracle's recursive node(), auth
paths, FORS signature and full signatures must agree byte for byte, and the
oracle's verify must accept each signature.
"""
import hashlib
import hmac
import random

import pytest

N, H, D, HP, A, K, W = 16, 4, 2, 2, 3, 4, 16
LEN1, LEN2 = 2 * N, 3
LEN = LEN1 + LEN2
WOTS_HASH, WOTS_PK, TREE, FORS_TREE, FORS_ROOTS, WOTS_PRF, FORS_PRF = range(7)


class Toy:
    def __init__(self, seed, robust=False):
        self.sk_seed, self.sk_prf, self.pk_seed = seed[:N], seed[N:2 * N], seed[2 * N:3 * N]
        self.robust = robust
        self._leaves = {}

    @staticmethod
    def adrs(layer, tree, typ, kp=0, w6=0, w7=0):
        return (bytes([layer]) + tree.to_bytes(8, "big") + bytes([typ])
                + kp.to_bytes(4, "big") + w6.to_bytes(4, "big") + w7.to_bytes(4, "big"))

    def th(self, ad, data, prf=False):
        """Tweakable hash.  Robust instantiation: F, H and T_l (not PRF) hash
        data xor MGF1-SHA-256(PK.seed || ADRSc, |data|)."""
        if self.robust and not prf:
            mask = b"".join(hashlib.sha256(self.pk_seed + ad + c.to_bytes(4, "big")).digest()
                            for c in range(-(-len(data) // 32)))
            data = bytes(x ^ y for x, y in zip(data, mask))
        return hashlib.sha256(self.pk_seed + bytes(64 - N) + ad + data).digest()[:N]

    def chain_values(self, layer, tree, kp, i):
        """All 16 positions of chain i."""
        x = self.th(self.adrs(layer, tree, WOTS_PRF, kp, i, 0), self.sk_seed, prf=True)
        vals = [x]
        for q in range(W - 1):
            x = self.th(self.adrs(layer, tree, WOTS_HASH, kp, i, q), x)
            vals.append(x)
        return vals

    def wots_leaf(self, layer, tree, kp):
        key = (layer, tree, kp)
        if key not in self._leaves:
            ends = b"".join(self.chain_values(layer, tree, kp, i)[-1] for i in range(LEN))
            self._leaves[key] = self.th(self.adrs(layer, tree, WOTS_PK, kp), ends)
        return self._leaves[key]

    def xmss_levels(self, layer, tree):
        lv = [[self.wots_leaf(layer, tree, kp) for kp in range(2 ** HP)]]
        for z in range(1, HP + 1):
            prev = lv[-1]
            lv.append([self.th(self.adrs(layer, tree, TREE, 0, z, i), prev[2 * i] + prev[2 * i + 1])
                       for i in range(len(prev) // 2)])
        return lv

    def fors_levels(self, tree, kp):
        """levels[z][g] for all k trees side by side (global index g)."""
        leaves = []
        for g in range(K * 2 ** A):
            s = self.th(self.adrs(0, tree, FORS_PRF, kp, 0, g), self.sk_seed, prf=True)
            leaves.append(self.th(self.adrs(0, tree, FORS_TREE, kp, 0, g), s))
        lv = [leaves]
        for z in range(1, A + 1):
            prev = lv[-1]
            lv.append([self.th(self.adrs(0, tree, FORS_TREE, kp, z, g), prev[2 * g] + prev[2 * g + 1])
                       for g in range(len(prev) // 2)])
        return lv

    @staticmethod
    def digits(msg):
        d = []
        for b in msg:
            d += [b >> 4, b & 15]
        c = sum(15 - x for x in d) << 4
        return d + [(c >> 12) & 15, (c >> 8) & 15, (c >> 4) & 15]

    def pk_root(self):
        return self.xmss_levels(D - 1, 0)[HP][0]

    def sign_fields(self, R, fidx, idx_tree, idx_leaf):
        sig = bytearray(R)
        flv = self.fors_levels(idx_tree, idx_leaf)
        for i in range(K):
            g = (i << A) + fidx[i]
            sig += self.th(self.adrs(0, idx_tree, FORS_PRF, idx_leaf, 0, g), self.sk_seed, prf=True)
            for z in range(A):
                sig += flv[z][(g >> z) ^ 1]
        roots = b"".join(flv[A][i] for i in range(K))
        root = self.th(self.adrs(0, idx_tree, FORS_ROOTS, idx_leaf), roots)
        tree, leaf = idx_tree, idx_leaf
        for j in range(D):
            dg = self.digits(root)
            for i in range(LEN):
                sig += self.chain_values(j, tree, leaf, i)[dg[i]]
            lv = self.xmss_levels(j, tree)
            for z in range(HP):
                sig += lv[z][(leaf >> z) ^ 1]
            root = lv[HP][0]
            leaf, tree = tree & (2 ** HP - 1), tree >> HP
        return bytes(sig)

    def sign(self, m):
        R = hmac.new(self.sk_prf, self.pk_seed + m, hashlib.sha256).digest()[:N]
        pk_root = self.pk_root()
        seed = R + self.pk_seed + hashlib.sha256(R + self.pk_seed + pk_root + m).digest()
        digest = hashlib.sha256(seed + bytes(4)).digest()[:4]
        q = [(digest[b // 8] >> (b % 8)) & 1 for b in range(16)]
        fidx = [sum(q[i * A + j] << j for j in range(A)) for i in range(K)]
        return self.sign_fields(R, fidx, digest[2] & 3, digest[3] & 3)


@pytest.fixture(scope="module", params=["toy", "robust-toy"])
def ps(request):
    """The simple toy set and its robust instantiation."""
    return request.param


@pytest.fixture(scope="module")
def toy(ps):
    rng = random.Random(4242)
    return Toy(bytes(rng.getrandbits(8) for _ in range(3 * N)), robust=ps.startswith("robust-"))


@pytest.fixture(scope="module")
def toy_keys(O, toy, ps):
    pk, sk = O.keygen(ps, toy.sk_seed + toy.sk_prf + toy.pk_seed)
    return pk, sk


def test_toy_pk_root(O, ps, toy, toy_keys):
    pk, sk = toy_keys
    assert pk == toy.pk_seed + toy.pk_root()


def test_toy_every_xmss_node(O, ps, toy, toy_keys):
    pk, sk = toy_keys
    for layer, trees in ((0, range(2 ** (H - HP))), (1, [0])):
        for t in trees:
            lv = toy.xmss_levels(layer, t)
            for z in range(HP + 1):
                for i in range(2 ** (HP - z)):
                    assert O.xmss_node(ps, sk, layer, t, i, z) == lv[z][i]


def test_toy_every_fors_node(O, ps, toy, toy_keys):
    pk, sk = toy_keys
    for t in range(2 ** (H - HP)):
        for kp in range(2 ** HP):
            lv = toy.fors_levels(t, kp)
            for z in range(A + 1):
                for g in range(K * 2 ** (A - z)):
                    assert O.fors_node(ps, sk, t, kp, g, z) == lv[z][g]


def test_toy_all_index_pairs(O, ps, toy, toy_keys):
    pk, sk = toy_keys
    rng = random.Random(77)
    R = bytes(rng.getrandbits(8) for _ in range(N))
    for idx_tree in range(2 ** (H - HP)):
        for idx_leaf in range(2 ** HP):
            fidx = [rng.randrange(2 ** A) for _ in range(K)]
            want = toy.sign_fields(R, fidx, idx_tree, idx_leaf)
            got = O.sign_fields(ps, sk, R, fidx, idx_tree, idx_leaf)
            assert got == want, (idx_tree, idx_leaf)


def test_toy_full_sign_and_verify(O, ps, toy, toy_keys):
    pk, sk = toy_keys
    for i in range(6):
        m = bytes([i * 7 % 256]) * (i * 11)
        sig = O.sign(ps, sk, m)
        assert sig == toy.sign(m)
        assert O.verify(ps, pk, m, sig)
