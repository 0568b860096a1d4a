"""ctypes binding for the plain-C SPHINCS+ oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may use
this module.  Every call releases the GIL (ctypes foreign calls do), so a
thread pool signs on several host cores at once.
"""
import ctypes as C
from dataclasses import dataclass

from . import build as _build

PARAM_IDS = {"128f": 0, "192f": 1, "256f": 2, "toy": 3, "128s": 4, "192s": 5, "256s": 6,
             # the same sets in FIPS 205 mode (MSB-first FORS indices)
             "slh-128f": 16, "slh-192f": 17, "slh-256f": 18, "slh-toy": 19,
             "slh-128s": 20, "slh-192s": 21, "slh-256s": 22}
# the SHAKE instantiation of each set: id + 32 ("shake-128f", "slh-shake-128f", ...)
PARAM_IDS.update({"shake-" + k: v + 32 for k, v in list(PARAM_IDS.items()) if not k.startswith("slh-")})
PARAM_IDS.update({"slh-shake-" + k[4:]: v + 32 for k, v in list(PARAM_IDS.items()) if k.startswith("slh-")})
# the robust SHA2 instantiation of each round-3.1 set ("robust-128f", ...): id + 64
PARAM_IDS.update({"robust-" + k: v + 64 for k, v in list(PARAM_IDS.items()) if v < 16})

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        u8p = C.POINTER(C.c_uint8)
        L.oracle_params.argtypes = [C.c_int, C.POINTER(C.c_int64)]
        L.oracle_sha256.argtypes = [C.c_char_p, C.c_size_t, C.c_char_p]
        L.oracle_sha512.argtypes = [C.c_char_p, C.c_size_t, C.c_char_p]
        L.oracle_hmac.argtypes = [C.c_int, C.c_char_p, C.c_size_t, C.c_char_p, C.c_size_t, C.c_char_p]
        L.oracle_mgf1.argtypes = [C.c_int, C.c_char_p, C.c_size_t, C.c_char_p, C.c_size_t]
        L.oracle_sha_tables.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                        C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]
        L.oracle_adrs_compress.argtypes = [C.POINTER(C.c_uint32), C.c_char_p]
        L.oracle_thash.argtypes = [C.c_int, C.c_int, C.c_char_p, C.c_char_p,
                                   C.POINTER(C.c_uint32), C.c_char_p, C.c_int, C.c_char_p]
        L.oracle_wots_digits.argtypes = [C.c_int, C.c_char_p, C.POINTER(C.c_int32)]
        L.oracle_hash_message.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.c_size_t, C.c_char_p,
                                          C.c_char_p, C.POINTER(C.c_uint32), C.POINTER(C.c_uint64),
                                          C.POINTER(C.c_uint32)]
        L.oracle_split_digest.argtypes = [C.c_int, C.c_char_p, C.POINTER(C.c_uint32),
                                          C.POINTER(C.c_uint64), C.POINTER(C.c_uint32)]
        L.oracle_wots_chain.argtypes = [C.c_int, C.c_char_p, C.c_uint32, C.c_uint64, C.c_uint32,
                                        C.c_int, C.c_char_p, C.c_int, C.c_int, C.c_char_p]
        L.oracle_wots_sk.argtypes = [C.c_int, C.c_char_p, C.c_uint32, C.c_uint64, C.c_uint32,
                                     C.c_int, C.c_char_p]
        L.oracle_wots_pkgen.argtypes = [C.c_int, C.c_char_p, C.c_uint32, C.c_uint64, C.c_uint32, C.c_char_p]
        L.oracle_wots_sign.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.c_uint32, C.c_uint64,
                                       C.c_uint32, C.c_char_p]
        L.oracle_wots_pk_from_sig.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.c_char_p, C.c_uint32,
                                              C.c_uint64, C.c_uint32, C.c_char_p]
        L.oracle_xmss_node.argtypes = [C.c_int, C.c_char_p, C.c_uint32, C.c_uint64, C.c_uint32,
                                       C.c_int, C.c_char_p]
        L.oracle_xmss_root_from_sig.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.c_char_p, C.c_uint32,
                                                C.c_uint64, C.c_uint32, C.c_char_p]
        L.oracle_fors_node.argtypes = [C.c_int, C.c_char_p, C.c_uint64, C.c_uint32, C.c_uint32,
                                       C.c_int, C.c_char_p]
        L.oracle_fors_sk.argtypes = [C.c_int, C.c_char_p, C.c_uint64, C.c_uint32, C.c_uint32, C.c_char_p]
        L.oracle_fors_pk_from_sig.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.POINTER(C.c_uint32),
                                              C.c_uint64, C.c_uint32, C.c_char_p]
        L.oracle_keygen.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.c_char_p]
        L.oracle_sign.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.c_size_t, C.c_char_p]
        L.oracle_sign_fields.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.POINTER(C.c_uint32),
                                         C.c_uint64, C.c_uint32, C.c_char_p]
        L.oracle_verify.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.c_size_t, C.c_char_p]
        L.oracle_slh_sign.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.c_size_t, C.c_char_p, C.c_size_t,
                                      C.c_char_p]
        L.oracle_slh_verify.argtypes = [C.c_int, C.c_char_p, C.c_char_p, C.c_size_t, C.c_char_p, C.c_size_t,
                                        C.c_char_p]
        L.oracle_counters.argtypes = [C.POINTER(C.c_uint64), C.c_int]
        L.oracle_shake256.argtypes = [C.c_char_p, C.c_size_t, C.c_char_p, C.c_size_t]
        L.oracle_keccak_f1600.argtypes = [C.POINTER(C.c_uint64)]
        for name in ("oracle_params", "oracle_thash", "oracle_wots_digits", "oracle_hash_message",
                     "oracle_split_digest", "oracle_wots_chain", "oracle_wots_sk", "oracle_wots_pkgen",
                     "oracle_wots_sign", "oracle_wots_pk_from_sig", "oracle_xmss_node",
                     "oracle_xmss_root_from_sig", "oracle_fors_node", "oracle_fors_sk",
                     "oracle_fors_pk_from_sig", "oracle_keygen", "oracle_sign", "oracle_sign_fields",
                     "oracle_verify", "oracle_slh_sign", "oracle_slh_verify"):
            getattr(L, name).restype = C.c_int
        for name in ("oracle_sha256", "oracle_sha512", "oracle_hmac", "oracle_mgf1",
                     "oracle_sha_tables", "oracle_adrs_compress", "oracle_counters"):
            getattr(L, name).restype = None
        _lib = L
    return _lib


class library:
    """Context manager that points every call of this module at another build
    of the oracle source (the tests use it to check that the pins catch
    deliberately planted mistakes), restoring the regular build on exit."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = lib()
        _lib = None
        real_build = _build.build
        _build.build = lambda force=False, _p=self.path: _p
        try:
            lib()
        finally:
            _build.build = real_build
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved


def _pid(ps):
    return PARAM_IDS[ps] if isinstance(ps, str) else int(ps)


def _check(rc):
    if rc < 0:
        raise ValueError("oracle: bad parameter set")
    return rc


@dataclass(frozen=True)
class Params:
    """Parameter set as the oracle derives it from Table 1 of the paper."""
    name: str
    n: int
    h: int
    d: int
    hp: int
    a: int
    k: int
    w: int
    big: int
    len1: int
    len2: int
    len: int
    md_bytes: int
    tree_bytes: int
    leaf_bytes: int
    m: int
    sig_bytes: int

    @property
    def fors_bytes(self):
        return self.k * (self.a + 1) * self.n

    @property
    def layer_bytes(self):
        return (self.len + self.hp) * self.n


def params(ps) -> Params:
    info = (C.c_int64 * 16)()
    _check(lib().oracle_params(_pid(ps), info))
    name = ps if isinstance(ps, str) else {v: k for k, v in PARAM_IDS.items()}[ps]
    return Params(name, *[int(x) for x in info])


def sha256(m: bytes) -> bytes:
    out = C.create_string_buffer(32)
    lib().oracle_sha256(m, len(m), out)
    return out.raw


def sha512(m: bytes) -> bytes:
    out = C.create_string_buffer(64)
    lib().oracle_sha512(m, len(m), out)
    return out.raw


def hmac(big: int, key: bytes, m: bytes) -> bytes:
    out = C.create_string_buffer(64 if big else 32)
    lib().oracle_hmac(big, key, len(key), m, len(m), out)
    return out.raw


def mgf1(big: int, seed: bytes, outlen: int) -> bytes:
    out = C.create_string_buffer(max(outlen, 1))
    lib().oracle_mgf1(big, seed, len(seed), out, outlen)
    return out.raw[:outlen]


def sha_tables():
    k256 = (C.c_uint32 * 64)(); iv256 = (C.c_uint32 * 8)()
    k512 = (C.c_uint64 * 80)(); iv512 = (C.c_uint64 * 8)()
    lib().oracle_sha_tables(k256, iv256, k512, iv512)
    return list(k256), list(iv256), list(k512), list(iv512)


def adrs_compress(words8) -> bytes:
    w = (C.c_uint32 * 8)(*words8)
    out = C.create_string_buffer(22)
    lib().oracle_adrs_compress(w, out)
    return out.raw


THASH_F, THASH_H, THASH_T, THASH_PRF = 0, 1, 2, 3


def thash(ps, which, pk_seed: bytes, words8, data: bytes = b"", l: int = 0, sk_seed: bytes = None) -> bytes:
    P = params(ps)
    out = C.create_string_buffer(32)
    w = (C.c_uint32 * 8)(*words8)
    _check(lib().oracle_thash(_pid(ps), which, pk_seed, sk_seed, w, data or b"\0", l, out))
    return out.raw[:P.n]


def wots_digits(ps, msg: bytes):
    P = params(ps)
    d = (C.c_int32 * P.len)()
    _check(lib().oracle_wots_digits(_pid(ps), msg, d))
    return list(d)


def hash_message(ps, sk: bytes, m: bytes):
    """(R, digest, fors_indices, idx_tree, idx_leaf) of message m under sk."""
    P = params(ps)
    R = C.create_string_buffer(32); dg = C.create_string_buffer(64)
    fidx = (C.c_uint32 * P.k)(); it = C.c_uint64(); il = C.c_uint32()
    _check(lib().oracle_hash_message(_pid(ps), sk, m, len(m), R, dg, fidx, C.byref(it), C.byref(il)))
    return R.raw[:P.n], dg.raw[:P.m], list(fidx), it.value, il.value


def split_digest(ps, digest: bytes):
    P = params(ps)
    fidx = (C.c_uint32 * P.k)(); it = C.c_uint64(); il = C.c_uint32()
    _check(lib().oracle_split_digest(_pid(ps), digest, fidx, C.byref(it), C.byref(il)))
    return list(fidx), it.value, il.value


def wots_chain(ps, sk, layer, tree, kp, chain, x, start, steps):
    out = C.create_string_buffer(32)
    _check(lib().oracle_wots_chain(_pid(ps), sk, layer, tree, kp, chain, x, start, steps, out))
    return out.raw[:params(ps).n]


def wots_sk(ps, sk, layer, tree, kp, chain):
    out = C.create_string_buffer(32)
    _check(lib().oracle_wots_sk(_pid(ps), sk, layer, tree, kp, chain, out))
    return out.raw[:params(ps).n]


def wots_pkgen(ps, sk, layer, tree, kp):
    out = C.create_string_buffer(32)
    _check(lib().oracle_wots_pkgen(_pid(ps), sk, layer, tree, kp, out))
    return out.raw[:params(ps).n]


def wots_sign(ps, sk, msg, layer, tree, kp):
    P = params(ps)
    out = C.create_string_buffer(P.len * P.n)
    _check(lib().oracle_wots_sign(_pid(ps), sk, msg, layer, tree, kp, out))
    return out.raw


def wots_pk_from_sig(ps, sk, sig, msg, layer, tree, kp):
    out = C.create_string_buffer(32)
    _check(lib().oracle_wots_pk_from_sig(_pid(ps), sk, sig, msg, layer, tree, kp, out))
    return out.raw[:params(ps).n]


def xmss_node(ps, sk, layer, tree, idx, z):
    out = C.create_string_buffer(32)
    _check(lib().oracle_xmss_node(_pid(ps), sk, layer, tree, idx, z, out))
    return out.raw[:params(ps).n]


def xmss_root_from_sig(ps, sk, sig, msg, layer, tree, leaf):
    out = C.create_string_buffer(32)
    _check(lib().oracle_xmss_root_from_sig(_pid(ps), sk, sig, msg, layer, tree, leaf, out))
    return out.raw[:params(ps).n]


def fors_node(ps, sk, idx_tree, idx_leaf, g, z):
    out = C.create_string_buffer(32)
    _check(lib().oracle_fors_node(_pid(ps), sk, idx_tree, idx_leaf, g, z, out))
    return out.raw[:params(ps).n]


def fors_sk(ps, sk, idx_tree, idx_leaf, g):
    out = C.create_string_buffer(32)
    _check(lib().oracle_fors_sk(_pid(ps), sk, idx_tree, idx_leaf, g, out))
    return out.raw[:params(ps).n]


def fors_pk_from_sig(ps, sk, sig_fors, fidx, idx_tree, idx_leaf):
    P = params(ps)
    f = (C.c_uint32 * P.k)(*fidx)
    out = C.create_string_buffer(32)
    _check(lib().oracle_fors_pk_from_sig(_pid(ps), sk, sig_fors, f, idx_tree, idx_leaf, out))
    return out.raw[:P.n]


def keygen(ps, seed: bytes):
    """(pk, sk) from a 3n-byte seed SK.seed || SK.prf || PK.seed."""
    P = params(ps)
    if len(seed) != 3 * P.n:
        raise ValueError("seed must be 3n bytes")
    pk = C.create_string_buffer(2 * P.n); sk = C.create_string_buffer(4 * P.n)
    _check(lib().oracle_keygen(_pid(ps), seed, pk, sk))
    return pk.raw, sk.raw


def sign(ps, sk: bytes, m: bytes) -> bytes:
    P = params(ps)
    sig = C.create_string_buffer(P.sig_bytes)
    _check(lib().oracle_sign(_pid(ps), sk, m, len(m), sig))
    return sig.raw


def sign_fields(ps, sk, R, fidx, idx_tree, idx_leaf) -> bytes:
    P = params(ps)
    f = (C.c_uint32 * P.k)(*fidx)
    sig = C.create_string_buffer(P.sig_bytes)
    _check(lib().oracle_sign_fields(_pid(ps), sk, R, f, idx_tree, idx_leaf, sig))
    return sig.raw


def verify(ps, pk: bytes, m: bytes, sig: bytes) -> bool:
    return _check(lib().oracle_verify(_pid(ps), pk, m, len(m), sig)) == 1


def slh_sign(ps, sk: bytes, ctx: bytes, m: bytes) -> bytes:
    """FIPS 205 pure SLH-DSA signature (deterministic) of m under context ctx;
    ps is the base set ("128f", ...)."""
    P = params(ps)
    sig = C.create_string_buffer(P.sig_bytes)
    _check(lib().oracle_slh_sign(_pid(ps), sk, ctx, len(ctx), m, len(m), sig))
    return sig.raw


def slh_verify(ps, pk: bytes, ctx: bytes, m: bytes, sig: bytes) -> bool:
    return _check(lib().oracle_slh_verify(_pid(ps), pk, ctx, len(ctx), m, len(m), sig)) == 1


def shake256(m: bytes, outlen: int) -> bytes:
    out = C.create_string_buffer(max(outlen, 1))
    lib().oracle_shake256(m, len(m), out, outlen)
    return out.raw[:outlen]


def keccak_f1600(lanes):
    """One Keccak-f[1600] permutation of 25 little-endian 64-bit lanes A[x + 5y]."""
    st = (C.c_uint64 * 25)(*lanes)
    lib().oracle_keccak_f1600(st)
    return list(st)


def counters(reset=False):
    """[SHA-256 blocks, SHA-512 blocks, F, PRF, H, T, Keccak permutations] of
    the calling thread."""
    out = (C.c_uint64 * 7)()
    lib().oracle_counters(out, 1 if reset else 0)
    return list(out)
