"""Thin Python binding of libhs.so (include/hs.h).

Argument marshalling only: tensors (CUDA or CPU) and numpy arrays are passed
to the C ABI as raw pointers with the current CUDA stream; every step of
signing and verifying runs in the library's kernels.  There is no fallback:
if ``libhs.so`` is missing or cannot be loaded, :func:`load` raises.
"""
import ctypes as C
import os

import numpy as np

PARAMS = {"128f": 0, "192f": 1, "256f": 2, "toy": 3, "128s": 4, "192s": 5, "256s": 6,
          "shake-128f": 7, "shake-192f": 8, "shake-256f": 9, "shake-128s": 10, "shake-192s": 11, "shake-256s": 12,
          "robust-128f": 13, "robust-192f": 14, "robust-256f": 15}
N_BYTES = {"128f": 16, "192f": 24, "256f": 32, "toy": 16, "128s": 16, "192s": 24, "256s": 32}
N_BYTES.update({"shake-" + k: v for k, v in list(N_BYTES.items()) if k != "toy"})
N_BYTES.update({"robust-" + k: N_BYTES[k] for k in ("128f", "192f", "256f")})
NUM_PARAMS = 16
_N_BY_ID = [16, 24, 32, 16, 16, 24, 32, 16, 24, 32, 16, 24, 32, 16, 24, 32]
STATUS = {0: "HS_OK", 1: "HS_EINVAL", 2: "HS_ENOMEM", 3: "HS_ECUDA", 4: "HS_ETIMEOUT", 5: "HS_EKEY",
          6: "HS_ECANCELED", 7: "HS_EBUDGET"}
LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libhs.so")

_lib = None


class HSError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (STATUS.get(code, code), msg))
        self.code = code


def load():
    """Load libhs.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libhs.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, u32, u64p = C.c_void_p, C.c_uint32, C.c_void_p
    for name in ("hs_sig_bytes", "hs_pk_bytes", "hs_sk_bytes", "hs_seed_bytes"):
        getattr(L, name).argtypes = [C.c_int]
        getattr(L, name).restype = C.c_size_t
    L.hs_keygen.argtypes = [C.c_int, vp, u32, vp, vp, vp]
    L.hs_sign_batch.argtypes = [C.c_int, vp, u32, vp, vp, u64p, u32, vp, vp]
    L.hs_verify_batch.argtypes = [C.c_int, vp, u32, vp, vp, u64p, vp, u32, vp, vp]
    L.hs_check_status.argtypes = [vp, C.POINTER(C.c_uint32)]
    L.hs_last_error.restype = C.c_char_p
    L.hs_last_error_copy.argtypes = [C.c_char_p, C.c_size_t]
    L.hs_last_error_copy.restype = C.c_int
    L.hs_profile_enable.argtypes = [C.c_int]
    L.hs_profile_read.argtypes = [C.POINTER(C.c_float), C.POINTER(C.c_char_p), C.c_int]
    L.hs_profile_read.restype = C.c_int
    L.hs_sign_kernel_count.restype = C.c_int
    L.hs_sign_batch_noalloc.argtypes = [C.c_int, vp, u32, vp, vp, u64p, u32, vp, vp]
    L.hs_sign_batch_noalloc.restype = C.c_int
    L.hs_probe_int_pipes.argtypes = [C.POINTER(C.c_float), C.c_int]
    L.hs_probe_int_pipes.restype = C.c_int
    L.hs_probe_sha_mix.argtypes = [C.POINTER(C.c_float), C.c_int]
    L.hs_probe_sha_mix.restype = C.c_int
    L.hs_sign_mixed.argtypes = [C.c_void_p, C.c_uint32, C.c_int, C.c_void_p]
    L.hs_sign_mixed.restype = C.c_int
    L.hs_server_create.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]
    L.hs_server_submit.argtypes = [C.c_void_p, C.c_int, C.c_uint32, C.c_void_p, C.c_uint64, C.c_void_p,
                                   C.POINTER(C.c_uint64)]
    L.hs_server_wait.argtypes = [C.c_void_p, C.c_uint64, C.c_uint32]
    L.hs_server_poll.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    L.hs_server_poll.restype = C.c_int
    L.hs_server_get_stats.argtypes = [C.c_void_p, C.c_void_p]
    L.hs_server_replay.argtypes = [C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_uint32]
    L.hs_server_destroy.argtypes = [C.c_void_p]
    L.hs_slh_sign_batch.argtypes = [C.c_int, vp, u32, vp, vp, u32, vp, u64p, u32, vp, vp]
    L.hs_slh_sign_batch.restype = C.c_int
    L.hs_slh_verify_batch.argtypes = [C.c_int, vp, u32, vp, vp, u32, vp, u64p, vp, u32, vp, vp]
    L.hs_slh_verify_batch.restype = C.c_int
    L.hs_keyset_create.argtypes = [C.c_int, vp, u32, u32, vp, C.POINTER(C.c_void_p)]
    L.hs_keyset_create.restype = C.c_int
    L.hs_keyset_bytes.argtypes = [vp]
    L.hs_keyset_bytes.restype = C.c_size_t
    L.hs_sign_keyset.argtypes = [vp, vp, vp, u64p, u32, vp, vp]
    L.hs_sign_keyset.restype = C.c_int
    L.hs_keyset_destroy.argtypes = [vp]
    L.hs_keyset_destroy.restype = C.c_int
    L.hs_server_cancel.argtypes = [C.c_void_p, C.c_uint64]
    L.hs_server_cancel.restype = C.c_int
    L.hs_server_inject_launch_failures.argtypes = [C.c_void_p, C.c_uint32]
    L.hs_server_inject_launch_failures.restype = C.c_int
    for name in ("hs_server_create", "hs_server_submit", "hs_server_wait", "hs_server_get_stats",
                 "hs_server_replay", "hs_server_destroy"):
        getattr(L, name).restype = C.c_int
    L.hs_set_tree_sharing.argtypes = [C.c_int]
    L.hs_set_tree_sharing.restype = C.c_int
    L.hs_set_host_direct.argtypes = [C.c_int]
    L.hs_set_host_direct.restype = C.c_int
    L.hs_set_chain_checkpoint.argtypes = [C.c_uint32]
    L.hs_set_chain_checkpoint.restype = C.c_int
    for name in ("hs_keygen", "hs_sign_batch", "hs_verify_batch", "hs_check_status"):
        getattr(L, name).restype = C.c_int
    _lib = L
    return L


def _pid(params):
    return PARAMS[params] if isinstance(params, str) else int(params)


def last_error(maxlen=512):
    """The calling thread's most recent error text (hs_last_error_copy)."""
    buf = C.create_string_buffer(maxlen)
    load().hs_last_error_copy(buf, maxlen)
    return buf.value.decode(errors="replace")


def _check(rc):
    if rc != 0:
        raise HSError(rc, last_error())


def _ptr(x):
    """Raw address of a tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data if x.size else None
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return x.data_ptr() if x.numel() else None


def _numel(x):
    return int(x.size) if isinstance(x, np.ndarray) else int(x.numel())


def _buf(x, name, itemsize, min_elems=0):
    """Check a buffer before its address goes to the C ABI: the element size
    the library reads (1 for bytes, 4 for key indices, 8 for lengths) and at
    least min_elems elements, so that a wrong dtype or a short buffer raises
    here instead of being read past its end.  None passes (NULL)."""
    if x is None:
        return None
    isz = int(x.itemsize) if isinstance(x, np.ndarray) else int(x.element_size())
    if isz != itemsize:
        raise ValueError("%s: elements of %d bytes expected, got %d" % (name, itemsize, isz))
    if _numel(x) < min_elems:
        raise ValueError("%s: at least %d elements needed, got %d" % (name, min_elems, _numel(x)))
    return x


def _msgs_lens(msgs, lens, key_idx=None):
    """Checks shared by the signing and verification calls: lens (8-byte
    lengths, one per message), key_idx (4-byte, one per message), msgs
    (bytes; covering the lengths when they are on the host)."""
    count = int(lens.shape[0])
    _buf(lens, "lens", 8)
    _buf(key_idx, "key_idx", 4, count)
    if msgs is not None:
        _buf(msgs, "msgs", 1)
        if isinstance(lens, np.ndarray) and count:
            need = int(lens.astype(np.uint64).sum())
            if _numel(msgs) < need:
                raise ValueError("msgs: the lengths add up to %d bytes, the buffer has %d" % (need, _numel(msgs)))
    return count


def _stream(stream):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    import torch
    return torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None


def _like(x, n, dtype_np, dtype_torch_name):
    """Allocate an output on the same side (device / host) as x."""
    if isinstance(x, np.ndarray):
        return np.empty(n, dtype=dtype_np)
    import torch
    return torch.empty(n, dtype=getattr(torch, dtype_torch_name), device=x.device)


def _nonempty(msgs, lens):
    """A batch whose messages are all empty still passes a valid message
    buffer (the C ABI accepts NULL only with host-side lengths)."""
    if msgs is None or (msgs.size if isinstance(msgs, np.ndarray) else msgs.numel()) == 0:
        return _like(lens, 16, np.uint8, "uint8")
    return msgs


def sig_bytes(params):
    return int(load().hs_sig_bytes(_pid(params)))


def hs_keygen(params, seeds, pk=None, sk=None, stream=None):
    """(pk, sk) for each 3n-byte seed row of ``seeds`` (uint8 [count, 3n])."""
    n = N_BYTES[params] if isinstance(params, str) else _N_BY_ID[params]
    count = seeds.shape[0] if seeds.ndim == 2 else seeds.shape[0] // (3 * n)
    _buf(seeds, "seeds", 1, count * 3 * n)
    pk = _like(seeds, count * 2 * n, np.uint8, "uint8") if pk is None else _buf(pk, "pk", 1, count * 2 * n)
    sk = _like(seeds, count * 4 * n, np.uint8, "uint8") if sk is None else _buf(sk, "sk", 1, count * 4 * n)
    _check(load().hs_keygen(_pid(params), _ptr(seeds), count, _ptr(pk), _ptr(sk), _stream(stream)))
    return pk.reshape(count, 2 * n), sk.reshape(count, 4 * n)


def hs_sign_batch(params, sk, msgs, lens, key_idx=None, sigs=None, num_keys=None, stream=None):
    """Signatures (uint8 [count, SIG]) of the packed messages ``msgs`` with lengths ``lens``."""
    count = _msgs_lens(msgs, lens, key_idx)
    n = N_BYTES[params] if isinstance(params, str) else _N_BY_ID[params]
    if num_keys is None:
        num_keys = (sk.shape[0] if sk.ndim == 2 else sk.shape[0] // (4 * n))
    _buf(sk, "sk", 1, int(num_keys) * 4 * n)
    S = sig_bytes(params)
    sigs = _like(lens, count * S, np.uint8, "uint8") if sigs is None else _buf(sigs, "sigs", 1, count * S)
    msgs = _nonempty(msgs, lens)
    _check(load().hs_sign_batch(_pid(params), _ptr(sk), int(num_keys), _ptr(key_idx), _ptr(msgs), _ptr(lens),
                                count, _ptr(sigs), _stream(stream)))
    return sigs.reshape(count, S)


SLH_INTERNAL = 0xFFFFFFFF


def _ctx(ctx):
    """(buffer, length) of a context string; None = the internal functions."""
    if ctx is None:
        return None, SLH_INTERNAL
    ctx = bytes(ctx)
    return (C.create_string_buffer(ctx, len(ctx)) if ctx else None), len(ctx)


def hs_slh_sign_batch(params, sk, msgs, lens, ctx=b"", key_idx=None, sigs=None, num_keys=None, stream=None):
    """FIPS 205 SLH-DSA signatures (deterministic) of every message under one
    context string; ctx=None signs the messages as given (internal function)."""
    count = _msgs_lens(msgs, lens, key_idx)
    n = N_BYTES[params] if isinstance(params, str) else _N_BY_ID[params]
    if num_keys is None:
        num_keys = (sk.shape[0] if sk.ndim == 2 else sk.shape[0] // (4 * n))
    _buf(sk, "sk", 1, int(num_keys) * 4 * n)
    S = sig_bytes(params)
    sigs = _like(lens, count * S, np.uint8, "uint8") if sigs is None else _buf(sigs, "sigs", 1, count * S)
    msgs = _nonempty(msgs, lens)
    cbuf, clen = _ctx(ctx)
    _check(load().hs_slh_sign_batch(_pid(params), _ptr(sk), int(num_keys), _ptr(key_idx), cbuf, clen, _ptr(msgs),
                                    _ptr(lens), count, _ptr(sigs), _stream(stream)))
    return sigs.reshape(count, S)


def hs_slh_verify_batch(params, pk, msgs, lens, sigs, ctx=b"", key_idx=None, ok=None, num_keys=None, stream=None):
    """1/0 per FIPS 205 signature under one context string."""
    count = _msgs_lens(msgs, lens, key_idx)
    n = N_BYTES[params] if isinstance(params, str) else _N_BY_ID[params]
    if num_keys is None:
        num_keys = (pk.shape[0] if pk.ndim == 2 else pk.shape[0] // (2 * n))
    _buf(pk, "pk", 1, int(num_keys) * 2 * n)
    _buf(sigs, "sigs", 1, count * sig_bytes(params))
    ok = _like(lens, count, np.uint8, "uint8") if ok is None else _buf(ok, "ok", 1, count)
    msgs = _nonempty(msgs, lens)
    cbuf, clen = _ctx(ctx)
    _check(load().hs_slh_verify_batch(_pid(params), _ptr(pk), int(num_keys), _ptr(key_idx), cbuf, clen, _ptr(msgs),
                                      _ptr(lens), _ptr(sigs), count, _ptr(ok), _stream(stream)))
    return ok


class KeySet:
    """Resident signing keys with their top ``cache_layers`` hypertree layers
    prebuilt (hs_keyset_* of include/hs.h); ``sign`` gives the same bytes as
    hs_sign_batch with these keys."""

    def __init__(self, params, sk, cache_layers=0, stream=None):
        L = load()
        n = N_BYTES[params] if isinstance(params, str) else _N_BY_ID[params]
        self.params = params
        self.num_keys = int(sk.shape[0] if sk.ndim == 2 else sk.shape[0] // (4 * n))
        _buf(sk, "sk", 1, self.num_keys * 4 * n)
        h = C.c_void_p()
        _check(L.hs_keyset_create(_pid(params), _ptr(sk), self.num_keys, int(cache_layers), _stream(stream),
                                  C.byref(h)))
        self._h = h
        self.cache_layers = int(cache_layers)

    @property
    def nbytes(self):
        return int(load().hs_keyset_bytes(self._h))

    def sign(self, msgs, lens, key_idx=None, sigs=None, stream=None):
        count = _msgs_lens(msgs, lens, key_idx)
        S = sig_bytes(self.params)
        sigs = _like(lens, count * S, np.uint8, "uint8") if sigs is None else _buf(sigs, "sigs", 1, count * S)
        msgs = _nonempty(msgs, lens)
        _check(load().hs_sign_keyset(self._h, _ptr(key_idx), _ptr(msgs), _ptr(lens), count, _ptr(sigs),
                                     _stream(stream)))
        return sigs.reshape(count, S)

    def close(self):
        if getattr(self, "_h", None):
            load().hs_keyset_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hs_verify_batch(params, pk, msgs, lens, sigs, key_idx=None, ok=None, num_keys=None, stream=None):
    """1/0 per signature (uint8 [count])."""
    count = _msgs_lens(msgs, lens, key_idx)
    n = N_BYTES[params] if isinstance(params, str) else _N_BY_ID[params]
    if num_keys is None:
        num_keys = (pk.shape[0] if pk.ndim == 2 else pk.shape[0] // (2 * n))
    _buf(pk, "pk", 1, int(num_keys) * 2 * n)
    _buf(sigs, "sigs", 1, count * sig_bytes(params))
    ok = _like(lens, count, np.uint8, "uint8") if ok is None else _buf(ok, "ok", 1, count)
    msgs = _nonempty(msgs, lens)
    _check(load().hs_verify_batch(_pid(params), _ptr(pk), int(num_keys), _ptr(key_idx), _ptr(msgs), _ptr(lens),
                                  _ptr(sigs), count, _ptr(ok), _stream(stream)))
    return ok


def hs_check_status(stream=None):
    """Synchronize the stream; return the device status flags (and clear them)."""
    flags = C.c_uint32(0)
    rc = load().hs_check_status(_stream(stream), C.byref(flags))
    return rc, flags.value


def hs_profile_enable(on=True):
    load().hs_profile_enable(1 if on else 0)


def hs_profile_read():
    """{stage name: ms} of the most recent profiled hs_sign_batch call."""
    ms = (C.c_float * 16)()
    names = (C.c_char_p * 16)()
    n = load().hs_profile_read(ms, names, 16)
    if n < 0:
        return {}
    return {names[i].decode(): float(ms[i]) for i in range(n)}


def hs_sign_kernel_count():
    return int(load().hs_sign_kernel_count())


def hs_set_chain_checkpoint(stride):
    """Stride of the WOTS+ chain positions TREE_Sign keeps for WOTS+_Sign (0 = none)."""
    _check(load().hs_set_chain_checkpoint(int(stride)))


def hs_sign_batch_noalloc(params, sk, msgs, lens, sigs, key_idx=None, num_keys=None, stream=None):
    """Like hs_sign_batch, for callers that cannot allocate device memory:
    all buffers (including the output ``sigs``) are caller-provided device
    tensors, and the library works in its fixed 8 MiB device buffer."""
    count = _msgs_lens(msgs, lens, key_idx)
    n = N_BYTES[params] if isinstance(params, str) else _N_BY_ID[params]
    if num_keys is None:
        num_keys = (sk.shape[0] if sk.ndim == 2 else sk.shape[0] // (4 * n))
    _buf(sk, "sk", 1, int(num_keys) * 4 * n)
    _buf(sigs, "sigs", 1, count * sig_bytes(params))
    _check(load().hs_sign_batch_noalloc(_pid(params), _ptr(sk), int(num_keys), _ptr(key_idx), _ptr(msgs),
                                        _ptr(lens), count, _ptr(sigs), _stream(stream)))
    return sigs


PIPE_FORMS = ("lop3", "shf", "iadd", "imad", "imad_hi", "prmt", "lop3+imad")


def hs_probe_int_pipes():
    """{instruction form: measured lane-ops per clock per SM} on the current GPU."""
    r = (C.c_float * 8)()
    n = load().hs_probe_int_pipes(r, 8)
    if n < 0:
        raise HSError(3, "hs_probe_int_pipes failed")
    return {PIPE_FORMS[i]: round(float(r[i]), 2) for i in range(n)}


SHA_MIX_FORMS = ("sha256_per_clk_sm", "sha512_per_clk_sm", "add64_lane_ops_per_clk_sm", "sha256_plain_per_clk_sm")


def hs_probe_sha_mix():
    """{form: measured rate per clock per SM} of the SHA-2 instruction mix on
    the current GPU: SHA-256 (the signer's round code) and SHA-512
    compressions, 64-bit additions, and SHA-256 as FIPS 180-4 writes it."""
    r = (C.c_float * 4)()
    n = load().hs_probe_sha_mix(r, 4)
    if n < 0:
        raise HSError(3, "hs_probe_sha_mix failed")
    return {SHA_MIX_FORMS[i]: round(float(r[i]), 2 if i == 2 else 5) for i in range(n)}


class SignJob(C.Structure):
    """hs_sign_job of include/hs.h."""
    _fields_ = [("params", C.c_int), ("sk", C.c_void_p), ("num_keys", C.c_uint32), ("key_idx", C.c_void_p),
                ("msgs", C.c_void_p), ("lens", C.c_void_p), ("count", C.c_uint32), ("sigs", C.c_void_p)]


def hs_sign_mixed(jobs, use_graph=True, stream=None):
    """Sign several batches (possibly different parameter sets) in one call.
    ``jobs``: sequence of dicts with params, sk, msgs, lens, sigs and
    optionally key_idx, num_keys (device tensors).  Returns the sigs tensors."""
    arr = (SignJob * len(jobs))()
    for j, jb in enumerate(jobs):
        ps = jb["params"]
        n = N_BYTES[ps] if isinstance(ps, str) else _N_BY_ID[ps]
        sk = jb["sk"]
        nk = jb.get("num_keys") or (sk.shape[0] if sk.ndim == 2 else sk.shape[0] // (4 * n))
        cnt = _msgs_lens(jb["msgs"], jb["lens"], jb.get("key_idx"))
        _buf(sk, "sk", 1, int(nk) * 4 * n)
        _buf(jb["sigs"], "sigs", 1, cnt * sig_bytes(ps))
        msgs = _nonempty(jb["msgs"], jb["lens"])
        arr[j] = SignJob(_pid(ps), _ptr(sk), int(nk), _ptr(jb.get("key_idx")), _ptr(msgs), _ptr(jb["lens"]),
                         int(jb["lens"].shape[0]), _ptr(jb["sigs"]))
    _check(load().hs_sign_mixed(C.cast(arr, C.c_void_p), len(jobs), 1 if use_graph else 0, _stream(stream)))
    return [jb["sigs"] for jb in jobs]


class ServerConfig(C.Structure):
    _fields_ = [("max_inflight", C.c_uint32), ("max_batch", C.c_uint32), ("mem_budget_bytes", C.c_uint64),
                ("pinned_bytes", C.c_uint64), ("cache_layers", C.c_uint32)]


class ServerStats(C.Structure):
    _fields_ = [("completed", C.c_uint64), ("batches", C.c_uint64), ("batched_requests", C.c_uint64),
                ("pending", C.c_uint64), ("max_device_bytes_in_use", C.c_uint64),
                ("max_inflight_batches", C.c_uint32), ("failed", C.c_uint64), ("cancelled", C.c_uint64)]


class Server:
    """Continuous-batching signing server (hs_server_* of include/hs.h).

    ``keys``: {params: sk array/tensor [num_keys, 4n]} for the sets it serves.
    """

    def __init__(self, keys, max_inflight=4, max_batch=1024, mem_budget=8 << 30, pinned=0, cache_layers=0):
        L = load()
        self._keepalive = []
        sks = (C.c_void_p * NUM_PARAMS)()
        nk = (C.c_uint32 * NUM_PARAMS)()
        for ps, sk in keys.items():
            pid = PARAMS[ps]
            self._keepalive.append(sk)
            sks[pid] = _ptr(sk)
            nk[pid] = int(sk.shape[0])
        cfg = ServerConfig(int(max_inflight), int(max_batch), int(mem_budget), int(pinned), int(cache_layers))
        h = C.c_void_p()
        _check(L.hs_server_create(C.byref(cfg), sks, nk, C.byref(h)))
        self._h = h
        self.budget = int(mem_budget)

    def submit(self, params, key, msg, out=None):
        """Queue one request; returns (id, out) where out receives the signature."""
        msg = bytes(msg)
        if out is None:
            out = np.empty(sig_bytes(params), dtype=np.uint8)
        else:                        # the server copies the signature into it from the host
            if not isinstance(out, np.ndarray) and out.is_cuda:
                raise ValueError("out: host memory expected (the server writes it on the host)")
            _buf(out, "out", 1, sig_bytes(params))
        rid = C.c_uint64()
        buf = C.create_string_buffer(msg, len(msg)) if msg else None
        _check(load().hs_server_submit(self._h, _pid(params), int(key), buf, len(msg), _ptr(out), C.byref(rid)))
        return rid.value, out

    def wait(self, rid, timeout_ms=60000):
        _check(load().hs_server_wait(self._h, int(rid), int(timeout_ms)))

    def poll(self, max_n=4096, with_status=False):
        """Finished requests as (id, latency_ns), or (id, latency_ns, status)."""
        ids = np.empty(max_n, dtype=np.uint64)
        lat = np.empty(max_n, dtype=np.uint64)
        st = np.empty(max_n, dtype=np.int32)
        n = load().hs_server_poll(self._h, _ptr(ids), _ptr(lat), _ptr(st), max_n)
        if with_status:
            return list(zip(ids[:n].tolist(), lat[:n].tolist(), st[:n].tolist()))
        return list(zip(ids[:n].tolist(), lat[:n].tolist()))

    def stats(self):
        st = ServerStats()
        rc = load().hs_server_get_stats(self._h, C.byref(st))
        d = {f: getattr(st, f) for f, _ in ServerStats._fields_}
        d["status"] = rc
        return d

    def replay(self, params, keys, pool_idx, pool_msgs, pool_lens, arrival_ns, keep_signatures=False,
               timeout_ms=600000):
        """Open-loop load: request i arrives arrival_ns[i] after the start.
        Returns (latency_ns array, signatures list or None)."""
        params = np.ascontiguousarray(params, dtype=np.uint8)
        keys = np.ascontiguousarray(keys, dtype=np.uint32)
        pool_idx = np.ascontiguousarray(pool_idx, dtype=np.uint32)
        pool_lens = np.ascontiguousarray(pool_lens, dtype=np.uint64)
        arrival_ns = np.ascontiguousarray(arrival_ns, dtype=np.uint64)
        n = int(params.shape[0])
        for name, a in (("keys", keys), ("pool_idx", pool_idx), ("arrival_ns", arrival_ns)):
            if a.shape[0] != n:
                raise ValueError("%s: %d entries for %d requests" % (name, a.shape[0], n))
        if pool_msgs is not None:
            pool_msgs = np.ascontiguousarray(pool_msgs, dtype=np.uint8)
        need = int(pool_lens.sum())
        if need and (pool_msgs is None or pool_msgs.size < need):
            raise ValueError("pool_msgs: the pool lengths add up to %d bytes, the buffer has %d"
                             % (need, 0 if pool_msgs is None else pool_msgs.size))
        lat = np.zeros(n, dtype=np.uint64)
        sigs = offs = None
        if keep_signatures:
            sizes = np.array([SIG_BY_ID[int(p)] for p in params], dtype=np.uint64)
            offs = np.zeros(n, dtype=np.uint64)
            if n > 1:
                np.cumsum(sizes[:-1], out=offs[1:])
            sigs = np.zeros(int(sizes.sum()), dtype=np.uint8)
        msgs = pool_msgs if pool_msgs is not None and pool_msgs.size else np.zeros(16, np.uint8)
        _check(load().hs_server_replay(self._h, n, _ptr(params), _ptr(keys), _ptr(pool_idx), _ptr(msgs),
                                       _ptr(pool_lens), int(pool_lens.shape[0]), _ptr(arrival_ns), _ptr(sigs),
                                       _ptr(offs), _ptr(lat), int(timeout_ms)))
        out = None
        if keep_signatures:
            out = [sigs[int(o):int(o) + SIG_BY_ID[int(p)]].tobytes() for o, p in zip(offs, params)]
        return lat, out

    def cancel(self, rid):
        """Drop a request that has not started; raises if it already runs or ran."""
        _check(load().hs_server_cancel(self._h, int(rid)))

    def inject_launch_failures(self, n):
        """Test hook: the next n batches fail as if their launch had failed."""
        _check(load().hs_server_inject_launch_failures(self._h, int(n)))

    def close(self):
        if getattr(self, "_h", None):
            load().hs_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


SIG_BY_ID = {0: 17088, 1: 35664, 2: 49856, 3: 1456, 4: 7856, 5: 16224, 6: 29792,
             7: 17088, 8: 35664, 9: 49856, 10: 7856, 11: 16224, 12: 29792, 13: 17088, 14: 35664, 15: 49856}


def hs_set_host_direct(on=True):
    """Write signatures straight into mapped page-locked host buffers (default on)."""
    _check(load().hs_set_host_direct(1 if on else 0))


def hs_set_tree_sharing(on=True):
    """Share repeated upper-layer XMSS trees within a batch (same bytes, less work)."""
    _check(load().hs_set_tree_sharing(1 if on else 0))
