"""hs_sign_batch_noalloc: signing for callers that cannot allocate device memory.

Some callers reserve all their device memory at start-up or embed this
library without letting it allocate; they use the no-allocation entry point,
which works in a fixed device buffer inside the library.  These tests call it
through the C ABI and require its signatures to equal, byte for byte (the
tolerance every parity test here uses):
  * the CPU oracle's, for both forms of TREE_Sign it can run -- chain-parallel
    (a small batch whose chain ends fit the buffer) and one thread per leaf
    (a batch too large for the chain ends) -- at 128f, 192f without key
    indices, and the wide-tree set 128s;
  * hs_sign_batch's, on two calls in a row (different sets, sizes and keys,
    so the second call runs on whatever the first left in the shared buffer).
They also check that an oversized batch and a host buffer are refused with a
clear message, and that an out-of-range key index is reported by
hs_check_status once the device is set up.

The file name makes pytest collect it last.
"""
import ctypes as C
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu
THREADS = max(1, len(os.sched_getaffinity(0)))
SCRATCH = 8 << 20                                  # HS_NOALLOC_SCRATCH_BYTES


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _noalloc(L, pid, sk, num_keys, kidx, msgs, lens, count, sigs, stream):
    return L.hs_sign_batch_noalloc(pid, sk.data_ptr(), num_keys, None if kidx is None else kidx.data_ptr(),
                                   msgs.data_ptr(), lens.data_ptr(), count, sigs.data_ptr(), stream)


def _sign_noalloc(hs, ps, wl, sk, with_kidx=True):
    import torch
    L = hs.load()
    msgs, lens = _dev(wl.msgs), _dev(wl.lens)
    kidx = _dev(wl.key_idx) if with_kidx else None
    sigs = torch.full((wl.count * hs.sig_bytes(ps),), 0xA5, dtype=torch.uint8, device="cuda")
    rc = _noalloc(L, hs.PARAMS[ps], sk, wl.num_keys, kidx, msgs, lens, wl.count, sigs,
                  torch.cuda.current_stream().cuda_stream)
    assert rc == 0, hs.last_error()
    torch.cuda.synchronize()
    return sigs.view(wl.count, -1).cpu().numpy()


def _oracle(O, ps, wl, idxs, with_kidx=True):
    sks = [O.keygen(ps, bytes(s))[1] for s in wl.seeds]

    def one(i):
        return O.sign(ps, sks[int(wl.key_idx[i]) if with_kidx else 0], wl.message(i))
    with ThreadPoolExecutor(THREADS) as ex:
        return list(ex.map(one, idxs))


def _per_msg_split_bytes(ps):
    """Chain-end bytes per message of the chain-parallel TREE_Sign form."""
    n, d, hp, length = {"128f": (16, 22, 3, 35), "192f": (24, 22, 3, 51), "128s": (16, 7, 9, 35)}[ps]
    return d * (1 << hp) * length * n


@pytest.mark.parametrize("ps,count,keys,with_kidx,form", [
    ("128f", 40, 3, True, "chain-parallel"),
    ("128f", 300, 4, True, "per-leaf"),
    ("192f", 8, 1, False, "chain-parallel"),
    ("128s", 3, 2, True, "chain-parallel"),
    ("128s", 5, 2, True, "per-leaf"),
])
def test_noalloc_matches_oracle(hs, O, ps, count, keys, with_kidx, form):
    # which form the entry point takes follows from the buffer size: the
    # chain ends of the whole batch either fit in it or they do not
    fits = count * _per_msg_split_bytes(ps) < SCRATCH - (1 << 20)
    assert fits == (form == "chain-parallel")
    wl = inputs.make(ps, count, num_keys=keys, lengths=("uniform", 0, 300), seed=610 + count)
    if not with_kidx:
        wl.key_idx[:] = 0
    _, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    got = _sign_noalloc(hs, ps, wl, sk, with_kidx)
    idxs = list(range(count)) if count <= 40 else [0, 1, 2, count // 3, count // 2, count - 2, count - 1]
    want = _oracle(O, ps, wl, idxs, with_kidx)
    for k, i in enumerate(idxs):
        assert got[i].tobytes() == want[k], "%s %s: message %d differs from the oracle" % (ps, form, i)
    if count > 40:                                   # the rest against the pooled-scratch entry point
        ref = hs.hs_sign_batch(ps, sk, _dev(wl.msgs), _dev(wl.lens), key_idx=_dev(wl.key_idx),
                               num_keys=wl.num_keys).cpu().numpy()
        assert np.array_equal(got, ref)


def test_noalloc_matches_sign_batch_on_two_calls(hs):
    import torch
    L = hs.load()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [("128f", 0, inputs.make("128f", 40, num_keys=3, lengths=("uniform", 0, 300), seed=601)),
             ("256f", 2, inputs.make("256f", 9, num_keys=2, lengths=("uniform", 1, 200), seed=602))]
    for ps, pid, wl in cases:
        pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
        msgs, lens, kidx = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)
        want = hs.hs_sign_batch(ps, sk, msgs, lens, key_idx=kidx, num_keys=wl.num_keys)
        sigs = torch.full((wl.count * hs.sig_bytes(ps),), 0xA5, dtype=torch.uint8, device="cuda")
        rc = _noalloc(L, pid, sk, wl.num_keys, kidx, msgs, lens, wl.count, sigs, stream)
        assert rc == 0, hs.last_error()
        torch.cuda.synchronize()
        assert torch.equal(sigs.view(wl.count, -1), want), ps


def test_noalloc_refuses_oversized_batch_and_host_buffers(hs):
    import torch
    L = hs.load()
    stream = torch.cuda.current_stream().cuda_stream
    count = 20000                                  # > 8 MiB of 128f scratch
    sk = torch.zeros(64, dtype=torch.uint8, device="cuda")
    lens = torch.zeros(count, dtype=torch.uint64, device="cuda")
    msgs = torch.zeros(16, dtype=torch.uint8, device="cuda")
    kidx = torch.zeros(count, dtype=torch.int32, device="cuda")
    sigs = torch.empty(16, dtype=torch.uint8, device="cuda")
    assert _noalloc(L, 0, sk, 1, kidx, msgs, lens, count, sigs, stream) == 1
    assert "bytes of scratch" in hs.last_error()
    host_sigs = torch.empty(17088, dtype=torch.uint8).pin_memory()
    assert _noalloc(L, 0, sk, 1, kidx, msgs, lens, 1, host_sigs, stream) == 1
    assert "memory of the current device" in hs.last_error()


def test_noalloc_reports_bad_key_index(hs):
    wl = inputs.make("128f", 4, num_keys=2, lengths=("uniform", 1, 64), seed=640)
    _, sk = hs.hs_keygen("128f", _dev(wl.seeds))      # sets the device up
    hs.hs_check_status()                               # start from a clear status word
    wl.key_idx[2] = 7                                  # only 2 keys
    got = _sign_noalloc(hs, "128f", wl, sk)
    rc, flags = hs.hs_check_status()
    assert rc == 5 and flags & (1 << 5)                # HS_EKEY
    assert not got[2].any()
    ref = hs.hs_sign_batch("128f", sk, _dev(wl.msgs), _dev(wl.lens), key_idx=_dev(wl.key_idx),
                           num_keys=2).cpu().numpy()
    hs.hs_check_status()
    for i in (0, 1, 3):
        assert got[i].tobytes() == ref[i].tobytes()
