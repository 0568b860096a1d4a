"""hs_sign_batch_noalloc: signing for callers that cannot allocate device memory.

Some callers reserve all their device memory at start-up or embed this
library without letting it allocate; they use the no-allocation entry point,
which works in a fixed device buffer inside the library.  This test calls it
through the C ABI twice in a row (different parameter sets, sizes and keys,
so the second call runs on whatever the first left in the shared buffer) and
requires its signatures to equal hs_sign_batch's byte for byte, the
tolerance every parity test here uses.  It also checks that a batch too big
for the buffer is refused with a clear message.

The file name makes pytest collect it last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _noalloc(L, pid, sk, num_keys, kidx, msgs, lens, count, sigs, stream):
    return L.hs_sign_batch_noalloc(pid, sk.data_ptr(), num_keys, kidx.data_ptr(), msgs.data_ptr(),
                                   lens.data_ptr(), count, sigs.data_ptr(), stream)


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
        assert rc == 0, L.hs_last_error()
        torch.cuda.synchronize()
        assert torch.equal(sigs.view(wl.count, -1), want), ps


def test_noalloc_refuses_oversized_batch(hs):
    import torch
    L = hs.load()
    count = 20000                                  # > 8 MiB of 128f scratch
    sk = torch.zeros(64, dtype=torch.uint8, device="cuda")
    lens = torch.zeros(count, dtype=torch.uint64, device="cuda")
    msgs = torch.zeros(16, dtype=torch.uint8, device="cuda")
    kidx = torch.zeros(count, dtype=torch.int32, device="cuda")
    sigs = torch.empty(16, dtype=torch.uint8, device="cuda")
    rc = _noalloc(L, 0, sk, 1, kidx, msgs, lens, count, sigs, torch.cuda.current_stream().cuda_stream)
    assert rc == 1
    assert b"bytes of scratch" in L.hs_last_error()
