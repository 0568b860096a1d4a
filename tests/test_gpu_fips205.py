"""FIPS 205 (SLH-DSA) mode on the GPU: hs_slh_sign_batch is byte-identical
to the oracle's pure SLH-DSA signing for every set, context strings of 0, 1
and 255 bytes, ragged and empty messages, and the internal functions
(ctx=None); hs_slh_verify_batch accepts them and rejects another context."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _oracle_all(O, fn, items):
    with ThreadPoolExecutor(16) as ex:
        return list(ex.map(fn, items))


@pytest.mark.parametrize("ps,count", [("toy", 40), ("128f", 8), ("192f", 3), ("256f", 2)])
@pytest.mark.parametrize("ctx", [b"", b"\x07", bytes(range(255)), None], ids=["ctx0", "ctx1", "ctx255", "internal"])
def test_slh_sign_equals_oracle(hs, O, ps, count, ctx):
    wl = inputs.make(ps, count, num_keys=2, lengths=("uniform", 0, 300), seed=205 + count, key_mode="random")
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    d_msgs, d_lens, d_kidx = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)
    sigs = hs.hs_slh_sign_batch(ps, sk, d_msgs, d_lens, ctx=ctx, key_idx=d_kidx, num_keys=2)
    got = sigs.cpu().numpy()
    osks = [O.keygen(ps, bytes(s))[1] for s in wl.seeds]

    def ref(i):
        m, k = wl.message(i), osks[int(wl.key_idx[i])]
        return O.sign("slh-" + ps, k, m) if ctx is None else O.slh_sign(ps, k, ctx, m)

    want = _oracle_all(O, ref, range(count))
    for i in range(count):
        assert got[i].tobytes() == want[i], i
    ok = hs.hs_slh_verify_batch(ps, pk, d_msgs, d_lens, sigs, ctx=ctx, key_idx=d_kidx, num_keys=2).cpu().numpy()
    assert ok.all()
    other = b"x" if ctx is None else ctx + b"!" if len(ctx) < 255 else ctx[:-1]
    bad = hs.hs_slh_verify_batch(ps, pk, d_msgs, d_lens, sigs, ctx=other, key_idx=d_kidx, num_keys=2).cpu().numpy()
    assert not bad.any()


def test_slh_full_size_launch_sampled(hs, O):
    """The per-leaf TREE_Sign launch shape (8192 messages) against the oracle on a sample."""
    wl = inputs.make("128f", 8192, num_keys=16, lengths=32, seed=2051)
    pk, sk = hs.hs_keygen("128f", _dev(wl.seeds))
    d_msgs, d_lens, d_kidx = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)
    ctx = b"batch-context"
    sigs = hs.hs_slh_sign_batch("128f", sk, d_msgs, d_lens, ctx=ctx, key_idx=d_kidx, num_keys=16)
    ok = hs.hs_slh_verify_batch("128f", pk, d_msgs, d_lens, sigs, ctx=ctx, key_idx=d_kidx, num_keys=16)
    assert int(ok.sum().item()) == 8192
    plain = hs.hs_verify_batch("128f", pk, d_msgs, d_lens, sigs, key_idx=d_kidx, num_keys=16)
    assert int(plain.sum().item()) == 0                      # not round-3.1 signatures
    got = sigs.cpu().numpy()
    sample = np.random.default_rng(7).choice(8192, 6, replace=False)
    osks = {}

    def ref(i):
        k = int(wl.key_idx[i])
        if k not in osks:
            osks[k] = O.keygen("128f", bytes(wl.seeds[k]))[1]
        return O.slh_sign("128f", osks[k], ctx, wl.message(int(i)))

    want = [ref(i) for i in sample]
    for i, w in zip(sample, want):
        assert got[i].tobytes() == w, int(i)


def test_slh_errors(hs):
    wl = inputs.make("toy", 4, num_keys=1, lengths=8, seed=3)
    pk, sk = hs.hs_keygen("toy", _dev(wl.seeds))
    with pytest.raises(hs.HSError) as e:
        hs.hs_slh_sign_batch("toy", sk, _dev(wl.msgs), _dev(wl.lens), ctx=bytes(256))
    assert e.value.code == 1
    empty = hs.hs_slh_sign_batch("toy", sk, np.zeros(0, np.uint8), np.zeros(0, np.uint64), ctx=b"c")
    assert empty.shape[0] == 0
