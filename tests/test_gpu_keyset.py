"""Keysets (resident keys with their top hypertree layers prebuilt): every
signature is byte-identical to hs_sign_batch's with the same keys -- and to
the oracle on a sample -- for every parameter set, several cache depths,
chain checkpoint strides 0/2/4, both TREE_Sign forms (chain-parallel below
the split size, per-leaf above), ragged batches and bad key indices; the
server with a cache serves the same bytes."""
import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _batch(hs, ps, count, num_keys, seed, lengths=("uniform", 0, 300)):
    wl = inputs.make(ps, count, num_keys=num_keys, lengths=lengths, seed=seed, key_mode="random")
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    return wl, pk, sk


@pytest.mark.parametrize("ps,layers,count,num_keys", [
    ("toy", 1, 37, 3),
    ("128f", 1, 300, 5),
    ("128f", 3, 1000, 7),
    ("128f", 4, 8200, 16),          # per-leaf TREE_Sign (>= the split size)
    ("192f", 2, 500, 4),
    ("256f", 3, 260, 3),
    ("128s", 1, 70, 3),             # a 512-leaf top tree per key (wide-tree builder)
    ("256s", 2, 20, 2),             # 1 + 256 wide trees per key
    ("shake-128f", 2, 300, 4),
])
def test_keyset_equals_sign_batch(hs, O, ps, layers, count, num_keys):
    import torch
    wl, pk, sk = _batch(hs, ps, count, num_keys, 500 + layers)
    d_msgs, d_lens, d_kidx = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)
    ref = hs.hs_sign_batch(ps, sk, d_msgs, d_lens, key_idx=d_kidx, num_keys=num_keys).cpu().numpy()
    with hs.KeySet(ps, sk, cache_layers=layers) as ks:
        assert ks.nbytes > 0
        got = ks.sign(d_msgs, d_lens, key_idx=d_kidx).cpu().numpy()
        again = ks.sign(d_msgs, d_lens, key_idx=d_kidx).cpu().numpy()
    assert np.array_equal(got, ref)
    assert np.array_equal(again, ref)
    ok = hs.hs_verify_batch(ps, pk, d_msgs, d_lens, torch.from_numpy(got).cuda(), key_idx=d_kidx,
                            num_keys=num_keys).cpu().numpy()
    assert ok.all()
    for i in np.random.default_rng(layers).choice(count, 2, replace=False):
        osk = O.keygen(ps, bytes(wl.seeds[int(wl.key_idx[i])]))[1]
        assert got[i].tobytes() == O.sign(ps, osk, wl.message(int(i)))


@pytest.mark.parametrize("stride", [0, 4])
def test_keyset_checkpoint_strides(hs, stride):
    wl, pk, sk = _batch(hs, "128f", 200, 4, 77)
    d_msgs, d_lens, d_kidx = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)
    ref = hs.hs_sign_batch("128f", sk, d_msgs, d_lens, key_idx=d_kidx, num_keys=4).cpu().numpy()
    hs.hs_set_chain_checkpoint(stride)
    try:
        ks = hs.KeySet("128f", sk, cache_layers=3)
    finally:
        hs.hs_set_chain_checkpoint(2)
    with ks:
        got = ks.sign(d_msgs, d_lens, key_idx=d_kidx).cpu().numpy()   # the keyset keeps its own stride
    assert np.array_equal(got, ref)


def test_keyset_host_buffers_empty_and_bad_keys(hs):
    wl, pk, sk = _batch(hs, "toy", 20, 2, 78)
    ref = hs.hs_sign_batch("toy", sk, _dev(wl.msgs), _dev(wl.lens), key_idx=_dev(wl.key_idx),
                           num_keys=2).cpu().numpy()
    with hs.KeySet("toy", sk.cpu().numpy(), cache_layers=1) as ks:
        got = ks.sign(wl.msgs, wl.lens, key_idx=wl.key_idx)          # host in, host out
        assert np.array_equal(np.asarray(got), ref)
        empty = ks.sign(np.zeros(0, np.uint8), np.zeros(0, np.uint64))
        assert empty.shape[0] == 0
        bad = wl.key_idx.copy()
        bad[3] = 9
        out = ks.sign(_dev(wl.msgs), _dev(wl.lens), key_idx=_dev(bad))
        rc, flags = hs.hs_check_status()
        assert rc == 5 and flags & (1 << 5)
        out = out.cpu().numpy()
        keep = np.arange(20) != 3
        assert np.array_equal(out[keep], ref[keep])                   # the others are unaffected
    with pytest.raises(hs.HSError):
        hs.KeySet("toy", sk, cache_layers=2)                          # d - 1 = 1 at most
    with pytest.raises(hs.HSError):
        hs.KeySet("128f", sk[:0], cache_layers=1)                      # no keys


def test_server_with_cache_serves_same_bytes(hs):
    wl, pk, sk = _batch(hs, "128f", 96, 6, 79)
    ref = hs.hs_sign_batch("128f", sk, _dev(wl.msgs), _dev(wl.lens), key_idx=_dev(wl.key_idx),
                           num_keys=6).cpu().numpy()
    with hs.Server({"128f": sk}, max_inflight=3, max_batch=16, mem_budget=256 << 20, cache_layers=3) as srv:
        reqs = [srv.submit("128f", int(wl.key_idx[i]), wl.message(i)) for i in range(96)]
        for i, (rid, out) in enumerate(reqs):
            srv.wait(rid, timeout_ms=60000)
            assert out.tobytes() == ref[i].tobytes(), i
        assert srv.stats()["status"] == 0
