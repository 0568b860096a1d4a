"""GPU parity of the robust SHA2 instantiation (robust-128f / 192f / 256f).

Keys and signatures must equal the CPU oracle's byte for byte (the
tolerance of every parity test here) in both forms of TREE_Sign (a thread
per chain for small batches, a thread per leaf), with WOTS+_Sign from chain
checkpoints and recomputed, from a keyset with cached top layers, and GPU
verify must accept them, reject a flipped byte and reject them under the
simple set.  FIPS 205 mode has no robust sets and refuses them.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu
THREADS = max(1, len(os.sched_getaffinity(0)))
SETS = ("robust-128f", "robust-192f", "robust-256f")


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _oracle(O, ps, wl, idxs):
    sks = [O.keygen(ps, bytes(s))[1] for s in wl.seeds]
    with ThreadPoolExecutor(THREADS) as ex:
        return list(ex.map(lambda i: O.sign(ps, sks[int(wl.key_idx[i])], wl.message(i)), idxs))


@pytest.mark.parametrize("ps", SETS)
def test_robust_keygen_and_sign_match_oracle(hs, O, ps):
    import torch
    from paper_2512_23969_gb300 import autotune
    wl = inputs.make(ps, 10, num_keys=3, lengths=("uniform", 0, 300), seed=910)
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    opk = [O.keygen(ps, bytes(s)) for s in wl.seeds]
    assert [bytes(x) for x in pk.cpu().numpy()] == [p for p, _ in opk]
    assert [bytes(x) for x in sk.cpu().numpy()] == [s for _, s in opk]
    want = _oracle(O, ps, wl, range(wl.count))
    msgs, lens, kidx = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)
    saved_split = autotune.get(ps, "tree_split_below")
    try:
        for split in (1 << 20, 0):               # chain-parallel, then per leaf
            autotune.set(ps, "tree_split_below", split)
            for ck in (2, 0):                      # WOTS+_Sign from checkpoints / recomputed
                hs.hs_set_chain_checkpoint(ck)
                got = hs.hs_sign_batch(ps, sk, msgs, lens, key_idx=kidx, num_keys=wl.num_keys).cpu().numpy()
                for i in range(wl.count):
                    assert got[i].tobytes() == want[i], (ps, split, ck, i)
    finally:
        hs.hs_set_chain_checkpoint(2)
        autotune.set(ps, "tree_split_below", saved_split)
    ok = hs.hs_verify_batch(ps, pk, msgs, lens, _dev(got), key_idx=kidx, num_keys=wl.num_keys)
    assert ok.cpu().numpy().tolist() == [1] * wl.count
    bad = got.copy()
    bad[3, 77] ^= 1
    ok = hs.hs_verify_batch(ps, pk, msgs, lens, _dev(bad), key_idx=kidx, num_keys=wl.num_keys)
    assert ok.cpu().numpy().tolist() == [1, 1, 1, 0] + [1] * (wl.count - 4)
    simple = ps[len("robust-"):]                 # same keys and sizes, other hashes: rejected
    ok = hs.hs_verify_batch(simple, pk, msgs, lens, _dev(got), key_idx=kidx, num_keys=wl.num_keys)
    assert not ok.cpu().numpy().any()
    torch.cuda.synchronize()


def test_robust_large_batch_sampled_and_keyset(hs, O):
    """A batch of the per-leaf size at robust-128f, sampled against the
    oracle; the same batch from a keyset with two cached layers is
    byte-identical."""
    ps = "robust-128f"
    wl = inputs.make(ps, 2048, num_keys=4, lengths=32, seed=911)
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    msgs, lens, kidx = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)
    got = hs.hs_sign_batch(ps, sk, msgs, lens, key_idx=kidx, num_keys=wl.num_keys).cpu().numpy()
    idxs = [0, 1, 777, 2046, 2047]
    for k, w in zip(idxs, _oracle(O, ps, wl, idxs)):
        assert got[k].tobytes() == w, k
    ok = hs.hs_verify_batch(ps, pk, msgs, lens, _dev(got), key_idx=kidx, num_keys=wl.num_keys)
    assert int(ok.sum().item()) == wl.count
    with hs.KeySet(ps, sk, cache_layers=2) as ks:
        from_cache = ks.sign(msgs, lens, key_idx=kidx).cpu().numpy()
    assert np.array_equal(from_cache, got)


def test_robust_sets_refused_in_fips_mode(hs):
    wl = inputs.make("robust-128f", 2, num_keys=1, lengths=8, seed=912)
    _, sk = hs.hs_keygen("robust-128f", _dev(wl.seeds))
    with pytest.raises(hs.HSError) as e:
        hs.hs_slh_sign_batch("robust-128f", sk, _dev(wl.msgs), _dev(wl.lens))
    assert e.value.code == 1
