"""The SHAKE instantiation on the GPU: keys and signatures byte-identical
to the oracle (whose SHAKE256 is pinned against hashlib) for the f and s
sets, messages across the 136-byte rate boundary, both TREE_Sign forms,
the FIPS 205 mode and GPU verify."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2512_23969_gb300 import autotune, inputs

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _pool(fn, items):
    with ThreadPoolExecutor(16) as ex:
        return list(ex.map(fn, items))


@pytest.mark.parametrize("ps,count", [("shake-128f", 6), ("shake-192f", 3), ("shake-256f", 3), ("shake-128s", 2),
                                      ("shake-192s", 1), ("shake-256s", 1)])
def test_keys_and_signatures_equal_oracle(hs, O, ps, count):
    import torch
    wl = inputs.make(ps, count, num_keys=2, lengths=("uniform", 0, 600), seed=700 + count, key_mode="random")
    wl.lens[0] = 0                                      # an empty message
    wl = inputs.make(ps, count, num_keys=2, lengths=wl.lens.tolist(), seed=700 + count, key_mode="random")
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    okeys = _pool(lambda s: O.keygen(ps, bytes(s)), list(wl.seeds))
    for i, (opk, osk) in enumerate(okeys):
        assert pk[i].cpu().numpy().tobytes() == opk and sk[i].cpu().numpy().tobytes() == osk
    d = [_dev(x) for x in (wl.msgs, wl.lens, wl.key_idx)]
    got = hs.hs_sign_batch(ps, sk, d[0], d[1], key_idx=d[2], num_keys=2).cpu().numpy()
    want = _pool(lambda i: O.sign(ps, okeys[int(wl.key_idx[i])][1], wl.message(i)), range(count))
    for i in range(count):
        assert got[i].tobytes() == want[i], i
    ok = hs.hs_verify_batch(ps, pk, d[0], d[1], torch.from_numpy(got).cuda(), key_idx=d[2], num_keys=2)
    assert ok.cpu().numpy().all()
    bad = got.copy()
    bad[:, 40] ^= 2
    ok = hs.hs_verify_batch(ps, pk, d[0], d[1], torch.from_numpy(bad).cuda(), key_idx=d[2], num_keys=2)
    assert not ok.cpu().numpy().any()


def test_tree_forms_agree_and_fips_mode(hs, O):
    ps = "shake-128f"
    wl = inputs.make(ps, 300, num_keys=4, lengths=("uniform", 1, 300), seed=705, key_mode="random")
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    d = [_dev(x) for x in (wl.msgs, wl.lens, wl.key_idx)]
    ref = hs.hs_sign_batch(ps, sk, d[0], d[1], key_idx=d[2], num_keys=4).cpu().numpy()   # chain-parallel form
    split0 = autotune.get(ps, "tree_split_below")
    try:
        autotune.set(ps, "tree_split_below", 0)                                          # one thread per leaf
        assert np.array_equal(hs.hs_sign_batch(ps, sk, d[0], d[1], key_idx=d[2], num_keys=4).cpu().numpy(), ref)
    finally:
        autotune.set(ps, "tree_split_below", split0)
    osk = {k: O.keygen(ps, bytes(wl.seeds[k]))[1] for k in range(4)}
    for i in (0, 150, 299):
        assert ref[i].tobytes() == O.sign(ps, osk[int(wl.key_idx[i])], wl.message(i)), i
    slh = hs.hs_slh_sign_batch(ps, sk, d[0], d[1], ctx=b"shake-ctx", key_idx=d[2], num_keys=4)
    g = slh.cpu().numpy()
    for i in (0, 7):
        assert g[i].tobytes() == O.slh_sign(ps, osk[int(wl.key_idx[i])], b"shake-ctx", wl.message(i)), i
    ok = hs.hs_slh_verify_batch(ps, pk, d[0], d[1], slh, ctx=b"shake-ctx", key_idx=d[2], num_keys=4)
    assert ok.cpu().numpy().all()
