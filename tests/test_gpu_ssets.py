"""The small-signature sets (128s / 192s / 256s) on the GPU: keys and
signatures byte-identical to the oracle for both TREE_Sign forms (the
chain-parallel form below the split size and one thread per leaf above
it), every compiled FORS lane count, chain checkpoint strides 0/2/4, the
FIPS 205 mode, mixed batches and the server; GPU verify accepts them and
rejects tampering."""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2512_23969_gb300 import autotune, inputs

pytestmark = pytest.mark.gpu
SETS = ("128s", "192s", "256s")


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _pool(fn, items):
    with ThreadPoolExecutor(16) as ex:
        return list(ex.map(fn, items))


def _setup(hs, ps, count, seed, num_keys=2):
    wl = inputs.make(ps, count, num_keys=num_keys, lengths=("uniform", 0, 200), seed=seed, key_mode="random")
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    return wl, pk, sk


@pytest.mark.parametrize("ps", SETS)
def test_keygen_equals_oracle(hs, O, ps):
    wl, pk, sk = _setup(hs, ps, 1, 11, num_keys=3)
    want = _pool(lambda s: O.keygen(ps, bytes(s)), list(wl.seeds))
    for i, (opk, osk) in enumerate(want):
        assert pk[i].cpu().numpy().tobytes() == opk
        assert sk[i].cpu().numpy().tobytes() == osk


@pytest.mark.parametrize("ps", SETS)
def test_small_batch_equals_oracle(hs, O, ps):
    """5 messages: the chain-parallel TREE_Sign form."""
    import torch
    wl, pk, sk = _setup(hs, ps, 5, 12)
    d = [_dev(x) for x in (wl.msgs, wl.lens, wl.key_idx)]
    got = hs.hs_sign_batch(ps, sk, d[0], d[1], key_idx=d[2], num_keys=2).cpu().numpy()
    osks = [O.keygen(ps, bytes(s))[1] for s in wl.seeds]
    want = _pool(lambda i: O.sign(ps, osks[int(wl.key_idx[i])], wl.message(i)), range(5))
    for i in range(5):
        assert got[i].tobytes() == want[i], i
    ok = hs.hs_verify_batch(ps, pk, d[0], d[1], torch.from_numpy(got).cuda(), key_idx=d[2], num_keys=2)
    assert ok.cpu().numpy().all()
    bad = got.copy()
    bad[0, 100] ^= 1                                    # a FORS byte
    bad[1, -5] ^= 1                                     # the top layer's last auth node
    ok = hs.hs_verify_batch(ps, pk, d[0], d[1], torch.from_numpy(bad).cuda(), key_idx=d[2], num_keys=2)
    assert ok.cpu().numpy().tolist() == [0, 0, 1, 1, 1]


@pytest.mark.parametrize("ps", SETS)
def test_forms_lanes_and_strides_agree(hs, O, ps):
    """80 messages: per-leaf TREE_Sign (default) equals the chain-parallel
    form, every FORS lane count and every checkpoint stride; a sample is
    checked against the oracle and all pass GPU verify."""
    wl, pk, sk = _setup(hs, ps, 80, 13, num_keys=3)
    d = [_dev(x) for x in (wl.msgs, wl.lens, wl.key_idx)]
    sign = lambda: hs.hs_sign_batch(ps, sk, d[0], d[1], key_idx=d[2], num_keys=3).cpu().numpy()
    ref = sign()
    split0, lanes0 = autotune.get(ps, "tree_split_below"), autotune.get(ps, "fors_lanes")
    try:
        autotune.set(ps, "tree_split_below", 1 << 30)
        assert np.array_equal(sign(), ref)
        autotune.set(ps, "tree_split_below", split0)
        for v in autotune.options(ps, "fors_lanes"):
            autotune.set(ps, "fors_lanes", v)
            assert np.array_equal(sign(), ref), v
        autotune.set(ps, "fors_lanes", lanes0)
        for stride in (0, 4):
            hs.hs_set_chain_checkpoint(stride)
            assert np.array_equal(sign(), ref), stride
    finally:
        hs.hs_set_chain_checkpoint(2)
        autotune.set(ps, "tree_split_below", split0)
        autotune.set(ps, "fors_lanes", lanes0)
    import torch
    ok = hs.hs_verify_batch(ps, pk, d[0], d[1], torch.from_numpy(ref).cuda(), key_idx=d[2], num_keys=3)
    assert ok.cpu().numpy().all()
    osks = [O.keygen(ps, bytes(s))[1] for s in wl.seeds]
    sample = [0, 41, 79]
    want = _pool(lambda i: O.sign(ps, osks[int(wl.key_idx[i])], wl.message(i)), sample)
    for i, w in zip(sample, want):
        assert ref[i].tobytes() == w, i


def test_fips205_mode_128s(hs, O):
    wl, pk, sk = _setup(hs, "128s", 3, 14)
    d = [_dev(x) for x in (wl.msgs, wl.lens, wl.key_idx)]
    got = hs.hs_slh_sign_batch("128s", sk, d[0], d[1], ctx=b"ctx", key_idx=d[2], num_keys=2)
    osks = [O.keygen("128s", bytes(s))[1] for s in wl.seeds]
    want = _pool(lambda i: O.slh_sign("128s", osks[int(wl.key_idx[i])], b"ctx", wl.message(i)), range(3))
    g = got.cpu().numpy()
    for i in range(3):
        assert g[i].tobytes() == want[i], i
    ok = hs.hs_slh_verify_batch("128s", pk, d[0], d[1], got, ctx=b"ctx", key_idx=d[2], num_keys=2)
    assert ok.cpu().numpy().all()


def test_mixed_and_server_with_s_sets(hs):
    jobs, refs = [], []
    for ps, count, seed in (("128s", 7, 15), ("128f", 20, 16), ("256s", 3, 17)):
        wl, pk, sk = _setup(hs, ps, count, seed)
        d = [_dev(x) for x in (wl.msgs, wl.lens, wl.key_idx)]
        refs.append((ps, wl, sk, hs.hs_sign_batch(ps, sk, d[0], d[1], key_idx=d[2], num_keys=2).cpu().numpy()))
        import torch
        jobs.append({"params": ps, "sk": sk, "msgs": d[0], "lens": d[1], "key_idx": d[2], "num_keys": 2,
                     "sigs": torch.empty(count * hs.sig_bytes(ps), dtype=torch.uint8, device="cuda")})
    hs.hs_sign_mixed(jobs, use_graph=True)
    for j, (ps, wl, sk, ref) in zip(jobs, refs):
        assert np.array_equal(j["sigs"].view(wl.count, -1).cpu().numpy(), ref), ps
    ps, wl, sk, ref = refs[0]
    with hs.Server({"128s": sk, "128f": refs[1][2]}, max_inflight=2, max_batch=4, mem_budget=512 << 20,
                   cache_layers=2) as srv:
        reqs = [srv.submit("128s", int(wl.key_idx[i]), wl.message(i)) for i in range(wl.count)]
        for i, (rid, out) in enumerate(reqs):
            srv.wait(rid, timeout_ms=120000)
            assert out.tobytes() == ref[i].tobytes(), i
