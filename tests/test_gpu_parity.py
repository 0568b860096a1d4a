"""GPU parity: libhs.so signatures are byte-identical to the CPU oracle.

Tolerance: 0 differing bytes (integer hashing; exactly one valid signature
per key and message under deterministic signing).  Every call goes through
the C ABI via the thin binding; inputs come from the seeded generators in
paper_2512_23969_gb300.inputs.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu
THREADS = max(1, len(os.sched_getaffinity(0)))


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _oracle_keys(O, ps, seeds):
    out = [O.keygen(ps, bytes(s)) for s in seeds]
    return [p for p, _ in out], [s for _, s in out]


def _oracle_sign_many(O, ps, sks, wl, idxs):
    def one(i):
        return O.sign(ps, sks[int(wl.key_idx[i])], wl.message(i))
    with ThreadPoolExecutor(THREADS) as ex:
        return list(ex.map(one, idxs))


def _gpu_sign(hs, wl, sk_dev):
    import torch
    sigs = hs.hs_sign_batch(wl.params, sk_dev, _dev(wl.msgs), _dev(wl.lens), key_idx=_dev(wl.key_idx),
                            num_keys=wl.num_keys)
    torch.cuda.synchronize()
    rc, flags = hs.hs_check_status()
    assert rc == 0 and flags == 0
    return sigs.cpu().numpy()


def _first_diff(a, b):
    d = np.nonzero(np.frombuffer(a, np.uint8) != np.frombuffer(b, np.uint8))[0]
    return int(d[0]) if d.size else -1


def _compare(O, ps, got, want, idxs):
    for k, i in enumerate(idxs):
        g = got[i].tobytes()
        w = want[k]
        assert len(g) == len(w)
        assert g == w, "message %d: first differing byte %d of %d" % (i, _first_diff(g, w), len(w))


@pytest.mark.parametrize("ps", ["toy", "128f", "192f", "256f"])
def test_keygen_matches_oracle(hs, O, ps):
    wl = inputs.make(ps, 1, num_keys=5, seed=900 + len(ps))
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    opk, osk = _oracle_keys(O, ps, wl.seeds)
    assert pk.cpu().numpy().tobytes() == b"".join(opk)
    assert sk.cpu().numpy().tobytes() == b"".join(osk)


def test_toy_ragged_multikey(hs, O):
    """Toy set: 37 messages (ragged against every block size), lengths 0..300
    including empty, 3 keys in random order; every signature checked."""
    lens = np.random.default_rng(10).integers(0, 301, size=37)
    lens[0] = lens[5] = 0
    wl = inputs.make("toy", 37, num_keys=3, lengths=list(lens), seed=11, key_mode="random")
    pk, sk = hs.hs_keygen("toy", _dev(wl.seeds))
    got = _gpu_sign(hs, wl, sk)
    _, osk = _oracle_keys(O, "toy", wl.seeds)
    want = _oracle_sign_many(O, "toy", osk, wl, range(wl.count))
    _compare(O, "toy", got, want, range(wl.count))


def test_128f_config0_all_64(hs, O):
    """128f, one key from a seeded 48-byte seed, 64 x 32-byte messages: all
    64 signatures byte-compared with the oracle."""
    wl = inputs.config(0)
    assert wl.seeds.shape == (1, 48)
    pk, sk = hs.hs_keygen("128f", _dev(wl.seeds))
    got = _gpu_sign(hs, wl, sk)
    _, osk = _oracle_keys(O, "128f", wl.seeds)
    want = _oracle_sign_many(O, "128f", osk, wl, range(wl.count))
    _compare(O, "128f", got, want, range(wl.count))


@pytest.mark.parametrize("ps", ["192f", "256f"])
def test_192f_256f_variable_lengths(hs, O, ps):
    """192f / 256f: 12 messages of U{32..1024} bytes over 4 keys."""
    wl = inputs.make(ps, 12, num_keys=4, lengths=("uniform", 32, 1024), seed=5000 + int(ps[:3]))
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    got = _gpu_sign(hs, wl, sk)
    _, osk = _oracle_keys(O, ps, wl.seeds)
    want = _oracle_sign_many(O, ps, osk, wl, range(wl.count))
    _compare(O, ps, got, want, range(wl.count))


@pytest.mark.parametrize("ps", ["toy", "128f", "192f", "256f"])
def test_edge_lengths(hs, O, ps):
    """Message lengths at SHA block boundaries, empty messages, count = 1."""
    lens = [0, 1, 55, 56, 63, 64, 65, 111, 112, 127, 128, 129, 4096]
    if ps != "toy":
        lens = lens[:6] + [lens[-1]]
    wl = inputs.make(ps, len(lens), num_keys=1, lengths=lens, seed=77)
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    got = _gpu_sign(hs, wl, sk)
    _, osk = _oracle_keys(O, ps, wl.seeds)
    want = _oracle_sign_many(O, ps, osk, wl, range(wl.count))
    _compare(O, ps, got, want, range(wl.count))
    one = inputs.make(ps, 1, num_keys=1, lengths=[0], seed=78)
    got1 = _gpu_sign(hs, one, hs.hs_keygen(ps, _dev(one.seeds))[1])
    want1 = O.sign(ps, O.keygen(ps, bytes(one.seeds[0]))[1], b"")
    assert got1[0].tobytes() == want1


def test_128f_config1_full_size(hs, O):
    """128f, 16 keys, 16384 x 32-byte messages in one batched call (the
    benchmark's launch configuration): oracle parity on the seeded
    256-message subset, GPU verify accepts all 16384."""
    import torch
    wl = inputs.config(1)
    pk, sk = hs.hs_keygen("128f", _dev(wl.seeds))
    msgs, lens, kidx = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)
    sigs = hs.hs_sign_batch("128f", sk, msgs, lens, key_idx=kidx, num_keys=16)
    ok = hs.hs_verify_batch("128f", pk, msgs, lens, sigs, key_idx=kidx, num_keys=16)
    torch.cuda.synchronize()
    assert int(ok.sum().item()) == wl.count
    got = sigs.cpu().numpy()
    _, osk = _oracle_keys(O, "128f", wl.seeds)
    want = _oracle_sign_many(O, "128f", osk, wl, list(wl.subset))
    _compare(O, "128f", got, want, list(wl.subset))


@pytest.mark.parametrize("ps", ["toy", "128f", "192f", "256f"])
def test_gpu_verify_accepts_and_rejects(hs, O, ps):
    import torch
    wl = inputs.make(ps, 8, num_keys=2, lengths=("uniform", 0, 200), seed=31)
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    msgs, lens, kidx = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)
    sigs = hs.hs_sign_batch(ps, sk, msgs, lens, key_idx=kidx, num_keys=2)
    ok = hs.hs_verify_batch(ps, pk, msgs, lens, sigs, key_idx=kidx, num_keys=2)
    assert ok.cpu().numpy().tolist() == [1] * 8
    S = sigs.shape[1]
    rng = np.random.default_rng(5)
    bad = sigs.clone()
    flips = [int(rng.integers(0, S)) for _ in range(8)]
    flips[0] = 0                      # R
    flips[1] = S - 1                  # last auth node
    for m, pos in enumerate(flips):
        bad[m, pos] ^= 1 << int(rng.integers(0, 8))
    ok2 = hs.hs_verify_batch(ps, pk, msgs, lens, bad, key_idx=kidx, num_keys=2)
    assert ok2.cpu().numpy().tolist() == [0] * 8
    # oracle agrees on the tampered ones
    pkh = pk.cpu().numpy()
    for m in range(2):
        assert not O.verify(ps, pkh[int(wl.key_idx[m])].tobytes(), wl.message(m), bad[m].cpu().numpy().tobytes())
    # wrong key
    ok3 = hs.hs_verify_batch(ps, pk, msgs, lens, sigs, key_idx=_dev(1 - wl.key_idx), num_keys=2)
    assert ok3.cpu().numpy().tolist() == [0] * 8
    torch.cuda.synchronize()


def test_host_buffers_equal_device_path(hs, O):
    """The C ABI accepts host (numpy) buffers and stages them itself."""
    wl = inputs.make("toy", 9, num_keys=2, lengths=("uniform", 0, 90), seed=44)
    pk_h, sk_h = hs.hs_keygen("toy", wl.seeds)
    assert isinstance(sk_h, np.ndarray)
    sig_h = hs.hs_sign_batch("toy", sk_h, wl.msgs, wl.lens, key_idx=wl.key_idx, num_keys=2)
    sig_d = _gpu_sign(hs, wl, _dev(sk_h))
    assert sig_h.tobytes() == sig_d.tobytes()
    ok = hs.hs_verify_batch("toy", pk_h, wl.msgs, wl.lens, sig_h, key_idx=wl.key_idx, num_keys=2)
    assert ok.tolist() == [1] * 9


@pytest.mark.parametrize("direct", [True, False])
def test_pinned_host_signatures(hs, O, direct):
    """Page-locked host buffers: signatures written straight into the mapped
    host buffer (direct) or staged and copied back -- the same bytes as the
    device path, and as the oracle on a sample; sets of every hash family
    and tree width, ragged messages."""
    import torch
    hs.hs_set_host_direct(direct)
    try:
        for ps, count in (("128f", 300), ("192f", 40), ("256s", 3), ("shake-128f", 20)):
            wl = inputs.make(ps, count, num_keys=3, lengths=("uniform", 0, 400), seed=4400 + count,
                             key_mode="random")
            pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
            dev = _gpu_sign(hs, wl, sk)
            pinned = torch.zeros(count * hs.sig_bytes(ps), dtype=torch.uint8).pin_memory()
            out = hs.hs_sign_batch(ps, sk, torch.from_numpy(wl.msgs).pin_memory(),
                                   torch.from_numpy(wl.lens).pin_memory(),
                                   key_idx=torch.from_numpy(wl.key_idx).pin_memory(), sigs=pinned, num_keys=3)
            assert out.numpy().tobytes() == dev.tobytes(), ps
            i = count - 1
            osk = O.keygen(ps, bytes(wl.seeds[int(wl.key_idx[i])]))[1]
            assert pinned.numpy()[i * hs.sig_bytes(ps):(i + 1) * hs.sig_bytes(ps)].tobytes() == \
                O.sign(ps, osk, wl.message(i))
    finally:
        hs.hs_set_host_direct(True)


def test_key_index_out_of_range(hs, O):
    import torch
    wl = inputs.make("toy", 4, num_keys=2, lengths=16, seed=45)
    pk, sk = hs.hs_keygen("toy", _dev(wl.seeds))
    kidx = wl.key_idx.copy()
    kidx[2] = 7
    sigs = hs.hs_sign_batch("toy", sk, _dev(wl.msgs), _dev(wl.lens), key_idx=_dev(kidx), num_keys=2)
    rc, flags = hs.hs_check_status()
    assert rc == 5 and flags & (1 << 5)
    s = sigs.cpu().numpy()
    assert not s[2].any()
    _, osk = _oracle_keys(O, "toy", wl.seeds)
    assert s[0].tobytes() == O.sign("toy", osk[kidx[0]], wl.message(0))
    rc, flags = hs.hs_check_status()
    assert rc == 0 and flags == 0
    torch.cuda.synchronize()


def test_invalid_arguments(hs):
    import torch
    from paper_2512_23969_gb300.hs import HSError
    L = hs.load()
    assert L.hs_sign_batch(9, None, 1, None, None, None, 1, None, None) == 1
    lens = torch.zeros(1, dtype=torch.uint64, device="cuda")
    sigs = torch.empty(17088, dtype=torch.uint8, device="cuda")
    sk = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert L.hs_sign_batch(0, sk.data_ptr(), 0, None, None, lens.data_ptr(), 1, sigs.data_ptr(), None) == 1
    # NULL msgs with device lengths cannot be validated -> rejected
    assert L.hs_sign_batch(0, sk.data_ptr(), 1, None, None, lens.data_ptr(), 1, sigs.data_ptr(), None) == 1
    assert L.hs_sign_batch(0, sk.data_ptr(), 1, None, None, lens.data_ptr(), 0, sigs.data_ptr(), None) == 0
    with pytest.raises(HSError):
        hs.hs_sign_batch("128f", sk, None, lens, num_keys=0)


@pytest.mark.parametrize("ps", ["192f", "256f"])
def test_config2_full_size(hs, O, ps):
    """192f / 256f, 16 keys, 8192 messages of U{32..1024} bytes in one call
    (the bench's launch shape for these sets): oracle on the seeded
    32-message subset, GPU verify accepts all."""
    import torch
    wl = inputs.config(2, ps)
    assert wl.count == 8192 and wl.num_keys == 16
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    msgs, lens, kidx = _dev(wl.msgs), _dev(wl.lens), _dev(wl.key_idx)
    sigs = hs.hs_sign_batch(ps, sk, msgs, lens, key_idx=kidx, num_keys=16)
    ok = hs.hs_verify_batch(ps, pk, msgs, lens, sigs, key_idx=kidx, num_keys=16)
    torch.cuda.synchronize()
    assert int(ok.sum().item()) == wl.count
    got = sigs.cpu().numpy()
    _, osk = _oracle_keys(O, ps, wl.seeds)
    want = _oracle_sign_many(O, ps, osk, wl, list(wl.subset))
    _compare(O, ps, got, want, list(wl.subset))


def test_mixed_full_size_graph(hs, O):
    """The mixed recipe at full size -- 32768 messages 50/30/20 over
    128f/192f/256f, log-uniform 16 B - 64 KB, 64 keys -- in one graph launch:
    GPU verify accepts all, and 4 seeded messages per set equal the oracle."""
    import numpy as np
    import torch
    wls = inputs.mixed()
    assert sum(wl.count for wl in wls) == 32768
    jobs, pks = [], []
    for wl in wls:
        pk, sk = hs.hs_keygen(wl.params, _dev(wl.seeds))
        pks.append(pk)
        jobs.append({"params": wl.params, "sk": sk, "msgs": _dev(wl.msgs), "lens": _dev(wl.lens),
                     "key_idx": _dev(wl.key_idx), "num_keys": wl.num_keys,
                     "sigs": torch.empty(wl.count * hs.sig_bytes(wl.params), dtype=torch.uint8, device="cuda")})
    hs.hs_sign_mixed(jobs, use_graph=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(23969)
    for wl, j, pk in zip(wls, jobs, pks):
        sig = j["sigs"].view(wl.count, -1)
        ok = hs.hs_verify_batch(wl.params, pk, j["msgs"], j["lens"], sig, key_idx=j["key_idx"],
                                num_keys=wl.num_keys)
        assert int(ok.sum().item()) == wl.count, wl.params
        sample = sorted(rng.choice(wl.count, 4, replace=False).tolist())
        _, osk = _oracle_keys(O, wl.params, wl.seeds)
        want = _oracle_sign_many(O, wl.params, osk, wl, sample)
        _compare(O, wl.params, sig.cpu().numpy(), want, sample)


def test_out_of_memory_is_an_error_status(hs):
    """A batch whose scratch cannot be allocated (terabytes of chain
    checkpoints) returns HS_ENOMEM; nothing is launched and the library keeps
    working."""
    import torch
    count = 4 << 20                                    # 4 Mi 256f messages, all empty
    lens = torch.zeros(count, dtype=torch.uint64, device="cuda")
    msgs = torch.zeros(16, dtype=torch.uint8, device="cuda")
    wl = inputs.make("256f", 2, num_keys=1, lengths=8, seed=9)
    pk, sk = hs.hs_keygen("256f", _dev(wl.seeds))
    # never written: the call fails before any launch (1.2 TB of scratch).
    # The C ABI is called directly: the binding would reject this short
    # signature buffer before the library could report HS_ENOMEM.
    sigs = torch.empty(16, dtype=torch.uint8, device="cuda")
    L = hs.load()
    rc = L.hs_sign_batch(hs.PARAMS["256f"], sk.data_ptr(), 1, None, msgs.data_ptr(), lens.data_ptr(), count,
                         sigs.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == 2                                     # HS_ENOMEM
    assert b"out of memory" in L.hs_last_error() or b"alloc" in L.hs_last_error()
    with pytest.raises(ValueError):                    # the binding's own check
        hs.hs_sign_batch("256f", sk, msgs, lens, sigs=sigs, num_keys=1)
    torch.cuda.synchronize()
    ok = hs.hs_verify_batch("256f", pk, _dev(wl.msgs), _dev(wl.lens),
                            hs.hs_sign_batch("256f", sk, _dev(wl.msgs), _dev(wl.lens), num_keys=1), num_keys=1)
    assert ok.cpu().numpy().all()
