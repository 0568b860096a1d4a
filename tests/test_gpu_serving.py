"""Continuous-batching server: every request's signature equals the same
request signed alone (hs_sign_batch with one message) -- byte for byte --
while requests of all parameter sets arrive over time, batch together and
overlap on the device; admission respects the device-memory budget."""
import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _keys(hs, trace, nkeys):
    out = {}
    for ps in ("128f", "192f", "256f"):
        pk, sk = hs.hs_keygen(ps, _dev(trace["seeds"][ps][:nkeys]))
        out[ps] = sk
    return out


@pytest.mark.parametrize("budget_mb,inflight", [(1024, 4), (48, 2)])
def test_served_equals_alone(hs, O, budget_mb, inflight):
    import torch
    trace = inputs.serving_trace(rate=2000, seconds=0.15, keys=(6, 4, 3), pool=64, lengths=(16, 700), seed=99)
    n = len(trace["params"])
    assert n > 100
    keys = _keys(hs, trace, 6)
    with hs.Server(keys, max_inflight=inflight, max_batch=64, mem_budget=budget_mb << 20) as srv:
        lat, sigs = srv.replay(trace["params"], trace["keys"], trace["pool_idx"], trace["pool_msgs"],
                               trace["pool_lens"], trace["arrival_ns"], keep_signatures=True, timeout_ms=120000)
        st = srv.stats()
    assert st["status"] == 0 and st["completed"] == n
    assert st["max_device_bytes_in_use"] <= budget_mb << 20
    assert st["batches"] > 1
    if budget_mb >= 1024:
        assert st["max_inflight_batches"] >= 2          # batches overlapped on the device
    names = ("128f", "192f", "256f")
    offs = np.zeros(len(trace["pool_lens"]) + 1, dtype=np.int64)
    np.cumsum(trace["pool_lens"].astype(np.int64), out=offs[1:])
    for i in range(n):
        ps = names[int(trace["params"][i])]
        q = int(trace["pool_idx"][i])
        m = trace["pool_msgs"][offs[q]:offs[q + 1]]
        alone = hs.hs_sign_batch(ps, keys[ps], _dev(m if m.size else np.zeros(1, np.uint8)),
                                 _dev(np.array([m.size], np.uint64)),
                                 key_idx=_dev(np.array([trace["keys"][i]], np.uint32)),
                                 num_keys=int(keys[ps].shape[0]))       # 6 / 4 / 3 keys per set
        assert alone.cpu().numpy().tobytes() == sigs[i], i
        if i % 50 == 0:   # and the oracle on a sample
            osk = O.keygen(ps, bytes(trace["seeds"][ps][int(trace["keys"][i])]))[1]
            assert sigs[i] == O.sign(ps, osk, m.tobytes())
    assert (lat > 0).all()
    torch.cuda.synchronize()


def test_submit_wait_poll_and_errors(hs):
    wl = inputs.make("toy", 3, num_keys=2, lengths=20, seed=5)
    pk, sk = hs.hs_keygen("toy", _dev(wl.seeds))
    with hs.Server({"toy": sk}, max_inflight=2, max_batch=8, mem_budget=16 << 20) as srv:
        ids = [srv.submit("toy", int(wl.key_idx[i]), wl.message(i)) for i in range(3)]
        for rid, out in ids:
            srv.wait(rid, timeout_ms=60000)
        got = dict(srv.poll())
        assert set(got) == {rid for rid, _ in ids}
        ref = hs.hs_sign_batch("toy", sk, _dev(wl.msgs), _dev(wl.lens), key_idx=_dev(wl.key_idx), num_keys=2)
        for i, (rid, out) in enumerate(ids):
            assert out.tobytes() == ref[i].cpu().numpy().tobytes()
        with pytest.raises(hs.HSError) as e:
            srv.submit("toy", 9, b"x")
        assert e.value.code == 5
        with pytest.raises(hs.HSError):
            srv.submit("128f", 0, b"x")              # set not served: no keys
        with pytest.raises(hs.HSError):
            srv.wait(123456789, timeout_ms=10)
