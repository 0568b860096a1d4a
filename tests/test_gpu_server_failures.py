"""Server failure handling without a GPU fault: a batch whose launch fails
(simulated on the host -- nothing of it reaches the GPU) completes its
requests with HS_ECUDA and the server keeps serving byte-exact signatures;
requests still waiting for a batch can be cancelled."""
import numpy as np
import pytest

from paper_2512_23969_gb300 import inputs

pytestmark = pytest.mark.gpu

HS_EINVAL, HS_ECUDA, HS_ECANCELED, HS_EBUDGET = 1, 3, 6, 7


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _setup(hs, ps, count, num_keys, seed):
    wl = inputs.make(ps, count, num_keys=num_keys, lengths=("uniform", 1, 200), seed=seed)
    pk, sk = hs.hs_keygen(ps, _dev(wl.seeds))
    ref = hs.hs_sign_batch(ps, sk, _dev(wl.msgs), _dev(wl.lens), key_idx=_dev(wl.key_idx),
                           num_keys=num_keys).cpu().numpy()
    return wl, sk, ref


def _wait_status(hs, srv, rid):
    try:
        srv.wait(rid, timeout_ms=60000)
        return 0
    except hs.HSError as e:
        return e.code


def test_injected_launch_failure_then_recovery(hs):
    wl, sk, ref = _setup(hs, "toy", 64, 3, 71)
    with hs.Server({"toy": sk}, max_inflight=2, max_batch=8, mem_budget=32 << 20) as srv:
        srv.inject_launch_failures(2)
        reqs = [srv.submit("toy", int(wl.key_idx[i]), wl.message(i)) for i in range(len(wl.lens))]
        codes = [_wait_status(hs, srv, rid) for rid, _ in reqs]
        st = srv.stats()
        failed = [i for i, c in enumerate(codes) if c]
        assert all(codes[i] == HS_ECUDA for i in failed)
        assert 2 <= len(failed) <= 16                       # exactly two batches of at most 8 failed
        assert st["failed"] == len(failed) and st["completed"] == len(reqs)
        assert st["status"] == 0                            # a failed launch is not a dead server
        for i, (rid, out) in enumerate(reqs):
            if not codes[i]:
                assert out.tobytes() == ref[i].tobytes(), i
        polled = srv.poll(with_status=True)
        assert {r for r, _, c in polled if c == HS_ECUDA} == {reqs[i][0] for i in failed}
        # the server keeps working: every request after the failures succeeds, byte-exact
        again = [srv.submit("toy", int(wl.key_idx[i]), wl.message(i)) for i in range(len(wl.lens))]
        for i, (rid, out) in enumerate(again):
            srv.wait(rid, timeout_ms=60000)
            assert out.tobytes() == ref[i].tobytes(), i
        assert srv.stats()["failed"] == len(failed)


def test_replay_reports_failed_batches(hs):
    wl, sk, ref = _setup(hs, "toy", 32, 2, 72)
    trace_params = np.full(32, 3, np.uint8)
    arrival = np.arange(32, dtype=np.uint64) * 1000
    with hs.Server({"toy": sk}, max_inflight=1, max_batch=4, mem_budget=32 << 20) as srv:
        srv.inject_launch_failures(1)
        with pytest.raises(hs.HSError) as e:
            srv.replay(trace_params, wl.key_idx, np.arange(32, dtype=np.uint32), wl.msgs, wl.lens, arrival,
                       keep_signatures=True, timeout_ms=60000)
        assert e.value.code == HS_ECUDA
        lat, sigs = srv.replay(trace_params, wl.key_idx, np.arange(32, dtype=np.uint32), wl.msgs, wl.lens,
                               arrival, keep_signatures=True, timeout_ms=60000)
        assert all(sigs[i] == ref[i].tobytes() for i in range(32))
        assert srv.stats()["status"] == 0


def test_cancel_pending_requests(hs):
    wl, sk, ref = _setup(hs, "128f", 16, 4, 73)
    n = 1200
    with hs.Server({"128f": sk}, max_inflight=1, max_batch=16, mem_budget=256 << 20) as srv:
        reqs = [srv.submit("128f", int(wl.key_idx[i % 16]), wl.message(i % 16)) for i in range(n)]
        # the tail of a burst this deep is still queued behind one small batch at a time
        cancelled = set()
        for i in range(n - 1, n - 201, -1):
            try:
                srv.cancel(reqs[i][0])
                cancelled.add(i)
            except hs.HSError as e:
                assert e.code == 1                          # it had already started: it completes
        assert len(cancelled) > 0
        for i, (rid, out) in enumerate(reqs):
            code = _wait_status(hs, srv, rid)
            if i in cancelled:
                assert code == HS_ECANCELED
            else:
                assert code == 0 and out.tobytes() == ref[i % 16].tobytes(), i
        st = srv.stats()
        assert st["cancelled"] == len(cancelled) and st["completed"] == n and st["failed"] == 0
        done = srv.poll(max_n=n + 8, with_status=True)
        assert sorted(r for r, _, c in done if c == HS_ECANCELED) == sorted(reqs[i][0] for i in cancelled)
        with pytest.raises(hs.HSError):
            srv.cancel(reqs[0][0])                          # finished and collected: unknown


def test_request_beyond_budget_is_ebudget(hs):
    """A request that alone needs more memory than the server reserved can
    never be admitted: HS_EBUDGET, distinct from HS_EINVAL for malformed
    arguments; the server keeps serving."""
    wl, sk, ref = _setup(hs, "toy", 4, 1, 74)
    with hs.Server({"toy": sk}, max_inflight=1, max_batch=4, mem_budget=1 << 20, pinned=1 << 20) as srv:
        with pytest.raises(hs.HSError) as e:
            srv.submit("toy", 0, bytes(2 << 20))               # 2 MiB message, 1 MiB budget
        assert e.value.code == HS_EBUDGET
        assert "budget" in hs.last_error()
        L = hs.load()
        assert L.hs_server_submit(srv._h, 99, 0, None, 0, None, None) == HS_EINVAL     # no such set
        rid, out = srv.submit("toy", int(wl.key_idx[0]), wl.message(0))
        srv.wait(rid, timeout_ms=60000)
        assert out.tobytes() == ref[0].tobytes()
