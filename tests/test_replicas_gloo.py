"""The N > 1 (replica) path of bench.py on CPU: two gloo ranks combine their
step times as the maximum, and the job rate counts both ranks' signatures."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2512_23969_gb300 import replicas
    ws, r, local = replicas.init_from_env()
    local_ms = 100.0 + 50.0 * r                  # rank 1 is slower
    m = replicas.max_over_ranks(local_ms)
    replicas.barrier()
    q.put((r, ws, local, m, replicas.job_rate(ws, 16384, 5, m)))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_gloo_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    assert all(r[1] == 2 for r in res)
    assert all(r[3] == pytest.approx(150.0) for r in res)
    assert all(r[4] == pytest.approx(2 * 16384 * 5 / 0.150) for r in res)


def test_single_process_defaults():
    from paper_2512_23969_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_rate(1, 100, 2, 1000.0) == pytest.approx(200.0)
