"""The benchmark's multi-rank plumbing (replicas: one independent problem per
rank, only timings cross ranks) on CPU with the gloo backend, world size 2."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    from paper_1811_10573_gb300 import harness
    d = harness.init(backend="gloo")
    d.barrier()
    m = d.max(1.5 + rank)
    g = d.gather(10.0 * rank)
    d.barrier()
    d.close()
    q.put((rank, m, g))


def test_max_and_gather_over_two_ranks():
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
    assert [r[1] for r in res] == [2.5, 2.5]
    assert all(r[2] == [0.0, 10.0] for r in res)


def test_single_process_is_identity(monkeypatch):
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    from paper_1811_10573_gb300 import harness
    d = harness.init()
    assert not d.active and d.max(3.0) == 3.0 and d.gather(2.0) == [2.0]
    d.barrier()
