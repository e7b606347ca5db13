"""The N > 1 bookkeeping of bench.py on CPU: two gloo ranks, distinct seeds,
barrier, and the max / sum reductions of per-rank timings."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    from paper_2505_05919_gb300 import dist
    dist.init("gloo")
    r, w, _ = dist.env()
    dist.barrier()
    mx = dist.max_over_ranks(1.5 + r)     # rank 1 is the slowest
    sm = dist.sum_over_ranks(10.0 * (r + 1))
    out[r] = (r, w, dist.seed_offset(r), mx, sm)
    dist.finalize()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = dict(out)
    assert set(res) == {0, 1}
    assert res[0][1] == res[1][1] == 2
    assert res[0][2] != res[1][2]                 # replicas differ across ranks
    assert res[0][3] == res[1][3] == 2.5          # max over ranks
    assert res[0][4] == res[1][4] == 30.0         # sum over ranks


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2505_05919_gb300 import dist
    assert dist.env() == (0, 1, 0)
    assert dist.max_over_ranks(3.25) == 3.25
