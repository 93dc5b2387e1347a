"""The replica harness of `bench.py --gpus N` on CPU with the gloo backend:
whole-job throughput = work summed over ranks / max over ranks of the timed
region, and per-rank independent random keys."""
import os
import socket

import pytest

from paper_2512_24970_gb300.replicas import aggregate, replica_seed


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        v, ms, units = aggregate(100.0 + 50.0 * rank, 1000.0 * (rank + 1), dist, torch.device("cpu"))
        q.put((rank, v, ms, units, replica_seed(7, rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_single_process():
    v, ms, units = aggregate(250.0, 5000.0)
    assert (ms, units) == (250.0, 5000.0)
    assert v == pytest.approx(20000.0)


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, v, ms, units, seed in out:
        assert ms == 150.0                        # the slower rank's time
        assert units == 3000.0                    # both ranks' work
        assert v == pytest.approx(3000.0 / 0.150)
    assert [o[4] for o in out] == [7, 1007]       # independent Philox keys
