"""Multi-process host logic of bench.py (gloo, world size 2, CPU only)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1208_2643_gb300 import replicas
    r, w, lr = replicas.rank_info()
    local_ms = 100.0 + 50.0 * r          # rank 1 is slower
    job = replicas.job_time_ms(local_ms)
    out.put((r, w, lr, replicas.instance_seed(1, r), job, replicas.throughput(10, w, job)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1] and all(x[1] == 2 for x in res)
    assert [x[3] for x in res] == [1, 2]                 # distinct instance seeds
    assert all(x[4] == 150.0 for x in res)               # max over ranks
    assert all(abs(x[5] - 2 * 10 / 0.150) < 1e-9 for x in res)


def test_single_process_is_identity():
    from paper_1208_2643_gb300 import replicas
    assert replicas.job_time_ms(12.5) == 12.5
    assert replicas.throughput(100, 1, 1000.0) == 100.0
