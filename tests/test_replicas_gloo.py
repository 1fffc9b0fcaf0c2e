"""The N > 1 path on CPU: two gloo ranks run independent replicas (no data
collective) and the whole-job rate is the units of all ranks over the time of
the slowest rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from workloads import generators as gen


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2511_05895_gb300 import replicas
    import oracle
    r, w, _ = replicas.rank_world()
    # each rank: its own seeded graph and batches (what bench.py does per GPU)
    g = gen.random_graph(n=300, m=2000, seed=100 + r)
    cap = g.cap.copy()
    flows = []
    for i in range(2):
        b = gen.mixed_batch(cap, 20, 1, 50, seed=100 + r, index=i)
        gen.apply_batch(cap, b)
        flows.append(oracle.maxflow_fifo(g.n, g.row_ptr, g.col, cap, g.s, g.t))
    seconds = 1.0 + r                      # rank 1 is the slower one
    rate = replicas.whole_job_rate(10, seconds)
    mx = replicas.max_over_ranks(seconds)
    out[r] = (r, w, rate, mx, flows)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(90)
        assert p.exitcode == 0
    for r in range(world):
        rr, w, rate, mx, flows = out[r]
        assert rr == r and w == world
        assert mx == 2.0                      # max over ranks
        assert abs(rate - world * 10 / 2.0) < 1e-12
        assert all(f >= 0 for f in flows)
    assert out[0][4] != out[1][4]             # independent replicas, different graphs
