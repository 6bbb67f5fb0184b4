"""The N > 1 benchmark path on CPU: independent replicas over torch.distributed
(gloo, world size 2).  The step itself has no exchange; the only collective
logic is the barrier and the max-time / summed-work reduction that turns the
ranks' results into the whole-job rate."""
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


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    ms = [40.0, 50.0][rank]          # the slower rank sets the job time
    work = [1.0e9, 3.0e9][rank]      # particle-steps each replica processed
    rate, ms_max, ps_sum = bench.replica_rate(world, ms, work)
    q.put((rank, rate, ms_max, ps_sum))
    dist.destroy_process_group()


def test_replica_rate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, ms_max, ps_sum in out:
        assert ms_max == 50.0 and ps_sum == 4.0e9
        assert rate == pytest.approx(4.0e9 / 0.05)
