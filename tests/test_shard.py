"""Host logic of the sharded batched scan (CPU): the greedy LPT assignment
of whole targets to ranks and the end-of-run FP64 tally reduction over
torch.distributed (gloo, world size 2)."""
import itertools
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2107_01723_gb300 import shard
from paper_2107_01723_gb300 import workloads as W


def test_lpt_assigns_every_target_once_and_balances():
    w = [l["n_macro"] for l in W.config4()["lasers"]]
    for n in (1, 2, 3, 4, 8):
        a = shard.lpt_assign(w, n)
        assert sorted(itertools.chain(*a)) == list(range(len(w)))
        loads = [sum(w[t] for t in r) for r in a]
        # LPT bound: max load <= 4/3 of optimum; the optimum is >= max(mean, largest)
        lower = max(sum(w) / n, max(w))
        assert max(loads) <= 4 / 3 * lower + 1e-9
    assert shard.lpt_assign([5, 5, 5, 5], 2) == [[0, 2], [1, 3]]


def test_lpt_matches_brute_force_on_small_cases():
    cases = [[7, 6, 5, 4, 3, 3, 2], [10, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1], [3, 3, 2, 2, 2]]
    for w in cases:
        for n in (2, 3):
            best = min(max(sum(w[i] for i in range(len(w)) if lab[i] == r) for r in range(n))
                       for lab in itertools.product(range(n), repeat=len(w)))
            lpt = max(sum(w[t] for t in r) for r in shard.lpt_assign(w, n))
            assert best <= lpt <= 4 / 3 * best


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
    from paper_2107_01723_gb300 import shard as S
    tot = S.reduce_tallies(world, {"E_xray_above": [1.5, 2.25][rank], "E_injected": [10.0, 30.0][rank]})
    q.put((rank, tot))
    dist.destroy_process_group()


def test_tally_reduction_two_ranks():
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
    for _, tot in out:
        assert tot == {"E_xray_above": 3.75, "E_injected": 40.0}
