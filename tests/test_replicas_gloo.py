"""Multi-process path of the benchmark on CPU: two gloo ranks.

The solve shards as independent replicas (no data-path collective); what the
ranks share is the right-hand-side numbering and the max-over-ranks timing.
Checked here with world_size 2 on the CPU: the maximum reaches every rank, the
ranks' right-hand-side indices are disjoint and give different vectors, and
the job total counts every rank's solves.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import synth
    from paper_1912_02868_gb300 import replicas
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = replicas.rank_env()
        replicas.barrier()
        mx = replicas.max_over_ranks(10.0 * (rank + 1))
        idx = [replicas.rhs_index(r, s) for s in range(3)]
        b0 = synth.rhs(16, 0, idx[0])[0]
        out.put((rank, r, w, local, mx, idx, float(np.abs(b0).sum())))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas():
    import torch.multiprocessing as mp
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
    (r0, e0, w0, l0, m0, i0, s0), (r1, e1, w1, l1, m1, i1, s1) = res
    assert (e0, w0, l0) == (0, 2, 0) and (e1, w1, l1) == (1, 2, 1)
    assert m0 == m1 == 20.0                      # the max reaches both ranks
    assert not set(i0) & set(i1)                 # disjoint right-hand sides
    assert s0 != s1                              # and different vectors


def test_single_process_defaults():
    from paper_1912_02868_gb300 import replicas
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.rhs_index(0, 7) == 7 and replicas.rhs_index(2, 7) == 2 * replicas.RHS_STRIDE + 7
    assert replicas.total_units(4, 5, 10) == 200
    with pytest.raises(ValueError):
        replicas.rhs_index(0, replicas.RHS_STRIDE)
