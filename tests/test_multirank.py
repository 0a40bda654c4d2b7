"""The multi-process harness of bench.py on the host (gloo, world size 2): every rank
contracts its own sub-cube batch (independent problems, weak scaling) and the job time is
the maximum over the ranks.  No GPU work: the device path per rank is the one-GPU path."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, circ, fixed, open_q = bench.workload("t12", rank)
        bits = torch.from_numpy(fixed.astype(np.int64))
        gathered = [torch.zeros_like(bits) for _ in range(world)]
        dist.all_gather(gathered, bits)
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
        out[rank] = (ms, [g.numpy().tolist() for g in gathered], list(open_q))
    finally:
        dist.destroy_process_group()


def test_two_ranks_independent_batches_and_max_time():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        ms, gathered, open_q = res[r]
        assert ms == 15.0  # the slowest rank
        assert gathered[0] != gathered[1]  # each rank has its own sub-cube batch
        assert open_q == res[0][2]  # same open qubits, same plan shape
