"""The multi-rank path on CPU with two gloo ranks: disjoint shot ranges per rank, step time as the
maximum over ranks, counts as the sum; the summed per-weight counts of the ranks equal one process
sampling the union of their ranges (shots are independent, Sec. 5.1)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from oracle import sampler
from oracle.circuit import parse
from synth import tiny_circuit

TEXT = tiny_circuit(3, 2, seed=3)
DRAWN = 128


def _counts(shot0, n):
    counts, _ = sampler.sample(parse(TEXT), p=2e-2, seed=1, shots=range(shot0, shot0 + n), engine="sv")
    out = np.zeros((8, 3), dtype=np.int64)
    for w, (a, b, c) in counts.items():
        out[min(w, 7)] += (a, b, c)
    return out


def _worker(rank, world, port, out_q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        starts = [bench.rank_shot0(rank, s, DRAWN) for s in range(2)]
        gathered = [None] * world
        dist.all_gather_object(gathered, starts)
        c = sum(_counts(s0, DRAWN) for s0 in starts)
        t = torch.tensor(c.reshape(-1), dtype=torch.int64)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        ms, acc, surv = bench.reduce_over_ranks(dist, "cpu", 10.0 * (rank + 1), int(c[:, 1].sum()), int(c[:, 0].sum()))
        if rank == 0:
            out_q.put((gathered, t.numpy().reshape(8, 3), ms, acc, surv))
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.slow
def test_two_gloo_ranks_partition_and_sum():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p_ in procs:
        p_.start()
    gathered, total, ms, acc, surv = q.get(timeout=300)
    for p_ in procs:
        p_.join(timeout=60)
        assert p_.exitcode == 0
    ranges = [(s0, s0 + DRAWN) for starts in gathered for s0 in starts]
    ranges.sort()
    assert all(a % 64 == 0 for a, _ in ranges)
    assert all(ranges[i][1] <= ranges[i + 1][0] for i in range(len(ranges) - 1))  # disjoint
    union = sum(_counts(a, b - a) for a, b in ranges)
    assert np.array_equal(total, union)
    assert ms == 20.0 and acc == int(union[:, 1].sum()) and surv == int(union[:, 0].sum())
