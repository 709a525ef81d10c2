"""Sharding of slices over ranks on CPU: two gloo ranks each contract their
share of the slices with the FP64 oracle; the all-reduced sum equals the
unsliced contraction, whatever the rank count."""
import os

import numpy as np
import pytest

from paper_2410_15080_b300.shard import slice_range


@pytest.mark.parametrize("n,w", [(16, 2), (17, 3), (5, 8), (1024, 8), (0, 4)])
def test_slice_range_partitions(n, w):
    got = [slice_range(r, w, n) for r in range(w)]
    assert sum(c for _, c in got) == n
    pos = 0
    for f, c in got:
        assert f == pos and c >= 0
        pos += c
    assert max(c for _, c in got) - min(c for _, c in got) <= 1


def _worker(rank, world, port, q):
    import itertools
    import torch
    import torch.distributed as dist
    import synth
    from oracle import planner, tn
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    net = synth.ring_htn(n_sub=4, gates_per_edge=1, wires_per_edge=1, k=3, seed=7)
    p = planner.make_plan(net.inds(), net.dims(), net.output, n_slices=16, slice_dim=4)
    dims = net.dims()
    assign = list(itertools.product(*[range(dims[i]) for i in p.sliced]))
    first, count = slice_range(rank, world, len(assign))
    part = np.zeros(3)
    for vals in assign[first:first + count]:
        sub = tn.slice_network(net.pairs(), dict(zip(p.sliced, vals)))
        part = part + tn.contract_pairwise(sub, net.output, planner.order_of(p))
    t = torch.from_numpy(part)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        full = tn.contract_pairwise(net.pairs(), net.output, planner.order_of(p))
        q.put(float(np.abs(t.numpy() - full).max() / np.abs(full).max()))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slice_sum_over_gloo_ranks(world):
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert q.get(timeout=10) < 1e-12
