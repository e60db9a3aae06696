"""Multi-process slice sharding on CPU (gloo, world size 2).

Each rank contracts its own block of slices (here with the FP64 oracle, the
CPU stand-in for one GPU's share), the partial amplitudes are summed with
one all-reduce, and the result must equal the whole slice range contracted
at once and the state-vector amplitudes.
"""

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2005_06787_gb300.shard import all_reduce_amplitudes, slice_range
from synthetic.circuits import grid_layout, random_bits, random_circuit

SLICED = [(4, 2), (1, 3), (7, 1), (3, 4), (8, 2)]


def _case():
    c = random_circuit(grid_layout(3, 3), 5, 37)
    oq = [2, 5, 8]
    cb = list(random_bits(6, 8))
    return c, oq, cb


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c, oq, cb = _case()
    net = oracle.build_network(c, oq, cb)
    lo, hi = slice_range(rank, world, 1 << len(SLICED))
    part = oracle.contract_sliced_sum(net, SLICED, slices=list(range(lo, hi))).reshape(-1)
    t = torch.from_numpy(np.ascontiguousarray(part).view(np.float64).copy())
    all_reduce_amplitudes(t)
    if rank == 0:
        out_q.put(t.numpy().view(np.complex128).copy())
    dist.barrier()
    dist.destroy_process_group()


def test_slice_range_partitions():
    for total in [0, 1, 7, 256, 1000]:
        for world in [1, 2, 3, 8]:
            blocks = [slice_range(r, world, total, begin=5) for r in range(world)]
            assert blocks[0][0] == 5 and blocks[-1][1] == 5 + total
            for (a, b), (c_, d) in zip(blocks, blocks[1:]):
                assert b == c_
            sizes = [b - a for a, b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slice_range(2, 2, 10)


def test_two_rank_slice_sum_equals_whole_range():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    port = _free_port()
    mp.spawn(_worker, args=(world, port, q), nprocs=world, join=True)
    got = q.get(timeout=60)
    c, oq, cb = _case()
    net = oracle.build_network(c, oq, cb)
    whole = oracle.contract_sliced_sum(net, SLICED).reshape(-1)
    np.testing.assert_allclose(got, whole, atol=1e-13)
    np.testing.assert_allclose(got, oracle.sv_amplitudes(c, oq, cb), atol=1e-13)
