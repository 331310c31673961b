"""The N > 1 path on the CPU: two gloo ranks shard the frequency grid with no data-path
collective (disjoint batches per step, the grid covered in order), and the timing
reduction takes the maximum over ranks, as bench.py does under torchrun."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2310_04734_gb300.sharding import batch_indices


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, n, batch, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = torch.tensor(np.stack([batch_indices(n, batch, world, rank, s) for s in range(steps)]))
    gathered = [torch.zeros_like(idx) for _ in range(world)]
    dist.all_gather(gathered, idx)
    t = torch.tensor([1.0 + rank], dtype=torch.float64)   # a per-rank "elapsed time"
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put((torch.stack(gathered).numpy(), float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_frequencies_and_take_the_max_time():
    world, n, batch, steps = 2, 481, 96, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, batch, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    idx, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert tmax == 2.0
    # idx[rank, step, :]: within a step the ranks' batches are disjoint
    for s in range(steps):
        assert len(set(idx[0, s]) & set(idx[1, s])) == 0
    # in step order the ranks walk the grid contiguously, wrapping at its end
    walk = np.concatenate([idx[r, s] for s in range(steps) for r in range(world)])
    assert np.array_equal(walk, np.arange(world * batch * steps) % n)


def test_sharding_rejects_bad_arguments():
    with pytest.raises(ValueError):
        batch_indices(10, 4, 2, 2, 0)
