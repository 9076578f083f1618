"""Multi-GPU host logic on CPU: instance shards are disjoint, cover the batch and are balanced; the
timing reduction is the maximum over ranks.  Two gloo ranks on 127.0.0.1 (no GPU)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2507_04115_gb300 import inputs, sharding
    wl = inputs.uneven_batch(n=2000, seed=2)
    costs = sharding.instance_cost(wl.N, wl.n_steps)
    mine = sharding.lpt(costs, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine.tolist())
    t = torch.tensor([float(rank + 1) * 1.5])          # stand-in for each rank's measured time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    blocks = [sharding.contiguous(8192 * world, world, r) for r in range(world)]
    if rank == 0:
        q.put((gathered, float(t.item()), [(b.start, b.stop) for b in blocks], float(costs.sum()),
               [float(costs[np.array(g)].sum()) for g in gathered], float(costs.max())))
    dist.barrier()
    dist.destroy_process_group()


def test_lpt_shards_on_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    gathered, tmax, blocks, total, loads, cmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    allidx = np.concatenate([np.array(g) for g in gathered])
    assert np.array_equal(np.sort(allidx), np.arange(2000))          # disjoint and complete
    assert abs(sum(loads) - total) < 1e-6 * total
    assert max(loads) <= total / world + cmax                         # LPT bound
    assert tmax == 3.0                                                # max over ranks
    assert blocks == [(0, 8192), (8192, 16384)]


def test_contiguous_blocks_cover_ragged_sizes():
    from paper_2507_04115_gb300 import sharding
    for n, world in [(10, 3), (8192, 8), (7, 7), (5, 8)]:
        spans = [sharding.contiguous(n, world, r) for r in range(world)]
        covered = np.concatenate([np.arange(s.start, s.stop) for s in spans])
        assert np.array_equal(covered, np.arange(n))
        sizes = [s.stop - s.start for s in spans]
        assert max(sizes) - min(sizes) <= 1
