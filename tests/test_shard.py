"""Host-side sharding of the batched sweep across ranks: the assignment covers every
lattice once and balances the site counts; the gathered table equals the one-process
table, checked with two gloo ranks on the CPU (no GPU)."""
import os
import socket

import numpy as np
import pytest

from paper_1306_6445_gb300 import inputs as I
from paper_1306_6445_gb300 import shard

torch = pytest.importorskip("torch")


def sweep_sizes(n=512):
    return [d["side"] ** 2 for d in I.batch_draws(n)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_assignment_covers_each_lattice_once_and_balances_sites(world):
    sizes = np.array(sweep_sizes())
    parts = shard.assign(sizes, world)
    allidx = np.concatenate(parts)
    assert len(allidx) == len(sizes) and np.array_equal(np.sort(allidx), np.arange(len(sizes)))
    loads = np.array([sizes[p].sum() for p in parts])
    # greedy largest-first: the spread is at most one lattice
    assert loads.max() - loads.min() <= sizes.max()
    assert shard.assign(sizes, world)[0].tolist() == parts[0].tolist()   # deterministic


def fake_measure(idx):
    """Stand-in for lb_batch_measure: a row that depends only on the lattice index."""
    i = np.asarray(idx, dtype=np.float64)
    return np.stack([i * 0.5, np.sin(i), np.cos(i) + 2.0], axis=1)


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = sweep_sizes(64)
    mine = shard.assign(sizes, world)[rank]
    table = shard.gather_rows(fake_measure(mine), mine, len(sizes), dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, table))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_gather_the_full_table():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = fake_measure(np.arange(64))
    for r in range(2):
        assert np.array_equal(got[r], want)


def test_gather_without_a_group_needs_full_coverage():
    with pytest.raises(ValueError):
        shard.gather_rows(fake_measure([0, 1]), [0, 1], 3)
    assert np.array_equal(shard.gather_rows(fake_measure([2, 0, 1]), [2, 0, 1], 3),
                          fake_measure([0, 1, 2]))
