"""Sharding of independent lattices across ranks (one process per GPU).

The batched sweep's lattices are independent problems, so ranks split them with no
data-path communication: `assign` balances the site counts (largest first onto the least
loaded rank, deterministic), each rank advances its own lattices, and `gather_rows` puts
the per-lattice results back in the global order on the host at the end (an
all_gather_object of the small result rows; it works on gloo and NCCL groups alike)."""
from __future__ import annotations

import numpy as np


def assign(sizes, world: int):
    """Lattice indices per rank for lattices of the given site counts: largest first, each
    onto the rank with the fewest sites so far (ties to the lower rank). Returns a list of
    `world` sorted index arrays covering every lattice exactly once."""
    sizes = np.asarray(sizes, dtype=np.int64)
    if world < 1:
        raise ValueError("world must be >= 1")
    load = np.zeros(world, dtype=np.int64)
    parts = [[] for _ in range(world)]
    for i in sorted(range(len(sizes)), key=lambda k: (-sizes[k], k)):
        r = int(np.argmin(load))
        parts[r].append(i)
        load[r] += sizes[i]
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def gather_rows(rows, idx, n: int, dist=None):
    """Assemble the global n x k table from this rank's rows (len(idx) x k) for lattices
    idx. Without a process group the local rows must already cover everything."""
    rows = np.asarray(rows, dtype=np.float64)
    pieces = [(np.asarray(idx), rows)]
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        out = [None] * dist.get_world_size()
        dist.all_gather_object(out, (np.asarray(idx).tolist(), rows.tolist()))
        pieces = [(np.asarray(i, dtype=np.int64), np.asarray(r, dtype=np.float64).reshape(len(i), -1))
                  for i, r in out]
    k = next((p[1].shape[1] for p in pieces if len(p[0])), 0)
    table = np.full((n, k), np.nan)
    seen = np.zeros(n, dtype=bool)
    for i, r in pieces:
        if len(i):
            if seen[i].any():
                raise ValueError("a lattice was measured by two ranks")
            table[i] = r
            seen[i] = True
    if not seen.all():
        raise ValueError("some lattices were measured by no rank")
    return table
