"""Host-side partitioning of search work across GPUs (one process per GPU).

Targets and tables are independent (the paper removes the only carried
dependency, the hunt-and-locate bound, Sec. 1 and 3.1), so no collective is
needed on the data path: each rank searches its own slice.

* one table, many targets: contiguous slices of the target array;
* many tables: whole tables per rank, assigned by longest-processing-time
  (largest target count first, to the least-loaded rank), so each table is
  prepared on exactly one rank.
"""
from __future__ import annotations

import heapq

import numpy as np


def target_slice(m: int, world: int, rank: int) -> tuple[int, int]:
    """[start, end) of rank's contiguous share of m targets (sizes differ by at most 1)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(m, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def lpt_tables(counts, world: int) -> list[np.ndarray]:
    """Table indices per rank: greedy longest-processing-time on target counts.
    Ties go to the lower rank, tables keep ascending order within a rank."""
    counts = np.asarray(counts, dtype=np.int64)
    order = np.argsort(-counts, kind="stable")
    heap = [(0, r) for r in range(world)]
    owner = np.empty(len(counts), dtype=np.int64)
    for k in order:
        load, r = heapq.heappop(heap)
        owner[k] = r
        heapq.heappush(heap, (load + int(counts[k]), r))
    return [np.flatnonzero(owner == r) for r in range(world)]


def gather_batch(X_off, X, Y_off, Y, tables):
    """The sub-batch of the given tables: (X_off, X, Y_off, Y, positions of
    its targets in the full Y) with offsets rebased to the sub-batch."""
    X_off = np.asarray(X_off)
    Y_off = np.asarray(Y_off)
    xs, ys, pos = [], [], []
    xo, yo = [0], [0]
    for k in tables:
        xs.append(X[X_off[k]:X_off[k + 1]])
        ys.append(Y[Y_off[k]:Y_off[k + 1]])
        pos.append(np.arange(Y_off[k], Y_off[k + 1]))
        xo.append(xo[-1] + X_off[k + 1] - X_off[k])
        yo.append(yo[-1] + Y_off[k + 1] - Y_off[k])
    cat = (lambda a: np.concatenate(a)) if xs else (lambda a: np.zeros(0))
    return (np.asarray(xo, dtype=np.int64), cat(xs), np.asarray(yo, dtype=np.int64), cat(ys),
            np.concatenate(pos) if pos else np.zeros(0, dtype=np.int64))
