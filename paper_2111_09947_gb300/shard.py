"""Multi-GPU sharding of masked products (host logic).

Rows of C are independent (Sec. 4: row-by-row algorithms parallelise over
rows with no dependencies), so a product splits into contiguous row blocks
balanced by push work, and a batch splits by product, with no data exchange.
Only bookkeeping crosses ranks: the row offsets that stitch the blocks'
outputs into one CSR (an all-gather of per-rank entry counts) and the timing
reduction of the benchmark (max of times, sum of work).  Every function
takes an optional torch.distributed group and works on any backend (gloo on
CPU for tests, NCCL on GPUs).
"""
from __future__ import annotations

import numpy as np


def partition_rows(work: np.ndarray, parts: int) -> np.ndarray:
    """Boundaries b[0..parts] of contiguous row blocks with roughly equal
    total work (e.g. flops per row); b[0] = 0, b[parts] = len(work)."""
    work = np.asarray(work, dtype=np.float64)
    n = len(work)
    if parts <= 0:
        raise ValueError("parts must be positive")
    csum = np.concatenate([[0.0], np.cumsum(np.maximum(work, 0.0))])
    total = csum[-1]
    if total <= 0:
        return np.linspace(0, n, parts + 1).round().astype(np.int64)
    targets = total * np.arange(parts + 1) / parts
    b = np.searchsorted(csum, targets, side="left").astype(np.int64)
    b[0], b[-1] = 0, n
    return np.maximum.accumulate(np.clip(b, 0, n))


def partition_products(costs, parts: int) -> list[list[int]]:
    """Greedy longest-first assignment of products to ranks by cost."""
    order = sorted(range(len(costs)), key=lambda p: -costs[p])
    load = [0.0] * parts
    out: list[list[int]] = [[] for _ in range(parts)]
    for p in order:
        r = min(range(parts), key=lambda x: load[x])
        out[r].append(p)
        load[r] += costs[p]
    return [sorted(x) for x in out]


def reduce_timing(total_ms: float, work: float, device=None, group=None) -> tuple[float, float]:
    """(max of per-rank times, sum of per-rank work) over the group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    w = torch.tensor([work], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(w, op=dist.ReduceOp.SUM, group=group)
    return float(t.item()), float(w.item())


def gather_row_offsets(local_nnz: int, device=None, group=None) -> list[int]:
    """Exclusive prefix of every rank's entry count: where each row block's
    output starts in the stitched CSR."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    x = torch.tensor([local_nnz], dtype=torch.int64, device=device)
    parts = [torch.zeros_like(x) for _ in range(world)]
    dist.all_gather(parts, x, group=group)
    counts = [int(p.item()) for p in parts]
    return [0] + list(np.cumsum(counts)[:-1].tolist()) if world else []
