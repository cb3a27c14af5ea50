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


def row_block(X, r0: int, r1: int):
    """Rows [r0, r1) of a CSR matrix X (numpy or torch arrays) as a CSR of
    r1 - r0 rows over the same columns: row pointers rebased, column and
    value slices are views.  Returns an object of X's type when it accepts
    (nrows, ncols, rowptr, colidx, values), else a dict."""
    base = int(X.rowptr[r0])
    end = int(X.rowptr[r1])
    rp = X.rowptr[r0:r1 + 1] - base
    ci = X.colidx[base:end]
    vals = getattr(X, "values", None)
    v = vals[base:end] if vals is not None else None
    try:
        return type(X)(r1 - r0, X.ncols, rp, ci, v)
    except TypeError:
        return {"nrows": r1 - r0, "ncols": X.ncols, "rowptr": rp, "colidx": ci, "values": v}


def push_work(A, B) -> np.ndarray:
    """Push products per row of A B (sum over A_i* of nnz(B_k*)), on host."""
    def host(x):
        return x.cpu().numpy() if hasattr(x, "cpu") else np.asarray(x)
    arp, aci, brp = host(A.rowptr).astype(np.int64), host(A.colidx), host(B.rowptr).astype(np.int64)
    blen = np.diff(brp)
    cs = np.concatenate([[0], np.cumsum(blen[aci])]) if len(aci) else np.zeros(1, np.int64)
    return cs[arp[1:]] - cs[arp[:-1]]


def sharded_product(M, A, B, compute, rank: int, world: int, group=None, device=None):
    """This rank's share of C = M .* (A B) (or its complement, as compute
    decides): the contiguous block of rows [r0, r1) that partition_rows gives
    it by push work, computed by compute(M_block, A_block, B) (the library's
    GPU product in use; any CSR-returning function in tests), plus the number
    of entries of C before the block (an all-gather of per-rank counts), so
    the blocks stitch into one CSR.  B is replicated on every rank.

    Returns dict(r0, r1, offset, nnz, result)."""
    b = partition_rows(push_work(A, B), world)
    r0, r1 = int(b[rank]), int(b[rank + 1])
    res = compute(row_block(M, r0, r1), row_block(A, r0, r1), B)
    rp = res["rowptr"] if isinstance(res, dict) else res.rowptr
    nnz = int(rp[-1]) if len(rp) else 0
    offsets = gather_row_offsets(nnz, device=device, group=group)
    return {"r0": r0, "r1": r1, "offset": int(offsets[rank]), "nnz": nnz, "result": res}


def allreduce_sum(x, group=None):
    """In-place sum of a tensor over the group (the one data-path exchange of
    a row-sharded triangle count: each rank's partial count)."""
    import torch.distributed as dist
    dist.all_reduce(x, op=dist.ReduceOp.SUM, group=group)
    return x


def sharded_triangle_count(L, count_block, rank: int, world: int, group=None, device=None):
    """Triangle count of the strict lower triangle L (C = L .* (L L) on
    plus-pair, count = sum(C), Sec. 8.2) split by rows: this rank computes the
    block of rows that partition_rows gives it by push work (L replicated as
    the right operand), count_block(L_block, L) returns its partial count as
    a one-element int64 tensor on `device`, and an all-reduce sums the
    partial counts.  Returns dict(r0, r1, local, total)."""
    b = partition_rows(push_work(L, L), world)
    r0, r1 = int(b[rank]), int(b[rank + 1])
    Lb = row_block(L, r0, r1)
    part = count_block(Lb, L)
    local = int(part.item())
    total = allreduce_sum(part, group=group)
    return {"r0": r0, "r1": r1, "local": local, "total": int(total.item())}
