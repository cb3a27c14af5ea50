"""The masked heap procedure of Sec. 5.5 (Alg. 4 with the insertion of Alg. 5),
written out as the paper states it -- one binary heap of row iterators, one
pop at a time -- must reach the definition of the masked product that the
oracle computes, for NInspect 0, 1, 2 and unbounded, with a plain mask, and
with NInspect 0 under a complement.  This pins the reading the heap kinds
follow: an iterator whose look-ahead runs off the end of the mask leaves the
queue, and the main loop stops once the mask is exhausted (plain only).
"""
import heapq
import itertools

import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_09947_gb300 import synth

INF = None   # NInspect unbounded


def heap_row(m, a_cols, a_vals, B, ninspect, complement):
    """One row: m sorted mask columns, (a_cols, a_vals) the row u of A."""
    queue = []
    tie = itertools.count()

    def insert(k, a, p, mi):
        e = B.rowptr[k + 1]
        if p >= e:
            return
        if ninspect == 0 or complement:
            heapq.heappush(queue, (int(B.colidx[p]), next(tie), k, a, p))
            return
        left = ninspect
        while p < e and mi < len(m):
            bc, mc = int(B.colidx[p]), int(m[mi])
            if bc == mc:
                heapq.heappush(queue, (bc, next(tie), k, a, p))
                return
            if bc < mc:
                p += 1
            else:
                mi += 1
                if left is not None:
                    left -= 1
                    if left == 0:
                        heapq.heappush(queue, (bc, next(tie), k, a, p))
                        return

    mi = 0
    for k, a in zip(a_cols, a_vals):
        insert(int(k), a, int(B.rowptr[k]), mi)
    out_c, out_v = [], []
    prev = None
    while queue:
        j, _, k, a, p = heapq.heappop(queue)
        while mi < len(m) and m[mi] < j:
            mi += 1
        if mi == len(m) and not complement:
            break
        in_mask = mi < len(m) and m[mi] == j
        if in_mask != complement:
            prod = a * (B.values[p] if B.values is not None else 1)
            if prev == j:
                out_v[-1] += prod
            else:
                prev = j
                out_c.append(j)
                out_v.append(prod)
        insert(k, a, p + 1, mi)
    return out_c, out_v


def heap_product(M, A, B, ninspect, complement):
    rp, ci, vals = [0], [], []
    for i in range(M.nrows):
        m = M.colidx[M.rowptr[i]:M.rowptr[i + 1]]
        s, e = A.rowptr[i], A.rowptr[i + 1]
        av = A.values[s:e] if A.values is not None else np.ones(e - s, np.int64)
        c, v = heap_row(m, A.colidx[s:e], av, B, ninspect, complement)
        ci += c
        vals += v
        rp.append(len(ci))
    return np.array(rp), np.array(ci, dtype=np.int64), np.array(vals)


CASES = [(30, 20, 25, 3.0, 3.0, 6.0), (40, 30, 50, 1.0, 2.0, 20.0), (25, 40, 30, 6.0, 5.0, 2.0),
         (12, 12, 12, 12.0, 12.0, 12.0), (20, 0, 10, 0.0, 0.0, 3.0)]


@pytest.mark.parametrize("ninspect", [0, 1, 2, INF])
def test_heap_plain_reaches_definition(ninspect):
    for s, (m, k, n, da, db, dm) in enumerate(CASES):
        p = synth.random_problem(m, k, n, min(da, max(k, 1)), db, dm, 700 + s, "i64")
        ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64")
        rp, ci, v = heap_product(p["M"], p["A"], p["B"], ninspect, False)
        assert np.array_equal(rp, ref["rowptr"]) and np.array_equal(ci, ref["colidx"])
        assert np.array_equal(v.astype(np.int64), ref["values"])


def test_heap_complement_reaches_definition():
    for s, (m, k, n, da, db, dm) in enumerate(CASES):
        p = synth.random_problem(m, k, n, min(da, max(k, 1)), db, dm, 800 + s, "i64")
        ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64", complement=True, method=O.ESC)
        rp, ci, v = heap_product(p["M"], p["A"], p["B"], 0, True)
        assert np.array_equal(rp, ref["rowptr"]) and np.array_equal(ci, ref["colidx"])
        assert np.array_equal(v.astype(np.int64), ref["values"])


def test_heap_look_ahead_skips_products():
    """With NInspect unbounded every queued iterator sits on a mask column, so
    the pops are exactly the masked products (the plus-pair sum of C); with
    NInspect 0 the queue also carries the products the mask discards."""
    p = synth.random_problem(40, 30, 400, 4.0, 40.0, 5.0, 901, "i64")
    M, A, B = p["M"], p["A"], p["B"]
    pops = {0: 0, INF: 0}
    orig = heapq.heappop
    for ni in pops:
        def counting(q, _ni=ni):
            pops[_ni] += 1
            return orig(q)
        heapq.heappop = counting
        try:
            heap_product(M, A, B, ni, False)
        finally:
            heapq.heappop = orig
    masked = int(O.masked_spgemm(M, A, B, "plus_pair_i64")["values"].sum())
    assert pops[INF] == masked
    assert pops[0] > 4 * masked
