"""Multi-rank host logic on CPU (gloo, world size 2): the timing reduction the
benchmark uses under torchrun, the global row offsets that stitch row blocks
into one CSR, and the partition helpers."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2111_09947_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _sharded_worker(rank, world, port, q):
    """Each rank computes its row block of one product with the oracle as the
    compute function; rank 0 stitches the blocks."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        from oracle import oracle as O
        from paper_2111_09947_gb300 import synth
        p = synth.random_problem(300, 200, 250, 6.0, 9.0, 20.0, 91, "i64")

        def compute(Mb, Ab, B):
            return O.masked_spgemm(Mb, Ab, B, "plus_times_i64")
        out = shard.sharded_product(p["M"], p["A"], p["B"], compute, rank, world)
        parts = [None] * world
        dist.all_gather_object(parts, {k: out[k] for k in ("r0", "r1", "offset", "nnz")} |
                               {"rowptr": out["result"]["rowptr"], "colidx": out["result"]["colidx"],
                                "values": out["result"]["values"]})
        q.put((rank, parts))
    finally:
        dist.destroy_process_group()


def _tc_worker(rank, world, port, q):
    """Each rank counts the triangles of its row block of L with the oracle;
    the all-reduce gives every rank the whole count."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        from oracle import oracle as O
        from paper_2111_09947_gb300 import synth
        L = synth.triangle_counting(scale=10, ef=8, seed=3)["M"]

        def count_block(Lb, Lfull):
            r = O.masked_spgemm(Lb, Lb, Lfull, "plus_pair_i64")
            return torch.tensor([int(r["values"].sum())], dtype=torch.int64)
        out = shard.sharded_triangle_count(L, count_block, rank, world)
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_triangle_count():
    """A triangle count split by rows over two gloo ranks: the blocks cover
    the rows once, and the all-reduced count equals the whole product's."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from oracle import oracle as O
    from paper_2111_09947_gb300 import synth
    L = synth.triangle_counting(scale=10, ef=8, seed=3)["M"]
    want = int(O.masked_spgemm(L, L, L, "plus_pair_i64")["values"].sum())
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_tc_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0]["r0"] == 0 and res[0]["r1"] == res[1]["r0"] and res[1]["r1"] == L.nrows
    assert res[0]["local"] + res[1]["local"] == want
    assert res[0]["total"] == res[1]["total"] == want
    assert res[0]["local"] > 0 and res[1]["local"] > 0


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms, work = shard.reduce_timing(10.0 + 5 * rank, 100.0 * (rank + 1))
        offs = shard.gather_row_offsets(7 + 3 * rank)
        q.put((rank, ms, work, offs))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_and_offsets():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, work, offs in res:
        assert ms == 15.0 and work == 300.0
        assert offs == [0, 7]


def test_partition_rows_balances_work():
    rng = np.random.default_rng(0)
    work = rng.pareto(1.5, 10000) * 100
    b = shard.partition_rows(work, 4)
    assert b[0] == 0 and b[-1] == len(work) and np.all(np.diff(b) >= 0)
    sums = [work[b[i]:b[i + 1]].sum() for i in range(4)]
    assert max(sums) <= work.sum() / 4 + work.max() + 1e-9
    assert list(shard.partition_rows(np.zeros(10), 3)) == [0, 3, 7, 10]
    with pytest.raises(ValueError):
        shard.partition_rows(work, 0)


def test_partition_products_covers_all():
    costs = [5, 1, 1, 1, 9, 3, 2]
    parts = shard.partition_products(costs, 3)
    assert sorted(sum(parts, [])) == list(range(len(costs)))
    loads = [sum(costs[p] for p in part) for part in parts]
    assert max(loads) - min(loads) <= max(costs)


def test_two_rank_row_sharded_product_stitches():
    from oracle import oracle as O
    from paper_2111_09947_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = res[0]
    assert parts[0]["r0"] == 0 and parts[0]["r1"] == parts[1]["r0"] and parts[1]["r1"] == 300
    assert parts[0]["offset"] == 0 and parts[1]["offset"] == parts[0]["nnz"]
    # stitched CSR: row pointers shifted by each block's offset
    rp = np.concatenate([parts[0]["rowptr"][:-1] + parts[0]["offset"], parts[1]["rowptr"] + parts[1]["offset"]])
    ci = np.concatenate([x["colidx"] for x in parts])
    va = np.concatenate([x["values"] for x in parts])
    p = synth.random_problem(300, 200, 250, 6.0, 9.0, 20.0, 91, "i64")
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64")
    assert np.array_equal(rp, ref["rowptr"]) and np.array_equal(ci, ref["colidx"])
    assert np.array_equal(va, ref["values"])
    # the split balances push work
    w = shard.push_work(p["A"], p["B"])
    b = parts[0]["r1"]
    assert abs(w[:b].sum() - w[b:].sum()) <= w.max()
