"""Larger-scale parity: the sorted transpose across its three sort tiers,
the backward pass through column-tiled rows, and the workloads at (or near)
full size, checked on every row or on sampled rows the oracle computes one
by one."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2111_09947_gb300 import _lib, synth
from gpu_util import assert_parity, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    h = _lib.Handle()
    yield h
    h.close()


def test_transpose_sorted_all_tiers(handle):
    # A^T row lengths: 30000 (global-memory sort), 5000 (shared-memory CTA
    # sort), ~30 (warp sort)
    m, n = 30000, 64
    rng = np.random.default_rng(3)
    rows, cols = [], []
    for i in range(m):
        c = {0}
        if i % 6 == 0:
            c.add(1)
        c.update(rng.choice(np.arange(2, n), size=2, replace=False).tolist())
        for j in sorted(c):
            rows.append(i)
            cols.append(j)
    A = synth.coo_to_csr(m, n, np.array(rows, np.int32), np.array(cols, np.int32))
    A = A.with_values(synth.uniform_f32(A.nnz, 3, 1))
    d = _lib.DeviceCsr.from_host(A)
    At = _lib.msgemm_transpose(handle, d, 4, sorted_rows=True)
    torch.cuda.synchronize()
    ar = np.repeat(np.arange(m), np.diff(A.rowptr))
    order = np.lexsort((ar, A.colidx))        # by column, then row
    want_ci = ar[order]
    want_v = A.values[order]
    want_rp = np.concatenate([[0], np.cumsum(np.bincount(A.colidx, minlength=n))])
    assert np.array_equal(At.rowptr.cpu().numpy(), want_rp)
    assert np.array_equal(At.colidx.cpu().numpy(), want_ci)
    assert np.array_equal(At.values.cpu().numpy(), want_v)


@pytest.mark.parametrize("force", ["auto", "msa", "hash", "mca", "dot"])
def test_backward_tiled_rows(handle, force):
    # 60000 columns exceed one shared-memory tile: forced MSA runs tiled rows
    m, k, n = 200, 60000, 60000
    p = synth.random_problem(m, k, n, 40.0, 3.0, 30.0, 314, "f32")
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
    G = synth.Csr(m, n, ref["rowptr"].astype(np.int32), ref["colidx"], synth.upstream_grad(len(ref["colidx"]), 2))
    dA_ref, dB_ref = O.grad(p["A"], p["B"], G)
    d = to_dev(p, "plus_times_f32")
    handle.force(force)
    dA, dB = _lib.msgemm_backward(handle, d["A"], d["B"], _lib.DeviceCsr.from_host(G))
    handle.sync_status()
    handle.force("auto")
    Aabs = p["A"].with_values(np.abs(p["A"].values))
    Babs = p["B"].with_values(np.abs(p["B"].values))
    Gabs = G.with_values(np.abs(G.values))
    SA, SB = O.grad(Aabs, Babs, Gabs)          # sum of |g||b| and |a||g| per entry
    assert np.all(np.abs(dA.cpu().numpy() - dA_ref) <= 1e-5 * SA + 1e-30)
    assert np.all(np.abs(dB.cpu().numpy() - dB_ref) <= 1e-5 * SB + 1e-30)


def test_triangle_count_full_scale20(handle):
    p = synth.triangle_counting(scale=20, ef=16)
    d = to_dev(p, "plus_pair_i64")
    res = _lib.msgemm_run(handle, d["M"], d["A"], d["B"], "plus_pair_i64")
    tri = int(_lib.msgemm_reduce_sum(handle, res, "plus_pair_i64").item())
    handle.sync_status()
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_pair_i64")
    assert tri == int(ref["values"].sum())
    assert_parity(res.trimmed(), ref, "plus_pair_i64")


def test_bfs_step_full_scale20_sampled_rows(handle):
    p = synth.bfs_step(scale=20, ef=16, nsrc=512)
    d = to_dev(p, "plus_times_i64")
    res = _lib.msgemm_run(handle, d["M"], d["A"], d["B"], "plus_times_i64", complement=True).trimmed()
    handle.sync_status()
    flops = np.array([np.diff(p["B"].rowptr)[p["A"].row(i)].sum() for i in range(p["A"].nrows)])
    rows = np.unique(np.concatenate([np.argsort(flops)[-2:], np.argsort(flops)[:2],
                                     np.random.default_rng(1).choice(p["A"].nrows, 6, replace=False)])).astype(np.int32)
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64", complement=True, method=O.ESC, rows=rows)
    assert_parity(res, ref, "plus_times_i64", rows=rows)


def test_bfs_step_scale16_all_rows(handle):
    p = synth.bfs_step(scale=16, ef=16, nsrc=512, seed=17)
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64", complement=True, method=O.ESC)
    for force in ("auto", "msa"):
        handle.force(force)
        d = to_dev(p, "plus_times_i64")
        res = _lib.msgemm_run(handle, d["M"], d["A"], d["B"], "plus_times_i64", complement=True).trimmed()
        handle.sync_status()
        assert_parity(res, ref, "plus_times_i64", ctx=force)
    handle.force("auto")


def test_autograd_problem_scale14(handle):
    p = synth.autograd_problem(scale=14, ef=16, seed=23)
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
    d = to_dev(p, "plus_times_f32")
    res = _lib.msgemm_run(handle, d["M"], d["A"], d["B"], "plus_times_f32").trimmed()
    assert_parity(res, ref, "plus_times_f32")
    G = synth.Csr(p["M"].nrows, p["M"].ncols, ref["rowptr"].astype(np.int32), ref["colidx"],
                  synth.upstream_grad(len(ref["colidx"]), 23))
    dA_ref, dB_ref = O.grad(p["A"], p["B"], G)
    dA, dB = _lib.msgemm_backward(handle, d["A"], d["B"], _lib.DeviceCsr.from_host(G))
    handle.sync_status()
    SA, SB = O.grad(p["A"].with_values(np.abs(p["A"].values)), p["B"].with_values(np.abs(p["B"].values)),
                    G.with_values(np.abs(G.values)))
    assert np.all(np.abs(dA.cpu().numpy() - dA_ref) <= 1e-5 * SA + 1e-30)
    assert np.all(np.abs(dB.cpu().numpy() - dB_ref) <= 1e-5 * SB + 1e-30)


def test_batched_full_size_sampled_products(handle):
    ps = synth.batched_problems(nprod=256)
    devs = [to_dev(q, "plus_times_f32") for q in ps]
    outs = _lib.msgemm_run_batched(handle, [x["M"] for x in devs], [x["A"] for x in devs], [x["B"] for x in devs],
                                   "plus_times_f32")
    handle.sync_status()
    for pidx in (0, 1, 2, 100, 255):
        q = ps[pidx]
        ref = O.masked_spgemm(q["M"], q["A"], q["B"], "plus_times_f32")
        assert_parity(outs[pidx].trimmed(), ref, "plus_times_f32", ctx=f"product {pidx}")


@pytest.mark.parametrize("tile_index", [0, 1])
def test_tiled_rows_index_and_cursor_paths(handle, tile_index):
    """Rows wider than one shared-memory tile, walked through the per-row tile
    index of B (default) and through per-entry cursors (fallback)."""
    handle.set_option(_lib.OPT_TILE_INDEX, tile_index)
    try:
        p = synth.bfs_step(scale=16, ef=16, nsrc=256, seed=29)        # 65536 columns: 3 int64 tiles
        ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64", complement=True, method=O.ESC)
        handle.force("msa")
        d = to_dev(p, "plus_times_i64")
        res = _lib.msgemm_run(handle, d["M"], d["A"], d["B"], "plus_times_i64", complement=True).trimmed()
        handle.sync_status()
        assert_parity(res, ref, "plus_times_i64", ctx=f"bfs tile_index={tile_index}")
        for sr, gen in (("plus_times_f32", "f32"), ("plus_pair_i64", "pair")):
            q = synth.random_problem(900, 400, 120000, 20.0, 500.0, 60.0, 55, gen)
            ref = O.masked_spgemm(q["M"], q["A"], q["B"], sr)
            dq = to_dev(q, sr)
            res = _lib.msgemm_run(handle, dq["M"], dq["A"], dq["B"], sr).trimmed()
            handle.sync_status()
            assert_parity(res, ref, sr, ctx=f"{sr} tile_index={tile_index}")
    finally:
        handle.force("auto")
        handle.set_option(_lib.OPT_TILE_INDEX, 1)
