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


def test_autograd_problem_scale18_full(handle):
    """The differentiable workload at its full size (R-MAT scale 18, edge
    factor 16, fp32 N(0,1)): the forward C on every row, and dA, dB on every
    entry, against the fp64 oracle at the per-entry bounds 1e-5 * sum |a||b|
    (C), 1e-5 * sum |g||b| (dA) and 1e-5 * sum |a||g| (dB)."""
    p = synth.autograd_problem(scale=18, ef=16)
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
    d = to_dev(p, "plus_times_f32")
    res = _lib.msgemm_run(handle, d["M"], d["A"], d["B"], "plus_times_f32").trimmed()
    handle.sync_status()
    assert_parity(res, ref, "plus_times_f32", ctx="autograd scale 18 forward")
    G = synth.Csr(p["M"].nrows, p["M"].ncols, ref["rowptr"].astype(np.int32), ref["colidx"],
                  synth.upstream_grad(len(ref["colidx"])))
    dA_ref, dB_ref = O.grad(p["A"], p["B"], G)
    SA, SB = O.grad(p["A"].with_values(np.abs(p["A"].values)), p["B"].with_values(np.abs(p["B"].values)),
                    G.with_values(np.abs(G.values)))
    for rep in range(2):   # the second call reuses whatever the first left in the handle
        dA, dB = _lib.msgemm_backward(handle, d["A"], d["B"], _lib.DeviceCsr.from_host(G))
        handle.sync_status()
        eA = np.abs(dA.cpu().numpy().astype(np.float64) - dA_ref)
        eB = np.abs(dB.cpu().numpy().astype(np.float64) - dB_ref)
        assert np.all(eA <= 1e-5 * SA + 1e-30), f"dA: {(eA > 1e-5 * SA).sum()} entries outside (rep {rep})"
        assert np.all(eB <= 1e-5 * SB + 1e-30), f"dB: {(eB > 1e-5 * SB).sum()} entries outside (rep {rep})"


@pytest.mark.parametrize("use_graph", [False, True])
def test_batched_full_size_all_products(handle, use_graph):
    """The 256-product batch at its full size, every product against the
    oracle (eagerly, and replayed from a captured CUDA graph)."""
    ps = synth.batched_problems(nprod=256)
    devs = [to_dev(q, "plus_times_f32") for q in ps]
    args = ([x["M"] for x in devs], [x["A"] for x in devs], [x["B"] for x in devs])
    outs = _lib.msgemm_run_batched(handle, *args, "plus_times_f32", use_graph=use_graph)
    if use_graph:   # a second call replays the graph
        outs = _lib.msgemm_run_batched(handle, *args, "plus_times_f32", use_graph=True)
    handle.sync_status()
    assert handle.bin_counts()["mca_q"] > 0
    for pidx, q in enumerate(ps):
        ref = O.masked_spgemm(q["M"], q["A"], q["B"], "plus_times_f32")
        assert_parity(outs[pidx].trimmed(), ref, "plus_times_f32", ctx=f"product {pidx}")


@pytest.mark.parametrize("tile_index", [0, 1])
def test_tiled_rows_index_and_cursor_paths(handle, tile_index):
    """Rows wider than one shared-memory tile, walked through the per-row tile
    index of B (default) and through per-entry cursors (fallback)."""
    handle.set_option(_lib.OPT_TILE_INDEX, tile_index)
    try:
        p = synth.bfs_step(scale=16, ef=16, nsrc=256, seed=29)        # 65536 columns: 2 tiles
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


def _varied_rows(m, k, n, a_deg, m_deg, seed, gen):
    """A (m x k) and M (m x n) whose rows cycle through the given degrees,
    columns uniform without replacement; B (k x n) Erdos-Renyi, 400 per row."""
    rng = np.random.default_rng(seed)

    def csr(rows, ncols, degs):
        d = np.array([degs[i % len(degs)] for i in range(rows)], np.int64)
        rp = np.concatenate([[0], np.cumsum(d)]).astype(np.int32)
        ci = np.concatenate([np.sort(rng.choice(ncols, size=x, replace=False)) for x in d]).astype(np.int32) \
            if d.sum() else np.zeros(0, np.int32)
        return synth.Csr(rows, ncols, rp, ci)
    A, M = csr(m, k, a_deg), csr(m, n, m_deg)
    B = synth.er_pattern(k, n, 400.0, seed, 1)
    if gen == "f32":
        A = A.with_values(rng.uniform(-1, 1, A.nnz).astype(np.float32))
        B = B.with_values(rng.uniform(-1, 1, B.nnz).astype(np.float32))
    elif gen == "i64":
        A = A.with_values(rng.integers(-3, 4, A.nnz).astype(np.int64))
        B = B.with_values(rng.integers(-3, 4, B.nnz).astype(np.int64))
    return {"M": M, "A": A, "B": B}


@pytest.mark.parametrize("grid", [0, 1, 2])
@pytest.mark.parametrize("semiring", ["plus_times_i64", "plus_times_f32", "plus_pair_i64"])
def test_complemented_heavy_rows_grid_modes(handle, grid, semiring):
    """Heavy complemented rows: one CTA walking every tile of a row (grid 0),
    the tile-major grid of (row, tile) items for dense-output rows (1) or for
    every heavy row (2).  130000 columns: 3 tiles of 52000 columns (every
    semiring keeps 4 bytes per column in shared memory), the last partial.  A's rows give 400 to 240000 products (sparse to
    dense outputs); masks range from empty to half the columns."""
    gen = {"plus_times_i64": "i64", "plus_times_f32": "f32", "plus_pair_i64": "pair"}[semiring]
    q = _varied_rows(240, 3000, 130000, (1, 60, 600, 10, 300), (0, 2000, 65000, 50, 9000, 120000), 61, gen)
    ref = O.masked_spgemm(q["M"], q["A"], q["B"], semiring, complement=True, method=O.ESC)
    handle.set_option(_lib.OPT_GRID, grid)
    try:
        for force in ("msa", "auto"):
            handle.force(force)
            dq = to_dev(q, semiring)
            for rep in range(2):   # a second call finds the tile arrays as the first left them
                res = _lib.msgemm_run(handle, dq["M"], dq["A"], dq["B"], semiring, complement=True).trimmed()
                handle.sync_status()
                assert_parity(res, ref, semiring, ctx=f"grid={grid} force={force} rep={rep}")
            counts = handle.bin_counts()
            if grid == 2 and force == "msa":
                assert counts["cmsa_g"] > 0 and counts["cmsa_t"] == 0
            if grid == 1:
                assert counts["cmsa_g"] > 0
            if grid == 0:
                assert counts["cmsa_g"] == 0
    finally:
        handle.force("auto")
        handle.set_option(_lib.OPT_GRID, 1)


def test_bfs_grid_rows_scale16(handle):
    """The BFS step at scale 16 with the default policy: its heavy rows take
    the grid kind; every row against the oracle."""
    p = synth.bfs_step(scale=16, ef=16, nsrc=128, seed=30)
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64", complement=True, method=O.ESC)
    d = to_dev(p, "plus_times_i64")
    res = _lib.msgemm_run(handle, d["M"], d["A"], d["B"], "plus_times_i64", complement=True).trimmed()
    handle.sync_status()
    assert handle.bin_counts()["cmsa_g"] > 0
    assert_parity(res, ref, "plus_times_i64", ctx="bfs scale 16 grid")


@pytest.mark.parametrize("grid", [0, 2])
@pytest.mark.parametrize("complement", [False, True])
def test_int64_tiled_high_words(handle, grid, complement):
    """int64 through the column-tiled kinds, whose shared memory keeps only
    each column's low word: values near +-2^50 make every product carry a
    non-zero high half, sums wrap mod 2^64, and the high words must come back
    exactly and be cleared for the next row and call."""
    rng = np.random.default_rng(71 + grid + 2 * complement)
    q = _varied_rows(160, 2000, 120000, (3, 40, 400), (0, 900, 60000, 20), 72 + grid, "i64")
    big = np.int64(1) << np.int64(50)
    q["A"] = q["A"].with_values(rng.integers(-big, big, q["A"].nnz, dtype=np.int64))
    q["B"] = q["B"].with_values(rng.integers(-(1 << 12), 1 << 12, q["B"].nnz, dtype=np.int64))
    method = O.ESC if complement else O.MERGE
    ref = O.masked_spgemm(q["M"], q["A"], q["B"], "plus_times_i64", complement=complement, method=method)
    handle.set_option(_lib.OPT_GRID, grid)
    try:
        handle.force("msa")
        dq = to_dev(q, "plus_times_i64")
        for rep in range(2):
            res = _lib.msgemm_run(handle, dq["M"], dq["A"], dq["B"], "plus_times_i64", complement=complement).trimmed()
            handle.sync_status()
            assert_parity(res, ref, "plus_times_i64", ctx=f"grid={grid} complement={complement} rep={rep}")
    finally:
        handle.force("auto")
        handle.set_option(_lib.OPT_GRID, 1)


@pytest.mark.parametrize("grid", [0, 1, 2])
@pytest.mark.parametrize("semiring", ["plus_times_f32", "plus_times_i64", "plus_pair_i64"])
def test_plain_heavy_rows_grid_modes(handle, grid, semiring):
    """Heavy plain-mask rows of a product wider than one tile: one CTA per row
    (grid 0), (row, tile) items for rows over the flop bound (1, bound lowered
    so the heavy rows qualify) or for every CTA row (2)."""
    gen = {"plus_times_i64": "i64", "plus_times_f32": "f32", "plus_pair_i64": "pair"}[semiring]
    q = _varied_rows(200, 3000, 130000, (2, 60, 900, 20), (0, 30, 4000, 60000, 700), 81 + grid, gen)
    ref = O.masked_spgemm(q["M"], q["A"], q["B"], semiring)
    handle.set_option(_lib.OPT_GRID, grid)
    handle.set_option(_lib.OPT_GRID_MIN_FLOPS, 1 << 16)
    try:
        for force in ("auto", "msa"):
            handle.force(force)
            dq = to_dev(q, semiring)
            for rep in range(2):
                res = _lib.msgemm_run(handle, dq["M"], dq["A"], dq["B"], semiring).trimmed()
                handle.sync_status()
                assert_parity(res, ref, semiring, ctx=f"grid={grid} force={force} rep={rep}")
            counts = handle.bin_counts()
            if grid == 0:
                assert counts["msa_g"] == 0
            else:
                assert counts["msa_g"] > 0
    finally:
        handle.force("auto")
        handle.set_option(_lib.OPT_GRID, 1)
        handle.set_option(_lib.OPT_GRID_MIN_FLOPS, 1 << 20)


def test_backward_through_grid_rows(tmp_path):
    """Gradient form (values written at each mask entry's own slot) through
    the (row, tile) items: every row made a CTA row by a policy loaded from an
    autotuner cache (warp flop bound 0), grid mode 2; dA and dB against the
    oracle's closed forms."""
    import json
    m, k, n = 150, 60000, 60000
    p = synth.random_problem(m, k, n, 300.0, 3.0, 30.0, 315, "f32")
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
    G = synth.Csr(m, n, ref["rowptr"].astype(np.int32), ref["colidx"], synth.upstream_grad(len(ref["colidx"]), 3))
    dA_ref, dB_ref = O.grad(p["A"], p["B"], G)
    d = to_dev(p, "plus_times_f32")
    cache = tmp_path / "policy.json"
    entry = {"warp_flops_max": 0, "dot_ratio": 2, "warp_slab": 4608, "grid_min_flops": 1 << 20,
             "pref": [[1, 2, 3, 0]] * 16}
    cache.write_text(json.dumps({torch.cuda.get_device_name() + "|plus_times_f32": entry}))
    h = _lib.Handle()
    try:
        _lib.msgemm_autotune(h, [], [], [], "plus_times_f32", cache_path=cache)
        h.set_option(_lib.OPT_GRID, 2)
        dA, dB = _lib.msgemm_backward(h, d["A"], d["B"], _lib.DeviceCsr.from_host(G))
        h.sync_status()
        assert h.bin_counts()["msa_g"] > 0
    finally:
        h.close()
    Aabs = p["A"].with_values(np.abs(p["A"].values))
    Babs = p["B"].with_values(np.abs(p["B"].values))
    Gabs = G.with_values(np.abs(G.values))
    SA, SB = O.grad(Aabs, Babs, Gabs)
    assert np.all(np.abs(dA.cpu().numpy() - dA_ref) <= 1e-5 * SA + 1e-30)
    assert np.all(np.abs(dB.cpu().numpy() - dB_ref) <= 1e-5 * SB + 1e-30)


@pytest.mark.parametrize("complement", [True, False])
@pytest.mark.parametrize("values", ["small_positive", "carry", "f32_positive"])
def test_grid_speculation_paths(handle, complement, values):
    """Dense grid tiles (push work per tile >= 8x the tile width) first run
    without SET bits: small positive values stay on that path; a value that
    carries into the int64 high word forces the tracked rerun (and stops
    speculation for the launch); positive fp32 stays speculative."""
    semiring = "plus_times_f32" if values == "f32_positive" else "plus_times_i64"
    gen = "f32" if values == "f32_positive" else "i64"
    q = _varied_rows(16, 4000, 130000, (3900,), (0, 3000, 60000), 91, gen)
    rng = np.random.default_rng(92)
    if gen == "i64":
        q["A"] = q["A"].with_values(rng.integers(1, 4, q["A"].nnz).astype(np.int64))
        q["B"] = q["B"].with_values(rng.integers(1, 4, q["B"].nnz).astype(np.int64))
        if values == "carry":
            va = q["A"].values.copy()
            va[len(va) // 2] = np.int64(1) << np.int64(40)
            q["A"] = q["A"].with_values(va)
    else:
        q["A"] = q["A"].with_values(rng.uniform(0.5, 1.5, q["A"].nnz).astype(np.float32))
        q["B"] = q["B"].with_values(rng.uniform(0.5, 1.5, q["B"].nnz).astype(np.float32))
    ref = O.masked_spgemm(q["M"], q["A"], q["B"], semiring, complement=complement,
                          method=O.ESC if complement else O.MERGE)
    handle.set_option(_lib.OPT_GRID, 2)
    try:
        dq = to_dev(q, semiring)
        res = _lib.msgemm_run(handle, dq["M"], dq["A"], dq["B"], semiring, complement=complement).trimmed()
        handle.sync_status()
        assert handle.bin_counts()["cmsa_g" if complement else "msa_g"] > 0
        assert_parity(res, ref, semiring, ctx=f"{values} complement={complement}")
    finally:
        handle.set_option(_lib.OPT_GRID, 1)
