"""Input generators: reproducibility and the structure each workload needs."""
import numpy as np

from paper_2111_09947_gb300 import synth


def _valid(c):
    assert c.rowptr[0] == 0 and np.all(np.diff(c.rowptr) >= 0)
    for i in range(c.nrows):
        r = c.row(i)
        assert np.all(np.diff(r) > 0) and (len(r) == 0 or (r[0] >= 0 and r[-1] < c.ncols))


def test_counter_rng_is_reproducible_and_addressable():
    k = synth.key(2111, 3)
    a = synth.uniform_f32(1000, 2111, 3)
    b = synth.uniform_f32(1000, 2111, 3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, synth.uniform_f32(1000, 2111, 4))
    assert a.min() >= -1.0 and a.max() < 1.0
    # values sit on the 2^-23 grid (exact in fp32 and fp64)
    assert np.all((a.astype(np.float64) + 1.0) * 2 ** 23 == np.round((a.astype(np.float64) + 1.0) * 2 ** 23))
    z = synth.normal_f32(200000, 1, 1)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1) < 0.02
    assert k == synth.key(2111, 3)


def test_erdos_renyi_density_and_validity():
    c = synth.er_pattern(4096, 4096, 8.0, 2111, 1)
    _valid(c)
    assert abs(c.nnz / 4096 - 8.0) < 0.3
    full = synth.er_pattern(5, 7, 7.0, 1, 1)
    assert full.nnz == 35


def test_rmat_graph_is_simple_and_symmetric():
    g = synth.rmat_graph(10, 16, seed=3)
    _valid(g)
    d = g.to_dense(np.int64) if False else g.pattern_dense()
    assert np.array_equal(d, d.T)
    assert not np.any(np.diag(d))
    # skewed degrees (R-MAT): max degree well above the mean
    deg = np.diff(g.rowptr)
    assert deg.max() > 8 * deg.mean()


def test_degree_relabel_lower():
    g = synth.rmat_graph(9, 8, seed=4)
    L = synth.degree_relabel_lower(g)
    _valid(L)
    assert L.nnz * 2 == g.nnz
    rows = np.repeat(np.arange(L.nrows), np.diff(L.rowptr))
    assert np.all(L.colidx < rows)
    # relabelled degrees are non-increasing in the new ids
    full = synth.coo_to_csr(L.nrows, L.ncols, rows, L.colidx, symmetrize=True)
    assert np.all(np.diff(np.diff(full.rowptr)) <= 0)


def test_bfs_frontier_structure():
    g = synth.rmat_graph(9, 8, seed=6)
    p = synth.bfs_step(graph=g, nsrc=16, seed=6)
    F, V = p["A"], p["M"]
    _valid(F)
    _valid(V)
    assert len(set(p["sources"].tolist())) == len(p["sources"])
    for q, s in enumerate(p["sources"].tolist()):
        assert s in V.row(q).tolist()
        assert set(F.row(q).tolist()) <= set(V.row(q).tolist())
        assert np.all(F.values[F.rowptr[q]:F.rowptr[q + 1]] >= 1)


def test_batched_sizes_span_range():
    ps = synth.batched_problems(nprod=12, seed=9, log2_range=(10, 12))
    ns = [p["n"] for p in ps]
    assert min(ns) >= 2 ** 10 and max(ns) <= 2 ** 12
    assert [p["dm"] for p in ps[:3]] == [1, 16, 256]
    for p in ps:
        _valid(p["A"])
        assert p["A"].nrows == p["B"].nrows == p["M"].nrows == p["n"]
