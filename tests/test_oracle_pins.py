"""Pins of the CPU oracle against facts that do not come from the oracle.

* dense brute force (numpy matmul) on tiny rectangular inputs, every
  semiring, both mask forms, both oracle algorithms;
* triangle counts with closed forms (Sec. 8.2: count = sum(L .* L^2)):
  K_n -> C(n, 3), complete bipartite -> 0, cycles -> 0, wheels -> rim size;
* an independent node-iterator triangle count on small R-MAT graphs;
* the complement partition C_M + C_!M = A B with disjoint patterns;
* the BFS meaning of a complemented step (Sec. 8.4): the row of source s is
  the level-3 vertex set with its shortest-path counts, from a plain BFS;
* gradients: exact central differences of the bilinear loss on dyadic data,
  and fp64 central differences on an R-MAT scale-8 problem.
"""
import itertools
import math
from collections import deque

import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_09947_gb300 import synth
from paper_2111_09947_gb300.synth import Csr
from dense_ref import dense_masked, to_dense_result

SEMIRINGS = ["plus_times_f32", "plus_times_i64", "plus_pair_i64"]


def tiny_cases():
    shapes = [(1, 1, 1), (3, 5, 4), (7, 2, 9), (16, 16, 16), (5, 0, 6), (0, 4, 3), (12, 20, 8), (33, 17, 40)]
    dens = [(0.5, 0.5, 0.5), (3.0, 3.0, 2.0), (1.0, 4.0, 8.0), (100.0, 100.0, 100.0), (0.0, 2.0, 2.0)]
    seed = 10
    for (m, k, n), (da, db, dm) in itertools.product(shapes, dens):
        seed += 1
        yield m, k, n, da, db, dm, seed


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("complement", [False, True])
def test_oracle_vs_dense_bruteforce(semiring, complement):
    methods = [O.ESC] if complement else [O.MERGE, O.ESC]
    sr_gen = {"plus_times_f32": "f32", "plus_times_i64": "i64", "plus_pair_i64": "pair"}[semiring]
    ncase = 0
    for m, k, n, da, db, dm, seed in tiny_cases():
        p = synth.random_problem(m, k, n, min(da, max(k, 1)), min(db, max(n, 1)), min(dm, max(n, 1)), seed, sr_gen)
        M, A, B = p["M"], p["A"], p["B"]
        present, vals, S = dense_masked(M, A, B, semiring, complement)
        for meth in methods:
            res = O.masked_spgemm(M, A, B, semiring, complement=complement, method=meth)
            # rows sorted ascending
            for i in range(m):
                row = res["colidx"][res["rowptr"][i]:res["rowptr"][i + 1]]
                assert np.all(np.diff(row) > 0)
            got_p, got_v = to_dense_result(res, m, n, np.float64 if semiring == "plus_times_f32" else np.int64)
            assert np.array_equal(got_p, present), (m, k, n, seed, meth)
            if semiring == "plus_times_f32":
                np.testing.assert_allclose(got_v[present], vals[present], rtol=0, atol=1e-12)
                got_S, _ = None, None
                Sd = np.zeros((m, n))
                rows = np.repeat(np.arange(m), np.diff(res["rowptr"]))
                Sd[rows, res["colidx"]] = res["S"]
                np.testing.assert_allclose(Sd[present], S[present], rtol=1e-12, atol=0)
            else:
                assert np.array_equal(got_v[present], vals[present])
        ncase += 1
    assert ncase >= 40


def test_structural_zero_sum_is_kept():
    # a_00 * b_00 + a_01 * b_10 = 1*1 + 1*(-1) = 0: entry present with value 0
    A = Csr(1, 2, np.array([0, 2], np.int32), np.array([0, 1], np.int32), np.array([1, 1], np.int64))
    B = Csr(2, 1, np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([1, -1], np.int64))
    M = Csr(1, 1, np.array([0, 1], np.int32), np.array([0], np.int32))
    for meth in (O.MERGE, O.ESC):
        r = O.masked_spgemm(M, A, B, "plus_times_i64", method=meth)
        assert list(r["colidx"]) == [0] and list(r["values"]) == [0]


def test_mask_entry_without_product_is_absent():
    # Fig. 1: the mask may hold entries for which the product yields nothing
    A = Csr(2, 2, np.array([0, 1, 1], np.int32), np.array([0], np.int32), np.array([2.0], np.float32))
    B = Csr(2, 2, np.array([0, 1, 1], np.int32), np.array([1], np.int32), np.array([3.0], np.float32))
    M = Csr(2, 2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32))
    r = O.masked_spgemm(M, A, B, "plus_times_f32")
    assert list(r["rowptr"]) == [0, 1, 1] and list(r["colidx"]) == [1] and r["values"][0] == 6.0


def test_validation_flags_bad_inputs():
    good = Csr(2, 3, np.array([0, 2, 3], np.int32), np.array([0, 2, 1], np.int32))
    assert O.validate(good) == 0
    assert O.validate(Csr(2, 3, np.array([0, 2, 3], np.int32), np.array([2, 0, 1], np.int32))) == 3
    assert O.validate(Csr(2, 3, np.array([0, 2, 3], np.int32), np.array([0, 0, 1], np.int32))) == 3
    assert O.validate(Csr(2, 3, np.array([0, 2, 3], np.int32), np.array([0, 3, 1], np.int32))) == 2
    assert O.validate(Csr(2, 3, np.array([0, 3, 2], np.int32), np.array([0, 1, 2], np.int32))) == 1
    with pytest.raises(O.OracleError):
        O.masked_spgemm(good, Csr(2, 2, np.array([0, 2, 2], np.int32), np.array([1, 0], np.int32)),
                        Csr(2, 3, np.array([0, 0, 0], np.int32), np.array([], np.int32)), "plus_pair_i64")


# ---------------------------------------------------------------- triangles

def graph_from_edges(n, edges):
    src = np.array([e[0] for e in edges], np.int32)
    dst = np.array([e[1] for e in edges], np.int32)
    return synth.coo_to_csr(n, n, src, dst, symmetrize=True, drop_loops=True)


def tc_oracle(g, relabel=True):
    L = synth.degree_relabel_lower(g) if relabel else synth.strict_lower(g)
    r = O.masked_spgemm(L, L, L, "plus_pair_i64")
    return int(r["values"].astype(np.uint64).sum())


@pytest.mark.parametrize("relabel", [True, False])
def test_triangle_closed_forms(relabel):
    for n in (3, 4, 5, 10, 50):
        g = graph_from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
        assert tc_oracle(g, relabel) == math.comb(n, 3)
    for a, b in ((1, 1), (3, 4), (10, 7)):
        g = graph_from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)])
        assert tc_oracle(g, relabel) == 0
    for n in (4, 5, 9, 100):
        g = graph_from_edges(n, [(i, (i + 1) % n) for i in range(n)])
        assert tc_oracle(g, relabel) == 0
    for r in (4, 5, 17):
        edges = [(0, 1 + i) for i in range(r)] + [(1 + i, 1 + (i + 1) % r) for i in range(r)]
        assert tc_oracle(graph_from_edges(r + 1, edges), relabel) == r


def node_iterator_triangles(g):
    adj = [set(g.row(v).tolist()) for v in range(g.nrows)]
    t = 0
    for v in range(g.nrows):
        for u in adj[v]:
            if u > v:
                t += sum(1 for w in adj[v] & adj[u] if w > u)
    return t


@pytest.mark.parametrize("scale", [6, 8, 10])
def test_triangles_vs_node_iterator(scale):
    g = synth.rmat_graph(scale, 16, seed=77 + scale)
    assert tc_oracle(g, True) == node_iterator_triangles(g) == tc_oracle(g, False)


# ---------------------------------------------------------------- complement

@pytest.mark.parametrize("semiring", ["plus_times_i64", "plus_pair_i64"])
def test_complement_partition(semiring):
    sr_gen = "i64" if semiring == "plus_times_i64" else "pair"
    for seed, (m, k, n, d) in enumerate([(40, 30, 50, 4.0), (64, 64, 64, 8.0), (25, 60, 33, 12.0)]):
        p = synth.random_problem(m, k, n, d, d, d, 500 + seed, sr_gen)
        M, A, B = p["M"], p["A"], p["B"]
        cm = O.masked_spgemm(M, A, B, semiring, complement=False, method=O.MERGE)
        cn = O.masked_spgemm(M, A, B, semiring, complement=True, method=O.ESC)
        empty = Csr(m, n, np.zeros(m + 1, np.int32), np.zeros(0, np.int32))
        full = O.masked_spgemm(empty, A, B, semiring, complement=True, method=O.ESC)
        pm, vm = to_dense_result(cm, m, n, np.int64)
        pn, vn = to_dense_result(cn, m, n, np.int64)
        pf, vf = to_dense_result(full, m, n, np.int64)
        assert not np.any(pm & pn)
        assert np.array_equal(pm | pn, pf)
        assert np.array_equal(vm + vn, vf)
        # the unmasked product equals the dense product on its pattern
        Ad = A.to_dense(np.int64) if semiring == "plus_times_i64" else A.pattern_dense().astype(np.int64)
        Bd = B.to_dense(np.int64) if semiring == "plus_times_i64" else B.pattern_dense().astype(np.int64)
        assert np.array_equal(vf, np.where(pf, Ad @ Bd, 0))


def test_merge_and_esc_agree_midsize():
    p = synth.random_problem(600, 500, 700, 9.0, 11.0, 20.0, 4242, "f32")
    a = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32", method=O.MERGE)
    b = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32", method=O.ESC)
    assert np.array_equal(a["rowptr"], b["rowptr"]) and np.array_equal(a["colidx"], b["colidx"])
    # same ascending-k summation order in both: identical fp64 sums
    assert np.array_equal(a["values"], b["values"])


def test_row_selection_matches_full():
    p = synth.random_problem(300, 200, 250, 6.0, 6.0, 30.0, 99, "i64")
    full = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64")
    rows = np.array([5, 0, 299, 17, 17], np.int32)
    part = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64", rows=rows)
    for r, i in enumerate(rows):
        a = slice(full["rowptr"][i], full["rowptr"][i + 1])
        b = slice(part["rowptr"][r], part["rowptr"][r + 1])
        assert np.array_equal(full["colidx"][a], part["colidx"][b])
        assert np.array_equal(full["values"][a], part["values"][b])


# ---------------------------------------------------------------- BFS step

def bfs_levels(g, s, depth):
    level = {s: 0}
    sigma = {s: 1}
    frontier = [s]
    for d in range(1, depth + 1):
        nxt = {}
        for u in frontier:
            for v in g.row(u).tolist():
                if v in level and level[v] < d:
                    continue
                if v not in nxt:
                    nxt[v] = 0
                nxt[v] += sigma[u]
        for v, c in nxt.items():
            level[v] = d
            sigma[v] = c
        frontier = sorted(nxt)
    return level, sigma


def test_bfs_step_is_level3_with_path_counts():
    g = synth.rmat_graph(10, 8, seed=31)
    p = synth.bfs_step(graph=g, nsrc=24, seed=31)
    F, V, A = p["A"], p["M"], p["B"]
    res = O.masked_spgemm(V, F, A, "plus_times_i64", complement=True, method=O.ESC)
    for q, s in enumerate(p["sources"].tolist()):
        level, sigma = bfs_levels(g, s, 3)
        l2 = sorted(v for v, d in level.items() if d == 2)
        assert F.row(q).tolist() == l2
        assert F.values[F.rowptr[q]:F.rowptr[q + 1]].tolist() == [sigma[v] for v in l2]
        l3 = sorted(v for v, d in level.items() if d == 3)
        row = slice(res["rowptr"][q], res["rowptr"][q + 1])
        assert res["colidx"][row].tolist() == l3
        assert res["values"][row].tolist() == [sigma[v] for v in l3]


# ---------------------------------------------------------------- gradients

def loss(M, A, B, G):
    """l = sum_ij G_ij C_ij, C = M .* (A B), from the oracle's forward (fp64)."""
    c = O.masked_spgemm(M, A, B, "plus_times_f32")
    Gd = G.to_dense(np.float64)
    rows = np.repeat(np.arange(M.nrows), np.diff(c["rowptr"]))
    return float(np.sum(Gd[rows, c["colidx"]] * c["values"]))


def test_gradients_exact_central_differences_dyadic():
    # dyadic values (multiples of 1/8 in [-2, 2)) make every product and sum
    # exact, and the loss is bilinear, so central differences are exact.
    m, k, n = 9, 7, 11
    p = synth.random_problem(m, k, n, 3.0, 3.0, 6.0, 1234, "f32")
    M, A, B = p["M"], p["A"], p["B"]
    A = A.with_values((np.round(A.values * 16) / 8).astype(np.float32))
    B = B.with_values((np.round(B.values * 16) / 8).astype(np.float32))
    c = O.masked_spgemm(M, A, B, "plus_times_f32")
    G = Csr(m, n, c["rowptr"].astype(np.int32), c["colidx"],
            (np.round(synth.uniform_f32(len(c["colidx"]), 1234, synth.S_G) * 16) / 8).astype(np.float32))
    dA, dB = O.grad(A, B, G)
    h = 0.5
    for t in range(A.nnz):
        ap, am = A.values.copy(), A.values.copy()
        ap[t] += h
        am[t] -= h
        fd = (loss(M, A.with_values(ap), B, G) - loss(M, A.with_values(am), B, G)) / (2 * h)
        assert fd == dA[t]
    for t in range(B.nnz):
        bp, bm = B.values.copy(), B.values.copy()
        bp[t] += h
        bm[t] -= h
        fd = (loss(M, A, B.with_values(bp), G) - loss(M, A, B.with_values(bm), G)) / (2 * h)
        assert fd == dB[t]
    # dense closed form: dA = pattern(A) .* (Gd B^T), dB = pattern(B) .* (A^T Gd)
    Gd, Ad, Bd = G.to_dense(), A.to_dense(), B.to_dense()
    rows = np.repeat(np.arange(m), np.diff(A.rowptr))
    assert np.array_equal(dA, (Gd @ Bd.T)[rows, A.colidx])
    rows = np.repeat(np.arange(k), np.diff(B.rowptr))
    assert np.array_equal(dB, (Ad.T @ Gd)[rows, B.colidx])


def test_gradients_fd_rmat_scale8():
    p = synth.autograd_problem(scale=8, ef=16, seed=5)
    M, A, B = p["M"], p["A"], p["B"]
    c = O.masked_spgemm(M, A, B, "plus_times_f32")
    G = Csr(M.nrows, M.ncols, c["rowptr"].astype(np.int32), c["colidx"], synth.upstream_grad(len(c["colidx"]), 5))
    dA, dB = O.grad(A, B, G)
    # l is linear in each A entry: its partial is exact from any two points.
    # Rows of C touched by A_ik are row i only, so evaluate single rows.
    Gd = G.to_dense(np.float64)
    h = 2.0 ** -3
    rng = np.random.default_rng(0)
    for t in rng.choice(A.nnz, size=min(A.nnz, 300), replace=False):
        i = int(np.searchsorted(A.rowptr, t, side="right") - 1)
        vals = []
        for s in (+h, -h):
            av = A.values.astype(np.float64).copy()
            av[t] += s
            # exact in fp32 only if representable: fall back to fp64 dense row
            Arow = np.zeros(A.ncols)
            Arow[A.row(i)] = av[A.rowptr[i]:A.rowptr[i + 1]]
            crow = Arow @ B.to_dense(np.float64)
            mrow = np.zeros(M.ncols, bool)
            mrow[M.row(i)] = True
            vals.append(float(np.sum(Gd[i] * crow * mrow)))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dA[t]) <= 1e-9 * (1 + abs(fd))
    Bd = B.to_dense(np.float64)
    Ad = A.to_dense(np.float64)
    Mp = M.pattern_dense()
    for t in rng.choice(B.nnz, size=min(B.nnz, 300), replace=False):
        kk = int(np.searchsorted(B.rowptr, t, side="right") - 1)
        j = int(B.colidx[t])
        vals = []
        for s in (+h, -h):
            col = Bd[:, j].copy()
            col[kk] += s
            ccol = Ad @ col
            vals.append(float(np.sum(Gd[:, j] * ccol * Mp[:, j])))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - dB[t]) <= 1e-9 * (1 + abs(fd))
