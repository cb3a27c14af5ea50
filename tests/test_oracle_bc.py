"""Pins of the oracle's betweenness centrality (Brandes, the application of
Sec. 8.3), independent of its own code: closed forms on paths, stars and
complete graphs; networkx's Brandes implementation on random undirected and
directed graphs; additivity over source batches.  All sources are used where
a closed form or networkx gives the whole-graph value (ordered pairs: an
undirected graph counts each pair twice, networkx counts it once)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_09947_gb300 import synth


def _csr_from_edges(n, edges, symmetric=True):
    src = np.array([e[0] for e in edges], np.int64)
    dst = np.array([e[1] for e in edges], np.int64)
    if symmetric:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    keep = np.ones(len(src), bool)
    keep[1:] = (src[1:] != src[:-1]) | (dst[1:] != dst[:-1])
    src, dst = src[keep], dst[keep]
    rp = np.zeros(n + 1, np.int32)
    np.add.at(rp, src + 1, 1)
    return synth.Csr(n, n, np.cumsum(rp).astype(np.int32), dst.astype(np.int32))


def test_path_star_complete_closed_forms():
    n = 9
    P = _csr_from_edges(n, [(v, v + 1) for v in range(n - 1)])
    bc = O.bc(P, np.arange(n))
    assert np.allclose(bc, [2 * v * (n - 1 - v) for v in range(n)])
    S = _csr_from_edges(n, [(0, v) for v in range(1, n)])
    bc = O.bc(S, np.arange(n))
    assert np.isclose(bc[0], (n - 1) * (n - 2)) and np.allclose(bc[1:], 0)
    K = _csr_from_edges(n, [(a, b) for a in range(n) for b in range(a + 1, n)])
    assert np.allclose(O.bc(K, np.arange(n)), 0)
    # cycle of 4: each vertex lies on one shortest path of the two between its
    # neighbours (in both directions): 2 * 1/2 = 1
    C4 = _csr_from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)])
    assert np.allclose(O.bc(C4, np.arange(4)), 1.0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_against_networkx_undirected(seed):
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(seed)
    n = 70
    edges = [(a, b) for a in range(n) for b in range(a + 1, n) if rng.random() < 0.06]
    A = _csr_from_edges(n, edges)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from(edges)
    ref = nx.betweenness_centrality(G, normalized=False)
    bc = O.bc(A, np.arange(n))
    assert np.allclose(bc, [2 * ref[v] for v in range(n)], rtol=1e-12, atol=1e-9)


def test_against_networkx_directed_rmat():
    nx = pytest.importorskip("networkx")
    A = synth.rmat_directed(256, 6, 11, 1)
    G = nx.DiGraph()
    G.add_nodes_from(range(A.nrows))
    for v in range(A.nrows):
        for w in A.colidx[A.rowptr[v]:A.rowptr[v + 1]]:
            if w != v:
                G.add_edge(v, int(w))
    # self loops never lie on a shortest path; drop them from the CSR too
    keep = A.colidx != np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))[keep]
    A = _csr_from_edges(A.nrows, list(zip(rows.tolist(), A.colidx[keep].tolist())), symmetric=False)
    ref = nx.betweenness_centrality(G, normalized=False)
    assert np.allclose(O.bc(A, np.arange(A.nrows)), [ref[v] for v in range(A.nrows)], rtol=1e-12, atol=1e-9)


def test_additive_over_source_batches():
    g = synth.rmat_graph(9, 8, 5, 1)
    rng = np.random.default_rng(4)
    s = rng.choice(g.nrows, 40, replace=False)
    whole = O.bc(g, s)
    parts = O.bc(g, s[:17]) + O.bc(g, s[17:])
    assert np.allclose(whole, parts, rtol=1e-12, atol=1e-9)
    assert np.all(whole >= 0)
