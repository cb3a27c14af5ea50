"""Pins of the oracle's k-truss (Sec. 8.2, k = 5 in the paper's benchmark):
closed forms on complete graphs and on a clique with pendant structure, and
networkx's k_truss on random graphs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_09947_gb300 import synth
from test_oracle_bc import _csr_from_edges


def _edges(A, keep):
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    return {(int(u), int(v)) for u, v, kk in zip(rows, A.colidx, keep) if kk and u < v}


def test_complete_graphs():
    K6 = _csr_from_edges(6, [(a, b) for a in range(6) for b in range(a + 1, 6)])
    keep, sup, _ = O.ktruss(K6, 5)
    assert keep.all() and (sup == 4).all()          # each edge of K6 lies on 4 triangles
    keep, _, _ = O.ktruss(K6, 7)
    assert not keep.any()                            # needs 5 triangles per edge
    K4 = _csr_from_edges(4, [(a, b) for a in range(4) for b in range(a + 1, 4)])
    assert not O.ktruss(K4, 5)[0].any()


def test_clique_with_tails_and_triangles():
    # K5 on 0..4, a triangle 5-6-7 hanging off vertex 0, a path 8-9-10 off 4
    edges = [(a, b) for a in range(5) for b in range(a + 1, 5)]
    edges += [(0, 5), (5, 6), (6, 7), (7, 5), (4, 8), (8, 9), (9, 10)]
    A = _csr_from_edges(11, edges)
    keep, sup, it = O.ktruss(A, 5)
    assert _edges(A, keep) == {(a, b) for a in range(5) for b in range(a + 1, 5)}
    keep3, _, _ = O.ktruss(A, 3)                     # 3-truss: every edge on a triangle
    assert _edges(A, keep3) == {(a, b) for a in range(5) for b in range(a + 1, 5)} | {(5, 6), (6, 7), (5, 7)}


@pytest.mark.parametrize("seed,k", [(1, 4), (2, 5), (3, 6)])
def test_against_networkx(seed, k):
    nx = pytest.importorskip("networkx")
    g = synth.rmat_graph(8, 12, seed, 1)
    rows = np.repeat(np.arange(g.nrows), np.diff(g.rowptr))
    G = nx.Graph()
    G.add_edges_from((int(u), int(v)) for u, v in zip(rows, g.colidx) if u < v)
    ref = {tuple(sorted(e)) for e in nx.k_truss(G, k).edges()}
    keep, sup, _ = O.ktruss(g, k)
    assert _edges(g, keep) == ref
    assert (sup[keep] >= k - 2).all()
