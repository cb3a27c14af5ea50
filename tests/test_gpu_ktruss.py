"""k-truss through the C ABI (msgemm_ktruss) against the oracle: the truss's
pattern, each edge's support and the number of rounds are exact (integer
work).  R-MAT graphs at several scales and k, a graph with self loops, a
complete graph, an empty graph."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2111_09947_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    h = _lib.Handle()
    yield h
    h.close()


def _check(h, g, k):
    A = _lib.DeviceCsr.from_host(synth.Csr(g.nrows, g.ncols, g.rowptr, g.colidx))
    res, rounds, products = _lib.msgemm_ktruss(h, A, k)
    h.sync_status()
    keep, sup, it = O.ktruss(g, k)
    rows = np.repeat(np.arange(g.nrows), np.diff(g.rowptr))
    rp = np.zeros(g.nrows + 1, np.int64)
    np.add.at(rp, rows[keep] + 1, 1)
    r = res.trimmed()
    assert np.array_equal(r.rowptr.cpu().numpy().astype(np.int64), np.cumsum(rp))
    assert np.array_equal(r.colidx.cpu().numpy(), g.colidx[keep])
    assert np.array_equal(r.values.cpu().numpy(), sup[keep])
    assert rounds == it
    assert products >= int(sup[keep].sum())
    return int(keep.sum())


@pytest.mark.parametrize("scale,k", [(9, 3), (11, 5), (13, 5), (12, 7)])
def test_rmat(handle, scale, k):
    g = synth.rmat_graph(scale, 16, 50 + scale, 1)
    _check(handle, g, k)


def test_self_loops_complete_and_empty(handle):
    n = 7
    rp = np.arange(0, n * n + 1, n).astype(np.int32)              # K7 with every self loop
    ci = np.tile(np.arange(n, dtype=np.int32), n)
    K = synth.Csr(n, n, rp, ci)
    assert _check(handle, K, 5) == n * (n - 1)                     # loops dropped, every edge kept
    assert _check(handle, K, 8) == 0                               # needs 6 triangles per edge
    E = synth.Csr(5, 5, np.zeros(6, np.int32), np.zeros(0, np.int32))
    assert _check(handle, E, 5) == 0
