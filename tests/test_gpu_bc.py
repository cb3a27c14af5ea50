"""Batched betweenness centrality through the C ABI (msgemm_bc) against the
oracle's Brandes: undirected R-MAT graphs (the BFS workload's graph family),
a directed graph, a path (closed form), repeated and single sources, empty
batches.  The forward path counts are exact (int64); the backward runs the
fp32 semiring on positive terms only, so each level adds at most
(k + 3) u relative error (u = 2^-24: k - 1 for a sum of k terms in any order,
one each for 1/sigma, the sum with T and the product with sigma), and a
centrality is within D (Delta + 4) u of the oracle's, relatively, for D
levels and maximum degree Delta."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2111_09947_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def handle():
    h = _lib.Handle()
    yield h
    h.close()


def _check(h, g, sources):
    A = _lib.DeviceCsr.from_host(synth.Csr(g.nrows, g.ncols, g.rowptr, g.colidx))
    bc, levels = _lib.msgemm_bc(h, A, torch.from_numpy(np.asarray(sources, np.int32)).cuda())
    h.sync_status()
    ref = O.bc(g, sources)
    got = bc.cpu().numpy()
    delta = 0
    if g.nrows and len(g.colidx):   # terms of a sum: in- or out-neighbours
        delta = int(max(np.diff(g.rowptr).max(), np.bincount(g.colidx, minlength=g.ncols).max()))
    rel = max(levels, 1) * (delta + 4) * 2.0 ** -24
    err = np.abs(got - ref)
    assert np.all(err <= rel * np.abs(ref) + 1e-12), (float(err.max()), rel)
    return levels


@pytest.mark.parametrize("scale,nsrc", [(8, 16), (11, 64), (13, 200)])
def test_undirected_rmat(handle, scale, nsrc):
    g = synth.rmat_graph(scale, 16, 31 + scale, 1)
    src = synth.pick_sources(g, nsrc, 7)
    levels = _check(handle, g, src)
    assert levels >= 2


def test_directed_and_path(handle):
    A = synth.rmat_directed(2048, 8, 5, 1)
    rng = np.random.default_rng(2)
    _check(handle, A, rng.choice(2048, 50, replace=False))
    n = 300   # path: closed form 2 v (n - 1 - v) with every vertex a source
    rp = np.concatenate([[0], np.cumsum([1] + [2] * (n - 2) + [1])]).astype(np.int32)
    ci = np.concatenate([[1]] + [[v - 1, v + 1] for v in range(1, n - 1)] + [[n - 2]]).astype(np.int32)
    P = synth.Csr(n, n, rp, ci)
    levels = _check(handle, P, np.arange(n))
    assert levels == n


def test_repeated_single_and_empty_sources(handle):
    g = synth.rmat_graph(10, 8, 41, 1)
    s = synth.pick_sources(g, 5, 3)
    _check(handle, g, np.concatenate([s, s[:2]]))   # repeats count twice, as in the oracle
    _check(handle, g, s[:1])
    A = _lib.DeviceCsr.from_host(synth.Csr(g.nrows, g.ncols, g.rowptr, g.colidx))
    bc, levels = _lib.msgemm_bc(handle, A, torch.zeros(0, dtype=torch.int32, device="cuda"))
    assert levels == 0 and float(bc.abs().sum()) == 0.0
    with pytest.raises(_lib.MsgemmError):
        _lib.msgemm_bc(handle, A, torch.tensor([g.nrows], dtype=torch.int32, device="cuda"))


def test_bfs_workload_graph_scale16(handle):
    p = synth.bfs_step(scale=16, ef=16, nsrc=128, seed=30)
    _check(handle, p["graph"], p["sources"])
