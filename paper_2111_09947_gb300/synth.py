"""Seeded synthetic workloads for masked SpGEMM (host side, numpy arrays).

The paper evaluates on Erdos-Renyi and Graph500 R-MAT graphs (Sec. 7) and on
SuiteSparse matrices; the generators here produce the synthetic families with
the shapes of its workloads: the Erdos-Renyi density grid (Sec. 8.1), triangle
counting on a degree-relabelled strict lower triangle (Sec. 8.2) and the
complemented-mask forward step of multi-source betweenness centrality
(Sec. 8.4).  Matrices are CSR with int32 indices, rows sorted and free of
duplicates.  The generator code is C (``synth.c``, SplitMix64 counter-based
stream per (seed, stream id)); this file only marshals arrays.

Nothing here computes a masked product: both the CUDA path and the CPU oracle
consume these arrays.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
from typing import Optional

import numpy as np

from . import _build

BASE_SEED = 2111

# Stream ids: one per matrix role, fixed so that every workload is reproducible.
S_A, S_B, S_M, S_AV, S_BV, S_G, S_SRC, S_BATCH = 1, 2, 3, 4, 5, 6, 7, 8

RMAT_ABC = (0.57, 0.19, 0.19)

_lib: Optional[C.CDLL] = None


def _load() -> C.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    path = _build.SYNTH_LIB
    if not os.path.exists(path):
        _build.build_synth()
    lib = C.CDLL(path)
    u64, i64, i32, f64, vp = C.c_uint64, C.c_int64, C.c_int, C.c_double, C.c_void_p
    sig = {
        "synth_key": (u64, [u64, u64]),
        "synth_draw": (u64, [u64, u64]),
        "synth_uniform_f32": (None, [u64, i64, vp]),
        "synth_normal_f32": (None, [u64, i64, vp]),
        "synth_er_count": (i64, [u64, i64, i64, f64, vp]),
        "synth_er_fill": (None, [u64, i64, i64, f64, vp, vp]),
        "synth_rmat": (i64, [u64, i32, i64, i64, f64, f64, f64, vp, vp]),
        "synth_coo_to_csr": (i64, [i64, i64, vp, vp, i32, i32, vp, vp]),
        "synth_degree_order": (None, [i64, vp, vp]),
        "synth_relabel_coo": (i64, [i64, vp, vp, vp, i32, vp, vp]),
        "synth_pick_sources": (i64, [u64, i64, vp, i64, vp]),
        "synth_bfs2": (None, [i64, vp, vp, i64, vp, i32, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclasses.dataclass
class Csr:
    """Host CSR matrix: int32 rowptr/colidx, optional values (float32 or int64)."""
    nrows: int
    ncols: int
    rowptr: np.ndarray
    colidx: np.ndarray
    values: Optional[np.ndarray] = None

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1]) if len(self.rowptr) else 0

    def row(self, i: int) -> np.ndarray:
        return self.colidx[self.rowptr[i]:self.rowptr[i + 1]]

    def with_values(self, values: Optional[np.ndarray]) -> "Csr":
        return Csr(self.nrows, self.ncols, self.rowptr, self.colidx, values)

    def to_dense(self, dtype=np.float64) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols), dtype=dtype)
        rows = np.repeat(np.arange(self.nrows), np.diff(self.rowptr))
        vals = self.values if self.values is not None else np.ones(self.nnz)
        d[rows, self.colidx] = vals
        return d

    def pattern_dense(self) -> np.ndarray:
        d = np.zeros((self.nrows, self.ncols), dtype=bool)
        rows = np.repeat(np.arange(self.nrows), np.diff(self.rowptr))
        d[rows, self.colidx] = True
        return d


def key(seed: int, stream: int) -> int:
    return int(_load().synth_key(seed & (2**64 - 1), stream))


def uniform_f32(count: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(count, np.float32)
    if count:
        _load().synth_uniform_f32(key(seed, stream), count, _p(out))
    return out


def normal_f32(count: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(count, np.float32)
    if count:
        _load().synth_normal_f32(key(seed, stream), count, _p(out))
    return out


def er_pattern(m: int, n: int, d: float, seed: int, stream: int) -> Csr:
    """Erdos-Renyi m x n pattern, each entry present with probability d / n."""
    lib = _load()
    k = key(seed, stream)
    rp = np.empty(m + 1, np.int64)
    nnz = lib.synth_er_count(k, m, n, float(d), _p(rp))
    ci = np.empty(max(nnz, 1), np.int32)
    lib.synth_er_fill(k, m, n, float(d), _p(rp), _p(ci))
    return Csr(m, n, rp.astype(np.int32), ci[:nnz])


def coo_to_csr(nrows: int, ncols: int, src: np.ndarray, dst: np.ndarray,
               symmetrize: bool = False, drop_loops: bool = False) -> Csr:
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    ne = len(src)
    rp = np.empty(nrows + 1, np.int32)
    ci = np.empty(max(1, ne * (2 if symmetrize else 1)), np.int32)
    nnz = _load().synth_coo_to_csr(nrows, ne, _p(src), _p(dst), int(symmetrize), int(drop_loops),
                                   _p(rp), _p(ci))
    return Csr(nrows, ncols, rp, ci[:nnz].copy())


def rmat_edges(scale: int, n: int, nedges: int, seed: int, stream: int,
               abc=RMAT_ABC) -> tuple[np.ndarray, np.ndarray]:
    src = np.empty(max(nedges, 1), np.int32)
    dst = np.empty(max(nedges, 1), np.int32)
    kept = _load().synth_rmat(key(seed, stream), scale, n, nedges, *abc, _p(src), _p(dst))
    return src[:kept], dst[:kept]


def rmat_graph(scale: int, ef: int, seed: int = BASE_SEED, stream: int = S_A) -> Csr:
    """Undirected R-MAT graph: ef * 2^scale edges, symmetrised, loops and
    duplicates removed (pattern only)."""
    n = 1 << scale
    s, d = rmat_edges(scale, n, ef * n, seed, stream)
    return coo_to_csr(n, n, s, d, symmetrize=True, drop_loops=True)


def rmat_directed(n: int, ef: int, seed: int, stream: int) -> Csr:
    """Directed R-MAT pattern on n vertices (n need not be a power of two):
    ef * n edges drawn at scale ceil(log2 n), endpoints >= n rejected,
    duplicates removed, self-loops kept."""
    scale = max(1, math.ceil(math.log2(max(n, 2))))
    s, d = rmat_edges(scale, n, ef * n, seed, stream)
    return coo_to_csr(n, n, s, d)


def degree_relabel_lower(g: Csr) -> Csr:
    """Relabels vertices by non-increasing degree (ties: ascending id) and
    returns the strict lower triangle L of the relabelled adjacency."""
    lib = _load()
    n = g.nrows
    new_id = np.empty(n, np.int32)
    lib.synth_degree_order(n, _p(g.rowptr), _p(new_id))
    src = np.empty(max(g.nnz, 1), np.int32)
    dst = np.empty(max(g.nnz, 1), np.int32)
    cnt = lib.synth_relabel_coo(n, _p(g.rowptr), _p(g.colidx), _p(new_id), 1, _p(src), _p(dst))
    return coo_to_csr(n, n, src[:cnt], dst[:cnt])


def strict_lower(g: Csr) -> Csr:
    """Strict lower triangle of g without relabelling."""
    rows = np.repeat(np.arange(g.nrows, dtype=np.int32), np.diff(g.rowptr))
    keep = g.colidx < rows
    return coo_to_csr(g.nrows, g.ncols, rows[keep], g.colidx[keep])


def transpose_pattern(a: Csr) -> Csr:
    rows = np.repeat(np.arange(a.nrows, dtype=np.int32), np.diff(a.rowptr))
    return coo_to_csr(a.ncols, a.nrows, a.colidx, rows)


def pick_sources(g: Csr, nsrc: int, seed: int, stream: int = S_SRC) -> np.ndarray:
    out = np.empty(max(nsrc, 1), np.int32)
    got = _load().synth_pick_sources(key(seed, stream), g.nrows, _p(g.rowptr), nsrc, _p(out))
    return out[:got]


def bfs_frontier(g: Csr, sources: np.ndarray) -> tuple[Csr, Csr]:
    """Two-level BFS from each source: returns (F, Visited), both
    len(sources) x n.  Row s of F holds level-2 vertices with their shortest
    path counts sigma (int64); row s of Visited holds levels 0, 1 and 2."""
    lib = _load()
    n, q = g.nrows, len(sources)
    sources = np.ascontiguousarray(sources, np.int32)
    frp = np.empty(q + 1, np.int64)
    vrp = np.empty(q + 1, np.int64)
    lib.synth_bfs2(n, _p(g.rowptr), _p(g.colidx), q, _p(sources), 0, _p(frp), None, None, _p(vrp), None)
    fci = np.empty(max(int(frp[-1]), 1), np.int32)
    fsg = np.empty(max(int(frp[-1]), 1), np.int64)
    vci = np.empty(max(int(vrp[-1]), 1), np.int32)
    lib.synth_bfs2(n, _p(g.rowptr), _p(g.colidx), q, _p(sources), 1, _p(frp), _p(fci), _p(fsg), _p(vrp), _p(vci))
    F = Csr(q, n, frp.astype(np.int32), fci[:frp[-1]], fsg[:frp[-1]])
    V = Csr(q, n, vrp.astype(np.int32), vci[:vrp[-1]])
    return F, V


# ---------------------------------------------------------------------------
# Workloads.  Each returns plain Csr objects; values are generated on the host
# so that every consumer sees identical bytes.

def random_problem(m: int, k: int, n: int, da: float, db: float, dm: float, seed: int,
                   semiring: str = "f32") -> dict:
    """Independent Erdos-Renyi A (m x k), B (k x n), M (m x n) with values for
    the semiring: f32 -> uniform[-1, 1); i64 -> small signed integers; pair -> none."""
    A = er_pattern(m, k, da, seed, S_A)
    B = er_pattern(k, n, db, seed, S_B)
    M = er_pattern(m, n, dm, seed, S_M)
    if semiring == "f32":
        A = A.with_values(uniform_f32(A.nnz, seed, S_AV))
        B = B.with_values(uniform_f32(B.nnz, seed, S_BV))
    elif semiring == "i64":
        A = A.with_values(np.floor(uniform_f32(A.nnz, seed, S_AV) * 8).astype(np.int64))
        B = B.with_values(np.floor(uniform_f32(B.nnz, seed, S_BV) * 8).astype(np.int64))
    return {"M": M, "A": A, "B": B}


def er_plain_f32(n: int = 4096, d: float = 8.0, seed: int = BASE_SEED) -> dict:
    """Plain fp32 masked product on independent Erdos-Renyi A, B, M (n x n,
    average d entries per row, values uniform[-1, 1))."""
    return random_problem(n, n, n, d, d, d, seed, "f32")


def triangle_counting(scale: int = 20, ef: int = 16, seed: int = BASE_SEED, relabel: bool = True) -> dict:
    """L = strict lower triangle of an undirected R-MAT graph (degree
    relabelled); the masked product is C = L .* (L L) on plus-pair."""
    g = rmat_graph(scale, ef, seed, S_A)
    L = degree_relabel_lower(g) if relabel else strict_lower(g)
    return {"M": L, "A": L, "B": L, "graph_nnz": g.nnz}


def bfs_step(scale: int = 20, ef: int = 16, nsrc: int = 512, seed: int = BASE_SEED,
             graph: Optional[Csr] = None) -> dict:
    """One complemented-mask step of multi-source BFS: C = !Visited .* (F A) on
    plus-times int64, with A the undirected R-MAT adjacency (values 1) and F
    the level-2 frontier of nsrc random sources carrying path counts."""
    g = graph if graph is not None else rmat_graph(scale, ef, seed, S_A)
    src = pick_sources(g, nsrc, seed)
    F, V = bfs_frontier(g, src)
    A = g.with_values(np.ones(g.nnz, np.int64))
    return {"M": V, "A": F, "B": A, "sources": src, "graph": g}


def autograd_problem(scale: int = 18, ef: int = 16, seed: int = BASE_SEED) -> dict:
    """A: directed R-MAT (duplicates removed) with N(0,1) fp32 values;
    B: pattern of A^T with fresh N(0,1) values; M: pattern of A."""
    n = 1 << scale
    A = rmat_directed(n, ef, seed, S_A)
    A = A.with_values(normal_f32(A.nnz, seed, S_AV))
    Bp = transpose_pattern(A)
    B = Bp.with_values(normal_f32(Bp.nnz, seed, S_BV))
    M = Csr(A.nrows, A.ncols, A.rowptr, A.colidx)
    return {"M": M, "A": A, "B": B}


def upstream_grad(nnz: int, seed: int = BASE_SEED) -> np.ndarray:
    return normal_f32(nnz, seed, S_G)


def batched_problems(nprod: int = 256, seed: int = BASE_SEED, ef: int = 8,
                     mask_degrees=(1, 16, 256), log2_range=(10, 16)) -> list[dict]:
    """nprod independent fp32 products.  Product p: n = round(2^s) with s
    uniform in log2_range; A, B directed R-MAT (ef * n edges); M Erdos-Renyi
    with average degree mask_degrees[p % 3]; values uniform[-1, 1)."""
    out = []
    kb = key(seed, S_BATCH)
    lo, hi = log2_range
    lib = _load()
    for p in range(nprod):
        u = (int(lib.synth_draw(kb, p)) >> 11) * (1.0 / 9007199254740992.0)
        n = int(round(2.0 ** (lo + (hi - lo) * u)))
        ps = seed * 1000003 + p
        A = rmat_directed(n, ef, ps, S_A)
        B = rmat_directed(n, ef, ps, S_B)
        dm = mask_degrees[p % len(mask_degrees)]
        M = er_pattern(n, n, dm, ps, S_M)
        A = A.with_values(uniform_f32(A.nnz, ps, S_AV))
        B = B.with_values(uniform_f32(B.nnz, ps, S_BV))
        out.append({"M": M, "A": A, "B": B, "n": n, "dm": dm})
    return out
