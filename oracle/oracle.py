"""ctypes wrapper of the CPU oracle (oracle.c) -- TEST INFRASTRUCTURE.

Only tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this module.  It shares no code with the CUDA library.

Matrices are passed as any object with ``nrows``, ``ncols``, ``rowptr``,
``colidx`` and ``values`` attributes holding numpy arrays (int32 indices;
float32 values for plus-times fp32, int64 for plus-times int64, ignored for
plus-pair and for the mask).
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

from . import build as _build

PT_F32, PT_I64, PP_I64 = 0, 1, 2
MERGE, ESC = 0, 1
SEMIRINGS = {"plus_times_f32": PT_F32, "plus_times_i64": PT_I64, "plus_pair_i64": PP_I64}
ERRORS = {1: "bad rowptr", 2: "column out of range", 3: "unsorted or duplicate columns",
          4: "bad arguments", 5: "out of memory"}

_lib: Optional[C.CDLL] = None


def _load() -> C.CDLL:
    global _lib
    if _lib is None:
        path = _build.build()
        lib = C.CDLL(path)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
        lib.oracle_masked_spgemm.restype = vp
        lib.oracle_masked_spgemm.argtypes = [i32, i32, i32, i64, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp,
                                             i64, vp, C.POINTER(C.c_int)]
        lib.oracle_result_nrows.restype = i64
        lib.oracle_result_nrows.argtypes = [vp]
        lib.oracle_result_nnz.restype = i64
        lib.oracle_result_nnz.argtypes = [vp]
        lib.oracle_result_copy.restype = None
        lib.oracle_result_copy.argtypes = [vp, vp, vp, vp, vp]
        lib.oracle_result_free.restype = None
        lib.oracle_result_free.argtypes = [vp]
        lib.oracle_validate_csr.restype = i32
        lib.oracle_validate_csr.argtypes = [i64, i64, vp, vp]
        lib.oracle_grad.restype = i32
        lib.oracle_grad.argtypes = [i64, i64, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.oracle_bc.argtypes = [i64, vp, vp, i64, vp, vp]
        lib.oracle_ktruss.argtypes = [i64, vp, vp, i64, vp, vp, vp]
        lib.oracle_ktruss.restype = i32
        lib.oracle_bc.restype = i32
        lib.oracle_set_threads.restype = None
        lib.oracle_set_threads.argtypes = [i32]
        _lib = lib
    return _lib


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (results do not
    depend on it)."""
    _load().oracle_set_threads(int(n))


def _arr(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def _ptr(a) -> Optional[int]:
    return None if a is None else a.ctypes.data


class OracleError(RuntimeError):
    pass


def _sr(semiring) -> int:
    return SEMIRINGS[semiring] if isinstance(semiring, str) else int(semiring)


def validate(mat) -> int:
    rp = _arr(mat.rowptr, np.int32)
    ci = _arr(mat.colidx, np.int32)
    return int(_load().oracle_validate_csr(mat.nrows, mat.ncols, _ptr(rp), _ptr(ci)))


def masked_spgemm(M, A, B, semiring, complement: bool = False, method: int = MERGE,
                  rows: Optional[np.ndarray] = None) -> dict:
    """C = M .* (A B) (or !M .* (A B)).  Returns dict(rowptr int64, colidx
    int32, values float64|int64, S float64|None).  With ``rows`` only those
    rows of C are computed, in the given order."""
    sr = _sr(semiring)
    lib = _load()
    if not (M.nrows == A.nrows and A.ncols == B.nrows and M.ncols == B.ncols):
        raise OracleError("shape mismatch")
    vdt = np.float32 if sr == PT_F32 else np.int64
    Mrp, Mci = _arr(M.rowptr, np.int32), _arr(M.colidx, np.int32)
    Arp, Aci = _arr(A.rowptr, np.int32), _arr(A.colidx, np.int32)
    Brp, Bci = _arr(B.rowptr, np.int32), _arr(B.colidx, np.int32)
    Av = _arr(A.values, vdt) if sr != PP_I64 else None
    Bv = _arr(B.values, vdt) if sr != PP_I64 else None
    sel = _arr(rows, np.int32)
    err = C.c_int(0)
    h = lib.oracle_masked_spgemm(sr, int(bool(complement)), int(method), A.nrows, A.ncols, B.ncols,
                                 _ptr(Mrp), _ptr(Mci), _ptr(Arp), _ptr(Aci), _ptr(Av),
                                 _ptr(Brp), _ptr(Bci), _ptr(Bv),
                                 0 if sel is None else len(sel), _ptr(sel), C.byref(err))
    if not h:
        raise OracleError(ERRORS.get(err.value, f"error {err.value}"))
    try:
        nr = lib.oracle_result_nrows(h)
        nnz = lib.oracle_result_nnz(h)
        rp = np.empty(nr + 1, np.int64)
        ci = np.empty(nnz, np.int32)
        vals = np.empty(nnz, np.float64 if sr == PT_F32 else np.int64)
        S = np.empty(nnz, np.float64) if sr == PT_F32 else None
        lib.oracle_result_copy(h, _ptr(rp), _ptr(ci), _ptr(vals), _ptr(S))
    finally:
        lib.oracle_result_free(h)
    return {"rowptr": rp, "colidx": ci, "values": vals, "S": S}


def grad(A, B, G) -> tuple[np.ndarray, np.ndarray]:
    """Gradients of l = sum G_ij C_ij for C = M .* (A B) (fp32 inputs, fp64
    result).  G is stored on C's pattern.  Returns (dA aligned with A's
    storage, dB aligned with B's storage)."""
    lib = _load()
    Arp, Aci, Av = _arr(A.rowptr, np.int32), _arr(A.colidx, np.int32), _arr(A.values, np.float32)
    Brp, Bci, Bv = _arr(B.rowptr, np.int32), _arr(B.colidx, np.int32), _arr(B.values, np.float32)
    Grp, Gci, Gv = _arr(G.rowptr, np.int32), _arr(G.colidx, np.int32), _arr(G.values, np.float32)
    dA = np.empty(len(Aci), np.float64)
    dB = np.empty(len(Bci), np.float64)
    e = lib.oracle_grad(A.nrows, A.ncols, B.ncols, _ptr(Arp), _ptr(Aci), _ptr(Av), _ptr(Brp), _ptr(Bci), _ptr(Bv),
                        _ptr(Grp), _ptr(Gci), _ptr(Gv), _ptr(dA), _ptr(dB))
    if e:
        raise OracleError(ERRORS.get(e, f"error {e}"))
    return dA, dB


def bc(A, sources) -> np.ndarray:
    """Betweenness centrality of every vertex from the given sources (Brandes,
    fp64; the application benchmarked in Sec. 8.3): for each source s, the
    dependencies delta_s(v) of a breadth-first search over the stored entries
    of A (edge v -> w for entry (v, w)); bc(v) = sum over sources s != v of
    delta_s(v)."""
    lib = _load()
    if A.nrows != A.ncols:
        raise OracleError("shape mismatch")
    rp, ci = _arr(A.rowptr, np.int32), _arr(A.colidx, np.int32)
    src = _arr(sources, np.int32)
    out = np.zeros(A.nrows, np.float64)
    err = lib.oracle_bc(A.nrows, _ptr(rp), _ptr(ci), len(src), _ptr(src), _ptr(out))
    if err:
        raise OracleError(ERRORS.get(err, f"error {err}"))
    return out


def ktruss(A, k: int):
    """k-truss of a symmetric pattern A (Sec. 8.2): the largest subgraph where
    every edge lies on at least k - 2 of its triangles, by repeated support
    counting and pruning.  Returns (keep mask over A's entries, final support
    per entry, iterations)."""
    lib = _load()
    if A.nrows != A.ncols:
        raise OracleError("shape mismatch")
    rp, ci = _arr(A.rowptr, np.int32), _arr(A.colidx, np.int32)
    keep = np.zeros(len(ci), np.uint8)
    sup = np.zeros(len(ci), np.int64)
    it = np.zeros(1, np.int64)
    err = lib.oracle_ktruss(A.nrows, _ptr(rp), _ptr(ci), int(k), _ptr(keep), _ptr(sup), _ptr(it))
    if err:
        raise OracleError(ERRORS.get(err, f"error {err}"))
    return keep.astype(bool), sup, int(it[0])
