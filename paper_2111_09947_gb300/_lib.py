"""ctypes binding of the C ABI in include/msgemm.h (argument marshalling only).

Every step of the computation runs in the CUDA library ``libmsgemm.so``; this
module converts torch tensors to the ABI's plain structs, supplies torch's
caching allocator as the library's allocation callbacks, and wraps outputs
back into tensors.  A missing library is an error: there is no CPU fallback.
"""
from __future__ import annotations

import bisect
import ctypes as C
import weakref
import os
from collections.abc import Sequence
from dataclasses import dataclass
from typing import Optional

import torch

from . import _build

PLUS_TIMES_F32, PLUS_TIMES_I64, PLUS_PAIR_I64 = 0, 1, 2
SEMIRINGS = {"plus_times_f32": PLUS_TIMES_F32, "plus_times_i64": PLUS_TIMES_I64, "plus_pair_i64": PLUS_PAIR_I64}
ACC_AUTO, ACC_MSA, ACC_HASH, ACC_MCA, ACC_DOT, ACC_HEAP, ACC_HEAPDOT = 0, 1, 2, 3, 4, 5, 6
ACCUMULATORS = {"auto": 0, "msa": 1, "hash": 2, "mca": 3, "dot": 4, "heap": 5, "heapdot": 6}
OPT_FORCE_ACCUM, OPT_VALIDATE, OPT_DOT, OPT_PROFILE, OPT_TILE_INDEX, OPT_GRID, OPT_WARP_SLAB, OPT_GRID_MIN_FLOPS = 1, 2, 3, 4, 5, 6, 7, 8
OPT_PHASES = 9
OPT_HASH_KICKS = 10
OPT_QTEAM_FLOPS = 11
OPT_HASH_SLAB = 12
STATUS = {0: "OK", 1: "ERR_INVALID", 2: "ERR_SHAPE", 3: "ERR_UNSORTED", 4: "ERR_UNSUPPORTED", 5: "ERR_OOM",
          6: "ERR_OVERFLOW", 7: "ERR_CUDA", 8: "ERR_TIMEOUT"}
KIND_NAMES = ["empty", "msa_w", "msa_t", "hash_w", "hash_b", "mca_w", "mca_b", "dot_w", "dot_b",
              "chash_w", "chash_b", "cmsa_t", "cmsa_g", "msa_g", "heap_w", "heapdot_w", "cheap_w", "mca_q", "dot_q",
              "hash_l"]

# Exported symbols that include/msgemm.h declares.
EXPORTS = ["msgemm_create", "msgemm_set_stream", "msgemm_set_option", "msgemm_run", "msgemm_backward",
           "msgemm_run_batched", "msgemm_autotune", "msgemm_transpose", "msgemm_reduce_sum",
           "msgemm_sync_status", "msgemm_last_error_detail", "msgemm_num_kinds", "msgemm_bin_counts",
           "msgemm_profile_count", "msgemm_profile_entry", "msgemm_last_row_kinds", "msgemm_kernel_launches",
           "msgemm_transpose_noalloc", "msgemm_bc", "msgemm_ktruss", "msgemm_destroy",
           "msgemm_backward_plan_create", "msgemm_backward_planned", "msgemm_backward_plan_destroy"]


class MsgemmError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"{STATUS.get(status, status)}: {detail}")


class Csr(C.Structure):
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("colidx", C.c_void_p), ("values", C.c_void_p)]


class CsrOut(C.Structure):
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("rowptr", C.c_void_p), ("colidx", C.c_void_p),
                ("values", C.c_void_p), ("capacity", C.c_int64), ("d_nnz", C.c_void_p)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib: Optional[C.CDLL] = None


def lib_path() -> str:
    return _build.CUDA_LIB


def load(build_if_missing: bool = False) -> C.CDLL:
    """Loads libmsgemm.so; raises if it is absent (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        if build_if_missing:
            _build.build_cuda()
        else:
            raise ImportError(f"{path} is missing: build it with __graft_entry__.build() "
                              "(the masked SpGEMM has no CPU fallback)")
    lib = C.CDLL(path)
    vp, i32, i64, sz = C.c_void_p, C.c_int, C.c_int64, C.c_size_t
    P = C.POINTER
    sigs = {
        "msgemm_create": (i32, [P(vp), vp, ALLOC_FN, FREE_FN, vp]),
        "msgemm_set_stream": (i32, [vp, vp]),
        "msgemm_set_option": (i32, [vp, i32, i64]),
        "msgemm_run": (i32, [vp, P(Csr), i32, P(Csr), P(Csr), i32, P(CsrOut)]),
        "msgemm_backward": (i32, [vp, P(Csr), P(Csr), P(Csr), i32, vp, vp]),
        "msgemm_run_batched": (i32, [vp, i32, P(Csr), vp, P(Csr), P(Csr), i32, P(CsrOut), i32]),
        "msgemm_autotune": (i32, [vp, i32, P(Csr), vp, P(Csr), P(Csr), i32, C.c_char_p]),
        "msgemm_transpose": (i32, [vp, P(Csr), i32, i32, P(CsrOut)]),
        "msgemm_reduce_sum": (i32, [vp, P(CsrOut), i32, vp]),
        "msgemm_sync_status": (i32, [vp]),
        "msgemm_last_error_detail": (i32, [vp, C.c_char_p, sz]),
        "msgemm_num_kinds": (i32, []),
        "msgemm_bin_counts": (i32, [vp, P(i64), i32]),
        "msgemm_profile_count": (i32, [vp]),
        "msgemm_profile_entry": (i32, [vp, i32, C.c_char_p, sz, P(C.c_float)]),
        "msgemm_last_row_kinds": (i32, [vp, vp, i64]),
        "msgemm_kernel_launches": (i64, []),
        "msgemm_transpose_noalloc": (i32, [P(Csr), i32, i32, vp, vp, vp, vp]),
        "msgemm_bc": (i32, [vp, P(Csr), vp, i32, vp, P(C.c_int32)]),
        "msgemm_ktruss": (i32, [vp, P(Csr), i64, P(CsrOut), P(C.c_int32), P(C.c_int64)]),
        "msgemm_destroy": (None, [vp]),
        "msgemm_backward_plan_create": (i32, [vp, P(Csr), P(Csr), P(vp)]),
        "msgemm_backward_planned": (i32, [vp, vp, P(Csr), P(Csr), P(Csr), vp, vp]),
        "msgemm_backward_plan_destroy": (None, [vp, vp]),
    }
    for name, (res, args) in sigs.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


@dataclass
class DeviceCsr:
    """CSR matrix on the device: int32 rowptr/colidx, optional values."""
    nrows: int
    ncols: int
    rowptr: torch.Tensor
    colidx: torch.Tensor
    values: Optional[torch.Tensor] = None

    @property
    def nnz(self) -> int:
        return int(self.colidx.numel())

    def abi(self) -> Csr:
        # the checked struct is kept while the fields hold the same objects
        sig = (self.nrows, self.ncols, id(self.rowptr), id(self.colidx), id(self.values))
        memo = self.__dict__.get("_abi")
        if memo is not None and memo[0] == sig:
            return memo[1]
        for t in (self.rowptr, self.colidx):
            assert t.is_cuda and t.dtype == torch.int32 and t.is_contiguous()
        v = self.values
        if v is not None:
            assert v.is_cuda and v.is_contiguous() and v.numel() == self.nnz
        c = Csr(self.nrows, self.ncols, self.nnz, self.rowptr.data_ptr(),
                self.colidx.data_ptr() if self.nnz else 0, v.data_ptr() if v is not None and self.nnz else 0)
        self.__dict__["_abi"] = (sig, c)
        return c

    @staticmethod
    def from_host(m, device="cuda", values_dtype=None) -> "DeviceCsr":
        """From any host CSR with numpy rowptr/colidx/values attributes."""
        rp = torch.from_numpy(m.rowptr).to(device=device, dtype=torch.int32)
        ci = torch.from_numpy(m.colidx).to(device=device, dtype=torch.int32)
        v = None
        if m.values is not None:
            v = torch.from_numpy(m.values)
            if values_dtype is not None:
                v = v.to(values_dtype)
            v = v.to(device)
        return DeviceCsr(m.nrows, m.ncols, rp.contiguous(), ci.contiguous(), v)


_ESIZE: dict = {}


def _esize(dtype: torch.dtype) -> int:
    n = _ESIZE.get(dtype)
    if n is None:
        n = _ESIZE[dtype] = torch.empty((), dtype=dtype).element_size()
    return n


class _Blocks:
    """Output allocations taken over from the library; product arrays are
    views into them."""

    def __init__(self):
        self.base: list[int] = []
        self.mem: list[torch.Tensor] = []

    def add(self, ptr: int, t: torch.Tensor):
        i = bisect.bisect(self.base, ptr)
        self.base.insert(i, ptr)
        self.mem.insert(i, t)

    def view(self, ptr: int, dtype: torch.dtype, count: int) -> torch.Tensor:
        i = bisect.bisect(self.base, ptr) - 1
        if i < 0:
            raise KeyError("pointer outside the output allocations")
        off = ptr - self.base[i]
        nb = count * _esize(dtype)
        raw = self.mem[i]
        if off + nb > raw.numel():
            raise KeyError("array outside its allocation")
        return raw[off:off + nb].view(dtype)

    def result(self, out: CsrOut, out_dtype: torch.dtype) -> "Result":
        cap = out.capacity
        return Result(out.nrows, out.ncols, self.view(out.rowptr, torch.int32, out.nrows + 1),
                      self.view(out.colidx, torch.int32, cap), self.view(out.values, out_dtype, cap),
                      self.view(out.d_nnz, torch.int64, 1))


class BatchResult(Sequence):
    """Outputs of msgemm_run_batched; each product's Result is made on first
    access (views into the batch's shared allocations)."""

    def __init__(self, blocks: _Blocks, outs, out_dtype: torch.dtype):
        self._blocks, self._outs, self._dt = blocks, outs, out_dtype
        self._cache: dict[int, "Result"] = {}

    def __len__(self):
        return len(self._outs)

    def __getitem__(self, p):
        if isinstance(p, slice):
            return [self[i] for i in range(*p.indices(len(self)))]
        if p < 0:
            p += len(self)
        if not 0 <= p < len(self):
            raise IndexError(p)
        r = self._cache.get(p)
        if r is None:
            r = self._cache[p] = self._blocks.result(self._outs[p], self._dt)
        return r


@dataclass
class Result:
    """Output CSR: tensors sized to the capacity; nnz is a device scalar."""
    nrows: int
    ncols: int
    rowptr: torch.Tensor
    colidx: torch.Tensor
    values: torch.Tensor
    d_nnz: torch.Tensor

    def nnz(self) -> int:
        return int(self.d_nnz.item())

    def trimmed(self) -> DeviceCsr:
        k = self.nnz()
        return DeviceCsr(self.nrows, self.ncols, self.rowptr, self.colidx[:k], self.values[:k])


class Handle:
    """Owns a msgemm handle bound to the current device; allocations go
    through torch's caching allocator on the current stream."""

    def __init__(self, device: Optional[torch.device] = None):
        self.lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self._live: dict[int, torch.Tensor] = {}
        self._plans = weakref.WeakSet()   # backward plans made with this handle
        self._alloc_cb = ALLOC_FN(self._alloc)
        self._free_cb = FREE_FN(self._free)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            st = torch.cuda.current_stream().cuda_stream
            self._check(self.lib.msgemm_create(C.byref(h), st, self._alloc_cb, self._free_cb, None), None)
        self.h = h

    def _alloc(self, nbytes, ctx):
        try:
            t = torch.empty(int(nbytes), dtype=torch.uint8, device=self.device)
        except RuntimeError:
            return None
        p = t.data_ptr()
        self._live[p] = t
        return p

    def _free(self, ptr, ctx):
        self._live.pop(ptr, None)

    def _check(self, status, h):
        if status != 0:
            detail = ""
            if h is not None:
                buf = C.create_string_buffer(512)
                self.lib.msgemm_last_error_detail(h, buf, 512)
                detail = buf.value.decode(errors="replace")
            raise MsgemmError(status, detail)

    def check(self, status):
        self._check(status, self.h)

    def bind_stream(self):
        self.check(self.lib.msgemm_set_stream(self.h, torch.cuda.current_stream(self.device).cuda_stream))

    def set_option(self, opt: int, value: int):
        self.check(self.lib.msgemm_set_option(self.h, opt, int(value)))

    def force(self, accumulator: str):
        self.set_option(OPT_FORCE_ACCUM, ACCUMULATORS[accumulator])

    def adopt(self, ptr: int, dtype: torch.dtype, count: int) -> torch.Tensor:
        """Takes ownership of a library-allocated output buffer as a tensor."""
        raw = self._live.pop(ptr)
        return raw.view(dtype)[:count] if count else raw.view(dtype)[:0]

    def claim(self, outs) -> "_Blocks":
        """Takes ownership of the allocations that hold these outputs' arrays
        (a batch carves each array kind of all its products from one
        allocation whose base is the first product's array)."""
        blocks = _Blocks()
        live = self._live
        for o in outs:
            for ptr in (o.rowptr, o.colidx, o.values, o.d_nnz):
                if ptr and ptr in live:
                    blocks.add(ptr, live.pop(ptr))
        return blocks

    def result(self, out: CsrOut, out_dtype: torch.dtype) -> Result:
        return self.claim([out]).result(out, out_dtype)

    def sync_status(self):
        self.check(self.lib.msgemm_sync_status(self.h))

    def bin_counts(self) -> dict:
        n = self.lib.msgemm_num_kinds()
        arr = (C.c_int64 * n)()
        self.check(self.lib.msgemm_bin_counts(self.h, arr, n))
        return {KIND_NAMES[k] if k < len(KIND_NAMES) else str(k): int(arr[k]) for k in range(n)}

    def profile(self) -> list:
        """[(phase name, device ms)] of the last call made with profiling on."""
        out = []
        for i in range(self.lib.msgemm_profile_count(self.h)):
            buf = C.create_string_buffer(64)
            ms = C.c_float()
            self.check(self.lib.msgemm_profile_entry(self.h, i, buf, 64, C.byref(ms)))
            out.append((buf.value.decode(), float(ms.value)))
        return out

    def row_kinds(self, nrows: int):
        import numpy as np
        out = np.empty(nrows, np.uint8)
        self.check(self.lib.msgemm_last_row_kinds(self.h, out.ctypes.data if nrows else None, nrows))
        return out

    def close(self):
        if getattr(self, "h", None):
            for plan in list(self._plans):   # their memory came from this handle
                plan.close()
            self.lib.msgemm_destroy(self.h)
            self.h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def out_dtype(semiring: int) -> torch.dtype:
    return torch.float32 if semiring == PLUS_TIMES_F32 else torch.int64


def _sr(semiring) -> int:
    return SEMIRINGS[semiring] if isinstance(semiring, str) else int(semiring)


def msgemm_run(h: Handle, M: DeviceCsr, A: DeviceCsr, B: DeviceCsr, semiring="plus_times_f32",
               complement: bool = False) -> Result:
    """C = M .* (A B) (or !M .* (A B)) through msgemm_run."""
    sr = _sr(semiring)
    h.bind_stream()
    m, a, b = M.abi(), A.abi(), B.abi()
    out = CsrOut()
    h.check(h.lib.msgemm_run(h.h, C.byref(m), int(bool(complement)), C.byref(a), C.byref(b), sr, C.byref(out)))
    return h.result(out, out_dtype(sr))


class BackwardPlan:
    """Transposed patterns of A and B for repeated backward passes
    (msgemm_backward_plan_create); keeps A, B and the handle alive and is
    destroyed before its handle closes."""

    def __init__(self, h: Handle, A: DeviceCsr, B: DeviceCsr):
        self.h, self.A, self.B = h, A, B
        self.p = None
        h.bind_stream()
        p = C.c_void_p()
        a, b = A.abi(), B.abi()
        h.check(h.lib.msgemm_backward_plan_create(h.h, C.byref(a), C.byref(b), C.byref(p)))
        self.p = p
        h._plans.add(self)

    def close(self):
        if self.p is not None and getattr(self.h, "h", None):
            self.h.lib.msgemm_backward_plan_destroy(self.h.h, self.p)
        self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def msgemm_backward(h: Handle, A: DeviceCsr, B: DeviceCsr, G: DeviceCsr, need_dA=True, need_dB=True,
                    plan: Optional[BackwardPlan] = None):
    """(dA values aligned with A's storage, dB values aligned with B's).
    With a plan made for A's and B's patterns the transposes are not rebuilt."""
    h.bind_stream()
    dA = torch.empty(A.nnz, dtype=torch.float32, device=A.colidx.device) if need_dA else None
    dB = torch.empty(B.nnz, dtype=torch.float32, device=B.colidx.device) if need_dB else None
    a, b, g = A.abi(), B.abi(), G.abi()
    pa = dA.data_ptr() if dA is not None and dA.numel() else None
    pb = dB.data_ptr() if dB is not None and dB.numel() else None
    if plan is not None:
        if plan.p is None:
            raise MsgemmError(1, "backward plan is closed")
        h.check(h.lib.msgemm_backward_planned(h.h, plan.p, C.byref(a), C.byref(b), C.byref(g), pa, pb))
    else:
        h.check(h.lib.msgemm_backward(h.h, C.byref(a), C.byref(b), C.byref(g), PLUS_TIMES_F32, pa, pb))
    return dA, dB


def msgemm_run_batched(h: Handle, Ms, As, Bs, semiring="plus_times_f32", complement=None, use_graph=False):
    sr = _sr(semiring)
    h.bind_stream()
    n = len(Ms)
    marr = (Csr * n)(*[x.abi() for x in Ms])
    aarr = (Csr * n)(*[x.abi() for x in As])
    barr = (Csr * n)(*[x.abi() for x in Bs])
    outs = (CsrOut * n)()
    comp = None
    if complement is not None:
        comp = (C.c_int * n)(*[int(bool(c)) for c in complement])
    h.check(h.lib.msgemm_run_batched(h.h, n, marr, comp, aarr, barr, sr, outs, int(bool(use_graph))))
    return BatchResult(h.claim(outs), outs, out_dtype(sr))


def msgemm_autotune(h: Handle, Ms, As, Bs, semiring="plus_times_f32", complement=None, cache_path=None):
    """Tune the handle's binning policy on this batch (or load it from the
    JSON cache at cache_path when it holds this device and semiring)."""
    sr = _sr(semiring)
    h.bind_stream()
    n = len(Ms)
    marr = (Csr * max(n, 1))(*[x.abi() for x in Ms])
    aarr = (Csr * max(n, 1))(*[x.abi() for x in As])
    barr = (Csr * max(n, 1))(*[x.abi() for x in Bs])
    comp = None
    if complement is not None:
        comp = (C.c_int * max(n, 1))(*[int(bool(c)) for c in complement])
    path = None if cache_path is None else str(cache_path).encode()
    h.check(h.lib.msgemm_autotune(h.h, n, marr, comp, aarr, barr, sr, path))


def msgemm_reduce_sum(h: Handle, res: Result, semiring) -> torch.Tensor:
    """Device scalar: int64 (wrapping) sum for the int64 semirings, float64 for fp32."""
    sr = _sr(semiring)
    h.bind_stream()
    out = torch.empty(1, dtype=torch.float64 if sr == PLUS_TIMES_F32 else torch.int64, device=res.values.device)
    co = CsrOut(res.nrows, res.ncols, res.rowptr.data_ptr(), res.colidx.data_ptr(), res.values.data_ptr(),
                res.values.numel(), res.d_nnz.data_ptr())
    h.check(h.lib.msgemm_reduce_sum(h.h, C.byref(co), sr, out.data_ptr()))
    return out


def msgemm_transpose(h: Handle, A: DeviceCsr, value_bytes: int, sorted_rows: bool = False) -> Result:
    h.bind_stream()
    a = A.abi()
    out = CsrOut()
    h.check(h.lib.msgemm_transpose(h.h, C.byref(a), int(value_bytes), int(bool(sorted_rows)), C.byref(out)))
    dt = {0: torch.uint8, 4: torch.float32, 8: torch.int64}[value_bytes]
    rp = h.adopt(out.rowptr, torch.int32, out.nrows + 1)
    ci = h.adopt(out.colidx, torch.int32, out.capacity)
    v = h.adopt(out.values, dt, out.capacity) if value_bytes else None
    nz = h.adopt(out.d_nnz, torch.int64, 1)
    return Result(out.nrows, out.ncols, rp, ci, v, nz)


def msgemm_transpose_noalloc(A: DeviceCsr, value_bytes: int, sorted_rows: bool = False):
    """Transpose through the entry point that allocates nothing: the output
    arrays are allocated here (by the caller), the library only fills them.
    Returns (rowptr, colidx, values-or-None)."""
    lib = load()
    dev = A.rowptr.device
    rp = torch.empty(A.ncols + 1, dtype=torch.int32, device=dev)
    ci = torch.empty(max(A.nnz, 1), dtype=torch.int32, device=dev)
    dt = {0: None, 4: torch.float32, 8: torch.int64}[value_bytes]
    v = torch.empty(max(A.nnz, 1), dtype=dt, device=dev) if dt is not None else None
    a = A.abi()
    # the entry point takes its scratch and SM count from the current device:
    # make A's device current for the call
    with torch.cuda.device(dev):
        st = lib.msgemm_transpose_noalloc(C.byref(a), int(value_bytes), int(bool(sorted_rows)), rp.data_ptr(),
                                          ci.data_ptr(), v.data_ptr() if v is not None else None,
                                          torch.cuda.current_stream(dev).cuda_stream)
    if st != 0:
        raise MsgemmError(st, "msgemm_transpose_noalloc")
    return rp, ci[:A.nnz], (v[:A.nnz] if v is not None else None)


def msgemm_bc(h: Handle, A: DeviceCsr, sources: torch.Tensor):
    """Betweenness centrality of every vertex from the given sources (device
    int32): returns (centrality fp64 tensor of n, number of BFS levels)."""
    h.bind_stream()
    src = sources.to(device=A.rowptr.device, dtype=torch.int32).contiguous()
    out = torch.empty(max(A.nrows, 1), dtype=torch.float64, device=A.rowptr.device)
    a = A.abi()
    lv = C.c_int32(0)
    h.check(h.lib.msgemm_bc(h.h, C.byref(a), src.data_ptr() if src.numel() else None, int(src.numel()),
                            out.data_ptr(), C.byref(lv)))
    return out[:A.nrows], int(lv.value)


def msgemm_ktruss(h: Handle, A: DeviceCsr, k: int):
    """k-truss of a symmetric pattern: (Result with each edge's support as
    int64 values, rounds, products kept over all rounds)."""
    h.bind_stream()
    a = A.abi()
    out = CsrOut()
    it = C.c_int32(0)
    prod = C.c_int64(0)
    h.check(h.lib.msgemm_ktruss(h.h, C.byref(a), int(k), C.byref(out), C.byref(it), C.byref(prod)))
    return h.result(out, torch.int64), int(it.value), int(prod.value)
