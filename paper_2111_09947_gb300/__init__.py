"""Masked sparse matrix-matrix products on NVIDIA GB300 (sm_103a).

C = M .* (A B) and C = !M .* (A B) over CSR operands on the plus-times fp32,
plus-times int64 and plus-pair int64 semirings ("Parallel Algorithms for
Masked Sparse Matrix-Matrix Products", Sec. 2).  The computation runs in the
CUDA library behind the C ABI of include/msgemm.h; this package marshals
arguments (``_lib``), offers a differentiable form (``autograd``) and the
seeded input generators (``synth``).
"""
from ._lib import (DeviceCsr, Handle, MsgemmError, Result, load, msgemm_autotune, msgemm_backward,  # noqa: F401
                   msgemm_bc, msgemm_ktruss, msgemm_reduce_sum, msgemm_run, msgemm_run_batched, msgemm_transpose,
                   msgemm_transpose_noalloc)

_default_handle = None


def default_handle() -> Handle:
    global _default_handle
    if _default_handle is None:
        _default_handle = Handle()
    return _default_handle


def masked_spgemm(M: DeviceCsr, A: DeviceCsr, B: DeviceCsr, semiring: str = "plus_times_f32",
                  complement: bool = False, handle: Handle = None) -> DeviceCsr:
    """C = M .* (A B) (complement=False) or !M .* (A B); returns C trimmed to
    its entry count (reads the count back, one host synchronisation)."""
    h = handle or default_handle()
    return msgemm_run(h, M, A, B, semiring, complement).trimmed()


_SR_DTYPES = {"plus_times_f32": "float32", "plus_times_i64": "int64", "plus_pair_i64": None}


def _from_torch_csr(X, values: bool, semiring: str) -> DeviceCsr:
    import torch
    if X.layout != torch.sparse_csr:
        raise TypeError("expected a torch.sparse_csr tensor or a DeviceCsr")
    crow, col = X.crow_indices(), X.col_indices()
    if crow.dtype != torch.int32 or col.dtype != torch.int32:
        raise TypeError("sparse_csr operands need int32 crow and col indices")
    v = None
    if values and _SR_DTYPES[semiring] is not None:
        v = X.values().to(getattr(torch, _SR_DTYPES[semiring])).contiguous()
    return DeviceCsr(X.shape[0], X.shape[1], crow.contiguous(), col.contiguous(), v)


def masked_spgemm_csr(M, A, B, semiring: str = "plus_times_f32", complement: bool = False, handle: Handle = None):
    """torch.sparse_csr tensors in (int32 crow/col indices, on the GPU), a
    torch.sparse_csr tensor out: C = M .* (A B) or !M .* (A B).  Only M's
    pattern is read.  For gradients use autograd.masked_spgemm_autograd."""
    import torch
    h = handle or default_handle()
    Md = _from_torch_csr(M, False, semiring)
    Ad = _from_torch_csr(A, True, semiring)
    Bd = _from_torch_csr(B, True, semiring)
    c = msgemm_run(h, Md, Ad, Bd, semiring, complement).trimmed()
    return torch.sparse_csr_tensor(c.rowptr, c.colidx, c.values, size=(c.nrows, c.ncols))
