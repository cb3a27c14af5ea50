"""Masked sparse matrix-matrix products on NVIDIA GB300 (sm_103a).

C = M .* (A B) and C = !M .* (A B) over CSR operands on the plus-times fp32,
plus-times int64 and plus-pair int64 semirings ("Parallel Algorithms for
Masked Sparse Matrix-Matrix Products", Sec. 2).  The computation runs in the
CUDA library behind the C ABI of include/msgemm.h; this package marshals
arguments (``_lib``), offers a differentiable form (``autograd``) and the
seeded input generators (``synth``).
"""
from ._lib import (DeviceCsr, Handle, MsgemmError, Result, load, msgemm_backward, msgemm_reduce_sum,  # noqa: F401
                   msgemm_run, msgemm_run_batched, msgemm_transpose)

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
