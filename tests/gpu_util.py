"""Helpers for GPU-vs-oracle parity tests."""
import numpy as np
import torch

from paper_2111_09947_gb300 import _lib

# fp32 bound (per entry): |c - c_ref| <= 1e-5 * sum_k |a_ik| |b_kj|, c_ref in fp64
FP32_REL = 1e-5


def to_dev(p: dict, semiring: str) -> dict:
    vd = {"plus_times_f32": torch.float32, "plus_times_i64": torch.int64, "plus_pair_i64": None}[semiring]
    out = {}
    for k in ("M", "A", "B"):
        m = p[k]
        d = _lib.DeviceCsr.from_host(m, values_dtype=vd if k != "M" else None)
        if k == "M" or semiring == "plus_pair_i64":
            d.values = None
        out[k] = d
    return out


def host(res):
    """(rowptr, colidx, values) numpy arrays of a trimmed DeviceCsr."""
    return res.rowptr.cpu().numpy(), res.colidx.cpu().numpy(), res.values.cpu().numpy()


def assert_parity(res, ref, semiring, rows=None, ctx=""):
    """Element-wise parity: identical row pointers and columns; integer values
    bit-exact; fp32 within the per-entry bound.  With ``rows`` the oracle holds
    only those rows (in order) and the GPU result is sliced to match."""
    rp, ci, v = host(res)
    if rows is not None:
        parts_c, parts_v, lens = [], [], []
        for i in rows:
            s, e = rp[i], rp[i + 1]
            parts_c.append(ci[s:e])
            parts_v.append(v[s:e])
            lens.append(e - s)
        ci = np.concatenate(parts_c) if parts_c else ci[:0]
        v = np.concatenate(parts_v) if parts_v else v[:0]
        rp = np.concatenate([[0], np.cumsum(lens)])
    assert np.array_equal(rp.astype(np.int64), ref["rowptr"]), f"rowptr differs {ctx}"
    assert np.array_equal(ci, ref["colidx"]), f"colidx differs {ctx}"
    if semiring == "plus_times_f32":
        err = np.abs(v.astype(np.float64) - ref["values"])
        bad = err > FP32_REL * ref["S"]
        assert not bad.any(), f"{bad.sum()} fp32 values outside the bound {ctx}: max err/S " \
                              f"{np.max(err / np.maximum(ref['S'], 1e-300)):.3e}"
    else:
        assert np.array_equal(v.astype(np.int64), ref["values"]), f"int values differ {ctx}"
