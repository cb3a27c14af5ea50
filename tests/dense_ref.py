"""Dense brute force for tiny inputs (numpy matmul), used to pin the oracle.

For C = M .* (A B): the output pattern is {(i, j) allowed by the mask : some
k has A_ik and B_kj stored}; values are the dense product restricted to it.
"""
import numpy as np


def dense_masked(M, A, B, semiring: str, complement: bool):
    Ap = A.pattern_dense().astype(np.int64)
    Bp = B.pattern_dense().astype(np.int64)
    hits = Ap @ Bp                      # number of k with both stored
    allowed = M.pattern_dense()
    if complement:
        allowed = ~allowed
    present = (hits > 0) & allowed
    if semiring == "plus_times_f32":
        vals = A.to_dense(np.float64) @ B.to_dense(np.float64)
        S = np.abs(A.to_dense(np.float64)) @ np.abs(B.to_dense(np.float64))
    elif semiring == "plus_times_i64":
        vals = A.to_dense(np.int64) @ B.to_dense(np.int64)
        S = None
    else:
        vals = hits
        S = None
    return present, vals, S


def to_dense_result(res, nrows, ncols, dtype):
    rp, ci, v = res["rowptr"], res["colidx"], res["values"]
    present = np.zeros((nrows, ncols), bool)
    vals = np.zeros((nrows, ncols), dtype)
    rows = np.repeat(np.arange(nrows), np.diff(rp))
    present[rows, ci] = True
    vals[rows, ci] = v
    return present, vals
