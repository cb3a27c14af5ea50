"""The transpose entry point that allocates nothing (msgemm_transpose_noalloc).

It exists for callers that cannot allocate device memory where they need a
transpose (fixed memory pools, hosts without an allocator, paths that cannot
afford cudaMalloc's possible device synchronisation):
it keeps its scratch in a fixed device array inside the library.  Checked
against msgemm_transpose, the entry point that allocates, on two calls in a
row over different matrices (the second call finds the first one's scratch
contents and must clear what it needs).  Transposes are exact: equality.
This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2111_09947_gb300 import _lib, synth

pytestmark = pytest.mark.gpu


def _mat(m, n, d, seed):
    c = synth.er_pattern(m, n, d, seed, 1)
    c = c.with_values(synth.uniform_f32(c.nnz, seed, 2))
    return _lib.DeviceCsr.from_host(c)


@pytest.fixture(scope="module")
def handle():
    h = _lib.Handle()
    yield h
    h.close()


def _rows_as_sets(rp, ci, v):
    out = []
    for i in range(len(rp) - 1):
        s, e = rp[i], rp[i + 1]
        out.append(sorted(zip(ci[s:e].tolist(), v[s:e].tolist())))
    return out


def test_noalloc_transpose_matches_allocating_transpose(handle):
    mats = [_mat(3000, 70000, 9.0, 41), _mat(50000, 1200, 3.0, 42)]   # second call: fewer columns
    for A in mats:
        ref = _lib.msgemm_transpose(handle, A, 4, sorted_rows=True)
        rp, ci, v = _lib.msgemm_transpose_noalloc(A, 4, sorted_rows=True)
        torch.cuda.synchronize()
        assert torch.equal(rp, ref.rowptr)
        assert torch.equal(ci, ref.colidx[:A.nnz])
        assert torch.equal(v, ref.values[:A.nnz])
        # unsorted form: same rows as sets
        rp2, ci2, v2 = _lib.msgemm_transpose_noalloc(A, 4, sorted_rows=False)
        torch.cuda.synchronize()
        assert torch.equal(rp2, ref.rowptr)
        r = rp2.cpu().numpy()
        assert _rows_as_sets(r, ci2.cpu().numpy(), v2.cpu().numpy()) == \
            _rows_as_sets(r, ref.colidx[:A.nnz].cpu().numpy(), ref.values[:A.nnz].cpu().numpy())


def _numpy_transpose(m, n, rp, ci, v):
    """A^T on the host: rows of A^T in ascending row order of A (the sorted form)."""
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rp))
    order = np.lexsort((rows, ci))
    trp = np.concatenate([[0], np.cumsum(np.bincount(ci, minlength=n))]).astype(np.int32)
    return trp, rows[order].astype(np.int32), (v[order] if v is not None else None)


def _host_case(m, n, d, seed, value_bytes, last_col_rows=()):
    """Erdos-Renyi pattern plus, for the rows listed, an entry in the last column."""
    c = synth.er_pattern(m, n, d, seed, 1)
    rp, ci = c.rowptr.astype(np.int64), c.colidx.astype(np.int64)
    extra = set(int(i) for i in last_col_rows)
    rows_l, cols_l = [], []
    for i in range(m):
        cols = ci[rp[i]:rp[i + 1]].tolist()
        if i in extra and (not cols or cols[-1] != n - 1):
            cols.append(n - 1)
        rows_l += [i] * len(cols)
        cols_l += cols
    c = synth.coo_to_csr(m, n, np.array(rows_l, np.int32), np.array(cols_l, np.int32))
    rng = np.random.default_rng(seed)
    if value_bytes == 4:
        v = rng.uniform(-1, 1, c.nnz).astype(np.float32)
    elif value_bytes == 8:
        v = rng.integers(-(1 << 60), 1 << 60, c.nnz, dtype=np.int64)
    else:
        v = None
    return c.with_values(v)


@pytest.mark.parametrize("value_bytes", [0, 4, 8])
@pytest.mark.parametrize("sorted_rows", [True, False])
def test_noalloc_transpose_at_the_column_cap(value_bytes, sorted_rows):
    """ncols = 2^20, the largest accepted size (it fills the cursor area and
    the scan's tile sums exactly), with entries in the last column; checked
    against a transpose computed on the host with numpy, not against the
    library.  The unsorted form is checked row by row as a set."""
    n = 1 << 20
    m = 5000
    h = _host_case(m, n, 6.0, 77 + value_bytes, value_bytes, last_col_rows=range(0, m, 97))
    vd = {0: None, 4: torch.float32, 8: torch.int64}[value_bytes]
    A = _lib.DeviceCsr.from_host(h, values_dtype=vd)
    if value_bytes == 0:
        A.values = None
    want_rp, want_ci, want_v = _numpy_transpose(m, n, h.rowptr, h.colidx, h.values)
    assert want_rp[-1] - want_rp[-2] >= m // 97    # the last column is populated
    for rep in range(2):   # the second call finds the first one's scratch contents
        rp, ci, v = _lib.msgemm_transpose_noalloc(A, value_bytes, sorted_rows=sorted_rows)
        torch.cuda.synchronize()
        assert np.array_equal(rp.cpu().numpy(), want_rp)
        got_ci = ci.cpu().numpy()
        got_v = v.cpu().numpy() if v is not None else None
        if sorted_rows:
            assert np.array_equal(got_ci, want_ci)
            if value_bytes:
                assert np.array_equal(got_v, want_v)
        else:
            # same (row, value) pairs per row of A^T
            key_got = np.lexsort((got_ci, np.repeat(np.arange(n), np.diff(want_rp))))
            assert np.array_equal(got_ci[key_got], want_ci)
            if value_bytes:
                assert np.array_equal(got_v[key_got], want_v)


def test_noalloc_transpose_rejects_too_many_columns():
    rp = torch.zeros(2, dtype=torch.int32, device="cuda")
    A = _lib.DeviceCsr(1, (1 << 20) + 1, rp, torch.zeros(0, dtype=torch.int32, device="cuda"), None)
    with pytest.raises(_lib.MsgemmError) as e:
        _lib.msgemm_transpose_noalloc(A, 0)
    assert e.value.status == 6
