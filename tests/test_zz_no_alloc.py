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


def test_noalloc_transpose_rejects_too_many_columns():
    rp = torch.zeros(2, dtype=torch.int32, device="cuda")
    A = _lib.DeviceCsr(1, (1 << 20) + 1, rp, torch.zeros(0, dtype=torch.int32, device="cuda"), None)
    with pytest.raises(_lib.MsgemmError) as e:
        _lib.msgemm_transpose_noalloc(A, 0)
    assert e.value.status == 6
