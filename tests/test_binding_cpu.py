"""Host logic of the Python binding, without a GPU: output arrays of a batch are
views into the few allocations the library carved them from, and a batch's
per-product results are made on access.  Plain CPU tensors stand in for the
device allocations (only pointers and sizes are involved)."""
import pytest
import torch

from paper_2111_09947_gb300 import _lib


def _carve(sizes, align=16):
    """One uint8 allocation holding slices of the given byte sizes, carved as
    the library carves a call's outputs (each slice >= 1 byte, 16-aligned)."""
    offs, total = [], 0
    for b in sizes:
        offs.append(total)
        total += (max(b, 1) + align - 1) // align * align
    mem = torch.zeros(total, dtype=torch.uint8)
    base = mem.data_ptr()
    return mem, [base + o for o in offs]


def _batch(nrows, caps, vbytes=4):
    """Fake outputs of len(nrows) products: one allocation per array kind."""
    n = len(nrows)
    rp_mem, rp = _carve([4 * (m + 1) for m in nrows])
    nz_mem, nz = _carve([8] * n)
    ci_mem, ci = _carve([4 * c for c in caps])
    v_mem, v = _carve([vbytes * c for c in caps])
    outs = (_lib.CsrOut * n)()
    for p in range(n):
        outs[p].nrows, outs[p].ncols = nrows[p], 10
        outs[p].rowptr, outs[p].colidx, outs[p].values = rp[p], ci[p], v[p]
        outs[p].capacity, outs[p].d_nnz = caps[p], nz[p]
    return outs, {rp[0]: rp_mem, nz[0]: nz_mem, ci[0]: ci_mem, v[0]: v_mem}


class _FakeHandle:
    """The part of Handle that claim() uses: the live allocations by pointer."""

    def __init__(self, live):
        self._live = dict(live)

    claim = _lib.Handle.claim


def test_batch_views_and_lazy_results():
    nrows, caps = [3, 0, 5, 2], [4, 0, 7, 1]
    outs, live = _batch(nrows, caps)
    workspace = torch.zeros(64, dtype=torch.uint8)
    h = _FakeHandle({**live, workspace.data_ptr(): workspace})
    res = _lib.BatchResult(h.claim(outs), outs, torch.float32)
    # the four output allocations are taken over; the workspace stays live
    assert list(h._live) == [workspace.data_ptr()]
    assert len(res) == 4
    for p, r in enumerate(res):
        assert r.rowptr.dtype == torch.int32 and r.rowptr.numel() == nrows[p] + 1
        assert r.colidx.numel() == caps[p] and r.values.numel() == caps[p]
        assert r.values.dtype == torch.float32 and r.d_nnz.dtype == torch.int64 and r.d_nnz.numel() == 1
        assert r.rowptr.data_ptr() == outs[p].rowptr
        if caps[p]:
            assert r.values.data_ptr() == outs[p].values and r.colidx.data_ptr() == outs[p].colidx
    # views write through to the shared allocation
    res[2].colidx.fill_(7)
    ci_mem = live[outs[0].colidx]
    assert int((ci_mem.view(torch.int32) == 7).sum()) == caps[2]
    assert res[-1] is res[3] and len(res[1:3]) == 2
    with pytest.raises(IndexError):
        res[4]


def test_view_outside_allocation_raises():
    outs, live = _batch([2], [3])
    blocks = _FakeHandle(live).claim(outs)
    with pytest.raises(KeyError):
        blocks.view(outs[0].rowptr - 64, torch.int32, 1)
    with pytest.raises(KeyError):
        blocks.view(outs[0].colidx, torch.int32, 1000)


def test_single_product_result_claims_its_arrays():
    outs, live = _batch([4], [6], vbytes=8)
    h = _FakeHandle(live)
    r = _lib.Handle.result(h, outs[0], torch.int64)
    assert not h._live
    assert r.values.dtype == torch.int64 and r.values.numel() == 6 and r.rowptr.numel() == 5
