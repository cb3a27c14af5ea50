"""Row-sharded products on the GPU: the row blocks partition_rows gives for
three ranks, each run through the C ABI on device row slices (views of the
same device arrays), stitched, equal the whole product from the oracle; and
sharded_product itself in a one-rank gloo group."""
import os
import socket

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2111_09947_gb300 import _lib, shard, synth
from gpu_util import assert_parity, to_dev

pytestmark = pytest.mark.gpu


def _stitch(blocks):
    rp, ci, va, off = [np.zeros(1, np.int64)], [], [], 0
    for b in blocks:
        r = b.trimmed()
        brp = r.rowptr.cpu().numpy().astype(np.int64)
        rp.append(brp[1:] + off)
        ci.append(r.colidx.cpu().numpy())
        va.append(r.values.cpu().numpy())
        off += int(brp[-1])
    return np.concatenate(rp), np.concatenate(ci), np.concatenate(va)


@pytest.mark.parametrize("semiring,gen,complement", [("plus_times_f32", "f32", False),
                                                      ("plus_times_i64", "i64", True)])
def test_row_blocks_stitch_to_the_whole_product(semiring, gen, complement):
    p = synth.random_problem(2000, 1500, 3000, 8.0, 12.0, 40.0, 97, gen)
    d = to_dev(p, semiring)
    h = _lib.Handle()
    try:
        b = shard.partition_rows(shard.push_work(p["A"], p["B"]), 3)
        blocks = []
        for r in range(3):
            Mb = shard.row_block(d["M"], int(b[r]), int(b[r + 1]))
            Ab = shard.row_block(d["A"], int(b[r]), int(b[r + 1]))
            blocks.append(_lib.msgemm_run(h, Mb, Ab, d["B"], semiring, complement))
        h.sync_status()
        rp, ci, va = _stitch(blocks)
    finally:
        h.close()
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], semiring, complement=complement,
                          method=O.ESC if complement else O.MERGE)
    whole = synth.Csr(p["M"].nrows, p["M"].ncols, rp.astype(np.int32), ci, va)
    assert_parity(_lib.DeviceCsr.from_host(whole), ref, semiring)


def test_sharded_product_one_rank_group():
    import torch.distributed as dist
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        p = synth.random_problem(500, 400, 600, 6.0, 8.0, 30.0, 98, "f32")
        d = to_dev(p, "plus_times_f32")
        h = _lib.Handle()
        out = shard.sharded_product(d["M"], d["A"], d["B"],
                                    lambda Mb, Ab, B: _lib.msgemm_run(h, Mb, Ab, B, "plus_times_f32").trimmed(),
                                    0, 1)
        h.sync_status()
        assert out["r0"] == 0 and out["r1"] == 500 and out["offset"] == 0
        assert_parity(out["result"], O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32"), "plus_times_f32")
        h.close()
    finally:
        dist.destroy_process_group()


def test_torch_sparse_csr_interface():
    """masked_spgemm_csr: torch.sparse_csr tensors in and out."""
    import paper_2111_09947_gb300 as pkg
    p = synth.random_problem(400, 300, 500, 6.0, 8.0, 30.0, 99, "f32")

    def t(x, vals=True):
        v = torch.from_numpy(x.values if vals else np.ones(x.nnz, np.float32)).cuda()
        return torch.sparse_csr_tensor(torch.from_numpy(x.rowptr).cuda(), torch.from_numpy(x.colidx).cuda(), v,
                                       size=(x.nrows, x.ncols))
    C = pkg.masked_spgemm_csr(t(p["M"], False), t(p["A"]), t(p["B"]))
    assert C.layout == torch.sparse_csr and tuple(C.shape) == (400, 500)
    res = _lib.DeviceCsr(400, 500, C.crow_indices(), C.col_indices(), C.values())
    assert_parity(res, O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32"), "plus_times_f32")
