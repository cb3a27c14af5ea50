"""Heap accumulators (Sec. 5.5, Alg. 4 and 5) and the two-phase form (Sec. 6)
against the CPU oracle, through the C ABI.

Heap: forced on every row it fits (at most 128 stored entries in A_i*), with
NInspect 1 (Heap), unbounded (HeapDot) and, for complemented masks, 0; the
bin counts must show the heap kinds really ran, and rows too long for them
must fall back without changing the result.  A cached policy that ranks heap
first must route AUTO rows to it.

Two-phase: a symbolic pass (indices only) sizes C exactly, then a numeric pass
writes every row in place.  Results must equal the oracle's, C's capacity must
equal its entry count, and every accumulator family (and the batched entry
point) must go through it.
"""
import json

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2111_09947_gb300 import _lib, synth
from gpu_util import assert_parity, to_dev

pytestmark = pytest.mark.gpu

SEMIRINGS = ["plus_times_f32", "plus_times_i64", "plus_pair_i64"]
GEN = {"plus_times_f32": "f32", "plus_times_i64": "i64", "plus_pair_i64": "pair"}

SHAPES = [
    # m, k, n, dA, dB, dM
    (1, 1, 1, 1.0, 1.0, 1.0),
    (37, 23, 41, 3.0, 4.0, 5.0),
    (2500, 1500, 3000, 8.0, 8.0, 8.0),         # several compaction tiles, ragged
    (400, 300, 500, 2.0, 2.0, 200.0),          # inputs much sparser than the mask
    (700, 600, 900, 12.0, 40.0, 2.0),          # mask much sparser than the inputs
    (50, 0, 60, 0.0, 0.0, 10.0),               # k = 0
    (64, 64, 64, 64.0, 64.0, 64.0),            # dense
    (2000, 300, 70000, 6.0, 300.0, 40.0),      # wide rows
]


@pytest.fixture()
def handle():
    h = _lib.Handle()
    h.set_option(_lib.OPT_VALIDATE, 1)
    yield h
    h.close()


def _problem(s, shape, semiring, seed0):
    m, k, n, da, db, dm = shape
    return synth.random_problem(m, k, n, min(da, max(k, 1)), min(db, max(n, 1)), min(dm, max(n, 1)), seed0 + s,
                                GEN[semiring])


def _ref(p, semiring, complement):
    return O.masked_spgemm(p["M"], p["A"], p["B"], semiring, complement=complement,
                           method=O.ESC if complement else O.MERGE)


def _run(h, p, semiring, complement):
    d = to_dev(p, semiring)
    res = _lib.msgemm_run(h, d["M"], d["A"], d["B"], semiring, complement)
    h.sync_status()
    return res


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("force", ["heap", "heapdot"])
@pytest.mark.parametrize("complement", [False, True])
def test_heap_forced(handle, semiring, force, complement):
    handle.force(force)
    kind = "cheap_w" if complement else {"heap": "heap_w", "heapdot": "heapdot_w"}[force]
    used = 0
    for s, shape in enumerate(SHAPES):
        p = _problem(s, shape, semiring, 4100)
        res = _run(handle, p, semiring, complement)
        used += handle.bin_counts()[kind]
        assert_parity(res.trimmed(), _ref(p, semiring, complement), semiring, ctx=f"shape {s}")
    assert used > 1000, "the heap kind took too few rows to test it"


@pytest.mark.parametrize("complement", [False, True])
def test_heap_long_rows_fall_back(handle, complement):
    """Rows with more than 128 stored entries in A_i* do not fit the heap's
    registers and take the tiled MSA; short rows of the same call keep the heap."""
    handle.force("heap")
    p = synth.random_problem(300, 4000, 3000, 200.0, 3.0, 60.0, 4200, "i64")
    # a few short rows too: cut A's rows 0..49 down to 5 entries
    A = p["A"]
    keep = np.ones(A.nnz, bool)
    for i in range(50):
        keep[A.rowptr[i] + 5:A.rowptr[i + 1]] = False
    rp = np.concatenate([[0], np.cumsum([keep[A.rowptr[i]:A.rowptr[i + 1]].sum() for i in range(A.nrows)])])
    p["A"] = synth.Csr(A.nrows, A.ncols, rp.astype(np.int32), A.colidx[keep], A.values[keep])
    res = _run(handle, p, "plus_times_i64", complement)
    counts = handle.bin_counts()
    assert_parity(res.trimmed(), _ref(p, "plus_times_i64", complement), "plus_times_i64")
    heap = counts["cheap_w" if complement else "heap_w"]
    assert 0 < heap <= 50
    assert counts["cmsa_t" if complement else "msa_t"] + counts["cmsa_g" if complement else "msa_g"] >= 250


def test_heap_int64_wrap(handle):
    """int64 values over +-2^50: products and sums wrap modulo 2^64."""
    rng = np.random.default_rng(78)
    p = synth.random_problem(300, 200, 400, 12.0, 30.0, 40.0, 607, "pair")
    p = {k: (v if k == "M" else v.with_values(rng.integers(-2 ** 50, 2 ** 50, v.nnz, dtype=np.int64)))
         for k, v in p.items()}
    for force in ("heap", "heapdot"):
        handle.force(force)
        for complement in (False, True):
            res = _run(handle, p, "plus_times_i64", complement)
            assert_parity(res.trimmed(), _ref(p, "plus_times_i64", complement), "plus_times_i64",
                          ctx=f"{force} complement={complement}")


def test_heap_from_cached_policy(tmp_path):
    """A cached policy with HeapDot first (then MCA) for every class sends the
    AUTO rows that fit it to the heap kind."""
    key = torch.cuda.get_device_name() + "|plus_times_f32"
    entry = {"warp_flops_max": 65536, "dot_ratio": 1e6, "warp_slab": 4608, "grid_min_flops": 1 << 62,
             "pref": [[6, 3, 0, 0]] * 16}
    cache = tmp_path / "tune.json"
    cache.write_text(json.dumps({key: entry}))
    p = synth.random_problem(3000, 2000, 2500, 4.0, 6.0, 30.0, 4300, "f32")
    h = _lib.Handle()
    try:
        _lib.msgemm_autotune(h, [], [], [], "plus_times_f32", cache_path=cache)
        res = _run(h, p, "plus_times_f32", False)
        counts = h.bin_counts()
    finally:
        h.close()
    assert_parity(res.trimmed(), _ref(p, "plus_times_f32", False), "plus_times_f32")
    assert counts["heapdot_w"] > 2500


# ------------------------------------------------------------- two phases

@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("force", ["auto", "msa", "hash", "mca", "dot", "heap"])
@pytest.mark.parametrize("complement", [False, True])
def test_two_phase(handle, semiring, force, complement):
    if complement and force in ("mca", "dot"):
        pytest.skip("no complemented form")
    handle.set_option(_lib.OPT_PHASES, 2)
    handle.force(force)
    for s, shape in enumerate(SHAPES):
        p = _problem(s, shape, semiring, 4400)
        res = _run(handle, p, semiring, complement)
        ref = _ref(p, semiring, complement)
        nnz = len(ref["colidx"])
        assert int(res.nnz()) == nnz
        assert res.colidx.numel() == nnz, "two-phase output must be sized exactly"
        assert_parity(res.trimmed(), ref, semiring, ctx=f"shape {s}")


def test_two_phase_matches_one_phase_triangles(handle):
    """Triangle counting at R-MAT scale 14 in both forms: the same C."""
    p = synth.triangle_counting(scale=14, ef=16, seed=5)
    d = to_dev(p, "plus_pair_i64")
    one = _lib.msgemm_run(handle, d["M"], d["A"], d["B"], "plus_pair_i64").trimmed()
    handle.set_option(_lib.OPT_PHASES, 2)
    two = _lib.msgemm_run(handle, d["M"], d["A"], d["B"], "plus_pair_i64")
    assert two.colidx.numel() == int(two.nnz())
    two = two.trimmed()
    for a, b in ((one.rowptr, two.rowptr), (one.colidx, two.colidx), (one.values, two.values)):
        assert torch.equal(a, b)


def test_two_phase_batched(handle):
    """The batched entry point in two phases (the graph flag is ignored)."""
    ps = synth.batched_problems(nprod=10, seed=44, log2_range=(8, 12))
    comp = [i % 3 == 0 for i in range(len(ps))]
    devs = [to_dev(p, "plus_times_f32") for p in ps]
    handle.set_option(_lib.OPT_PHASES, 2)
    outs = _lib.msgemm_run_batched(handle, [d["M"] for d in devs], [d["A"] for d in devs], [d["B"] for d in devs],
                                   "plus_times_f32", complement=comp, use_graph=True)
    handle.sync_status()
    for o, p, c in zip(outs, ps, comp):
        ref = _ref(p, "plus_times_f32", c)
        assert o.colidx.numel() == len(ref["colidx"])
        assert_parity(o.trimmed(), ref, "plus_times_f32")


def test_two_phase_empty_and_errors(handle):
    handle.set_option(_lib.OPT_PHASES, 2)
    p = synth.random_problem(0, 5, 7, 1.0, 1.0, 1.0, 1, "f32")
    res = _run(handle, p, "plus_times_f32", False)
    assert int(res.nnz()) == 0 and res.rowptr.numel() == 1
    with pytest.raises(_lib.MsgemmError):
        handle.set_option(_lib.OPT_PHASES, 3)


@pytest.mark.parametrize("force", ["heap", "heapdot"])
def test_heap_gradient_form(handle, force):
    """Backward (values written at each mask entry's own slot) through the heap
    kinds: dA and dB against the oracle's closed forms."""
    m, k, n = 300, 400, 500
    p = synth.random_problem(m, k, n, 6.0, 5.0, 30.0, 4500, "f32")
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
    G = synth.Csr(m, n, ref["rowptr"].astype(np.int32), ref["colidx"], synth.upstream_grad(len(ref["colidx"]), 4))
    dA_ref, dB_ref = O.grad(p["A"], p["B"], G)
    d = to_dev(p, "plus_times_f32")
    handle.force(force)
    dA, dB = _lib.msgemm_backward(handle, d["A"], d["B"], _lib.DeviceCsr.from_host(G))
    handle.sync_status()
    assert handle.bin_counts()[{"heap": "heap_w", "heapdot": "heapdot_w"}[force]] > 100
    Aabs = p["A"].with_values(np.abs(p["A"].values))
    Babs = p["B"].with_values(np.abs(p["B"].values))
    Gabs = G.with_values(np.abs(G.values))
    SA, SB = O.grad(Aabs, Babs, Gabs)
    assert np.all(np.abs(dA.cpu().numpy() - dA_ref) <= 1e-5 * SA + 1e-30)
    assert np.all(np.abs(dB.cpu().numpy() - dB_ref) <= 1e-5 * SB + 1e-30)


@pytest.mark.parametrize("complement", [False, True])
def test_heap_register_limit(handle, complement):
    """A row with exactly 128 stored entries in A_i* fits the heap's registers
    (4 iterators per lane); one with 129 takes the tiled MSA; both exact."""
    rng = np.random.default_rng(46)
    m, k, n = 6, 400, 300
    rows = [128, 129, 1, 127, 0, 5]
    rp = np.concatenate([[0], np.cumsum(rows)]).astype(np.int32)
    ci = np.concatenate([np.sort(rng.choice(k, size=r, replace=False)) for r in rows]).astype(np.int32)
    A = synth.Csr(m, k, rp, ci, rng.integers(-9, 9, len(ci)).astype(np.int64))
    p = synth.random_problem(m, k, n, 4.0, 3.0, 40.0, 4600, "i64")
    p["A"] = A
    handle.force("heap")
    res = _run(handle, p, "plus_times_i64", complement)
    kinds = handle.row_kinds(m)
    assert_parity(res.trimmed(), _ref(p, "plus_times_i64", complement), "plus_times_i64")
    heap = _lib.KIND_NAMES.index("cheap_w" if complement else "heap_w")
    assert kinds[0] == heap and kinds[3] == heap and kinds[1] != heap


def test_two_phase_rejects_invalid_input(handle):
    """Validation runs before the symbolic pass: an unsorted row is refused."""
    p = synth.random_problem(40, 30, 50, 4.0, 4.0, 6.0, 4700, "f32")
    A = p["A"]
    ci = A.colidx.copy()
    r = next(i for i in range(A.nrows) if A.rowptr[i + 1] - A.rowptr[i] >= 2)
    ci[A.rowptr[r]], ci[A.rowptr[r] + 1] = ci[A.rowptr[r] + 1], ci[A.rowptr[r]]
    p["A"] = synth.Csr(A.nrows, A.ncols, A.rowptr, ci, A.values)
    handle.set_option(_lib.OPT_PHASES, 2)
    d = to_dev(p, "plus_times_f32")
    with pytest.raises(_lib.MsgemmError) as e:
        _lib.msgemm_run(handle, d["M"], d["A"], d["B"], "plus_times_f32")
    assert e.value.status == 3
    handle.sync_status()
