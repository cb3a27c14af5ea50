"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Every accumulator family is forced on every row (and AUTO lets the binning
mix them); shapes span several tiles and ragged tails, empty rows, empty
matrices and degenerate dimensions; both mask forms; all three semirings.
"""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2111_09947_gb300 import _lib, synth
from golden_io import worked_example
from gpu_util import assert_parity, to_dev

pytestmark = pytest.mark.gpu

SEMIRINGS = ["plus_times_f32", "plus_times_i64", "plus_pair_i64"]
FORCES = ["auto", "msa", "hash", "mca", "dot", "heap", "heapdot"]
GEN = {"plus_times_f32": "f32", "plus_times_i64": "i64", "plus_pair_i64": "pair"}


@pytest.fixture(scope="module")
def handle():
    h = _lib.Handle()
    h.set_option(_lib.OPT_VALIDATE, 1)
    yield h
    h.close()


def run(h, p, semiring, complement=False, force="auto"):
    h.force(force)
    d = to_dev(p, semiring)
    res = _lib.msgemm_run(h, d["M"], d["A"], d["B"], semiring, complement).trimmed()
    h.sync_status()
    return res


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("force", FORCES)
def test_worked_example(handle, semiring, force):
    g = worked_example()
    vals = {"plus_times_f32": np.float32, "plus_times_i64": np.int64}
    p = {"M": g["M"], "A": g["A"], "B": g["B"]}
    if semiring in vals:
        p = {k: v.with_values(v.values.astype(vals[semiring])) for k, v in p.items()}
    key = "C_plus_pair" if semiring == "plus_pair_i64" else "C_plus_times"
    res = run(handle, p, semiring, False, force)
    want = g[key]
    assert np.array_equal(res.rowptr.cpu().numpy(), want.rowptr)
    assert np.array_equal(res.colidx.cpu().numpy(), want.colidx)
    assert np.array_equal(res.values.cpu().numpy().astype(np.int64), want.values)
    res = run(handle, p, semiring, True, force)
    want = g["C_complement_" + key[2:]]
    assert np.array_equal(res.colidx.cpu().numpy(), want.colidx)
    assert np.array_equal(res.values.cpu().numpy().astype(np.int64), want.values)


SHAPES = [
    # m, k, n, dA, dB, dM
    (1, 1, 1, 1.0, 1.0, 1.0),
    (37, 23, 41, 3.0, 4.0, 5.0),
    (300, 200, 250, 6.0, 6.0, 30.0),
    (2500, 1500, 3000, 8.0, 8.0, 8.0),          # several compaction tiles, ragged
    (700, 600, 900, 12.0, 40.0, 2.0),           # mask much sparser than inputs (pull regime)
    (400, 300, 500, 2.0, 2.0, 200.0),           # inputs much sparser than mask
    (50, 0, 60, 0.0, 0.0, 10.0),                # k = 0: no products at all
    (64, 64, 64, 64.0, 64.0, 64.0),             # dense
    (2000, 300, 70000, 6.0, 300.0, 40.0),       # wide rows: tiled MSA, CTA kinds
]


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("force", FORCES)
def test_random_plain(handle, semiring, force):
    for s, (m, k, n, da, db, dm) in enumerate(SHAPES):
        p = synth.random_problem(m, k, n, min(da, max(k, 1)), min(db, max(n, 1)), min(dm, max(n, 1)), 900 + s,
                                 GEN[semiring])
        ref = O.masked_spgemm(p["M"], p["A"], p["B"], semiring)
        res = run(handle, p, semiring, False, force)
        assert_parity(res, ref, semiring, ctx=f"shape {s} force {force}")


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("force", ["auto", "hash", "msa"])
def test_random_complement(handle, semiring, force):
    for s, (m, k, n, da, db, dm) in enumerate(SHAPES):
        p = synth.random_problem(m, k, n, min(da, max(k, 1)), min(db, max(n, 1)), min(dm, max(n, 1)), 1900 + s,
                                 GEN[semiring])
        ref = O.masked_spgemm(p["M"], p["A"], p["B"], semiring, complement=True, method=O.ESC)
        res = run(handle, p, semiring, True, force)
        assert_parity(res, ref, semiring, ctx=f"shape {s} force {force}")


@pytest.mark.parametrize("semiring", ["plus_times_f32", "plus_times_i64"])
@pytest.mark.parametrize("which", ["A", "B", "AB"])
@pytest.mark.parametrize("force", ["auto", "msa", "hash", "mca", "dot", "heap"])
def test_pattern_operands(handle, semiring, which, force):
    """Under plus-times an operand passed without values is a pattern: every
    stored value is 1 (the oracle gets explicit ones).  Plain and
    complemented masks; the pull kind reads B^T built without values."""
    one = {"plus_times_f32": np.float32, "plus_times_i64": np.int64}[semiring]
    for s in (1, 2, 3, 4, 8):
        m, k, n, da, db, dm = SHAPES[s]
        p = synth.random_problem(m, k, n, min(da, max(k, 1)), min(db, max(n, 1)), min(dm, max(n, 1)), 3900 + s,
                                 GEN[semiring])
        q = dict(p)
        for x in which:
            q[x] = p[x].with_values(np.ones(p[x].nnz, dtype=one))
        for comp in ((False, True) if force in ("auto", "msa", "hash") else (False,)):
            ref = O.masked_spgemm(q["M"], q["A"], q["B"], semiring, complement=comp,
                                  method=O.ESC if comp else O.MERGE)
            d = to_dev(p, semiring)
            for x in which:
                d[x].values = None
            handle.force(force)
            res = _lib.msgemm_run(handle, d["M"], d["A"], d["B"], semiring, comp).trimmed()
            handle.sync_status()
            assert_parity(res, ref, semiring, ctx=f"shape {s} {which} complement={comp}")


@pytest.mark.parametrize("complement", [False, True])
@pytest.mark.parametrize("force", ["auto", "msa", "hash", "mca", "dot"])
def test_int64_wide_values_wrap(handle, complement, force):
    """int64 values spread over +-2^50: products and sums wrap mod 2^64;
    the 64-bit shared-memory accumulation (two 32-bit words with carry) must
    match the oracle bit for bit."""
    if complement and force in ("mca", "dot"):
        pytest.skip("no complemented form")
    rng = np.random.default_rng(77)
    p = synth.random_problem(300, 200, 70000 if force == "msa" else 400, 12.0, 30.0, 40.0, 606, "pair")
    p = {k: (v if k == "M" else v.with_values(rng.integers(-2 ** 50, 2 ** 50, v.nnz, dtype=np.int64)))
         for k, v in p.items()}
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64", complement=complement,
                          method=O.ESC if complement else O.MERGE)
    res = run(handle, p, "plus_times_i64", complement, force)
    assert_parity(res, ref, "plus_times_i64", ctx=force)


def test_empty_matrices(handle):
    for m, k, n in [(0, 5, 7), (5, 7, 0), (0, 0, 0), (3, 4, 5)]:
        p = synth.random_problem(m, k, n, 0.0, 0.0, 0.0, 5, "f32")
        for comp in (False, True):
            res = run(handle, p, "plus_times_f32", comp)
            assert res.rowptr.numel() == m + 1
            assert int(res.rowptr[-1]) == 0 if m else True
            assert res.colidx.numel() == 0


def test_errors(handle):
    p = synth.random_problem(10, 8, 12, 2.0, 2.0, 2.0, 3, "f32")
    d = to_dev(p, "plus_times_f32")
    with pytest.raises(_lib.MsgemmError) as e:
        _lib.msgemm_run(handle, d["M"], d["B"], d["B"], "plus_times_f32")
    assert e.value.status == 2
    with pytest.raises(_lib.MsgemmError) as e:
        _lib.msgemm_backward(handle, d["A"], d["B"], d["M"]) if False else \
            handle.check(handle.lib.msgemm_backward(handle.h, None, None, None, 1, None, None))
    assert e.value.status in (1, 4)
    # unsorted row found by device validation
    A = p["A"]
    ci = A.colidx.copy()
    r = next(i for i in range(A.nrows) if A.rowptr[i + 1] - A.rowptr[i] >= 2)
    s = A.rowptr[r]
    ci[s], ci[s + 1] = ci[s + 1], ci[s]
    bad = synth.Csr(A.nrows, A.ncols, A.rowptr, ci, A.values)
    d2 = to_dev({"M": p["M"], "A": bad, "B": p["B"]}, "plus_times_f32")
    handle.force("auto")
    with pytest.raises(_lib.MsgemmError) as e:
        _lib.msgemm_run(handle, d2["M"], d2["A"], d2["B"], "plus_times_f32")
    assert e.value.status == 3
    handle.sync_status()   # error word was cleared
    # a row pointer beyond nnz is rejected before any product kernel reads it
    rp = p["M"].rowptr.copy()
    rp[-1] += 5
    d3 = to_dev({"M": synth.Csr(p["M"].nrows, p["M"].ncols, rp, p["M"].colidx), "A": p["A"], "B": p["B"]},
                "plus_times_f32")
    with pytest.raises(_lib.MsgemmError) as e:
        _lib.msgemm_run(handle, d3["M"], d3["A"], d3["B"], "plus_times_f32")
    assert e.value.status == 1
    handle.sync_status()


def test_er_plain_fp32_full(handle):
    """Erdos-Renyi n = 4096, 8 entries per row, fp32: the whole output."""
    p = synth.er_plain_f32()
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
    for force in FORCES:
        res = run(handle, p, "plus_times_f32", False, force)
        assert_parity(res, ref, "plus_times_f32", ctx=force)


@pytest.mark.parametrize("scale", [10, 14])
def test_triangle_count_rmat(handle, scale):
    p = synth.triangle_counting(scale=scale, ef=16, seed=21)
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_pair_i64")
    for force in FORCES:
        res = run(handle, p, "plus_pair_i64", False, force)
        assert_parity(res, ref, "plus_pair_i64", ctx=force)
        full = _lib.msgemm_run(handle, *[to_dev(p, "plus_pair_i64")[k] for k in ("M", "A", "B")], "plus_pair_i64")
        tri = int(_lib.msgemm_reduce_sum(handle, full, "plus_pair_i64").item())
        assert tri == int(ref["values"].sum())


def test_bfs_step_small(handle):
    p = synth.bfs_step(scale=12, ef=16, nsrc=64, seed=8)
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_i64", complement=True, method=O.ESC)
    for force in ["auto", "msa", "hash"]:
        res = run(handle, p, "plus_times_i64", True, force)
        assert_parity(res, ref, "plus_times_i64", ctx=force)


def test_batched_matches_plain(handle):
    ps = synth.batched_problems(nprod=10, seed=4, log2_range=(8, 11))
    devs = [to_dev(p, "plus_times_f32") for p in ps]
    handle.force("auto")
    outs = _lib.msgemm_run_batched(handle, [d["M"] for d in devs], [d["A"] for d in devs], [d["B"] for d in devs],
                                   "plus_times_f32")
    for p, o in zip(ps, outs):
        ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
        assert_parity(o.trimmed(), ref, "plus_times_f32")


def test_backward_vs_oracle(handle):
    for seed, (m, k, n) in enumerate([(60, 50, 70), (300, 200, 250)]):
        p = synth.random_problem(m, k, n, 5.0, 5.0, 12.0, 70 + seed, "f32")
        ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
        G = synth.Csr(m, n, ref["rowptr"].astype(np.int32), ref["colidx"],
                      synth.upstream_grad(len(ref["colidx"]), seed))
        dA_ref, dB_ref = O.grad(p["A"], p["B"], G)
        d = to_dev(p, "plus_times_f32")
        Gd = _lib.DeviceCsr.from_host(G)
        handle.force("auto")
        dA, dB = _lib.msgemm_backward(handle, d["A"], d["B"], Gd)
        handle.sync_status()
        # bound: sum of |g||b| (dA) and |a||g| (dB), fp64 via dense products
        Ad, Bd, Gdd = p["A"].to_dense(), p["B"].to_dense(), G.to_dense()
        SA = (np.abs(Gdd) @ np.abs(Bd).T)[np.repeat(np.arange(m), np.diff(p["A"].rowptr)), p["A"].colidx]
        SB = (np.abs(Ad).T @ np.abs(Gdd))[np.repeat(np.arange(k), np.diff(p["B"].rowptr)), p["B"].colidx]
        assert np.all(np.abs(dA.cpu().numpy() - dA_ref) <= 1e-5 * SA + 1e-30)
        assert np.all(np.abs(dB.cpu().numpy() - dB_ref) <= 1e-5 * SB + 1e-30)


def test_autograd_function(handle):
    from paper_2111_09947_gb300.autograd import masked_spgemm_autograd
    p = synth.autograd_problem(scale=8, ef=16, seed=5)
    d = to_dev(p, "plus_times_f32")
    a = d["A"].values.clone().requires_grad_(True)
    b = d["B"].values.clone().requires_grad_(True)
    handle.force("auto")
    cv, crp, cci = masked_spgemm_autograd(a, b, d["M"], d["A"], d["B"], handle)
    g = torch.from_numpy(synth.upstream_grad(cv.numel(), 5)).cuda()
    (cv * g).sum().backward()
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
    G = synth.Csr(p["M"].nrows, p["M"].ncols, ref["rowptr"].astype(np.int32), ref["colidx"],
                  synth.upstream_grad(len(ref["colidx"]), 5))
    dA_ref, dB_ref = O.grad(p["A"], p["B"], G)
    # per-entry bound: 1e-5 * sum |g||b| (dA) and 1e-5 * sum |a||g| (dB), fp64
    SA, SB = O.grad(p["A"].with_values(np.abs(p["A"].values)), p["B"].with_values(np.abs(p["B"].values)),
                    G.with_values(np.abs(G.values)))
    assert np.all(np.abs(a.grad.cpu().numpy().astype(np.float64) - dA_ref) <= 1e-5 * SA + 1e-30)
    assert np.all(np.abs(b.grad.cpu().numpy().astype(np.float64) - dB_ref) <= 1e-5 * SB + 1e-30)
    # the forward values of the same call, at the forward bound
    err = np.abs(cv.detach().cpu().numpy().astype(np.float64) - ref["values"])
    assert np.array_equal(crp.cpu().numpy(), ref["rowptr"]) and np.array_equal(cci.cpu().numpy(), ref["colidx"])
    assert np.all(err <= 1e-5 * ref["S"])


@pytest.mark.parametrize("kicks", [0, 1, 64])
@pytest.mark.parametrize("semiring", SEMIRINGS)
def test_hash_build_paths(handle, semiring, kicks):
    """Hash rows (Sec. 5.3) forced on every row, with the cuckoo insertion's
    move limit at its default (64), at 1 (insertions run out often: the retry
    with the second hash pair and the linear fallback both run) and at 0
    (linear probing only).  Mask rows from 1 to 1500 entries put warp and CTA
    rows (both slab sizes) at load factors from 1/8 up to 1/2; the gradient
    form (values at the mask's slots) and the two-phase form go through the
    same lookups."""
    rng = np.random.default_rng(500 + kicks)
    m, k, n = 600, 500, 40000
    mdeg = np.array([1, 7, 60, 140, 230, 287, 700, 1500])[np.arange(m) % 8]
    rows, cols = [], []
    for i in range(m):
        c = np.sort(rng.choice(n, size=int(mdeg[i]), replace=False))
        rows.append(np.full(len(c), i))
        cols.append(c)
    M = synth.coo_to_csr(m, n, np.concatenate(rows).astype(np.int32), np.concatenate(cols).astype(np.int32))
    q = synth.random_problem(m, k, n, 12.0, 300.0, 1.0, 501 + kicks, GEN[semiring])
    q["M"] = M
    ref = O.masked_spgemm(q["M"], q["A"], q["B"], semiring)
    handle.set_option(_lib.OPT_HASH_KICKS, kicks)
    try:
        for phases in (1, 2):
            handle.set_option(_lib.OPT_PHASES, phases)
            # repeated: a lookup that reads the table before the build is
            # visible loses products only in some runs
            for rep in range(3):
                res = run(handle, q, semiring, False, "hash")
                assert_parity(res, ref, semiring, ctx=f"kicks={kicks} phases={phases} rep={rep}")
            counts = handle.bin_counts()
            assert counts["hash_w"] > 0 and counts["hash_b"] > 0
            if semiring == "plus_times_i64":   # 12-byte slots: the 1500-entry rows need the large slab
                assert counts["hash_l"] > 0
    finally:
        handle.set_option(_lib.OPT_PHASES, 1)
        handle.set_option(_lib.OPT_HASH_KICKS, 64)
        handle.force("auto")


def _grad_bounds(p, G):
    SA, SB = O.grad(p["A"].with_values(np.abs(p["A"].values)), p["B"].with_values(np.abs(p["B"].values)),
                    G.with_values(np.abs(G.values)))
    return SA, SB


@pytest.mark.parametrize("force", ["auto", "hash", "mca", "msa"])
def test_backward_plan(handle, force):
    """The planned backward (transposed patterns built once) against the
    oracle's gradients at the per-entry bounds, on two value sets of the same
    pattern in a row; a plan refuses operands with another pattern."""
    m, k, n = 700, 900, 800
    p = synth.random_problem(m, k, n, 9.0, 7.0, 40.0, 606, "f32")
    d = to_dev(p, "plus_times_f32")
    handle.force(force)
    try:
        plan = _lib.BackwardPlan(handle, d["A"], d["B"])
        for rep in range(2):
            if rep:
                p["A"] = p["A"].with_values(synth.normal_f32(p["A"].nnz, 700, 4))
                p["B"] = p["B"].with_values(synth.normal_f32(p["B"].nnz, 700, 5))
                d["A"].values.copy_(torch.from_numpy(p["A"].values))
                d["B"].values.copy_(torch.from_numpy(p["B"].values))
            ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
            G = synth.Csr(m, n, ref["rowptr"].astype(np.int32), ref["colidx"],
                          synth.upstream_grad(len(ref["colidx"]), 60 + rep))
            dA_ref, dB_ref = O.grad(p["A"], p["B"], G)
            SA, SB = _grad_bounds(p, G)
            dA, dB = _lib.msgemm_backward(handle, d["A"], d["B"], _lib.DeviceCsr.from_host(G), plan=plan)
            handle.sync_status()
            assert np.all(np.abs(dA.cpu().numpy().astype(np.float64) - dA_ref) <= 1e-5 * SA + 1e-30)
            assert np.all(np.abs(dB.cpu().numpy().astype(np.float64) - dB_ref) <= 1e-5 * SB + 1e-30)
            # only dB, then only dA
            _, dB1 = _lib.msgemm_backward(handle, d["A"], d["B"], _lib.DeviceCsr.from_host(G), need_dA=False,
                                          plan=plan)
            dA1, _ = _lib.msgemm_backward(handle, d["A"], d["B"], _lib.DeviceCsr.from_host(G), need_dB=False,
                                          plan=plan)
            handle.sync_status()
            assert np.all(np.abs(dA1.cpu().numpy().astype(np.float64) - dA_ref) <= 1e-5 * SA + 1e-30)
            assert np.all(np.abs(dB1.cpu().numpy().astype(np.float64) - dB_ref) <= 1e-5 * SB + 1e-30)
        # another pattern (a copy of A's arrays at other addresses) is refused
        A2 = _lib.DeviceCsr(d["A"].nrows, d["A"].ncols, d["A"].rowptr.clone(), d["A"].colidx.clone(), d["A"].values)
        with pytest.raises(_lib.MsgemmError) as e:
            _lib.msgemm_backward(handle, A2, d["B"], _lib.DeviceCsr.from_host(G), plan=plan)
        assert e.value.status == 1
        plan.close()
    finally:
        handle.force("auto")


def test_backward_plan_outlived_by_handle_close():
    """Closing a handle destroys the plans made with it first (their memory
    came from its allocator); a closed plan is refused."""
    p = synth.random_problem(50, 40, 60, 4.0, 4.0, 6.0, 9, "f32")
    d = to_dev(p, "plus_times_f32")
    h = _lib.Handle()
    plan = _lib.BackwardPlan(h, d["A"], d["B"])
    h.close()
    assert plan.p is None
    h2 = _lib.Handle()
    try:
        ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
        G = _lib.DeviceCsr.from_host(synth.Csr(50, 60, ref["rowptr"].astype(np.int32), ref["colidx"],
                                               synth.upstream_grad(len(ref["colidx"]), 1)))
        with pytest.raises(_lib.MsgemmError):
            _lib.msgemm_backward(h2, d["A"], d["B"], G, plan=plan)
    finally:
        h2.close()


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("qflops", [0, 1024, 1 << 20])
def test_team_of_eight_mca(handle, semiring, qflops):
    """Rows with at most 8 mask entries and at most MSGEMM_OPT_QTEAM_FLOPS
    push products take the mask-compressed accumulator on an eight-lane team
    (Sec. 5.4; mask row and accumulators in registers).  Mask rows of 0 to 12
    entries, A rows of 0 to 40 entries over B rows of 1 to 300: some rows
    qualify, some are too heavy or have too many mask entries.  AUTO and forced
    MCA, one and two phases, against the oracle."""
    rng = np.random.default_rng(77)
    m, k, n = 900, 700, 5000
    mdeg = np.arange(m) % 13
    rows, cols = [], []
    for i in range(m):
        c = np.sort(rng.choice(n, size=int(mdeg[i]), replace=False))
        rows.append(np.full(len(c), i))
        cols.append(c)
    M = synth.coo_to_csr(m, n, np.concatenate(rows).astype(np.int32), np.concatenate(cols).astype(np.int32))
    q = synth.random_problem(m, k, n, 10.0, 30.0, 1.0, 78, GEN[semiring])
    q["M"] = M
    ref = O.masked_spgemm(q["M"], q["A"], q["B"], semiring)
    handle.set_option(_lib.OPT_QTEAM_FLOPS, qflops)
    try:
        for force in ("auto", "mca"):
            for phases in (1, 2):
                handle.set_option(_lib.OPT_PHASES, phases)
                res = run(handle, q, semiring, False, force)
                assert_parity(res, ref, semiring, ctx=f"q={qflops} force={force} phases={phases}")
                nq = handle.bin_counts()["mca_q"]
                assert (nq > 0) == (qflops > 0), nq
    finally:
        handle.set_option(_lib.OPT_PHASES, 1)
        handle.set_option(_lib.OPT_QTEAM_FLOPS, 1024)
        handle.force("auto")


def test_team_of_eight_gradient_form(handle):
    """The backward's dA product (mask = pattern(A), values at each mask
    entry's own slot) through the team-of-eight rows: every row of A has at
    most 8 entries, so with a high flop bound every row qualifies."""
    m, k, n = 600, 500, 700
    p = synth.random_problem(m, k, n, 4.0, 5.0, 30.0, 79, "f32")
    ref = O.masked_spgemm(p["M"], p["A"], p["B"], "plus_times_f32")
    G = synth.Csr(m, n, ref["rowptr"].astype(np.int32), ref["colidx"], synth.upstream_grad(len(ref["colidx"]), 79))
    dA_ref, dB_ref = O.grad(p["A"], p["B"], G)
    SA, SB = _grad_bounds(p, G)
    d = to_dev(p, "plus_times_f32")
    handle.set_option(_lib.OPT_QTEAM_FLOPS, 1 << 20)
    handle.set_option(_lib.OPT_DOT, 0)
    try:
        dA, dB = _lib.msgemm_backward(handle, d["A"], d["B"], _lib.DeviceCsr.from_host(G))
        handle.sync_status()
    finally:
        handle.set_option(_lib.OPT_QTEAM_FLOPS, 1024)
        handle.set_option(_lib.OPT_DOT, 1)
    assert np.all(np.abs(dA.cpu().numpy().astype(np.float64) - dA_ref) <= 1e-5 * SA + 1e-30)
    assert np.all(np.abs(dB.cpu().numpy().astype(np.float64) - dB_ref) <= 1e-5 * SB + 1e-30)


@pytest.mark.parametrize("semiring", SEMIRINGS)
@pytest.mark.parametrize("qflops", [0, 1024, 1 << 20])
def test_team_of_eight_dot(handle, semiring, qflops):
    """Pull rows (Sec. 4.1) with at most 8 mask entries and at most
    MSGEMM_OPT_QTEAM_FLOPS pull pairs run on an eight-lane team that
    binary-searches A_i* in global memory.  Mask rows of 0 to 36 entries (the
    longer ones take the warp kinds), A rows up to ~200 entries (so pull is cheaper
    than push), forced pull and AUTO, one and two phases, against the oracle."""
    rng = np.random.default_rng(88)
    m, k, n = 800, 900, 3000
    mdeg = np.arange(m) % 37
    rows, cols = [], []
    for i in range(m):
        c = np.sort(rng.choice(n, size=int(mdeg[i]), replace=False))
        rows.append(np.full(len(c), i))
        cols.append(c)
    M = synth.coo_to_csr(m, n, np.concatenate(rows).astype(np.int32), np.concatenate(cols).astype(np.int32))
    q = synth.random_problem(m, k, n, 60.0, 20.0, 1.0, 89, GEN[semiring])
    q["M"] = M
    ref = O.masked_spgemm(q["M"], q["A"], q["B"], semiring)
    handle.set_option(_lib.OPT_QTEAM_FLOPS, qflops)
    try:
        for force in ("dot", "auto"):
            for phases in (1, 2):
                handle.set_option(_lib.OPT_PHASES, phases)
                res = run(handle, q, semiring, False, force)
                assert_parity(res, ref, semiring, ctx=f"q={qflops} force={force} phases={phases}")
                nq = handle.bin_counts()["dot_q"]
                if force == "dot":
                    assert (nq > 0) == (qflops > 0), nq
    finally:
        handle.set_option(_lib.OPT_PHASES, 1)
        handle.set_option(_lib.OPT_QTEAM_FLOPS, 1024)
        handle.force("auto")
