"""Host-side helpers of bench.py (no GPU): byte models and the CPU-baseline
sampling loop, and the reference arm's JSON line."""
import json
import os
import subprocess
import sys

import numpy as np

import bench
from paper_2111_09947_gb300 import synth


def test_q_min_and_kernel_bytes():
    p = synth.random_problem(50, 40, 60, 4.0, 4.0, 6.0, 3, "f32")
    M, A, B = p["M"], p["A"], p["B"]
    q = bench.q_min_bytes(M, A, B, 10, 4, 4)
    assert q == 4 * 51 + A.nnz * 8 + 4 * 41 + B.nnz * 8 + 4 * 51 + 4 * M.nnz + 4 * 51 + 10 * 8
    kinds = np.zeros(50, np.uint8)
    kinds[::2] = 3
    crp = np.zeros(51, np.int32)
    kb = bench.kernel_bytes(kinds, 3, M, A, B, crp, 4, 4)
    rows = np.arange(0, 50, 2)
    anz = np.diff(A.rowptr)
    ks = np.unique(np.concatenate([A.row(i) for i in rows]))
    want = (8 + anz[rows] * 8).sum() + (8 + np.diff(M.rowptr)[rows] * 4).sum() + \
        (8 + np.diff(B.rowptr)[ks] * 8).sum()
    assert kb == want
    assert bench.kernel_bytes(kinds, 5, M, A, B, crp, 4, 4) == 0
    # a pattern B (no value array) reads no value bytes of B
    assert bench.q_min_bytes(M, A, B, 10, 4, 4, vb_b=0) == q - B.nnz * 4
    assert bench.kernel_bytes(kinds, 3, M, A, B, crp, 4, 4, 0) == want - (np.diff(B.rowptr)[ks] * 4).sum()


def test_oracle_sample_rate_runs():
    p = synth.triangle_counting(scale=10, ef=8, seed=1)
    L = p["M"]
    kfn = bench.kept_fn_for("plus_pair_i64", L, L, L, False)
    rate, secs, rows, res = bench.oracle_sample_rate(L, L, L, "plus_pair_i64", False, 5.0, kept_fn=kfn)
    assert rate >= 0 and secs > 0 and rows == L.nrows      # a small C fits the budget whole
    # the whole-C count equals the oracle's triangle count
    from oracle import oracle as O
    assert kfn(None, res) == int(O.masked_spgemm(L, L, L, "plus_pair_i64")["values"].sum())


def test_oracle_plan_budget():
    """The planner takes the whole C when it fits the budget and otherwise a
    row sample that fits it."""
    p = synth.triangle_counting(scale=12, ef=16, seed=1)
    L = p["M"]
    whole, fixed, per_row = bench.oracle_plan(L, L, L, "plus_pair_i64", False, 100.0)
    assert whole is None and fixed >= 0 and per_row > 0
    part, fixed, per_row = bench.oracle_plan(L, L, L, "plus_pair_i64", False, fixed + per_row * 100)
    assert part is not None and 1 <= part < L.nrows


def test_kept_fn_for_semirings():
    """Kept products from an fp32 result (a plus-pair call on the same rows)
    equal the plus-pair sum."""
    from oracle import oracle as O
    q = synth.random_problem(80, 60, 90, 5.0, 5.0, 9.0, 4, "f32")
    rows = np.array([1, 5, 7, 40], np.int32)
    res = O.masked_spgemm(q["M"], q["A"], q["B"], "plus_times_f32", rows=rows)
    pp = O.masked_spgemm(q["M"], q["A"], q["B"], "plus_pair_i64", rows=rows)
    assert bench.kept_fn_for("plus_times_f32", q["M"], q["A"], q["B"], False)(rows, res) == int(pp["values"].sum())


def test_reference_arm_line():
    env = dict(os.environ, OMP_NUM_THREADS="2")
    out = subprocess.run([sys.executable, bench.__file__, "--impl", "reference", "--scale", "10", "--steps", "2",
                          "--warmup", "1"], capture_output=True, text=True, env=env, timeout=300)
    assert out.returncode == 0, out.stderr
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "masked GFLOP/s"
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
    # the same config dict as the GPU arm builds for this workload
    assert line["config"] == bench.build_workload("tc", 10, synth.BASE_SEED).config


def test_oracle_threads_form_and_thread_independence():
    """The one-core / all-core oracle figure runs, and the oracle's result does
    not depend on its thread count."""
    from oracle import oracle as O
    wl = bench.build_workload("er", None, synth.BASE_SEED)
    out = bench.oracle_threads_form(wl, seconds=0.05)
    assert out["threads_1"] > 0 and out["threads_all"] > 0 and out["cores"] == os.cpu_count()
    M, A, B, _ = wl.mats[0]
    try:
        O.set_threads(1)
        one = O.masked_spgemm(M, A, B, "plus_times_f32")
    finally:
        O.set_threads(os.cpu_count())
    many = O.masked_spgemm(M, A, B, "plus_times_f32")
    for k in ("rowptr", "colidx", "values", "S"):
        assert np.array_equal(one[k], many[k])
