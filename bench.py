#!/usr/bin/env python
"""Masked SpGEMM benchmark on GB300.

Default workload (--workload tc): triangle counting on an R-MAT graph of
scale 20 (edge factor 16, Graph500 quadrant probabilities), symmetrised,
loops and duplicates removed, degree-relabelled; C = L .* (L L) on plus-pair
int64 and the count sum(C) (Sec. 8.2).  One step = the whole path on resident
inputs: binning, accumulators, compaction and the count reduction.  The
metric is masked GFLOP/s = 2 x (products kept by the mask) / time.

Other workloads (also reported under "forms" of the default run):
  er        plain fp32 product, Erdos-Renyi n = 4096, 8 entries per row
  bfs       complemented step of multi-source BFS (512 sources, scale 20)
  batched   256 independent fp32 products in one call (vs 256 calls)
  autograd  forward + backward of the differentiable form (R-MAT scale 18)
  bc        (form only) betweenness centrality from 512 sources, R-MAT scale
            20, reported in TEPS
  ktruss    (form only) 5-truss of the R-MAT scale-20 graph, masked flops of
            all rounds / time

--impl reference times the CPU oracle (the plain C program under oracle/)
on bounded row samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

REPO = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, REPO)

import numpy as np  # noqa: E402

L2_FLUSH_BYTES = 256 << 20     # > 129 MB L2
PEAKS_FALLBACK = {"hbm_gbs": 6800.0}
SMS = 152                      # GB300 streaming multiprocessors
SM_MAX_MHZ = 2070.0
WORKLOADS = ("tc", "er", "bfs", "batched", "autograd")
_T0 = time.perf_counter()


def log(msg: str) -> None:
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=WORKLOADS, default="tc")
    ap.add_argument("--scale", type=int, default=None, help="R-MAT scale (tc: 20, bfs: 20, autograd: 18)")
    ap.add_argument("--no-forms", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="time the default policy (no untimed tuning first)")
    ap.add_argument("--sweep", choices=["er", "rmat"], default=None,
                    help="policy sweeps instead of the benchmark line: Erdos-Renyi n x degrees with every "
                         "accumulator forced vs AUTO, or triangle counting over R-MAT scales")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--batch-products", type=int, default=256,
                    help="products of the batched workload (256; fewer for a small profiling case)")
    ap.add_argument("--sweep-out", default=None, help="write the sweep's table (with the kernel source hash) "
                                                       "to this JSON file")
    ap.add_argument("--sweep-max-log2", type=int, default=22, help="largest n = 2^x of the Erdos-Renyi sweep")
    return ap.parse_args(argv)


def peaks():
    path = os.path.join(REPO, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    except Exception:
        return {"hbm_gbs": PEAKS_FALLBACK["hbm_gbs"], "source": "fallback 6.8 TB/s"}


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return summarize_clocks(self.lines)


def summarize_clocks(lines):
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 9:
            continue
        try:
            sm.append(float(parts[1]))
            smax.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- byte / flop models
def push_products(A, B) -> int:
    bl = np.diff(B.rowptr).astype(np.int64)
    return int(bl[A.colidx].sum())


def q_min_bytes(M, A, B, nnz_c, vb_in, vb_out, complement=False, vb_b=None) -> int:
    """Compulsory bytes (read A, B, M once, write C once); vb_b = value bytes
    of B (0 for a pattern operand), by default vb_in."""
    vb_b = vb_in if vb_b is None else vb_b
    q = 4 * (A.nrows + 1) + A.nnz * (4 + vb_in)
    q += 4 * (B.nrows + 1) + B.nnz * (4 + vb_b)
    q += 4 * (M.nrows + 1) + 4 * M.nnz
    q += 4 * (M.nrows + 1) + nnz_c * (4 + vb_out)
    return int(q)


def kernel_bytes(kinds, kind_id, M, A, B, C_rp, vb_in, vb_out, vb_b=None) -> int:
    """Compulsory bytes of the rows one accumulator kernel processes: their
    rows of A and M, the distinct rows of B they touch (vb_b value bytes per
    entry: 0 for a pattern operand, by default vb_in), their output."""
    vb_b = vb_in if vb_b is None else vb_b
    rows = np.nonzero(kinds == kind_id)[0]
    if len(rows) == 0:
        return 0
    anz = np.diff(A.rowptr).astype(np.int64)
    mnz = np.diff(M.rowptr).astype(np.int64)
    cnz = np.diff(C_rp).astype(np.int64)
    q = int((8 + anz[rows] * (4 + vb_in)).sum() + (8 + mnz[rows] * 4).sum() + (cnz[rows] * (4 + vb_out)).sum())
    sel = np.zeros(A.nrows, bool)
    sel[rows] = True
    rowmask = np.repeat(sel, anz)
    ks = np.unique(A.colidx[rowmask])
    bl = np.diff(B.rowptr).astype(np.int64)
    q += int((8 + bl[ks] * (4 + vb_b)).sum())
    return q


def kernel_products(kinds, kind_id, A, B) -> int:
    """Push products (sum of |B_k*| over A_i*) of the rows of one kind."""
    rows = np.nonzero(kinds == kind_id)[0]
    if len(rows) == 0:
        return 0
    anz = np.diff(A.rowptr).astype(np.int64)
    sel = np.zeros(A.nrows, bool)
    sel[rows] = True
    bl = np.diff(B.rowptr).astype(np.int64)
    return int(bl[A.colidx[np.repeat(sel, anz)]].sum())


def code_only(src: str) -> str:
    """C/CUDA source without comments and blank lines (what the compiler sees
    of it, up to layout), so that comment edits do not count as changes."""
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    return "\n".join(line.rstrip() for line in src.splitlines() if line.strip())


def source_hash() -> str:
    """Hash of the kernel sources (comments excluded)."""
    h = hashlib.sha1()
    cdir = os.path.join(REPO, "paper_2111_09947_gb300", "csrc")
    for name in sorted(os.listdir(cdir)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(cdir, name), encoding="utf-8") as f:
                h.update(name.encode())
                h.update(code_only(f.read()).encode())
    return h.hexdigest()[:12]


def profile_entry(kernel: str, workload: str) -> dict:
    """The committed ncu figures of a kernel on a workload (DRAM bytes per
    launch, L2 hit rate), if they were taken on the current kernel sources;
    else an empty dict."""
    path = os.path.join(REPO, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return {}
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("source_sha") != source_hash():
        return {}
    return e


def traffic_for(kernel: str, workload: str):
    return profile_entry(kernel, workload).get("dram_bytes_per_launch")


VB = {"plus_times_f32": (4, 4), "plus_times_i64": (8, 8), "plus_pair_i64": (0, 8)}


# ----------------------------------------------------------------- workloads
class Workload:
    """A benchmark workload: host inputs and its counts.

    mats: list of (M, A, B, complement) host products one step runs;
    kept: products kept by the masks per step; masked flops = 2 * kept."""

    def __init__(self, name, semiring, config, mats, dtype, pattern_b=False):
        self.name = name
        self.pattern_b = pattern_b   # B goes to the device without values (every value 1)
        self.semiring = semiring
        self.config = dict(config, l2="GPU arm: flushed before every timed step (256 MiB write)")
        self.mats = mats
        self.dtype = dtype
        self.kept = None
        self.nnz_c = None


def build_workload(name, scale, seed, nprod=256):
    from paper_2111_09947_gb300 import synth
    if name == "tc":
        scale = scale or 20
        tc = synth.triangle_counting(scale=scale, ef=16, seed=seed)
        L = tc["M"]
        cfg = {"workload": f"triangle counting: R-MAT scale {scale}, edge factor 16, (a,b,c)=(0.57,0.19,0.19), "
                           "symmetrised, loops/duplicates removed, degree-relabelled, L strict lower; "
                           "C = L .* (L L) plus-pair int64 + count", "n": L.nrows, "nnz_L": L.nnz}
        return Workload(name, "plus_pair_i64", cfg, [(L, L, L, False)], "int64")
    if name == "er":
        p = synth.er_plain_f32(seed=seed)
        cfg = {"workload": "plain masked product, fp32: A, B, M independent Erdos-Renyi n=4096, 8 entries per row, "
                           "values uniform[-1,1)", "n": 4096, "nnz_A": p["A"].nnz, "nnz_M": p["M"].nnz}
        return Workload(name, "plus_times_f32", cfg, [(p["M"], p["A"], p["B"], False)], "f32")
    if name == "bfs":
        scale = scale or 20
        b = synth.bfs_step(scale=scale, ef=16, nsrc=512, seed=seed)
        cfg = {"workload": f"multi-source BFS step, complemented mask: C = !Visited .* (F A), plus-times int64; "
                           f"A = R-MAT scale {scale} ef 16 symmetrised (values 1, passed as a pattern operand), "
                           "F = level-2 frontier of 512 random sources with path counts", "n": b["B"].nrows,
               "nnz_F": b["A"].nnz, "nnz_visited": b["M"].nnz, "nnz_A": b["B"].nnz}
        return Workload(name, "plus_times_i64", cfg, [(b["M"], b["A"], b["B"], True)], "int64", pattern_b=True)
    if name == "batched":
        ps = synth.batched_problems(nprod=nprod, seed=seed)
        cfg = {"workload": f"{nprod} independent fp32 products in one call: n log-uniform in [2^10, 2^16], A/B R-MAT "
                           "ef 8, M Erdos-Renyi with {1,16,256} entries per row",
               "rows": int(sum(p["n"] for p in ps)), "nnz_M": int(sum(p["M"].nnz for p in ps))}
        return Workload(name, "plus_times_f32", cfg, [(p["M"], p["A"], p["B"], False) for p in ps], "f32")
    if name == "autograd":
        scale = scale or 18
        a = synth.autograd_problem(scale=scale, ef=16, seed=seed)
        cfg = {"workload": f"differentiable masked product, fp32, forward + backward: A R-MAT scale {scale} ef 16 "
                           "N(0,1), B = pattern(A^T) N(0,1), M = pattern(A), G N(0,1) on C",
               "n": a["A"].nrows, "nnz_A": a["A"].nnz}
        return Workload(name, "plus_times_f32", cfg, [(a["M"], a["A"], a["B"], False)], "f32")
    raise ValueError(name)


class DeviceRun:
    """Device copies of a workload's inputs and its step callable."""

    def __init__(self, torch, _lib, synth, h, wl, dev):
        self.torch, self._lib, self.h, self.wl, self.dev = torch, _lib, h, wl, dev
        sr = wl.semiring
        vd = {"plus_times_f32": torch.float32, "plus_times_i64": torch.int64, "plus_pair_i64": None}[sr]
        keep = sr != "plus_pair_i64"
        cache = {}

        def dv(m, values):
            key = (id(m), values)
            if key not in cache:
                d = _lib.DeviceCsr.from_host(m, device=dev, values_dtype=vd if values else None)
                if not values:
                    d.values = None
                cache[key] = d
            return cache[key]
        self.prods = [(dv(M, False), dv(A, keep), dv(B, keep and not wl.pattern_b), c) for (M, A, B, c) in wl.mats]
        self.G = None
        self.plan = None
        self.allreduce = None
        if wl.name == "autograd":
            M, A, B, _ = self.prods[0]
            res = _lib.msgemm_run(h, M, A, B, sr).trimmed()
            self.G = _lib.DeviceCsr(res.nrows, res.ncols, res.rowptr, res.colidx,
                                    torch.from_numpy(synth.upstream_grad(res.nnz)).to(dev))
            # the transposed patterns, built once as the autograd function does
            # on its first backward (patterns are fixed across steps)
            self.plan = _lib.BackwardPlan(h, A, B)

    def step(self):
        """One step; returns (result object, a device scalar to read back)."""
        _lib, h, sr = self._lib, self.h, self.wl.semiring
        name = self.wl.name
        if name == "tc":
            M, A, B, _ = self.prods[0]   # L, L, L; or a row block of L, its rows of L, and L
            r = _lib.msgemm_run(h, M, A, B, sr)
            cnt = _lib.msgemm_reduce_sum(h, r, sr)
            if self.allreduce is not None:   # row-sharded: sum the partial counts over the ranks
                self.allreduce(cnt)
            return r, cnt
        if name == "batched":
            Ms, As, Bs = [p[0] for p in self.prods], [p[1] for p in self.prods], [p[2] for p in self.prods]
            outs = _lib.msgemm_run_batched(h, Ms, As, Bs, sr)
            return outs[0], outs[-1].d_nnz
        M, A, B, comp = self.prods[0]
        if name == "autograd":
            r = _lib.msgemm_run(h, M, A, B, sr)
            _lib.msgemm_backward(h, A, B, self.G, plan=self.plan)
            return r, r.d_nnz
        r = _lib.msgemm_run(h, M, A, B, sr, comp)
        return r, r.d_nnz

    def per_product_step(self):
        """The batched workload as separate calls (the plain path)."""
        for (M, A, B, c) in self.prods:
            self._lib.msgemm_run(self.h, M, A, B, self.wl.semiring, c)

    def count_kept(self):
        """Products kept by the masks: the sum of the plus-pair result."""
        _lib, h = self._lib, self.h

        def pat(d):
            return _lib.DeviceCsr(d.nrows, d.ncols, d.rowptr, d.colidx, None)
        kept, nnz_c = 0, 0
        for (M, A, B, c) in self.prods:
            r = _lib.msgemm_run(h, pat(M), pat(A), pat(B), "plus_pair_i64", c)
            kept += int(_lib.msgemm_reduce_sum(h, r, "plus_pair_i64").item())
            nnz_c += r.nnz()
        if self.wl.name == "autograd":
            # backward: dA = pattern(A) .* (G B^T), dB = pattern(B) .* (A^T G)
            M, A, B, _ = self.prods[0]
            Bt = _lib.msgemm_transpose(h, pat(B), 0, True)
            At = _lib.msgemm_transpose(h, pat(A), 0, True)
            for (mm, aa, bb) in ((pat(A), pat(self.G), pat(Bt)), (pat(B), pat(At), pat(self.G))):
                r = _lib.msgemm_run(h, mm, aa, bb, "plus_pair_i64")
                kept += int(_lib.msgemm_reduce_sum(h, r, "plus_pair_i64").item())
        return kept, nnz_c


def timed_steps(torch, step, steps, flush_buf, stream, after=None):
    """Per-step device times (ms) with CUDA events on the launching stream;
    L2 flushed (a write larger than L2) before each step, outside the timing."""
    times = []
    for s in range(steps):
        flush_buf.fill_(s & 0xFF)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
        if after:
            after()
    return times


def oracle_plan(M, A, B, semiring, complement, target_s, rng_seed=7):
    """Sizes one oracle call to about target_s seconds.  Every call of the
    merge method transposes all of B once (a fixed cost per call), so the
    cost is fitted as t = fixed + per_row * rows from two untimed probe calls
    (k and 4k uniformly drawn rows); the plan is the whole C when that fits
    the budget, else the number of rows that does.  Returns (rows or None for
    the whole C, the fitted fixed seconds, the fitted seconds per row)."""
    from oracle import oracle as O
    rng = np.random.default_rng(rng_seed)
    m = M.nrows
    method = O.ESC if complement else O.MERGE
    k = max(1, min(m, int(m * 0.002)))
    ts = []
    for kk in (k, min(m, 4 * k)):
        rows = np.sort(rng.choice(m, size=kk, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        O.masked_spgemm(M, A, B, semiring, complement=complement, method=method, rows=rows)
        ts.append((kk, time.perf_counter() - t0))
    (k1, t1), (k2, t2) = ts
    per_row = max((t2 - t1) / max(k2 - k1, 1), t2 / k2 * 0.05, 1e-9)
    fixed = max(0.0, t2 - per_row * k2)
    if fixed + per_row * m <= target_s:
        return None, fixed, per_row
    return max(1, min(m, int((target_s - fixed) / per_row))), fixed, per_row


def oracle_timed_call(M, A, B, semiring, complement, nrows, rng, kept_fn):
    """One timed oracle call on the whole C (nrows None) or on nrows uniformly
    drawn rows; returns (seconds, masked flops of what it computed, rows)."""
    from oracle import oracle as O
    method = O.ESC if complement else O.MERGE
    rows = None if nrows is None else np.sort(rng.choice(M.nrows, size=nrows, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    res = O.masked_spgemm(M, A, B, semiring, complement=complement, method=method, rows=rows)
    dt = time.perf_counter() - t0
    return dt, 2 * kept_fn(rows, res), (M.nrows if rows is None else len(rows)), res


def oracle_sample_rate(M, A, B, semiring, complement, target_s, rng_seed=7, kept_fn=None):
    """The CPU oracle timed on one call of about target_s seconds (the whole C
    when it fits); returns (masked GFLOP/s, seconds, rows, result)."""
    nrows, _, _ = oracle_plan(M, A, B, semiring, complement, target_s, rng_seed)
    dt, flops, nr, res = oracle_timed_call(M, A, B, semiring, complement, nrows,
                                           np.random.default_rng(rng_seed + 1), kept_fn)
    return flops / dt / 1e9, dt, nr, res


def oracle_threads_form(wl, seconds=1.5):
    """The oracle on one host core and on all of them, on row samples of a
    one-product workload (its first product), as masked GFLOP/s."""
    from oracle import oracle as O
    M, A, B, comp = wl.mats[0]
    kfn = kept_fn_for(wl.semiring, M, A, B, comp)
    cores = os.cpu_count()
    out = {"unit": "GFLOP/s", "kind": "oracle", "cores": cores}
    try:
        for label, n in (("threads_1", 1), ("threads_all", cores)):
            O.set_threads(n)
            rate, secs, rows, _ = oracle_sample_rate(M, A, B, wl.semiring, comp, seconds, kept_fn=kfn)
            out[label] = round(rate, 5)
            out[label + "_sample"] = f"{rows} of {M.nrows} rows, {secs:.2f} s"
    finally:
        O.set_threads(cores)
    return out


def kept_fn_for(semiring, M, A, B, complement):
    """Products kept in an oracle result: its sum on plus-pair (each entry
    counts its products), else a plus-pair oracle call on the same rows."""
    if semiring == "plus_pair_i64":
        return lambda rows, res: int(res["values"].sum())
    return kept_from_oracle(M, A, B, complement)


def kept_from_oracle(M, A, B, complement):
    """kept_fn for oracle samples: products kept in the sampled rows, counted
    by the oracle in plus-pair (not part of the timed oracle call)."""
    from oracle import oracle as O

    def fn(rows, res):
        pp = O.masked_spgemm(M, A, B, "plus_pair_i64", complement=complement,
                             method=O.ESC if complement else O.MERGE, rows=rows)
        return int(pp["values"].sum())
    return fn


# ----------------------------------------------------------------- measurement
def measure(torch, _lib, synth, h, wl, dev, stream, flush, steps, warmup, clocks_gpu=None, autotune=True,
            allreduce=None, dist_sync=False):
    """Times `steps` steps of a workload; returns a dict of measurements.
    With autotune, a fresh handle's policy is first tuned on the workload's
    products by the library's autotuner (untimed; its duration is reported)."""
    if autotune:
        h = _lib.Handle(dev)
    run = DeviceRun(torch, _lib, synth, h, wl, dev)
    wl.kept, wl.nnz_c = run.count_kept()
    run.allreduce = allreduce
    tune_s = None
    if autotune:
        t0 = time.perf_counter()
        Ms, As, Bs, comps = (list(x) for x in zip(*run.prods))
        _lib.msgemm_autotune(h, Ms, As, Bs, wl.semiring, complement=comps)
        torch.cuda.synchronize()
        tune_s = round(time.perf_counter() - t0, 2)
    # the timed steps run as a user would run them: the library's phase
    # profiler off (it records events around every phase)
    h.set_option(_lib.OPT_PROFILE, 0)
    for _ in range(warmup):
        run.step()
    torch.cuda.synchronize()
    kinds = h.row_kinds(wl.mats[0][0].nrows) if len(wl.mats) == 1 and wl.name != "autograd" else None
    clocks = ClockSampler(clocks_gpu) if clocks_gpu is not None else None
    if clocks:
        clocks.start()
    per_phase = {}
    l0 = _lib.load().msgemm_kernel_launches()

    def collect():
        for name, ms in h.profile():
            per_phase.setdefault(name, []).append(ms)

    def sync_all():
        # every rank enters and leaves the timed region together (the main
        # measurement only: the forms run on rank 0 alone)
        torch.cuda.synchronize()
        if dist_sync:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
    sync_all()
    # profiler range = the timed region (for ncu --profile-from-start off; no effect otherwise)
    torch.cuda.profiler.start()
    times = timed_steps(torch, run.step, steps, flush, stream)
    torch.cuda.profiler.stop()
    sync_all()
    launches = _lib.load().msgemm_kernel_launches() - l0
    clk = clocks.stop() if clocks else None
    # per-phase device times: a separate, untimed pass of the same steps with
    # the library's event profile on (same stream, L2 flushed before each)
    h.set_option(_lib.OPT_PROFILE, 1)
    timed_steps(torch, run.step, max(3, min(steps, 10)), flush, stream, after=collect)
    h.set_option(_lib.OPT_PROFILE, 0)
    kind_rows = {k: v for k, v in h.bin_counts().items() if v} if wl.name != "autograd" else None
    out = {"times": times, "launches": launches, "clocks": clk, "per_phase": per_phase, "kinds": kinds, "run": run,
           "autotune_s": tune_s, "kind_rows": kind_rows}
    if wl.name == "batched":
        run.per_product_step()
        torch.cuda.synchronize()
        out["per_product_ms"] = statistics.median(timed_steps(torch, run.per_product_step, 3, flush, stream))
    if wl.name in ("batched", "er"):
        # the same products replayed from a captured CUDA graph (plain masks)
        Ms, As, Bs = [p[0] for p in run.prods], [p[1] for p in run.prods], [p[2] for p in run.prods]

        def graph_step():
            return _lib.msgemm_run_batched(h, Ms, As, Bs, wl.semiring, use_graph=True)
        for _ in range(3):
            graph_step()
        torch.cuda.synchronize()
        out["graph_ms"] = statistics.median(timed_steps(torch, graph_step, 5, flush, stream))
    if wl.name == "autograd":
        M, A, B, _ = run.prods[0]
        fwd = lambda: _lib.msgemm_run(h, M, A, B, wl.semiring)  # noqa: E731
        bwd = lambda: _lib.msgemm_backward(h, A, B, run.G, plan=run.plan)  # noqa: E731
        bwd0 = lambda: _lib.msgemm_backward(h, A, B, run.G)  # noqa: E731
        out["fwd_ms"] = statistics.median(timed_steps(torch, fwd, 5, flush, stream))
        out["bwd_ms"] = statistics.median(timed_steps(torch, bwd, 5, flush, stream))
        out["bwd_unplanned_ms"] = statistics.median(timed_steps(torch, bwd0, 5, flush, stream))
    return out


def bc_form(torch, _lib, synth, dev, stream, flush, steps, warmup, scale=20, nsrc=512):
    """Betweenness centrality from 512 sources on the R-MAT scale-20 graph
    (forward and backward stages, Sec. 8.3), timed as whole calls; TEPS =
    sources x edges / time, edges = undirected edges (stored entries / 2)."""
    g = synth.rmat_graph(scale, 16, synth.BASE_SEED, synth.S_A)
    src = synth.pick_sources(g, nsrc, synth.BASE_SEED)
    h = _lib.Handle(dev)
    A = _lib.DeviceCsr.from_host(synth.Csr(g.nrows, g.ncols, g.rowptr, g.colidx), device=dev)
    s = torch.from_numpy(np.asarray(src, np.int32)).to(dev)
    out = {}

    def step():
        out["r"] = _lib.msgemm_bc(h, A, s)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    times = timed_steps(torch, step, steps, flush, stream)
    h.close()
    ms = statistics.median(times)
    edges = g.nnz / 2
    return {"config": f"betweenness centrality, {nsrc} sources, R-MAT scale {scale} ef 16 symmetrised "
                      f"(forward: complemented int64 products, backward: plain fp32 products)",
            "ms_per_step": round(ms, 3), "levels": out["r"][1], "edges": int(edges),
            "gteps": round(nsrc * edges / (ms * 1e-3) / 1e9, 3)}


def ktruss_form(torch, _lib, synth, dev, stream, flush, steps, warmup, scale=20, k=5, autotune=True):
    """5-truss of the R-MAT scale-20 graph (Sec. 8.2): rounds of supports
    A .* (A A) on plus-pair and pruning until stable; metric = masked flops of
    all rounds / total time, the paper's.  The policy is tuned (untimed) on
    the first round's product."""
    g = synth.rmat_graph(scale, 16, synth.BASE_SEED, synth.S_A)
    h = _lib.Handle(dev)
    A = _lib.DeviceCsr.from_host(synth.Csr(g.nrows, g.ncols, g.rowptr, g.colidx), device=dev)
    tune_s = None
    if autotune:
        t0 = time.perf_counter()
        _lib.msgemm_autotune(h, [A], [A], [A], "plus_pair_i64")
        torch.cuda.synchronize()
        tune_s = round(time.perf_counter() - t0, 2)
    out = {}

    def step():
        out["r"] = _lib.msgemm_ktruss(h, A, k)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    times = timed_steps(torch, step, steps, flush, stream)
    h.close()
    ms = statistics.median(times)
    res, rounds, prods = out["r"]
    return {"config": f"{k}-truss, R-MAT scale {scale} ef 16 symmetrised: rounds of supports A .* (A A) on "
                      "plus-pair and pruning until no edge drops",
            "ms_per_step": round(ms, 3), "rounds": rounds, "masked_products": prods, "truss_edges": res.nnz() // 2,
            "masked_gflops": round(2 * prods / (ms * 1e-3) / 1e9, 3), "autotune_s": tune_s}


def roofline_of(_lib, wl, meas):
    """Roofline of the dominant accumulator kernel (single-product workloads):
    its compulsory bytes (rows of A and M it processes, distinct rows of B
    they touch, their output) over its mean launch time."""
    pk = peaks()
    kind_ids = {n: i for i, n in enumerate(_lib.KIND_NAMES)}
    cand = {n: statistics.mean(v) for n, v in meas["per_phase"].items() if n in kind_ids and n != "empty"}
    if not cand or meas["kinds"] is None:
        return None
    dom = max(cand, key=cand.get)
    dom_ms = cand[dom]
    M, A, B, comp = wl.mats[0]
    vb_in, vb_out = VB[wl.semiring]
    r, _ = meas["run"].step()
    C_rp = r.rowptr.cpu().numpy()
    kb = kernel_bytes(meas["kinds"], kind_ids[dom], M, A, B, C_rp, vb_in, vb_out, 0 if wl.pattern_b else vb_in)
    achieved = kb / (dom_ms * 1e-3) / 1e9
    prof = profile_entry(dom, wl.name)
    roof = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 2), "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / pk["hbm_gbs"], 5), "traffic": prof.get("dram_bytes_per_launch"),
            "l2_hit_pct": prof.get("l2_hit_pct"), "peak_source": pk["source"],
            "algorithmic_bytes_per_launch": kb, "kernel_ms": round(dom_ms, 4),
            "kernel_ms_source": "library event profile on the launching stream, separate pass of the same steps"}
    # The same kernel against the shared-memory pipe: every enumerated (push)
    # product needs at least one shared-memory access (a probe or an insert);
    # one SM retires one 32-lane shared-memory wavefront per clock.
    prods = kernel_products(meas["kinds"], kind_ids[dom], A, B)
    clk = (meas.get("clocks") or {}).get("sm_max_mhz") or SM_MAX_MHZ
    speak = SMS * 32 * clk * 1e6 / 1e9
    lookups = prods / (dom_ms * 1e-3) / 1e9
    smem = {"bound": "smem", "kernel": dom, "achieved": round(lookups, 2), "peak": round(speak, 1),
            "unit": "G shared accesses/s", "frac": round(lookups / speak, 5), "push_products_per_launch": prods,
            "peak_source": f"{SMS} SMs x 32 lanes x {clk:.0f} MHz (one conflict-free wavefront per SM per clock)"}
    # the committed full-set capture of the same kernel: shared-memory
    # wavefronts actually issued (bank conflicts included) per SM and clock,
    # and the busy share of the L1/shared data pipe
    if prof.get("smem_wavefronts_per_launch") and prof.get("smem_duration_ns"):
        wps = prof["smem_wavefronts_per_launch"] / (prof["smem_duration_ns"] * 1e-9)
        smem["ncu_wavefronts_per_sm_clock"] = round(wps / (SMS * clk * 1e6), 3)
    if prof.get("l1tex_throughput_pct") is not None:
        smem["ncu_l1tex_throughput_pct"] = prof["l1tex_throughput_pct"]
    return roof, smem


def e2e_measure(torch, run, flush, stream, steps):
    """Same workload through the C ABI from pinned host buffers: every step
    copies its inputs host->device, runs, and reads a result scalar back."""
    wl = run.wl
    seen, uniq, h2d = set(), [], 0
    for (Md, Ad, Bd, _c) in run.prods:
        for d in (Md, Ad, Bd):
            for t in (d.rowptr, d.colidx, d.values):
                if t is None or t.numel() == 0 or t.data_ptr() in seen:
                    continue
                seen.add(t.data_ptr())
                uniq.append((t.cpu().pin_memory(), t))
                h2d += t.numel() * t.element_size()
    out_h = torch.empty(1, dtype=torch.int64).pin_memory()

    def step():
        for hsrc, dst in uniq:
            dst.copy_(hsrc, non_blocking=True)
        _, scalar = run.step()
        out_h.copy_(scalar.view(-1)[:1].view(torch.int64), non_blocking=True)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    t = timed_steps(torch, step, steps, flush, stream)
    ms = statistics.mean(t)
    return {"value": round(2 * wl.kept / (ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": 8, "ms_per_step": round(ms, 4)}


def form_summary(wl, meas):
    ms = statistics.mean(meas["times"])
    d = {"ms_per_step": round(ms, 4), "masked_products": wl.kept,
         "masked_gflops": round(2 * wl.kept / (ms * 1e-3) / 1e9, 3), "autotune_s": meas.get("autotune_s")}
    if len(wl.mats) == 1:
        M, A, B, comp = wl.mats[0]
        vb_in, vb_out = VB[wl.semiring]
        d["hbm_min_gbs"] = round(q_min_bytes(M, A, B, wl.nnz_c, vb_in, vb_out, vb_b=0 if wl.pattern_b else None)
                                 / (ms * 1e-3) / 1e9, 2)
        d["push_products"] = push_products(A, B)
    if meas["per_phase"]:
        d["phase_ms"] = {n: round(statistics.mean(v), 4) for n, v in meas["per_phase"].items()}
    if meas.get("kind_rows"):
        d["kind_rows"] = meas["kind_rows"]
    for k in ("per_product_ms", "graph_ms", "fwd_ms", "bwd_ms", "bwd_unplanned_ms"):
        if k in meas:
            d[k] = round(meas[k], 3)
    if "per_product_ms" in meas:
        d["batched_speedup"] = round(meas["per_product_ms"] / ms, 2)
        if "graph_ms" in meas:
            d["graph_vs_per_product"] = round(meas["per_product_ms"] / meas["graph_ms"], 2)
    return d


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2111_09947_gb300 import _lib, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    # triangle counting on N ranks: one product split by rows (strong
    # scaling, the count all-reduced every step); other workloads: one seeded
    # instance per rank (weak scaling)
    sharded = world > 1 and args.workload == "tc"
    seed = synth.BASE_SEED if sharded or world == 1 else synth.BASE_SEED + 7919 * rank
    h = _lib.Handle(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    log(f"generating {args.workload} workload")
    t_gen = time.perf_counter()
    wl = build_workload(args.workload, args.scale, seed, args.batch_products)
    sharding = None
    if sharded:
        from paper_2111_09947_gb300 import shard
        L = wl.mats[0][0]
        b = shard.partition_rows(shard.push_work(L, L), world)
        r0, r1 = int(b[rank]), int(b[rank + 1])
        Lb = shard.row_block(L, r0, r1)
        wl.mats = [(Lb, Lb, L, False)]
        sharding = {"kind": "rows of L in contiguous blocks balanced by push work, L replicated as the right "
                            "operand, partial counts all-reduced every step", "ranks": world}
    gen_s = time.perf_counter() - t_gen
    log("measuring")
    if world > 1:
        dist.barrier()
    meas = measure(torch, _lib, synth, h, wl, dev, stream, flush, args.steps, args.warmup, local,
                   autotune=not args.no_autotune, allreduce=(lambda t: dist.all_reduce(t)) if sharded else None,
                   dist_sync=world > 1)
    total_ms = sum(meas["times"])
    flops = 2.0 * wl.kept
    if world > 1:
        from paper_2111_09947_gb300.shard import reduce_timing
        total_ms, flops = reduce_timing(total_ms, flops, device=dev)
    ms_per_step = total_ms / args.steps
    value = flops * args.steps / (total_ms * 1e-3) / 1e9
    summary = form_summary(wl, meas)
    log("roofline and end-to-end")
    rr = roofline_of(_lib, wl, meas)
    roof, roof_smem = rr if rr is not None else (None, None)
    if roof is None:
        pk = peaks()
        q = summary.get("hbm_min_gbs")
        roof = {"bound": "hbm", "kernel": "whole step", "achieved": q, "peak": pk["hbm_gbs"], "unit": "GB/s",
                "frac": round(q / pk["hbm_gbs"], 5) if q else None, "traffic": None, "peak_source": pk["source"]}
    e2e = e2e_measure(torch, meas["run"], flush, stream, max(3, args.steps // 2))
    cfg = dict(wl.config)
    line = {
        "metric": "masked GFLOP/s", "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": wl.dtype,
        "data": "synthetic (seeded R-MAT / Erdos-Renyi; the paper's SuiteSparse graphs are not used)",
        "config": cfg, "gpu_launches": int(meas["launches"]), "roofline": roof,
        "hbm_min_gbs": summary.get("hbm_min_gbs"), "phase_ms": summary.get("phase_ms"),
        "kind_rows": summary.get("kind_rows"),
        "clocks": meas["clocks"], "e2e": e2e, "gen_seconds": round(gen_s, 2), "autotune_s": meas["autotune_s"],
        "counts": {"masked_products": wl.kept, "nnz_C": wl.nnz_c, "seed_per_rank": world > 1 and not sharded},
    }
    if sharding is not None:
        # the all-reduced count of the last step, and the kept products of all blocks
        _, cnt = meas["run"].step()
        sharding["triangles"] = int(cnt.item())
        sharding["masked_products_all_ranks"] = int(flops / 2)
        line["sharding"] = sharding
    if roof_smem is not None:
        line["roofline_smem"] = roof_smem
    if "push_products" in summary:
        line["push_gflops"] = round(2 * summary["push_products"] / (ms_per_step * 1e-3) / 1e9, 2)
    for k in ("per_product_ms", "batched_speedup", "graph_ms", "graph_vs_per_product", "fwd_ms", "bwd_ms",
              "bwd_unplanned_ms"):
        if k in summary:
            line[k] = summary[k]

    if rank == 0 and world == 1 and not args.no_cpu_baseline and len(wl.mats) == 1:
        log("cpu baseline")
        M, A, B, comp = wl.mats[0]
        kfn = kept_fn_for(wl.semiring, M, A, B, comp)
        rate, secs, nrows, res = oracle_sample_rate(M, A, B, wl.semiring, comp, args.cpu_seconds, kept_fn=kfn)
        what = "the whole C" if nrows >= M.nrows else f"{nrows} uniformly drawn rows of the same C"
        line["cpu_baseline"] = {"value": round(rate, 4), "unit": "GFLOP/s", "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{what} ({'expand-sort-compress' if comp else 'merge per mask entry'}, "
                                          f"all cores), {secs:.1f} s"}
        if nrows >= M.nrows and wl.name != "autograd":
            # the flop numerator (counted on the GPU) against the oracle's count of the whole C
            o_kept = kfn(None, res)
            line["kept_check"] = {"gpu": wl.kept, "oracle": o_kept, "nnz_C_gpu": wl.nnz_c,
                                  "nnz_C_oracle": int(len(res["colidx"])),
                                  "equal": bool(o_kept == wl.kept and len(res["colidx"]) == wl.nnz_c)}

    if rank == 0 and not args.no_forms:
        forms = {}
        if len(wl.mats) == 1 and not wl.mats[0][3] and wl.name != "autograd":
            log("form: two_phase")
            forms["two_phase"] = two_phase_form(torch, _lib, meas["run"], flush, stream, wl, ms_per_step)
        for name in WORKLOADS:
            if name == args.workload:
                continue
            log(f"form: {name}")
            fw = build_workload(name, None, synth.BASE_SEED)
            fm = measure(torch, _lib, synth, h, fw, dev, stream, flush, 5, 2, None, autotune=not args.no_autotune)
            forms[name] = dict(config=fw.config["workload"], **form_summary(fw, fm))
            if name in ("er", "autograd") and world == 1:
                # the CPU oracle on one core and on all (the forward product for autograd)
                try:
                    forms[name]["cpu_oracle"] = oracle_threads_form(fw)
                except Exception as e:   # a side figure: never lose the line for it
                    forms[name]["cpu_oracle"] = {"error": repr(e)[:200]}
            del fm
            torch.cuda.empty_cache()
        log("form: bc")
        forms["bc"] = bc_form(torch, _lib, synth, dev, stream, flush, 3, 2)
        torch.cuda.empty_cache()
        log("form: ktruss")
        forms["ktruss"] = ktruss_form(torch, _lib, synth, dev, stream, flush, 2, 1, autotune=not args.no_autotune)
        torch.cuda.empty_cache()
        line["forms"] = forms

    h.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def two_phase_form(torch, _lib, run, flush, stream, wl, ms_one):
    """A workload of one plain product in the two-phase form (Sec. 6) on the
    same (tuned) handle: a symbolic pass counts, C is allocated exactly, a
    numeric pass writes in place.  Output memory: one phase holds a temporary
    and C, both of the mask's size; two phases hold C alone, of its own size."""
    h = run.h
    h.set_option(_lib.OPT_PHASES, 2)
    try:
        for _ in range(2):
            run.step()
        torch.cuda.synchronize()
        t = statistics.median(timed_steps(torch, run.step, 5, flush, stream))
    finally:
        h.set_option(_lib.OPT_PHASES, 1)
    M = wl.mats[0][0]
    ent = 4 + (4 if wl.semiring == "plus_times_f32" else 8)   # column index + value
    return {"config": "the main workload in the two-phase form: symbolic count, exact allocation, numeric pass "
                      "in place (same tuned policy; the (row, tile) grid kinds are not used)",
            "ms_per_step": round(t, 4), "one_phase_ms": round(ms_one, 4),
            "masked_gflops_2p": round(2 * wl.kept / (t * 1e-3) / 1e9, 3),
            "output_bytes_one_phase": 2 * M.nnz * ent, "output_bytes_two_phase": wl.nnz_c * ent}


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle, as it stands, timed on the same workload and config as
    the GPU arm.  Each step is one oracle call: the whole C when the fitted
    cost says it fits the per-step budget (so the call's one transpose of B is
    amortised as in the cpu_baseline leg), else a uniform row sample sized to
    the budget; the budget keeps the whole run within a few minutes."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    from paper_2111_09947_gb300 import synth
    name = args.workload if args.workload in ("tc", "er", "bfs", "autograd") else "tc"
    wl = build_workload(name, args.scale, synth.BASE_SEED, args.batch_products)
    M, A, B, comp = wl.mats[0]
    per_step = max(0.5, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    nrows, fixed, per_row = oracle_plan(M, A, B, wl.semiring, comp, per_step, rng_seed=11)
    kfn = kept_fn_for(wl.semiring, M, A, B, comp)
    rng = np.random.default_rng(12)
    times, flops = [], []
    for s in range(args.warmup + args.steps):
        dt, fl, nr, _ = oracle_timed_call(M, A, B, wl.semiring, comp, nrows, rng, kfn)
        if s >= args.warmup:
            times.append(dt)
            flops.append(fl)
    value = sum(flops) / sum(times) / 1e9
    what = "the whole C per step" if nrows is None else f"{nrows} uniformly drawn rows per step (of {M.nrows})"
    sample = f"{what}, oracle " + ("expand-sort-compress" if comp else "merge per mask entry") + \
             f", all {cores} cores (fitted fixed cost per call {fixed:.2f} s)"
    line = {"impl": "reference", "metric": "masked GFLOP/s", "value": round(value, 4), "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(times) / len(times), 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic (seeded R-MAT / Erdos-Renyi; the paper's "
            "SuiteSparse graphs are not used)",
            "config": wl.config,
            "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """Sweeps of the policy (one JSON line per point, then a summary line).
    er: plain fp32 products of independent Erdos-Renyi A, B, M (n x n) over
    n, the input degree and the mask degree (the density study of Sec. 8.1),
    each timed with every accumulator family forced and with AUTO; AUTO's
    time over the best forced one says how well the binning picks.  rmat:
    triangle counting over R-MAT scales (the scaling study of Sec. 8.2)."""
    import torch
    from paper_2111_09947_gb300 import _lib, synth
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    h = _lib.Handle(dev)
    rows = []
    if args.sweep == "er":
        for lg in range(12, args.sweep_max_log2 + 1, 2):
            n = 1 << lg
            for din in (4, 16, 64):
                for dm in (1, 16, 256):
                    if n * max(din, dm) > (1 << 28):
                        continue
                    p = synth.random_problem(n, n, n, float(din), float(din), float(dm), synth.BASE_SEED + lg, "f32")
                    d = {k: _lib.DeviceCsr.from_host(p[k], device=dev) for k in ("M", "A", "B")}
                    d["M"].values = None
                    t = {}
                    # every family forced (one phase), AUTO, and AUTO in two phases (Sec. 6); the
                    # dense MSA forced on every row is left out from n = 2^22 (at 2^20 it already
                    # takes 0.2-0.6 s a call: every row clears and gathers n columns)
                    fams = ["auto", "msa", "hash", "mca", "dot", "heap", "heapdot", "auto_2p"]
                    if lg >= 22:
                        fams.remove("msa")
                    for force in fams:
                        h.force("auto" if force == "auto_2p" else force)
                        h.set_option(_lib.OPT_PHASES, 2 if force == "auto_2p" else 1)
                        fn = lambda: _lib.msgemm_run(h, d["M"], d["A"], d["B"], "plus_times_f32")  # noqa: E731
                        for _ in range(2):
                            fn()
                        torch.cuda.synchronize()
                        t[force] = round(statistics.median(timed_steps(torch, fn, 5, flush, stream)), 4)
                    h.force("auto")
                    h.set_option(_lib.OPT_PHASES, 1)
                    # the autotuner on this product (fresh handle, no cache), then timed
                    ht = _lib.Handle(dev)
                    _lib.msgemm_autotune(ht, [d["M"]], [d["A"]], [d["B"]], "plus_times_f32")
                    fn = lambda: _lib.msgemm_run(ht, d["M"], d["A"], d["B"], "plus_times_f32")  # noqa: E731
                    for _ in range(2):
                        fn()
                    torch.cuda.synchronize()
                    t["tuned"] = round(statistics.median(timed_steps(torch, fn, 5, flush, stream)), 4)
                    ht.close()
                    forced = {k: v for k, v in t.items() if k not in ("auto", "auto_2p", "tuned")}
                    best = min(forced.values())
                    row = {"n": n, "d_in": din, "d_mask": dm, "ms": t,
                           "best": min((v, k) for k, v in forced.items())[1],
                           "auto_over_best": round(t["auto"] / best, 3),
                           "tuned_over_best": round(t["tuned"] / best, 3),
                           "two_phase_over_one": round(t["auto_2p"] / t["auto"], 3)}
                    rows.append(row)
                    print(json.dumps(row), flush=True)
                    del d
        r = np.array([x["auto_over_best"] for x in rows])
        r2 = np.array([x["two_phase_over_one"] for x in rows])
        rt = np.array([x["tuned_over_best"] for x in rows])
        wins = {}
        for x in rows:
            wins[x["best"]] = wins.get(x["best"], 0) + 1
        summary = {"sweep": "er", "points": len(rows), "auto_over_best_median": round(float(np.median(r)), 3),
                   "auto_over_best_max": round(float(r.max()), 3),
                   "auto_within_10pct": int((r <= 1.10).sum()), "best_family_counts": wins,
                   "tuned_over_best_median": round(float(np.median(rt)), 3),
                   "tuned_over_best_max": round(float(rt.max()), 3),
                   "tuned_within_10pct": int((rt <= 1.10).sum()),
                   "two_phase_over_one_median": round(float(np.median(r2)), 3)}
        print(json.dumps(summary), flush=True)
    else:
        for scale in range(8, 21, 2):
            wl = build_workload("tc", scale, synth.BASE_SEED)
            meas = measure(torch, _lib, synth, h, wl, dev, stream, flush, 5, 3, None, autotune=not args.no_autotune)
            ms = statistics.mean(meas["times"])
            row = {"scale": scale, "nnz_L": wl.config["nnz_L"], "masked_products": wl.kept, "ms": round(ms, 4),
                   "masked_gflops": round(2 * wl.kept / (ms * 1e-3) / 1e9, 3)}
            row.update(two_phase_form(torch, _lib, meas["run"], flush, stream, wl, ms))
            row.pop("config")
            rows.append(row)
            print(json.dumps(row), flush=True)
        summary = {"sweep": "rmat", "points": len(rows)}
        print(json.dumps(summary), flush=True)
    h.close()
    if args.sweep_out:
        doc = {"sweep": args.sweep, "source_sha": source_hash(), "device": torch.cuda.get_device_name(dev),
               "when": time.strftime("%Y-%m-%dT%H:%M:%SZ", time.gmtime()),
               "command": "python bench.py " + " ".join(sys.argv[1:]),
               "timing": "median of 5 CUDA-event-timed calls after 2 untimed, L2 flushed before each (ms)",
               "summary": summary, "rows": rows}
        with open(args.sweep_out, "w") as f:
            json.dump(doc, f, indent=1)


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.sweep:
        run_sweep(args)
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
    run_ours(args)


if __name__ == "__main__":
    main()
