#!/usr/bin/env python
"""Masked SpGEMM benchmark on GB300.

Default workload: triangle counting on an R-MAT graph of scale 20 (edge
factor 16, Graph500 quadrant probabilities), symmetrised, loops and
duplicates removed, degree-relabelled; C = L .* (L L) on plus-pair int64 and
the count sum(C) (Sec. 8.2).  One step = the whole path on resident inputs:
binning, accumulators, compaction and the count reduction.  The metric is
masked GFLOP/s = 2 x (products kept by the mask) / time.

Also reported (key "forms"): the plain fp32 product on Erdos-Renyi n = 4096,
the complemented BFS step of multi-source betweenness centrality (512
sources, scale 20), 256 batched products against per-product calls, and the
forward + backward pass of the differentiable form (R-MAT scale 18).

--impl reference times the CPU oracle (the plain C program under oracle/)
on bounded row samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
_T0 = time.perf_counter()


def log(msg: str) -> None:
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f}s] {msg}", file=sys.stderr, flush=True)
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--scale", type=int, default=20, help="R-MAT scale of the triangle-count workload")
    ap.add_argument("--no-forms", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    return ap.parse_args()


def peaks():
    path = os.path.join(REPO, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": PEAKS_FALLBACK["hbm_gbs"], "source": "fallback"}


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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
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
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- workload math
def masked_products_from_pp(res_pp) -> int:
    """Products kept by the mask = sum of the plus-pair result."""
    v = res_pp.values[: res_pp.nnz()]
    return int(v.sum().item())


def push_products(A, B) -> int:
    bl = np.diff(B.rowptr).astype(np.int64)
    return int(bl[A.colidx].sum())


def q_min_bytes(M, A, B, nnz_c, vb_in, vb_out, complement=False) -> int:
    """Compulsory bytes (read A, B, M once, write C once)."""
    q = 4 * (A.nrows + 1) + A.nnz * (4 + vb_in)
    q += 4 * (B.nrows + 1) + B.nnz * (4 + vb_in)
    q += 4 * (M.nrows + 1) + 4 * M.nnz
    q += 4 * (M.nrows + 1) + nnz_c * (4 + vb_out)
    return int(q)


def kernel_bytes(kinds, kind_id, M, A, B, C_rp, vb_in, vb_out) -> int:
    """Compulsory bytes of the rows one accumulator kernel processes: their
    rows of A and M, the distinct rows of B they touch, their output."""
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
    q += int((8 + bl[ks] * (4 + vb_in)).sum())
    return q


def source_hash() -> str:
    h = hashlib.sha1()
    cdir = os.path.join(REPO, "paper_2111_09947_gb300", "csrc")
    for name in sorted(os.listdir(cdir)):
        if name.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(cdir, name), "rb") as f:
                h.update(name.encode())
                h.update(f.read())
    return h.hexdigest()[:12]


def traffic_for(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources."""
    path = os.path.join(REPO, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    e = d.get(workload, {}).get(kernel)
    if not e or e.get("source_sha") != source_hash():
        return None
    return e.get("dram_bytes_per_launch")


# ----------------------------------------------------------------- timing
def timed_steps(torch, step, steps, flush_buf, stream):
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
    return times


def oracle_sample_rate(M, A, B, semiring, complement, target_s, rng_seed=7, kept_fn=None):
    """Times the CPU oracle on random row samples until about target_s of
    work; returns (masked GFLOP/s, seconds, rows, sample description)."""
    from oracle import oracle as O
    rng = np.random.default_rng(rng_seed)
    m = M.nrows
    frac = 0.002
    method = O.ESC if complement else O.MERGE
    total_t, total_f, total_rows = 0.0, 0, 0
    while True:
        k = max(1, min(m, int(m * frac)))
        rows = np.sort(rng.choice(m, size=k, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        res = O.masked_spgemm(M, A, B, semiring, complement=complement, method=method, rows=rows)
        dt = time.perf_counter() - t0
        kept = kept_fn(rows, res)
        total_t += dt
        total_f += 2 * kept
        total_rows += k
        if total_t >= target_s or k == m:
            total_rows = min(total_rows, m) if k == m else total_rows
            break
        remaining = target_s - total_t
        frac = min(1.0, frac * max(2.0, remaining / max(dt, 1e-3)))
    return total_f / total_t / 1e9, total_t, total_rows


# ----------------------------------------------------------------- main arm
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
    seed = synth.BASE_SEED + 7919 * rank      # weak scaling: one instance per rank

    # ---- workload (host), then resident on the device
    log('generating triangle-count workload')
    t_gen = time.perf_counter()
    tc = synth.triangle_counting(scale=args.scale, ef=16, seed=seed)
    L = tc["M"]
    gen_s = time.perf_counter() - t_gen
    Ld = _lib.DeviceCsr.from_host(L, device=dev)
    Ld.values = None
    h = _lib.Handle(dev)
    h.set_option(_lib.OPT_PROFILE, 1)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        r = _lib.msgemm_run(h, Ld, Ld, Ld, "plus_pair_i64")
        s = _lib.msgemm_reduce_sum(h, r, "plus_pair_i64")
        return r, s

    log('warm-up')
    for _ in range(args.warmup):
        r, s = step()
    torch.cuda.synchronize()
    triangles = int(s.item())
    nnz_c = r.nnz()
    kept = triangles                       # plus-pair: each kept product counts 1
    masked_flops = 2 * kept
    kinds = h.row_kinds(L.nrows)
    C_rp = r.rowptr.cpu().numpy()

    # ---- timed region
    log('timed steps')
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    l0 = _lib.load().msgemm_kernel_launches()
    per_kernel = {}
    times = []
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        r, s = step()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
        for name, ms in h.profile():
            per_kernel.setdefault(name, []).append(ms)
    launches = _lib.load().msgemm_kernel_launches() - l0
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_ms = sum(times)
    if world > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        f = torch.tensor([masked_flops], dtype=torch.float64, device=dev)
        dist.all_reduce(f, op=dist.ReduceOp.SUM)
        flops_all = float(f.item())
    else:
        flops_all = float(masked_flops)
    ms_per_step = total_ms / args.steps
    value = flops_all * args.steps / (total_ms * 1e-3) / 1e9
    assert int(s.item()) == triangles

    # ---- roofline of the dominant accumulator kernel
    pk = peaks()
    kind_ids = {n: i for i, n in enumerate(_lib.KIND_NAMES)}
    cand = {n: statistics.mean(v) for n, v in per_kernel.items() if n in kind_ids and n != "empty"}
    dom = max(cand, key=cand.get)
    dom_ms = cand[dom]
    kb = kernel_bytes(kinds, kind_ids[dom], L, L, L, C_rp, 0, 8)
    achieved = kb / (dom_ms * 1e-3) / 1e9
    traffic = traffic_for(dom, f"tc_scale{args.scale}")
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 2), "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": round(achieved / pk["hbm_gbs"], 5), "traffic": traffic,
                "peak_source": pk["source"] + " (MEASURED_PEAKS.json hbm_gbs)" if pk["source"] == "measured"
                else "fallback 6.8 TB/s", "algorithmic_bytes_per_launch": kb, "kernel_ms": round(dom_ms, 4)}
    qmin = q_min_bytes(L, L, L, nnz_c, 0, 8)
    pushp = push_products(L, L)
    phase_ms = {n: round(statistics.mean(v), 4) for n, v in per_kernel.items()}

    # ---- end to end through the C ABI from pinned host buffers
    log('end-to-end steps')
    rp_h = torch.from_numpy(L.rowptr).pin_memory()
    ci_h = torch.from_numpy(L.colidx).pin_memory()
    rp_d = torch.empty_like(rp_h, device=dev)
    ci_d = torch.empty_like(ci_h, device=dev)
    out_h = torch.empty(1, dtype=torch.int64).pin_memory()
    Le = _lib.DeviceCsr(L.nrows, L.ncols, rp_d, ci_d, None)

    def e2e_step():
        rp_d.copy_(rp_h, non_blocking=True)
        ci_d.copy_(ci_h, non_blocking=True)
        rr = _lib.msgemm_run(h, Le, Le, Le, "plus_pair_i64")
        ss = _lib.msgemm_reduce_sum(h, rr, "plus_pair_i64")
        out_h.copy_(ss, non_blocking=True)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    et = timed_steps(torch, e2e_step, max(3, args.steps // 2), flush, stream)
    assert int(out_h.item()) == triangles
    e2e_ms = statistics.mean(et)
    h2d = rp_h.numel() * 4 + ci_h.numel() * 4

    line = {
        "metric": "masked GFLOP/s", "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (seeded R-MAT; the paper's SuiteSparse graphs are not used)",
        "config": {"workload": f"triangle counting: R-MAT scale {args.scale}, edge factor 16, (a,b,c)=(0.57,0.19,0.19), "
                               "symmetrised, loops/duplicates removed, degree-relabelled, L strict lower; "
                               "C = L .* (L L) plus-pair int64 + count",
                   "n": L.nrows, "nnz_L": L.nnz, "triangles": triangles, "nnz_C": nnz_c,
                   "masked_products": kept, "push_products": pushp,
                   "l2": "flushed before every timed step (256 MiB write)", "seed_per_rank": True},
        "gpu_launches": int(launches),
        "roofline": roofline,
        "hbm_min_gbs": round(qmin / (ms_per_step * 1e-3) / 1e9, 2),
        "push_effective_gbs": round(pushp * 4 / (ms_per_step * 1e-3) / 1e9, 2),
        "push_gflops": round(2 * pushp / (ms_per_step * 1e-3) / 1e9, 2),
        "phase_ms": phase_ms,
        "clocks": clk,
        "e2e": {"value": round(2 * kept / (e2e_ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 8, "ms_per_step": round(e2e_ms, 4)},
        "gen_seconds": round(gen_s, 2),
    }

    # ---- CPU baseline: the oracle on a bounded row sample (rank 0, N = 1)
    log('cpu baseline')
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rp_pp = C_rp
        cvals = r.values[:nnz_c].cpu().numpy()

        def kept_fn(rows, res):
            return int(res["values"].sum())
        cores = os.cpu_count()
        rate, secs, nrows = oracle_sample_rate(L, L, L, "plus_pair_i64", False, args.cpu_seconds, kept_fn=kept_fn)
        what = ("the whole C" if nrows >= L.nrows else f"{nrows} uniformly drawn rows of the same C")
        line["cpu_baseline"] = {"value": round(rate, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                                "sample": f"{what} (oracle merge per mask entry, all cores), {secs:.1f} s"}
        del rp_pp, cvals

    if rank == 0 and not args.no_forms:
        line["forms"] = other_forms(torch, h, dev, stream, flush, synth, _lib)

    h.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def other_forms(torch, h, dev, stream, flush, synth, _lib):
    forms = {}
    h.set_option(_lib.OPT_PROFILE, 0)
    K = 10

    # plain fp32, Erdos-Renyi n = 4096, 8 per row
    log('form: er plain fp32')
    p = synth.er_plain_f32()
    d = {k: _lib.DeviceCsr.from_host(v, device=dev) for k, v in p.items()}
    d["M"].values = None
    pp = {k: _lib.DeviceCsr(v.nrows, v.ncols, v.rowptr, v.colidx, None) for k, v in d.items()}
    kept = masked_products_from_pp(_lib.msgemm_run(h, pp["M"], pp["A"], pp["B"], "plus_pair_i64"))
    step = lambda: _lib.msgemm_run(h, d["M"], d["A"], d["B"], "plus_times_f32")  # noqa: E731
    for _ in range(5):
        step()
    t = timed_steps(torch, step, K, flush, stream)
    ms = statistics.median(t)
    forms["er_plain_f32"] = {"n": 4096, "avg_per_row": 8, "us_per_call": round(ms * 1e3, 2),
                             "masked_products": kept, "masked_gflops": round(2 * kept / (ms * 1e-3) / 1e9, 4)}

    # complemented BFS step, 512 sources
    log('form: bfs step')
    b = synth.bfs_step(scale=20, ef=16, nsrc=512)
    db = {k: _lib.DeviceCsr.from_host(v, device=dev) for k, v in (("M", b["M"]), ("A", b["A"]), ("B", b["B"]))}
    db["M"].values = None
    dpp = {k: _lib.DeviceCsr(v.nrows, v.ncols, v.rowptr, v.colidx, None) for k, v in db.items()}
    rpp = _lib.msgemm_run(h, dpp["M"], dpp["A"], dpp["B"], "plus_pair_i64", complement=True)
    kept = masked_products_from_pp(rpp)
    nnz_c = rpp.nnz()
    del rpp
    step = lambda: _lib.msgemm_run(h, db["M"], db["A"], db["B"], "plus_times_i64", complement=True)  # noqa: E731
    for _ in range(2):
        step()
    torch.cuda.synchronize()
    t = timed_steps(torch, step, 5, flush, stream)
    ms = statistics.median(t)
    q = q_min_bytes(b["M"], b["A"], b["B"], nnz_c, 8, 8, True)
    forms["bfs_complement_i64"] = {"sources": int(b["A"].nrows), "ms_per_step": round(ms, 3),
                                   "masked_products": kept, "nnz_C": nnz_c,
                                   "masked_gflops": round(2 * kept / (ms * 1e-3) / 1e9, 3),
                                   "hbm_min_gbs": round(q / (ms * 1e-3) / 1e9, 2),
                                   "push_products": push_products(b["A"], b["B"])}
    del db, dpp, b
    torch.cuda.empty_cache()

    # batched: 256 products in one call vs 256 calls
    log('form: batched')
    ps = synth.batched_problems(nprod=256)
    devs = []
    for q in ps:
        x = {k: _lib.DeviceCsr.from_host(v, device=dev) for k, v in (("M", q["M"]), ("A", q["A"]), ("B", q["B"]))}
        x["M"].values = None
        devs.append(x)
    Ms, As, Bs = [x["M"] for x in devs], [x["A"] for x in devs], [x["B"] for x in devs]

    def per_product():
        for x in devs:
            _lib.msgemm_run(h, x["M"], x["A"], x["B"], "plus_times_f32")

    def batched():
        _lib.msgemm_run_batched(h, Ms, As, Bs, "plus_times_f32")

    for _ in range(2):
        per_product()
        batched()
    tp = statistics.median(timed_steps(torch, per_product, 3, flush, stream))
    tb = statistics.median(timed_steps(torch, batched, 5, flush, stream))
    forms["batched_256_f32"] = {"products": len(ps), "per_product_ms": round(tp, 3), "batched_ms": round(tb, 3),
                                "speedup": round(tp / tb, 2)}
    del devs, Ms, As, Bs
    torch.cuda.empty_cache()

    # differentiable form: forward, backward, forward + backward
    log('form: autograd')
    a = synth.autograd_problem(scale=18, ef=16)
    da = {k: _lib.DeviceCsr.from_host(v, device=dev) for k, v in a.items()}
    da["M"].values = None
    res = _lib.msgemm_run(h, da["M"], da["A"], da["B"], "plus_times_f32").trimmed()
    G = _lib.DeviceCsr(res.nrows, res.ncols, res.rowptr, res.colidx,
                       torch.from_numpy(synth.upstream_grad(res.nnz)).to(dev))
    fwd = lambda: _lib.msgemm_run(h, da["M"], da["A"], da["B"], "plus_times_f32")  # noqa: E731
    bwd = lambda: _lib.msgemm_backward(h, da["A"], da["B"], G)  # noqa: E731

    def fwdbwd():
        fwd()
        bwd()
    for _ in range(2):
        fwdbwd()
    tf = statistics.median(timed_steps(torch, fwd, 5, flush, stream))
    tbw = statistics.median(timed_steps(torch, bwd, 5, flush, stream))
    tfb = statistics.median(timed_steps(torch, fwdbwd, 5, flush, stream))
    forms["autograd_f32_scale18"] = {"nnz_A": int(a["A"].nnz), "fwd_ms": round(tf, 3), "bwd_ms": round(tbw, 3),
                                     "fwd_bwd_ms": round(tfb, 3), "bwd_over_fwd": round(tbw / tf, 2)}
    return forms


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle, as it stands, on bounded row samples of the same workload."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = os.cpu_count()
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    from oracle import oracle as O
    from paper_2111_09947_gb300 import synth
    tc = synth.triangle_counting(scale=args.scale, ef=16, seed=synth.BASE_SEED)
    L = tc["M"]
    rng = np.random.default_rng(11)
    # size one step's sample to ~ a few seconds
    frac = 0.002
    t0 = time.perf_counter()
    rows = np.sort(rng.choice(L.nrows, size=max(1, int(L.nrows * frac)), replace=False)).astype(np.int32)
    O.masked_spgemm(L, L, L, "plus_pair_i64", rows=rows)
    dt = time.perf_counter() - t0
    frac = min(1.0, frac * max(1.0, 4.0 / max(dt, 1e-3)))
    nrow = max(1, int(L.nrows * frac))
    times, flops = [], []
    for s in range(args.warmup + args.steps):
        rows = np.sort(rng.choice(L.nrows, size=nrow, replace=False)).astype(np.int32)
        t0 = time.perf_counter()
        res = O.masked_spgemm(L, L, L, "plus_pair_i64", rows=rows)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            flops.append(2 * int(res["values"].sum()))
    value = sum(flops) / sum(times) / 1e9
    sample = f"{nrow} uniformly drawn rows per step (of {L.nrows}), oracle merge per mask entry"
    line = {"impl": "reference", "metric": "masked GFLOP/s", "value": round(value, 4), "unit": "GFLOP/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * sum(times) / len(times), 2), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic (seeded R-MAT)",
            "config": {"workload": f"triangle counting: R-MAT scale {args.scale}, edge factor 16, relabelled, "
                                   "C = L .* (L L) plus-pair int64", "n": L.nrows, "nnz_L": L.nnz},
            "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count()))
    run_ours(args)


if __name__ == "__main__":
    main()
