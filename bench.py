#!/usr/bin/env python
"""Benchmark of the Ozaki-scheme multi-component product on GB300.

Workload (the headline one): double-double C = A B with m = n = k = 4096,
operands of Eq. 1 with exponent spread phi = 1 (synthetic, seeded), the
slice count chosen automatically for the 2^-100 target; the digit form is
selectable (default: the automatic form, balanced radix-32 e4m3 digits on
tcgen05).  A step is the whole hot path:
exponent reduce + digit split (K1, K2) and the fused slice products with
exact accumulation (K3).  Metric: effective GFLOP/s = 2 m n k / time.

Printed: one JSON line (rank 0).  Besides the contract keys it carries
  roofline      -- the slice-product kernel: algorithmic tensor FLOPs
                   (pairs * 2 m n k) / its CUDA-event time, against the
                   e4m3 dense peak derived from the measured bf16 peak;
  splitter      -- algorithmic HBM bytes of K1 + K2 (operands read once,
                   digits written once) / their time, against measured HBM;
  e2e           -- the same metric through the C ABI with host buffers
                   (pinned H2D of A, B and D2H of C inside the timed region);
  cpu_baseline  -- the oracle (exact product rounded to 512 bits) on the
                   host cores, on a bounded block of the same product, with
                   the GPU result's error against it;
  variants      -- single timed passes of the other forms/precisions
                   (DD and QD; balanced and 4-bit e4m3 / int8 / binary64
                   digits) at 4096^3;
  multiprecision_2048 -- 8 and 16 binary64 components (424 / 848 bits)
                   at 2048^3, balanced and 4-bit e4m3 digits on tcgen05;
  lu_4096       -- the LU application: DD n = 4096 and TD n = 2048 LU
                   without pivoting on Ozaki products, and the solve;
  literal_vs_truncating_1024 -- Algorithm 1 as printed against the
                   truncating binary64-digit form, error and time per D.

--impl reference times the oracle itself (the CPU reference of this repo)
on a bounded block per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 2 ** 20


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.dev), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons, pw = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
                pw.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(pw) if pw else None}


# ---------------------------------------------------------------------------
# ranks: one replica per GPU, each with its own problem (no data-path
# collective); the time of the job is the slowest rank's
# ---------------------------------------------------------------------------
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _rank_seed(rank: int) -> int:
    """Seed of a rank's operands (rank 0: the single-GPU workload)."""
    return 1000 * rank


def _max_over_ranks(x: float, device) -> float:
    """Largest x over the ranks of the default process group."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _host_operands(prec, m, n, k, phi, seed):
    from ozmp_inputs import gen_problem
    return gen_problem(prec, m, n, k, phi=phi, seed=seed)


def target_bits(prec) -> int:
    """Normwise target of a precision: 2^-(50 q) for q binary64 components, 2^-66 for TS."""
    if prec == "ts":
        return 66
    q = {"dd": 2, "td": 3, "qd": 4}.get(prec)
    if q is None:
        q = int(str(prec)[1:])      # "q5" .. "q16"
    return 50 * q


def sample_idx(m, n, b):
    """b evenly spaced rows and columns (first and last included)."""
    import numpy as np
    rows = sorted(set(np.linspace(0, m - 1, min(m, b)).astype(int).tolist()))
    cols = sorted(set(np.linspace(0, n - 1, min(n, b)).astype(int).tolist()))
    return rows, cols


def sampled_error(torch, C, A, B, rows, cols, prec, ex=None):
    """Normwise and largest elementwise relative error of the device result C
    on a block of entries (full k), against the exact product rounded to 512
    bits (the oracle); only that block is read back."""
    from oracle import _clib
    from oracle import exact as X
    if ex is None:
        ex = _clib.exact_block(A, B, rows, cols)
    ri = torch.tensor(rows, device=C[0].device)
    ci = torch.tensor(cols, device=C[0].device)
    blk = [c.index_select(0, ri).index_select(1, ci).cpu().numpy() for c in C]
    chat = [[[float(b[a, c]) for b in blk] for c in range(len(cols))] for a in range(len(rows))]
    em = X.error_metrics(chat, ex)
    out = {"err_nw": em["err_nw"], "err_max_rel": em["err_max"], "err_block": f"{len(rows)}x{len(cols)}, full k",
           "target": 2.0 ** -target_bits(prec)}
    if target_bits(prec) > 480:
        # the oracle's 512-bit rounding limits what can be resolved
        out["resolution"] = 2.0 ** -510
    return out


def run_variant(oz, torch, prec, form, n, phi, steps, warmup, nslices=0, err=True):
    """Device-resident timing of one (precision, form), with the error of the
    result on a 64 x 64 block against the oracle: returns a dict."""
    import numpy as np
    A, B = _host_operands(prec, n, n, n, phi, 0)
    Ad = [oz.colmajor(a) for a in A]
    Bd = [oz.colmajor(b) for b in B]
    dt = torch.float32 if prec == "ts" else torch.float64
    q = len(A)
    C = [torch.empty((n, n), dtype=dt, device="cuda").T for _ in range(q)]
    p = oz.Plan(prec, n, n, n, form, nslices)
    for _ in range(warmup):
        p.split(Ad, Bd)
        p.multiply(C)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for s in range(steps):
        ev[s][0].record()
        p.split(Ad, Bd)
        ev[s][1].record()
        p.multiply(C)
        ev[s][2].record()
    torch.cuda.synchronize()
    split_ms = [e[0].elapsed_time(e[1]) for e in ev]
    gemm_ms = [e[1].elapsed_time(e[2]) for e in ev]
    tot = ev[0][0].elapsed_time(ev[-1][2]) / steps
    st = p.status()
    i = p.info
    flops = 2.0 * n * n * n
    out = {"prec": prec, "form": oz.Form(i.form).name.lower(), "beta": i.beta, "nslices": i.nslices,
           "pairs": i.npairs, "ms_per_step": tot, "gflops": flops / (tot * 1e-3) / 1e9,
           "split_ms": sum(split_ms) / steps, "gemm_ms": sum(gemm_ms) / steps,
           "slice_tflops": i.npairs * flops / (sum(gemm_ms) / steps * 1e-3) / 1e12, "status": st.name}
    if err:
        rows, cols = sample_idx(n, n, 64)
        out.update(sampled_error(torch, C, A, B, rows, cols, prec))
    del p, Ad, Bd, C
    torch.cuda.empty_cache()
    return out


def literal_variant(oz, torch, n=1024):
    """Accuracy and time against the division count D: Algorithm 1 as printed
    (binary64 round-to-nearest slices, binary64 tensor-core products) and the
    truncating binary64-digit form with s = D, both against the exact
    product rounded to 512 bits (the oracle) on a 64 x 64 block (full k); DD,
    n^3, phi = 1."""
    from oracle import _clib
    A, B = _host_operands("dd", n, n, n, 1.0, 0)
    Ad = [oz.colmajor(a) for a in A]
    Bd = [oz.colmajor(b) for b in B]
    rows, cols = sample_idx(n, n, 64)
    ex = _clib.exact_block(A, B, rows, cols)
    out = []
    for D in (3, 4, 5, 6, 7, 8):
        row = {"D": D}
        try:
            C = [torch.empty((n, n), dtype=torch.float64, device="cuda").T for _ in range(2)]
            oz.ozmp_gemm_literal(Ad, Bd, C, D)
            t0 = time.time()
            st = oz.ozmp_gemm_literal(Ad, Bd, C, D)
            row["literal_ms"] = (time.time() - t0) * 1e3
            row["literal_err"] = sampled_error(torch, C, A, B, rows, cols, "dd", ex)["err_nw"]
            row["literal_status"] = st.name
            p = oz.Plan("dd", n, n, n, "fp64", D)
            C2 = [torch.empty((n, n), dtype=torch.float64, device="cuda").T for _ in range(2)]
            p.execute(Ad, Bd, C2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            p.execute(Ad, Bd, C2)
            e1.record()
            torch.cuda.synchronize()
            row["truncating_fp64_ms"] = e0.elapsed_time(e1)
            row["truncating_fp64_err"] = sampled_error(torch, C2, A, B, rows, cols, "dd", ex)["err_nw"]
            row["truncating_status"] = p.status().name
            del p
        except Exception as ex_:
            row["error"] = repr(ex_)[:200]
        out.append(row)
    return {"vs": "exact product rounded to 512 bits, 64 x 64 block, full k", "rows": out}


def lu_variant(oz, torch):
    """The LU application (Sec. 4.6): in-place LU without pivoting of a random
    n x n matrix (a_ij = U[0,1), the paper's test matrix) in DD and TD, and
    the solve of A x = b with b_i = 1 / i; time of the second call (the first
    creates the product plans), (2/3) n^3 / time."""
    import numpy as np
    out = []
    for q, n in ((2, 4096), (3, 2048)):
        try:
            rng = np.random.default_rng(0)
            A = rng.random((n, n))
            comps = [np.asfortranarray(A)] + [np.zeros((n, n), order="F") for _ in range(q - 1)]
            Ad = [oz.colmajor(c) for c in comps]
            W = [a.clone() for a in Ad]
            oz.ozmp_lu(W)
            W = [a.clone() for a in Ad]
            torch.cuda.synchronize()
            t0 = time.time()
            st = oz.ozmp_lu(W)
            t_lu = time.time() - t0
            b = [oz.colmajor(np.asfortranarray(1.0 / np.arange(1, n + 1, dtype=np.float64)[:, None]))] + \
                [torch.zeros((1, n), dtype=torch.float64, device="cuda").T for _ in range(q - 1)]
            t0 = time.time()
            st2 = oz.ozmp_lu_solve(W, b)
            t_s = time.time() - t0
            out.append({"prec": {2: "dd", 3: "td"}[q], "n": n, "lu_s": t_lu, "gflops": 2 * n ** 3 / 3 / t_lu / 1e9,
                        "solve_s": t_s, "status": st.name, "solve_status": st2.name})
            del Ad, W, b
            torch.cuda.empty_cache()
        except Exception as ex:
            out.append({"q": q, "n": n, "error": repr(ex)[:200]})
    return out


def td_qd_1024_variant(oz, torch):
    """TD and QD 1024^3, binary64 slices (and e4m3 slices), with the simple
    multi-component GEMM as the side baseline (one timed pass each)."""
    out = []
    n = 1024
    for prec in ("td", "qd"):
        for form in ("fp64", "fp8bal", "fp8"):
            try:
                out.append(run_variant(oz, torch, prec, form, n, 1.0, 1, 1))
            except Exception as ex:
                out.append({"prec": prec, "form": form, "error": repr(ex)[:200]})
        A, B = _host_operands(prec, n, n, n, 1.0, 0)
        Ad = [oz.colmajor(a) for a in A]
        Bd = [oz.colmajor(b) for b in B]
        C = [torch.empty((n, n), dtype=torch.float64, device="cuda").T for _ in A]
        oz.ozmp_gemm_naive(prec, Ad, Bd, C)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        oz.ozmp_gemm_naive(prec, Ad, Bd, C)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        row = {"prec": prec, "form": "naive (multi-component triple loop)", "ms_per_step": ms,
               "gflops": 2.0 * n ** 3 / (ms * 1e-3) / 1e9}
        rows, cols = sample_idx(n, n, 64)
        row.update(sampled_error(torch, C, A, B, rows, cols, prec))
        out.append(row)
    return out


def batched_512_variant(oz, torch):
    """512 uneven DD/TD problems (m, n, k log-uniform in [32, 768], seed 1):
    one graph replay of the batched plan vs a loop of single calls."""
    from ozmp_inputs import batched_problem_shapes, gen_problem
    shapes = batched_problem_shapes(512, seed=1)
    probs = []
    flops = 0.0
    for idx, (m, n, k, prec) in enumerate(shapes):
        A, B = gen_problem(prec, m, n, k, phi=1.0, seed=1000 + idx)
        C = [torch.empty((n, m), dtype=torch.float64, device="cuda").T for _ in A]
        probs.append((prec, [oz.colmajor(a) for a in A], [oz.colmajor(b) for b in B], C, 0))
        flops += 2.0 * m * n * k
    plan = oz.ozmp_gemm_batched(probs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 3
    e0.record()
    for _ in range(reps):
        oz.ozmp_gemm_batched(probs, plan=plan)
    e1.record()
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1) / reps
    st = oz.ozmp_plan_get_status(plan)
    oz.ozmp_plan_destroy(plan)
    # error of 8 DD and 8 TD problems on up to 32 x 32 entries, against the oracle
    import numpy as np
    rng = np.random.default_rng(11)
    picks = []
    for want in ("dd", "td"):
        idx = [i for i, sh in enumerate(shapes) if sh[3] == want]
        picks += [int(x) for x in rng.choice(idx, 8, replace=False)]
    errs = {"dd": [], "td": []}
    for idx in picks:
        m, n, k, prec = shapes[idx]
        A, B = gen_problem(prec, m, n, k, phi=1.0, seed=1000 + idx)
        rows, cols = sample_idx(m, n, 32)
        errs[prec].append(sampled_error(torch, probs[idx][3], A, B, rows, cols, prec)["err_nw"])
    # the loop of single calls does the same work: the automatic (fixed-rule) counts of the batch
    def rule_count(p):
        return oz.Plan(p[0], p[1][0].shape[0], p[2][0].shape[1], p[1][0].shape[1], "auto", 0,
                       workspace=False).info.nslices
    plans = [oz.Plan(p[0], p[1][0].shape[0], p[2][0].shape[1], p[1][0].shape[1], "auto", rule_count(p))
             for p in probs]
    for pl, p in zip(plans, probs):
        pl.execute(p[1], p[2], p[3])
    torch.cuda.synchronize()
    e0.record()
    for pl, p in zip(plans, probs):
        pl.execute(p[1], p[2], p[3])
    e1.record()
    torch.cuda.synchronize()
    ms_l = e0.elapsed_time(e1)
    return {"problems": len(probs), "gflops_total": flops / 1e9, "batched_ms": ms_b,
            "batched_gflops": flops / (ms_b * 1e-3) / 1e9, "loop_ms": ms_l,
            "loop_gflops": flops / (ms_l * 1e-3) / 1e9, "status": st.name,
            "err_nw_max": {p: max(v) for p, v in errs.items()},
            "err_sample": "8 DD and 8 TD problems (seed 11), up to 32 x 32 entries each, full k, against the exact "
                          "product rounded to 512 bits",
            "target": {"dd": 2.0 ** -100, "td": 2.0 ** -150}}


# peak of the slice-product engine of a form (TFLOP/s or TOPS) and its source
def engine_peak(form, bf16, bf16_sus, src, burst):
    if form in ("fp8", "fp8_bal", "fp8bal", "fp8_mma", "fp8mma"):
        if burst:
            return bf16 * 2.0, f"e4m3 dense = bf16 {src} burst x 2 (nominal ratio)"
        return bf16_sus * 2.0, f"e4m3 dense = bf16 {src} sustained x 2 (nominal ratio)"
    if form == "fp16":
        # kind::f16 runs at the bf16 rate
        if burst:
            return bf16, f"f16 dense = bf16 {src} burst"
        return bf16_sus, f"f16 dense = bf16 {src} sustained"
    if form == "int8":
        return 151.3, "IMMA mma.sync s8 microbenchmark on this GB300 (no MEASURED_PEAKS entry)"
    return 1.05, "DMMA mma.sync f64 microbenchmark on this GB300 (no MEASURED_PEAKS entry)"


def timed_product(oz, torch, prec, form, m, n, k, Ad, Bd, warm, nslices=0):
    """One timed product through a plan (split, then multiply, CUDA events on
    the current stream; the product kernel alone from the plan's timing
    ring).  Returns (row, C, plan)."""
    dt = torch.float32 if prec == "ts" else torch.float64
    C = [torch.empty((n, m), dtype=dt, device="cuda").T for _ in Ad]
    p = oz.Plan(prec, m, n, k, form, nslices)
    for _ in range(warm):
        p.split(Ad, Bd)
        p.multiply(C)
    torch.cuda.synchronize()
    p.set_timing(1)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ev[0].record()
    p.split(Ad, Bd)
    ev[1].record()
    p.multiply(C)
    ev[2].record()
    torch.cuda.synchronize()
    kern = p.read_timing(1)
    p.set_timing(0)
    i = p.info
    flops = 2.0 * m * n * k
    tot = ev[0].elapsed_time(ev[2])
    split_ms = ev[0].elapsed_time(ev[1])
    kms = kern[0] if kern else ev[1].elapsed_time(ev[2])
    q = len(Ad)
    w = 4 if prec == "ts" else 8
    sb = splitter_bytes(q, w, m, n, k, i.nslices, i.digit_bytes)
    row = {"prec": prec, "form": oz.Form(i.form).name.lower(), "beta": i.beta, "nslices": i.nslices,
           "pairs": i.npairs, "ms": tot, "gflops": flops / (tot * 1e-3) / 1e9, "split_ms": split_ms,
           "product_kernel_ms": kms, "slice_tflops": i.npairs * flops / (kms * 1e-3) / 1e12,
           "splitter_gbs": sb / (split_ms * 1e-3) / 1e9, "status": p.status().name}
    return row, C, p


def min_slices(oz, torch, prec, form, As, Bs, ex, k, start):
    """The smallest forced slice count whose result meets the precision's
    target on the sampled block, found on the sampled rows and columns alone
    (full k): their exponents, digits and sums equal those of the whole
    product, so the block's error is the same."""
    from oracle import exact as X
    ms, ns = As[0].shape[0], Bs[0].shape[1]
    tgt = 2.0 ** -target_bits(prec)
    dt = torch.float32 if prec == "ts" else torch.float64

    def err(s):
        C = [torch.empty((ns, ms), dtype=dt, device="cuda").T for _ in As]
        p = oz.Plan(prec, ms, ns, k, form, s)
        p.execute(As, Bs, C)
        torch.cuda.synchronize()
        Cg = [c.cpu().numpy() for c in C]
        chat = [[[float(c[a, b]) for c in Cg] for b in range(ns)] for a in range(ms)]
        return X.error_metrics(chat, ex)["err_nw"]

    s = start
    if err(s) <= tgt:
        while s > 1 and err(s - 1) <= tgt:
            s -= 1
        return s
    while s < start + 16:
        s += 1
        if err(s) <= tgt:
            return s
    return None


def config3_variant(oz, torch, n=4096):
    """DD and QD n^3 with exponent spread phi in {0, 1, 4}: the balanced e4m3
    (tcgen05), int8 (IMMA) and binary64 (DMMA) digit forms, each at the
    slice count the library chooses from the data (nslices = 0): its time,
    and its error on a 64 x 64 block against the oracle; beside it the
    smallest slice count that still meets the target on that block."""
    import numpy as np
    from oracle import _clib
    out = []
    for prec in ("dd", "qd"):
        for phi in (0.0, 1.0, 4.0):
            A, B = _host_operands(prec, n, n, n, phi, 0)
            rows, cols = sample_idx(n, n, 64)
            ex = _clib.exact_block(A, B, rows, cols)
            Ad = [oz.colmajor(a) for a in A]
            Bd = [oz.colmajor(b) for b in B]
            As = [oz.colmajor(np.ascontiguousarray(a[rows])) for a in A]
            Bs = [oz.colmajor(np.ascontiguousarray(b[:, cols])) for b in B]
            for form in ("fp8bal", "int8", "fp64"):
                try:
                    row, C, p = timed_product(oz, torch, prec, form, n, n, n, Ad, Bd, 0 if form == "fp64" else 1)
                    row["phi"] = phi
                    row.update(sampled_error(torch, C, A, B, rows, cols, prec, ex))
                    row["s_min_on_block"] = min_slices(oz, torch, prec, form, As, Bs, ex, n, row["nslices"])
                    del C, p
                except Exception as e:  # report, do not hide
                    row = {"prec": prec, "phi": phi, "form": form, "error": repr(e)[:200]}
                out.append(row)
            del Ad, Bd, As, Bs
            torch.cuda.empty_cache()
    return out


def config5_variant(oz, torch):
    """QD m = n = 8192, k = 16384 and TS 8192^3 (phi = 1): the balanced e4m3
    and int8 forms (and, for TS, the binary32-slice form in binary16 digits
    and binary64 digits), each with the fraction of its engine's peak, the
    splitter's HBM rate and the error on a 32 x 32 block."""
    from oracle import _clib
    hbm, bf16, bf16_sus, src = measured_peaks()
    out = []
    for prec, m, n, k, forms in (("qd", 8192, 8192, 16384, ("fp8bal", "int8")),
                                 ("ts", 8192, 8192, 8192, ("fp8bal", "fp16", "int8", "fp64"))):
        A, B = _host_operands(prec, m, n, k, 1.0, 0)
        rows, cols = sample_idx(m, n, 32)
        ex = _clib.exact_block(A, B, rows, cols)
        Ad = [oz.colmajor(a) for a in A]
        Bd = [oz.colmajor(b) for b in B]
        for form in forms:
            try:
                row, C, p = timed_product(oz, torch, prec, form, m, n, k, Ad, Bd, 1 if form == "fp8bal" else 0)
                row.update({"m": m, "n": n, "k": k})
                peak, note = engine_peak(form, bf16, bf16_sus, src, burst=True)
                row["slice_frac_of_peak"] = row["slice_tflops"] / peak
                row["peak"] = peak
                row["peak_source"] = note
                row["splitter_frac_of_hbm"] = row["splitter_gbs"] / hbm
                row.update(sampled_error(torch, C, A, B, rows, cols, prec, ex))
                del C, p
            except Exception as e:
                row = {"prec": prec, "form": form, "error": repr(e)[:200]}
            out.append(row)
        del Ad, Bd
        torch.cuda.empty_cache()
    out.append({"not_timed": "QD 8192^2 x 16384 in binary64 digits: about 80 DMMA slice products of 2.2 TFLOP each, "
                             "near 3 minutes at the measured 1.05 TFLOP/s (bench.py --side config5_qd_fp64)"})
    return out


def config5_qd_fp64(oz, torch):
    from oracle import _clib
    prec, m, n, k = "qd", 8192, 8192, 16384
    A, B = _host_operands(prec, m, n, k, 1.0, 0)
    rows, cols = sample_idx(m, n, 32)
    Ad = [oz.colmajor(a) for a in A]
    Bd = [oz.colmajor(b) for b in B]
    row, C, p = timed_product(oz, torch, prec, "fp64", m, n, k, Ad, Bd, 0)
    row.update(sampled_error(torch, C, A, B, rows, cols, prec))
    return row


def launches_per_step(oz, info, Bd, k, w, adaptive=True, check=True):
    """Kernels of one plan execution (the register splitter, q <= 4).

    Slice count chosen from the data (adaptive): exponent init, the row
    exponent pass with the norms folded in, then for B either the one-pass
    column digit kernel, which also reduces B's exponents and norms (the
    conditions below), or a column exponent pass with the norms; the choice;
    the row digits (and the column digits when B took two kernels).  Fixed
    slice count: exponent init,
    row exponents, then for B either one pass (e4m3 forms, 16-byte aligned
    column starts and lengths, at most 112 KB a column) or column exponents
    + column digits, the row digits, and the exponent statistics of the
    check.  Then the slice-product kernel and, for the tcgen05 forms, its
    rounding pass (which runs the check); the other engines take a check
    pass over C.  (Exponents beyond +-230 add the scaled norm launches.)"""
    form = oz.Form(info.form)
    e4m3 = form in (oz.Form.FP8, oz.Form.FP8_BAL, oz.Form.FP8_MMA)
    tc = form in (oz.Form.FP8, oz.Form.FP8_BAL, oz.Form.FP16)
    ldb = Bd[0].stride(1)
    one_pass = (e4m3 and (k * w) % 16 == 0 and (ldb * w) % 16 == 0 and len(Bd) * k * w <= 112 * 1024
                and all(b.data_ptr() % 16 == 0 for b in Bd))
    if adaptive:
        split = 5 if one_pass else 6
    else:
        split = 3 + (1 if one_pass else 2) + (1 if check else 0)
    return split + 1 + (1 if tc else (1 if check else 0))


def splitter_bytes(q, w, m, n, k, s, db):
    # algorithmic bytes of K1 + K2: both operands read once, every digit
    # written once (the row exponents of A take a second read of A, which
    # counts as time, not as algorithmic bytes)
    return q * w * (m * k + k * n) + s * db * (m * k + k * n)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="dd")
    ap.add_argument("--form", default="auto")
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--phi", type=float, default=1.0)
    ap.add_argument("--nslices", type=int, default=0)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--side", default=None, choices=sorted(SIDE),
                    help="run one side measurement alone (one GPU) and print its JSON")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.side:
        import torch
        import paper_2301_09960_gb300 as oz
        torch.cuda.set_device(0)
        oz.load()
        print(json.dumps({"side": args.side, "result": SIDE[args.side](oz, torch)}))
        return
    ws, rank, local = _dist()
    workload = f"{args.prec} gemm m=n=k={args.n}, phi={args.phi}, Eq. 1 operands"
    metric = "DD/QD GEMM effective GFLOP/s (2mnk/s) and % of slice roofline, INT8 vs FP64"

    if args.impl == "reference":
        if rank != 0:
            return
        from oracle import _clib
        m = n = k = args.n
        A, B = _host_operands(args.prec, m, n, k, args.phi, 0)
        blk = 48
        rows, cols = list(range(blk)), list(range(blk))
        for _ in range(args.warmup):
            _clib.exact_block(A, B, rows[:8], cols[:8])
        t0 = time.time()
        for s in range(args.steps):
            r0 = (s * blk) % m
            _clib.exact_block(A, B, [r0 + i for i in rows], cols)
        dt = (time.time() - t0) / args.steps
        val = 2.0 * blk * blk * k / dt / 1e9
        cores = os.cpu_count()
        line = {"impl": "reference", "metric": metric, "value": val, "unit": "GFLOP/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64 components, exact 512-bit",
                "data": "synthetic (Eq. 1, seeded)",
                "config": {"workload": workload, "sample": f"{blk}x{blk} block of C per step, full k={k}"},
                "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": cores, "kind": "oracle",
                                 "sample": f"{blk}x{blk} block of C, k={k}, exact dot products rounded to 512 bits"},
                "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    import paper_2301_09960_gb300 as oz

    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    oz.load()

    m = n = k = args.n
    prec, form = args.prec, args.form
    A, B = _host_operands(prec, m, n, k, args.phi, _rank_seed(rank))
    q = len(A)
    dt = torch.float32 if prec == "ts" else torch.float64
    w = 4 if prec == "ts" else 8
    Ad = [oz.colmajor(a) for a in A]
    Bd = [oz.colmajor(b) for b in B]
    C = [torch.empty((n, m), dtype=dt, device="cuda").T for _ in range(q)]
    plan = oz.Plan(prec, m, n, k, form, args.nslices)

    for _ in range(args.warmup):
        plan.split(Ad, Bd)
        plan.multiply(C)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()

    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    plan.set_timing(args.steps)     # event pair around each product-kernel launch
    for s in range(args.steps):
        ev[s][0].record()
        plan.split(Ad, Bd)
        ev[s][1].record()
        plan.multiply(C)
        ev[s][2].record()
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    total_ms = ev[0][0].elapsed_time(ev[-1][2])
    kernel_runs = plan.read_timing(args.steps)
    plan.set_timing(0)
    kernel_ms = sum(kernel_runs) / max(len(kernel_runs), 1)
    clk = clocks.stop()
    split_ms = sum(e[0].elapsed_time(e[1]) for e in ev) / args.steps
    gemm_ms = sum(e[1].elapsed_time(e[2]) for e in ev) / args.steps
    status = plan.status()
    info = plan.info          # the slice count the splits chose from the data
    if ws > 1:
        total_ms = _max_over_ranks(total_ms, "cuda")
    ms_per_step = total_ms / args.steps
    flops = 2.0 * m * n * k
    value = ws * flops / (ms_per_step * 1e-3) / 1e9

    # ---- end to end through the C ABI with host buffers ----
    Ah = [torch.from_numpy(a.T.copy()).pin_memory() for a in A]     # (k, m) rows = columns of A
    Bh = [torch.from_numpy(b.T.copy()).pin_memory() for b in B]
    Ch = [torch.empty((n, m), dtype=dt).pin_memory() for _ in range(q)]
    # Steps are independent products, so they are pipelined as a serving
    # loop would: while the product of step i runs on the compute stream, one
    # copy stream brings in step i+1's operands and another takes out step
    # i-1's result (two streams, so that an upload never queues behind a
    # download); device operands and results are double-buffered.  Both
    # copies wait until step i's split has finished: a copy running beside
    # the split kernels doubled the split (0.8 -> 1.7 ms at DD 4096^3), while
    # beside the product they cost nothing measurable.  So the loop calls the
    # split and the multiply entry points itself, with an event between them.
    # Every step still copies its inputs in from pinned host memory and its
    # result out inside the timed region.
    bufs = [([torch.empty((k, m), dtype=dt, device="cuda") for _ in range(q)],
             [torch.empty((n, k), dtype=dt, device="cuda") for _ in range(q)],
             [torch.empty((n, m), dtype=dt, device="cuda") for _ in range(q)]) for _ in range(2)]
    h2d = sum(t.numel() * t.element_size() for t in Ah + Bh)
    d2h = sum(t.numel() * t.element_size() for t in Ch)
    e2e_steps = max(1, args.steps)   # as many steps as the device-resident measurement
    comp = torch.cuda.current_stream()
    cs_in, cs_out = torch.cuda.Stream(), torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in range(2)]      # a set's operands are on the device
    ev_split = [torch.cuda.Event() for _ in range(2)]   # the split that read a set's operands is done
    ev_done = [torch.cuda.Event() for _ in range(2)]    # the product that wrote a set's result is done
    ev_out = [torch.cuda.Event() for _ in range(2)]     # a set's result is on the host

    def copy_in(i):
        # step i's operands into set i % 2, once step i-1's split is done (in
        # stream order after step i-2's, the last reader of this set)
        Ad2, Bd2, _ = bufs[i % 2]
        with torch.cuda.stream(cs_in):
            if i >= 1:
                cs_in.wait_event(ev_split[(i - 1) % 2])
            for x, y in zip(Ad2 + Bd2, Ah + Bh):
                x.copy_(y, non_blocking=True)
            ev_in[i % 2].record(cs_in)

    def copy_out(i, after):
        # step i's result to the host, behind `after` on the compute stream
        with torch.cuda.stream(cs_out):
            cs_out.wait_event(after)
            for x, y in zip(Ch, bufs[i % 2][2]):
                x.copy_(y, non_blocking=True)
            ev_out[i % 2].record(cs_out)

    def compute(i):
        Ad2, Bd2, Cd2 = bufs[i % 2]
        comp.wait_event(ev_in[i % 2])
        if i >= 2:
            comp.wait_event(ev_out[i % 2])      # step i-2's result, in the same set, is on the host
        plan.split([x.T for x in Ad2], [x.T for x in Bd2])
        ev_split[i % 2].record(comp)
        plan.multiply([x.T for x in Cd2])
        ev_done[i % 2].record(comp)

    copy_in(0)
    compute(0)
    copy_out(0, ev_done[0])
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    cs_in.wait_event(e0)
    copy_in(1)
    for i in range(1, e2e_steps + 1):
        compute(i)
        if i < e2e_steps:
            copy_in(i + 1)                      # during step i's product
        if i >= 2:
            copy_out(i - 1, ev_split[i % 2])    # during step i's product
    copy_out(e2e_steps, ev_done[e2e_steps % 2])
    comp.wait_event(ev_out[e2e_steps % 2])      # the last result is on the host
    e1.record(comp)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    if ws > 1:
        e2e_ms = _max_over_ranks(e2e_ms, "cuda")
    e2e_val = ws * flops / (e2e_ms * 1e-3) / 1e9
    # the last result read out equals the device-resident loop's, bit for bit
    e2e_same = all(torch.equal(Ch[c], C[c].T.cpu()) for c in range(q))

    # ---- roofline of the dominant kernel (slice products) ----
    hbm, bf16, bf16_sus, src = measured_peaks()
    alg_flops = info.npairs * flops
    achieved = alg_flops / (kernel_ms * 1e-3) / 1e12
    # the burst peak matches a kernel timed in a short region at full clock;
    # the sustained one (a seconds-long loop under the power cap) matches a
    # region of seconds or one whose SM clock sat below its maximum
    region_s = total_ms * 1e-3
    capped = (clk.get("sm_mhz") is not None and clk.get("sm_max_mhz")
              and clk["sm_mhz"] < 0.95 * clk["sm_max_mhz"])
    burst = region_s < 2.0 and not capped
    fname = oz.Form(info.form).name.lower()
    peak, peak_note = engine_peak(fname, bf16, bf16_sus, src, burst)
    peak_note += (f"; timed region {region_s:.2f} s at median SM {clk.get('sm_mhz')} of {clk.get('sm_max_mhz')} MHz"
                  f" -> {'burst' if burst else 'sustained'}")
    peak_other = engine_peak(fname, bf16, bf16_sus, src, not burst)[0]
    sbytes = splitter_bytes(q, w, m, n, k, info.nslices, info.digit_bytes)
    # DRAM bytes (read + write) of one launch of the product kernel, from the
    # one-pass ncu capture of this workload's launch in
    # profiles/k_gemm_tc_bal_dd4096_s25_dram.md; only for the workload captured
    # there, with the default tile and pair orders
    traffic = None
    if (oz.Form(info.form) == oz.Form.FP8_BAL and prec == "dd" and m == n == k == 4096 and info.nslices == 25
            and os.environ.get("OZMP_TC_LOCKSTEP", "1") == "1" and os.environ.get("OZMP_TC_GROUP", "8") == "8"
            and os.environ.get("OZMP_TC_WALK", "1") == "1"):
        traffic = 18.865e9 + 3.367e9

    line = {
        "metric": metric, "value": value, "unit": "GFLOP/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "e4m3" if info.form in (oz.Form.FP8, oz.Form.FP8_BAL, oz.Form.FP8_MMA) else
        ({oz.Form.INT8: "s8", oz.Form.FP16: "f16"}.get(oz.Form(info.form), "f64")),
        "acc_dtype": "f32 (integers below 2^24, exact) -> int64 carry-save limbs"
        if info.form in (oz.Form.FP8, oz.Form.FP8_BAL, oz.Form.FP16) else
        ("f32 (exact integers) -> int64" if info.form == oz.Form.FP8_MMA else
         ("s32 -> int64" if info.form == oz.Form.INT8 else "f64 (exact integers) -> int64")),
        "data": "synthetic (Eq. 1, seeded)",
        "config": {"workload": workload, "prec": prec, "form": oz.Form(info.form).name.lower(), "m": m, "n": n,
                   "k": k, "phi": args.phi, "beta": info.beta, "nslices": info.nslices, "pairs": info.npairs,
                   "parallelism": f"replicas x{ws}" if ws > 1 else "1 gpu",
                   "l2": "inputs larger than L2 (A, B and the digit workspace each exceed 129 MB)"},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": {oz.Form.FP8: "k_gemm_tc (tcgen05)",
                                oz.Form.FP8_BAL: "k_gemm_tc (tcgen05)", oz.Form.FP16: "k_gemm_tc (tcgen05 kind::f16)",
                                oz.Form.FP8_MMA: "k_gemm_b1<FP8> (mma.sync)",
                                oz.Form.INT8: "k_gemm_b1<INT8> (mma.sync)"}.get(oz.Form(info.form), "k_gemm_f64 (DMMA)"),
                     "peak_source": peak_note,
                     # context: the other figure of the pair
                     "peak_other": peak_other, "frac_other": achieved / peak_other},
        "splitter": {"ms": split_ms, "bytes": sbytes, "achieved_gbs": sbytes / (split_ms * 1e-3) / 1e9,
                     "peak_gbs": hbm, "frac": sbytes / (split_ms * 1e-3) / 1e9 / hbm},
        "stage_ms": {"split": split_ms, "products": gemm_ms, "product_kernel": kernel_ms},
        "e2e": {"value": e2e_val, "unit": "GFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": e2e_ms, "steps": e2e_steps, "result_equals_device": e2e_same,
                "pipelined": "operands of step i+1 copied in and the result of step i-1 copied out on two copy "
                             "streams during step i's product, after its split (double-buffered device "
                             "operands and results)"},
        "gpu_launches": launches_per_step(oz, info, Bd, k, w, adaptive=args.nslices == 0) * args.steps,
        "clocks": clk,
        "device_status": status.name,
    }

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # oracle on the host cores: exact product of a bounded block, and the
        # GPU result's error on that block
        from oracle import _clib
        from oracle import exact as X
        blk = 160
        rows = list(range(0, m, m // blk))[:blk]
        cols = list(range(0, n, n // blk))[:blk]
        t0 = time.time()
        ex = _clib.exact_block(A, B, rows, cols)
        tcpu = time.time() - t0
        Cg = [c.cpu().numpy() for c in C]
        chat = [[[float(c[a, b]) for c in Cg] for b in cols] for a in rows]
        em = X.error_metrics(chat, ex)
        line["cpu_baseline"] = {"value": 2.0 * len(rows) * len(cols) * k / tcpu / 1e9, "unit": "GFLOP/s",
                                "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{len(rows)}x{len(cols)} strided block of C, full k={k}: exact dot "
                                          f"products rounded to 512 bits ({tcpu:.1f} s)"}
        line["error"] = {"err_nw": em["err_nw"], "err_max_rel": em["err_max"],
                         "vs": "exact product rounded to 512 bits, same block", "target": 2.0 ** -100}

    if rank == 0 and ws == 1 and not args.no_variants:
        del Ad, Bd, C, bufs, plan
        torch.cuda.empty_cache()
        try:
            add_variants(line, oz, torch, args)
        except Exception as ex:  # the headline line is printed whatever a side measurement does
            line["variants_error"] = repr(ex)[:300]

    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        dist.destroy_process_group()


# the side measurements that can run alone (--side)
SIDE = {
    "batched_512_problems": lambda oz, torch: batched_512_variant(oz, torch),
    "lu_4096": lambda oz, torch: lu_variant(oz, torch),
    "literal_vs_truncating_1024": lambda oz, torch: literal_variant(oz, torch),
    "td_qd_1024": lambda oz, torch: td_qd_1024_variant(oz, torch),
    "config3_phi_sweep_4096": lambda oz, torch: config3_variant(oz, torch),
    "config5_large": lambda oz, torch: config5_variant(oz, torch),
    "config5_qd_fp64": lambda oz, torch: config5_qd_fp64(oz, torch),
}


def add_variants(line, oz, torch, args):
    """Side measurements of the default run (rank 0, one GPU): the other
    forms and precisions, more components, LU, Algorithm 1 as printed, TD/QD
    at 1024 and the batched problems."""
    # the batch first: its tile-width calibration times short launches, which
    # the heavy sections below would leave running on a hot, power-capped GPU
    line["batched_512_problems"] = batched_512_variant(oz, torch)
    var = []
    # (the int8 and binary64 forms at 4096^3 are in config3, per exponent spread)
    for vp, vf in [("dd", "fp8"), ("dd", "fp8mma"), ("dd", "fp16"), ("qd", "fp8bal"), ("qd", "fp8"),
                   ("qd", "fp8mma")]:
        try:
            var.append(run_variant(oz, torch, vp, vf, args.n, args.phi, 1, 1))
        except Exception as ex:  # report, do not hide
            var.append({"prec": vp, "form": vf, "error": repr(ex)[:200]})
    line["variants"] = var
    # more components (Sec. 5's multiple precisions beyond QD): q binary64
    # words, about 53 q bits, target 2^(-50 q); one timed pass at 2048^3
    md = []
    for q in (8, 16):
        for form in ("fp8bal", "fp8"):
            try:
                r = run_variant(oz, torch, f"q{q}", form, 2048, args.phi, 1, 1)
                r["bits"] = 53 * q
                md.append(r)
            except Exception as ex:
                md.append({"prec": f"q{q}", "form": form, "error": repr(ex)[:200]})
    line["multiprecision_2048"] = md
    line["lu_4096"] = lu_variant(oz, torch)
    line["literal_vs_truncating_1024"] = literal_variant(oz, torch)
    line["td_qd_1024"] = td_qd_1024_variant(oz, torch)
    line["config3_phi_sweep_4096"] = config3_variant(oz, torch)
    line["config5_large"] = config5_variant(oz, torch)


if __name__ == "__main__":
    main()
