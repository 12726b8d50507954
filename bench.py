"""Benchmark of the sparse spectral method's hot path on one GB300 (or N replicas).

Workload (default): the d = 10 plain-FP64 configuration - a with 10 cosines in
[-8,8]^10 (s_a = 21), manufactured u with 20 +-pairs, f_hat = L[a_hat] u_hat
(|supp f_hat| = 840), N = 3 (|S| = 334,440, 2.51e6 operator nonzeros), CBC
lattice with M = 10^6.  Synthetic, seeded (workloads.make_cfg2).  Secondary
sections: the d = 100 workload (FP32 sampling and FFT at M = 2^26 + 15, |S| =
1.15e6, FP32-refined solve) and the 512-instance batched solve (persistent,
graph-replayed) against a loop of single solves.

One step = the whole path: CBC lattice choice, sft_recover(a), sft_recover(f)
(lattice sampling + length-M FFT + bin extraction), stamp_build (S^3 and the
neighbour table), right-hand side on S, FP64 CG solve to 1e-12.

Metric: stamped Galerkin nonzeros per second = nnz(L) x operator applications in
the step / step time.  Also reported: time to solution of the FP64 and the
FP32-refined solves (solve only) with their errors against the exact
(manufactured) solution, per-stage times, the roofline of the dominant kernel,
and the CPU oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

L2_BYTES = 129 * 2**20
FLUSH_BYTES = 512 * 2**20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the d=100 and batched sections")
    ap.add_argument("--apply-only", action="store_true",
                    help="run only the galerkin_apply section and print it (profiling the operator kernels)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in self.rows for n, v in zip(names, r[5:9]) if v.strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------- oracle legs

def oracle_setup(inst):
    """The oracle's stamping set (BFS), explicit sparse operator, right-hand
    side and Jacobi diagonal for the workload, from the exact coefficients."""
    from oracle import pipeline as op
    from oracle import solve as osol
    from oracle import stamp as ostamp
    from oracle import galerkin as ogal
    from oracle.sft import true_coefficients
    a = true_coefficients(inst.a.freq, inst.a.coef)
    af = np.array(list(a.keys()), np.int64)
    av = np.array(list(a.values()), np.complex128)
    ff, fv = op.forcing(inst)
    keep = np.abs(fv) > 0
    ff, fv = ff[keep], fv[keep]
    t0 = time.perf_counter()
    S, _ = ostamp.stamp_bfs(af, ff, inst.N)
    L, nnz = ogal.galerkin_matrix(S, af, av)
    b = op.rhs_on(S, ff, fv)
    D = osol.jacobi_diag(S, av[~af.any(axis=1)][0])
    return {"L": L, "b": b, "D": D, "nnz": nnz, "size": len(S), "seconds": time.perf_counter() - t0}


def run_reference(args, inst, budget_s=120.0):
    """The oracle as the reference arm: its operator is assembled once
    (stamping BFS and explicit matrix, reported as setup), then every warm-up
    and timed step runs the oracle's Jacobi PCG toward 1e-12 for at most as
    many applications as keep the whole run within about two minutes (the
    full solve takes 15); throughput = nonzeros x applications / PCG time."""
    from oracle import solve as osol
    world, rank, _ = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
        if rank != 0:
            dist.barrier()
            return
    st = oracle_setup(inst)
    t0 = time.perf_counter()
    _, it_full, _ = osol.pcg(st["L"], st["b"], st["D"], 1e-12, max_iter=1)
    per_apply = max(time.perf_counter() - t0, 1e-3) / 2.0          # one iteration + the initial residual
    per_step = budget_s / max(1, args.steps + args.warmup)
    cap = int(max(1, min(15, per_step / per_apply - 1)))
    for _ in range(args.warmup):
        osol.pcg(st["L"], st["b"], st["D"], 1e-12, max_iter=cap)
    tot, work = 0.0, 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, it, _ = osol.pcg(st["L"], st["b"], st["D"], 1e-12, max_iter=cap)
        tot += time.perf_counter() - t0
        work += st["nnz"] * (it + 1)
    value = work / tot
    sample = (f"oracle Jacobi PCG (numpy/scipy, FP64) on the explicit operator of the full workload "
              f"(|S| = {st['size']}, nnz = {st['nnz']}), at most {cap} of the 15 applications per step; "
              f"operator assembly (BFS stamping + matrix) {st['seconds']:.1f} s once, not in the steps")
    line = {
        "impl": "reference", "metric": "stamped Galerkin nnz/s", "value": value, "unit": "nnz/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "cfg2: d=10 plain FP64, s_a=21, |supp f|=840, N=3, |S|=334440"},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "setup_seconds": st["seconds"],
    }
    print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- helpers

def count_launches(fn):
    """Kernels of this library launched by fn() (CUPTI through torch.profiler);
    None when the profiler is unavailable."""
    import torch
    try:
        from torch.autograd import DeviceType
        from torch.profiler import ProfilerActivity, profile
        # device events are listed only beside CPU activity, and the first
        # profiling session of a process records none: open one to warm up
        with profile(activities=[ProfilerActivity.CPU, ProfilerActivity.CUDA]):
            torch.zeros(1, device="cuda").add_(1)
            torch.cuda.synchronize()
        with profile(activities=[ProfilerActivity.CPU, ProfilerActivity.CUDA]) as prof:
            fn()
            torch.cuda.synchronize()
        import re
        mine = re.compile(r"(^|[^A-Za-z])k_[a-z]")   # this library's kernels are k_* (mangled or not)
        names = [e.name for e in prof.events()
                 if e.device_type == DeviceType.CUDA and mine.search(e.name) and "at::" not in e.name]
        return len(names)
    except Exception:
        return None


def load_peaks():
    """The measured copy bandwidth and GEMM peaks of this GPU type, when present."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def fp64_peak_gflops(sm_mhz):
    """FP64 ALU peak: one FP64 FMA per SM clock (GB300; the per-SM rate comes
    from the ncu FP64-pipe counters of a pure-FP64 sampling kernel,
    k_sample<double>) x 152 SMs x 2 flops x clock."""
    return 152 * 2 * sm_mhz * 1e6 / 1e9


def d100_section(B, gp, flush, steps=2, smooth=False):
    """The d = 100 workload: FP32 samples and FFT at M = 2^26 + 15 (prime; with
    smooth=True the 7-smooth M = 2^26, no Bluestein chirp), |S| = 1.15e6,
    FP32-refined solve.  Times the whole path and its stages."""
    import torch
    inst = W.make_cfg5(smooth=smooth)
    prep = gp.prepare(inst)
    out = {"workload": "cfg5: d=100, s_a=41, 50 f pairs, N=3, FP32 sampling/FFT, FP32-refined solve"
                       + (", 7-smooth M" if smooth else ", prime M")}
    times = []
    for it in range(steps + 1):
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record()
        prep.z, prep.M = gp.choose_lattice(prep.extra["lattice"], prep.cand)
        ev[1].record()
        af, av = B.sft_recover(prep.z, prep.M, prep.a_freq, prep.a_coef, prep.cand, tau=1e-4, precision="fp32")
        ff, fv = B.sft_recover(prep.z, prep.M, prep.f_freq, prep.f_coef, prep.cand, tau=1e-4, precision="fp32")
        ev[2].record()
        stamp = B.stamp_build(af, av, ff, inst.N)
        f_on, _ = stamp.scatter(ff, fv)
        ev[3].record()
        u, st = B.solve(stamp, f_on, 1e-12, 1000, "fp32")
        ev[4].record()
        ev[4].synchronize()
        if it:
            times.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)] + [st["kernel_ms"]])
        if it < steps:
            stamp.destroy()
    med = np.median(np.array(times), axis=0)
    # the step itself: one sparse_spectral_solve call (as the headline step)
    fused_ms = []
    for it in range(steps + 1):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = gp.run_fused(prep, tol=1e-12, max_iter=1000, solve_precision="fp32_refined")
        e1.record()
        e1.synchronize()
        if r.stats["status"] != "SS_OK" or r.stamp.size != stamp.size:
            raise RuntimeError(f"d = 100 one-call step failed: {r.stats}")
        if it:
            fused_ms.append(e0.elapsed_time(e1))
        fst = r.stats
        r.stamp.destroy()
    step_ms = float(np.median(fused_ms))
    out.update({"M": int(prep.M), "stamp_size": stamp.size, "nnz": stamp.nnz,
                "ms_per_step": step_ms, "staged_ms_per_step": float(sum(med[:4])),
                "step_form": "ms_per_step: one sparse_spectral_solve call; breakdown_ms: the stages called one by one",
                "breakdown_ms": {"lattice": med[0], "sft": med[1], "stamp": med[2], "solve": med[3],
                                 "solve_kernel": med[4]},
                "solve": {"applies": fst["applies"], "outer_iters": fst["outer_iters"],
                          "inner_iters": fst["inner_iters"], "rel_residual": fst["rel_residual"],
                          "status": fst["status"]},
                "nnz_per_s": stamp.nnz * fst["applies"] / (step_ms / 1e3)})
    # FP32 operator alone (the inner-CG kernel): algorithmic bytes per apply
    x = torch.randn(stamp.size, dtype=torch.complex64, device="cuda")
    for _ in range(3):
        B.galerkin_apply(stamp, x)
    reps = 20
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        B.galerkin_apply(stamp, x)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    out["apply_fp32"] = {"ms": ms, "nnz_per_s": stamp.nnz / (ms / 1e3),
                         "note": "standalone FP32 galerkin_apply (one kernel), L2-warm back-to-back (host launch rate included)"}
    stamp.destroy()
    return out


def apply_section(B, gp, flush, peaks, reps=10):
    """galerkin_apply alone (pack of u into gather records + the operator), L2
    flushed before every call, on the d = 100 set (FP32 operator) and the
    d = 10 set (FP64 and FP32).  Algorithmic HBM bytes per call: the index
    stream (4 B per nonzero) plus, per row, u read, |k|^2 read and y written
    (FP32: 8 + 4 + 8 B, the norm as its 4-byte FP32 norm word; FP64 also reads
    the 16 B entry coefficient per nonzero and moves 16 B values with the
    8 B int64 norm).  FP64 is also given as FP64 flops (four
    FMAs per nonzero) against the FP64 ALU peak."""
    import torch
    out = {}
    hbm = peaks.get("hbm_gbs", 6783.5)
    for name, inst, precs in (("cfg5", W.make_cfg5(), ("fp32",)), ("cfg2", W.make_cfg2(), ("fp64", "fp32"))):
        p = gp.prepare(inst)
        r = gp.run(p, solve=False)
        st = r.stamp
        res = {"size": st.size, "nnz": st.nnz}
        for prec in precs:
            dt = torch.complex64 if prec == "fp32" else torch.complex128
            x = torch.randn(st.size, dtype=dt, device="cuda")
            y = B.galerkin_apply(st, x, prec)
            for _ in range(3):
                B.galerkin_apply(st, x, prec)
            # everything is queued before the first wait, so the host never
            # holds the GPU back: each apply starts right after its flush
            evs = []
            for _ in range(reps):
                flush.zero_()
                flush.sum()        # evicts the flush's dirty lines outside the timed region
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                B.galerkin_apply(st, x, prec)
                b.record()
                evs.append((a, b))
            torch.cuda.synchronize()
            ms = statistics.median([a.elapsed_time(b) for a, b in evs])
            realc = bool(st.real_coefficients) if prec == "fp64" else False
            if prec == "fp32":
                byts = 4 * st.nnz + st.size * (8 + 4 + 8)
            else:
                # index and coefficient per nonzero (8 B when the coefficients are real)
                byts = (4 + (8 if realc else 16)) * st.nnz + st.size * (16 + 8 + 16)
            d = {"ms": ms, "nnz_per_s": st.nnz / (ms / 1e3), "algorithmic_bytes": byts,
                 "achieved_gbs": byts / (ms / 1e3) / 1e9, "hbm_frac": byts / (ms / 1e3) / 1e9 / hbm}
            if prec == "fp64":
                d["fp64_gflops"] = (4.0 if realc else 8.0) * st.nnz / (ms / 1e3) / 1e9
                d["real_coefficients"] = realc
            res[prec] = d
        st.destroy()
        out[name] = res
    out["note"] = ("CUDA events around one galerkin_apply call (FP32: one kernel; FP64: pack + operator) after "
                   "a 512 MB L2 flush (write, "
                   "then read so that no dirty line is written back inside the timed call), all calls queued "
                   "before the first wait; fraction of the measured HBM copy bandwidth")
    return out


def adr_section(B, gp, flush, Q=1000):
    """The three-dimensional advection-diffusion-reaction data (Remark ADR,
    Section "Three-dimensional exactly sparse advection-diffusion-reaction
    equation"): 45 operator terms, 5 forcing terms, frequencies in
    [-49, 50]^3, N = 1 and 2.  Whole pipeline (lattice, 6 SFTs, union stamp,
    BiCGStab), then the exact and Monte Carlo proxy on S^{N+1}."""
    import torch
    out = {}
    for N in (1, 2):
        inst = W.make_adr(0, N=N)
        for it in range(2):   # the first pass warms up
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            res = gp.run_adr(inst)
            b.record()
            b.synchronize()
            if it == 0:
                res.stamp.destroy()
        st = res.stamp
        d = {"size": st.size, "nnz": st.nnz, "pipeline_ms": a.elapsed_time(b),
             "solve_kernel_ms": res.stats["kernel_ms"], "iterations": res.stats["inner_iters"],
             "applies": res.stats["applies"], "rel_residual": res.stats["rel_residual"],
             "status": res.stats["status"]}
        X = W.mc_points(0, Q, inst.d)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record()
        st.extend(1)
        e[1].record()
        f1, _ = st.scatter(res.f_freq, res.f_val)
        num, den = B.proxy_residual(st, res.u, f1)
        e[2].record()
        r, fx = B.proxy_mc(st, res.u, inst.f.freq, inst.f.coef, X)
        e[3].record()
        e[3].synchronize()
        d.update({"size_N_plus_1": st.size, "extend_ms": e[0].elapsed_time(e[1]),
                  "exact_proxy": float(np.sqrt(num / den)), "exact_proxy_ms": e[1].elapsed_time(e[2]),
                  "mc_proxy": float(torch.sqrt((r * r).sum() / (fx * fx).sum())), "mc_points": Q,
                  "mc_ms": e[2].elapsed_time(e[3])})
        st.destroy()
        out[f"N{N}"] = d
    return out


def identify_section(B, gp, flush):
    """Support identification without candidates (d + 1 shifted samplings and
    FFTs) of the d = 10 workload's forcing: 840 frequencies on the
    component-by-component lattice (M = 10^6) chosen for the known support."""
    import torch
    inst = W.make_cfg2()
    p = gp.prepare(inst)
    z, M = gp.choose_lattice(p.extra["lattice"], p.cand)
    K = int(p.cand.abs().max())
    P = next_prime_py(2 * K + 1)
    n_true = int(len(p.f_freq))
    times = []
    for it in range(3):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        f, v = B.sft_identify(z, M, p.f_freq, p.f_coef, P, s_max=4 * n_true + 8, tau=1e-9)
        b.record()
        b.synchronize()
        if it:
            times.append(a.elapsed_time(b))
    return {"workload": "cfg2 forcing (d=10, M=10^6)", "P": P, "identified": int(len(f)),
            "ms": statistics.median(times), "samplings_and_ffts": inst.d + 1}


def next_prime_py(n):
    def prime(m):
        if m < 2:
            return False
        i = 2
        while i * i <= m:
            if m % i == 0:
                return False
            i += 1
        return True
    while not prime(n):
        n += 1
    return n


DF_OPS_PER_PAIR = 150   # ten double-float multiply-adds of 15 FP32 instructions per (term, point)


def multiscale_section(B, gp, flush, reps=5):
    """The d = 3 multiscale workload (frequencies up to 2^10 per coordinate,
    N = 4): FP32-refined against plain FP64 on the same stamp, time to
    solution at relative residual 1e-10 and 1e-12, and the relative l2
    difference of the two solutions."""
    import torch
    inst = W.make_cfg3()
    res = gp.run(gp.prepare(inst), solve=False)
    st_ = res.stamp
    out = {"size": st_.size, "nnz": st_.nnz}
    for tol in (1e-10, 1e-12):
        sols = {}
        for prec in ("fp64", "fp32"):
            times = []
            for _ in range(reps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                u, stt = B.solve(st_, res.f_on_S, tol, 2000, prec)
                b.record()
                b.synchronize()
                times.append(a.elapsed_time(b))
            sols[prec] = u
            out[f"{prec}@{tol:g}"] = {"time_to_solution_ms": statistics.median(times), "kernel_ms": stt["kernel_ms"],
                                      "applies": stt["applies"], "rel_residual": stt["rel_residual"],
                                      "half_system": stt["half_system"], "status": stt["status"]}
        out[f"rel_l2_fp32_vs_fp64@{tol:g}"] = float(torch.linalg.norm(sols["fp32"] - sols["fp64"]) /
                                                   torch.linalg.norm(sols["fp64"]))
    st_.destroy()
    return out


def proxy_section(B, gp, flush, Q=1000):
    """Lemma ProxyError after the solve: extension to S^{N+1}, the exact proxy
    and its Monte Carlo estimate at Q = 1000 uniform points (the paper uses 200
    and 1000), for the d = 3 multiscale workload (given f, truncation error
    visible) and the d = 10 workload (manufactured: the proxy is the solver's
    tolerance)."""
    import torch
    out = {}
    for name, inst in (("cfg3", W.make_cfg3()), ("cfg2", W.make_cfg2())):
        prep = gp.prepare(inst)
        res = gp.run(prep, tol=1e-12)
        X = W.mc_points(0, Q, inst.d)
        n_u = res.stamp.size
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        res.stamp.extend(1)
        ev[1].record()
        f1, _ = res.stamp.scatter(res.f_freq, res.f_val)
        num, den = B.proxy_residual(res.stamp, res.u.to(torch.complex128), f1)
        ev[2].record()
        u128 = res.u.to(torch.complex128)
        r, fx = B.proxy_mc(res.stamp, u128, prep.f_freq, prep.f_coef, X)   # warm
        reps = 3
        ev[2].synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            r, fx = B.proxy_mc(res.stamp, u128, prep.f_freq, prep.f_coef, X)
        b.record()
        b.synchronize()
        mc_ms = a.elapsed_time(b) / reps
        pairs = (res.stamp.size + len(prep.f_freq)) * Q
        mc = float(torch.sqrt((r * r).sum() / (fx * fx).sum()))
        peak = 152 * 128 * 2070e6   # FP32 instructions per second at the maximum SM clock
        out[name] = {"n_u": n_u, "size_N_plus_1": res.stamp.size, "extend_ms": ev[0].elapsed_time(ev[1]),
                     "exact_proxy_ms": ev[1].elapsed_time(ev[2]), "exact": float(np.sqrt(num / den)),
                     "mc": mc, "points": Q, "mc_ms": mc_ms, "term_point_pairs": pairs,
                     "pairs_per_s": pairs / (mc_ms / 1e3),
                     "mc_fp32_frac": pairs * DF_OPS_PER_PAIR / (mc_ms / 1e3) / peak,
                     "note": "mc_ms: whole proxy_mc call (operator, export, three kernels); fraction of the "
                             "FP32 instruction peak at 150 double-float instructions per pair"}
        res.stamp.destroy()
    return out


def batched_section(B, flush, n_inst=512, reps=3, world=1, rank=0):
    """The batched workload: 512 instances of uneven d, s_a and |S| (1e3..1e5),
    FP32-refined, in one persistent graph-replayed launch vs a loop of single
    solves.  With several ranks the instances are split by estimated cost
    (paper_2302_00752_gb300.shard; no data-path collective) and the time is the
    slowest rank's.  Instance set-up (recovery and stamping) is not timed."""
    import torch
    from paper_2302_00752_gb300 import pipeline as gp
    from paper_2302_00752_gb300.shard import partition_instances
    insts = W.make_cfg4(n=n_inst)
    cost = [W.generic_stamp_count(2 * len(i.f.freq), 2 * len(i.a.freq) - 1, i.N) * (2 * len(i.a.freq) - 1)
            for i in insts]
    mine = partition_instances(cost, world)[rank]
    insts = [insts[i] for i in mine]
    stamps, fs = [], []
    t0 = time.perf_counter()
    for inst in insts:
        p = gp.prepare(inst)
        r = gp.run(p, tol=1e-12, solve_precision=None, solve=False)
        stamps.append(r.stamp)
        fs.append(r.f_on_S)
    setup_s = time.perf_counter() - t0
    batch = B.Batch(stamps)
    us = [torch.empty_like(f) for f in fs]
    best_ms, cfg = batch.autotune(fs, us, tol=1e-12, max_iter=500, precision="fp32")
    batch.solve(fs, us, tol=1e-12, max_iter=500, precision="fp32", use_graph=True)
    bt, lt = [], []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _, stats = batch.solve(fs, us, tol=1e-12, max_iter=500, precision="fp32", use_graph=True)
        b.record()
        b.synchronize()
        bt.append(a.elapsed_time(b))
        flush.zero_()
        a.record()
        single = [B.solve(s, f, 1e-12, 500, "fp32") for s, f in zip(stamps, fs)]
        b.record()
        b.synchronize()
        lt.append(a.elapsed_time(b))
    # the same batch in the plain FP64 form (graph, same tiles), for comparison
    batch.solve(fs, us, tol=1e-12, max_iter=500, precision="fp64", use_graph=True)
    ft = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        _, stats64 = batch.solve(fs, us, tol=1e-12, max_iter=500, precision="fp64", use_graph=True)
        b.record()
        b.synchronize()
        ft.append(a.elapsed_time(b))
    fp64_ok = all(st["status"] == "SS_OK" for st in stats64)
    applies = sum(st["applies"] for st in stats)
    nnz_applied = sum(s.nnz * st["applies"] for s, st in zip(stamps, stats))
    ok = all(st["status"] == "SS_OK" for st in stats)
    sizes = [s.size for s in stamps]
    t_b, t_l = statistics.median(bt), statistics.median(lt)
    if world > 1:
        dev = torch.device("cuda", torch.cuda.current_device())
        v = torch.tensor([t_b, t_l], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(v, op=torch.distributed.ReduceOp.MAX)
        w = torch.tensor([nnz_applied, float(ok is False)], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(w)
        t_b, t_l = float(v[0]), float(v[1])
        nnz_applied, ok = float(w[0]), bool(w[1] == 0)
    out = {"workload": f"cfg4: {n_inst} instances, d 6..30, s_a 5..41, |S| {min(sizes)}..{max(sizes)} (rank 0)",
           "ranks": world, "instances_rank0": len(stamps),
           "total_rows_rank0": int(sum(sizes)), "total_nnz_rank0": int(sum(s.nnz for s in stamps)),
           "persistent_graph_ms": t_b, "loop_of_single_solves_ms": t_l,
           "speedup": t_l / t_b, "nnz_per_s": nnz_applied / (t_b / 1e3), "applies_rank0": applies,
           "all_converged": ok, "autotuned": cfg, "autotune_best_ms": best_ms, "setup_s": setup_s,
           "fp64_persistent_graph_ms_rank0": statistics.median(ft), "fp64_all_converged_rank0": fp64_ok,
           "fp32_refined_vs_fp64_speedup_rank0": statistics.median(ft) / statistics.median(bt)}
    batch.destroy()
    for s in stamps:
        s.destroy()
    return out


# ---------------------------------------------------------------- our path

def main():
    args = parse()
    inst = W.make_cfg2()
    if args.impl == "reference":
        run_reference(args, inst)
        return
    import torch
    if args.apply_only:
        from paper_2302_00752_gb300 import binding as B
        from paper_2302_00752_gb300 import pipeline as gp
        flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
        print(json.dumps({"apply": apply_section(B, gp, flush, load_peaks())}))
        return
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2302_00752_gb300 import binding as B
    from paper_2302_00752_gb300 import pipeline as gp

    dev = torch.device("cuda", local)
    prep = gp.prepare(inst)                         # manufactured f_hat built by the library (untimed)
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    u_buf = torch.empty(1 << 20, dtype=torch.complex128, device=dev)   # solution buffer, reused by every step

    def step(p, keep=False):
        """One pass of Algorithm 1 through the single library call
        (sparse_spectral_solve): the timed step."""
        r = gp.run_fused(p, tol=1e-12, max_iter=1000, tau=1e-9, solve_precision="fp64", out=u_buf)
        st = r.stats
        if st["status"] != "SS_OK":
            raise RuntimeError(f"solve failed: {st}")
        out = {"nnz": r.stamp.nnz, "size": r.stamp.size, "zero_index": r.stamp.zero_index, "applies": st["applies"],
               "iters": st["inner_iters"], "times": {"solve_kernel": st["kernel_ms"]}, "u": r.u, "stats": st}
        if keep:
            out["stamp"] = r.stamp
        else:
            r.stamp.destroy()
        return out

    def staged_step(p, keep=False):
        """The same stages called one by one from Python, with CUDA events
        between them (the per-stage breakdown; not the timed step)."""
        t = {}
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
        ev[0].record()
        p.z, p.M = gp.choose_lattice(p.extra["lattice"], p.cand)
        ev[1].record()
        af, av = B.sft_recover(p.z, p.M, p.a_freq, p.a_coef, p.cand, tau=1e-9, precision="fp64")
        ff, fv = B.sft_recover(p.z, p.M, p.f_freq, p.f_coef, p.cand, tau=1e-9, precision="fp64")
        ev[2].record()
        stamp = B.stamp_build(af, av, ff, inst.N)
        f_on, _ = stamp.scatter(ff, fv, count_outside=False)
        ev[3].record()
        u, st = B.solve(stamp, f_on, 1e-12, 1000, "fp64")
        ev[4].record()
        ev[4].synchronize()
        t["lattice"] = ev[0].elapsed_time(ev[1])
        t["sft"] = ev[1].elapsed_time(ev[2])
        t["stamp"] = ev[2].elapsed_time(ev[3])
        t["solve"] = ev[3].elapsed_time(ev[4])
        t["solve_kernel"] = st["kernel_ms"]
        out = {"nnz": stamp.nnz, "size": stamp.size, "applies": st["applies"], "iters": st["inner_iters"],
               "times": t, "u": u, "stats": st}
        if keep:
            out["stamp"], out["f_on"] = stamp, f_on
        else:
            stamp.destroy()
        return out

    for _ in range(max(3, args.warmup)):
        step(prep)

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms, work, stage = [], 0, {}
    for _ in range(args.steps):
        flush.zero_()                               # L2 flushed between steps
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = step(prep)
        e1.record()
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        work += r["nnz"] * r["applies"]
        for k, v in r["times"].items():
            stage.setdefault(k, []).append(v)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks.stop()
    total_ms = sum(step_ms)
    if world > 1:
        tt = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(tt.item())
    value = world * work / (total_ms / 1e3)

    # per-stage breakdown from the staged form (same kernels, Python between the stages)
    staged_ms = []
    for _ in range(max(3, args.steps)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = staged_step(prep)
        e1.record()
        e1.synchronize()
        staged_ms.append(e0.elapsed_time(e1))
        for k, v in r["times"].items():
            if k != "solve_kernel":
                stage.setdefault(k, []).append(v)

    # solve-only time to solution, FP64 vs FP32-refined, errors against the exact solution
    keep = staged_step(prep, keep=True)
    stamp, f_on = keep["stamp"], keep["f_on"]
    S, lv = stamp.export()
    S = S.cpu().numpy()
    # stamping throughput: every set member of levels 0..N-1 tries every step of supp a_hat
    counts = np.bincount(lv.cpu().numpy().astype(np.int64), minlength=inst.N + 1)
    af = np.asarray(inst.a.freq, np.int64)
    s_a = len({tuple(k) for k in np.vstack([af, -af]).tolist()})   # |supp a_hat| of the real coefficient
    cand = int(sum(counts[n] for n in range(inst.N)) * s_a)
    stamp_stats = {"level_sizes": counts.tolist(), "candidates": cand,
                   "candidates_per_s": cand / (statistics.median(stage["stamp"]) / 1e3),
                   "stamp_ms": statistics.median(stage["stamp"]),
                   "note": "whole stamp_build + scatter call (levels, hash, neighbour table, coefficients)"}
    idx = {tuple(k): i for i, k in enumerate(S.tolist())}
    exact = np.zeros(len(S), complex)
    for k, v in zip(inst.u_freq.tolist(), inst.u_val):
        exact[idx[tuple(k)]] = v
    tts = {}
    for prec in ("fp64", "fp64_full", "fp32", "df64", "fp64@1e-10", "fp32@1e-10"):
        times, kern = [], []
        stamp.set_symmetry(prec != "fp64_full")        # fp64_full: the full system, for comparison
        base, tol_p = (prec.split("@")[0], 1e-10) if "@" in prec else (prec, 1e-12)
        for _ in range(5):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            u, st = B.solve(stamp, f_on, tol_p, 1000, "fp64" if base == "fp64_full" else base)
            b.record()
            b.synchronize()
            times.append(a.elapsed_time(b))
            kern.append(st["kernel_ms"])
        uu = u.cpu().numpy()
        err = float(np.linalg.norm(uu - exact) / np.linalg.norm(exact))
        tts[prec] = {"time_to_solution_ms": statistics.median(times), "kernel_ms": statistics.median(kern),
                     "rel_l2_err_vs_exact": err, "rel_residual": st["rel_residual"], "applies": st["applies"],
                     "outer_iters": st["outer_iters"], "inner_iters": st["inner_iters"],
                     "half_system": st["half_system"],
                     "nnz_per_s": stamp.nnz * st["applies"] / (statistics.median(kern) / 1e3)}

    # end to end through the C ABI with host buffers: H2D of the data, D2H of u
    host = {k: getattr(prep, k).cpu().pin_memory() for k in ("a_freq", "a_coef", "f_freq", "f_coef", "cand")}
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    u_host = torch.empty(stamp.size, dtype=torch.complex128).pin_memory()
    d2h = u_host.numel() * u_host.element_size()
    stamp.destroy()
    e2e_ms, e2e_work = [], 0
    for _ in range(args.steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        p2 = gp.Prepared(prep.d, prep.N, *[host[k].to(dev, non_blocking=True) for k in
                                           ("a_freq", "a_coef", "f_freq", "f_coef", "cand")],
                         sft_precision="fp64", solve_precision="fp64", extra=prep.extra)
        r = step(p2)
        u_host.copy_(r["u"], non_blocking=True)
        b.record()
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
        e2e_work += r["nnz"] * r["applies"]
    e2e_value = world * e2e_work / (sum(e2e_ms) / 1e3)

    # roofline of the dominant kernel: the persistent FP64 CG (FP64 ALU bound;
    # algorithmic flops: 8 per processed nonzero and application (4 FP64 FMAs
    # of the complex product), 4 when the entry coefficients are real, and 30
    # per processed row and CG iteration for the vector updates and the three
    # inner products).  With the Hermitian half system the CG processes the
    # rows k >lex 0 and their nonzeros, half of S and half of L's nonzeros
    # (symmetric S; the zero row stores none).
    med = {k: statistics.median(v) for k, v in stage.items()}
    nnz, size, iters = r["nnz"], r["size"], r["iters"]
    applies = r["applies"]
    half = bool(r["stats"].get("half_system"))
    realc = bool(r["stats"].get("real_coefficients"))
    nnz_p = nnz / 2 if half else nnz
    rows_p = (size - (1 if r["zero_index"] >= 0 else 0)) // 2 if half else size
    # real entry coefficients (a_hat real): 2 FP64 FMAs per nonzero, else 4
    flops_nnz = 4.0 if realc else 8.0
    solve_flops = flops_nnz * nnz_p * applies + 30.0 * rows_p * iters
    kms = med["solve_kernel"]
    clk = clocks.summary()
    sm_max = clk.get("sm_max_mhz") or 2070.0
    peak64 = fp64_peak_gflops(sm_max)
    achieved = solve_flops / (kms / 1e3) / 1e9
    # DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
    # the ncu capture in profiles/k_solve_fp64_half_system_cfg2.md, taken on
    # this kernel for this workload (half system, real coefficients)
    traffic = 41.355008e6 + 2.038272e6 if (half and realc) else None
    roofline = {"kernel": "k_solve<0> (persistent FP64 CG)", "bound": "alu", "achieved": achieved, "peak": peak64,
                "unit": "GFLOP/s (FP64)", "frac": achieved / peak64, "traffic": traffic,
                "traffic_unit": "DRAM bytes per launch (one ncu capture of this kernel on this workload)",
                "peak_source": "derived: 1 FP64 FMA/clk/SM (ncu FP64-pipe counters) x 152 SMs x 2 x sm_max_mhz",
                "flops_per_launch": solve_flops, "kernel_ms": kms, "half_system": half,
                "real_coefficients": realc, "flops_per_processed_nnz": flops_nnz,
                "processed_nnz": nnz_p, "processed_rows": rows_p}
    launches_per_step = count_launches(lambda: step(prep))
    gpu_launches = launches_per_step * args.steps if launches_per_step is not None else None

    extra = {}
    if not args.no_extra:
        if rank == 0:
            try:
                extra["d100"] = d100_section(B, gp, flush)
            except Exception as e:  # reported, not hidden
                extra["d100"] = {"error": repr(e)}
            try:
                extra["d100_smooth_M"] = d100_section(B, gp, flush, smooth=True)
            except Exception as e:
                extra["d100_smooth_M"] = {"error": repr(e)}
            try:
                extra["apply"] = apply_section(B, gp, flush, load_peaks())
            except Exception as e:
                extra["apply"] = {"error": repr(e)}
            try:
                extra["identify"] = identify_section(B, gp, flush)
            except Exception as e:
                extra["identify"] = {"error": repr(e)}
            try:
                extra["adr"] = adr_section(B, gp, flush)
            except Exception as e:
                extra["adr"] = {"error": repr(e)}
            try:
                extra["multiscale"] = multiscale_section(B, gp, flush)
            except Exception as e:
                extra["multiscale"] = {"error": repr(e)}
            try:
                extra["proxy"] = proxy_section(B, gp, flush)
            except Exception as e:
                extra["proxy"] = {"error": repr(e)}
        if world > 1:
            torch.distributed.barrier()
        extra["batched"] = batched_section(B, flush, world=world, rank=rank)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import solve as osol
        o = oracle_setup(inst)
        t0 = time.perf_counter()
        _, it, _ = osol.pcg(o["L"], o["b"], o["D"], 1e-12)
        dt = time.perf_counter() - t0
        cpu = {"value": o["nnz"] * (it + 1) / dt, "unit": "nnz/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle Jacobi PCG to 1e-12 (numpy/scipy FP64, {it + 1} applications, {dt:.2f} s) on "
                         f"the explicit operator of the full workload; its assembly (BFS stamping + matrix, "
                         f"{o['seconds']:.1f} s) and the DFT recovery are not in the time",
               "full_path_nnz_per_s": o["nnz"] * (it + 1) / (dt + o["seconds"])}
        try:
            from oracle import cpu_pcg
            t0 = time.perf_counter()
            n_cores = len(os.sched_getaffinity(0))
            _, it_c = cpu_pcg.pcg(o["L"], o["b"], o["D"], 1e-12, n_threads=n_cores)
            dt_c = time.perf_counter() - t0
            cpu["all_cores"] = {"value": o["nnz"] * (it_c + 1) / dt_c, "unit": "nnz/s", "cores": n_cores,
                                "kind": "oracle (C, OpenMP)",
                                "sample": f"the same Jacobi PCG in C with OpenMP row-parallel products on the same "
                                          f"CSR operator ({it_c + 1} applications, {dt_c:.2f} s)"}
        except Exception as e:
            cpu["all_cores"] = {"error": repr(e)}

    if rank == 0:
        line = {
            "metric": "stamped Galerkin nnz/s", "value": value, "unit": "nnz/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cfg2: d=10 plain FP64, s_a=21, manufactured u (20 pairs), |supp f|=840, N=3",
                       "stamp_size": size, "nnz": nnz, "M": int(prep.M), "l2_flush": True,
                       "nnz_counting": ("value counts the nonzeros of L_{N,s} per operator application; the FP64 "
                                        "CG runs the Hermitian half system (rows k >lex 0, half of the stored "
                                        "nonzeros per application, the rest by u_{-k} = conj(u_k)) when "
                                        "half_system is true; processed_nnz_per_s counts the nonzeros it reads"),
                       "parallelism": "replicas" if world > 1 else "single"},
            "e2e": {"value": e2e_value, "unit": "nnz/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": sum(e2e_ms) / len(e2e_ms)},
            "breakdown_ms": med,
            "staged_ms_per_step": statistics.median(staged_ms),
            "step_form": ("timed step: sparse_spectral_solve (one library call for lattice, both SFTs, stamp, "
                          "right-hand side, solve); breakdown_ms and staged_ms_per_step from the same stages "
                          "called one by one from Python with events between them"),
            "processed_nnz_per_s": value * (nnz_p / nnz if nnz else 1.0),
            "half_system": half,
            "solve_only": tts,
            "stamp": stamp_stats,
            "roofline": roofline,
            "gpu_launches": gpu_launches,
            "gpu_launches_per_step": launches_per_step,
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        line.update(extra)
        print(json.dumps(line))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
