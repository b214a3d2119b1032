#!/usr/bin/env python
"""Benchmark: inertia-validated factorizations per second and time to lambda_k on the synthetic
tight-binding workload (default: n = 1,048,576, the periodic diamond pencil of 32x32x32 cells).

A step is one pass of the whole hot path on the GPU: numeric LDL^T of A - sigma*B (assembly,
extend-add, Bunch-Kaufman pivoting, Schur updates, inertia reduction), one solve with the factor,
and one A/B sparse product.  Every step uses a new shift.  After the timed steps the counts are
validated (non-decreasing in sigma, and equal to those of a second, independently ordered
analysis at two of the timed shifts: Sylvester's law makes the count independent of the
ordering and of every pivot choice), and Algorithm 4 runs once for the time to lambda_k with the
paper's bisection in Algorithm 1', then once more with the interpolating shift rule (the
root-finder variant the paper proposes; same start vectors, lambda_k compared).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead (bounded sample).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD_N = {"scale": "524,288", "million": "1,048,576", "mid": "49,768", "small": "2,048"}


def metric_for(workload: str) -> str:
    return f"inertia-validated factorizations/s (n={WORKLOAD_N[workload]} tight-binding pencil)"


UNIT = "factorizations/s"
# FP64 FMA issue rate of GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (max SM clock).
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.07e9
# DRAM bytes (read + write) of lf_flush_tc_kernel per FP64-equivalent update flop, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) over all 832 flush launches of one factorization
# of the n = 49,768 workload: 18.41 GB for 4.095e11 flop
FLUSH_DRAM_BYTES_PER_FP64_FLOP = 0.04496
WORKLOAD_DESC = {
    "scale": "periodic diamond 32x32x18 cells, 16,384 random vacancies, 131,072 atoms x 4 sp3 orbitals, "
             "n=524,288, jitter 0.05 A, 2.9 A cutoff",
    "million": "periodic diamond 32x32x32 cells, 262,144 atoms x 4 sp3 orbitals, n=1,048,576, jitter 0.05 A, "
               "2.9 A cutoff",
    "mid": "periodic diamond 12x12x12 cells, 1,382 vacancies, n=49,768",
    "small": "periodic diamond 4x4x4 cells, n=2,048",
}
# cpu_baseline sample: the same generator (jitter, vacancy fraction) on a smaller periodic box
CPU_SAMPLE = dict(nx=5, ny=5, nz=4, vacancies=89)
# the oracle's work is scaled to the full workload by the ratio of the default-ordering GPU plan's
# flop counts (the oracle runs its own ordering whichever ordering the GPU arm uses)
CPU_SCALE_NOTE = "scaled by the ratio of the default nested-dissection plan's flop counts (sample / full)"


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def make_workload(name: str):
    from gen import workload
    return workload(name, seed=0)


def shifts_for(k: int, count: int):
    # shifts walking through the middle of the spectrum (where Algorithm 1' bisects)
    return [0.30 + 0.013 * i for i in range(count)]


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.device)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _measured_peaks():
    """Peaks from MEASURED_PEAKS.json when present (bf16 FLOP/s burst and sustained, HBM B/s), else
    the fallback figures; each with its source."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    out = {"bf16": (1.9e15, "of fallback: 1.9 PFLOP/s bf16 burst"),
           "bf16_sustained": (1.7e15, "of fallback: 1.7 PFLOP/s bf16 sustained"),
           "hbm": (6.8e12, "of fallback: 6.8 TB/s")}
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return out
    for key, field, scale in (("bf16", "bf16_tflops", 1e12), ("bf16_sustained", "bf16_tflops_sustained", 1e12),
                              ("hbm", "hbm_gbs", 1e9)):
        try:
            out[key] = (float(d[field]) * scale, f"of measured: MEASURED_PEAKS.json {field}")
        except (KeyError, TypeError, ValueError):
            pass
    return out


def measure_fp64_peak(torch, n: int = 8192, reps: int = 3):
    """FP64 rate of this GPU measured with the vendor library (cuBLAS DGEMM through torch.mm,
    n x n, best of reps): the denominator for the FP64 fractions (not on the hot path)."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    torch.mm(a, b)
    best = None
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.mm(a, b)
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 1e3
        best = t if best is None else min(best, t)
    del a, b
    torch.cuda.empty_cache()
    return 2.0 * n ** 3 / best


def flops_of(p, refined: bool = False) -> float:
    """Symbolic factorization flops of the GPU plan for pencil p (host analysis only, no device)."""
    import paper_1710_05134_gb300 as kep
    return kep.symbolic_info(p.n, p.rowptr, p.colind, p.coords, refined_order=refined).flops_factor


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_oracle_run(seconds: float, first_shift: int = 0):
    """The oracle's sparse LDL^T (c3, plain C, as it stands) on the sample pencil, one factorization
    per thread at a time on every host core (independent shifts; the C call releases the GIL), for
    about `seconds` of wall time.  Returns (sample pencil, factorizations done, wall seconds, cores)."""
    from gen import make_pair
    from oracle import core
    s = CPU_SAMPLE
    p = make_pair(s["nx"], s["ny"], s["nz"], seed=0, vacancies=s["vacancies"])
    core.sparse_inertia(p.rowptr, p.colind, p.a, p.b, 1.0, -0.3)   # compile/load outside timing
    cores = host_cores()
    counter = [first_shift]
    done = [0]
    lock = threading.Lock()
    deadline = [0.0]

    def worker():
        while True:
            with lock:
                if time.perf_counter() >= deadline[0]:
                    return
                i = counter[0]
                counter[0] += 1
            core.sparse_inertia(p.rowptr, p.colind, p.a, p.b, 1.0, -(0.30 + 0.013 * (i % 64)))
            with lock:
                done[0] += 1

    threads = [threading.Thread(target=worker) for _ in range(cores)]
    t0 = time.perf_counter()
    deadline[0] = t0 + seconds
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    return p, done[0], time.perf_counter() - t0, cores


def cpu_sample_desc(p, done, wall, cores, ratio, n_full):
    s = CPU_SAMPLE
    return (f"oracle sparse LDL^T (c3, plain C, own nested dissection) on the same generator at "
            f"{s['nx']}x{s['ny']}x{s['nz']} cells with {s['vacancies']} vacancies (n={p.n}): {done} factorizations "
            f"at independent shifts on {cores} threads in {wall:.1f} s, {CPU_SCALE_NOTE}, "
            f"{ratio:.3e}, to n={n_full}")


def run_reference(args):
    """The CPU oracle timed on the host cores: each step is a bounded run of the oracle on the
    sample pencil on every core, scaled to the workload."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    full = make_workload(args.workload)
    p0 = _cpu_sample_pencil()
    ratio = flops_of(p0) / flops_of(full)
    per_step = 4.0
    if args.warmup > 0:
        cpu_oracle_run(1.0)                            # warm-up
    done_all, wall_all, cores = 0, 0.0, 1
    for i in range(args.steps):
        p, done, wall, cores = cpu_oracle_run(per_step, first_shift=i)
        done_all += done
        wall_all += wall
    value = done_all / wall_all * ratio
    sample = cpu_sample_desc(p0, done_all, wall_all, cores, ratio, full.n)
    line = {"impl": "reference", "metric": metric_for(args.workload), "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 / value if value > 0 else None,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "desc": WORKLOAD_DESC.get(args.workload)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _cpu_sample_pencil():
    from gen import make_pair
    s = CPU_SAMPLE
    return make_pair(s["nx"], s["ny"], s["nz"], seed=0, vacancies=s["vacancies"])


VARIANTS = ("grad", "fp32_factor_ir", "two_shifts_in_flight", "autotune_schur", "gershgorin_multisection8",
            "stage3_f32_ir", "hermitian_mid")
# variants on a workload of their own (run after the main problem is released)
SEPARATE_VARIANTS = ("multisection_batch", "graph_replay", "hermitian_full", "precision_full")
# run only when named (minutes each): the n = 524,288 complex workload and the n = 1,500,000
# mixed-precision workload at their stated sizes
EXPLICIT_VARIANTS = ("hermitian_full", "precision_full")


def measure_variants(P, p, torch, kth, which="all"):
    """Timings of the next rows on the same problem (device-synchronised wall clock)."""
    want = set(VARIANTS) if which == "all" else set(which.split(",")) - set(SEPARATE_VARIANTS)
    unknown = want - set(VARIANTS)
    if unknown:
        raise ValueError(f"unknown variants {sorted(unknown)}")
    out = {}
    sync = torch.cuda.synchronize
    n = p.n
    # kep_grad: d lambda / d (A, B) values for an eigenvector (the one of --kth if it ran)
    lam = kth["lambda_k"] if kth else 0.0
    xk = getattr(P, "_last_x", None)
    if xk is None:
        xk = np.random.default_rng(0).normal(size=n)
    if "grad" in want:
        x = torch.from_numpy(np.ascontiguousarray(xk)).cuda()
        P.grad(lam, x)
        sync(); t0 = time.perf_counter()
        for _ in range(5):
            P.grad(lam, x)
        sync(); dt = (time.perf_counter() - t0) / 5
        out["grad"] = {"ms": 1e3 * dt, "entries": P.nnz,
                       "bytes_per_call": P.nnz * (8 + 4 + 16) + 2 * 8 * n}
    if "fp32_factor_ir" in want:
        out["fp32_factor_ir"] = measure_fp32_factor(P, p, torch)
    if "two_shifts_in_flight" in want:
        out["two_shifts_in_flight"] = measure_two_in_flight(P, p, torch)
    if "autotune_schur" in want:
        from paper_1710_05134_gb300 import tune
        try:
            r = tune.tune_schur(P, [0.31, 0.33], sync=sync)
            out["autotune_schur"] = {"best": list(r["best"]), "nu": r["nu"],
                                     "seconds": {f"{k[0]}/{k[1]}": v for k, v in r["seconds"].items()}}
        except Exception as exc:
            out["autotune_schur"] = {"error": str(exc)}
        P.set_schur_mode(True)                         # back to the defaults for what follows
        P.set_schur_tile(64)
    # Algorithm 4 variants
    for name, kw in (("gershgorin_multisection8", {"init": "gershgorin", "nshift": 8}),
                     ("stage3_f32_ir", {"solve_precision": "f32_ir"})):
        if name not in want:
            continue
        sync(); t0 = time.perf_counter()
        try:
            lam_v, _, rep = P.kth_eigenpair(p.k, want_vector=False, **kw)
        except Exception as exc:       # e.g. refinement that does not reach its tolerance
            out[name] = {"error": str(exc), "seconds": time.perf_counter() - t0,
                         "report": getattr(exc, "report", None)}
            continue
        t = time.perf_counter() - t0
        out[name] = {"time_to_lambda_k_s": t, "lambda_k": lam_v,
                     "n_factor": rep["n_factor"], "n_bisect": rep["n_bisect"], "n_si_iter": rep["n_si_iter"],
                     "init_interval": [rep["init_lo"], rep["init_hi"]], "t_stage": rep["t_stage"],
                     "n_refine": rep["n_refine"], "solve_berr": rep["solve_berr"],
                     "nu_interval": [rep["nu_lo"], rep["nu_hi"]], "rel_res": rep["rel_res"]}
        if kth:
            normA = float(np.abs(p.A()).sum(1).max())
            out[name]["lambda_diff_rel_to_bisection_run"] = abs(lam_v - kth["lambda_k"]) / normA
    if "hermitian_mid" in want:
        out["hermitian_mid"] = measure_hermitian(torch)
    return out


def measure_multisection_batch(torch, nshift: int = 8, reps: int = 2):
    """The multisection workload (n = 262,144, 32x16x16 cells, refined nested dissection): nshift
    shifts factored one after another (kep_factor each) against the same shifts in one
    kep_factor_multi call (all shifts' fronts in the same launches), best of reps, equal counts
    required."""
    import paper_1710_05134_gb300 as kep
    from gen import workload
    sync = torch.cuda.synchronize
    p = workload("batch")
    res = {"n": p.n, "shifts": nshift, "workload": "periodic diamond 32x16x16 cells, n=262,144"}
    sig = [0.30 + 0.011 * i for i in range(nshift)]
    with kep.Problem.from_pencil(p, refined_order=True) as P:
        res["flops_per_factorization"] = P.info.flops_factor
        P.factor(0.29)
        P.factor_multi(sig)                            # allocations of the batched path, untimed
        t_seq, t_multi = [], []
        for _ in range(reps):
            sync(); t0 = time.perf_counter()
            nu_seq = [P.factor(s).neg for s in sig]
            sync(); t_seq.append(time.perf_counter() - t0)
            sync(); t0 = time.perf_counter()
            nu_multi = [r.neg for r in P.factor_multi(sig)]
            sync(); t_multi.append(time.perf_counter() - t0)
        res.update(sequential_s=min(t_seq), batched_s=min(t_multi),
                   sequential_factorizations_per_s=nshift / min(t_seq),
                   batched_factorizations_per_s=nshift / min(t_multi),
                   speedup=min(t_seq) / min(t_multi), counts_equal=nu_seq == nu_multi, nu=nu_multi)
    return res


def measure_graph_replay(torch, reps: int = 5):
    """The n = 49,768 workload (where the pivot-step launches are latency-bound): factorizations
    with each level's step passes replayed as CUDA graphs against separate launches, best of
    reps each, equal counts required."""
    import paper_1710_05134_gb300 as kep
    from gen import workload
    sync = torch.cuda.synchronize
    p = workload("mid")
    sig = [0.30 + 0.013 * i for i in range(reps)]
    res = {"n": p.n, "factorizations": reps}
    with kep.Problem.from_pencil(p) as P:
        for mode in (False, True):
            P.set_graphs(mode)
            P.factor(0.29)                              # capture (graphs) / warm-up, untimed
            ts_, nus = [], []
            for s in sig:
                sync(); t0 = time.perf_counter()
                nus.append(P.factor(s).neg)
                sync(); ts_.append(time.perf_counter() - t0)
            res["graphs" if mode else "launches"] = {"best_s": min(ts_), "mean_s": sum(ts_) / len(ts_), "nu": nus}
        res["counts_equal"] = res["graphs"]["nu"] == res["launches"]["nu"]
        res["speedup"] = res["launches"]["best_s"] / res["graphs"]["best_s"]
    return res


def measure_fp32_factor(P, p, torch):
    """The reduced-precision factor (4-digit tensor-core splitting, FP32 tiles below order 512) +
    GMRES-refined solve against the FP64-accurate factor + plain solve, same shift and right-hand
    side; each with the normwise backward error ||b - M x||_inf / (||M||_inf ||x||_inf + ||b||_inf)
    of its solution (M = A - sigma B, products on the GPU)."""
    sync = torch.cuda.synchronize
    n = p.n
    sigma = float(shifts_for(p.k, 1)[0])
    rhs = np.random.default_rng(1).normal(size=n)
    nM = float(abs(p.A()).sum(1).max()) + abs(sigma) * float(abs(p.B()).sum(1).max())
    res = {"sigma": sigma}
    for mode in ("fp64_accurate", "fp32_refined"):
        P.set_schur_mode(True, fp32=(mode == "fp32_refined"))
        P.factor(sigma + 0.001)                        # warm-up (allocations, graphs)
        sync(); t0 = time.perf_counter()
        P.factor(sigma)
        sync(); tf = time.perf_counter() - t0
        t0 = time.perf_counter()
        if mode == "fp32_refined":
            try:
                xs, it, be = P.solve_refined(rhs, tol=1e-13)
            except Exception as exc:
                xs, it, be = None, None, str(exc)
        else:
            xs, it, be = P.solve(rhs), 0, None
        sync(); ts_ = time.perf_counter() - t0
        be_own = None
        if xs is not None:
            ax, bx = P.spmv(xs)
            r = rhs - (ax - sigma * bx)
            be_own = float(np.abs(r).max() / (nM * np.abs(xs).max() + np.abs(rhs).max()))
        res[mode] = {"factor_s": tf, "solve_s": ts_, "total_s": tf + ts_, "corrections": it,
                     "backward_error": be_own, "reported_backward_error": be}
    if isinstance(res["fp32_refined"].get("total_s"), float):
        res["speedup_same_backward_error"] = res["fp64_accurate"]["total_s"] / res["fp32_refined"]["total_s"]
    P.set_schur_mode(True)
    return res


def measure_two_in_flight(P, p, torch):
    """Four shifts factored one after another on one context, then two at a time on two contexts
    of the same pattern (own streams, own host threads): the latency-bound pivot kernels of one
    factorization overlap the tensor-core updates of the other."""
    import paper_1710_05134_gb300 as kep
    from paper_1710_05134_gb300 import multishift
    sync = torch.cuda.synchronize
    sig = [0.30 + 0.013 * i for i in range(4)]
    res = {"shifts": len(sig)}
    Q = None
    try:
        Q = kep.Problem.from_pencil(p)
        sq = torch.cuda.Stream()
        Q.set_stream(sq)
        Q.factor(0.29)                               # the second context's allocations, untimed
        sync(); t0 = time.perf_counter()
        nu_seq = [P.factor(s).neg for s in sig]
        sync(); res["sequential_s"] = time.perf_counter() - t0
        cc = multishift.ConcurrentCounter([lambda s: P.factor(s).neg, lambda s: Q.factor(s).neg])
        try:
            sync(); t0 = time.perf_counter()
            nu_con = cc.count_many(sig)
            sync(); res["two_in_flight_s"] = time.perf_counter() - t0
        finally:
            cc.close()
        res["speedup"] = res["sequential_s"] / res["two_in_flight_s"]
        res["counts_equal"] = nu_seq == nu_con
        res["nu"] = nu_con
    except Exception as exc:                         # e.g. the second context does not fit
        res["error"] = str(exc)
    finally:
        if Q is not None:
            Q.close()
    return res


def measure_precision(torch):
    """The mixed-precision workload (n = 1,500,000: 375,000 atoms, amorphous-like jitter 0.3 A,
    k = 0.3 n, refined nested dissection): Algorithm 4 with FP64-accurate stage-3 solves, then
    again with stage 3 on the reduced-precision factor and every shifted solve refined in FP64 to
    a backward error <= 1e-13.  Both runs draw the same start vectors, so stages 1-2 (the FP64
    inertia factorizations) take the same path; reported: the lambda_k difference relative to
    ||A||_inf, the angle between the two eigenvectors in the B inner product, and the speed-ups.
    A third run takes Algorithm 1' with the interpolating shift rule (FP64 solves)."""
    import paper_1710_05134_gb300 as kep
    from gen import workload
    p = workload("precision")
    normA = float(np.abs(p.A()).sum(1).max())
    res = {"workload": "precision", "n": p.n, "nnz": int(p.rowptr[-1]), "k": p.k,
           "desc": "periodic diamond 25x25x75 cells, 375,000 atoms, jitter 0.3 A, k = 0.3 n",
           "norm_A_inf": normA}
    t0 = time.perf_counter()
    with kep.Problem.from_pencil(p, refined_order=True) as P:
        res["analyze_s"] = time.perf_counter() - t0
        inf = P.info
        res.update(max_front=inf.max_front, flops_per_factorization=inf.flops_factor,
                   slot_gb=inf.slot_bytes / 1e9)
        xs = {}
        runs = {"f64": {}, "f32_ir": {"solve_precision": "f32_ir"}, "f64_interp": {"split": "interp"}}
        for mode, kw in runs.items():
            torch.cuda.synchronize(); t0 = time.perf_counter()
            try:
                lam, x, rep = P.kth_eigenpair(p.k, **kw)
            except Exception as exc:
                res[mode] = {"error": str(exc), "seconds": time.perf_counter() - t0}
                continue
            torch.cuda.synchronize()
            res[mode] = {"time_to_lambda_k_s": time.perf_counter() - t0, "lambda_k": lam,
                         "rel_res": rep["rel_res"], "n_factor": rep["n_factor"],
                         "n_si_iter": rep["n_si_iter"], "t_stage": rep["t_stage"],
                         "n_refine": rep["n_refine"], "solve_berr": rep["solve_berr"],
                         "n_bisect": rep["n_bisect"]}
            xs[mode] = x
        a, b = res.get("f64", {}), res.get("f32_ir", {})
        if "lambda_k" in a and "lambda_k" in b:
            _, bx = P.spmv(xs["f32_ir"])
            cos = abs(float(np.dot(xs["f64"], bx)))    # both B-normalised
            res.update(lambda_err_rel=abs(a["lambda_k"] - b["lambda_k"]) / normA,
                       eigvec_sin_angle_B=float(np.sqrt(max(0.0, 1.0 - min(cos, 1.0) ** 2))),
                       speedup_total=a["time_to_lambda_k_s"] / b["time_to_lambda_k_s"],
                       speedup_stage3=a["t_stage"][2] / b["t_stage"][2])
        c = res.get("f64_interp", {})
        if "lambda_k" in a and "lambda_k" in c:
            res.update(interp_lambda_diff_rel=abs(a["lambda_k"] - c["lambda_k"]) / normA,
                       interp_speedup_total=a["time_to_lambda_k_s"] / c["time_to_lambda_k_s"])
    return res


def measure_hermitian(torch, name: str = "mid_peierls", refined: bool = False):
    """A complex Hermitian pencil (the generator with Peierls phases on every atom pair: n = 49,768
    for mid_peierls, n = 524,288 for scale_peierls, the differentiation workload), through the
    real embedding of order 2n (each complex variable's two rows ordered together): analysis,
    factorization, Algorithm 4 and the complex derivatives."""
    import paper_1710_05134_gb300 as kep
    from gen import workload
    sync = torch.cuda.synchronize
    ph = workload(name)
    res = {"workload": name, "n": ph.n, "nnz": int(ph.rowptr[-1]), "k": ph.k,
           "ordering": "refined" if refined else "default"}
    t0 = time.perf_counter()
    with kep.Problem.from_pencil(ph, refined_order=refined) as H:
        res["analyze_s"] = time.perf_counter() - t0
        inf = H.info
        res.update(embedding_n=inf.n, max_front=inf.max_front, flops_per_factorization=inf.flops_factor)
        H.factor(0.31)
        sync(); t0 = time.perf_counter()
        nus = [H.factor(0.30 + 0.013 * i).neg for i in range(3)]
        sync(); res["factor_s"] = (time.perf_counter() - t0) / 3
        res["nu"] = nus
        res["device_free_gb_before_kth"] = torch.cuda.mem_get_info()[0] / 1e9
        t0 = time.perf_counter()
        try:
            lam, x, rep = H.kth_eigenpair(ph.k)
        except Exception as exc:
            res["kth_error"] = str(exc)
            res["storage_replans"] = H.info.replans
            return res
        res.update(time_to_lambda_k_s=time.perf_counter() - t0, lambda_k=lam, rel_res=rep["rel_res"],
                   n_factor=rep["n_factor"], n_si_iter=rep["n_si_iter"], t_stage=rep["t_stage"],
                   storage_replans=H.info.replans)
        xd = torch.from_numpy(x).cuda()
        H.grad(lam, xd)
        sync(); t0 = time.perf_counter()
        H.grad(lam, xd)
        sync(); res["grad_ms"] = 1e3 * (time.perf_counter() - t0)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kep", choices=["kep", "reference"])
    ap.add_argument("--workload", default="million", choices=["scale", "million", "mid", "small"])
    ap.add_argument("--ordering", default="refined", choices=["refined", "default"],
                    help="nested dissection of the timed analysis: refined (minimum-vertex-cover separators, "
                         "less fill) or default")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="wall time of the cpu_baseline run")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end leg (at most --steps)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-kth", action="store_true", help="skip Algorithm 4 (time to lambda_k)")
    ap.add_argument("--no-kth-interp", action="store_true",
                    help="skip the second Algorithm 4 run with the interpolating shift rule")
    ap.add_argument("--no-validate", action="store_true", help="skip the second-ordering count check")
    ap.add_argument("--variants", nargs="?", const="all", default=None,
                    help="also measure the next rows (all, or a comma list of: " + ", ".join(VARIANTS + SEPARATE_VARIANTS) + ")")
    ap.add_argument("--event-timing", type=int, default=1,
                    help="bracket the roofline kernels' launches with CUDA events (1) or not (0)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1710_05134_gb300 as kep
    from paper_1710_05134_gb300 import multishift

    rank, world, local = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1), _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    refined = args.ordering == "refined"
    fp64_peak = measure_fp64_peak(torch)
    p = make_workload(args.workload)
    t0 = time.perf_counter()
    P = kep.Problem.from_pencil(p, refined_order=refined)
    t_analyze = time.perf_counter() - t0
    info = P.info
    stream = torch.cuda.Stream()
    P.set_stream(stream)
    n = p.n
    gen = torch.Generator(device="cuda").manual_seed(1234 + rank)
    b = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
    x = torch.empty_like(b)
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    # each rank factors its own shifts (round-robin over one sequence): independent units, no
    # collective on the data path; the sequence increases, so each rank's counts must not decrease
    shifts = multishift.shard(shifts_for(p.k, world * (args.warmup + args.steps + e2e_steps + 2)), rank, world)

    nus = []

    def step(i):
        r = P.factor(shifts[i])
        nus.append(r.neg)
        P.solve(b, out=x)
        P.spmv(x)

    warm = None
    for i in range(args.warmup):
        last = i == args.warmup - 1
        if last:                       # per-class breakdown from the last warm-up step
            P.timing(reset=True)
            P.set_timing(True)
        step(i)
        if last:
            warm = P.timing(reset=True)
            P.set_timing(False)
    torch.cuda.synchronize()
    if warm is None:
        warm = P.timing(reset=True)
    warm_classes = {k: v for k, v in warm.items() if k not in ("total_launches", "flops")}
    dom = max(warm_classes, key=lambda k: warm_classes[k][1])

    # the timed region brackets only the roofline kernels' launches with events (events around
    # every launch would add their own cost to the step)
    P.timing(reset=True)
    P.set_timing(bool(args.event_timing), classes=sorted({dom, "update", "flush_tc"}))
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    w0 = time.perf_counter()
    for i in range(args.steps):
        step(args.warmup + i)
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - w0
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    timing = P.timing(reset=True)
    P.set_timing(False)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    value = world * args.steps / (ms / 1e3)
    timed_shifts = shifts[args.warmup:args.warmup + args.steps]
    timed_nus = nus[args.warmup:args.warmup + args.steps]

    # end to end through the public API with host buffers: copies inside the timed region
    e2e = None
    if not args.no_e2e:
        bh = torch.empty(n, dtype=torch.float64, pin_memory=True).copy_(b.cpu()).numpy()
        xh = np.empty(n)
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for i in range(e2e_steps):
            P.factor(shifts[args.warmup + args.steps + i])
            P.solve(bh, out=xh)
            P.spmv(xh)
        et = time.perf_counter() - e0
        if dist:
            t = torch.tensor([et], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            et = float(t.item())
        e2e = {"value": world * e2e_steps / et, "unit": UNIT, "steps": e2e_steps,
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 3 * 8 * n + 32,
               "path": "Problem.factor + Problem.solve (pageable host rhs in, x out) + Problem.spmv "
                       "(host x in, A x and B x out) through the C ABI"}

    # roofline of the dominant kernel class (dominant in the last warm-up step; its launches in
    # the timed region are event-timed)
    peaks = _measured_peaks()
    classes = {k: v for k, v in timing.items() if k not in ("total_launches", "flops")}
    fl = timing["flops"]
    roofline, rooflines = None, {}
    if classes["update"][1] > 0 and fl["update"] > 0:
        a = fl["update"] / (classes["update"][1] / 1e3)
        rooflines["update"] = {"bound": "alu", "kernel": "lf_schur_kernel (FP64 FMA tiles)",
                               "achieved": a / 1e12, "peak": fp64_peak / 1e12, "unit": "TFLOP/s",
                               "frac": a / fp64_peak,
                               "peak_source": "measured in this run: cuBLAS DGEMM 8192^3 (torch.mm), best of 3",
                               "peak_derived_tflops": FP64_PEAK_DERIVED / 1e12,
                               "launches": classes["update"][0], "kernel_ms": classes["update"][1]}
    if classes["flush_tc"][1] > 0 and fl["flush_tc"] > 0:
        sec = classes["flush_tc"][1] / 1e3
        pk, src = peaks["bf16_sustained"]
        method = fl["flush_fp64_equivalent"] / sec          # the FP64 update work carried out
        issued = fl["flush_tc"] / sec                       # bf16 products issued (36 per FP64 FMA)
        rooflines["flush_tc"] = {
            "bound": "tensor", "kernel": "lf_flush_tc_kernel (tcgen05 bf16, exact splitting of FP64)",
            "achieved": method / 1e12, "peak": pk / 1e12, "unit": "TFLOP/s", "frac": method / pk,
            "achieved_is": "the Schur-update flops of the method (2 per FP64 multiply-add) per second of the "
                           "kernel's launches",
            "peak_source": src + " (the kernel's own dtype)",
            "issued_bf16_tflops": issued / 1e12, "frac_issued_bf16": issued / pk,
            "fp64_peak_ratio": method / fp64_peak,
            "traffic_note": "DRAM bytes per launch scaled from ncu at n=49,768 (all 832 flush launches of one "
                            "factorization: 0.04496 B per FP64-equivalent flop) by this run's flops per launch",
            "launches": classes["flush_tc"][0], "kernel_ms": classes["flush_tc"][1]}
    if "flush_tc" in rooflines and classes["flush_tc"][0] > 0:
        rooflines["flush_tc"]["traffic"] = FLUSH_DRAM_BYTES_PER_FP64_FLOP * fl["flush_fp64_equivalent"] / classes["flush_tc"][0]
        rooflines["flush_tc"]["algorithmic_flops_per_launch"] = fl["flush_fp64_equivalent"] / classes["flush_tc"][0]
    roofline = rooflines.get(dom)
    if roofline is not None:
        roofline = dict(roofline)
        roofline.setdefault("traffic", None)
        roofline["share_of_step"] = roofline["kernel_ms"] / ms if ms > 0 else None
        roofline["class"] = dom

    kth = None
    if not args.no_kth and rank == 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            lam, xk, rep = P.kth_eigenpair(p.k)
            t_kth = time.perf_counter() - t0
            P._last_x = xk
            kth = {"time_to_lambda_k_s": t_kth, "k": p.k, "lambda_k": lam, "report": rep}
        except Exception as exc:
            kth = {"error": str(exc), "seconds": time.perf_counter() - t0,
                   "report": getattr(exc, "report", None)}
        # the same run with Algorithm 1''s interpolating shift rule (the root-finder variant the
        # paper proposes): same start vectors, so stage 1 is the same; lambda_k must agree
        if not args.no_kth_interp:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                lam_i, _, rep_i = P.kth_eigenpair(p.k, split="interp", want_vector=False)
                kth_i = {"time_to_lambda_k_s": time.perf_counter() - t0, "lambda_k": lam_i, "report": rep_i}
                if "lambda_k" in kth:
                    kth_i["lambda_diff_rel"] = abs(lam_i - kth["lambda_k"]) / float(np.abs(p.A()).sum(1).max())
            except Exception as exc:
                kth_i = {"error": str(exc), "seconds": time.perf_counter() - t0,
                         "report": getattr(exc, "report", None)}
            kth["split_interp"] = kth_i

    variants = None
    if args.variants and rank == 0:
        variants = measure_variants(P, p, torch, kth, args.variants)

    # validation of the timed counts: nu is non-decreasing in sigma, and a second analysis with the
    # other nested dissection (other fronts, pivots and update batches) gives the same count at the
    # first and last timed shift (Sylvester's law)
    validation = {"monotone": all(a <= b2 for a, b2 in zip(timed_nus, timed_nus[1:]))}
    P.close()
    if not args.no_validate:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        other = "default" if refined else "refined"
        check = sorted({0, len(timed_shifts) - 1})
        with kep.Problem.from_pencil(p, refined_order=not refined) as Q:
            got = [Q.factor(timed_shifts[i]).neg for i in check]
        want = [timed_nus[i] for i in check]
        validation.update({"second_ordering": other, "shifts": [timed_shifts[i] for i in check],
                           "nu_timed": want, "nu_second": got, "equal": got == want,
                           "seconds": time.perf_counter() - t0})
    validation["ok"] = validation["monotone"] and validation.get("equal", True)
    if args.variants and rank == 0:
        sep = [v for v in SEPARATE_VARIANTS if v not in EXPLICIT_VARIANTS] if args.variants == "all" else \
            [v for v in args.variants.split(",") if v in SEPARATE_VARIANTS]
        variants = variants or {}
        for name in sep:
            try:
                if name == "multisection_batch":
                    variants[name] = measure_multisection_batch(torch)
                elif name == "graph_replay":
                    variants[name] = measure_graph_replay(torch)
                elif name == "precision_full":
                    variants[name] = measure_precision(torch)
                else:
                    variants[name] = measure_hermitian(torch, "scale_peierls", refined=True)
            except Exception as exc:
                variants[name] = {"error": str(exc)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ps = _cpu_sample_pencil()
        ratio = flops_of(ps) / (info.flops_factor if not refined else flops_of(p))
        ps, done, cwall, cores = cpu_oracle_run(args.cpu_seconds)
        cpu_val = done / cwall * ratio
        cpu = {"value": cpu_val, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": cpu_sample_desc(ps, done, cwall, cores, ratio, n)}

    if rank == 0:
        line = {"metric": metric_for(args.workload), "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "desc": WORKLOAD_DESC.get(args.workload), "n": n,
                           "nnz": int(info.nnz), "k": p.k, "fronts": int(info.nfronts),
                           "max_front": int(info.max_front), "nnz_factor": int(info.nnz_factor),
                           "flops_per_factorization": info.flops_factor,
                           "step": "factor(A - sigma B) + solve + A/B SpMV, new sigma each step",
                           "l2": "inputs larger than L2 (front storage %.1f GB)" % (info.front_bytes / 1e9),
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "analyze_s": t_analyze, "wall_s": wall,
                           "ordering": ("refined nested dissection (minimum-vertex-cover separators)" if refined
                                        else "nested dissection"),
                           "event_timing": bool(args.event_timing),
                           "shifts": timed_shifts, "nu": timed_nus},
                "clocks": clocks, "e2e": e2e, "gpu_launches": timing["total_launches"],
                "roofline": roofline, "rooflines": rooflines, "cpu_baseline": cpu,
                "nu_validation": validation,
                "fp64_peak_measured_tflops": fp64_peak / 1e12,
                "factorization_fp64_equivalent_tflops": info.flops_factor * args.steps / (ms / 1e3) / 1e12,
                "kernels_ms_warmup_step": {k: v[1] for k, v in warm_classes.items()},
                "kernels_launches_warmup_step": {k: v[0] for k, v in warm_classes.items()},
                "kernels_ms_timed": {k: v[1] for k, v in classes.items() if v[1] > 0}}
        if kth is not None:
            line["time_to_lambda_k"] = kth
        if variants is not None:
            line["variants"] = variants
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
