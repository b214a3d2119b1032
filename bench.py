#!/usr/bin/env python
"""Benchmark: inertia-validated factorizations per second on the synthetic tight-binding workload.

A step is one pass of the whole hot path on the GPU: numeric LDL^T of A - sigma*B (assembly,
extend-add, Bunch-Kaufman pivoting, Schur updates, inertia reduction), one solve with the factor,
and one A/B sparse product.  Every step uses a new shift.  The default workload is the
n = 524,288 periodic diamond pencil with 11 % vacancies (32x32x18 cells, 16,384 sites removed).

Prints one JSON line (rank 0).  --impl reference times the CPU oracle instead (bounded sample).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "inertia-validated factorizations/s (n=524,288 tight-binding pencil)"
WORKLOAD_N = {"scale": "524,288", "million": "1,048,576", "mid": "49,768", "small": "2,048"}


def metric_for(workload: str) -> str:
    return f"inertia-validated factorizations/s (n={WORKLOAD_N[workload]} tight-binding pencil)"
UNIT = "factorizations/s"
# FP64 FMA issue rate of GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (max SM clock).
FP64_PEAK_DERIVED = 152 * 2 * 2 * 2.07e9
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
    """bf16 peaks (FLOP/s) from MEASURED_PEAKS.json when present, else the fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"bf16": (d["bf16_tflops"] * 1e12, "measured (MEASURED_PEAKS.json bf16_tflops, burst)"),
                "bf16_sustained": (d["bf16_tflops_sustained"] * 1e12,
                                   "measured (MEASURED_PEAKS.json bf16_tflops_sustained)")}
    except (OSError, KeyError, ValueError):
        return {"bf16": (1.9e15, "fallback 1.9 PFLOP/s bf16 burst"),
                "bf16_sustained": (1.7e15, "fallback 1.7 PFLOP/s bf16 sustained")}


def flops_of(p, refined: bool = False) -> float:
    """Symbolic factorization flops of the GPU plan for pencil p (host analysis only, no device)."""
    import paper_1710_05134_gb300 as kep
    return kep.symbolic_info(p.n, p.rowptr, p.colind, p.coords, refined_order=refined).flops_factor


def cpu_oracle_sample(reps: int = 1):
    """Time the oracle's sparse LDL^T (c3, single thread, as it stands) on the sample pencil."""
    from gen import make_pair
    from oracle import core
    s = CPU_SAMPLE
    p = make_pair(s["nx"], s["ny"], s["nz"], seed=0, vacancies=s["vacancies"])
    core.sparse_inertia(p.rowptr, p.colind, p.a, p.b, 1.0, -0.3)   # compile/load outside timing
    times = []
    for i in range(reps):
        t0 = time.perf_counter()
        core.sparse_inertia(p.rowptr, p.colind, p.a, p.b, 1.0, -(0.30 + 0.013 * i))
        times.append(time.perf_counter() - t0)
    return p, times


def run_reference(args):
    """The CPU oracle timed on the host cores: each step factors the bounded sample once."""
    rank = _env_int("RANK", 0)
    if rank != 0:
        return 0
    from gen import make_pair
    from oracle import core
    s = CPU_SAMPLE
    p = make_pair(s["nx"], s["ny"], s["nz"], seed=0, vacancies=s["vacancies"])
    full = make_workload(args.workload)
    ratio = flops_of(p) / flops_of(full)
    for i in range(args.warmup):
        core.sparse_inertia(p.rowptr, p.colind, p.a, p.b, 1.0, -(0.30 + 0.013 * i))
    t0 = time.perf_counter()
    for i in range(args.steps):
        core.sparse_inertia(p.rowptr, p.colind, p.a, p.b, 1.0, -(0.30 + 0.013 * i))
    dt = time.perf_counter() - t0
    value = args.steps / dt * ratio
    sample = (f"oracle sparse LDL^T (c3) on the same generator at {s['nx']}x{s['ny']}x{s['nz']} cells "
              f"(n={p.n}), {args.steps} factorizations in {dt:.2f} s, scaled to the full workload by the "
              f"GPU plan's flop ratio {ratio:.3e}")
    line = {"impl": "reference", "metric": metric_for(args.workload), "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps / 1.0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "desc": WORKLOAD_DESC.get(args.workload)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


VARIANTS = ("grad", "fp32_factor_ir", "two_shifts_in_flight", "autotune_min_front", "gershgorin_multisection8",
            "stage3_f32_ir", "hermitian_mid")


def measure_variants(P, p, torch, kth, which="all"):
    """Timings of the next rows on the same problem (device-synchronised wall clock)."""
    want = set(VARIANTS) if which == "all" else set(which.split(","))
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
    if "autotune_min_front" in want:
        from paper_1710_05134_gb300 import tune
        try:
            out["autotune_min_front"] = tune.tune_min_front(P, [0.31, 0.33], sync=sync)
        except Exception as exc:
            out["autotune_min_front"] = {"error": str(exc)}
        P.set_schur_mode(True)                         # back to the default for what follows
    # Algorithm 4 variants
    for name, kw in (("gershgorin_multisection8", {"init": "gershgorin", "nshift": 8}),
                     ("stage3_f32_ir", {"solve_precision": "f32_ir"})):
        if name not in want:
            continue
        sync(); t0 = time.perf_counter()
        try:
            lam_v, _, rep = P.kth_eigenpair(p.k, want_vector=False, **kw)
        except Exception as exc:       # e.g. refinement that does not reach its tolerance
            out[name] = {"error": str(exc), "seconds": time.perf_counter() - t0}
            continue
        t = time.perf_counter() - t0
        out[name] = {"time_to_lambda_k_s": t, "lambda_k": lam_v,
                     "n_factor": rep["n_factor"], "n_bisect": rep["n_bisect"], "n_si_iter": rep["n_si_iter"],
                     "init_interval": [rep["init_lo"], rep["init_hi"]], "t_stage": rep["t_stage"],
                     "n_refine": rep["n_refine"], "solve_berr": rep["solve_berr"]}
    if "hermitian_mid" in want:
        out["hermitian_mid"] = measure_hermitian(torch)
    return out


def measure_fp32_factor(P, p, torch):
    """FP32 factor + refined solve against the FP64-accurate factor + plain solve, same shift."""
    sync = torch.cuda.synchronize
    n = p.n
    sigma = float(shifts_for(p.k, 1)[0])
    rhs = np.random.default_rng(1).normal(size=n)
    res = {}
    for mode in ("fp64_accurate", "fp32_refined"):
        P.set_schur_mode(True, fp32=(mode == "fp32_refined"))
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
        res[mode] = {"factor_s": tf, "solve_s": ts_, "corrections": it, "backward_error": be}
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


def measure_hermitian(torch):
    """A complex Hermitian pencil (the n = 49,768 generator with Peierls phases on every atom
    pair), through the real embedding of order 2n: analysis, factorization, Algorithm 4 and the
    complex derivatives."""
    import paper_1710_05134_gb300 as kep
    from gen import workload
    sync = torch.cuda.synchronize
    ph = workload("mid_peierls")
    res = {"n": ph.n, "nnz": int(ph.rowptr[-1]), "k": ph.k}
    t0 = time.perf_counter()
    with kep.Problem.from_pencil(ph) as H:
        res["analyze_s"] = time.perf_counter() - t0
        inf = H.info
        res.update(embedding_n=inf.n, max_front=inf.max_front, flops_per_factorization=inf.flops_factor)
        H.factor(0.31)
        sync(); t0 = time.perf_counter()
        nus = [H.factor(0.30 + 0.013 * i).neg for i in range(3)]
        sync(); res["factor_s"] = (time.perf_counter() - t0) / 3
        res["nu"] = nus
        t0 = time.perf_counter()
        try:
            lam, x, rep = H.kth_eigenpair(ph.k)
        except Exception as exc:
            res["kth_error"] = str(exc)
            return res
        res.update(time_to_lambda_k_s=time.perf_counter() - t0, lambda_k=lam, rel_res=rep["rel_res"],
                   n_factor=rep["n_factor"], n_si_iter=rep["n_si_iter"])
        xd = torch.from_numpy(x).cuda()
        H.grad(lam, xd)
        sync(); t0 = time.perf_counter()
        H.grad(lam, xd)
        sync(); res["grad_ms"] = 1e3 * (time.perf_counter() - t0)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="kep", choices=["kep", "reference"])
    ap.add_argument("--workload", default="scale", choices=["scale", "million", "mid", "small"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--refined-order", action="store_true",
                    help="analyse with the refined nested dissection (minimum-vertex-cover separators)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kth", action="store_true",
                    help="also run Algorithm 4 once (k = n/2) and report the time to lambda_k")
    ap.add_argument("--variants", nargs="?", const="all", default=None,
                    help="also measure the next rows (all, or a comma list of: " + ", ".join(VARIANTS) + ")")
    ap.add_argument("--event-timing", type=int, default=1,
                    help="bracket every launch with CUDA events for the per-kernel roofline (1) or not (0)")
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

    p = make_workload(args.workload)
    t0 = time.perf_counter()
    P = kep.Problem.from_pencil(p, refined_order=args.refined_order)
    t_analyze = time.perf_counter() - t0
    info = P.info
    stream = torch.cuda.Stream()
    P.set_stream(stream)
    n = p.n
    gen = torch.Generator(device="cuda").manual_seed(1234 + rank)
    b = torch.randn(n, dtype=torch.float64, device="cuda", generator=gen)
    x = torch.empty_like(b)
    # each rank factors its own shifts (round-robin over one sequence): independent units, no
    # collective on the data path
    shifts = multishift.shard(shifts_for(p.k, world * (args.warmup + 2 * args.steps + 8)), rank, world)

    nus = []

    def step(i):
        r = P.factor(shifts[i])
        nus.append(r.neg)
        P.solve(b, out=x)
        P.spmv(x)

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

    # end to end through the public API with host buffers: copies inside the timed region
    e2e = None
    if not args.no_e2e:
        bh = torch.empty(n, dtype=torch.float64, pin_memory=True).copy_(b.cpu()).numpy()
        xh = np.empty(n)
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        for i in range(args.steps):
            P.factor(shifts[args.warmup + args.steps + i])
            P.solve(bh, out=xh)
            P.spmv(xh)
        et = time.perf_counter() - e0
        if dist:
            t = torch.tensor([et], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            et = float(t.item())
        e2e = {"value": world * args.steps / et, "unit": UNIT,
               "h2d_bytes_per_step": 2 * 8 * n,
               "d2h_bytes_per_step": 3 * 8 * n + 32}

    # roofline of the dominant kernel class (dominant in the last warm-up step; its launches in
    # the timed region are event-timed)
    peaks = _measured_peaks()
    classes = {k: v for k, v in timing.items() if k not in ("total_launches", "flops")}
    fl = timing["flops"]
    roofline, rooflines = None, {}
    if classes["update"][1] > 0 and fl["update"] > 0:
        a = fl["update"] / (classes["update"][1] / 1e3)
        rooflines["update"] = {"bound": "alu", "kernel": "lf_schur_kernel (FP64 FMA tiles)",
                               "achieved": a / 1e12, "peak": FP64_PEAK_DERIVED / 1e12, "unit": "TFLOP/s",
                               "frac": a / FP64_PEAK_DERIVED,
                               "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz",
                               "launches": classes["update"][0], "kernel_ms": classes["update"][1]}
    if classes["flush_tc"][1] > 0 and fl["flush_tc"] > 0:
        a = fl["flush_tc"] / (classes["flush_tc"][1] / 1e3)
        pk, src = peaks["bf16_sustained"]
        rooflines["flush_tc"] = {"bound": "tensor", "kernel": "lf_flush_tc_kernel (tcgen05 bf16, exact splitting)",
                                 "achieved": a / 1e12, "peak": pk / 1e12, "unit": "TFLOP/s", "frac": a / pk,
                                 "peak_source": src, "launches": classes["flush_tc"][0],
                                 "kernel_ms": classes["flush_tc"][1],
                                 "fp64_equivalent_tflops": fl["flush_fp64_equivalent"] / (classes["flush_tc"][1] / 1e3) / 1e12}
    roofline = rooflines.get(dom)
    if roofline is not None:
        roofline = dict(roofline)
        roofline["traffic"] = None
        roofline["share_of_step"] = roofline["kernel_ms"] / ms if ms > 0 else None
        roofline["class"] = dom

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        ps, times = cpu_oracle_sample(reps=1)
        ratio = flops_of(ps, args.refined_order) / info.flops_factor
        cpu_val = (1.0 / min(times)) * ratio
        cpu = {"value": cpu_val, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": (f"oracle sparse LDL^T (c3, single thread) on the same generator at "
                          f"{CPU_SAMPLE['nx']}x{CPU_SAMPLE['ny']}x{CPU_SAMPLE['nz']} cells (n={ps.n}): "
                          f"{min(times):.2f} s per factorization, scaled to n={n} by the GPU plan's flop "
                          f"ratio {ratio:.3e}")}

    kth = None
    if args.kth and rank == 0:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lam, xk, rep = P.kth_eigenpair(p.k)
        t_kth = time.perf_counter() - t0
        P._last_x = xk
        kth = {"time_to_lambda_k_s": t_kth, "k": p.k, "lambda_k": lam, "report": rep}

    variants = None
    if args.variants and rank == 0:
        variants = measure_variants(P, p, torch, kth, args.variants)

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
                           "ordering": "refined nested dissection" if args.refined_order else "nested dissection",
                           "event_timing": bool(args.event_timing),
                           "nu": nus[args.warmup:args.warmup + args.steps]},
                "clocks": clocks, "e2e": e2e, "gpu_launches": timing["total_launches"],
                "roofline": roofline, "rooflines": rooflines, "cpu_baseline": cpu,
                "factorization_fp64_equivalent_tflops": info.flops_factor * args.steps / (ms / 1e3) / 1e12,
                "kernels_ms_warmup_step": {k: v[1] for k, v in warm_classes.items()},
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
