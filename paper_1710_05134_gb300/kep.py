"""Thin Python binding of the kep C ABI (include/kep.h): argument marshalling only.

Every computation runs in libkep.so's CUDA kernels.  If the library cannot be loaded this module
raises; there is no CPU fallback.  Vectors may be numpy arrays (host) or CUDA torch tensors
(device, float64, contiguous); device tensors are used in place on the context's stream.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

KEP_OK, KEP_ERR_INVALID, KEP_ERR_NOT_SPD, KEP_ERR_SINGULAR = 0, 1, 2, 3
KEP_ERR_NOT_CONVERGED, KEP_ERR_CLUSTER, KEP_ERR_POOL, KEP_ERR_TIMEOUT = 4, 5, 6, 7
KEP_ERR_CUDA, KEP_ERR_NONFINITE, KEP_ERR_NOMEM = 8, 9, 10
KEP_HOST, KEP_DEVICE = 0, 1
KEP_PATTERN_FULL, KEP_PATTERN_LOWER, KEP_ORDER_GRAPH, KEP_ORDER_REFINED = 0, 1, 2, 4

# symbols declared in include/kep.h
EXPORTED = ["kep_default_params", "kep_analyze", "kep_analyze_hermitian", "kep_get_info", "kep_symbolic_info", "kep_set_stream", "kep_factor",
            "kep_factor_pencil", "kep_solve", "kep_spmv", "kep_kth_eigenpair", "kep_set_timing",
            "kep_set_timing_classes", "kep_grad", "kep_set_values", "kep_factor_multi", "kep_solve_refined",
            "kep_get_timing", "kep_destroy", "kep_status_str", "kep_dense_inertia_noalloc",
            "kep_multisection_points", "kep_multisection_update", "kep_set_graphs",
            "kep_set_schur_mode", "kep_set_schur_tile", "kep_get_schur_config",
            "kep_interp_init", "kep_interp_point", "kep_interp_update"]
KEP_SCHUR_FP64, KEP_SCHUR_EMULATED = 0, 1
KEP_INIT_LANCZOS, KEP_INIT_GERSHGORIN = 0, 1
KEP_SOLVE_F64, KEP_SOLVE_F32_IR = 0, 1
KEP_BFACTOR_AUTO, KEP_BFACTOR_SHARED, KEP_BFACTOR_OWN = 0, 1, 2
KEP_SPLIT_BISECT, KEP_SPLIT_INTERP = 0, 1
KEP_SCHUR_FP32 = 2
KERNEL_CLASSES = ["assemble", "panel", "l21", "apply", "update", "reduce", "solve_fwd", "solve_bwd",
                  "perm", "spmv", "vec", "slice", "flush_tc"]


class KepError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {status_str(code)} (code {code})")


class Inertia(ctypes.Structure):
    _fields_ = [("neg", ctypes.c_int64), ("zero", ctypes.c_int64), ("pos", ctypes.c_int64),
                ("delayed", ctypes.c_int64)]

    def astuple(self):
        return (self.neg, self.zero, self.pos)


class Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nfronts", ctypes.c_int64),
                ("nlevels", ctypes.c_int64), ("max_front", ctypes.c_int64),
                ("nnz_factor", ctypes.c_int64), ("flops_factor", ctypes.c_double),
                ("front_bytes", ctypes.c_int64), ("replans", ctypes.c_int64),
                ("cb_bytes", ctypes.c_int64), ("slot_bytes", ctypes.c_int64)]


class Params(ctypes.Structure):
    _fields_ = [("m_max", ctypes.c_int64), ("tau_res", ctypes.c_double), ("tau_diff", ctypes.c_double),
                ("max_lanczos", ctypes.c_int64), ("max_si", ctypes.c_int64),
                ("start_vectors", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("init", ctypes.c_int32), ("nshift", ctypes.c_int32),
                ("solve_precision", ctypes.c_int32), ("b_factor", ctypes.c_int32),
                ("split", ctypes.c_int32)]


class InterpState(ctypes.Structure):
    """kep_interp_state: the interpolating shift rule's bracket, weights and safeguard."""
    _fields_ = [("lo", ctypes.c_double), ("hi", ctypes.c_double), ("nu_lo", ctypes.c_int64),
                ("nu_hi", ctypes.c_int64), ("w_lo", ctypes.c_double), ("w_hi", ctypes.c_double),
                ("width", ctypes.c_int64 * 4), ("nwidth", ctypes.c_int32), ("last", ctypes.c_int32),
                ("bisect_next", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Timing(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64 * 13), ("ms", ctypes.c_double * 13),
                ("flops", ctypes.c_double * 13), ("flush_fp64_equivalent_flops", ctypes.c_double),
                ("total_launches", ctypes.c_int64)]


class Report(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("eta", ctypes.c_double), ("rel_res", ctypes.c_double),
                ("rel_res_normwise", ctypes.c_double), ("sigma_lo", ctypes.c_double),
                ("sigma_hi", ctypes.c_double), ("nu_lo", ctypes.c_int64), ("nu_hi", ctypes.c_int64),
                ("init_lo", ctypes.c_double), ("init_hi", ctypes.c_double),
                ("init_nu_lo", ctypes.c_int64), ("init_nu_hi", ctypes.c_int64),
                ("n_factor", ctypes.c_int64), ("n_lanczos", ctypes.c_int64),
                ("n_bisect", ctypes.c_int64), ("n_si_iter", ctypes.c_int64),
                ("si_iter_bound", ctypes.c_int64), ("t_stage", ctypes.c_double * 3),
                ("n_refine", ctypes.c_int64), ("solve_berr", ctypes.c_double), ("cap_cols", ctypes.c_int64),
                ("last_res", ctypes.c_double), ("last_diff", ctypes.c_double), ("last_res_explicit", ctypes.c_double),
                ("restarted", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def asdict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "t_stage"}
        d["lambda"] = d.pop("lambda_")
        d["t_stage"] = list(self.t_stage)
        return d


_LIB = None


def lib() -> ctypes.CDLL:
    """Load (building if needed) libkep.so; raises if it cannot be built or loaded."""
    global _LIB
    if _LIB is None:
        path = _build.build()        # rebuilds when a source is newer than the library
        L = ctypes.CDLL(path)
        P, I64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
        L.kep_default_params.argtypes = [ctypes.POINTER(Params)]
        L.kep_default_params.restype = None
        L.kep_analyze.argtypes = [I64, P, P, P, P, I, P, ctypes.POINTER(P)]
        L.kep_analyze_hermitian.argtypes = [I64, P, P, P, P, I, P, ctypes.POINTER(P)]
        L.kep_get_info.argtypes = [P, ctypes.POINTER(Info)]
        L.kep_symbolic_info.argtypes = [I64, P, P, I, P, ctypes.POINTER(Info)]
        L.kep_set_stream.argtypes = [P, P]
        L.kep_factor.argtypes = [P, D, ctypes.POINTER(Inertia)]
        L.kep_factor_pencil.argtypes = [P, D, D, ctypes.POINTER(Inertia)]
        L.kep_solve.argtypes = [P, P, P, I64, I]
        L.kep_spmv.argtypes = [P, P, P, P, I]
        L.kep_kth_eigenpair.argtypes = [P, I64, ctypes.POINTER(Params), ctypes.POINTER(D), P,
                                        ctypes.POINTER(Report)]
        L.kep_set_timing.argtypes = [P, I]
        L.kep_set_timing_classes.argtypes = [P, ctypes.c_uint]
        L.kep_grad.argtypes = [P, D, P, D, P, P, I]
        L.kep_set_values.argtypes = [P, P, P]
        L.kep_factor_multi.argtypes = [P, P, ctypes.c_int32, P]
        L.kep_solve_refined.argtypes = [P, P, P, I, D, ctypes.c_int32, P, P]
        L.kep_get_timing.argtypes = [P, ctypes.POINTER(Timing), I]
        L.kep_dense_inertia_noalloc.argtypes = [I64, P, P, I64, D, P, P]
        L.kep_set_graphs.argtypes = [P, I]
        L.kep_multisection_points.argtypes = [D, D, ctypes.c_int32, P]
        L.kep_multisection_points.restype = I
        L.kep_multisection_update.argtypes = [I64, ctypes.c_int32, P, P, P, P, P, P]
        L.kep_multisection_update.restype = I
        L.kep_interp_init.argtypes = [I64, D, D, I64, I64, P]
        L.kep_interp_init.restype = I
        L.kep_interp_point.argtypes = [P, I64, I64, P]
        L.kep_interp_point.restype = I
        L.kep_interp_update.argtypes = [P, I64, D, I64]
        L.kep_interp_update.restype = I
        L.kep_dense_inertia_noalloc.restype = I
        L.kep_set_schur_mode.argtypes = [P, I, I64]
        L.kep_set_schur_mode.restype = I
        L.kep_set_schur_tile.argtypes = [P, I]
        L.kep_set_schur_tile.restype = I
        L.kep_get_schur_config.argtypes = [P, P, P, P]
        L.kep_get_schur_config.restype = I
        L.kep_destroy.argtypes = [P]
        L.kep_destroy.restype = None
        L.kep_status_str.argtypes = [I]
        L.kep_status_str.restype = ctypes.c_char_p
        for name in ["kep_analyze", "kep_analyze_hermitian", "kep_get_info", "kep_symbolic_info", "kep_set_stream", "kep_factor", "kep_factor_pencil",
                     "kep_solve", "kep_spmv", "kep_kth_eigenpair", "kep_set_timing", "kep_get_timing",
                     "kep_set_timing_classes", "kep_grad", "kep_set_values", "kep_factor_multi",
                     "kep_solve_refined"]:
            getattr(L, name).restype = I
        _LIB = L
    return _LIB


def multisection_points(lo: float, hi: float, nshift: int) -> list[float]:
    """The shifts of one Algorithm 1' step on [lo, hi) (kep_multisection_points; host only)."""
    out = (ctypes.c_double * max(1, int(nshift)))()
    _check(lib().kep_multisection_points(float(lo), float(hi), int(nshift), out), "kep_multisection_points")
    return [float(v) for v in out[:int(nshift)]]


def multisection_update(k: int, sigmas, nus, lo: float, hi: float, nu_lo: int, nu_hi: int):
    """The bracket update of one Algorithm 1' step (kep_multisection_update; host only):
    returns (lo, hi, nu_lo, nu_hi)."""
    cnt = len(sigmas)
    s = (ctypes.c_double * max(1, cnt))(*[float(v) for v in sigmas])
    v = (ctypes.c_int64 * max(1, cnt))(*[int(x) for x in nus])
    lo_, hi_ = ctypes.c_double(lo), ctypes.c_double(hi)
    nl_, nh_ = ctypes.c_int64(nu_lo), ctypes.c_int64(nu_hi)
    _check(lib().kep_multisection_update(int(k), cnt, s, v, ctypes.byref(lo_), ctypes.byref(hi_), ctypes.byref(nl_),
                                         ctypes.byref(nh_)), "kep_multisection_update")
    return lo_.value, hi_.value, nl_.value, nh_.value


def interp_init(k: int, lo: float, hi: float, nu_lo: int, nu_hi: int) -> InterpState:
    """A state of the interpolating shift rule for the bracket [lo, hi) of k (kep_interp_init;
    host only)."""
    st = InterpState()
    _check(lib().kep_interp_init(int(k), float(lo), float(hi), int(nu_lo), int(nu_hi), ctypes.byref(st)),
           "kep_interp_init")
    return st


def interp_point(st: InterpState, k: int, m_max: int) -> float:
    """The rule's next shift (kep_interp_point; host only)."""
    s = ctypes.c_double()
    _check(lib().kep_interp_point(ctypes.byref(st), int(k), int(m_max), ctypes.byref(s)), "kep_interp_point")
    return s.value


def interp_update(st: InterpState, k: int, sigma: float, nu: int) -> None:
    """Advance the rule with nu(sigma) (kep_interp_update; host only)."""
    _check(lib().kep_interp_update(ctypes.byref(st), int(k), float(sigma), int(nu)), "kep_interp_update")


def symbolic_info(n, rowptr, colind, coords=None, *, lower: bool = False, graph_order: bool = False,
                  refined_order: bool = False) -> Info:
    """The symbolic facts (#nzf, flop count, fronts) of a pattern, computed on the host only."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    cp = None
    if coords is not None:
        coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1)
        cp = coords.ctypes.data_as(ctypes.c_void_p)
    flags = ((KEP_PATTERN_LOWER if lower else KEP_PATTERN_FULL) | (KEP_ORDER_GRAPH if graph_order else 0)
             | (KEP_ORDER_REFINED if refined_order else 0))
    inf = Info()
    _check(lib().kep_symbolic_info(int(n), rowptr.ctypes.data, colind.ctypes.data, flags, cp, ctypes.byref(inf)),
           "kep_symbolic_info")
    return inf


def status_str(code: int) -> str:
    return lib().kep_status_str(code).decode()


def _check(code: int, where: str, ok=(KEP_OK,)):
    if code not in ok:
        raise KepError(code, where)
    return code


def _is_device(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _dev_ptr(x, complex_ok: bool = False) -> int:
    import torch
    ok = (torch.float64, torch.complex128) if complex_ok else (torch.float64,)
    if x.dtype not in ok or not x.is_contiguous():
        raise ValueError("device vectors must be contiguous float64 (complex128 for a Hermitian "
                         "pencil) CUDA tensors")
    return x.data_ptr()


@dataclass
class FactorResult:
    neg: int
    zero: int
    pos: int
    delayed: int
    status: int

    @property
    def nu(self) -> int:
        return self.neg


class Problem:
    """A pencil (A, B) analysed once (ordering, tree, maps) and factored for any shift.

    Complex values make it a Hermitian pencil (kep_analyze_hermitian): vectors, eigenvectors and
    derivatives are then complex128, and inertia counts are those of the complex pencil."""

    def __init__(self, n, rowptr, colind, a, b, coords=None, *, lower: bool = False,
                 graph_order: bool = False, refined_order: bool = False):
        L = lib()
        self.n = int(n)
        rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
        colind = np.ascontiguousarray(colind, dtype=np.int32)
        self.hermitian = bool(np.iscomplexobj(a) or np.iscomplexobj(b))
        self.vdtype = np.complex128 if self.hermitian else np.float64
        a = np.ascontiguousarray(a, dtype=self.vdtype)
        b = np.ascontiguousarray(b, dtype=self.vdtype)
        cp = None
        if coords is not None:
            coords = np.ascontiguousarray(coords, dtype=np.float64).reshape(-1)
            if coords.size != 3 * self.n:
                raise ValueError("coords must hold 3 values per row")
            cp = coords.ctypes.data_as(ctypes.c_void_p)
        flags = ((KEP_PATTERN_LOWER if lower else KEP_PATTERN_FULL) | (KEP_ORDER_GRAPH if graph_order else 0)
                 | (KEP_ORDER_REFINED if refined_order else 0))
        h = ctypes.c_void_p()
        fn, name = (L.kep_analyze_hermitian, "kep_analyze_hermitian") if self.hermitian else (L.kep_analyze, "kep_analyze")
        _check(fn(self.n, rowptr.ctypes.data, colind.ctypes.data, a.ctypes.data, b.ctypes.data, flags, cp,
                  ctypes.byref(h)), name)
        self._h = h
        self._stream = None
        self.nnz = int(rowptr[-1])

    def _dptr(self, x) -> int:
        return _dev_ptr(x, complex_ok=self.hermitian)

    def _host(self, x):
        return np.ascontiguousarray(x, dtype=self.vdtype)

    @classmethod
    def from_pencil(cls, p, **kw):
        return cls(p.n, p.rowptr, p.colind, p.a, p.b, p.coords, **kw)

    def close(self):
        if getattr(self, "_h", None):
            lib().kep_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def info(self) -> Info:
        inf = Info()
        _check(lib().kep_get_info(self._h, ctypes.byref(inf)), "kep_get_info")
        return inf

    def set_stream(self, stream):
        """Order the context's work on a torch.cuda.Stream (or a raw cudaStream_t int)."""
        handle = getattr(stream, "cuda_stream", stream)
        self._stream = stream
        _check(lib().kep_set_stream(self._h, ctypes.c_void_p(int(handle) if handle else 0)), "kep_set_stream")

    def set_schur_mode(self, emulated: bool, min_front: int = 512, *, fp32: bool = False):
        """Deferred Schur updates of fronts of order >= min_front on the tensor cores (FP64-accurate
        splitting) when emulated, else FP64 FMA everywhere; fp32: a reduced-precision factor for
        solve_refined (fronts of order >= min_front: 4-digit tensor-core splitting, smaller ones
        FP32 tiles)."""
        mode = KEP_SCHUR_FP32 if fp32 else (KEP_SCHUR_EMULATED if emulated else KEP_SCHUR_FP64)
        _check(lib().kep_set_schur_mode(self._h, mode, int(min_front)), "kep_set_schur_mode")

    def set_schur_tile(self, edge: int):
        """Edge (32 or 64) of the Schur tiles of fronts below the tensor-core threshold."""
        _check(lib().kep_set_schur_tile(self._h, int(edge)), "kep_set_schur_tile")

    def schur_config(self) -> dict:
        """{"mode": KEP_SCHUR_*, "min_front": tensor-core threshold, "tile": tile edge}."""
        mode, mf, tile = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
        _check(lib().kep_get_schur_config(self._h, ctypes.byref(mode), ctypes.byref(mf), ctypes.byref(tile)),
               "kep_get_schur_config")
        return {"mode": mode.value, "min_front": mf.value, "tile": tile.value}

    def solve_refined(self, rhs, tol: float = 1e-13, max_iter: int = 100):
        """(x, GMRES steps, backward error): GMRES-based iterative refinement preconditioned by the
        last factor, to a normwise backward error <= tol."""
        it = ctypes.c_int32()
        be = ctypes.c_double()
        if _is_device(rhs):
            import torch
            x = torch.empty_like(rhs)
            code = lib().kep_solve_refined(self._h, self._dptr(rhs), self._dptr(x), KEP_DEVICE, float(tol), int(max_iter),
                                           ctypes.byref(it), ctypes.byref(be))
        else:
            rhs = self._host(rhs)
            x = np.empty_like(rhs)
            code = lib().kep_solve_refined(self._h, rhs.ctypes.data, x.ctypes.data, KEP_HOST, float(tol), int(max_iter),
                                           ctypes.byref(it), ctypes.byref(be))
        _check(code, "kep_solve_refined")
        return x, it.value, be.value

    def set_graphs(self, enable: bool):
        """Replay each factorization level's pivot-step passes as CUDA graphs (default on)."""
        _check(lib().kep_set_graphs(self._h, 1 if enable else 0), "kep_set_graphs")

    def set_timing(self, enable: bool, classes=None):
        """Per-launch CUDA-event timing of this context's kernels (launch counts are always kept);
        classes: names from KERNEL_CLASSES to time (default: all)."""
        mask = 0xFFFFFFFF if classes is None else sum(1 << KERNEL_CLASSES.index(c) for c in classes)
        _check(lib().kep_set_timing_classes(self._h, mask), "kep_set_timing_classes")
        _check(lib().kep_set_timing(self._h, 1 if enable else 0), "kep_set_timing")

    def timing(self, reset: bool = False) -> dict:
        """{class: (launches, milliseconds)} since the last reset, plus 'total_launches' and
        'flops' ({class: device-counted algorithmic flops}, 'flush_fp64_equivalent')."""
        t = Timing()
        _check(lib().kep_get_timing(self._h, ctypes.byref(t), 1 if reset else 0), "kep_get_timing")
        d = {name: (int(t.launches[i]), float(t.ms[i])) for i, name in enumerate(KERNEL_CLASSES)}
        d["total_launches"] = int(t.total_launches)
        d["flops"] = {name: float(t.flops[i]) for i, name in enumerate(KERNEL_CLASSES)}
        d["flops"]["flush_fp64_equivalent"] = float(t.flush_fp64_equivalent_flops)
        return d

    def factor_multi(self, sigmas):
        """Inertia (neg, zero, pos, delayed) of A - sigma B for each shift of one multisection
        step; the factor of the last shift stays for solve()."""
        s = np.ascontiguousarray(sigmas, dtype=np.float64)
        out = (Inertia * s.size)()
        _check(lib().kep_factor_multi(self._h, s.ctypes.data, int(s.size), ctypes.byref(out)), "kep_factor_multi")
        return [FactorResult(o.neg, o.zero, o.pos, o.delayed, KEP_OK) for o in out]

    def set_values(self, a, b):
        """New values of A and B on the analysed pattern (same layout and dtype as at
        construction)."""
        a = self._host(a)
        b = self._host(b)
        if a.size != self.nnz or b.size != self.nnz:
            raise ValueError("values must match the analysed pattern")
        _check(lib().kep_set_values(self._h, a.ctypes.data, b.ctypes.data), "kep_set_values")

    def grad(self, lam: float, x, lam_bar: float = 1.0):
        """(d lambda / d a_vals, d lambda / d b_vals) in the layout of the analysed pattern
        (Hellmann-Feynman), times lam_bar; complex G_ij = lam_bar x_i conj(x_j) / x^H B x for a
        Hermitian pencil."""
        if _is_device(x):
            import torch
            ga = torch.empty(self.nnz, dtype=torch.complex128 if self.hermitian else torch.float64, device=x.device)
            gb = torch.empty_like(ga)
            _check(lib().kep_grad(self._h, float(lam), self._dptr(x), float(lam_bar), self._dptr(ga), self._dptr(gb),
                                  KEP_DEVICE), "kep_grad")
            return ga, gb
        x = self._host(x)
        ga, gb = np.empty(self.nnz, dtype=self.vdtype), np.empty(self.nnz, dtype=self.vdtype)
        _check(lib().kep_grad(self._h, float(lam), x.ctypes.data, float(lam_bar), ga.ctypes.data, gb.ctypes.data,
                              KEP_HOST), "kep_grad")
        return ga, gb

    def factor(self, sigma: float, *, allow_singular: bool = True) -> FactorResult:
        """LDL^T of A - sigma*B; .nu is the number of eigenvalues below sigma."""
        return self.factor_pencil(1.0, -float(sigma), allow_singular=allow_singular)

    def factor_pencil(self, ca: float, cb: float, *, allow_singular: bool = True) -> FactorResult:
        inr = Inertia()
        ok = (KEP_OK, KEP_ERR_SINGULAR) if allow_singular else (KEP_OK,)
        code = _check(lib().kep_factor_pencil(self._h, float(ca), float(cb), ctypes.byref(inr)),
                      "kep_factor_pencil", ok)
        return FactorResult(inr.neg, inr.zero, inr.pos, inr.delayed, code)

    def solve(self, rhs, out=None):
        """x = M^{-1} rhs with the last factorization; rhs of shape (n,) or (nrhs, n)."""
        if _is_device(rhs):
            import torch
            x = torch.empty_like(rhs) if out is None else out
            nrhs = 1 if rhs.dim() == 1 else rhs.shape[0]
            _check(lib().kep_solve(self._h, self._dptr(rhs), self._dptr(x), nrhs, KEP_DEVICE), "kep_solve")
            return x
        rhs = self._host(rhs)
        x = np.empty_like(rhs) if out is None else out
        nrhs = 1 if rhs.ndim == 1 else rhs.shape[0]
        _check(lib().kep_solve(self._h, rhs.ctypes.data, x.ctypes.data, nrhs, KEP_HOST), "kep_solve")
        return x

    def spmv(self, x):
        """(A x, B x)."""
        if _is_device(x):
            import torch
            ax, bx = torch.empty_like(x), torch.empty_like(x)
            _check(lib().kep_spmv(self._h, self._dptr(x), self._dptr(ax), self._dptr(bx), KEP_DEVICE), "kep_spmv")
            return ax, bx
        x = self._host(x)
        ax, bx = np.empty_like(x), np.empty_like(x)
        _check(lib().kep_spmv(self._h, x.ctypes.data, ax.ctypes.data, bx.ctypes.data, KEP_HOST), "kep_spmv")
        return ax, bx

    def kth_eigenpair(self, k: int, *, m_max: int = 20, tau_res: float = 1e-10, tau_diff: float = 1e-10,
                      max_lanczos: int = 200, max_si: int = 300, start_vectors=None, seed: int = 0x5eed,
                      want_vector: bool = True, init: str = "lanczos", nshift: int = 1,
                      solve_precision: str = "f64", b_factor: str = "auto", split: str = "bisect"):
        """Algorithm 4: (lambda_k, x_k (B-normalized), report dict).  init: "lanczos" (Algorithm 2)
        or "gershgorin" (an interval holding the whole spectrum); nshift: shifts per Algorithm 1'
        step (1 = bisection); b_factor: "auto", "shared" or "own" (where B's factor lives);
        split: "bisect" (the paper's Algorithm 1') or "interp" (the interpolating shift rule)."""
        prm = Params()
        lib().kep_default_params(ctypes.byref(prm))
        prm.m_max, prm.tau_res, prm.tau_diff = int(m_max), float(tau_res), float(tau_diff)
        prm.max_lanczos, prm.max_si, prm.seed = int(max_lanczos), int(max_si), int(seed)
        prm.init = {"lanczos": KEP_INIT_LANCZOS, "gershgorin": KEP_INIT_GERSHGORIN}[init]
        prm.nshift = int(nshift)
        prm.solve_precision = {"f64": KEP_SOLVE_F64, "f32_ir": KEP_SOLVE_F32_IR}[solve_precision]
        prm.b_factor = {"auto": KEP_BFACTOR_AUTO, "shared": KEP_BFACTOR_SHARED, "own": KEP_BFACTOR_OWN}[b_factor]
        prm.split = {"bisect": KEP_SPLIT_BISECT, "interp": KEP_SPLIT_INTERP}[split]
        sv = None
        if start_vectors is not None:
            sv = np.ascontiguousarray(start_vectors, dtype=np.float64).reshape(-1)
            nv = 2 * self.n if self.hermitian else self.n      # real vectors of the (embedded) pencil
            if sv.size != 2 * nv:
                raise ValueError(f"start_vectors must hold {2 * nv} values")
            prm.start_vectors = sv.ctypes.data
        lam = ctypes.c_double()
        x = np.empty(self.n, dtype=self.vdtype) if want_vector else None
        rep = Report()
        st = lib().kep_kth_eigenpair(self._h, int(k), ctypes.byref(prm), ctypes.byref(lam),
                                     x.ctypes.data if x is not None else None, ctypes.byref(rep))
        if st != KEP_OK:
            err = KepError(st, "kep_kth_eigenpair")
            err.report = rep.asdict()                  # what the stages reached
            raise err
        return lam.value, x, rep.asdict()


class KthEigenvalue:
    """lambda_k of A x = lambda B x as a differentiable function of the stored values of A and B
    (torch.autograd; gradients by the Hellmann-Feynman theorem through kep_grad).

        lam = KthEigenvalue.apply(problem, k, a_vals, b_vals)

    a_vals, b_vals: float64 tensors (complex128 for a Hermitian problem) in the layout of the
    problem's pattern; the forward pass loads them with set_values and runs Algorithm 4 (kwargs of
    kth_eigenpair via problem.kth_kwargs).  For complex values the gradient is
    d lambda / d Re + i d lambda / d Im of each stored entry (PyTorch's convention for a real
    output)."""

    @staticmethod
    def _fn():
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(ctx, problem, k, a_vals, b_vals):
                problem.set_values(a_vals.detach().cpu().numpy(), b_vals.detach().cpu().numpy())
                lam, x, _ = problem.kth_eigenpair(int(k), **getattr(problem, "kth_kwargs", {}))
                ctx.problem, ctx.lam, ctx.x = problem, lam, x
                return torch.tensor(lam, dtype=torch.float64, device=a_vals.device)

            @staticmethod
            def backward(ctx, lam_bar):
                ga, gb = ctx.problem.grad(ctx.lam, ctx.x, float(lam_bar))
                dev = lam_bar.device
                return (None, None, torch.from_numpy(ga).to(dev), torch.from_numpy(gb).to(dev))

        return _F

    @classmethod
    def apply(cls, problem, k, a_vals, b_vals):
        return cls._fn().apply(problem, k, a_vals, b_vals)
