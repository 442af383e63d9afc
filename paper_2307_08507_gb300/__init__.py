"""Python binding of libmdot, the GB300 (sm_103a) MDOT-PNCG library (include/mdot.h).

Argument marshalling only: every step of the solve runs in the library's CUDA kernels.  Device
arrays are torch CUDA tensors (torch provides device memory and the stream); host arrays for
``solve_host`` are numpy arrays.  The library must have been built (``build.build()``); importing
the binding never falls back to anything else.
"""
from __future__ import annotations

import ctypes as ct
import os
from dataclasses import dataclass

from . import build as _build

__all__ = ["Params", "Info", "Handle", "lib", "MDOT_OK", "status_string", "MdotError"]

MDOT_OK = 0
MDOT_ERR_INVALID_ARG = 1
MDOT_ERR_NOT_CONVERGED = 2
MDOT_ERR_NUMERIC = 3
MDOT_ERR_TIMEOUT = 4
MDOT_ERR_OOM = 5
MDOT_ERR_CUDA = 6
PREC_AUTO, PREC_FP32, PREC_FP64, PREC_FP32A = 0, 1, 2, 3
PREC_TENSOR_CORES = 256      # OR'ed into a dual evaluation's precision: grid costs on the tensor cores
COST_SQEUCLID, COST_L1 = 1, 2


class Params(ct.Structure):
    _fields_ = [("gamma_i", ct.c_double), ("gamma_f", ct.c_double), ("p", ct.c_double),
                ("q", ct.c_double), ("ls_c1", ct.c_double), ("ls_c2", ct.c_double),
                ("ls_max_trials", ct.c_int32), ("max_iter", ct.c_int32), ("precision", ct.c_int32),
                ("warm_start", ct.c_int32), ("final_tol", ct.c_double), ("fp32_floor", ct.c_double),
                ("profile", ct.c_int32), ("smoothing", ct.c_int32), ("projector", ct.c_int32),
                ("stop_entropy", ct.c_int32), ("precond", ct.c_int32), ("ls_init", ct.c_int32),
                ("wait_limit_us", ct.c_int32), ("tensor_cores", ct.c_int32), ("polish_iters", ct.c_int32),
                ("reserved", ct.c_int32)]


class Info(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("stages", ct.c_int32), ("evals", ct.c_int64),
                ("evals_fp64", ct.c_int64), ("iters", ct.c_int64), ("ls_trials", ct.c_int64),
                ("grad_l1", ct.c_double), ("gamma_f", ct.c_double), ("H_min", ct.c_double),
                ("cost", ct.c_double), ("lower_bound", ct.c_double), ("gap_cert", ct.c_double),
                ("t_stage_fp32_ms", ct.c_double), ("t_stage_fp64_ms", ct.c_double),
                ("t_round_ms", ct.c_double), ("t_bound_ms", ct.c_double), ("launches", ct.c_int32),
                ("stage_launches_fp32", ct.c_int32), ("stalls", ct.c_int32), ("tensor_cores", ct.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class TraceRow(ct.Structure):
    """mdot_trace_row: one kernel launch of a profiled solve."""
    _fields_ = [("kind", ct.c_int32), ("reserved", ct.c_int32), ("ms", ct.c_double), ("evals", ct.c_int64)]


class MdotError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = lib().mdot_last_error().decode() if status == MDOT_ERR_CUDA else ""
        super().__init__(f"{where}: {status_string(status)} {msg}".strip())


_lib = None
_P = ct.c_void_p


_lib_path = None


def use_phase_timer_build():
    """Load the diagnostic build with stage-kernel phase timers (build.py --phases; built here if
    needed) instead of the default library.  Must be called before anything else loads it."""
    global _lib_path
    if _lib is not None:
        raise RuntimeError("libmdot is already loaded")
    _lib_path = _build.build(phases=True)


def phase_timers(clear: bool = True, max_ctas: int = 160):
    """mdot_phase_timers: per CTA, cycles per phase (9) and the evaluation count, as a numpy array
    (max_ctas x 10); None when the loaded library has no phase timers."""
    import numpy as np
    L = lib()
    L.mdot_phase_timers.argtypes = [_P, ct.c_int32, ct.c_int32]
    L.mdot_phase_timers.restype = ct.c_int32
    buf = (ct.c_uint64 * (max_ctas * 10))()
    s = L.mdot_phase_timers(ct.cast(buf, _P), max_ctas, 1 if clear else 0)
    if s == MDOT_NOT_READY:
        return None
    if s != MDOT_OK:
        raise MdotError(s, "mdot_phase_timers")
    return np.frombuffer(buf, dtype=np.uint64).reshape(max_ctas, 10).copy()


def lib():
    """Load libmdot.so (built in-tree).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = _lib_path or _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libmdot is not built ({path} missing): run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` first")
    L = ct.CDLL(path)
    L.mdot_default_params.argtypes = [ct.POINTER(Params)]
    L.mdot_default_params.restype = None
    L.mdot_status_string.argtypes = [ct.c_int32]
    L.mdot_status_string.restype = ct.c_char_p
    L.mdot_last_error.argtypes = []
    L.mdot_last_error.restype = ct.c_char_p
    L.mdot_create.argtypes = [ct.POINTER(_P), ct.c_int64, _P]
    L.mdot_destroy.argtypes = [_P]
    L.mdot_dual_eval.argtypes = [_P, _P, _P, ct.c_double, _P, ct.c_int64, _P, ct.c_int32, _P, _P, _P, _P,
                                 ct.POINTER(ct.c_double)]
    L.mdot_round.argtypes = [_P, _P, _P, ct.c_double, _P, _P, _P, ct.c_int64,
                             ct.POINTER(ct.c_double), _P]
    L.mdot_lower_bound.argtypes = [_P, _P, ct.c_double, _P, _P, _P, ct.c_int64, ct.POINTER(ct.c_double)]
    L.mdot_solve.argtypes = [_P, _P, _P, _P, ct.c_int64, ct.c_double, ct.POINTER(Params), _P, _P,
                             ct.POINTER(ct.c_double), ct.POINTER(ct.c_double), ct.POINTER(Info)]
    L.mdot_solve_host.argtypes = L.mdot_solve.argtypes
    L.mdot_solve_points.argtypes = [_P, _P, _P, _P, _P, ct.c_int32, ct.c_float, ct.c_int64, ct.c_double,
                                    ct.POINTER(Params), _P, _P, ct.POINTER(ct.c_double),
                                    ct.POINTER(ct.c_double), ct.POINTER(Info)]
    L.mdot_dual_eval_points.argtypes = [_P, _P, _P, ct.c_double, _P, _P, ct.c_int32, ct.c_float, ct.c_int64,
                                        _P, ct.c_int32, _P, _P, _P, _P, ct.POINTER(ct.c_double)]
    L.mdot_dual_eval_time.argtypes = [_P, ct.POINTER(ct.c_double)]
    for name in ("mdot_create", "mdot_destroy", "mdot_dual_eval", "mdot_round", "mdot_lower_bound",
                 "mdot_solve", "mdot_solve_host", "mdot_solve_points", "mdot_dual_eval_points",
                 "mdot_dual_eval_time"):
        getattr(L, name).restype = ct.c_int32
    _lib = L
    return L


def status_string(s: int) -> str:
    return lib().mdot_status_string(int(s)).decode()


def default_params(**kw) -> Params:
    prm = Params()
    lib().mdot_default_params(ct.byref(prm))
    for k, v in kw.items():
        if not hasattr(prm, k) or k == "reserved":
            raise KeyError(k)
        setattr(prm, k, v)
    return prm


def _ptr(t, dtype, n=None, name="array"):
    """Device pointer of a contiguous CUDA tensor of the given torch dtype (checked)."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, has {t.numel()}")
    return ct.c_void_p(t.data_ptr())


def _hptr(a, dtype, n, name):
    import numpy as np
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous or a.size != n:
        raise TypeError(f"{name} must be a contiguous numpy {dtype} array of {n} elements")
    return ct.c_void_p(a.ctypes.data)


@dataclass
class SolveResult:
    status: int
    cost: float
    gap_cert: float
    info: Info


class Handle:
    """Owns an mdot_handle (workspace for problems of size <= max_n) bound to a CUDA stream."""

    def __init__(self, max_n: int, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.max_n = int(max_n)
        h = _P()
        s = lib().mdot_create(ct.byref(h), self.max_n, ct.c_void_p(stream.cuda_stream))
        if s != MDOT_OK:
            raise MdotError(s, "mdot_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().mdot_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- calls -------------------------------------------------------------------------------
    def dual_eval(self, u, v, gamma: float, C, ref_log_rP=None, precision: int = PREC_FP32, r=None, c=None):
        """mdot_dual_eval: (log r(P), log c(P)); with the marginals r, c also the dual objective g
        of Eq. (4): (log r(P), log c(P), g)."""
        import torch
        n = u.numel()
        lr = torch.empty(n, dtype=torch.float64, device=u.device)
        lc = torch.empty(n, dtype=torch.float64, device=u.device)
        ref = _ptr(ref_log_rP, torch.float64, n, "ref_log_rP") if ref_log_rP is not None else None
        want_g = r is not None or c is not None
        g = ct.c_double(0.0)
        s = lib().mdot_dual_eval(self._h, _ptr(u, torch.float64, n, "u"), _ptr(v, torch.float64, n, "v"),
                                 float(gamma), _ptr(C, torch.float32, n * n, "C"), n, ref,
                                 int(precision), _ptr(lr, torch.float64), _ptr(lc, torch.float64),
                                 _ptr(r, torch.float64, n, "r") if r is not None else None,
                                 _ptr(c, torch.float64, n, "c") if c is not None else None,
                                 ct.byref(g) if want_g else None)
        if s != MDOT_OK:
            raise MdotError(s, "mdot_dual_eval")
        return (lr, lc, g.value) if want_g else (lr, lc)

    def solve_trace(self):
        """mdot_solve_trace: one dict per kernel launch of the last profiled solve (kind: 0 fp32-entry
        stage, 1 fp64-entry stage, 2 rounding, 3 bound; device ms; evaluations it made)."""
        L = lib()
        if not hasattr(L, "_trace_typed"):
            L.mdot_solve_trace.argtypes = [_P, ct.c_int32, ct.POINTER(TraceRow), ct.POINTER(ct.c_int32)]
            L.mdot_solve_trace.restype = ct.c_int32
            L._trace_typed = True
        rows = (TraceRow * 512)()
        cnt = ct.c_int32(0)
        s = L.mdot_solve_trace(self._h, 512, rows, ct.byref(cnt))
        if s != MDOT_OK:
            raise MdotError(s, "mdot_solve_trace")
        return [{"kind": rows[k].kind, "ms": rows[k].ms, "evals": rows[k].evals} for k in range(min(cnt.value, 512))]

    def dual_eval_time(self) -> float:
        """mdot_dual_eval_time: device milliseconds of the last dual-evaluation kernel."""
        ms = ct.c_double(0.0)
        s = lib().mdot_dual_eval_time(self._h, ct.byref(ms))
        if s != MDOT_OK:
            raise MdotError(s, "mdot_dual_eval_time")
        return ms.value

    def round(self, u, v, gamma: float, C, r, c, want_G: bool = False):
        import torch
        n = u.numel()
        G = torch.empty((n, n), dtype=torch.float64, device=u.device) if want_G else None
        cost = ct.c_double(0.0)
        s = lib().mdot_round(self._h, _ptr(u, torch.float64, n, "u"), _ptr(v, torch.float64, n, "v"),
                             float(gamma), _ptr(C, torch.float32, n * n, "C"), _ptr(r, torch.float64, n, "r"),
                             _ptr(c, torch.float64, n, "c"), n, ct.byref(cost),
                             _ptr(G, torch.float64) if want_G else None)
        if s != MDOT_OK:
            raise MdotError(s, "mdot_round")
        return cost.value, G

    def lower_bound(self, u, gamma: float, C, r, c) -> float:
        import torch
        n = u.numel()
        lb = ct.c_double(0.0)
        s = lib().mdot_lower_bound(self._h, _ptr(u, torch.float64, n, "u"), float(gamma),
                                   _ptr(C, torch.float32, n * n, "C"), _ptr(r, torch.float64, n, "r"),
                                   _ptr(c, torch.float64, n, "c"), n, ct.byref(lb))
        if s != MDOT_OK:
            raise MdotError(s, "mdot_lower_bound")
        return lb.value

    def solve(self, r, c, C, eps_target: float = 1e-6, params: Params | None = None,
              u_out=None, v_out=None, check: bool = True):
        """mdot_solve on device tensors; returns (u, v, SolveResult)."""
        import torch
        n = r.numel()
        u = u_out if u_out is not None else torch.empty(n, dtype=torch.float64, device=r.device)
        v = v_out if v_out is not None else torch.empty(n, dtype=torch.float64, device=r.device)
        cost, gap, info = ct.c_double(0.0), ct.c_double(0.0), Info()
        s = lib().mdot_solve(self._h, _ptr(r, torch.float64, n, "r"), _ptr(c, torch.float64, n, "c"),
                             _ptr(C, torch.float32, n * n, "C"), n, float(eps_target),
                             ct.byref(params) if params is not None else None,
                             _ptr(u, torch.float64, n, "u_out"), _ptr(v, torch.float64, n, "v_out"),
                             ct.byref(cost), ct.byref(gap), ct.byref(info))
        if check and s not in (MDOT_OK, MDOT_ERR_NOT_CONVERGED):
            raise MdotError(s, "mdot_solve")
        return u, v, SolveResult(s, cost.value, gap.value, info)

    def dual_eval_points(self, u, v, gamma: float, x, y, kind: int, scale: float, ref_log_rP=None,
                         precision: int = PREC_FP32, r=None, c=None):
        """mdot_dual_eval_points: C regenerated from coordinates x, y (CUDA float32 tensors n x 3);
        with r, c also the dual objective g of Eq. (4)."""
        import torch
        n = u.numel()
        lr = torch.empty(n, dtype=torch.float64, device=u.device)
        lc = torch.empty(n, dtype=torch.float64, device=u.device)
        ref = _ptr(ref_log_rP, torch.float64, n, "ref_log_rP") if ref_log_rP is not None else None
        want_g = r is not None or c is not None
        g = ct.c_double(0.0)
        s = lib().mdot_dual_eval_points(self._h, _ptr(u, torch.float64, n, "u"), _ptr(v, torch.float64, n, "v"),
                                        float(gamma), _ptr(x, torch.float32, 3 * n, "x"),
                                        _ptr(y, torch.float32, 3 * n, "y"), int(kind), float(scale), n, ref,
                                        int(precision), _ptr(lr, torch.float64), _ptr(lc, torch.float64),
                                        _ptr(r, torch.float64, n, "r") if r is not None else None,
                                        _ptr(c, torch.float64, n, "c") if c is not None else None,
                                        ct.byref(g) if want_g else None)
        if s != MDOT_OK:
            raise MdotError(s, "mdot_dual_eval_points")
        return (lr, lc, g.value) if want_g else (lr, lc)

    def solve_points(self, r, c, x, y, kind: int, scale: float, eps_target: float = 1e-6,
                     params: Params | None = None, u_out=None, v_out=None, check: bool = True):
        """mdot_solve_points: MDOT-PNCG with C regenerated from coordinates (memory O(n))."""
        import torch
        n = r.numel()
        u = u_out if u_out is not None else torch.empty(n, dtype=torch.float64, device=r.device)
        v = v_out if v_out is not None else torch.empty(n, dtype=torch.float64, device=r.device)
        cost, gap, info = ct.c_double(0.0), ct.c_double(0.0), Info()
        s = lib().mdot_solve_points(self._h, _ptr(r, torch.float64, n, "r"), _ptr(c, torch.float64, n, "c"),
                                    _ptr(x, torch.float32, 3 * n, "x"), _ptr(y, torch.float32, 3 * n, "y"),
                                    int(kind), float(scale), n, float(eps_target),
                                    ct.byref(params) if params is not None else None,
                                    _ptr(u, torch.float64, n, "u_out"), _ptr(v, torch.float64, n, "v_out"),
                                    ct.byref(cost), ct.byref(gap), ct.byref(info))
        if check and s not in (MDOT_OK, MDOT_ERR_NOT_CONVERGED):
            raise MdotError(s, "mdot_solve_points")
        return u, v, SolveResult(s, cost.value, gap.value, info)

    def solve_host(self, r, c, C, eps_target: float = 1e-6, params: Params | None = None,
                   u_out=None, v_out=None, check: bool = True):
        """mdot_solve_host on numpy arrays (host memory; the copies are part of the call)."""
        import numpy as np
        n = r.size
        u = u_out if u_out is not None else np.empty(n, np.float64)
        v = v_out if v_out is not None else np.empty(n, np.float64)
        cost, gap, info = ct.c_double(0.0), ct.c_double(0.0), Info()
        s = lib().mdot_solve_host(self._h, _hptr(r, np.float64, n, "r"), _hptr(c, np.float64, n, "c"),
                                  _hptr(C, np.float32, n * n, "C"), n, float(eps_target),
                                  ct.byref(params) if params is not None else None,
                                  _hptr(u, np.float64, n, "u_out"), _hptr(v, np.float64, n, "v_out"),
                                  ct.byref(cost), ct.byref(gap), ct.byref(info))
        if check and s not in (MDOT_OK, MDOT_ERR_NOT_CONVERGED):
            raise MdotError(s, "mdot_solve_host")
        return u, v, SolveResult(s, cost.value, gap.value, info)


def cost_matrix(x, y, kind: int, scale: float, stream=None):
    """mdot_cost_matrix: the regenerated n x n cost of coordinates x, y (CUDA float32 tensors n x 3),
    computed as the solver's passes compute it; returns a new CUDA float32 tensor."""
    import torch
    L = lib()
    if not hasattr(L, "_cost_typed"):
        L.mdot_cost_matrix.argtypes = [_P, _P, ct.c_int32, ct.c_float, ct.c_int64, _P, _P]
        L.mdot_cost_matrix.restype = ct.c_int32
        L._cost_typed = True
    n = x.shape[0]
    if stream is None:
        stream = torch.cuda.current_stream()
    C = torch.empty((n, n), dtype=torch.float32, device=x.device)
    s = L.mdot_cost_matrix(_ptr(x, torch.float32, 3 * n, "x"), _ptr(y, torch.float32, 3 * n, "y"), int(kind),
                           float(scale), n, _ptr(C, torch.float32), ct.c_void_p(stream.cuda_stream))
    if s != MDOT_OK:
        raise MdotError(s, "mdot_cost_matrix")
    return C


def read_probe(buf, reps: int, stream=None):
    """mdot_read_probe: read the float32 CUDA tensor buf `reps` times (128-bit loads); returns the
    checksum tensor (the caller times the call with CUDA events on `stream`)."""
    import torch
    L = lib()
    if not hasattr(L, "_probe_typed"):
        L.mdot_read_probe.argtypes = [_P, ct.c_int64, ct.c_int32, _P, _P]
        L.mdot_read_probe.restype = ct.c_int32
        L._probe_typed = True
    if stream is None:
        stream = torch.cuda.current_stream()
    out = torch.empty(1, dtype=torch.float32, device=buf.device)
    s = L.mdot_read_probe(_ptr(buf, torch.float32, None, "buf"), buf.numel(), int(reps), _ptr(out, torch.float32),
                          ct.c_void_p(stream.cuda_stream))
    if s != MDOT_OK:
        raise MdotError(s, "mdot_read_probe")
    return out


NOALLOC_MAX_N = 4096


def dual_eval_noalloc(u, v, gamma: float, C, log_rP, log_cP, ref_log_rP=None, stream=None) -> int:
    """mdot_dual_eval_noalloc: fp32-entry dual evaluation that allocates no device memory (its
    scratch is a static device array inside the library).  For callers that cannot allocate;
    u, v, C, log_rP, log_cP are caller-owned CUDA tensors.  Returns the mdot_status."""
    import torch
    L = lib()
    if not hasattr(L, "_noalloc_typed"):
        L.mdot_dual_eval_noalloc.argtypes = [_P, _P, ct.c_double, _P, ct.c_int64, _P, _P, _P, _P]
        L.mdot_dual_eval_noalloc.restype = ct.c_int32
        L._noalloc_typed = True
    n = u.numel()
    if stream is None:
        stream = torch.cuda.current_stream()
    ref = _ptr(ref_log_rP, torch.float64, n, "ref_log_rP") if ref_log_rP is not None else None
    return L.mdot_dual_eval_noalloc(_ptr(u, torch.float64, n, "u"), _ptr(v, torch.float64, n, "v"),
                                    float(gamma), _ptr(C, torch.float32, n * n, "C"), n, ref,
                                    _ptr(log_rP, torch.float64, n, "log_rP"),
                                    _ptr(log_cP, torch.float64, n, "log_cP"),
                                    ct.c_void_p(stream.cuda_stream))


BATCH_MAX_N = 8192


class Problem(ct.Structure):
    """mdot_problem: one problem of a batch (device pointers)."""
    _fields_ = [("n", ct.c_int64), ("r", _P), ("c", _P), ("C", _P), ("x", _P), ("y", _P),
                ("cost_kind", ct.c_int32), ("scale", ct.c_float), ("eps_target", ct.c_double),
                ("gamma_f", ct.c_double), ("u_out", _P), ("v_out", _P)]


class Result(ct.Structure):
    """mdot_result: outcome of one problem of a batch."""
    _fields_ = [("status", ct.c_int32), ("stages", ct.c_int32), ("evals", ct.c_int64), ("iters", ct.c_int64),
                ("cost", ct.c_double), ("lower_bound", ct.c_double), ("gap_cert", ct.c_double),
                ("grad_l1", ct.c_double), ("gamma_f", ct.c_double), ("H_min", ct.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def make_problem(r, c, C=None, x=None, y=None, kind: int = COST_SQEUCLID, scale: float = 1.0,
                 eps_target: float = 1e-6, gamma_f: float = 0.0, u_out=None, v_out=None) -> Problem:
    """Fill an mdot_problem from CUDA tensors (the tensors must outlive the solve)."""
    import torch
    n = r.numel()
    p = Problem()
    p.n = n
    p.r = _ptr(r, torch.float64, n, "r")
    p.c = _ptr(c, torch.float64, n, "c")
    if C is not None:
        p.C = _ptr(C, torch.float32, n * n, "C")
    else:
        p.x = _ptr(x, torch.float32, 3 * n, "x")
        p.y = _ptr(y, torch.float32, 3 * n, "y")
        p.cost_kind = int(kind)
        p.scale = float(scale)
    p.eps_target = float(eps_target)
    p.gamma_f = float(gamma_f)
    if u_out is not None:
        p.u_out = _ptr(u_out, torch.float64, n, "u_out")
    if v_out is not None:
        p.v_out = _ptr(v_out, torch.float64, n, "v_out")
    return p


def _batch_lib():
    L = lib()
    if not hasattr(L, "_batch_typed"):
        L.mdot_solve_batch.argtypes = [_P, ct.c_int32, ct.POINTER(Problem), ct.POINTER(Params), ct.POINTER(Result)]
        L.mdot_solve_batch.restype = ct.c_int32
        L._batch_typed = True
    return L


def _solve_batch(self, problems, params: Params | None = None):
    """mdot_solve_batch: every problem of the list in one persistent launch (per cost form)."""
    k = len(problems)
    arr = (Problem * k)(*problems)
    res = (Result * k)()
    s = _batch_lib().mdot_solve_batch(self._h, k, arr, ct.byref(params) if params is not None else None, res)
    if s != MDOT_OK:
        raise MdotError(s, "mdot_solve_batch")
    return list(res)


Handle.solve_batch = _solve_batch


class BatchTuning(ct.Structure):
    """mdot_batch_tuning: the batched form's tile variant per size bucket, the tuner's pick (buckets
    below narrow_below narrow) and the timing batch's seconds under each candidate table."""
    _fields_ = [("variant", ct.c_int32 * 5), ("narrow_below", ct.c_int32), ("seconds", ct.c_double * 6)]

    def as_dict(self) -> dict:
        return {"variant": list(self.variant), "narrow_below": self.narrow_below, "seconds": list(self.seconds)}


def _tune_batch(self, problems, params: Params | None = None, sample: int = 64) -> BatchTuning:
    """mdot_tune_batch: time the batch (up to `sample` problems, gamma_f <= 2^12) under each table
    "buckets below k narrow" and keep the fastest (in the handle)."""
    L = _batch_lib()
    if not hasattr(L, "_tune_typed"):
        L.mdot_tune_batch.argtypes = [_P, ct.c_int32, ct.POINTER(Problem), ct.POINTER(Params), ct.c_int32,
                                      ct.POINTER(BatchTuning)]
        L.mdot_tune_batch.restype = ct.c_int32
        L.mdot_set_batch_tuning.argtypes = [_P, ct.POINTER(BatchTuning)]
        L.mdot_set_batch_tuning.restype = ct.c_int32
        L._tune_typed = True
    k = len(problems)
    arr = (Problem * k)(*problems)
    out = BatchTuning()
    s = L.mdot_tune_batch(self._h, k, arr, ct.byref(params) if params is not None else None, int(sample),
                          ct.byref(out))
    if s != MDOT_OK:
        raise MdotError(s, "mdot_tune_batch")
    return out


def _set_batch_tuning(self, table: BatchTuning):
    """mdot_set_batch_tuning: install a stored table of tile variants in the handle."""
    L = _batch_lib()
    L.mdot_set_batch_tuning.argtypes = [_P, ct.POINTER(BatchTuning)]
    L.mdot_set_batch_tuning.restype = ct.c_int32
    s = L.mdot_set_batch_tuning(self._h, ct.byref(table))
    if s != MDOT_OK:
        raise MdotError(s, "mdot_set_batch_tuning")


Handle.tune_batch = _tune_batch
Handle.set_batch_tuning = _set_batch_tuning


MDOT_NOT_READY = 7


def _server_lib():
    L = lib()
    if not hasattr(L, "_server_typed"):
        L.mdot_server_create.argtypes = [ct.POINTER(_P), ct.c_uint64, ct.POINTER(Params), ct.POINTER(ServerConfig)]
        L.mdot_server_submit.argtypes = [_P, ct.POINTER(Problem), ct.POINTER(ct.c_uint64)]
        L.mdot_server_poll.argtypes = [_P, ct.c_uint64, ct.POINTER(Result)]
        L.mdot_server_wait.argtypes = [_P, ct.c_uint64, ct.c_double, ct.POINTER(Result)]
        L.mdot_server_destroy.argtypes = [_P]
        for name in ("mdot_server_create", "mdot_server_submit", "mdot_server_poll", "mdot_server_wait",
                     "mdot_server_destroy"):
            getattr(L, name).restype = ct.c_int32
        L._server_typed = True
    return L


class ServerConfig(ct.Structure):
    """mdot_server_config: routing of the serving runtime (big_n, big_lanes, lane_ctas)."""
    _fields_ = [("big_n", ct.c_int64), ("big_lanes", ct.c_int32), ("lane_ctas", ct.c_int32)]


class Server:
    """mdot_server_*: request loop with continuous batching on the current device.

    submit() takes an mdot_problem (see make_problem) and returns a ticket; the problem's tensors
    are kept referenced here until its result has been collected (poll/wait returned it)."""

    def __init__(self, workspace_bytes: int, params: Params | None = None, big_n: int | None = None,
                 big_lanes: int | None = None, lane_ctas: int | None = None):
        L = _server_lib()
        self._s = _P()
        cfg = None
        if big_n is not None or big_lanes is not None or lane_ctas is not None:
            cfg = ServerConfig(big_n if big_n is not None else 2048, big_lanes if big_lanes is not None else 3,
                               lane_ctas or 0)
        s = L.mdot_server_create(ct.byref(self._s), int(workspace_bytes), ct.byref(params) if params is not None else None,
                                 ct.byref(cfg) if cfg is not None else None)
        if s != MDOT_OK:
            raise MdotError(s, "mdot_server_create")
        self._keep = {}

    def submit(self, problem: Problem, keep=()) -> int:
        t = ct.c_uint64(0)
        s = _server_lib().mdot_server_submit(self._s, ct.byref(problem), ct.byref(t))
        if s != MDOT_OK:
            raise MdotError(s, "mdot_server_submit")
        self._keep[t.value] = (problem, keep)
        return t.value

    def poll(self, ticket: int):
        """Result once solved, else None."""
        r = Result()
        s = _server_lib().mdot_server_poll(self._s, int(ticket), ct.byref(r))
        if s == MDOT_NOT_READY:
            return None
        if s != MDOT_OK:
            raise MdotError(s, "mdot_server_poll")
        self._keep.pop(int(ticket), None)
        return r

    def wait(self, ticket: int, timeout: float = 60.0):
        r = Result()
        s = _server_lib().mdot_server_wait(self._s, int(ticket), float(timeout), ct.byref(r))
        if s == MDOT_NOT_READY:
            return None
        if s != MDOT_OK:
            raise MdotError(s, "mdot_server_wait")
        self._keep.pop(int(ticket), None)
        return r

    def close(self):
        if getattr(self, "_s", None):
            _server_lib().mdot_server_destroy(self._s)
            self._s = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune_server(workspace_bytes: int, requests, candidates=None, params: Params | None = None,
                timeout: float = 600.0):
    """Pick the served form's routing by measurement on this device: for each candidate
    (big_n, big_lanes, lane_ctas) a fresh Server replays `requests` -- a list of
    (arrival offset in seconds, mdot_problem, tensors to keep alive) -- at their arrival times and
    the wall time to the last result is taken.  Returns (best candidate as a dict, one dict per
    candidate with problems_per_s, seconds and the per-request statuses and costs in request
    order).  Candidates default to the built-in routing and two around it."""
    import time
    import torch
    if candidates is None:
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        candidates = [dict(big_n=2048, big_lanes=3, lane_ctas=sms * 29 // 100),
                      dict(big_n=2048, big_lanes=2, lane_ctas=sms * 42 // 100),
                      dict(big_n=1024, big_lanes=4, lane_ctas=sms * 21 // 100)]
    table = []
    for cand in candidates:
        torch.cuda.synchronize()
        srv = Server(workspace_bytes, params, **cand)
        try:
            tickets = []
            t0 = time.perf_counter()
            for (ta, prob, keep) in sorted(requests, key=lambda q: q[0]):
                delay = t0 + ta - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                tickets.append(srv.submit(prob, keep))
            results = [srv.wait(t, timeout) for t in tickets]
            dt = time.perf_counter() - t0
        finally:
            srv.close()
        if any(r is None for r in results):
            raise MdotError(MDOT_ERR_TIMEOUT, "tune_server")
        table.append(dict(cand, problems_per_s=len(results) / dt, seconds=dt,
                          statuses=[r.status for r in results], costs=[r.cost for r in results]))
    best = max(table, key=lambda row: row["problems_per_s"])
    return {k: best[k] for k in ("big_n", "big_lanes", "lane_ctas")}, table
