"""ctypes binding of the CPU FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg are the only callers.  The product library never imports this package.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

_D = ct.POINTER(ct.c_double)
_DPHI = ct.CFUNCTYPE(ct.c_double, ct.c_void_p, ct.c_double)
_KEEP = ct.CFUNCTYPE(None, ct.c_void_p)


class OrParams(ct.Structure):
    _fields_ = [("gamma_i", ct.c_double), ("gamma_f", ct.c_double), ("p", ct.c_double),
                ("q", ct.c_double), ("ls_c1", ct.c_double), ("ls_c2", ct.c_double),
                ("ls_max_trials", ct.c_int), ("max_iter", ct.c_int), ("projector", ct.c_int),
                ("warm_start", ct.c_int), ("precond", ct.c_int), ("smoothing", ct.c_int),
                ("final_tol", ct.c_double), ("stop_entropy", ct.c_int), ("ls_init", ct.c_int)]


class OrStats(ct.Structure):
    _fields_ = [("stages", ct.c_int), ("evals", ct.c_long), ("half_evals", ct.c_long),
                ("iters", ct.c_long), ("ls_trials", ct.c_long), ("status", ct.c_int),
                ("grad_l1", ct.c_double), ("gamma_last", ct.c_double), ("grad_l1_init", ct.c_double)]


_SO_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so with gcc (plain -O2, IEEE semantics kept).
    openmp=True builds _build/liboracle_omp.so from the same source with -fopenmp (the dual
    evaluation's rows and column strips on every host core, same arithmetic), used only to time
    the CPU baseline."""
    src = os.path.join(_HERE, "oracle.c")
    so = _SO_OMP if openmp else _SO
    if not force and os.path.exists(so) and os.path.getmtime(so) >= max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return so
    os.makedirs(os.path.dirname(so), exist_ok=True)
    tmp = so + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                    "-ffp-contract=off", *(["-fopenmp"] if openmp else []), "-o", tmp, src, "-lm"],
                   check=True)
    os.replace(tmp, so)
    return so


def omp_dual_eval_timer():
    """(seconds per call of or_dual_eval, threads) on the OpenMP build: a callable timing one dual
    evaluation of (C, u, v, gamma) on every host core.  For the CPU baseline only."""
    L = ct.CDLL(build(openmp=True))
    L.or_dual_eval.argtypes = [ct.c_int, _D, _D, _D, ct.c_double, _D, _D]
    try:
        nthreads = int(ct.CFUNCTYPE(ct.c_int)(("omp_get_max_threads", L))())
    except Exception:
        nthreads = os.cpu_count() or 1

    def run(C, u, v, gamma):
        C, u, v = _f64(C), _f64(u), _f64(v)
        n = u.size
        lr, lc = np.empty(n), np.empty(n)
        L.or_dual_eval(n, _p(C), _p(u), _p(v), gamma, _p(lr), _p(lc))
        return lr, lc

    return run, nthreads


_use_omp = False


def use_openmp(flag: bool = True) -> None:
    """Make later calls load the OpenMP build (same arithmetic and summation order, so the same
    results; the dual evaluation runs on every host core).  Call before the first oracle call;
    used by the golden-value script for long solves."""
    global _use_omp, _lib
    if flag != _use_omp:
        _use_omp, _lib = flag, None


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build(openmp=_use_omp))
        L = _lib
        L.or_default_params.argtypes = [ct.POINTER(OrParams)]
        L.or_entropy.argtypes = [ct.c_int, _D]
        L.or_entropy.restype = ct.c_double
        L.or_dual_eval.argtypes = [ct.c_int, _D, _D, _D, ct.c_double, _D, _D]
        L.or_dual_value.argtypes = [ct.c_int, _D, _D, _D, ct.c_double, _D, _D]
        L.or_dual_value.restype = ct.c_double
        L.or_pncg.argtypes = [ct.c_int, _D, ct.c_double, _D, _D, ct.c_double, _D, _D,
                              ct.POINTER(OrParams), ct.POINTER(OrStats), _D, _D]
        L.or_sinkhorn.argtypes = [ct.c_int, _D, ct.c_double, _D, _D, ct.c_double, _D, _D,
                                  ct.POINTER(OrParams), ct.POINTER(OrStats), _D]
        L.or_mdot.argtypes = [ct.c_int, _D, _D, _D, ct.POINTER(OrParams), _D, _D,
                              ct.POINTER(OrStats), _D, ct.c_int]
        L.or_round.argtypes = [ct.c_int, _D, _D, _D, ct.c_double, _D, _D, _D]
        L.or_round.restype = ct.c_double
        L.or_ctransform_lb.argtypes = [ct.c_int, _D, _D, ct.c_double, _D, _D]
        L.or_ctransform_lb.restype = ct.c_double
        L.or_gamma_f_for_eps.argtypes = [ct.c_double] * 5
        L.or_gamma_f_for_eps.restype = ct.c_double
        L.or_ls_search.argtypes = [ct.c_double, ct.c_double, ct.POINTER(OrParams), _DPHI, _KEEP,
                                   ct.c_void_p, _D]
        L.or_ls_search.restype = ct.c_int
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def params(**kw) -> OrParams:
    prm = OrParams()
    lib().or_default_params(ct.byref(prm))
    for k, v in kw.items():
        if not hasattr(prm, k):
            raise KeyError(k)
        setattr(prm, k, v)
    return prm


def entropy(r) -> float:
    r = _f64(r)
    return lib().or_entropy(r.size, _p(r))


def dual_eval(C, u, v, gamma):
    C, u, v = _f64(C), _f64(u), _f64(v)
    n = u.size
    lr, lc = np.empty(n), np.empty(n)
    lib().or_dual_eval(n, _p(C), _p(u), _p(v), gamma, _p(lr), _p(lc))
    return lr, lc


def dual_value(C, u, v, gamma, r, c) -> float:
    C, u, v, r, c = map(_f64, (C, u, v, r, c))
    return lib().or_dual_value(u.size, _p(C), _p(u), _p(v), gamma, _p(r), _p(c))


def pncg(C, gamma, r, c, tol, u, v, **kw):
    C, r, c = map(_f64, (C, r, c))
    u, v = _f64(u).copy(), _f64(v).copy()
    n = u.size
    st = OrStats()
    lr, lc = np.empty(n), np.empty(n)
    prm = params(**kw)
    rc = lib().or_pncg(n, _p(C), gamma, _p(r), _p(c), tol, _p(u), _p(v), ct.byref(prm),
                       ct.byref(st), _p(lr), _p(lc))
    return u, v, rc, st, lr, lc


def sinkhorn(C, gamma, r, c, tol, u, v, **kw):
    C, r, c = map(_f64, (C, r, c))
    u, v = _f64(u).copy(), _f64(v).copy()
    st = OrStats()
    lr = np.empty(u.size)
    prm = params(**kw)
    rc = lib().or_sinkhorn(u.size, _p(C), gamma, _p(r), _p(c), tol, _p(u), _p(v), ct.byref(prm),
                           ct.byref(st), _p(lr))
    return u, v, rc, st, lr


def mdot(C, r, c, max_log: int = 256, **kw):
    C, r, c = map(_f64, (C, r, c))
    n = r.size
    u, v = np.empty(n), np.empty(n)
    st = OrStats()
    log = np.zeros((max_log, 6))
    prm = params(**kw)
    rc = lib().or_mdot(n, _p(C), _p(r), _p(c), ct.byref(prm), _p(u), _p(v), ct.byref(st),
                       _p(log), max_log)
    return u, v, rc, st, log[: min(st.stages, max_log)]


def round_plan(C, u, v, gamma, r, c, want_G: bool = False):
    C, u, v, r, c = map(_f64, (C, u, v, r, c))
    n = u.size
    G = np.empty((n, n)) if want_G else None
    cost = lib().or_round(n, _p(C), _p(u), _p(v), gamma, _p(r), _p(c),
                          _p(G) if want_G else ct.cast(None, _D))
    return cost, G


def ctransform_lb(C, u, gamma, r, c) -> float:
    C, u, r, c = map(_f64, (C, u, r, c))
    return lib().or_ctransform_lb(u.size, _p(C), _p(u), gamma, _p(r), _p(c))


def ls_search(dphi, d0: float, a0: float = 1.0, **kw):
    """The App. B line search (or_ls_search) on a Python function dphi(alpha) = phi'(alpha).
    Returns (rc, alpha, trials, lows): the return code, the step, every trial step in order and the
    trial steps that became the lower end of the bracket."""
    trials, lows = [], []

    def _dphi(_ctx, a):
        trials.append(a)
        return float(dphi(a))

    def _keep(_ctx):
        lows.append(trials[-1])

    f, k = _DPHI(_dphi), _KEEP(_keep)
    alpha = np.zeros(1)
    rc = lib().or_ls_search(float(d0), float(a0), ct.byref(params(**kw)), f, k, None, _p(alpha))
    return rc, float(alpha[0]), trials, lows


def gamma_f_for_eps(H, eps, gamma_i=16.0, q=2.0 ** (1.0 / 3.0), p=1.5) -> float:
    return lib().or_gamma_f_for_eps(H, eps, gamma_i, q, p)


@dataclass
class SolveResult:
    u: np.ndarray
    v: np.ndarray
    gamma_f: float
    cost: float
    lb: float
    gap_cert: float
    stats: OrStats
    stage_log: np.ndarray
    status: int


def solve(C, r, c, eps_target: float | None = None, gamma_f: float | None = None, **kw) -> SolveResult:
    """Alg. 1 followed by Alg. 3 and the c-transform lower bound, as one call.
    gamma_f is taken as given, or derived from eps_target by the Prop. 2 relation."""
    r, c = _f64(r), _f64(c)
    prm = params(**kw)
    if gamma_f is None:
        H = max(min(entropy(r), entropy(c)), 1e-12)
        gamma_f = gamma_f_for_eps(H, eps_target, prm.gamma_i, prm.q, prm.p)
    u, v, rc, st, log = mdot(C, r, c, gamma_f=gamma_f, **kw)
    cost, _ = round_plan(C, u, v, gamma_f, r, c)
    lb = ctransform_lb(C, u, gamma_f, r, c)
    return SolveResult(u, v, gamma_f, cost, lb, cost - lb, st, log, rc)
