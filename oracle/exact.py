"""Exact (unregularised) OT values used to pin the oracle and to measure true optimality gaps.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The paper measures errors against an exact
network-simplex solution (Sec. 5); here the exact optimum comes from textbook special cases and
from the HiGHS LP solver (a library routine):

* brute force over permutations (uniform marginals, n <= 8; by Birkhoff-von Neumann an optimal
  plan is a permutation matrix scaled by 1/n);
* the monotone (north-west corner) coupling of sorted supports for 1-D problems with a convex
  cost of x - y, optimal for any n;
* the full transportation LP (n <= ~300);
* column generation for large n: the LP restricted to a candidate arc set, priced against all
  n^2 reduced costs C_ij - f_i - g_j; it stops only when no arc prices out, so the returned dual
  (f, g) is feasible to the pricing tolerance and certifies the value.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.optimize import linprog
from scipy.sparse import coo_matrix


def brute_force_uniform(C: np.ndarray) -> float:
    """min over permutations sigma of (1/n) sum_i C[i, sigma(i)]."""
    n = C.shape[0]
    best = np.inf
    for perm in itertools.permutations(range(n)):
        best = min(best, float(C[np.arange(n), list(perm)].sum()))
    return best / n


def monotone_1d(x: np.ndarray, y: np.ndarray, r: np.ndarray, c: np.ndarray, cost) -> float:
    """OT between sum r_i delta_{x_i} and sum c_j delta_{y_j} on the real line for a convex
    cost(x - y): the north-west corner coupling of the sorted supports."""
    ix, iy = np.argsort(x, kind="stable"), np.argsort(y, kind="stable")
    xs, rs, ys, cs = x[ix], r[ix].astype(np.float64).copy(), y[iy], c[iy].astype(np.float64).copy()
    i = j = 0
    total = 0.0
    while i < len(xs) and j < len(ys):
        m = min(rs[i], cs[j])
        total += m * cost(xs[i] - ys[j])
        rs[i] -= m
        cs[j] -= m
        if rs[i] <= cs[j]:
            i += 1
        else:
            j += 1
    return total


_LP_DUAL_TOL = 1e-10          # HiGHS primal and dual feasibility tolerances used below


def _lp(Cflat, rows, cols, n, r, c):
    m = len(Cflat)
    A = coo_matrix((np.ones(2 * m), (np.concatenate([rows, n + cols]),
                                     np.concatenate([np.arange(m), np.arange(m)]))),
                   shape=(2 * n, m)).tocsr()
    b = np.concatenate([r, c])
    res = linprog(Cflat, A_eq=A, b_eq=b, bounds=(0, None), method="highs",
                  options={"primal_feasibility_tolerance": _LP_DUAL_TOL,
                           "dual_feasibility_tolerance": _LP_DUAL_TOL})
    if res.status != 0:
        raise RuntimeError(f"HiGHS failed: {res.message}")
    duals = res.eqlin.marginals
    return res.fun, duals[:n], duals[n:], res.x


def exact_ot_lp(C: np.ndarray, r: np.ndarray, c: np.ndarray) -> float:
    """Full transportation LP over all n^2 arcs."""
    n = C.shape[0]
    rows, cols = np.divmod(np.arange(n * n), n)
    val, _, _, _ = _lp(np.asarray(C, np.float64).reshape(-1), rows, cols, n,
                       np.asarray(r, np.float64), np.asarray(c, np.float64))
    return float(val)


def _northwest(r, c):
    """Arcs of the north-west corner rule: a feasible basis of the transportation polytope."""
    r, c = r.copy(), c.copy()
    i = j = 0
    arcs = []
    n = len(r)
    while i < n and j < n:
        arcs.append((i, j))
        m = min(r[i], c[j])
        r[i] -= m
        c[j] -= m
        if r[i] <= c[j] and i < n - 1:
            i += 1
        else:
            j += 1
    return arcs


def exact_ot_colgen(C: np.ndarray, r: np.ndarray, c: np.ndarray, k_init: int = 8,
                    tol: float = 1e-11, max_rounds: int = 200, add_per_row: int = 8,
                    seed_f: np.ndarray | None = None, seed_g: np.ndarray | None = None,
                    seed_width: float = 0.0):
    """Exact OT by column generation.  Returns (value, f, g, rounds).
    Candidate arcs start as the k_init cheapest arcs of every row and column plus a north-west
    corner basis (so the restricted LP is feasible); each round adds, per row, the add_per_row
    most negative reduced-cost arcs outside the set until none outside it is below -tol (the
    arcs inside it carry the LP's own duals, feasible to the solver's 1e-10 tolerance).
    With approximate dual potentials (seed_f, seed_g) -- e.g. f = u/gamma, g = v/gamma of an
    entropic solve -- every arc whose reduced cost C_ij - f_i - g_j is at most seed_width joins
    the first candidate set as well.  The seed only shortens the search: the returned value is
    still certified by pricing all n^2 arcs against the LP's own duals."""
    C = np.asarray(C, np.float64)
    r = np.asarray(r, np.float64)
    c = np.asarray(c, np.float64)
    n = C.shape[0]
    cand = set()
    part_r = np.argpartition(C, k_init, axis=1)[:, :k_init]
    for i in range(n):
        cand.update((i, int(j)) for j in part_r[i])
    part_c = np.argpartition(C, k_init, axis=0)[:k_init, :]
    for j in range(n):
        cand.update((int(i), j) for i in part_c[:, j])
    cand.update(_northwest(r, c))
    if seed_f is not None and seed_g is not None:
        red0 = C - np.asarray(seed_f, np.float64)[:, None] - np.asarray(seed_g, np.float64)[None, :]
        ii, jj = np.nonzero(red0 <= seed_width)
        cand.update(zip(ii.tolist(), jj.tolist()))
        del red0
    for rnd in range(max_rounds):
        arr = np.array(sorted(cand), dtype=np.int64)
        val, f, g, _ = _lp(C[arr[:, 0], arr[:, 1]], arr[:, 0], arr[:, 1], n, r, c)
        red = C - f[:, None] - g[None, :]
        # the LP's own arcs are dual feasible only to the solver's tolerance (1e-10): on
        # degenerate problems some price at -1e-10 < red < -tol, and re-adding them changes
        # nothing, so only arcs outside the set count as pricing out
        inside = red[arr[:, 0], arr[:, 1]]
        if inside.min() < -100 * _LP_DUAL_TOL:          # a sanity check of the solver's answer
            raise RuntimeError(f"LP duals infeasible on the LP's own arcs ({inside.min():.3e})")
        red[arr[:, 0], arr[:, 1]] = np.inf
        neg = red < -tol
        if not neg.any():
            return float(val), f, g, rnd + 1
        for i in np.nonzero(neg.any(axis=1))[0]:
            js = np.nonzero(neg[i])[0]
            js = js[np.argsort(red[i, js], kind="stable")[:add_per_row]]
            cand.update((int(i), int(j)) for j in js)
    raise RuntimeError("column generation did not converge")
