"""Seeded synthetic problem generators shared by the tests, the benchmark and the oracle checks.

This module holds problem *definitions* only (marginals, coordinates, cost matrices); it contains
none of the solver's arithmetic.  Every generator is deterministic in its seed (numpy PCG64).

Workload shapes follow Sec. 5.1 of the paper (64x64 pixel grids, L1 or squared-L2 pixel distance,
costs divided by their maximum so that C lies in [0, 1]) and App. C (3-D normal point clouds).  The
image datasets the paper uses are not available, so smooth random histograms stand in for them:
a mixture of three isotropic 2-D Gaussians evaluated at the cell centres plus a 1e-6 floor.

Cost matrices are built so that the dense and the on-the-fly (coordinate) forms agree bit for bit:
  grid costs:  C_ij = fl32(D_ij * s)  with D_ij an exact integer (squared or L1 cell distance) and
               s = fl32(1 / max_ij D_ij); both are exact in float32 up to the single final rounding.
  point costs: d = x_i - y_j per axis in float32, D = (d0*d0 + d1*d1) + d2*d2 with every product and
               sum rounded to float32 in that order, C_ij = fl32(D * s), s = fl32(1 / max_ij D).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "grid_histogram", "grid_coords", "grid_cost", "grid_problem",
    "point_cloud_problem", "point_cost", "line_problem", "entropy_problem", "serving_trace", "rng_for",
]


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def grid_histogram(k: int, seed: int, n_modes: int = 3) -> np.ndarray:
    """Histogram on a k x k grid: mixture of `n_modes` isotropic Gaussians (means ~ U[0,1]^2,
    sigma ~ U[0.05, 0.2], equal weights) evaluated at cell centres ((a+1/2)/k, (b+1/2)/k),
    plus a 1e-6 floor, L1-normalised.  Row-major cell order: index = a*k + b."""
    rng = rng_for(seed)
    means = rng.uniform(0.0, 1.0, size=(n_modes, 2))
    sig = rng.uniform(0.05, 0.2, size=n_modes)
    centres = (np.arange(k, dtype=np.float64) + 0.5) / k
    ga, gb = np.meshgrid(centres, centres, indexing="ij")
    dens = np.zeros((k, k), dtype=np.float64)
    for m in range(n_modes):
        d2 = (ga - means[m, 0]) ** 2 + (gb - means[m, 1]) ** 2
        dens += np.exp(-0.5 * d2 / sig[m] ** 2) / (2.0 * math.pi * sig[m] ** 2)
    dens = dens / dens.sum() + 1e-6
    h = dens.reshape(-1)
    return h / h.sum()


def grid_coords(k: int) -> np.ndarray:
    """Integer cell coordinates (a, b) of the k x k grid as float32, shape (k*k, 2)."""
    a, b = np.meshgrid(np.arange(k), np.arange(k), indexing="ij")
    return np.stack([a.reshape(-1), b.reshape(-1)], axis=1).astype(np.float32)


def coords3(xy: np.ndarray) -> np.ndarray:
    """n x 3 float32 coordinates (2-D data gets z = 0), the layout of the on-the-fly cost."""
    xy = np.asarray(xy, dtype=np.float32)
    if xy.shape[1] == 3:
        return np.ascontiguousarray(xy)
    out = np.zeros((xy.shape[0], 3), dtype=np.float32)
    out[:, : xy.shape[1]] = xy
    return out


def _grid_dist_int(k: int, kind: str) -> np.ndarray:
    xy = grid_coords(k).astype(np.int64)
    da = xy[:, None, 0] - xy[None, :, 0]
    db = xy[:, None, 1] - xy[None, :, 1]
    if kind == "l2sq":
        return da * da + db * db
    if kind == "l1":
        return np.abs(da) + np.abs(db)
    raise ValueError(f"unknown grid cost kind {kind!r}")


def grid_cost_scale(k: int, kind: str) -> np.float32:
    """s = fl32(1 / max D) for the k x k grid."""
    dmax = 2 * (k - 1) ** 2 if kind == "l2sq" else 2 * (k - 1)
    return np.float32(1.0 / dmax) if k > 1 else np.float32(1.0)


def grid_cost(k: int, kind: str = "l2sq", dtype=np.float32) -> np.ndarray:
    """Dense n x n (n = k*k) grid cost C_ij = fl32(D_ij * s), row-major, in [0, 1].
    float64 output holds the same float32 values promoted (so every precision solves one problem)."""
    d = _grid_dist_int(k, kind).astype(np.float32)
    c = d * grid_cost_scale(k, kind)          # one float32 rounding per entry
    return c.astype(dtype)


@dataclass
class Problem:
    n: int
    r: np.ndarray          # float64 [n], sums to 1
    c: np.ndarray          # float64 [n], sums to 1
    C: np.ndarray | None   # dense cost (float32 or float64), row-major n x n
    x: np.ndarray | None = None   # float32 [n, d] source coordinates (on-the-fly cost)
    y: np.ndarray | None = None   # float32 [n, d] target coordinates
    scale: float = 1.0            # s = fl32(1 / max D)
    kind: str = "l2sq"
    seed: int = 0


def grid_problem(k: int, seed: int, kind: str = "l2sq", dtype=np.float32, dense: bool = True) -> Problem:
    """Grid-histogram OT problem: r and c from independent draws (seeds 2*seed, 2*seed+1)."""
    r = grid_histogram(k, 2 * seed)
    c = grid_histogram(k, 2 * seed + 1)
    C = grid_cost(k, kind, dtype) if dense else None
    xy = grid_coords(k)
    return Problem(n=k * k, r=r, c=c, C=C, x=xy, y=xy.copy(),
                   scale=float(grid_cost_scale(k, kind)), kind=kind, seed=seed)


def _point_raw(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    x = x.astype(np.float32)
    y = y.astype(np.float32)
    d0 = x[:, None, 0] - y[None, :, 0]
    d1 = x[:, None, 1] - y[None, :, 1]
    d2 = x[:, None, 2] - y[None, :, 2]
    return (d0 * d0 + d1 * d1) + d2 * d2            # float32 ops, left to right


def point_cost(x: np.ndarray, y: np.ndarray, scale: np.float32) -> np.ndarray:
    return (_point_raw(x, y) * np.float32(scale)).astype(np.float32)


def point_cloud_problem(n: int, seed: int, dense: bool = True) -> Problem:
    """Point-cloud problem: x_i ~ N(0, I_3), y_j ~ U[-1, 1]^3 (float32), uniform weights,
    C = squared Euclidean distance / max (App. C style point clouds)."""
    rng = rng_for(seed)
    x = rng.standard_normal((n, 3)).astype(np.float32)
    y = rng.uniform(-1.0, 1.0, size=(n, 3)).astype(np.float32)
    raw = _point_raw(x, y)
    s = np.float32(1.0 / float(raw.max()))
    C = (raw * s).astype(np.float32) if dense else None
    w = np.full(n, 1.0 / n, dtype=np.float64)
    return Problem(n=n, r=w, c=w.copy(), C=C, x=x, y=y, scale=float(s), kind="points_l2sq", seed=seed)


def line_problem(n: int, seed: int, dense: bool = False) -> Problem:
    """Points on a line, for sizes where no n x n matrix is formed: x_i ~ U[0, 1], y_j ~ U[0.25, 1.25]
    (float32, stored as 3-D coordinates (t, 0, 0)), weights r, c proportional to Gamma(2, 1) draws plus a
    1e-3 floor, C = squared distance / max.  On a line a convex cost makes the monotone
    (north-west corner on the sorted supports) coupling optimal, so the exact cost is known at any
    n.  The cost's maximum is attained at the ends of the two supports (float32 rounding is
    monotone), so the scale takes O(n) work."""
    rng = rng_for(seed)
    t = (rng.uniform(0.0, 1.0, size=(2, n)) + np.array([[0.0], [0.25]])).astype(np.float32)
    x = np.zeros((n, 3), dtype=np.float32)
    y = np.zeros((n, 3), dtype=np.float32)
    x[:, 0], y[:, 0] = t[0], t[1]
    wr = rng.gamma(2.0, 1.0, size=n) + 1e-3
    wc = rng.gamma(2.0, 1.0, size=n) + 1e-3
    r, c = wr / wr.sum(), wc / wc.sum()
    dmax = max(np.float32(t[0].max() - t[1].min()), np.float32(t[1].max() - t[0].min()))
    s = np.float32(1.0 / float(np.float32(dmax * dmax)))
    C = (_point_raw(x, y) * s).astype(np.float32) if dense else None
    return Problem(n=n, r=r, c=c, C=C, x=x, y=y, scale=float(s), kind="line_l2sq", seed=seed)


def _raw_cost(x: np.ndarray, y: np.ndarray, kind: str) -> np.ndarray:
    """Unscaled cost in float32, in the order the coordinate form computes it: squared distance
    (d0*d0 + d1*d1) + d2*d2 or L1 distance (|d0| + |d1|) + |d2|."""
    if kind == "l2sq":
        return _point_raw(x, y)
    x, y = x.astype(np.float32), y.astype(np.float32)
    return (np.abs(x[:, None, 0] - y[None, :, 0]) + np.abs(x[:, None, 1] - y[None, :, 1])) + \
        np.abs(x[:, None, 2] - y[None, :, 2])


def entropy_problem(n: int, frac: float, seed: int, kind: str = "l2sq", dense: bool = False) -> Problem:
    """App. C's controlled-entropy problems: r with H(r) = frac * log n, c uniform (so H_min = H(r)),
    cost between n points x_i ~ N(0, I_3) and themselves, ||x_i - x_j||^2 or ||x_i - x_j||_1,
    divided by its maximum.  Reading of "a Dirichlet draw constructed to meet a target entropy":
    r proportional to U_i^beta with U_i ~ U(0, 1) (the small-concentration limit of a symmetric
    Dirichlet draw, whose Gamma(a) components behave like U^(1/a)), beta found by bisection so that
    H(r) matches the target to 1e-9 relative (H decreases monotonically in beta)."""
    rng = rng_for(seed)
    x = rng.standard_normal((n, 3)).astype(np.float32)
    U = rng.uniform(0.0, 1.0, size=n)
    target = frac * math.log(n)

    def dist(beta):
        with np.errstate(divide="ignore", under="ignore"):
            lw = beta * np.log(U)
        w = np.exp(lw - lw.max())
        return w / w.sum()

    def ent(r):
        nz = r[r > 0]
        return float(-(nz * np.log(nz)).sum())

    lo, hi = 0.0, 1.0
    while ent(dist(hi)) > target:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if ent(dist(mid)) > target:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-12 * hi:
            break
    r = dist(0.5 * (lo + hi))
    c = np.full(n, 1.0 / n)
    mx = np.float32(0.0)
    for i0 in range(0, n, 512):                      # max over all pairs, in row blocks
        mx = max(mx, _raw_cost(x[i0:i0 + 512], x, kind).max())
    s = np.float32(1.0 / float(mx))
    C = (_raw_cost(x, x, kind) * s).astype(np.float32) if dense else None
    return Problem(n=n, r=r, c=c, C=C, x=x, y=x.copy(), scale=float(s), kind=f"entropy_{kind}", seed=seed)


def batch_sizes(count: int, seed: int, lo: int = 256, hi: int = 4096) -> np.ndarray:
    """Problem sizes for the batched workload: n uniform on [lo, hi]."""
    return rng_for(seed).integers(lo, hi + 1, size=count)


def serving_trace(count: int, seed: int, rate: float = 200.0, n_lo: int = 128, n_hi: int = 8192,
                  gaps=(1e-4, 1e-5, 1e-6, 1e-7)):
    """Poisson arrivals (mean `rate`/s); n log-uniform on [n_lo, n_hi] rounded to the nearest
    square grid k*k (k*k <= n_hi); target gap uniform over `gaps`.  Returns a list of
    (t_arrival, k, eps, seed)."""
    rng = rng_for(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    n = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count))
    k = np.clip(np.rint(np.sqrt(n)), 2, math.isqrt(n_hi)).astype(int)      # n = k^2 stays <= n_hi
    eps = rng.choice(np.asarray(gaps), size=count)
    return [(float(t[i]), int(k[i]), float(eps[i]), int(seed * 100000 + i)) for i in range(count)]
