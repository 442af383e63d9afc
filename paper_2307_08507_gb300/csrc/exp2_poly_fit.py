"""Minimax fit of the polynomial behind exp2_acc (mdot_device.cuh), reproducible on the CPU.

exp2_acc evaluates 2^x on the reduced range [-1/2, 1/2] as p(x) = 1 + c1 x + ... + c6 x^6 (p(0) = 1
held exactly, so 2^k stays exact at the integers).  The coefficients c1..c6 minimise the largest
RELATIVE error max |p(x) / 2^x - 1| on that range; they are found with the Remez exchange
algorithm (E. Remez, 1934; see e.g. Cheney, "Introduction to Approximation Theory", ch. 3):
  1. start from 7 Chebyshev points;
  2. solve the linear system  p(x_i) / 2^x_i - 1 = (-1)^i E  for c1..c6 and the level E;
  3. move the points to the 7 alternating extrema of the error curve (found on a fine grid) and
     repeat until the level E and the largest error agree.
Run as a script to print the coefficients rounded to float32 (as they are written in the CUDA
source) and the largest relative error of that float32 polynomial, evaluated in float64.
"""
from __future__ import annotations

import numpy as np

DEGREE = 6
LO, HI = -0.5, 0.5


def rel_error(c, x):
    """p(x) / 2^x - 1 in float64 for p(x) = 1 + sum_k c[k-1] x^k."""
    x = np.asarray(x, dtype=np.float64)
    p = np.zeros_like(x)
    for ck in reversed(c):
        p = (p + ck) * x
    return (1.0 + p) / np.exp2(x) - 1.0


def remez(degree: int = DEGREE, iters: int = 60, grid: int = 200000):
    """Coefficients c1..c_degree of the relative-minimax fit with p(0) = 1, and its error level.

    With p(0) = 1 the error e(x) = p(x) / 2^x - 1 = (x / 2^x) (q(x) - (2^x - 1) / x) has a forced
    zero at x = 0, where the weight x / 2^x changes sign; the equioscillation (alternation) is that
    of h(x) = sign(x) e(x) at degree + 1 points, none of them 0."""
    m = degree + 1                                  # alternation points: degree unknowns + E
    k = np.arange(m)
    x = np.linspace(LO, HI, m) + 0.013              # no point at 0
    x[-1] = HI
    fine = np.linspace(LO, HI, grid)                # an even count: 0 is not a grid point
    c, E = None, None
    for _ in range(iters):
        A = np.zeros((m, m))
        for j in range(1, degree + 1):
            A[:, j - 1] = x ** j
        A[:, degree] = -((-1.0) ** k) * np.sign(x) * np.exp2(x)
        b = np.exp2(x) - 1.0
        sol = np.linalg.solve(A, b)
        c, E = sol[:degree], sol[degree]
        h = np.sign(fine) * rel_error(c, fine)
        # alternating extrema of h: split the grid at its sign changes, keep each segment's peak
        sgn = np.sign(h)
        sgn[sgn == 0] = 1
        cuts = np.nonzero(np.diff(sgn))[0] + 1
        segs = np.split(np.arange(fine.size), cuts)
        peaks = [s[np.argmax(np.abs(h[s]))] for s in segs]
        if len(peaks) < m:
            break
        vals = np.abs(h[peaks])
        best = int(np.argmax(vals))
        start = min(max(0, best - m // 2), len(peaks) - m)
        x = fine[peaks[start:start + m]]
        if abs(np.abs(h).max() - abs(E)) <= 1e-9 * abs(E):
            break
    return c, abs(E)


def float32_coefficients(c):
    return [float(np.float32(ck)) for ck in c]


if __name__ == "__main__":
    c, E = remez()
    c32 = float32_coefficients(c)
    fine = np.linspace(LO, HI, 400001)
    print("Remez level E = %.3e" % E)
    for j, ck in enumerate(c32, start=1):
        print("c%d = %.8e" % (j, ck))
    print("max |p32(x) / 2^x - 1| on [-1/2, 1/2] = %.3e" % np.abs(rel_error(c32, fine)).max())
