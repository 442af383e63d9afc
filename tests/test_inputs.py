"""CPU checks of the seeded input generators that the oracle, the GPU tests and the benchmark
share (paper_2307_08507_gb300/inputs.py): determinism, marginals in the simplex, costs in [0, 1]
with the fp32 arithmetic the coordinate form uses, the controlled-entropy target of App. C, and
the shapes of the batched and served workloads."""
import math

import numpy as np

from paper_2307_08507_gb300 import inputs as I


def test_grid_problem_is_seeded_and_in_the_simplex():
    a, b = I.grid_problem(12, 7), I.grid_problem(12, 7)
    assert np.array_equal(a.r, b.r) and np.array_equal(a.c, b.c) and np.array_equal(a.C, b.C)
    assert not np.array_equal(a.r, a.c)                          # r and c are independent draws
    for w in (a.r, a.c):
        assert abs(w.sum() - 1.0) <= 1e-12 and w.min() > 0.0
    assert not np.array_equal(I.grid_problem(12, 8).r, a.r)


def test_grid_cost_is_the_scaled_integer_distance():
    """C_ij = fl32(D_ij fl32(1 / max D)) with D the exact integer cell distance; symmetric, zero
    diagonal, maximum 1 (both costs)."""
    k = 9
    xy = I.grid_coords(k).astype(np.int64)
    for kind in ("l2sq", "l1"):
        C = I.grid_cost(k, kind)
        d = xy[:, None, :] - xy[None, :, :]
        D = (d * d).sum(-1) if kind == "l2sq" else np.abs(d).sum(-1)
        s = np.float32(1.0 / float(D.max()))
        assert np.array_equal(C, (D.astype(np.float32) * s).astype(np.float32))
        assert np.array_equal(C, C.T) and not C.diagonal().any()
        assert C.max() == np.float32(float(D.max())) * s
        assert I.grid_cost_scale(k, kind) == s


def test_point_cost_keeps_the_fp32_operation_order():
    """The dense point-cloud cost equals (d0 d0 + d1 d1) + d2 d2 times s, each step rounded to
    fp32, the order the regenerated cost uses."""
    p = I.point_cloud_problem(50, 3)
    x, y = p.x, p.y
    d = [(x[:, None, q] - y[None, :, q]).astype(np.float32) for q in range(3)]
    D = ((d[0] * d[0]).astype(np.float32) + (d[1] * d[1]).astype(np.float32)).astype(np.float32)
    D = (D + (d[2] * d[2]).astype(np.float32)).astype(np.float32)
    assert np.array_equal(p.C, (D * np.float32(p.scale)).astype(np.float32))
    assert p.C.max() <= 1.0 and p.C.min() >= 0.0
    assert np.allclose(p.r, 1.0 / 50) and np.allclose(p.c, 1.0 / 50)


def test_line_problem_scale_is_the_maximum_of_the_dense_cost():
    """The O(n) scale of the points-on-a-line problem equals 1 / max over all pairs."""
    p = I.line_problem(300, 11)
    dense = I.line_problem(300, 11, dense=True)
    raw = I._point_raw(dense.x, dense.y)
    assert dense.C.max() == np.float32(float(raw.max())) * np.float32(p.scale)
    assert abs(float(dense.C.max()) - 1.0) <= 1e-7
    assert abs(p.r.sum() - 1.0) <= 1e-12 and abs(p.c.sum() - 1.0) <= 1e-12


def test_entropy_problem_meets_its_target():
    """App. C reading: H(r) = frac log n to 1e-9 relative, c uniform, C symmetric in [0, 1]."""
    n = 400
    for frac in (0.03, 0.3, 0.9):
        p = I.entropy_problem(n, frac, 5, dense=True)
        nz = p.r[p.r > 0]
        H = float(-(nz * np.log(nz)).sum())
        assert abs(H - frac * math.log(n)) <= 1e-9 * frac * math.log(n), (frac, H)
        assert np.allclose(p.c, 1.0 / n)
        assert np.array_equal(p.C, p.C.T) and abs(float(p.C.max()) - 1.0) <= 1e-7


def test_batch_sizes_and_serving_trace():
    sizes = I.batch_sizes(512, 4000)
    assert sizes.min() >= 256 and sizes.max() <= 4096 and len(sizes) == 512
    assert np.array_equal(sizes, I.batch_sizes(512, 4000))
    trace = I.serving_trace(400, 5000)
    t = np.array([q[0] for q in trace])
    ks = np.array([q[1] for q in trace])
    assert np.all(np.diff(t) > 0.0)                               # arrivals in order
    assert abs(len(trace) / t[-1] - 200.0) <= 40.0                # Poisson rate 200/s
    assert (ks * ks).max() <= 8192 and ks.min() >= 2
    assert {q[2] for q in trace} <= {1e-4, 1e-5, 1e-6, 1e-7}
    assert len({q[3] for q in trace}) == len(trace)               # one problem seed per request
    assert trace == I.serving_trace(400, 5000)
