"""The squared-Euclidean cost of integer grid points on the tensor cores (mma.sync, bf16 inputs,
fp32 accumulation; mdot_params.tensor_cores / MDOT_PREC_TENSOR_CORES): |x|^2 + |y|^2 - 2 <x, y>
is exact for integer coordinates of magnitude <= 255, so the regenerated C has the bits of the
dense matrix the generator builds (inputs.grid_cost), and the solver on the regenerated cost
matches the CPU oracle on that matrix.  Points that are not such integers take the fp32 form (its
bits equal inputs.point_cost's)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2307_08507_gb300 as M
from paper_2307_08507_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]
DEV = "cuda:0"


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("k", [2, 5, 16, 45, 64, 128])
def test_grid_cost_bits_equal_the_dense_matrix(k):
    """Every entry, n = 4 ... 16384 (ragged tiles at k = 2, 5 and 45)."""
    torch.cuda.set_device(0)
    xy = t(I.coords3(I.grid_coords(k)))
    s = float(I.grid_cost_scale(k, "l2sq"))
    C = M.cost_matrix(xy, xy, M.COST_SQEUCLID, s)
    ref = I.grid_cost(k, "l2sq")
    assert torch.equal(C.cpu(), torch.from_numpy(ref))


def test_shifted_and_negative_integer_points_and_the_fp32_form():
    """Integer points with negative coordinates and |x| up to 255 (tensor cores), and the same
    points moved by half a unit (fp32 form): both against the generator's fp32 formula."""
    torch.cuda.set_device(0)
    rng = np.random.default_rng(3)
    x = rng.integers(-255, 256, size=(700, 3)).astype(np.float32)
    y = rng.integers(-255, 256, size=(700, 3)).astype(np.float32)
    for dx in (0.0, 0.5):
        xs, ys = x + np.float32(dx), y
        raw = I._point_raw(xs, ys)
        s = np.float32(1.0 / float(raw.max()))
        C = M.cost_matrix(t(xs), t(ys), M.COST_SQEUCLID, float(s))
        assert torch.equal(C.cpu(), torch.from_numpy(I.point_cost(xs, ys, s)))


def test_regenerated_grid_solve_uses_the_tensor_cores_and_matches_the_oracle():
    torch.cuda.set_device(0)
    p = I.grid_problem(24, 61)                       # n = 576: fp32 entries
    xy = t(I.coords3(p.x))
    gf = 2.0 ** 12
    tight = 1e-10
    with M.Handle(p.n) as h:
        u, v, res = h.solve_points(t(p.r), t(p.c), xy, xy, M.COST_SQEUCLID, p.scale, 1e-6,
                                   M.default_params(gamma_f=gf, final_tol=tight, tensor_cores=1))
        assert res.status == M.MDOT_OK and res.info.tensor_cores == 1
        ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, final_tol=tight)
        assert abs(res.cost - ref.cost) <= 1e-7, (res.cost, ref.cost)
        # the same problem from non-integer coordinates (the fp32 form): no tensor cores
        xs = t(I.coords3(p.x) * np.float32(0.5))
        _, _, r2 = h.solve_points(t(p.r), t(p.c), xs, xs, M.COST_SQEUCLID, p.scale * 4.0, 1e-6,
                                  M.default_params(gamma_f=gf, tensor_cores=1))
        assert r2.info.tensor_cores == 0
        # and the default: fp32 operations
        _, _, r3 = h.solve_points(t(p.r), t(p.c), xy, xy, M.COST_SQEUCLID, p.scale, 1e-6,
                                  M.default_params(gamma_f=gf, final_tol=tight))
        assert r3.info.tensor_cores == 0 and abs(r3.cost - ref.cost) <= 1e-7


@pytest.mark.parametrize("k,gamma", [(20, 2.0 ** 8), (64, 2.0 ** 14), (100, 2.0 ** 12)])
def test_tensor_core_dual_eval_matches_the_oracle(k, gamma):
    """Log-marginals of the tensor-core evaluation, every row and column, against the oracle on the
    dense matrix (fp32 and accurate fp32 tiers; n = 400, 4096, 10000)."""
    torch.cuda.set_device(0)
    p = I.grid_problem(k, 70 + k)
    xy = t(I.coords3(p.x))
    rng = np.random.default_rng(k)
    a = rng.uniform(0.0, 0.3, p.n)
    b = (p.C.astype(np.float64) - a[:, None]).min(axis=0)
    u = gamma * a + np.log(p.r)
    v = gamma * b + np.log(p.c)
    lr_o, lc_o = O.dual_eval(p.C.astype(np.float64), u, v, gamma)
    with M.Handle(p.n) as h:
        for prec, tol in ((M.PREC_FP32, 4e-6), (M.PREC_FP32A, 1e-6)):
            tc = prec | M.PREC_TENSOR_CORES
            lr, lc = h.dual_eval_points(t(u), t(v), gamma, xy, xy, M.COST_SQEUCLID, p.scale, precision=tc)
            np.testing.assert_allclose(lr.cpu().numpy(), lr_o, rtol=0, atol=tol)
            np.testing.assert_allclose(lc.cpu().numpy(), lc_o, rtol=0, atol=tol)
            lr2, lc2 = h.dual_eval_points(t(u), t(v), gamma, xy, xy, M.COST_SQEUCLID, p.scale, ref_log_rP=lr,
                                          precision=tc)
            np.testing.assert_allclose(lr2.cpu().numpy(), lr_o, rtol=0, atol=tol)
            np.testing.assert_allclose(lc2.cpu().numpy(), lc_o, rtol=0, atol=tol)
