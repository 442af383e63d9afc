"""On-the-fly cost (C regenerated from coordinates inside every pass): parity with the dense path
and with the CPU oracle run on the materialised matrix (the inputs module builds it with the same
fp32 operations, so both sides solve the identical problem)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2307_08507_gb300 as M
from paper_2307_08507_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]
DEV = "cuda:0"
TOL_F32 = 4e-6


@pytest.fixture(scope="module")
def h():
    torch.cuda.set_device(0)
    with M.Handle(4096) as handle:
        yield handle


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("kind,k", [("l2sq", 20), ("l1", 20), ("l2sq", 33)])
def test_dual_eval_points_matches_dense_and_oracle(h, kind, k):
    p = I.grid_problem(k, 5, kind=kind)
    xy = I.coords3(p.x)
    gamma = 2.0 ** 10
    rng = np.random.default_rng(k)
    u = np.log(p.r) + rng.normal(size=p.n)
    v = np.log(p.c) + rng.normal(size=p.n)
    ck = M.COST_SQEUCLID if kind == "l2sq" else M.COST_L1
    lr_o, lc_o = O.dual_eval(p.C.astype(np.float64), u, v, gamma)
    for prec, tol in ((M.PREC_FP32, TOL_F32), (M.PREC_FP32A, 1e-6), (M.PREC_FP64, 1e-11)):
        lr, lc = h.dual_eval_points(t(u), t(v), gamma, t(xy), t(xy), ck, p.scale, precision=prec)
        np.testing.assert_allclose(lr.cpu().numpy(), lr_o, rtol=0, atol=tol)
        np.testing.assert_allclose(lc.cpu().numpy(), lc_o, rtol=0, atol=tol)
        lr2, lc2 = h.dual_eval_points(t(u), t(v), gamma, t(xy), t(xy), ck, p.scale, ref_log_rP=lr, precision=prec)
        np.testing.assert_allclose(lr2.cpu().numpy(), lr_o, rtol=0, atol=tol)
        np.testing.assert_allclose(lc2.cpu().numpy(), lc_o, rtol=0, atol=tol)


@pytest.mark.parametrize("kind", ["l2sq", "l1"])
def test_solve_points_grid_matches_oracle(h, kind):
    p = I.grid_problem(16, 9, kind=kind)
    xy = I.coords3(p.x)
    ck = M.COST_SQEUCLID if kind == "l2sq" else M.COST_L1
    gf = 2.0 ** 13
    prm = M.default_params(gamma_f=gf)
    u, v, res = h.solve_points(t(p.r), t(p.c), t(xy), t(xy), ck, p.scale, 1e-6, prm)
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf)
    assert res.status == M.MDOT_OK
    # both solvers stop anywhere inside ||grad g||_1 <= eps_d / 2; rounding moves the plan by at
    # most 2 ||grad g||_1 in L1 (Altschuler's bound) and C lies in [0, 1], so the rounded costs
    # can differ by about the sum of the two tolerances, eps_d (plus the 1e-7 target)
    eps_d = res.info.H_min / gf ** 1.5
    assert abs(res.cost - ref.cost) <= max(1e-7, eps_d), (res.cost, ref.cost, eps_d)
    # and with the dense matrix through mdot_solve
    u2, v2, res2 = h.solve(t(p.r), t(p.c), t(p.C), 1e-6, prm)
    assert abs(res.cost - res2.cost) <= max(1e-7, eps_d)


def test_solve_points_point_cloud_matches_oracle(h):
    """App. C style point cloud: x ~ N(0, I3), y ~ U[-1, 1]^3, uniform weights, n = 600 (fp32
    entries: n > 512)."""
    p = I.point_cloud_problem(600, 4001)
    gf = 2.0 ** 12
    prm = M.default_params(gamma_f=gf)
    u, v, res = h.solve_points(t(p.r), t(p.c), t(p.x), t(p.y), M.COST_SQEUCLID, p.scale, 1e-6, prm)
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf)
    assert res.status == M.MDOT_OK
    eps_d = res.info.H_min / gf ** 1.5          # see test_solve_points_grid_matches_oracle
    assert abs(res.cost - ref.cost) <= max(1e-7, eps_d), (res.cost, ref.cost, eps_d)
    assert res.gap_cert >= -1e-12
