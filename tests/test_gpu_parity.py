"""GPU parity of the C-ABI library against the CPU FP64 oracle, element by element on the same
seeded inputs.

Tolerances (derived from the arithmetic of each tier):
* fp32 entries: each entry carries the ex2.approx error (max 2^-22.7 relative, measured) plus
  ~2^-23 |t| from the exponent t = log2 P_ij - A_i; weighted by the entries themselves the
  relative error of a row or column sum stays below ~1.5e-6 (|t| averages <= log2 n + 1 under
  those weights) -> 4e-6 absolute on log-marginals.
* fp64 entries: a few ulps of the largest term -> 1e-11.
* rounded-plan cost: 1e-7 absolute on costs normalised to max C = 1 (the target tolerance).
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import paper_2307_08507_gb300 as M
from paper_2307_08507_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]

TOL_F32 = 4e-6
TOL_F32A = 1e-6     # accurate fp32 tier: ~1.3 ulp per entry, unbiased, exponent in double-float
TOL_F64 = 1e-11
DEV = "cuda:0"


@pytest.fixture(scope="module")
def h():
    torch.cuda.set_device(0)
    with M.Handle(4096) as handle:
        yield handle


def t(a, dtype=None):
    a = np.ascontiguousarray(a)
    return torch.from_numpy(a if dtype is None else a.astype(dtype)).to(DEV)


def rand_potentials(n, gamma, seed, C):
    """Potentials of a plausible iterate: u_i = gamma a_i + log r_i, v_j = -gamma min_i(C_ij - a_i)
    + log c_j with random a; every row and column then has entries of order r_i c_j."""
    rng = np.random.default_rng(seed)
    r = rng.uniform(0.2, 1.0, n); r /= r.sum()
    c = rng.uniform(0.2, 1.0, n); c /= c.sum()
    a = rng.uniform(0.0, 0.3, n)
    b = (C.astype(np.float64) - a[:, None]).min(axis=0)
    u = gamma * a + np.log(r)
    v = gamma * b + np.log(c)
    return u, v, r, c


@pytest.mark.parametrize("n", [1, 2, 3, 31, 33, 257, 1000, 4096])
@pytest.mark.parametrize("gamma", [1.0, 64.0, 4096.0, 65536.0])
@pytest.mark.parametrize("precision", [M.PREC_FP32, M.PREC_FP64, M.PREC_FP32A])
def test_dual_eval_matches_oracle(h, n, gamma, precision):
    rng = np.random.default_rng(n * 7 + int(math.log2(gamma)))
    C = rng.uniform(0, 1, (n, n)).astype(np.float32)
    u, v, _, _ = rand_potentials(n, gamma, n + 1, C)
    lr_o, lc_o = O.dual_eval(C.astype(np.float64), u, v, gamma)
    lr, lc = h.dual_eval(t(u), t(v), gamma, t(C), precision=precision)
    tol = {M.PREC_FP32: TOL_F32, M.PREC_FP32A: TOL_F32A, M.PREC_FP64: TOL_F64}[precision]
    np.testing.assert_allclose(lr.cpu().numpy(), lr_o, rtol=0, atol=tol * max(1.0, 1e-12 * np.abs(lr_o).max()))
    np.testing.assert_allclose(lc.cpu().numpy(), lc_o, rtol=0, atol=tol * max(1.0, 1e-12 * np.abs(lc_o).max()))
    # the solver path: scales taken from a previous estimate give the same marginals
    lr2, lc2 = h.dual_eval(t(u), t(v), gamma, t(C), ref_log_rP=lr, precision=precision)
    np.testing.assert_allclose(lr2.cpu().numpy(), lr_o, rtol=0, atol=tol)
    np.testing.assert_allclose(lc2.cpu().numpy(), lc_o, rtol=0, atol=tol)


@pytest.mark.parametrize("n", [1, 33, 1000, 4096])
@pytest.mark.parametrize("gamma", [64.0, 65536.0])
@pytest.mark.parametrize("precision", [M.PREC_FP32, M.PREC_FP64, M.PREC_FP32A])
def test_dual_objective_matches_oracle(h, n, gamma, precision):
    """Eq. (4): g(u, v) = sum_ij P_ij - <u, r> - <v, c> from the same launch as the marginals,
    against the oracle's sum over every entry.  The fp64 sums of <u, r> and <v, c> are exact to
    n ulps of sum |u_i r_i| + sum |v_j c_j| at most; sum_i r(P)_i carries the per-tier relative error
    of the marginals (the log-marginal tolerances above), on both the one-pass and two-pass paths."""
    rng = np.random.default_rng(n * 3 + int(math.log2(gamma)))
    C = rng.uniform(0, 1, (n, n)).astype(np.float32)
    u, v, r, c = rand_potentials(n, gamma, n + 2, C)
    g_o = O.dual_value(C.astype(np.float64), u, v, gamma, r, c)
    scale = np.abs(u * r).sum() + np.abs(v * c).sum()
    rel = {M.PREC_FP32: TOL_F32, M.PREC_FP32A: TOL_F32A, M.PREC_FP64: TOL_F64}[precision]
    lr_o, _ = O.dual_eval(C.astype(np.float64), u, v, gamma)
    mass = np.exp(lr_o).sum()
    tol = rel * mass + 1e-12 * scale
    lr, lc, g = h.dual_eval(t(u), t(v), gamma, t(C), precision=precision, r=t(r), c=t(c))
    assert abs(g - g_o) <= tol, (g, g_o, tol)
    lr2, lc2, g2 = h.dual_eval(t(u), t(v), gamma, t(C), ref_log_rP=lr, precision=precision, r=t(r), c=t(c))
    assert abs(g2 - g_o) <= tol, (g2, g_o, tol)
    # the marginals of the same call are the ones of the call without g
    lr3, lc3 = h.dual_eval(t(u), t(v), gamma, t(C), ref_log_rP=lr, precision=precision)
    assert torch.equal(lr2, lr3) and torch.equal(lc2, lc3)


def test_dual_objective_needs_both_marginals(h):
    n = 8
    z = torch.zeros(n, dtype=torch.float64, device=DEV)
    C = torch.zeros((n, n), dtype=torch.float32, device=DEV)
    with pytest.raises(M.MdotError) as e:
        h.dual_eval(z, z, 1.0, C, r=z)
    assert e.value.status == M.MDOT_ERR_INVALID_ARG


def test_dual_eval_time_reports_the_kernel():
    """mdot_dual_eval_time: NOT_READY before any evaluation on the handle, then the device time of
    the last evaluation kernel (positive, below the host time of the whole call)."""
    import time
    torch.cuda.set_device(0)
    n = 512
    rng = np.random.default_rng(3)
    C = t(rng.uniform(0, 1, (n, n)).astype(np.float32))
    u = torch.zeros(n, dtype=torch.float64, device=DEV)
    with M.Handle(n) as hh:
        with pytest.raises(M.MdotError) as e:
            hh.dual_eval_time()
        assert e.value.status == M.MDOT_NOT_READY
        hh.dual_eval(u, u, 64.0, C)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hh.dual_eval(u, u, 64.0, C)
        wall = time.perf_counter() - t0
        ms = hh.dual_eval_time()
        assert 0.0 < ms < wall * 1e3


def test_dual_eval_huge_potentials(h):
    """Potentials of +-2000 (exp overflows without scaling): both log-marginals stay exact."""
    n, gamma = 64, 1e5
    rng = np.random.default_rng(4)
    C = rng.uniform(0, 1, (n, n)).astype(np.float32)
    u = rng.normal(size=n) + 2000.0
    v = rng.normal(size=n) - 2000.0
    lr_o, lc_o = O.dual_eval(C.astype(np.float64), u, v, gamma)
    for prec, tol in ((M.PREC_FP32, TOL_F32), (M.PREC_FP64, TOL_F64)):
        lr, lc = h.dual_eval(t(u), t(v), gamma, t(C), precision=prec)
        np.testing.assert_allclose(lr.cpu().numpy(), lr_o, rtol=1e-12, atol=tol)
        np.testing.assert_allclose(lc.cpu().numpy(), lc_o, rtol=1e-12, atol=tol)


def test_accurate_tier_removes_the_ex2_bias(h):
    """ex2.approx errs low by ~5e-8 on average, which biases every marginal; the accurate tier's
    polynomial exp2 is unbiased: its mean signed log-marginal error against the oracle is far
    smaller (n = 4096 grid at gamma = 2^16, every row and column)."""
    p = I.grid_problem(64, 2000)
    gamma = 2.0 ** 16
    u, v, _, _ = rand_potentials(p.n, gamma, 13, p.C)
    lr_o, lc_o = O.dual_eval(p.C.astype(np.float64), u, v, gamma)
    err = {}
    for prec in (M.PREC_FP32, M.PREC_FP32A):
        lr, lc = h.dual_eval(t(u), t(v), gamma, t(p.C), precision=prec)
        d = np.concatenate([lr.cpu().numpy() - lr_o, lc.cpu().numpy() - lc_o])
        err[prec] = (d.mean(), np.abs(d).max())
    assert abs(err[M.PREC_FP32A][0]) < 1e-8, err
    assert err[M.PREC_FP32A][1] < TOL_F32A, err
    assert abs(err[M.PREC_FP32A][0]) < abs(err[M.PREC_FP32][0]), err


def test_dual_eval_full_size_grid(h):
    """n = 4096 (64 x 64 grid, squared-L2 cost) at gamma = 2^14: every row and column."""
    p = I.grid_problem(64, 2000)
    gamma = 2.0 ** 14
    u, v, _, _ = rand_potentials(p.n, gamma, 11, p.C)
    lr_o, lc_o = O.dual_eval(p.C.astype(np.float64), u, v, gamma)
    lr, lc = h.dual_eval(t(u), t(v), gamma, t(p.C))
    np.testing.assert_allclose(lr.cpu().numpy(), lr_o, rtol=0, atol=TOL_F32)
    np.testing.assert_allclose(lc.cpu().numpy(), lc_o, rtol=0, atol=TOL_F32)


@pytest.mark.parametrize("n,gamma", [(1, 10.0), (3, 50.0), (33, 500.0), (256, 4096.0), (1000, 2.0 ** 15)])
def test_round_and_lower_bound_match_oracle(h, n, gamma):
    rng = np.random.default_rng(n)
    C = rng.uniform(0, 1, (n, n)).astype(np.float32)
    u, v, r, c = rand_potentials(n, gamma, n + 5, C)
    cost_o, G_o = O.round_plan(C.astype(np.float64), u, v, gamma, r, c, want_G=(n <= 256))
    cost, G = h.round(t(u), t(v), gamma, t(C), t(r), t(c), want_G=(n <= 256))
    assert abs(cost - cost_o) <= 1e-7 * max(1.0, cost_o), (cost, cost_o)
    if G is not None:
        Gn = G.cpu().numpy()
        assert (Gn >= 0).all()
        np.testing.assert_allclose(Gn.sum(1), r, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(Gn.sum(0), c, rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(Gn, G_o, rtol=0, atol=2e-6 * G_o.max())
    lb_o = O.ctransform_lb(C.astype(np.float64), u, gamma, r, c)
    lb = h.lower_bound(t(u), gamma, t(C), t(r), t(c))
    assert abs(lb - lb_o) <= 1e-12 * max(1.0, abs(lb_o)), (lb, lb_o)


def _solve_both(h, p, gamma_f, **kw):
    prm = M.default_params(gamma_f=gamma_f, **kw)
    u, v, res = h.solve(t(p.r), t(p.c), t(p.C), 1e-6, prm)
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gamma_f)
    return u.cpu().numpy(), v.cpu().numpy(), res, ref


@pytest.mark.parametrize("k,kind", [(12, "l2sq"), (16, "l2sq"), (16, "l1"), (32, "l2sq")])
def test_solve_matches_oracle(h, k, kind):
    """MDOT-PNCG end to end: rounded cost within 1e-7 of the oracle at the same gamma_f;
    potentials in cost units agree after fixing the additive shift."""
    p = I.grid_problem(k, 3 + k, kind=kind)
    gamma_f = 2.0 ** 14
    u, v, res, ref = _solve_both(h, p, gamma_f)
    assert res.status == M.MDOT_OK, M.status_string(res.status)
    assert abs(res.cost - ref.cost) <= 1e-7, (res.cost, ref.cost)
    assert res.info.grad_l1 <= ref.stage_log[-1, 1] / 2 * 1.0000001
    # potentials, shift fixed by sum_i u_i = 0 (footnote to Prop. 1), compared in cost units
    du = (u - u.mean()) - (ref.u - ref.u.mean())
    dv = (v + u.mean()) - (ref.v + ref.u.mean())
    assert np.abs(du).max() / gamma_f < 2e-4 and np.abs(dv).max() / gamma_f < 2e-4
    # certificate brackets the optimum and is consistent with the oracle's
    assert abs((res.cost - res.gap_cert) - ref.lb) <= 1e-6


def test_solve_fp64_tier_matches_oracle(h):
    """All-fp64 entries.  Rounding differs between the two sides, so line-search decisions near
    the Eq. (24) thresholds and the stopping point differ; both stop inside eps_d / 2 and the
    rounded costs agree to the target tolerance with similar work."""
    p = I.grid_problem(8, 5)
    gamma_f = 2.0 ** 12
    u, v, res, ref = _solve_both(h, p, gamma_f, precision=M.PREC_FP64)
    assert res.status == M.MDOT_OK
    assert res.info.evals_fp64 == res.info.evals
    assert abs(res.cost - ref.cost) <= 1e-7
    assert res.info.evals == pytest.approx(ref.stats.evals, rel=0.3)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_solve_tiny_problems(h, n):
    """n = 1 has H_min = 0 (a point mass): the floored tolerance still terminates."""
    rng = np.random.default_rng(n)
    C = rng.uniform(0, 1, (n, n)).astype(np.float32)
    r = np.full(n, 1.0 / n)
    u, v, res = h.solve(t(r), t(r), t(C), 1e-6, M.default_params(gamma_f=2.0 ** 12))
    ref = O.solve(C.astype(np.float64), r, r, gamma_f=2.0 ** 12)
    assert res.status == M.MDOT_OK
    assert abs(res.cost - ref.cost) <= 1e-7


def test_invalid_arguments_are_rejected(h):
    p = I.grid_problem(8, 1)
    bad_r = p.r.copy(); bad_r[0] = -1e-3; bad_r /= bad_r.sum()
    with pytest.raises(M.MdotError) as e:
        h.solve(t(bad_r), t(p.c), t(p.C), 1e-6)
    assert e.value.status == M.MDOT_ERR_INVALID_ARG
    with pytest.raises(M.MdotError) as e:
        h.solve(t(p.r * 1.01), t(p.c), t(p.C), 1e-6)
    assert e.value.status == M.MDOT_ERR_INVALID_ARG
    with pytest.raises(M.MdotError) as e:
        h.solve(t(p.r), t(p.c), t(p.C), -1.0)
    assert e.value.status == M.MDOT_ERR_INVALID_ARG
    # the handle still works after rejected calls
    u, v, res = h.solve(t(p.r), t(p.c), t(p.C), 1e-5)
    assert res.status == M.MDOT_OK


# Last-stage tolerances shared by the GPU and the oracle in the variant tests below, so that both
# stop at the same entropic optimum and the rounded costs must agree to the 1e-7 target:
# TIGHT where the GPU can finish in fp64 entries (AUTO: n <= 512, or the last fp32 stage polished
# in fp64), FLOOR (the fp32 floor, mdot_params.fp32_floor) where the tier is forced to fp32.
TIGHT, FLOOR = 1e-10, 2e-7


def _tol_for(prec):
    return TIGHT if prec in (M.PREC_AUTO, M.PREC_FP64) else FLOOR


@pytest.mark.parametrize("warm_start,smoothing,side,prec", [(1, 0, 16, 0), (0, 1, 16, 0), (1, 1, 16, 0),
                                                            (1, 0, 30, 3), (0, 1, 30, 3), (1, 1, 30, 0)])
def test_solve_ablation_variants_match_oracle(h, warm_start, smoothing, side, prec):
    """The ablation switches of Sec. 5 (eps-scaling instead of the Eq. (13) warm start; the
    smoothing weight fixed at its gamma_f value instead of eps_d), on the fp64 tier (n <= 512),
    on the accurate fp32 tier (a 30 x 30 grid) and on the automatic fp32 tiers with an fp64 last
    stage, against the oracle run with the same switch and the same last-stage tolerance."""
    p = I.grid_problem(side, 40 + warm_start + 3 * smoothing, kind="l2sq")
    gamma_f = 2.0 ** 12
    ft = _tol_for(prec)
    prm = M.default_params(gamma_f=gamma_f, warm_start=warm_start, smoothing=smoothing, precision=prec,
                           final_tol=ft)
    u, v, res = h.solve(t(p.r), t(p.c), t(p.C), 1e-6, prm)
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gamma_f, warm_start=warm_start, smoothing=smoothing,
                  final_tol=ft)
    assert res.status == M.MDOT_OK, M.status_string(res.status)
    assert res.info.grad_l1 <= ft
    assert abs(res.cost - ref.cost) <= 1e-7, (res.cost, ref.cost)
    assert res.info.stages == ref.stats.stages


@pytest.mark.parametrize("side,prec", [(16, 0), (30, 3)])
def test_solve_log_n_stopping_matches_oracle(h, side, prec):
    """App. C's comparison: log n in place of H_min in the stage tolerance eps_d, against the
    oracle run with the same switch (fp64 tier on a 16 x 16 grid, accurate fp32 tier on 30 x 30),
    the last stage at the shared tolerance; the stages before it stop at eps_d / 2 with log n."""
    p = I.grid_problem(side, 47, kind="l2sq")
    gamma_f = 2.0 ** 12
    ft = _tol_for(prec)
    prm = M.default_params(gamma_f=gamma_f, stop_entropy=1, precision=prec, final_tol=ft)
    u, v, res = h.solve(t(p.r), t(p.c), t(p.C), 1e-6, prm)
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gamma_f, stop_entropy=1, final_tol=ft)
    assert res.status == M.MDOT_OK, M.status_string(res.status)
    assert abs(res.cost - ref.cost) <= 1e-7, (res.cost, ref.cost)
    assert res.info.stages == ref.stats.stages
    assert res.info.grad_l1 <= ft
    # the switch is live: log n loosens every stage tolerance (App. C), fewer evaluations
    u1, v1, res1 = h.solve(t(p.r), t(p.c), t(p.C), 1e-6, M.default_params(gamma_f=gamma_f, precision=prec,
                                                                             final_tol=ft))
    assert res1.info.evals > res.info.evals


@pytest.mark.parametrize("side,prec", [(16, 0), (30, 3), (30, 0)])
def test_solve_diag_hessian_direction_matches_oracle(h, side, prec):
    """The diagonal-Hessian direction (Eq. (16), taken where every ratio r~/r(P), c~/c(P) lies in
    [0.01, 100], else the Sinkhorn direction) against the oracle run with the same variant: fp64
    tier (16 x 16), accurate fp32 tier (30 x 30), and the automatic tiers on 30 x 30 (the fast fp32
    tier for every stage tolerance above 2e-6, then the accurate tier and an fp64 last stage) --
    the barrier-synchronised stage kernel on each."""
    p = I.grid_problem(side, 48 + prec, kind="l2sq")
    gamma_f = 2.0 ** 12
    ft = _tol_for(prec)
    prm = M.default_params(gamma_f=gamma_f, precond=1, precision=prec, final_tol=ft)
    u, v, res = h.solve(t(p.r), t(p.c), t(p.C), 1e-6, prm)
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gamma_f, precond=1, final_tol=ft)
    assert res.status == M.MDOT_OK, M.status_string(res.status)
    assert abs(res.cost - ref.cost) <= 1e-7, (res.cost, ref.cost)
    assert res.info.stages == ref.stats.stages
    if side == 16:
        # same decisions as the oracle up to rounding: iteration counts agree closely
        assert abs(res.info.iters - ref.stats.iters) <= 0.02 * ref.stats.iters + ref.stats.stages
    # the plain direction on the same problem takes a different path (the switch is live)
    u0, v0, res0 = h.solve(t(p.r), t(p.c), t(p.C), 1e-6, M.default_params(gamma_f=gamma_f, precision=prec,
                                                                             final_tol=ft))
    assert res0.info.evals != res.info.evals


def test_diag_hessian_direction_regenerated_cost(h):
    p = I.point_cloud_problem(600, 4601)
    gf = 2.0 ** 11
    prm = M.default_params(gamma_f=gf, precond=1, final_tol=TIGHT)
    u, v, res = h.solve_points(t(p.r), t(p.c), t(p.x), t(p.y), M.COST_SQEUCLID, p.scale, 1e-6, prm)
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, precond=1, final_tol=TIGHT)
    assert res.status == M.MDOT_OK, M.status_string(res.status)
    assert abs(res.cost - ref.cost) <= 1e-7, (res.cost, ref.cost)
