"""Pins for the CPU FP64 oracle: each check compares the oracle with something other than itself
(closed forms, finite differences, identities proved in the paper, exact LP optima, brute force),
chosen so that a dropped term, a wrong sign or a transposed operand fails at least one."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import exact as E
from paper_2307_08507_gb300 import inputs as I


def _rand_problem(n, seed, kind="rand"):
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, (n, n))
    r = rng.uniform(0.2, 1, n); r /= r.sum()
    c = rng.uniform(0.2, 1, n); c /= c.sum()
    return C, r, c


# ---------------------------------------------------------------------------------------------
# Dual evaluation, Eq. (2)-(4) and the two reductions of Alg. 2
# ---------------------------------------------------------------------------------------------

def test_gradient_matches_finite_differences_of_dual():
    """grad g = (r(P) - r, c(P) - c) (Eq. (4)) vs central differences of g (Eq. (4))."""
    n, gamma = 6, 3.0
    C, r, c = _rand_problem(n, 1)
    rng = np.random.default_rng(2)
    u, v = rng.normal(size=n) - 2, rng.normal(size=n) - 2
    lr, lc = O.dual_eval(C, u, v, gamma)
    grad = np.concatenate([np.exp(lr) - r, np.exp(lc) - c])
    h = 1e-6
    fd = np.empty(2 * n)
    for a in range(2 * n):
        e = np.zeros(2 * n); e[a] = h
        gp = O.dual_value(C, u + e[:n], v + e[n:], gamma, r, c)
        gm = O.dual_value(C, u - e[:n], v - e[n:], gamma, r, c)
        fd[a] = (gp - gm) / (2 * h)
    np.testing.assert_allclose(grad, fd, rtol=0, atol=1e-8)


def test_dual_eval_separable_cost_closed_form():
    """C_ij = a_i + b_j makes P rank one: log r(P)_i = u_i - gamma a_i + log sum_j exp(v_j - gamma b_j)."""
    n, gamma = 9, 7.5
    rng = np.random.default_rng(3)
    a, b = rng.uniform(0, 0.5, n), rng.uniform(0, 0.5, n)
    C = a[:, None] + b[None, :]
    u, v = rng.normal(size=n), rng.normal(size=n)
    lr, lc = O.dual_eval(C, u, v, gamma)
    row_const = math.log(np.exp(v - gamma * b).sum())
    col_const = math.log(np.exp(u - gamma * a).sum())
    np.testing.assert_allclose(lr, u - gamma * a + row_const, rtol=0, atol=1e-12)
    np.testing.assert_allclose(lc, v - gamma * b + col_const, rtol=0, atol=1e-12)


def test_dual_eval_is_stabilised_for_huge_potentials():
    """Potentials of +-2000 overflow exp() without the max shift; the separable closed form
    still holds exactly in log space."""
    n, gamma = 5, 1e5
    rng = np.random.default_rng(4)
    a, b = rng.uniform(0, 0.01, n), rng.uniform(0, 0.01, n)
    C = a[:, None] + b[None, :]
    u, v = rng.normal(size=n) + 2000.0, rng.normal(size=n) - 2000.0
    lr, lc = O.dual_eval(C, u, v, gamma)
    z = v - gamma * b
    zm = z.max()
    np.testing.assert_allclose(lr, u - gamma * a + zm + math.log(np.exp(z - zm).sum()), rtol=1e-14)
    assert np.isfinite(lc).all()


def test_shift_invariance():
    """g(u + d1, v - d1) = g(u, v) (footnote to Prop. 1): P and both marginals are unchanged,
    while a one-sided shift u + d scales r(P) and c(P) by e^d."""
    n, gamma = 7, 11.0
    C, r, c = _rand_problem(n, 5)
    rng = np.random.default_rng(6)
    u, v = rng.normal(size=n) - 2, rng.normal(size=n) - 2
    d = 0.37
    lr, lc = O.dual_eval(C, u, v, gamma)
    lr2, lc2 = O.dual_eval(C, u + d, v - d, gamma)
    np.testing.assert_allclose(lr2, lr, atol=1e-13)
    np.testing.assert_allclose(lc2, lc, atol=1e-13)
    lr3, lc3 = O.dual_eval(C, u + d, v, gamma)
    np.testing.assert_allclose(lr3, lr + d, atol=1e-13)
    np.testing.assert_allclose(lc3, lc + d, atol=1e-13)
    assert abs(O.dual_value(C, u, v, gamma, r, c) - O.dual_value(C, u + d, v - d, gamma, r, c)) < 1e-13


def _kl(a, b):
    """Paper's KL: <a, log(a/b)> + <b - a, 1>."""
    return float(np.sum(a * np.log(a / b)) + np.sum(b - a))


def test_sinkhorn_direction_descent_identity():
    """Sec. 4: -<s, grad g> = KL(r(P)|r) + KL(r|r(P)) + KL(c(P)|c) + KL(c|c(P)) > 0."""
    n, gamma = 8, 5.0
    C, r, c = _rand_problem(n, 7)
    rng = np.random.default_rng(8)
    u, v = rng.normal(size=n) - 2, rng.normal(size=n) - 2
    lr, lc = O.dual_eval(C, u, v, gamma)
    rP, cP = np.exp(lr), np.exp(lc)
    s = np.concatenate([np.log(r) - lr, np.log(c) - lc])
    grad = np.concatenate([rP - r, cP - c])
    rhs = _kl(rP, r) + _kl(r, rP) + _kl(cP, c) + _kl(c, cP)
    assert rhs > 0
    assert abs(-float(s @ grad) - rhs) < 1e-12 * max(1.0, rhs)


# ---------------------------------------------------------------------------------------------
# Projections: Alg. 2 (PNCG) and Alg. 4 (Sinkhorn)
# ---------------------------------------------------------------------------------------------

def test_pncg_and_sinkhorn_reach_the_same_plan():
    """At fixed gamma the EOT plan P*(gamma) is unique (Sec. 2.1): both projectors agree."""
    n, gamma = 12, 40.0
    C, r, c = _rand_problem(n, 9)
    u0, v0 = np.log(r), np.log(c)
    u1, v1, rc1, st1, lr1, lc1 = O.pncg(C, gamma, r, c, 1e-13, u0, v0)
    u2, v2, rc2, st2, lr2 = O.sinkhorn(C, gamma, r, c, 1e-13, u0, v0)
    assert rc1 == 0 and rc2 == 0
    P1 = np.exp(u1[:, None] + v1[None, :] - gamma * C)
    P2 = np.exp(u2[:, None] + v2[None, :] - gamma * C)
    np.testing.assert_allclose(P1, P2, atol=1e-12)
    np.testing.assert_allclose(P1.sum(1), r, atol=1e-13)
    np.testing.assert_allclose(P1.sum(0), c, atol=1e-13)
    # PNCG is the faster projector (Fig. 4): fewer LSE passes than Sinkhorn here
    assert st1.evals < st2.half_evals / 2 + 1


def test_sinkhorn_column_residual_is_zero():
    """The column update of Alg. 4 sets v so that c(P) = c exactly after every iteration."""
    n, gamma = 10, 25.0
    C, r, c = _rand_problem(n, 10)
    u, v, rc, st, lr = O.sinkhorn(C, gamma, r, c, 1e-6, np.zeros(n), np.zeros(n))
    _, lc = O.dual_eval(C, u, v, gamma)
    np.testing.assert_allclose(np.exp(lc), c, rtol=1e-13)


def test_pncg_decreases_the_dual_monotonically():
    """Every accepted line-search step satisfies the approximate Wolfe conditions (Eq. (24)),
    so the dual objective never increases along the PNCG iterates."""
    n, gamma = 16, 60.0
    C, r, c = _rand_problem(n, 11)
    u, v = np.log(r), np.log(c)
    vals = [O.dual_value(C, u, v, gamma, r, c)]
    for k in range(1, 12):
        uk, vk, rc, st, _, _ = O.pncg(C, gamma, r, c, 0.0, u, v, max_iter=k)
        vals.append(O.dual_value(C, uk, vk, gamma, r, c))
    assert all(b <= a + 1e-15 for a, b in zip(vals, vals[1:]))
    assert vals[-1] < vals[0]


def test_line_search_trials_per_iteration_in_paper_range():
    """App. B reports 1.5-2.5 phi' evaluations per PNCG iteration on average: so does the line
    search with a first trial step of 1 (ls_init 0).  Starting each line search from the previous
    accepted step (ls_init 1, the default; App. B leaves the first trial open) takes fewer trials
    per iteration and fewer evaluations overall, and reaches the same plan cost to within the
    stage tolerance."""
    for k, seed in ((8, 3), (12, 4), (10, 5)):
        p = I.grid_problem(k, seed)
        gf = 2.0 ** 12
        r0 = O.solve(p.C, p.r, p.c, gamma_f=gf, ls_init=0)
        r1 = O.solve(p.C, p.r, p.c, gamma_f=gf, ls_init=1)
        q0 = r0.stats.ls_trials / r0.stats.iters
        q1 = r1.stats.ls_trials / r1.stats.iters
        assert 1.5 <= q0 <= 2.5, q0
        assert 1.0 <= q1 < q0, (q1, q0)
        assert r1.stats.evals < r0.stats.evals
        H = min(O.entropy(p.r), O.entropy(p.c))
        assert abs(r1.cost - r0.cost) <= H / gf ** 1.5, (r1.cost, r0.cost)


def test_line_search_hybrid_step_on_a_linear_derivative():
    """App. B on phi'(alpha) = alpha - 2.6 (a quadratic phi), with a narrow acceptance window
    (c1 = 0.49, c2 = 0.01: accept iff -0.026 <= phi'(alpha) <= 0.052).  Worked by hand: trials 1 and
    2 raise the lower end and double; 4 overshoots; inside the bracket every secant root is the
    exact root 2.6, so each next trial is alpha_hyb = 2.6 / 2 + (lo + hi) / 4 (Eq. (25)):
      lo = 2,   hi = 4   -> 2.8   (phi' = 0.2:   new upper end)
      lo = 2,   hi = 2.8 -> 2.5   (phi' = -0.1:  new lower end)
      lo = 2.5, hi = 2.8 -> 2.625 (phi' = 0.025: accepted).
    A pure secant step would stop at 2.6 after four trials, a pure bisection would try 3.0 fourth;
    a sign slip in the secant root sends the fourth trial to 1.6."""
    rc, alpha, trials, lows = O.ls_search(lambda a: a - 2.6, -2.6, 1.0, ls_c1=0.49, ls_c2=0.01)
    assert rc == 0
    assert trials == pytest.approx([1.0, 2.0, 4.0, 2.8, 2.5, 2.625], rel=1e-12, abs=1e-12)
    assert lows == pytest.approx([1.0, 2.0, 2.5], rel=1e-12)
    assert alpha == pytest.approx(2.625, rel=1e-12)


def test_line_search_cap_bisection_and_no_descent():
    """The readings around Eq. (24): after ls_max_trials the lower end is taken (rc 1); a
    non-finite phi' counts as an upper end and the next trial bisects; a non-negative phi'(0) is
    no descent direction (rc 2, no evaluation)."""
    rc, alpha, trials, lows = O.ls_search(lambda a: a - 2.6, -2.6, 1.0, ls_c1=0.49, ls_c2=0.01, ls_max_trials=3)
    assert rc == 1 and alpha == 2.0 and trials == [1.0, 2.0, 4.0] and lows == [1.0, 2.0]
    # phi' overflows beyond alpha = 5: the first trial 8 is an upper end, then (0 + 8) / 2 = 4 is
    # accepted (c1 = 0.1, c2 = 0.5, phi'(0) = -2.6: accept iff -1.3 <= phi' <= 2.08; phi'(4) = -0.5)
    rc, alpha, trials, _ = O.ls_search(lambda a: (a - 4.5) if a <= 5.0 else float("inf"), -2.6, 8.0)
    assert rc == 0 and trials == [8.0, 4.0] and alpha == 4.0
    rc, alpha, trials, _ = O.ls_search(lambda a: a, 0.0, 1.0)
    assert rc == 2 and trials == []


def test_diag_hessian_variant_converges_to_same_plan():
    n, gamma = 10, 30.0
    C, r, c = _rand_problem(n, 12)
    u1, v1, rc1, *_ = O.pncg(C, gamma, r, c, 1e-12, np.log(r), np.log(c), precond=0)
    u2, v2, rc2, *_ = O.pncg(C, gamma, r, c, 1e-12, np.log(r), np.log(c), precond=1)
    P1 = np.exp(u1[:, None] + v1[None, :] - gamma * C)
    P2 = np.exp(u2[:, None] + v2[None, :] - gamma * C)
    np.testing.assert_allclose(P1, P2, atol=1e-11)


# ---------------------------------------------------------------------------------------------
# MDOT (Alg. 1), Prop. 1, Eq. (13)
# ---------------------------------------------------------------------------------------------

def test_taylor_warm_start_tracks_linear_dual_paths():
    """For C_ij = a_i + b_j and fixed smoothing, u*(gamma) = log r~ - gamma a + const is linear in
    gamma, so the finite-difference step of Eq. (13) (from z^(0) = (log r~, log c~) at gamma = 0)
    predicts the next optimum exactly: a stage then starts at the previous stage's residual level.
    eps-scaling and no warm start start far away."""
    n = 10
    rng = np.random.default_rng(13)
    a, b = rng.uniform(0, 0.5, n), rng.uniform(0, 0.5, n)
    C = a[:, None] + b[None, :]
    r = rng.uniform(0.2, 1, n); r /= r.sum()
    c = rng.uniform(0.2, 1, n); c /= c.sum()
    logs = {}
    for ws in (0, 1, 2):
        u, v, rc, st, log = O.mdot(C, r, c, gamma_f=2.0 ** 10, smoothing=1, warm_start=ws)
        assert rc == 0
        logs[ws] = log
    def start_vs_prev_tol(log):
        return log[1:, 5] / (log[:-1, 1] / 2)
    # the stage starts within a small multiple of the previous stage's tolerance eps_d / 2 ...
    assert (start_vs_prev_tol(logs[0]) < 3.0).all(), start_vs_prev_tol(logs[0])
    # ... while eps-scaling and a cold start begin orders of magnitude further away
    assert (start_vs_prev_tol(logs[1]) > 50.0).all()
    assert (start_vs_prev_tol(logs[2]) > 50.0).all()
    assert logs[0][-1, 2] < logs[1][-1, 2] < logs[2][-1, 2]


def test_prop1_entropic_gap_bound_and_monotone_cost():
    """Prop. 1.3: <P*(gamma) - P*, C> <= H_min / gamma, checked on well-converged projections;
    the transport cost of P*(gamma) decreases as gamma grows."""
    p = I.grid_problem(5, 21)
    C, r, c = p.C.astype(np.float64), p.r, p.c
    ot = E.exact_ot_lp(C, r, c)
    H = min(O.entropy(r), O.entropy(c))
    costs = []
    for gamma in [4.0, 16.0, 64.0, 256.0, 1024.0]:
        u, v, rc, st, lr, lc = O.pncg(C, gamma, r, c, 1e-13, np.log(r), np.log(c))
        P = np.exp(u[:, None] + v[None, :] - gamma * C)
        cost = float((P * C).sum())
        assert cost - ot <= H / gamma + 1e-12
        costs.append(cost)
    assert all(b < a for a, b in zip(costs, costs[1:]))


def test_prop1_one_step_cost_decrease_equality():
    """Prop. 1.4: <P^(t) - P^(t+1), C> = (KL(P^(t)|P^(t+1)) + KL(P^(t+1)|P^(t))) / dgamma."""
    n = 8
    C, r, c = _rand_problem(n, 14)
    g0, dg = 20.0, 7.0
    def plan(g):
        u, v, rc, *_ = O.pncg(C, g, r, c, 1e-14, np.log(r), np.log(c))
        return np.exp(u[:, None] + v[None, :] - g * C)
    P0, P1 = plan(g0), plan(g0 + dg)
    lhs = float(((P0 - P1) * C).sum())
    rhs = (_kl(P0.ravel(), P1.ravel()) + _kl(P1.ravel(), P0.ravel())) / dg
    assert lhs > 0
    assert abs(lhs - rhs) < 1e-10 * rhs + 1e-14


def test_stage_schedule_and_counts():
    """Alg. 1: gamma_1 = min(gamma_i, gamma_f), gamma <- min(q gamma, gamma_f), exit at gamma_f;
    eps_d = H_min / gamma^p."""
    p = I.grid_problem(4, 2)
    q = 2.0 ** (1 / 3)
    u, v, rc, st, log = O.mdot(p.C, p.r, p.c, gamma_f=2.0 ** 8)
    expected = [16.0 * q ** k for k in range(13)]
    expected = [min(g, 256.0) for g in expected if g < 256.0 * (1 - 1e-12)] + [256.0]
    np.testing.assert_allclose(log[:, 0], expected, rtol=1e-12)
    H = min(O.entropy(p.r), O.entropy(p.c))
    np.testing.assert_allclose(log[:, 1], H / log[:, 0] ** 1.5, rtol=1e-12)
    # every stage met its tolerance eps_d / 2
    assert (log[:, 4] <= log[:, 1] / 2).all()
    # single stage when gamma_i >= gamma_f (the Sinkhorn-algorithm setting, Prop. 2)
    _, _, _, st1, log1 = O.mdot(p.C, p.r, p.c, gamma_i=64.0, gamma_f=64.0)
    assert st1.stages == 1


def test_log_n_stopping_bound():
    """App. C ablation: log n in place of H_min in eps_d.  The stage tolerances become
    log n / gamma^p (looser, since H_min <= log n), every stage meets its own one, and with uniform
    marginals (H_min = log n) the two choices run the same iterations."""
    p = I.grid_problem(5, 4)
    n = p.n
    _, _, _, st0, log0 = O.mdot(p.C, p.r, p.c, gamma_f=2.0 ** 9)
    _, _, _, st1, log1 = O.mdot(p.C, p.r, p.c, gamma_f=2.0 ** 9, stop_entropy=1)
    np.testing.assert_allclose(log1[:, 1], np.log(n) / log1[:, 0] ** 1.5, rtol=1e-12)
    assert (log1[:, 4] <= log1[:, 1] / 2).all()
    assert (log1[:, 1] > log0[:, 1]).all()
    assert st1.evals <= st0.evals
    w = np.full(n, 1.0 / n)
    _, _, _, su0, lu0 = O.mdot(p.C, w, w, gamma_f=2.0 ** 9)
    _, _, _, su1, lu1 = O.mdot(p.C, w, w, gamma_f=2.0 ** 9, stop_entropy=1)
    np.testing.assert_allclose(lu1[:, 1], lu0[:, 1], rtol=1e-13)
    assert su1.evals == su0.evals and su1.iters == su0.iters


# ---------------------------------------------------------------------------------------------
# Rounding (Alg. 3), c-transform bound, end-to-end against exact optima
# ---------------------------------------------------------------------------------------------

def test_round_feasible_and_within_altschuler_bound():
    """Alg. 3 output lies in U(r, c); ||G - P||_1 <= 2 (||r(P) - r||_1 + ||c(P) - c||_1)."""
    n, gamma = 30, 50.0
    C, r, c = _rand_problem(n, 15)
    rng = np.random.default_rng(16)
    u = np.log(r) + 0.3 * rng.normal(size=n)
    v = np.log(c) + 0.3 * rng.normal(size=n)
    cost, G = O.round_plan(C, u, v, gamma, r, c, want_G=True)
    P = np.exp(u[:, None] + v[None, :] - gamma * C)
    assert (G >= 0).all()
    np.testing.assert_allclose(G.sum(1), r, atol=1e-15 * n, rtol=1e-12)
    np.testing.assert_allclose(G.sum(0), c, atol=1e-15 * n, rtol=1e-12)
    g1 = np.abs(P.sum(1) - r).sum() + np.abs(P.sum(0) - c).sum()
    assert np.abs(G - P).sum() <= 2 * g1 + 1e-12
    assert abs(cost - float((G * C).sum())) < 1e-14


def test_brute_force_optimum_uniform_marginals():
    """n <= 7, uniform marginals: MDOT + rounding reaches the permutation optimum; the c-transform
    bound sits below it (weak duality)."""
    for seed in range(3):
        n = 6 + seed % 2
        rng = np.random.default_rng(100 + seed)
        C = rng.uniform(0, 1, (n, n))
        w = np.full(n, 1.0 / n)
        ot = E.brute_force_uniform(C)
        res = O.solve(C, w, w, gamma_f=2.0 ** 14)
        assert res.lb <= ot + 1e-12 <= res.cost + 2e-12
        assert res.cost - ot < 1e-6


def test_one_dimensional_monotone_coupling():
    """Points on a line with squared distance: the sorted north-west corner coupling is optimal."""
    n = 48
    rng = np.random.default_rng(17)
    x, y = np.sort(rng.uniform(0, 1, n)), rng.uniform(0, 1, n)
    C = (x[:, None] - y[None, :]) ** 2
    s = C.max()
    C /= s
    r = rng.uniform(0.5, 1, n); r /= r.sum()
    c = rng.uniform(0.5, 1, n); c /= c.sum()
    ot = E.monotone_1d(x, y, r, c, lambda d: d * d / s)
    assert abs(ot - E.exact_ot_lp(C, r, c)) < 1e-12
    res = O.solve(C, r, c, gamma_f=2.0 ** 19)
    assert res.lb <= ot + 1e-12 <= res.cost + 1e-12
    assert res.cost - ot < 1e-7


def test_equal_marginals_zero_diagonal_cost_is_free():
    """r = c with C_ii = 0 and C >= 0: the identity coupling costs 0."""
    p = I.grid_problem(6, 4)
    res = O.solve(p.C, p.r, p.r, gamma_f=2.0 ** 14)
    assert 0.0 <= res.cost < 5e-6
    assert res.lb <= 1e-15


@pytest.mark.parametrize("kind", ["l2sq", "l1"])
def test_grid_problem_against_lp(kind):
    """Grid histograms (n = 100): the rounded cost approaches the exact LP optimum; the true gap
    is below the Remark 1 / Prop. 2 target; the certificate brackets the optimum."""
    p = I.grid_problem(10, 31, kind=kind)
    ot = E.exact_ot_lp(p.C, p.r, p.c)
    res = O.solve(p.C, p.r, p.c, eps_target=1e-5)
    assert res.status == 0
    assert res.lb <= ot + 1e-12 <= res.cost + 1e-12
    assert res.cost - ot <= 1e-5
    # gap shrinks across the anneal: a larger gamma_f gives a smaller true gap
    res2 = O.solve(p.C, p.r, p.c, gamma_f=res.gamma_f * 8)
    assert res2.cost - ot <= res.cost - ot + 1e-12


def test_eps_dual_never_exceeds_primal():
    """Fenchel-Young form of weak duality for EOT: for every P in U(r, c),
    -g(u, v) <= gamma <P, C> - H(P) - 1 (here P = the rounded plan G)."""
    p = I.grid_problem(6, 8)
    C = p.C.astype(np.float64)
    for gamma in [16.0, 128.0, 1024.0]:
        u, v, rc, st, _, _ = O.pncg(C, gamma, p.r, p.c, 1e-9, np.log(p.r), np.log(p.c))
        cost, G = O.round_plan(C, u, v, gamma, p.r, p.c, want_G=True)
        Gp = G[G > 0]
        HG = -float((Gp * np.log(Gp)).sum())
        assert -O.dual_value(C, u, v, gamma, p.r, p.c) <= gamma * cost - HG - 1 + 1e-9


def test_ctransform_bound_is_tight_at_lp_duals():
    p = I.grid_problem(8, 9)
    C = p.C.astype(np.float64)
    val, f, g, _ = E.exact_ot_colgen(C, p.r, p.c)
    gamma = 1000.0
    # the bound is computed from u = gamma f: it must reproduce the LP value
    lb = O.ctransform_lb(C, gamma * f, gamma, p.r, p.c)
    assert abs(lb - val) < 1e-9
    # and any other potential gives a lower bound
    lb2 = O.ctransform_lb(C, gamma * f + np.random.default_rng(1).normal(size=p.n), gamma, p.r, p.c)
    assert lb2 <= val + 1e-12


@pytest.mark.parametrize("kind", ["l2sq", "l1"])
def test_seeded_column_generation_matches_full_lp(kind):
    """Column generation seeded with the nearly tight arcs of an entropic solve's potentials
    returns the full LP's value: the seed only changes the first arc set, and every round still
    prices all n^2 arcs.  A seed too narrow to contain any arc changes nothing either."""
    p = I.grid_problem(10, 33, kind=kind)
    C = p.C.astype(np.float64)
    ot = E.exact_ot_lp(C, p.r, p.c)
    res = O.solve(C, p.r, p.c, eps_target=1e-4)
    f, g = res.u / res.gamma_f, res.v / res.gamma_f
    red = C - f[:, None] - g[None, :]
    width = float(np.quantile(red, 0.05))           # about 5 arcs per row
    for w in (width, -1.0):
        val, fd, gd, _ = E.exact_ot_colgen(C, p.r, p.c, k_init=2, seed_f=f, seed_g=g, seed_width=w)
        assert abs(val - ot) <= 1e-10
        assert (C - fd[:, None] - gd[None, :]).min() >= -1e-9      # the returned duals are feasible


def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as fh:
        return json.load(fh)["cases"]


def test_stored_exact_optima_are_bracketed_by_the_oracle_records():
    """Weak duality on the stored values: every rounded oracle plan is feasible, so its cost is
    >= OT, and every c-transform bound is a feasible dual, so it is <= OT.  The exact optima stored
    for the n = 4096 benchmark instance (column generation) and the n = 256 instances (full LP)
    must lie inside every such bracket of the same instance."""
    checked = 0
    exact = {(c["kind"], c["seed"]): c["exact_ot"] for c in _golden("exact4096.json")
             if c.get("exact_ot") is not None}
    for rec in _golden("grid4096.json") + _golden("grid256.json"):
        ot = rec.get("exact_ot") if rec["n"] == 256 else exact.get((rec["kind"], rec["seed"]))
        if ot is None:
            continue
        assert rec["oracle_lb"] - 1e-12 <= ot <= rec["oracle_cost"] + 1e-12, rec
        checked += 1
    assert checked >= 10


def test_entropy_and_gamma_f_mapping():
    n = 64
    assert abs(O.entropy(np.full(n, 1.0 / n)) - math.log(n)) < 1e-13
    e = np.zeros(n); e[3] = 1.0
    assert O.entropy(e) == 0.0
    H, eps, q = 6.0, 1e-6, 2.0 ** (1 / 3)
    g = O.gamma_f_for_eps(H, eps)
    target = (5 * H / (2 * eps)) ** (1 / 1.5)
    k = math.log(g / 16.0) / math.log(q)
    assert g >= target * (1 - 1e-12) and g / q < target
    assert abs(k - round(k)) < 1e-9


def test_point_mass_marginal_has_a_single_feasible_plan():
    """r = e_i0 (H_min = 0): U(r, c) = {e_i0 c^T}, so the rounded cost is sum_j c_j C_i0j."""
    n, i0 = 7, 3
    rng = np.random.default_rng(23)
    C = rng.uniform(0, 1, (n, n))
    r = np.zeros(n); r[i0] = 1.0
    c = rng.uniform(0.2, 1, n); c /= c.sum()
    res = O.solve(C, r, c, gamma_f=2.0 ** 10)
    assert abs(res.cost - float(c @ C[i0])) < 1e-12
    assert res.lb <= res.cost + 1e-12
    one = np.ones(1)
    res1 = O.solve(np.array([[0.3]]), one, one, gamma_f=2.0 ** 10)
    assert abs(res1.cost - 0.3) < 1e-15

