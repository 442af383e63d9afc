"""Large n with the cost regenerated from coordinates (memory O(n), no n x n matrix): points on a
line, where the monotone coupling is optimal, so the exact cost is known at any n (stored by
tests/golden/make_golden.py --line).  Checks that hold at any size: the rounded plan is feasible
(cost >= OT), weak duality (lower bound <= OT <= cost, so the true gap <= the certificate), and the
returned potentials reproduce the smoothed marginals on sampled rows and columns to within the
reported ||grad g||_1 (each row and column recomputed one by one in fp64 on the host)."""
import json
import os

import numpy as np
import pytest
import torch

import oracle as O
import paper_2307_08507_gb300 as M
from paper_2307_08507_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]
DEV = "cuda:0"
HERE = os.path.dirname(os.path.abspath(__file__))


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def exact_cost(n, seed=11):
    with open(os.path.join(HERE, "golden", "line_exact.json")) as fh:
        for c in json.load(fh)["cases"]:
            if c["n"] == n and c["seed"] == seed:
                return c["exact_ot"]
    raise KeyError((n, seed))


def cost_rows(p, rows):
    """C[rows, :] in the float32 order the coordinate form defines."""
    return I.point_cost(p.x[rows], p.y, np.float32(p.scale)).astype(np.float64)


def test_line_problem_small_matches_oracle():
    torch.cuda.set_device(0)
    p = I.line_problem(200, 11, dense=True)
    gf = 2.0 ** 14
    tight = 1e-10           # the same last-stage tolerance on both sides (fp64 entries, n <= 512)
    with M.Handle(200) as h:
        u, v, res = h.solve_points(t(p.r), t(p.c), t(p.x), t(p.y), M.COST_SQEUCLID, p.scale, 1e-6,
                                   M.default_params(gamma_f=gf, final_tol=tight))
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, final_tol=tight)
    assert res.status == M.MDOT_OK
    assert abs(res.cost - ref.cost) <= 1e-7, (res.cost, ref.cost)
    ex = exact_cost(200)
    assert res.cost >= ex - 1e-12 and ref.cost >= ex - 1e-12
    assert res.cost - res.gap_cert <= ex + 1e-12


@pytest.mark.parametrize("n,eps", [(65536, 1e-5), (16384, 1e-6)])
def test_line_problem_large_n(n, eps):
    torch.cuda.set_device(0)
    p = I.line_problem(n, 11)
    with M.Handle(n) as h:
        u, v, res = h.solve_points(t(p.r), t(p.c), t(p.x), t(p.y), M.COST_SQEUCLID, p.scale, eps,
                                   M.default_params())
    assert res.status == M.MDOT_OK, M.status_string(res.status)
    ex = exact_cost(n)
    lb = res.cost - res.gap_cert
    # Alg. 3 returns a plan in U(r, c): its cost is at least the optimum (fp64 sums of n^2 terms)
    assert res.cost >= ex - 1e-10, (res.cost, ex)
    # the c-transform bound is a feasible dual: below the optimum
    assert lb <= ex + 1e-10, (lb, ex)
    gf, H = res.info.gamma_f, res.info.H_min
    w = H / gf ** 1.5
    # Prop. 1: the entropic optimum at gamma_f is within H_min / gamma_f of OT; rounding (Alg. 3)
    # and the smoothing move the plan by a few ||grad g||_1 and eps_d in L1, with C in [0, 1]
    assert res.cost - ex <= H / gf + 4 * (res.info.grad_l1 + w)
    # sampled rows and columns of P(u, v; gamma_f) against the smoothed marginals of the last stage
    rt = (1 - w / 4) * p.r + w / (4 * n)
    ct = (1 - w / 4) * p.c + w / (4 * n)
    un, vn = u.cpu().numpy(), v.cpu().numpy()
    rng = np.random.default_rng(5)
    rows = rng.choice(n, 48, replace=False)
    Cr = cost_rows(p, rows)
    z = un[rows, None] + vn[None, :] - gf * Cr
    m = z.max(axis=1, keepdims=True)
    rP = np.exp(m[:, 0]) * np.exp(z - m).sum(axis=1)
    cols = rng.choice(n, 48, replace=False)
    Cc = I.point_cost(p.x, p.y[cols], np.float32(p.scale)).astype(np.float64)
    zc = un[:, None] + vn[None, cols] - gf * Cc
    mc = zc.max(axis=0, keepdims=True)
    cP = np.exp(mc[0]) * np.exp(zc - mc).sum(axis=0)
    sampled = np.abs(rP - rt[rows]).sum() + np.abs(cP - ct[cols]).sum()
    assert sampled <= res.info.grad_l1 * 1.01 + 1e-12, (sampled, res.info.grad_l1)
    # and row by row: ||grad g||_1 ~ 1e-6 leaves relative marginal errors far below 1e-3
    assert np.median(np.abs(rP / rt[rows] - 1)) < 1e-3
    assert np.median(np.abs(cP / ct[cols] - 1)) < 1e-3
