"""MDOT-Sinkhorn (Alg. 4 as the projector of every stage of Alg. 1) on the GPU against the oracle
run with the same projector: rounded cost, stages, Sinkhorn iterations and passes over C."""
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


@pytest.fixture(scope="module")
def h():
    torch.cuda.set_device(0)
    with M.Handle(1024) as handle:
        yield handle


# The last stage of both sides runs to the same residual (1e-9 where the GPU can finish in fp64
# entries, the fp32 floor 2e-7 where the tier is forced to fp32), so both stop at the same
# entropic optimum and the rounded costs must agree to the 1e-7 target.
TIGHT, FLOOR = 1e-9, 2e-7


def _check(res, ref, gf, iter_slack):
    assert res.status == M.MDOT_OK, M.status_string(res.status)
    assert ref.status == 0
    assert abs(res.cost - ref.cost) <= 1e-7, (res.cost, ref.cost)
    assert res.info.stages == ref.stats.stages
    # one pass over C per half step, plus the residual pass at the start of each projection launch
    # (the stages and, when the last fp32 stage is finished in fp64 entries, that polish)
    projections = res.info.launches - 3          # less the validation, rounding and bound launches
    assert res.info.evals == projections + 2 * res.info.iters
    assert res.info.ls_trials == 0
    assert abs(res.info.iters - ref.stats.iters) <= iter_slack * ref.stats.iters + ref.stats.stages, \
        (res.info.iters, ref.stats.iters)
    assert res.gap_cert >= -1e-12


# grid 16 on the fp64 tier (n <= 512), grid 24 on the fast fp32 tier (automatic choice, every
# stage tolerance above the accurate tier's switch), grid 20 forced onto the accurate fp32 tier
# (whose last stage stops where the fp32 sums' noise lets the residual through: ~10 % slack)
@pytest.mark.parametrize("side,seed,prec,slack", [(16, 50, M.PREC_AUTO, 0.0), (24, 52, M.PREC_AUTO, 0.05),
                                                  (20, 53, M.PREC_FP32A, 0.1)])
def test_sinkhorn_projector_matches_oracle(h, side, seed, prec, slack):
    p = I.grid_problem(side, seed, kind="l2sq")
    gf = 2.0 ** 12
    ft = FLOOR if prec == M.PREC_FP32A else TIGHT
    prm = M.default_params(gamma_f=gf, projector=1, precision=prec, final_tol=ft)
    u, v, res = h.solve(t(p.r), t(p.c), t(p.C), 1e-6, prm)
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, projector=1, final_tol=ft)
    _check(res, ref, gf, slack)
    if side == 16:
        # the fp64 tier takes the oracle's decisions: the same iterations, dual values to rounding
        assert res.info.iters == ref.stats.iters
        np.testing.assert_allclose(u.cpu().numpy(), ref.u, rtol=0, atol=1e-9)
        np.testing.assert_allclose(v.cpu().numpy(), ref.v, rtol=0, atol=1e-9)


def test_sinkhorn_projector_regenerated_cost(h):
    """The same projector with C regenerated from point coordinates (fp64 and accurate fp32)."""
    p = I.point_cloud_problem(300, 4501)
    gf = 2.0 ** 11
    # fp32 entries: the last stage's residual falls through the floor at a point set by the noise
    # of the fp32 sums, so its iteration count can differ from the oracle's by ~10 %
    for prec, slack in ((M.PREC_AUTO, 0.0), (M.PREC_FP32A, 0.1)):
        ft = FLOOR if prec == M.PREC_FP32A else TIGHT
        ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, projector=1, final_tol=ft)
        prm = M.default_params(gamma_f=gf, projector=1, precision=prec, final_tol=ft)
        u, v, res = h.solve_points(t(p.r), t(p.c), t(p.x), t(p.y), M.COST_SQEUCLID, p.scale, 1e-6, prm)
        _check(res, ref, gf, slack)


def test_sinkhorn_projector_not_batched(h):
    p = I.point_cloud_problem(40, 4502)
    r, c, x, y = t(p.r), t(p.c), t(p.x), t(p.y)
    u, v = torch.empty(p.n, dtype=torch.float64, device=DEV), torch.empty(p.n, dtype=torch.float64, device=DEV)
    prob = M.make_problem(r, c, x=x, y=y, kind=M.COST_SQEUCLID, scale=p.scale, gamma_f=2.0 ** 8, u_out=u, v_out=v)
    with pytest.raises(M.MdotError) as e:
        h.solve_batch([prob], M.default_params(projector=1))
    assert e.value.status == M.MDOT_ERR_INVALID_ARG
