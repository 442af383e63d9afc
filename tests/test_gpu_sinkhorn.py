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


def _check(res, ref, gf, iter_slack):
    assert res.status == M.MDOT_OK, M.status_string(res.status)
    assert ref.status == 0
    # both stop anywhere inside ||r(P) - r~||_1 <= eps_d / 2 with c(P) = c~: the rounded costs may
    # differ by about eps_d (the same argument as for the PNCG projector)
    eps_d = res.info.H_min / gf ** 1.5
    assert abs(res.cost - ref.cost) <= max(1e-7, eps_d), (res.cost, ref.cost, eps_d)
    assert res.info.stages == ref.stats.stages
    # one pass over C per half step, plus the residual pass at the start of each stage
    assert res.info.evals == ref.stats.stages + 2 * res.info.iters
    assert res.info.ls_trials == 0
    assert abs(res.info.iters - ref.stats.iters) <= iter_slack * ref.stats.iters + ref.stats.stages, \
        (res.info.iters, ref.stats.iters)
    assert res.gap_cert >= -1e-12


# grid 16 on the fp64 tier (n <= 512), grid 24 on the fast fp32 tier (automatic choice, every
# stage tolerance above the accurate tier's switch), grid 20 forced onto the accurate fp32 tier
@pytest.mark.parametrize("side,seed,prec,slack", [(16, 50, M.PREC_AUTO, 0.0), (24, 52, M.PREC_AUTO, 0.05),
                                                  (20, 53, M.PREC_FP32A, 0.02)])
def test_sinkhorn_projector_matches_oracle(h, side, seed, prec, slack):
    p = I.grid_problem(side, seed, kind="l2sq")
    gf = 2.0 ** 12
    prm = M.default_params(gamma_f=gf, projector=1, precision=prec)
    u, v, res = h.solve(t(p.r), t(p.c), t(p.C), 1e-6, prm)
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, projector=1)
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
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, projector=1)
    for prec, slack in ((M.PREC_AUTO, 0.0), (M.PREC_FP32A, 0.02)):
        prm = M.default_params(gamma_f=gf, projector=1, precision=prec)
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
