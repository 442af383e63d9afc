"""Failure paths of the C ABI, made to happen without faulting the GPU:

* a non-finite entry in C: the first evaluation sees a non-finite marginal -> MDOT_ERR_NUMERIC
  (fp64 entries at n <= 512 and fp32 entries above);
* an iteration cap of one PNCG iteration per stage -> MDOT_ERR_NOT_CONVERGED, with the outputs
  filled from the last iterate (a feasible rounded plan whose cost is bracketed by the bound);
* a device-side wait limit of 1 microsecond (mdot_params.wait_limit_us) on a normal n = 4096
  solve: the CTAs wait for each other's flags every evaluation, so a wait runs out, the kernel
  raises its abort flag, every CTA leaves, and the call returns MDOT_ERR_TIMEOUT; the same handle
  then solves the problem normally.
"""
import numpy as np
import pytest
import torch

from oracle import exact as E
import paper_2307_08507_gb300 as M
from paper_2307_08507_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]
DEV = "cuda:0"


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.mark.parametrize("k", [16, 24])          # n = 256 (fp64 entries), n = 576 (fp32 entries)
def test_nan_in_cost_is_numeric(k):
    torch.cuda.set_device(0)
    p = I.grid_problem(k, 5)
    C = p.C.copy()
    C[3, 7] = np.nan
    with M.Handle(p.n) as h:
        u, v, res = h.solve(t(p.r), t(p.c), t(C), 1e-5, check=False)
        assert res.status == M.MDOT_ERR_NUMERIC, M.status_string(res.status)
        # the handle is still usable on a valid problem
        u, v, res = h.solve(t(p.r), t(p.c), t(p.C), 1e-5)
        assert res.status == M.MDOT_OK


@pytest.mark.parametrize("k", [16, 24])
def test_iteration_cap_is_not_converged_with_the_best_iterate(k):
    torch.cuda.set_device(0)
    p = I.grid_problem(k, 6)
    gf = 2.0 ** 10
    with M.Handle(p.n) as h:
        u, v, res = h.solve(t(p.r), t(p.c), t(p.C), 1e-6, M.default_params(gamma_f=gf, max_iter=1), check=False)
        assert res.status == M.MDOT_ERR_NOT_CONVERGED, M.status_string(res.status)
        assert res.info.iters <= res.info.stages        # one iteration per stage at most
        un, vn = u.cpu().numpy(), v.cpu().numpy()
        assert np.isfinite(un).all() and np.isfinite(vn).all()
        # the outputs come from the last iterate: its rounded plan is feasible, so its cost lies
        # above the exact optimum, and the certificate brackets it
        exact = E.exact_ot_lp(p.C.astype(np.float64), p.r, p.c) if p.n <= 300 else None
        assert np.isfinite(res.cost) and np.isfinite(res.gap_cert) and res.gap_cert >= 0.0
        if exact is not None:
            assert res.cost >= exact - 1e-9
            assert res.cost - res.gap_cert <= exact + 1e-9
        # same point as the rounding entry point gives for the returned potentials
        cost2, _ = h.round(u, v, gf, t(p.C), t(p.r), t(p.c))
        assert abs(cost2 - res.cost) <= 1e-7


def test_wait_limit_runs_out_and_the_handle_stays_usable():
    torch.cuda.set_device(0)
    p = I.grid_problem(64, 2000)
    r, c, C = t(p.r), t(p.c), t(p.C)
    with M.Handle(p.n) as h:
        u, v, ref = h.solve(r, c, C, 1e-4)
        assert ref.status == M.MDOT_OK
        u, v, res = h.solve(r, c, C, 1e-4, M.default_params(wait_limit_us=1), check=False)
        assert res.status == M.MDOT_ERR_TIMEOUT, M.status_string(res.status)
        # the next call starts from a cleared state and reproduces the first solve bit for bit
        u, v, again = h.solve(r, c, C, 1e-4)
        assert again.status == M.MDOT_OK
        assert again.cost == ref.cost and again.info.evals == ref.info.evals
