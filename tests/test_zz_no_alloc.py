"""mdot_dual_eval_noalloc, the dual evaluation for callers that cannot allocate device memory
(its scratch is a static device array inside the library).  Checked through the C ABI against
the handle-based mdot_dual_eval, within the fp32-entry tolerance of the parity tests, on two calls
in a row (the second call must not see anything the first left in the shared scratch)."""
import numpy as np
import pytest
import torch

import paper_2307_08507_gb300 as M
from paper_2307_08507_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]

TOL_F32 = 4e-6     # same bound as the fp32-entry parity tests (see test_gpu_parity.py)


def _case(k, seed, gamma):
    p = I.grid_problem(k, seed)
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 0.3, p.n)
    b = (p.C.astype(np.float64) - a[:, None]).min(axis=0)
    u = gamma * a + np.log(p.r)
    v = gamma * b + np.log(p.c)
    dev = "cuda:0"
    return (torch.from_numpy(u).to(dev), torch.from_numpy(v).to(dev),
            torch.from_numpy(p.C).to(dev))


def test_noalloc_matches_handle_entry_on_two_calls():
    torch.cuda.set_device(0)
    cases = [_case(64, 2000, 2.0 ** 13), _case(40, 7, 2.0 ** 9)]     # n = 4096, then n = 1600
    with M.Handle(4096) as h:
        for gamma, (u, v, C) in zip((2.0 ** 13, 2.0 ** 9), cases):
            n = u.numel()
            lr_ref, lc_ref = h.dual_eval(u, v, gamma, C)
            lr = torch.full((n,), float("nan"), dtype=torch.float64, device=u.device)
            lc = torch.full((n,), float("nan"), dtype=torch.float64, device=u.device)
            assert M.dual_eval_noalloc(u, v, gamma, C, lr, lc) == M.MDOT_OK
            np.testing.assert_allclose(lr.cpu().numpy(), lr_ref.cpu().numpy(), rtol=0, atol=TOL_F32)
            np.testing.assert_allclose(lc.cpu().numpy(), lc_ref.cpu().numpy(), rtol=0, atol=TOL_F32)
            # the one-pass form with a row-scale estimate, as inside the solver
            lr2 = torch.empty_like(lr)
            lc2 = torch.empty_like(lc)
            assert M.dual_eval_noalloc(u, v, gamma, C, lr2, lc2, ref_log_rP=lr_ref) == M.MDOT_OK
            np.testing.assert_allclose(lr2.cpu().numpy(), lr_ref.cpu().numpy(), rtol=0, atol=TOL_F32)
            np.testing.assert_allclose(lc2.cpu().numpy(), lc_ref.cpu().numpy(), rtol=0, atol=TOL_F32)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    torch.cuda.set_device(0)
    n = M.NOALLOC_MAX_N + 1
    dev = "cuda:0"
    u = torch.zeros(n, dtype=torch.float64, device=dev)
    C = torch.zeros((n, n), dtype=torch.float32, device=dev)
    out = torch.empty(n, dtype=torch.float64, device=dev)
    assert M.dual_eval_noalloc(u, u, 1.0, C, out, out.clone()) == M.MDOT_ERR_INVALID_ARG
