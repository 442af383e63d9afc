"""mdot_dual_eval_noalloc, the dual evaluation for callers that cannot allocate device memory
(its scratch is a static device array inside the library).  Checked through the C ABI against
the handle-based mdot_dual_eval, within the fp32-entry tolerance of the parity tests, on calls in a
row (no call may see anything an earlier one left in the shared scratch), and against the CPU
oracle.  Sizes: n = 4096 and 1600 (the vectorised path), 1601 (n not a multiple of 4: the scalar
path) and 100 (fewer rows than CTAs: some CTAs own no row or column)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2307_08507_gb300 as M
from paper_2307_08507_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(300)]

TOL_F32 = 4e-6     # same bound as the fp32-entry parity tests (see test_gpu_parity.py)


def _case(n, seed, gamma):
    rng = np.random.default_rng(seed)
    k = int(round(np.sqrt(n)))
    if k * k == n:
        p = I.grid_problem(k, seed)
        C, r, c = p.C, p.r, p.c
    else:
        C = rng.uniform(0.0, 1.0, (n, n)).astype(np.float32)
        r = rng.uniform(0.2, 1.0, n); r /= r.sum()
        c = rng.uniform(0.2, 1.0, n); c /= c.sum()
    a = rng.uniform(0.0, 0.3, n)
    b = (C.astype(np.float64) - a[:, None]).min(axis=0)
    u = gamma * a + np.log(r)
    v = gamma * b + np.log(c)
    return u, v, C


CASES = [(4096, 2000, 2.0 ** 13), (1600, 7, 2.0 ** 9), (1601, 8, 2.0 ** 11), (100, 9, 2.0 ** 6)]


def test_noalloc_matches_handle_entry_on_calls_in_a_row():
    torch.cuda.set_device(0)
    dev = "cuda:0"
    with M.Handle(4096) as h:
        for n, seed, gamma in CASES:
            un, vn, Cn = _case(n, seed, gamma)
            u, v, C = (torch.from_numpy(a).to(dev) for a in (un, vn, Cn))
            lr_ref, lc_ref = h.dual_eval(u, v, gamma, C)
            lr_o, lc_o = O.dual_eval(Cn.astype(np.float64), un, vn, gamma)
            for _ in range(2):                     # two calls in a row on the same size
                lr = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
                lc = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
                assert M.dual_eval_noalloc(u, v, gamma, C, lr, lc) == M.MDOT_OK
                np.testing.assert_allclose(lr.cpu().numpy(), lr_ref.cpu().numpy(), rtol=0, atol=TOL_F32)
                np.testing.assert_allclose(lc.cpu().numpy(), lc_ref.cpu().numpy(), rtol=0, atol=TOL_F32)
                np.testing.assert_allclose(lr.cpu().numpy(), lr_o, rtol=0, atol=TOL_F32)
                np.testing.assert_allclose(lc.cpu().numpy(), lc_o, rtol=0, atol=TOL_F32)
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
    msg = M.lib().mdot_last_error().decode()
    assert "MDOT_NOALLOC_MAX_N" in msg and str(n) in msg, msg
