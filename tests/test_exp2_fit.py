"""The polynomial of the accurate fp32 tier's exp2 (exp2_acc, csrc/mdot_device.cuh) against the
Remez exchange that the repository ships for it (csrc/exp2_poly_fit.py).  CPU only."""
import importlib.util
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_exp2_polynomial_is_a_minimax_fit():
    """The degree-6 polynomial of the accurate fp32 tier (exp2_acc in mdot_device.cuh, p(0) = 1) is
    a relative-minimax fit of 2^x on [-1/2, 1/2]: the Remez exchange (csrc/exp2_poly_fit.py) reaches
    a level below 2e-9 with the same leading coefficient, and the coefficients written in the CUDA
    source (float32) stay within 2 % of the best float32-rounded error, below 1.6e-8."""
    src_dir = os.path.join(ROOT, "paper_2307_08507_gb300", "csrc")
    spec = importlib.util.spec_from_file_location("exp2_poly_fit", os.path.join(src_dir, "exp2_poly_fit.py"))
    F = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(F)
    c, level = F.remez()
    assert level < 2e-9
    text = open(os.path.join(src_dir, "mdot_device.cuh")).read()
    body = text[text.index("__device__ __forceinline__ float exp2_acc("):]
    body = body[:body.index("return p * ex2f(kf);")]
    committed = [float(v) for v in re.findall(r"([0-9]\.[0-9]+e-?[0-9]+)f", body)][::-1]   # c1 .. c6
    assert len(committed) == 6
    assert np.float32(committed[0]) == np.float32(c[0])
    x = np.linspace(-0.5, 0.5, 400001)
    err_committed = np.abs(F.rel_error(committed, x)).max()
    err_remez32 = np.abs(F.rel_error(F.float32_coefficients(c), x)).max()
    assert err_committed < 1.6e-8
    assert err_committed <= 1.02 * err_remez32
