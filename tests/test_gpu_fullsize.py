"""Full-size parity: the n = 4096 benchmark instance (64 x 64 grid histograms, squared-Euclidean
cost, seed 2000, target gap 1e-6) solved exactly as bench.py solves it, against the stored CPU FP64
oracle result (tests/golden/grid4096.json, written by tests/golden/make_golden.py): rounded-plan
cost within 1e-7 absolute (costs normalised to max C = 1), same stage count, the certificate an
upper bound of the true gap."""
import json
import os

import numpy as np
import pytest
import torch

import paper_2307_08507_gb300 as M
from paper_2307_08507_gb300 import inputs as I

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(600)]
HERE = os.path.dirname(os.path.abspath(__file__))


def golden(kind="l2sq"):
    with open(os.path.join(HERE, "golden", "grid4096.json")) as fh:
        for c in json.load(fh)["cases"]:
            if c["kind"] == kind and c["seed"] == 2000 and c["eps_target"] == 1e-6:
                return c
    pytest.skip("no stored oracle result for this case")


def test_benchmark_instance_matches_the_oracle():
    g = golden()
    torch.cuda.set_device(0)
    p = I.grid_problem(64, 2000)
    dev = "cuda:0"
    r, c, C = (torch.from_numpy(a).to(dev) for a in (p.r, p.c, p.C))
    with M.Handle(4096) as h:
        u, v, res = h.solve(r, c, C, 1e-6)
    assert res.status == M.MDOT_OK
    assert res.info.gamma_f == g["gamma_f"]
    assert res.info.stages == g["oracle_stages"]
    assert abs(res.cost - g["oracle_cost"]) <= 1e-7, (res.cost, g["oracle_cost"])
    # the certificate bounds the gap to the oracle's own bound from above
    assert res.cost - res.info.lower_bound >= res.cost - g["oracle_cost"] - 1e-12
    # potentials: same plan up to the additive shift (compared in cost units)
    f = u.cpu().numpy() / res.info.gamma_f
    assert np.isfinite(f).all()
