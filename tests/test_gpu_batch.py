"""Batched solver (one persistent launch for many problems of uneven n): every result matches the
CPU oracle on its problem, and a problem solved alone and inside a mixed batch gives the same
result bit for bit (its reductions run in a fixed order on one CTA)."""
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
    with M.Handle(4096) as handle:
        yield handle


def _point_problems(sizes, seed0):
    out = []
    for k, n in enumerate(sizes):
        p = I.point_cloud_problem(int(n), seed0 + k)
        out.append(p)
    return out


def _tensors(p, dense=False):
    d = {"r": t(p.r), "c": t(p.c), "u": torch.empty(p.n, dtype=torch.float64, device=DEV),
         "v": torch.empty(p.n, dtype=torch.float64, device=DEV)}
    if dense:
        d["C"] = t(p.C)
    else:
        d["x"], d["y"] = t(p.x), t(p.y)
    return d


def _problem(p, d, gamma_f):
    if "C" in d:
        return M.make_problem(d["r"], d["c"], C=d["C"], gamma_f=gamma_f, u_out=d["u"], v_out=d["v"])
    return M.make_problem(d["r"], d["c"], x=d["x"], y=d["y"], kind=M.COST_SQEUCLID, scale=p.scale,
                          gamma_f=gamma_f, u_out=d["u"], v_out=d["v"])


# The fp32 tiers of the batched form drive a stage down to about their noise floor
# (mdot_params.fp32_floor, 2e-7); on problems of a few dozen points the fp32 noise of a row's few
# significant entries does not average out, so the tests of the fp32 path ask for 5e-7 (reached
# without the fp64 polish).  The oracle is run with the same last-stage tolerance, so both stop
# within 5e-7 (in L1) of the same entropic optimum and the rounded costs must agree to the 1e-7
# target.  A tighter last-stage tolerance is reached by the fp64 polish (test below).
FLOOR = 5e-7


def _grid_problem(k, seed, gf, dense=False):
    p = I.grid_problem(k, seed)
    d = {"r": t(p.r), "c": t(p.c), "u": torch.empty(p.n, dtype=torch.float64, device=DEV),
         "v": torch.empty(p.n, dtype=torch.float64, device=DEV)}
    if dense:
        d["C"] = t(p.C)
        prob = M.make_problem(d["r"], d["c"], C=d["C"], gamma_f=gf, u_out=d["u"], v_out=d["v"])
    else:
        d["xy"] = t(I.coords3(p.x))
        prob = M.make_problem(d["r"], d["c"], x=d["xy"], y=d["xy"], kind=M.COST_SQEUCLID, scale=p.scale,
                              gamma_f=gf, u_out=d["u"], v_out=d["v"])
    return p, d, prob


# the batched form floors every stage tolerance at fp32_floor; a caller who needs a tighter last
# stage lowers it, and the fp64 polish (at most polish_iters iterations) finishes the stage
TIGHT = 1e-10
TIGHT_PARAMS = dict(final_tol=TIGHT, fp32_floor=TIGHT, polish_iters=2000)


def test_batch_fp64_polish_reaches_a_tight_tolerance(h):
    """A last-stage tolerance below the accurate fp32 tier's noise: the fp32 part of the stage
    stalls above it and the batched solver continues in fp64 entries (as mdot_solve does) until it
    is reached, for the regenerated and the dense cost; the rounded costs match the oracle run to
    the same tolerance (grid histograms, whose last stage converges in some 100 fp64 iterations)."""
    tight = TIGHT
    gf = 2.0 ** 12
    cases = [_grid_problem(24, 4900, gf), _grid_problem(10, 4901, gf), _grid_problem(24, 4900, gf, dense=True)]
    res = h.solve_batch([prob for _, _, prob in cases], M.default_params(**TIGHT_PARAMS))
    refs = {}
    for (p, d, _), r in zip(cases, res):
        assert r.status == M.MDOT_OK, M.status_string(r.status)
        assert r.grad_l1 <= tight, (p.n, r.grad_l1)
        if p.n not in refs:
            refs[p.n] = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, final_tol=tight)
        assert abs(r.cost - refs[p.n].cost) <= 1e-7, (p.n, r.cost, refs[p.n].cost)


def test_batch_finishes_stalled_problems_on_every_sm(h):
    """A problem the batch kernel leaves above its last-stage tolerance (here: a one-iteration fp64
    polish on its SM cannot reach 1e-10) is finished by the single-problem solver's fp64 stage on
    every SM, from the batch's potentials; potentials the caller did not ask for are kept in the
    handle's scratch for that.  Results against the oracle at the same tolerance."""
    tight = TIGHT
    gf = 2.0 ** 12
    cases = [_grid_problem(24, 4910, gf), _grid_problem(10, 4911, gf, dense=True)]
    plist = [prob for _, _, prob in cases]
    plist[1].u_out = None                       # no potentials asked for: the handle's scratch
    plist[1].v_out = None
    res = h.solve_batch(plist, M.default_params(**{**TIGHT_PARAMS, "polish_iters": 1}))
    for (p, d, _), r in zip(cases, res):
        assert r.status == M.MDOT_OK, M.status_string(r.status)
        assert r.grad_l1 <= tight, (p.n, r.grad_l1)
        ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, final_tol=tight)
        assert abs(r.cost - ref.cost) <= 1e-7, (p.n, r.cost, ref.cost)


def test_batch_fp64_polish_over_two_row_chunks(h):
    """n = 2116 > 2048 rows: the fp64 pass adds the column sums of its two row chunks.  Against the
    single-problem solver (whose fp64 polish the parity tests check against the oracle) at the same
    tolerance, and the returned potentials' marginals recomputed by the oracle's dual evaluation."""
    tight = TIGHT
    gf = 2.0 ** 10
    p, d, prob = _grid_problem(46, 4902, gf)
    r = h.solve_batch([prob], M.default_params(**TIGHT_PARAMS))[0]
    assert r.status == M.MDOT_OK and r.grad_l1 <= tight, (M.status_string(r.status), r.grad_l1)
    _, _, one = h.solve_points(d["r"], d["c"], d["xy"], d["xy"], M.COST_SQEUCLID, p.scale, 1e-6,
                               M.default_params(gamma_f=gf, final_tol=tight))
    assert one.status == M.MDOT_OK
    assert abs(r.cost - one.cost) <= 1e-8, (r.cost, one.cost)
    # the gradient norm the batched solver reports, recomputed from its potentials by the oracle's
    # dual evaluation against the last stage's smoothed marginals (Alg. 1: weight w = eps_d)
    lr, lc = O.dual_eval(p.C.astype(np.float64), d["u"].cpu().numpy(), d["v"].cpu().numpy(), gf)
    w = r.H_min / gf ** M.default_params().p
    rt = (1.0 - w / 4.0) * p.r + w / (4.0 * p.n)
    ct = (1.0 - w / 4.0) * p.c + w / (4.0 * p.n)
    gnorm = np.abs(np.exp(lr) - rt).sum() + np.abs(np.exp(lc) - ct).sum()
    assert gnorm <= 2.0 * tight, gnorm


def test_batch_matches_oracle_and_single_solves(h):
    sizes = [300, 64, 129, 257, 40]
    probs = _point_problems(sizes, 4100)
    gf = 2.0 ** 10
    tens = [_tensors(p) for p in probs]
    res = h.solve_batch([_problem(p, d, gf) for p, d in zip(probs, tens)], M.default_params(final_tol=FLOOR))
    for p, r in zip(probs, res):
        assert r.status == M.MDOT_OK, M.status_string(r.status)
        assert r.grad_l1 <= FLOOR
        ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, final_tol=FLOOR)
        assert abs(r.cost - ref.cost) <= 1e-7, (p.n, r.cost, ref.cost)
        # the fp64 c-transform bound against the oracle's, and below the optimum
        lb_o = O.ctransform_lb(p.C.astype(np.float64), tens[probs.index(p)]["u"].cpu().numpy(), gf, p.r, p.c)
        assert abs(r.lower_bound - lb_o) <= 1e-12 * max(1.0, abs(lb_o)), (r.lower_bound, lb_o)
        assert r.lower_bound <= ref.cost + 1e-9
        assert r.evals > 0 and r.stages == ref.stats.stages


def test_batch_result_same_alone_and_in_the_mix(h):
    """Same problem, same inputs: alone in a batch of one and inside a batch of 9 uneven problems
    -> bitwise identical cost, bound, potentials and iteration counts."""
    gf = 2.0 ** 11
    probs = _point_problems([200, 513, 96, 1000, 33, 700, 256, 128, 400], 4200)
    target = 3                      # n = 1000
    tens = [_tensors(p) for p in probs]
    mixed = h.solve_batch([_problem(p, d, gf) for p, d in zip(probs, tens)])
    u_mix, v_mix = tens[target]["u"].clone(), tens[target]["v"].clone()
    alone = h.solve_batch([_problem(probs[target], tens[target], gf)])[0]
    assert alone.status == M.MDOT_OK
    a, m = alone, mixed[target]
    assert (a.cost, a.lower_bound, a.evals, a.iters) == (m.cost, m.lower_bound, m.evals, m.iters)
    assert torch.equal(u_mix, tens[target]["u"]) and torch.equal(v_mix, tens[target]["v"])


def test_batch_dense_and_mixed_forms(h):
    """Dense and regenerated problems in one call (one launch per form)."""
    gf = 2.0 ** 10
    pa = I.grid_problem(12, 31)
    pb = I.point_cloud_problem(150, 4300)
    da, db = _tensors(pa, dense=True), _tensors(pb)
    res = h.solve_batch([_problem(pa, da, gf), _problem(pb, db, gf)], M.default_params(final_tol=FLOOR))
    for p, r in zip((pa, pb), res):
        ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, final_tol=FLOOR)
        assert r.status == M.MDOT_OK
        assert abs(r.cost - ref.cost) <= 1e-7, (r.cost, ref.cost)


def test_batch_rejects_malformed_problems(h):
    p = I.point_cloud_problem(50, 4400)
    d = _tensors(p)
    bad = _problem(p, d, 2.0 ** 8)
    bad.scale = -1.0
    with pytest.raises(M.MdotError) as e:
        h.solve_batch([bad])
    assert e.value.status == M.MDOT_ERR_INVALID_ARG


def test_batch_grid_problems_on_the_tensor_cores_match_oracle(h):
    """Grid histograms with the squared-Euclidean cost regenerated from integer cell coordinates,
    mdot_params.tensor_cores = 1: the batched kernel forms the cost on the tensor cores (exact for
    such points), every result against the CPU oracle on the dense matrix."""
    gf = 2.0 ** 10
    probs, tens = [], []
    for q, k in enumerate((12, 20, 9)):
        p = I.grid_problem(k, 4500 + q)
        xy = I.coords3(p.x)
        d = {"r": t(p.r), "c": t(p.c), "x": t(xy), "y": t(xy.copy())}
        probs.append(p)
        tens.append(d)
    plist = [M.make_problem(d["r"], d["c"], x=d["x"], y=d["y"], kind=M.COST_SQEUCLID, scale=p.scale, gamma_f=gf)
             for p, d in zip(probs, tens)]
    res = h.solve_batch(plist, M.default_params(final_tol=FLOOR, tensor_cores=1))
    for p, r in zip(probs, res):
        assert r.status == M.MDOT_OK, M.status_string(r.status)
        ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, final_tol=FLOOR)
        assert abs(r.cost - ref.cost) <= 1e-7, (p.n, r.cost, ref.cost)


def test_batch_tile_variants_and_tuner(h):
    """Both tile variants of the batched kernel (256 threads and one problem per SM; 128 threads
    and two per SM) give results equal to the oracle's; the tuner times every candidate table on
    the batch and installs the fastest, which later solves use."""
    gf = 2.0 ** 10
    sizes = [300, 700, 64, 1500]
    probs = _point_problems(sizes, 4700)
    tens = [_tensors(p) for p in probs]
    plist = [_problem(p, d, gf) for p, d in zip(probs, tens)]
    prm = M.default_params(final_tol=FLOOR)
    refs = [O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, final_tol=FLOOR) for p in probs]
    for variant in (0, 1):
        table = M.BatchTuning()
        for b in range(5):
            table.variant[b] = variant
        h.set_batch_tuning(table)
        res = h.solve_batch(plist, prm)
        for p, r, ref in zip(probs, res, refs):
            assert r.status == M.MDOT_OK, M.status_string(r.status)
            assert abs(r.cost - ref.cost) <= 1e-7, (variant, p.n, r.cost, ref.cost)
    tuned = h.tune_batch(plist, prm, sample=3)
    secs = tuned.as_dict()["seconds"]
    k = tuned.narrow_below
    assert all(t > 0.0 for t in secs)                       # every candidate table was timed
    assert secs[k] == min(secs) and all(secs[q] > secs[k] for q in range(k))
    assert list(tuned.variant) == [1 if b < k else 0 for b in range(5)]
    res = h.solve_batch(plist, prm)                         # the installed table
    for p, r, ref in zip(probs, res, refs):
        assert r.status == M.MDOT_OK and abs(r.cost - ref.cost) <= 1e-7, (k, p.n, r.cost, ref.cost)
    h.set_batch_tuning(M.BatchTuning())      # back to the default (wide) variant for other tests
