"""Serving runtime (mdot_server_*): continuous batching of requests on one GPU.  A request's
result equals the batched solver's on the same problem bit for bit, whether it runs alone or in
a stream of other requests; requests above n = 4096 (row sums in chunks) and big-lane requests
match the CPU oracle; tickets and malformed requests behave as documented.

Oracle comparisons run both sides with the last-stage tolerance at the fp32 floor
(||grad g||_1 <= 2e-7, the lowest the fp32-entry batched route resolves), so both stop within 2e-7
of the same entropic optimum and the rounded costs must agree to the 1e-7 target."""
import time

import numpy as np
import pytest
import torch

import oracle as O
import paper_2307_08507_gb300 as M
from paper_2307_08507_gb300 import inputs as I

FLOOR = 2e-7

pytestmark = [pytest.mark.gpu, pytest.mark.timeout(900)]
DEV = "cuda:0"


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def grid_request(k, seed, eps=None, gamma_f=0.0):
    """k x k grid histograms, squared-Euclidean cost regenerated from the cell coordinates."""
    p = I.grid_problem(k, seed, dense=False)
    xy = I.coords3(p.x)
    d = {"r": t(p.r), "c": t(p.c), "x": t(xy), "y": t(xy.copy()),
         "u": torch.empty(p.n, dtype=torch.float64, device=DEV), "v": torch.empty(p.n, dtype=torch.float64, device=DEV)}
    prob = M.make_problem(d["r"], d["c"], x=d["x"], y=d["y"], kind=M.COST_SQEUCLID, scale=p.scale,
                          eps_target=eps or 1e-4, gamma_f=gamma_f, u_out=d["u"], v_out=d["v"])
    return p, d, prob


@pytest.fixture(scope="module")
def h():
    torch.cuda.set_device(0)
    with M.Handle(8192) as handle:
        yield handle


def test_server_matches_batch_alone_and_in_a_stream(h):
    gf = 2.0 ** 10
    ks = [12, 40, 9, 23, 31, 16, 50, 20, 11, 27]
    target = 4
    reqs = [grid_request(k, 7000 + i, gamma_f=gf) for i, k in enumerate(ks)]
    ref = h.solve_batch([grid_request(ks[target], 7000 + target, gamma_f=gf)[2]])[0]
    assert ref.status == M.MDOT_OK
    srv = M.Server(256 << 20)
    try:
        # alone
        p, d, prob = grid_request(ks[target], 7000 + target, gamma_f=gf)
        alone = srv.wait(srv.submit(prob, keep=(d,)), timeout=120)
        assert alone is not None and alone.status == M.MDOT_OK
        # in a stream: submitted one by one while the earlier ones run
        tickets = []
        for _, dd, pr in reqs:
            tickets.append(srv.submit(pr, keep=(dd,)))
            time.sleep(0.002)
        results = [srv.wait(tk, timeout=300) for tk in tickets]
    finally:
        srv.close()
    for r in results:
        assert r is not None and r.status == M.MDOT_OK
    m = results[target]
    for a in (alone, m):
        assert (a.cost, a.lower_bound, a.evals, a.iters, a.stages) == (ref.cost, ref.lower_bound, ref.evals,
                                                                       ref.iters, ref.stages)
    assert torch.equal(reqs[target][1]["u"], d["u"]) and torch.equal(reqs[target][1]["v"], d["v"])


def test_server_admits_within_a_small_budget():
    """A pool that holds about two requests still serves a queue of eight, in order."""
    reqs = [grid_request(k, 7100 + i, gamma_f=2.0 ** 8) for i, k in enumerate([30, 28, 26, 24, 22, 20, 18, 16])]
    per = 180 * 928          # workspace of one n = 900 request (180 bytes per padded element)
    srv = M.Server(2 * per + 4096)
    try:
        tickets = [srv.submit(pr, keep=(dd,)) for _, dd, pr in reqs]
        results = [srv.wait(tk, timeout=300) for tk in tickets]
    finally:
        srv.close()
    assert all(r is not None and r.status == M.MDOT_OK for r in results)


def test_batch_above_4096_matches_oracle(h):
    """n = 4100 (a point cloud: row sums in two chunks of 4096 and 4 rows) in the batched form,
    against the CPU oracle and against the cooperative solver on the same problem."""
    gf = 2.0 ** 9
    p = I.point_cloud_problem(4100, 7200)
    d = {"r": t(p.r), "c": t(p.c), "x": t(p.x), "y": t(p.y)}
    prob = M.make_problem(d["r"], d["c"], x=d["x"], y=d["y"], kind=M.COST_SQEUCLID, scale=p.scale, gamma_f=gf)
    prm = M.default_params(final_tol=FLOOR)
    r = h.solve_batch([prob], prm)[0]
    assert r.status == M.MDOT_OK, M.status_string(r.status)
    ref = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gf, final_tol=FLOOR)
    assert abs(r.cost - ref.cost) <= 1e-7, (r.cost, ref.cost)
    _, _, s = h.solve_points(d["r"], d["c"], d["x"], d["y"], M.COST_SQEUCLID, p.scale, 1e-6,
                             M.default_params(gamma_f=gf, final_tol=FLOOR))
    assert abs(r.cost - s.cost) <= 1e-7, (r.cost, s.cost)


def test_server_tickets_and_malformed_requests():
    srv = M.Server(64 << 20)
    try:
        p, d, prob = grid_request(8, 7300, gamma_f=2.0 ** 6)
        bad = M.make_problem(d["r"], d["c"], x=d["x"], y=d["y"], kind=M.COST_SQEUCLID, scale=-1.0, gamma_f=64.0)
        with pytest.raises(M.MdotError):
            srv.submit(bad)
        big = M.Problem()
        big.n = M.BATCH_MAX_N + 1
        with pytest.raises(M.MdotError):
            srv.submit(big)
        with pytest.raises(M.MdotError):
            srv.poll(123456789)
        tk = srv.submit(prob, keep=(d,))
        r = srv.wait(tk, timeout=120)
        assert r is not None and r.status == M.MDOT_OK
        with pytest.raises(M.MdotError):     # the ticket is released once collected
            srv.poll(tk)
    finally:
        srv.close()


def test_big_request_same_alone_and_in_a_stream(h):
    """Requests above 2048 go to a big lane (a cooperative solve on a share of the SMs): the same
    result bit for bit alone and while batched requests run beside it, and equal to the CPU
    oracle's on the same problem."""
    gf = 2.0 ** 11
    small = [grid_request(k, 7400 + i, gamma_f=gf) for i, k in enumerate([20, 33, 14, 41, 27, 18])]
    srv = M.Server(256 << 20, M.default_params(final_tol=FLOOR))
    try:
        p, d, prob = grid_request(48, 7450, gamma_f=gf)            # n = 2304
        alone = srv.wait(srv.submit(prob, keep=(d,)), timeout=300)
        u_alone = d["u"].clone()
        p2, d2, prob2 = grid_request(48, 7450, gamma_f=gf)
        tickets = [srv.submit(pr, keep=(dd,)) for _, dd, pr in small[:3]]
        tk = srv.submit(prob2, keep=(d2,))
        tickets += [srv.submit(pr, keep=(dd,)) for _, dd, pr in small[3:]]
        mixed = srv.wait(tk, timeout=300)
        others = [srv.wait(x, timeout=300) for x in tickets]
    finally:
        srv.close()
    assert alone is not None and mixed is not None
    assert alone.status == M.MDOT_OK and all(o is not None and o.status == M.MDOT_OK for o in others)
    assert (alone.cost, alone.lower_bound, alone.evals, alone.iters) == (mixed.cost, mixed.lower_bound, mixed.evals,
                                                                         mixed.iters)
    assert torch.equal(u_alone, d2["u"])
    pd = I.grid_problem(48, 7450)                                 # the same problem, dense C
    ref = O.solve(pd.C.astype(np.float64), pd.r, pd.c, gamma_f=gf, final_tol=FLOOR)
    assert abs(alone.cost - ref.cost) <= 1e-7, (alone.cost, ref.cost)


def test_tune_server_picks_a_measured_routing():
    """tune_server replays the same short trace under each candidate routing and returns the
    fastest.  Every request here is below both candidates' big_n, so all take the batched route
    and give bit-identical results under either routing."""
    torch.cuda.set_device(0)
    reqs, hold = [], []
    for q, k in enumerate((10, 12, 14, 16, 12, 10)):
        p, d, prob = grid_request(k, 7100 + q, eps=1e-5)
        reqs.append((0.01 * q, prob, tuple(d.values())))
        hold.append(d)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    cands = [dict(big_n=2048, big_lanes=2, lane_ctas=sms // 4), dict(big_n=1024, big_lanes=4, lane_ctas=sms // 8)]
    best, table = M.tune_server(1 << 28, reqs, cands)
    assert best in cands
    assert len(table) == 2 and all(row["problems_per_s"] > 0 for row in table)
    for row in table:
        assert row["statuses"] == [M.MDOT_OK] * len(reqs)
    assert table[0]["costs"] == table[1]["costs"]
