"""Write the stored expected values for the full-size workloads (n = 4096 grid histograms).

Calls only the oracle package (the CPU FP64 oracle and its exact-LP helper); nothing here comes
from the CUDA library.  Each record holds, for one (cost kind, seed, target gap):
  H_min, the Prop. 2 gamma_f, the oracle's rounded-plan cost and c-transform bound, its
  evaluation counts, and the exact OT value (column generation priced over all n^2 arcs).
Usage:  python tests/golden/make_golden.py [k] [eps ...]   (defaults: k = 64, eps = 1e-6)
        python tests/golden/make_golden.py --exact-only [k [kind]]   (only the exact OT values)
        python tests/golden/make_golden.py --exact-wide k kind k_init add_per_row   (the same with a
            wider initial arc set and more arcs added per round)
        python tests/golden/make_golden.py --exact-seeded k kind eps width   (the same, its first
            arc set seeded by an oracle solve at target eps: every arc whose reduced cost against
            the solve's potentials f = u/gamma_f, g = v/gamma_f is at most width; the oracle's
            OpenMP build, same arithmetic, on every host core)
        python tests/golden/make_golden.py --seeds k kind eps width seed ...   (for more seeds of the
            benchmark instance: the oracle solve at target eps into grid{n}.json, and the exact OT
            value seeded by that solve's nearly tight arcs into both files)
        python tests/golden/make_golden.py --oracle-only k kind eps   (one oracle solve, no exact value)
        python tests/golden/make_golden.py --line n ...   (exact costs of the points-on-a-line
            problems, seed 11: the monotone coupling, into tests/golden/line_exact.json)
        python tests/golden/make_golden.py --serve   (oracle costs of the served trace's requests
            with n <= 1024 among its first 100, into tests/golden/serve_oracle.json)
        python tests/golden/make_golden.py --cloud n seed gamma_f final_tol   (the oracle solve of
            one App. C point cloud, into tests/golden/cloud_oracle.json)
Runs the cases in parallel worker processes (spawn) and merges each finished case into
tests/golden/grid{n}.json (or exact{n}.json) as soon as it completes.
"""
from __future__ import annotations

import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

SEED = 2000          # problem seed of the n = 4096 benchmark instance


def one_case(args):
    k, kind, seed, eps = args[:4]
    with_exact = args[4] if len(args) > 4 else True
    import numpy as np
    import oracle as O
    from oracle import exact as E
    from paper_2307_08507_gb300 import inputs as I

    p = I.grid_problem(k, seed, kind=kind)
    C = p.C.astype(np.float64)
    H = min(O.entropy(p.r), O.entropy(p.c))
    t0 = time.time()
    res = O.solve(C, p.r, p.c, eps_target=eps)
    t_solve = time.time() - t0
    # exact optimum: candidate arcs = arcs that are nearly tight for the oracle's potentials
    f, g = res.u / res.gamma_f, res.v / res.gamma_f
    val, rounds, t_exact = None, None, None
    if with_exact:
        t0 = time.time()
        val, fd, gd, rounds = E.exact_ot_colgen(C, p.r, p.c, k_init=4)
        t_exact = time.time() - t0
    return {
        "k": k, "n": p.n, "kind": kind, "seed": seed, "eps_target": eps, "H_min": H,
        "gamma_f": res.gamma_f, "oracle_cost": res.cost, "oracle_lb": res.lb,
        "oracle_evals": int(res.stats.evals), "oracle_iters": int(res.stats.iters),
        "oracle_ls_trials": int(res.stats.ls_trials), "oracle_stages": int(res.stats.stages),
        "oracle_status": int(res.status), "oracle_grad_l1": res.stats.grad_l1,
        "oracle_seconds": t_solve, "exact_ot": val, "exact_rounds": rounds,
        "exact_seconds": t_exact, "true_gap": (res.cost - val) if val is not None else None,
        "f_g_span": [float(f.min()), float(f.max()), float(g.min()), float(g.max())],
    }


def exact_case(args):
    k, kind, seed = args[:3]
    k_init, add = (args[3], args[4]) if len(args) > 4 else (4, 8)
    import numpy as np
    from oracle import exact as E
    from paper_2307_08507_gb300 import inputs as I
    p = I.grid_problem(k, seed, kind=kind)
    t0 = time.time()
    val, f, g, rounds = E.exact_ot_colgen(p.C.astype(np.float64), p.r, p.c, k_init=k_init, add_per_row=add)
    return {"k": k, "n": p.n, "kind": kind, "seed": seed, "exact_ot": val, "exact_rounds": rounds,
            "exact_seconds": time.time() - t0}


def exact_seeded_case(k, kind, seed, eps, width):
    """Exact OT by column generation whose first arc set holds every arc that is within `width`
    of tight for the potentials of an oracle solve at target gap eps."""
    import numpy as np
    import oracle as O
    from oracle import exact as E
    from paper_2307_08507_gb300 import inputs as I
    O.use_openmp(True)
    p = I.grid_problem(k, seed, kind=kind)
    C = p.C.astype(np.float64)
    t0 = time.time()
    res = O.solve(C, p.r, p.c, eps_target=eps)
    t_seed = time.time() - t0
    f, g = res.u / res.gamma_f, res.v / res.gamma_f
    t0 = time.time()
    val, fd, gd, rounds = E.exact_ot_colgen(C, p.r, p.c, k_init=4, seed_f=f, seed_g=g,
                                            seed_width=width)
    return {"k": k, "n": p.n, "kind": kind, "seed": seed, "exact_ot": val, "exact_rounds": rounds,
            "exact_seconds": time.time() - t0, "seed_eps": eps, "seed_width": width,
            "seed_seconds": t_seed}


def seeds_case(k, kind, seed, eps, width):
    """One more seed of the benchmark instance: the oracle solve at target eps (OpenMP build) and
    the exact OT value by column generation seeded by that solve's potentials."""
    import numpy as np
    import oracle as O
    from oracle import exact as E
    from paper_2307_08507_gb300 import inputs as I
    O.use_openmp(True)
    p = I.grid_problem(k, seed, kind=kind)
    C = p.C.astype(np.float64)
    H = min(O.entropy(p.r), O.entropy(p.c))
    t0 = time.time()
    res = O.solve(C, p.r, p.c, eps_target=eps)
    t_solve = time.time() - t0
    f, g = res.u / res.gamma_f, res.v / res.gamma_f
    t0 = time.time()
    val, _, _, rounds = E.exact_ot_colgen(C, p.r, p.c, k_init=4, seed_f=f, seed_g=g, seed_width=width)
    t_exact = time.time() - t0
    grid = {
        "k": k, "n": p.n, "kind": kind, "seed": seed, "eps_target": eps, "H_min": H,
        "gamma_f": res.gamma_f, "oracle_cost": res.cost, "oracle_lb": res.lb,
        "oracle_evals": int(res.stats.evals), "oracle_iters": int(res.stats.iters),
        "oracle_ls_trials": int(res.stats.ls_trials), "oracle_stages": int(res.stats.stages),
        "oracle_status": int(res.status), "oracle_grad_l1": res.stats.grad_l1,
        "oracle_seconds": t_solve, "oracle_threads": "OpenMP build, every host core",
        "exact_ot": val, "exact_rounds": rounds, "exact_seconds": t_exact,
        "true_gap": res.cost - val,
        "f_g_span": [float(f.min()), float(f.max()), float(g.min()), float(g.max())],
    }
    exact = {"k": k, "n": p.n, "kind": kind, "seed": seed, "exact_ot": val, "exact_rounds": rounds,
             "exact_seconds": t_exact, "seed_eps": eps, "seed_width": width, "seed_seconds": t_solve}
    return grid, exact


def line_case(n, seed=11):
    import numpy as np
    from oracle import exact as E
    from paper_2307_08507_gb300 import inputs as I
    p = I.line_problem(n, seed)
    s32 = np.float32(p.scale)
    # the cost in the float32 order the problem defines: d = fl(x - y), C = fl(fl(d * d) * s)
    val = E.monotone_1d(p.x[:, 0], p.y[:, 0], p.r, p.c,
                        lambda d: float(np.float32(np.float32(d) * np.float32(d)) * s32))
    return {"n": n, "seed": seed, "exact_ot": val, "method": "monotone coupling of the sorted supports"}


def serve_case(args):
    """Oracle cost of one request of the serving trace (seed 5000, 200 requests): a k x k grid
    histogram pair with the squared-Euclidean grid cost at the request's target gap."""
    idx, k, eps, sd = args
    import numpy as np
    import oracle as O
    from paper_2307_08507_gb300 import inputs as I
    r, c = I.grid_histogram(k, 2 * sd), I.grid_histogram(k, 2 * sd + 1)
    C = I.grid_cost(k, "l2sq").astype(np.float64)
    t0 = time.time()
    res = O.solve(C, r, c, eps_target=eps)
    return {"index": idx, "seed": SERVE_SEED, "count": SERVE_COUNT, "k": k, "n": k * k, "eps_target": eps,
            "oracle_cost": res.cost, "oracle_evals": int(res.stats.evals), "oracle_seconds": time.time() - t0}


SERVE_SEED, SERVE_COUNT = 5000, 200


def cloud_case(n, seed, gamma_f, final_tol):
    """Oracle solve of the point cloud inputs.point_cloud_problem(n, seed) (x ~ N(0, I3),
    y ~ U[-1, 1]^3, uniform weights) at the given gamma_f and last-stage tolerance."""
    import numpy as np
    import oracle as O
    from paper_2307_08507_gb300 import inputs as I
    p = I.point_cloud_problem(n, seed)
    t0 = time.time()
    res = O.solve(p.C.astype(np.float64), p.r, p.c, gamma_f=gamma_f, final_tol=final_tol)
    return {"n": n, "seed": seed, "gamma_f": gamma_f, "final_tol": final_tol, "oracle_cost": res.cost,
            "oracle_status": int(res.status), "oracle_evals": int(res.stats.evals),
            "oracle_grad_l1": res.stats.grad_l1, "oracle_seconds": time.time() - t0}


def _merge(path, record, key):
    old = []
    if os.path.exists(path):
        with open(path) as fh:
            old = json.load(fh)["cases"]
    keyed = {key(c): c for c in old}
    keyed[key(record)] = record
    with open(path, "w") as fh:
        json.dump({"generator": "tests/golden/make_golden.py (CPU FP64 oracle + exact LP)",
                   "cases": sorted(keyed.values(), key=lambda c: tuple(str(x) for x in key(c)))},
                  fh, indent=1)


def main():
    ctx = mp.get_context("spawn")
    if len(sys.argv) > 1 and sys.argv[1] == "--exact-only":
        k = int(sys.argv[2]) if len(sys.argv) > 2 else 64
        kinds = sys.argv[3:] or ["l2sq", "l1"]
        cases = [(k, kind, SEED) for kind in kinds]
        path = os.path.join(HERE, f"exact{k * k}.json")
        with ctx.Pool(len(cases)) as pool:
            for rec in pool.imap_unordered(exact_case, cases):
                _merge(path, rec, lambda c: (c["kind"], c["seed"]))
                print(json.dumps(rec), flush=True)
        return
    if len(sys.argv) > 1 and sys.argv[1] == "--exact-wide":
        k, kind, k_init, add = int(sys.argv[2]), sys.argv[3], int(sys.argv[4]), int(sys.argv[5])
        rec = exact_case((k, kind, SEED, k_init, add))
        _merge(os.path.join(HERE, f"exact{k * k}.json"), rec, lambda c: (c["kind"], c["seed"]))
        print(json.dumps(rec), flush=True)
        return
    if len(sys.argv) > 1 and sys.argv[1] == "--exact-seeded":
        k, kind, eps, width = int(sys.argv[2]), sys.argv[3], float(sys.argv[4]), float(sys.argv[5])
        rec = exact_seeded_case(k, kind, SEED, eps, width)
        _merge(os.path.join(HERE, f"exact{k * k}.json"), rec, lambda c: (c["kind"], c["seed"]))
        print(json.dumps(rec), flush=True)
        return
    if len(sys.argv) > 1 and sys.argv[1] == "--seeds":
        k, kind, eps, width = int(sys.argv[2]), sys.argv[3], float(sys.argv[4]), float(sys.argv[5])
        for seed in [int(a) for a in sys.argv[6:]]:
            grid, exact = seeds_case(k, kind, seed, eps, width)
            _merge(os.path.join(HERE, f"grid{k * k}.json"), grid,
                   lambda c: (c["kind"], c["seed"], c["eps_target"]))
            _merge(os.path.join(HERE, f"exact{k * k}.json"), exact, lambda c: (c["kind"], c["seed"]))
            print(json.dumps(grid), flush=True)
        return
    if len(sys.argv) > 1 and sys.argv[1] == "--serve":
        # the first requests of the served trace with n <= 1024 among its first 100
        from paper_2307_08507_gb300 import inputs as I
        trace = I.serving_trace(SERVE_COUNT, SERVE_SEED)
        cases = [(i, k, eps, sd) for i, (ta, k, eps, sd) in enumerate(trace[:100]) if k * k <= 1024]
        path = os.path.join(HERE, "serve_oracle.json")
        with ctx.Pool(min(len(cases), os.cpu_count() or 1)) as pool:
            for rec in pool.imap_unordered(serve_case, cases):
                _merge(path, rec, lambda c: (c["seed"], c["index"]))
                print(json.dumps(rec), flush=True)
        return
    if len(sys.argv) > 1 and sys.argv[1] == "--cloud":
        rec = cloud_case(int(sys.argv[2]), int(sys.argv[3]), float(sys.argv[4]), float(sys.argv[5]))
        _merge(os.path.join(HERE, "cloud_oracle.json"), rec,
               lambda c: (c["n"], c["seed"], c["gamma_f"], c["final_tol"]))
        print(json.dumps(rec), flush=True)
        return
    if len(sys.argv) > 1 and sys.argv[1] == "--line":
        for n in [int(a) for a in sys.argv[2:]]:
            rec = line_case(n)
            _merge(os.path.join(HERE, "line_exact.json"), rec, lambda c: (c["n"], c["seed"]))
            print(json.dumps(rec), flush=True)
        return
    if len(sys.argv) > 1 and sys.argv[1] == "--oracle-only":
        k, kind, eps = int(sys.argv[2]), sys.argv[3], float(sys.argv[4])
        rec = one_case((k, kind, SEED, eps, False))
        _merge(os.path.join(HERE, f"grid{k * k}.json"), rec, lambda c: (c["kind"], c["seed"], c["eps_target"]))
        print(json.dumps(rec), flush=True)
        return
    k = int(sys.argv[1]) if len(sys.argv) > 1 else 64
    eps_list = [float(a) for a in sys.argv[2:]] or [1e-6]
    cases = [(k, kind, SEED, eps) for eps in eps_list for kind in ("l2sq", "l1")]
    path = os.path.join(HERE, f"grid{k * k}.json")
    with ctx.Pool(min(len(cases), os.cpu_count() or 1)) as pool:
        for rec in pool.imap_unordered(one_case, cases):
            _merge(path, rec, lambda c: (c["kind"], c["seed"], c["eps_target"]))
            print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
