"""Benchmark: time to rounded-plan optimality gap 1e-6 at n = 4096 (MDOT-PNCG, one GB300).

One step = one full solve through the C ABI (mdot_solve): H_min and validation, every MDOT stage
(PNCG + line search on the device), rounding (Alg. 3) and the lower bound, on a 64 x 64 grid-
histogram problem with squared-Euclidean cost (fp32 C, 64 MiB), eps_target = 1e-6 (gamma_f from
Prop. 2).  Inputs are resident in HBM when the timed region starts; L2 is flushed (256 MiB write)
between timed steps.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU FP64 oracle on this machine's host cores instead (a bounded sample
of its dual evaluations, scaled by the evaluation count of the full oracle solve).
N > 1 (torchrun): every rank solves its own instance (replicas, weak scaling); rank 0 reports the
max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 64                 # n = 4096
SEED = 2000
EPS = 1e-6
METRIC = "time to gap 1e-6 at n=4096"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample-evals", type=int, default=0, help="oracle evaluations in the CPU sample")
    ap.add_argument("--case", default="solve",
                    choices=["solve", "dual_eval", "dual_eval_regen", "dual_eval_regen_tc", "stage", "batch", "serve",
                             "tune_serve", "sinkhorn", "large_n", "nscale", "hmin", "phases"],
                    help="dual_eval / stage: run only that kernel (for profiler captures); sinkhorn, large_n, "
                         "nscale, hmin: the comparison studies (one JSON line per solve)")
    ap.add_argument("--grid", type=int, default=64, help="k of the k x k grid for --case runs")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-form measurement")
    ap.add_argument("--no-sweep", action="store_true", help="skip the n=4096 gap sweep (both costs, 1e-4..1e-7)")
    ap.add_argument("--serve-count", type=int, default=200,
                    help="requests of the serving trace replayed at the configured rate (half as many at 0.5x and "
                         "0.9x of the measured capacity and one problem per launch; 0: skip)")
    ap.add_argument("--serve-big-n", type=int, default=None, help="server routing: n above which a big lane solves")
    ap.add_argument("--serve-lanes", type=int, default=None, help="server routing: big lanes")
    ap.add_argument("--serve-lane-ctas", type=int, default=None, help="server routing: CTAs per big lane")
    return ap.parse_args()


# fp32 operations per entry of an evaluation with the squared-Euclidean cost regenerated in the
# exact order of the dense cost: 3 differences, 3 products, 2 sums, the scale (9); the exponent
# argument from the row and column constants (4: two adds, two fmas); the row and column sums (2)
ALU_OPS_PER_ENTRY = 15
# with the cost on the tensor cores: the scale of the exact integer distance (1), the exponent
# argument (4) and the row and column sums (2)
ALU_OPS_PER_ENTRY_TC = 7


def alu_peak_ops():
    """fp32 issue bound of the GPU: SMs x 128 fp32 lanes per SM per clock x the maximum SM clock
    (2070 MHz on GB300)."""
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count * 128 * 2070e6


def golden_case(kind="l2sq"):
    path = os.path.join(ROOT, "tests", "golden", f"grid{N_GRID * N_GRID}.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for c in json.load(fh)["cases"]:
            if c["kind"] == kind and c["seed"] == SEED and abs(c["eps_target"] - EPS) < 1e-15:
                return c
    return None


def golden_record(kind, eps):
    path = os.path.join(ROOT, "tests", "golden", f"grid{N_GRID * N_GRID}.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for c in json.load(fh)["cases"]:
            if c["kind"] == kind and c["seed"] == SEED and abs(c["eps_target"] - eps) <= 1e-15 * eps:
                return c
    return None


def exact_value(kind="l2sq"):
    """Exact OT value of the benchmark instance (column generation, tests/golden/make_golden.py)."""
    path = os.path.join(ROOT, "tests", "golden", f"exact{N_GRID * N_GRID}.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        for c in json.load(fh)["cases"]:
            if c["kind"] == kind and c["seed"] == SEED and c.get("exact_ot") is not None:
                return c["exact_ot"]
    return None


def gap_sweep(h, dev, stream):
    """The n = 4096 instance (64 x 64 grid, seed 2000) with both costs (squared Euclidean, L1) at
    target gaps 1e-4 ... 1e-7: one untimed and one timed solve each (CUDA events on the handle's
    stream), the true gap against the exact optimum where it is stored, an upper bound on the true
    gap (cost minus the c-transform bound of a gamma_f = 2^21 solve), the certificate, and the
    difference to the FP64 oracle's rounded cost on the same instance (tests/golden/)."""
    import torch
    import paper_2307_08507_gb300 as M
    from paper_2307_08507_gb300 import inputs as I
    rows = []
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for kind in ("l2sq", "l1"):
        p = I.grid_problem(N_GRID, SEED, kind=kind)
        r, c, C = (torch.from_numpy(a).to(dev) for a in (p.r, p.c, p.C))
        exact = exact_value(kind)
        for eps in (1e-4, 1e-5, 1e-6, 1e-7):
            h.solve(r, c, C, eps)
            ev0.record(stream)
            _, _, res = h.solve(r, c, C, eps, check=False)
            ev1.record(stream)
            torch.cuda.synchronize()
            g = golden_record(kind, eps)
            rows.append({"cost_kind": kind, "eps_target": eps, "status": M.status_string(res.status),
                         "seconds": ev0.elapsed_time(ev1) / 1e3, "gamma_f": res.info.gamma_f,
                         "evals": res.info.evals, "evals_fp64": res.info.evals_fp64, "cost": res.cost,
                         "true_gap": (res.cost - exact) if exact is not None else None,
                         "gap_cert": res.gap_cert,
                         "meets_target": (res.cost - exact <= eps) if exact is not None else None,
                         "cost_minus_oracle": (res.cost - g["oracle_cost"]) if g else None})
        # an upper bound on every row's true gap without the exact optimum: the c-transform bound of
        # a solve at gamma_f = 2^21 is a feasible OT dual value, so OT >= it (weak duality)
        _, _, hi = h.solve(r, c, C, 1e-6, M.default_params(gamma_f=2.0 ** 21), check=False)
        lb_hi = hi.cost - hi.gap_cert
        for row in rows:
            if row["cost_kind"] == kind:
                row["true_gap_bound"] = row["cost"] - lb_hi
        del C
    return rows


def max_over_ranks(x: float, dist, device) -> float:
    """Largest value over the ranks (the job's time is its slowest replica's)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# the sources the dense stage kernel (the roofline's kernel) is compiled from
STAGE_KERNEL_SOURCES = ("k_stage.cu", "mdot_device.cuh", "solver_kernels.cuh")


def kernel_source_hash() -> str:
    """sha256 over the CUDA sources the stage kernel is compiled from (STAGE_KERNEL_SOURCES in
    csrc/, in that order): a recorded ncu traffic figure stays valid while these are unchanged."""
    import hashlib
    hsh = hashlib.sha256()
    for name in STAGE_KERNEL_SOURCES:
        f = os.path.join(ROOT, "paper_2307_08507_gb300", "csrc", name)
        hsh.update(name.encode())
        with open(f, "rb") as fh:
            hsh.update(fh.read())
    return hsh.hexdigest()


def ncu_traffic(kernel: str):
    """DRAM bytes (read + write) per launch of `kernel` from the ncu capture recorded in
    profiles/ncu_traffic.json, or None when that capture was taken from other sources than the
    ones built now (the recorded sha256 of the CUDA sources differs)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    rec = d.get("kernels", {}).get(kernel)
    if rec is None or d.get("source_sha256") != kernel_source_hash():
        return None
    return float(rec["dram_bytes_per_launch"])


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index=0):
        self.proc = None
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"mdot_clocks_{os.getpid()}.csv")
        self.index = index

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines() if l.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() in ("active", "1", "0x1"):
                        reasons.append(nm) if False else reasons.add(nm)
            except Exception:
                continue
        if sm:
            sm.sort()
            out["sm_mhz"] = sm[len(sm) // 2]
            out["sm_max_mhz"] = max(mx)
            out["samples"] = len(sm)
        out["reasons"] = sorted(reasons)
        return out


# ---------------------------------------------------------------------------------------------
# reference arm and CPU baseline: the oracle as it stands, on the host cores
# ---------------------------------------------------------------------------------------------
def oracle_sample(n_evals: int):
    """Time n_evals oracle dual evaluations of the n = 4096 problem; return seconds per eval."""
    import numpy as np
    import oracle as O
    from paper_2307_08507_gb300 import inputs as I
    p = I.grid_problem(N_GRID, SEED)
    C = p.C.astype(np.float64)
    gamma = 2.0 ** 12
    u, v = np.log(p.r), np.log(p.c)
    O.dual_eval(C[:64, :64], u[:64], v[:64], gamma)          # load the library outside the timing
    t0 = time.perf_counter()
    for _ in range(n_evals):
        O.dual_eval(C, u, v, gamma)
    return (time.perf_counter() - t0) / n_evals


def oracle_sample_all_cores(n_evals: int):
    """The same timing on the OpenMP build of the oracle (rows and column strips of each dual
    evaluation on every host core, identical arithmetic); returns (seconds per eval, threads)."""
    import numpy as np
    import oracle as O
    from paper_2307_08507_gb300 import inputs as I
    run, threads = O.omp_dual_eval_timer()
    p = I.grid_problem(N_GRID, SEED)
    C = p.C.astype(np.float64)
    gamma = 2.0 ** 12
    u, v = np.log(p.r), np.log(p.c)
    run(C, u, v, gamma)                                          # warm (threads, pages)
    t0 = time.perf_counter()
    for _ in range(n_evals):
        run(C, u, v, gamma)
    return (time.perf_counter() - t0) / n_evals, threads


def cpu_solve_estimate(n_evals: int):
    g = golden_case()
    per_eval = oracle_sample(n_evals)
    evals = g["oracle_evals"] if g else 3000
    return per_eval * evals, per_eval, evals


def run_reference(args, rank, world):
    """The reference arm: the CPU FP64 oracle (the paper publishes no code), its dual evaluation on
    every host core (OpenMP build, same arithmetic).  One step = n_evals dual evaluations of the
    n = 4096 benchmark problem; ms_per_step is that step's measured wall time.  The metric (seconds
    to gap 1e-6, one full solve) is extrapolated: seconds per evaluation x the evaluation count of
    the full oracle solve of the same instance (tests/golden/grid4096.json)."""
    if rank != 0:
        return
    n_evals = args.cpu_sample_evals or 4
    g = golden_case()
    evals = g["oracle_evals"] if g else 3000
    for _ in range(args.warmup):
        oracle_sample_all_cores(1)
    per = []
    threads = 1
    for _ in range(args.steps):
        pe, threads = oracle_sample_all_cores(n_evals)
        per.append(pe)
    per_eval = sum(per) / len(per)
    value = per_eval * evals
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_eval * n_evals * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded grid histograms, Sec. 5.1 shapes)",
        "config": {"workload": "grid64x64_l2sq_n4096_eps1e-6", "n": N_GRID * N_GRID, "seed": SEED,
                   "eps_target": EPS, "l2": "oracle on CPU"},
        "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle",
                         "sample": f"per-evaluation x evaluations extrapolation: {n_evals} FP64 dual "
                                   f"evaluations at n=4096 per step on {threads} threads "
                                   f"({per_eval:.4f} s each), x the {evals} evaluations of the full "
                                   f"oracle solve"},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# batched form: 512 point-cloud problems, n uniform in [256, 4096], one persistent launch
# ---------------------------------------------------------------------------------------------
BATCH_COUNT = 512
BATCH_EPS = 1e-6
BATCH_SEED = 4000


def batch_problems(dev, count=BATCH_COUNT, seed=BATCH_SEED):
    """Point clouds x ~ N(0, I3), y ~ U[-1, 1]^3, uniform weights (App. C style), sizes from the
    seeded generator; the cost scale 1 / max D uses the generator's fp32 formula (on the GPU)."""
    import numpy as np
    import torch
    from paper_2307_08507_gb300 import inputs as I
    sizes = I.batch_sizes(count, seed)
    out = []
    for k, n in enumerate(sizes):
        rng = I.rng_for(seed + k)
        x = rng.standard_normal((int(n), 3)).astype(np.float32)
        y = rng.uniform(-1.0, 1.0, size=(int(n), 3)).astype(np.float32)
        xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
        d0 = xt[:, None, 0] - yt[None, :, 0]
        d1 = xt[:, None, 1] - yt[None, :, 1]
        d2 = xt[:, None, 2] - yt[None, :, 2]
        dmax = float(((d0 * d0 + d1 * d1) + d2 * d2).max().item())
        w = torch.full((int(n),), 1.0 / int(n), dtype=torch.float64, device=dev)
        out.append({"n": int(n), "x": xt, "y": yt, "r": w, "c": w.clone(),
                    "scale": float(np.float32(1.0 / dmax))})
        del d0, d1, d2
    return out


def _not_converged_summary(probs, res, M):
    """The problems whose last stage ended above its tolerance: how many, their sizes and their
    final ||grad g||_1 (quartiles), to set against the tolerance floor fp32_floor."""
    bad = [(probs[k]["n"], r.grad_l1) for k, r in enumerate(res) if r.status == M.MDOT_ERR_NOT_CONVERGED]
    if not bad:
        return {"count": 0}
    ns = sorted(b[0] for b in bad)
    gs = sorted(b[1] for b in bad)
    q = lambda v, f: v[min(len(v) - 1, int(f * len(v)))]
    return {"count": len(bad), "n_min": ns[0], "n_median": q(ns, 0.5), "n_max": ns[-1],
            "grad_l1_quartiles": [gs[0], q(gs, 0.25), q(gs, 0.5), q(gs, 0.75), gs[-1]],
            "fp32_floor": M.default_params().fp32_floor}


def measure_batch(h, dev, stream, sample_single=128):
    import torch
    import paper_2307_08507_gb300 as M
    probs = batch_problems(dev)
    plist = [M.make_problem(q["r"], q["c"], x=q["x"], y=q["y"], kind=M.COST_SQEUCLID, scale=q["scale"],
                            eps_target=BATCH_EPS) for q in probs]
    h.solve_batch(plist[:8])                                       # warm-up (small subset)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    # the fixed tiles (the default variant for every size) ...
    h.set_batch_tuning(M.BatchTuning())
    ev0.record(stream)
    res_fixed = h.solve_batch(plist)
    ev1.record(stream)
    torch.cuda.synchronize()
    t_fixed = ev0.elapsed_time(ev1) / 1e3
    # ... and the table the autotuner picks (each candidate timed on 128 problems of the batch,
    # evenly spaced in size, at gamma_f <= 2^12)
    t0 = time.perf_counter()
    tuned = h.tune_batch(plist, sample=128)
    t_tune = time.perf_counter() - t0
    if tuned.narrow_below == 0:
        # the tuner kept the fixed table: the same launches, so the fixed run stands for both
        res, t_batch = res_fixed, t_fixed
    else:
        ev0.record(stream)
        res = h.solve_batch(plist)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_batch = ev0.elapsed_time(ev1) / 1e3
    ok = sum(1 for r in res if r.status == M.MDOT_OK)
    # one problem per launch (cooperative multi-CTA solve) on a stratified sample, same accuracy
    order = sorted(range(len(probs)), key=lambda k: probs[k]["n"])
    pick = order[:: max(1, len(order) // sample_single)][:sample_single]
    t_single, dcost, evals_b, evals_s = 0.0, [], 0, 0
    st_single, st_batch_pick = {}, {}
    for k in pick:
        q = probs[k]
        ev0.record(stream)
        _, _, rs = h.solve_points(q["r"], q["c"], q["x"], q["y"], M.COST_SQEUCLID, q["scale"], BATCH_EPS,
                                  check=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_single += ev0.elapsed_time(ev1) / 1e3
        dcost.append(abs(rs.cost - res[k].cost))
        evals_b += res[k].evals
        evals_s += rs.info.evals
        st_single[M.status_string(rs.status)] = st_single.get(M.status_string(rs.status), 0) + 1
        st_batch_pick[M.status_string(res[k].status)] = st_batch_pick.get(M.status_string(res[k].status), 0) + 1
    t_single_all = t_single * len(probs) / len(pick)
    # entries of all evaluations of the batch per second, against the fp32 issue bound (the pass
    # regenerates the cost: ALU_OPS_PER_ENTRY fp32 operations per entry)
    entries = float(sum(r.evals * probs[k]["n"] ** 2 for k, r in enumerate(res)))
    alu = alu_peak_ops()
    return {"problems": len(probs), "n_range": [min(q["n"] for q in probs), max(q["n"] for q in probs)],
            "eps_target": BATCH_EPS, "cost": "regenerated squared Euclidean (point clouds)",
            "seconds": t_batch, "problems_per_s": len(probs) / t_batch, "ok": ok,
            "fixed_tiles": {"seconds": t_fixed, "problems_per_s": len(probs) / t_fixed,
                            "ok": sum(1 for r in res_fixed if r.status == M.MDOT_OK)},
            "tuning": {**tuned.as_dict(), "tuning_seconds": t_tune, "sample": 128,
                       "candidates": "table k: size buckets below k on variant 1, the rest on variant 0",
                       "buckets": ["n<512", "n<1024", "n<2048", "n<4096", "n<=8192"],
                       "variants": ["256 threads, 1 problem per SM", "128 threads, 2 problems per SM"]},
            "max_abs_cost_diff_tuned_vs_fixed": max(abs(a.cost - b.cost) for a, b in zip(res, res_fixed)),
            "statuses": {M.status_string(st): sum(1 for r in res if r.status == st) for st in {r.status for r in res}},
            "not_converged": _not_converged_summary(probs, res, M),
            "roofline": {"kernel": "batch_kernel<squared Euclidean> (one CTA per problem)", "bound": "alu",
                         "entries_per_s": entries / t_batch, "ops_per_entry": ALU_OPS_PER_ENTRY,
                         "achieved": entries * ALU_OPS_PER_ENTRY / t_batch / 1e12, "peak": alu / 1e12,
                         "unit": "Tops/s", "frac": entries * ALU_OPS_PER_ENTRY / t_batch / alu},
            "one_per_launch_sample": len(pick), "one_per_launch_seconds_sample": t_single,
            "one_per_launch_statuses": st_single, "batched_statuses_on_that_sample": st_batch_pick,
            "one_per_launch_problems_per_s": len(probs) / t_single_all,
            "speedup_vs_one_per_launch": t_single_all / t_batch,
            "max_abs_cost_diff_vs_one_per_launch": max(dcost), "evals_batch_sample": evals_b,
            "evals_single_sample": evals_s}


# ---------------------------------------------------------------------------------------------
# served form: a Poisson trace of grid-histogram requests replayed in real time
# ---------------------------------------------------------------------------------------------
SERVE_SEED = 5000
SERVE_WORKSPACE = 2 << 30          # HBM budget of the server's workspace pool (bytes)


def serving_oracle_costs():
    """Stored FP64 oracle costs of a sample of the serving trace's requests (tests/golden/
    serve_oracle.json, written by tests/golden/make_golden.py --serve): {trace index: cost}."""
    path = os.path.join(ROOT, "tests", "golden", "serve_oracle.json")
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return {c["index"]: c["oracle_cost"] for c in json.load(fh)["cases"] if c["seed"] == SERVE_SEED}


def serving_requests(dev, count, seed=SERVE_SEED):
    """Requests of the serving trace: k x k grid histograms (Sec. 5.1 shapes), squared-Euclidean
    cost regenerated from the cell coordinates, target gap from the trace; inputs resident on the
    device before the replay starts.  Each entry: (arrival s, n, eps, mdot_problem, tensors)."""
    import torch
    import paper_2307_08507_gb300 as M
    from paper_2307_08507_gb300 import inputs as I
    coords = {}
    reqs = []
    for (ta, k, eps, sd) in I.serving_trace(count, seed):
        if k not in coords:
            xy = torch.from_numpy(I.coords3(I.grid_coords(k))).to(dev)
            coords[k] = (xy, float(I.grid_cost_scale(k, "l2sq")))
        xy, scale = coords[k]
        r = torch.from_numpy(I.grid_histogram(k, 2 * sd)).to(dev)
        c = torch.from_numpy(I.grid_histogram(k, 2 * sd + 1)).to(dev)
        prob = M.make_problem(r, c, x=xy, y=xy, kind=M.COST_SQEUCLID, scale=scale, eps_target=eps)
        reqs.append((ta, k * k, eps, prob, (r, c, xy, scale)))
    return reqs


def measure_serving(dev, reqs, big_n=None, big_lanes=None, lane_ctas=None, rate=None):
    """Replay the requests (serving_requests) in real time through mdot_server_* (at the trace's
    200/s, or at mean rate `rate` with the same arrival pattern rescaled); latency = completion seen
    by the client - scheduled arrival.  Returns the summary and the costs in request order."""
    import numpy as np
    import torch
    import paper_2307_08507_gb300 as M
    if rate is not None:
        reqs = [(q[0] * 200.0 / rate,) + tuple(q[1:]) for q in reqs]
    torch.cuda.synchronize()
    srv = M.Server(SERVE_WORKSPACE, big_n=big_n, big_lanes=big_lanes, lane_ctas=lane_ctas)
    lat, done_at, evals, status_ok, statuses, big_lat = [], [], 0, 0, {}, []
    costs = [None] * len(reqs)
    try:
        # warm-up request (kernel load, first launch)
        srv.wait(srv.submit(reqs[0][3], keep=reqs[0][4]), timeout=600)
        pending = {}
        i = 0
        t0 = time.perf_counter()
        while i < len(reqs) or pending:
            now = time.perf_counter() - t0
            while i < len(reqs) and reqs[i][0] <= now:
                pending[srv.submit(reqs[i][3], keep=reqs[i][4])] = (reqs[i][0], reqs[i][1], i)
                i += 1
            for tk in list(pending):
                r = srv.poll(tk)
                if r is not None:
                    tn = time.perf_counter() - t0
                    ta, nq, idx = pending.pop(tk)
                    lat.append(tn - ta)
                    if nq > 2048:
                        big_lat.append(tn - ta)
                    done_at.append(tn)
                    evals += r.evals
                    costs[idx] = r.cost
                    status_ok += int(r.status == M.MDOT_OK)
                    key = M.status_string(r.status)
                    statuses[key] = statuses.get(key, 0) + 1
            time.sleep(0.0002)
        span = max(done_at) - reqs[0][0]
    finally:
        srv.close()
    lat = np.array(lat)
    n = np.array([q[1] for q in reqs])
    summary = {"requests": len(reqs), "offered_rate_per_s": len(reqs) / reqs[-1][0],
               "n_range": [int(n.min()), int(n.max())], "n_median": float(np.median(n)),
               "gaps": [1e-4, 1e-5, 1e-6, 1e-7], "workspace_bytes": SERVE_WORKSPACE,
               "cost": "regenerated squared Euclidean (grid histograms)",
               "problems_per_s": len(lat) / span, "latency_p50_s": float(np.percentile(lat, 50)),
               "latency_p99_s": float(np.percentile(lat, 99)), "latency_max_s": float(lat.max()),
               "latency_p50_n_gt_2048_s": float(np.percentile(big_lat, 50)) if big_lat else None,
               "routing": {"big_n": big_n if big_n is not None else 2048,
                           "big_lanes": big_lanes if big_lanes is not None else 3,
                           "lane_ctas": lane_ctas or "29 % of the SMs"},
               "ok": status_ok, "statuses": statuses, "evals_total": int(evals), "seconds": span}
    return summary, costs


def serving_oracle_costs():
    """Stored FP64 oracle costs of a sample of the serving trace's requests (tests/golden/
    serve_oracle.json, written by tests/golden/make_golden.py --serve): {trace index: cost}."""
    path = os.path.join(ROOT, "tests", "golden", "serve_oracle.json")
    if not os.path.exists(path):
        return {}
    with open(path) as fh:
        return {c["index"]: c["oracle_cost"] for c in json.load(fh)["cases"] if c["seed"] == SERVE_SEED}


def measure_serving_loads(dev, h, count_sat=200, count_sub=100):
    """Serving at three offered loads on the same trace: the configured Poisson rate (200/s, above
    capacity: the throughput, and queueing latency) and 0.5x / 0.9x of the capacity that run
    measured (latency below saturation); then the first count_sub requests solved one problem per
    launch (mdot_solve_points, in arrival order, default parameters) as the comparison, and the
    served costs against the stored FP64 oracle costs of a sample of the requests."""
    import torch
    import paper_2307_08507_gb300 as M
    trace = serving_requests(dev, count_sat)
    sat, costs = measure_serving(dev, trace)
    cap = sat["problems_per_s"]
    loads = {"configured_200_per_s": sat}
    reqs = trace[:count_sub]                     # the same requests, offered below capacity
    for f in (0.5, 0.9):
        loads[f"{f}x_capacity"], _ = measure_serving(dev, reqs, rate=f * cap)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    t_single, dcost = 0.0, []
    for q, (ta, nq, eps, prob, (r, c, xy, scale)) in enumerate(reqs):
        ev0.record(stream)
        _, _, rs = h.solve_points(r, c, xy, xy, M.COST_SQEUCLID, scale, eps, check=False)
        ev1.record(stream)
        torch.cuda.synchronize()
        t_single += ev0.elapsed_time(ev1) / 1e3
        if costs[q] is not None:
            dcost.append(abs(rs.cost - costs[q]))
    orc = serving_oracle_costs()
    d_or = [abs(costs[i] - v) for i, v in orc.items() if i < len(costs) and costs[i] is not None]
    single_rate = count_sub / t_single
    return {"loads": loads, "capacity_problems_per_s": cap,
            "one_per_launch": {"requests": count_sub, "seconds": t_single, "problems_per_s": single_rate,
                               "served_vs_one_per_launch_max_abs_cost_diff": max(dcost) if dcost else None},
            "served_speedup_vs_one_per_launch": cap / single_rate,
            "vs_oracle": {"sampled_requests": len(d_or), "max_abs_cost_diff": max(d_or) if d_or else None}}


# ---------------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------------
def run_ours(args, rank, world):
    import numpy as np
    import torch
    import paper_2307_08507_gb300 as M
    from paper_2307_08507_gb300 import inputs as I

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    p = I.grid_problem(N_GRID, SEED + rank)
    n = p.n
    stream = torch.cuda.current_stream()
    h = M.Handle(16384, stream)
    r = torch.from_numpy(p.r).to(dev)
    c = torch.from_numpy(p.c).to(dev)
    C = torch.from_numpy(p.C).to(dev)
    u = torch.empty(n, dtype=torch.float64, device=dev)
    v = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    prm = M.default_params()
    prm_prof = M.default_params(profile=1)

    def step(params):
        return h.solve(r, c, C, EPS, params, u_out=u, v_out=v)[2]

    for _ in range(args.warmup):
        res = step(prm)
    torch.cuda.synchronize()

    times = []
    results = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.fill_(1.0)                      # evict C from L2 between steps
            ev0.record(stream)
            res = step(prm)
            ev1.record(stream)
            torch.cuda.synchronize()
            times.append(ev0.elapsed_time(ev1) / 1e3)
            results.append(res)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
    t_step = max_over_ranks(sum(times) / len(times), dist, dev)
    res = results[-1]
    info = res.info

    # dominant kernel (fp32-entry stage launches): per-launch device time from CUDA events
    # recorded by the library on its stream, and algorithmic bytes = 4 n^2 per evaluation
    flush.fill_(1.0)
    res_p = step(prm_prof)
    ip = res_p.info
    evals32 = ip.evals - ip.evals_fp64
    launches32 = max(1, ip.stage_launches_fp32)
    bytes_per_launch = 4.0 * n * n * evals32 / launches32
    t_launch = ip.t_stage_fp32_ms / 1e3 / launches32
    hbm, peak_kind = peaks()
    achieved = bytes_per_launch / t_launch / 1e9 if t_launch > 0 else None
    trace = h.solve_trace()
    # per-evaluation device time of the stage launches (the accurate-tier launches dominate), to set
    # beside a profiler's per-launch durations
    acc_rows = [t for t in trace if t["kind"] == 0 and t["evals"] >= 100]
    us_per_eval_long = (1e3 * sum(t["ms"] for t in acc_rows) / max(1, sum(t["evals"] for t in acc_rows))
                        if acc_rows else None)

    # read rates of this GPU measured by the library's own streaming-read kernel: a 64 MiB buffer
    # (the size of C at n = 4096, held in L2 after the first pass) and a 4 GiB buffer (HBM)
    rates = {}
    for mib, reps in ((64, 50), (4096, 3)):
        buf = torch.ones(mib * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        M.read_probe(buf, 1)
        best = 1e30
        for _ in range(5):
            ev0.record(stream)
            M.read_probe(buf, reps)
            ev1.record(stream)
            torch.cuda.synchronize()
            best = min(best, ev0.elapsed_time(ev1) / 1e3)
        rates[f"read_{mib}MiB_GBps"] = buf.numel() * 4.0 * reps / best / 1e9
        del buf
    l2_gbs = rates["read_64MiB_GBps"]

    # single dual evaluation (K1 + K2, one pass, fp32 entries), n = 4096 and n = 16384
    dual = {}
    for kk in (64, 128):
        q = I.grid_problem(kk, SEED)
        Cq = torch.from_numpy(q.C).to(dev)
        uq = torch.from_numpy(np.log(q.r)).to(dev)
        vq = torch.from_numpy(np.log(q.c)).to(dev)
        gam = 2.0 ** 12
        lr, _ = h.dual_eval(uq, vq, gam, Cq)
        for _ in range(3):
            h.dual_eval(uq, vq, gam, Cq, ref_log_rP=lr)
        ts, tk = [], []
        for _ in range(10):
            flush.fill_(1.0)                      # C (64 MiB / 1 GiB) starts outside L2
            ev0.record(stream)
            h.dual_eval(uq, vq, gam, Cq, ref_log_rP=lr)
            ev1.record(stream)
            torch.cuda.synchronize()
            ts.append(ev0.elapsed_time(ev1) / 1e3)
            tk.append(h.dual_eval_time() / 1e3)   # the kernel alone: events around its launch
        tmed = sorted(ts)[len(ts) // 2]
        kmed = sorted(tk)[len(tk) // 2]
        gbs = 4.0 * q.n * q.n / kmed / 1e9
        dual[f"n{q.n}"] = {"us": kmed * 1e6, "GBps": gbs, "frac_hbm": gbs / hbm,
                           "us_call": tmed * 1e6, "bytes": 4 * q.n * q.n}
        del Cq
    # the same evaluation with C regenerated from the 2-D grid coordinates (n = 16384): no n^2
    # bytes, bound by the fp32 pipe (ALU_OPS_PER_ENTRY fp32 operations and one ex2 per entry)
    q = I.grid_problem(128, SEED, dense=False)
    xy = torch.from_numpy(I.coords3(q.x)).to(dev)
    uq = torch.from_numpy(np.log(q.r)).to(dev)
    vq = torch.from_numpy(np.log(q.c)).to(dev)
    alu_peak = alu_peak_ops()
    for name, prec, ops in (("n16384_regen", M.PREC_FP32, ALU_OPS_PER_ENTRY),
                            ("n16384_regen_tensor_cores", M.PREC_FP32 | M.PREC_TENSOR_CORES, ALU_OPS_PER_ENTRY_TC)):
        lr, _ = h.dual_eval_points(uq, vq, 2.0 ** 12, xy, xy, M.COST_SQEUCLID, q.scale, precision=prec)
        tk = []
        for _ in range(10):
            h.dual_eval_points(uq, vq, 2.0 ** 12, xy, xy, M.COST_SQEUCLID, q.scale, ref_log_rP=lr, precision=prec)
            tk.append(h.dual_eval_time() / 1e3)
        kmed = sorted(tk)[len(tk) // 2]
        ents = float(q.n) * q.n / kmed
        dual[name] = {"us": kmed * 1e6, "entries_per_s": ents, "bound": "alu",
                      "achieved_ops": ents * ops, "peak_ops": alu_peak, "frac_alu": ents * ops / alu_peak,
                      "ops_per_entry": ops}

    # the single-GPU studies (gap sweep, batched and served forms) run once, at N = 1: with N > 1
    # ranks the other replicas would wait minutes for rank 0 at the next collective
    solo = rank == 0 and world == 1
    sweep = gap_sweep(h, dev, stream) if (solo and not args.no_sweep) else None
    batch = measure_batch(h, dev, stream) if (solo and not args.no_batch) else None
    serving = (measure_serving_loads(dev, h, args.serve_count, max(1, args.serve_count // 2))
               if (solo and args.serve_count > 0) else None)

    # end to end through the public C ABI with host buffers (copies inside the timed region)
    Ch = torch.from_numpy(p.C).pin_memory().numpy()
    rh = torch.from_numpy(p.r).pin_memory().numpy()
    ch = torch.from_numpy(p.c).pin_memory().numpy()
    uh = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    vh = torch.empty(n, dtype=torch.float64).pin_memory().numpy()
    h.solve_host(rh, ch, Ch, EPS, prm, u_out=uh, v_out=vh)
    e2e = []
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, _, rr = h.solve_host(rh, ch, Ch, EPS, prm, u_out=uh, v_out=vh)
        e2e.append(time.perf_counter() - t0)
    e2e_t = sum(e2e) / len(e2e)

    g = golden_case()
    exact = exact_value()
    true_gap = (res.cost - exact) if exact is not None else None
    # a certificate of the target without the exact LP: the c-transform bound of a solve at
    # gamma_f = 2^21 is a feasible OT dual (weak duality), so OT >= lb_hi and the benchmark solve's
    # true gap is at most cost - lb_hi
    _, _, res_hi = h.solve(r, c, C, EPS, M.default_params(gamma_f=2.0 ** 21), check=False)
    lb_hi = res_hi.cost - res_hi.gap_cert
    cpu = None
    if rank == 0 and world == 1:
        n_evals = args.cpu_sample_evals or 40
        est1, per1, evals = cpu_solve_estimate(max(4, n_evals // 4))
        per_all, threads = oracle_sample_all_cores(n_evals)
        cpu = {"value": per_all * evals, "unit": "s", "cores": threads, "kind": "oracle",
               "sample": f"per-evaluation x evaluations extrapolation: {n_evals} FP64 dual evaluations "
                         f"of the same n=4096 problem on {threads} threads ({per_all:.4f} s each), x "
                         f"the {evals} evaluations of the full oracle solve",
               "single_core": {"value": est1, "unit": "s", "cores": 1,
                               "sample": f"{max(4, n_evals // 4)} evaluations on one core "
                                         f"({per1:.3f} s each) x {evals}"}}
    if rank == 0:
        line = {
            "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded grid histograms, Sec. 5.1 shapes)",
            "config": {"workload": "grid64x64_l2sq_n4096_eps1e-6", "n": n, "seed": SEED,
                       "eps_target": EPS, "gamma_f": info.gamma_f, "cost": "C fp32 dense, 64 MiB",
                       "l2": "flushed (256 MiB write) between timed steps", "replicas": world},
            "result": {"status": M.status_string(res.status), "cost": res.cost,
                       "true_gap": true_gap, "gap_cert": res.gap_cert,
                       "true_gap_bound": res.cost - lb_hi,
                       "true_gap_bound_how": "cost - c-transform lower bound of a gamma_f = 2^21 solve (weak duality)",
                       "oracle_cost": g["oracle_cost"] if g else None,
                       "cost_minus_oracle": (res.cost - g["oracle_cost"]) if g else None,
                       "evals": info.evals, "evals_fp64": info.evals_fp64, "iters": info.iters,
                       "stages": info.stages, "grad_l1": info.grad_l1},
            "roofline": {"kernel": "stage_kernel<fp32 entries> (one MDOT stage: PNCG + line search)",
                         "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": (achieved / hbm) if achieved else None,
                         "traffic": ncu_traffic("stage_kernel_flag<2, 0>"),
                         "peak_kind": peak_kind,
                         "bytes_per_launch": bytes_per_launch, "us_per_launch": t_launch * 1e6,
                         "us_per_eval": 1e6 * t_launch * launches32 / max(1, evals32),
                         "us_per_eval_launches_ge_100_evals": us_per_eval_long,
                         "l2_read_GBps": l2_gbs, "frac_l2": (achieved / l2_gbs) if achieved else None,
                         "read_rates": rates,
                         "launch_times_ms": {"stage_fp32": ip.t_stage_fp32_ms, "stage_fp64": ip.t_stage_fp64_ms,
                                             "round": ip.t_round_ms, "bound": ip.t_bound_ms},
                         "launches": [(t["kind"], round(t["ms"], 4), t["evals"]) for t in trace]},
            "gap_sweep": sweep,
            "dual_eval": dual,
            "batched": batch,
            "serving": serving,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_t, "unit": "s", "h2d_bytes_per_step": 4 * n * n + 16 * n,
                    "d2h_bytes_per_step": 16 * n},
            "gpu_launches": info.launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()


def _study_line(M, case, res, seconds, **extra):
    i = res.info
    d = {"study": case, **extra, "status": M.status_string(res.status), "seconds": seconds, "cost": res.cost,
         "gap_cert": res.gap_cert, "evals": i.evals, "evals_fp64": i.evals_fp64, "iters": i.iters,
         "ls_trials": i.ls_trials, "stages": i.stages, "gamma_f": i.gamma_f, "H_min": i.H_min,
         "grad_l1": i.grad_l1}
    print(json.dumps(d), flush=True)


def run_study(args):
    """Comparison studies, one timed solve per configuration (after one untimed solve of the same
    problem), wall time on the host around the synchronous call:
      sinkhorn: MDOT-PNCG against MDOT-Sinkhorn (Alg. 4 as the projector) on 32x32 and 64x64 grids
                at target gaps 1e-4, 1e-5, 1e-6;
      large_n:  points on a line (squared distance, regenerated cost, no n x n matrix) at
                n = 16384 ... 131072, against the exact cost of the monotone coupling;
      nscale:   time and evaluations against n = 36 ... 16384 (k x k grids), gap 1e-6 (Fig. 6 shape);
      hmin:     App. C: r drawn with H(r) / log n in {0.03, 0.1, 0.3, 0.9}, c uniform, 3-D normal
                points with L1 or squared-L2 cost; H_min against log n in the stage tolerance."""
    import numpy as np
    import torch
    import paper_2307_08507_gb300 as M
    from paper_2307_08507_gb300 import inputs as I
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)

    def to(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = fn()
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    if args.case == "sinkhorn":
        h = M.Handle(4096)
        for k in (32, 64):
            p = I.grid_problem(k, 7)
            r, c, C = to(p.r), to(p.c), to(p.C)
            for eps in (1e-4, 1e-5, 1e-6):
                for proj in (0, 1):
                    prm = M.default_params(projector=proj)
                    (_, _, res), dt = timed(lambda: h.solve(r, c, C, eps, prm))
                    _study_line(M, "sinkhorn", res, dt, n=p.n, eps_target=eps,
                                projector="sinkhorn" if proj else "pncg")
    elif args.case == "large_n":
        # exact costs (monotone coupling on the line) stored by tests/golden/make_golden.py --line
        with open(os.path.join(ROOT, "tests", "golden", "line_exact.json")) as fh:
            exact_of = {(c["n"], c["seed"]): c["exact_ot"] for c in json.load(fh)["cases"]}
        h = M.Handle(131072)
        for n, eps in ((16384, 1e-5), (16384, 1e-6), (65536, 1e-5), (65536, 1e-6), (131072, 1e-5)):
            p = I.line_problem(n, 11)
            exact = exact_of[(n, 11)]
            r, c, x, y = to(p.r), to(p.c), to(p.x), to(p.y)
            (_, _, res), dt = timed(lambda: h.solve_points(r, c, x, y, M.COST_SQEUCLID, p.scale, eps,
                                                           M.default_params(), check=False))
            _study_line(M, "large_n", res, dt, n=n, eps_target=eps, exact=exact, true_gap=res.cost - exact)
    elif args.case == "nscale":
        h = M.Handle(16384)
        for k in (6, 8, 12, 16, 24, 32, 48, 64, 96, 128):
            p = I.grid_problem(k, 7)
            r, c, C = to(p.r), to(p.c), to(p.C)
            (_, _, res), dt = timed(lambda: h.solve(r, c, C, 1e-6))
            _study_line(M, "nscale", res, dt, n=p.n, eps_target=1e-6)
    elif args.case == "hmin":
        n = 4096
        h = M.Handle(n)
        for kind, ck in (("l2sq", M.COST_SQEUCLID), ("l1", M.COST_L1)):
            for frac in (0.03, 0.1, 0.3, 0.9):
                p = I.entropy_problem(n, frac, 17, kind)
                r, c, x = to(p.r), to(p.c), to(p.x)
                for gf in (2.0 ** 10, 2.0 ** 13, 2.0 ** 16):
                    for se in (0, 1):
                        prm = M.default_params(gamma_f=gf, stop_entropy=se)
                        (_, _, res), dt = timed(lambda: h.solve_points(r, c, x, x, ck, p.scale, 1e-6, prm,
                                                                       check=False))
                        _study_line(M, "hmin", res, dt, n=n, cost_kind=kind, H_frac=frac,
                                    stop_entropy="log n" if se else "H_min")
    h.close()


def run_case(args):
    """Small fixed workloads for profiler captures: the one-pass dual evaluation (fp32 entries,
    row scales given) or one full solve of a k x k grid problem."""
    import numpy as np
    import torch
    import paper_2307_08507_gb300 as M
    from paper_2307_08507_gb300 import inputs as I
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    p = I.grid_problem(args.grid, SEED)
    h = M.Handle(p.n)
    C = torch.from_numpy(p.C).to(dev)
    if args.case == "batch":
        stream = torch.cuda.current_stream()
        print(json.dumps(measure_batch(h, dev, stream)))
        h.close()
        return
    if args.case == "tune_serve":
        # the served form's routing picked by measurement (M.tune_server) on the serving trace
        reqs = [(ta, prob, keep) for (ta, _, _, prob, keep) in serving_requests(dev, args.serve_count)]
        best, table = M.tune_server(SERVE_WORKSPACE, reqs)
        print(json.dumps({"best": best, "candidates": [{k: v for k, v in row.items() if k not in ("statuses", "costs")}
                                                      for row in table]}))
        h.close()
        return
    if args.case == "serve":
        print(json.dumps(measure_serving(dev, serving_requests(dev, args.serve_count), args.serve_big_n,
                                         args.serve_lanes, args.serve_lane_ctas)[0]))
        h.close()
        return
    if args.case == "dual_eval":
        u = torch.from_numpy(np.log(p.r)).to(dev)
        v = torch.from_numpy(np.log(p.c)).to(dev)
        lr, _ = h.dual_eval(u, v, 2.0 ** 12, C)
        for _ in range(args.reps):
            h.dual_eval(u, v, 2.0 ** 12, C, ref_log_rP=lr)
    elif args.case in ("dual_eval_regen", "dual_eval_regen_tc"):
        # the regenerated squared-Euclidean cost of the grid points: fp32 operations, or (_tc) the
        # contraction on the tensor cores
        prec = M.PREC_FP32 | (M.PREC_TENSOR_CORES if args.case == "dual_eval_regen_tc" else 0)
        u = torch.from_numpy(np.log(p.r)).to(dev)
        v = torch.from_numpy(np.log(p.c)).to(dev)
        xy = torch.from_numpy(I.coords3(p.x)).to(dev)
        lr, _ = h.dual_eval_points(u, v, 2.0 ** 12, xy, xy, M.COST_SQEUCLID, p.scale, precision=prec)
        for _ in range(args.reps):
            h.dual_eval_points(u, v, 2.0 ** 12, xy, xy, M.COST_SQEUCLID, p.scale, ref_log_rP=lr, precision=prec)
    else:
        r = torch.from_numpy(p.r).to(dev)
        c = torch.from_numpy(p.c).to(dev)
        for _ in range(args.reps):
            h.solve(r, c, C, EPS, M.default_params(profile=1))
        # the evaluations of every stage launch, counted by the kernel itself (State.evals): a
        # profiler's per-launch time divided by these gives its time per evaluation
        torch.cuda.synchronize()
        print(json.dumps({"stage_launches": [{"launch": q, "kind": t["kind"], "evals": t["evals"]}
                                             for q, t in enumerate(h.solve_trace())]}))
    torch.cuda.synchronize()
    h.close()
    print(f"case {args.case} n={p.n} reps={args.reps} done")


def run_phases(args):
    """Per-phase device time of an evaluation of the fp32-entry stage kernel on the benchmark solve
    (n = 4096 grid, target gap 1e-6), from the diagnostic build with phase timers
    (build.py --phases): per CTA, SM cycles per phase summed over the solve's launches, divided by
    its evaluations and by the median SM clock sampled during the solve."""
    import numpy as np
    import torch
    import paper_2307_08507_gb300 as M
    from paper_2307_08507_gb300 import inputs as I
    M.use_phase_timer_build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    names = ["loop_top", "pass", "row_epilogue", "wait_column_partials", "merge_column_epilogue",
             "cta_reduce_publish", "wait_scalar_partials", "decision", "commit_next_rows"]
    for kind in ("l2sq", "l1"):
        p = I.grid_problem(N_GRID, SEED, kind=kind)
        r, c, C = (torch.from_numpy(a).to(dev) for a in (p.r, p.c, p.C))
        with M.Handle(p.n) as h:
            h.solve(r, c, C, EPS)
            torch.cuda.synchronize()
            M.phase_timers(clear=True)
            with Clocks() as clk:
                _, _, res = h.solve(r, c, C, EPS, M.default_params(profile=1))
                torch.cuda.synchronize()
            ph = M.phase_timers(clear=True)
            trace = h.solve_trace()
        mhz = clk.summary()["sm_mhz"] or 2070.0
        G = int(np.count_nonzero(ph[:, 9]))
        cyc = ph[:G, :9].astype(np.float64) / ph[:G, 9:10].astype(np.float64)
        us = cyc / mhz
        st32 = [t for t in trace if t["kind"] == 0]
        print(json.dumps({
            "cost_kind": kind, "status": M.status_string(res.status), "evals": res.info.evals,
            "evals_per_cta": [int(ph[:G, 9].min()), int(ph[:G, 9].max())], "sm_mhz": mhz,
            "us_per_eval_fp32_launches": 1e3 * sum(t["ms"] for t in st32) / max(1, sum(t["evals"] for t in st32)),
            "phases_us_mean": dict(zip(names, us.mean(0).round(3).tolist())),
            "phases_us_min": dict(zip(names, us.min(0).round(3).tolist())),
            "phases_us_max": dict(zip(names, us.max(0).round(3).tolist())),
            "sum_us_mean": float(us.mean(0).sum())}), flush=True)


def main():
    args = parse()
    if args.case == "phases":
        run_phases(args)
        return
    if args.case in ("sinkhorn", "large_n", "nscale", "hmin"):
        run_study(args)
        return
    if args.case != "solve":
        run_case(args)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world)


if __name__ == "__main__":
    main()
