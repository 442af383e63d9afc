"""CPU checks of the benchmark's host logic: the ncu traffic record is reported only for the CUDA
sources it was captured from, and the max-over-ranks reduction of the replica timing."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_record_follows_the_source_hash(monkeypatch):
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    with open(path) as fh:
        rec = json.load(fh)
    name, entry = next(iter(rec["kernels"].items()))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: rec["source_sha256"])
    assert bench.ncu_traffic(name) == float(entry["dram_bytes_per_launch"])
    assert bench.ncu_traffic("no_such_kernel") is None
    # any change to the CUDA sources voids the record
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench.ncu_traffic(name) is None


def test_source_hash_covers_the_cuda_sources():
    h1 = bench.kernel_source_hash()
    assert len(h1) == 64 and h1 == bench.kernel_source_hash()


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks(1.25, None, None) == 1.25


def test_not_converged_summary_counts_and_quartiles():
    """The batched measurement's summary of the problems whose last stage ended above its
    tolerance: count, sizes, gradient-norm quartiles (no GPU: fake results)."""
    class R:
        def __init__(self, status, g):
            self.status, self.grad_l1 = status, g

    class FakeM:
        MDOT_ERR_NOT_CONVERGED = 2

        @staticmethod
        def default_params():
            class P:
                fp32_floor = 2e-7
            return P()

    probs = [{"n": n} for n in (300, 500, 700, 900)]
    res = [R(0, 1e-7), R(2, 4e-7), R(2, 1e-6), R(0, 5e-8)]
    s = bench._not_converged_summary(probs, res, FakeM)
    assert s["count"] == 2 and s["n_min"] == 500 and s["n_max"] == 700
    assert s["grad_l1_quartiles"][0] == 4e-7 and s["grad_l1_quartiles"][-1] == 1e-6
    assert bench._not_converged_summary(probs, [R(0, 1e-7)] * 4, FakeM) == {"count": 0}


def test_benchmark_instance_has_a_stored_exact_optimum():
    """The headline line reports the true gap of the n = 4096 solve (not only a bound): the exact
    optimum of the benchmark instance is stored for both costs of the gap sweep."""
    l2, l1 = bench.exact_value("l2sq"), bench.exact_value("l1")
    assert l2 is not None and l1 is not None
    assert 0.0 < l2 < 1.0 and 0.0 < l1 < 1.0          # costs normalised to max C = 1
