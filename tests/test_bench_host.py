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
