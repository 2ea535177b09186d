"""Host-side pieces of bench.py (no GPU): the workloads have the shapes and
sizes their names state, the algorithmic bytes per launch follow from them,
and the oracle baseline runs on a bounded prefix of the workload."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_headline_workload_and_bytes(bench):
    w = bench.workload(2, 0)
    assert w["kind"] == "indexed" and w["n"] == 128 ** 3 and w["n_nodes"] == 129 ** 3
    assert w["conn"].shape == (128 ** 3, 8) and w["nodes"].shape == (129 ** 3, 3)
    assert bench.algorithmic_bytes(w, "bulk32") == 49 * 128 ** 3 + 16 * 129 ** 3 == 137107472
    assert bench.algorithmic_bytes(w, "nodes32") == 40 * 129 ** 3


def test_small_workload(bench):
    w = bench.workload(1, 0)
    assert w["kind"] == "soa" and w["X"].shape == (8, 3, 10_000) and w["depth"] == 8
    assert bench.algorithmic_bytes(w, "bulk32") == 209 * 10_000
    # replicas draw their own inputs
    assert not (bench.workload(1, 1)["X"] == w["X"]).all()


def test_oracle_baseline_is_a_bounded_prefix(bench):
    w = bench.workload(1, 0)
    rate, sample = bench.oracle_rate(w, 0.01, 1)
    k = int(sample.split()[2])
    assert rate > 0 and sample.startswith("the first ") and k in (4096, 8192, 10_000)
