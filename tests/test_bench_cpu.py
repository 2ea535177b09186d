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
    # the scope table's 73.6 B per hexahedron: connectivity, outputs and one
    # FP64 node (24 B) per node of the mesh
    assert bench.algorithmic_bytes(w, "bulk32") == 49 * 128 ** 3 + 24 * 129 ** 3 == 154280984
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


def test_roofline_of_each_dominant_kernel(bench):
    """The dominant phase decides the roofline: bytes over HBM for the FP32
    pass, FP64 instructions for the FP64 pass, box expansions for the tail
    (the pipe with the larger fraction)."""
    w = bench.workload(1, 0)
    roof, share = bench.roofline_of(w, {"bulk32": (2.0, 10), "tail": (0.5, 10)}, {}, 10)
    assert roof["bound"] == "hbm" and roof["kernel"] == "bulk32"
    assert abs(roof["achieved"] - 209 * 10_000 / 0.2e-3 / 1e9) < 1e-9
    assert abs(sum(share.values()) - 1) < 1e-3
    roof, _ = bench.roofline_of(w, {"bulk64": (3.0, 3)}, {}, 3)
    assert roof["pipe"] == "fp64" and abs(roof["frac"] - 366 * 10_000 / 1e-3 / 1e12 / 0.625) < 1e-9
    stats = {"boxes": 3_000_000, "boxes_fp32": 1_000_000}
    roof, _ = bench.roofline_of(w, {"bulk32": (0.1, 1), "tail": (20.0, 10)}, stats, 10)
    assert roof["kernel"] == "tail" and roof["pipe"] == "fp64"
    assert roof["box_expansions_per_call"] == {"fp64": 200_000.0, "fp32": 100_000.0}
    assert abs(roof["fp64_frac"] - 147 * 200_000 / 2e-3 / 1e12 / 0.625) < 1e-9
    roof, _ = bench.roofline_of(w, {"bulk32": (0.1, 1), "tail": (2.0, 10)}, {}, 10)
    assert roof["bound"] == "latency"
    roof, _ = bench.roofline_of(w, {"bulk32": (0.1, 1), "tail": (2.0, 10)},
                                {"redone_tail": 1_000_000}, 10)
    assert roof["pipe"] == "fp64" and abs(roof["frac"] - 366 * 100_000 / 0.2e-3 / 1e12 / 0.625) < 1e-9
