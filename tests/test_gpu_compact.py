"""Compaction by verdict and candidate filtering on the GPU (through the C
ABI): the ids must equal numpy's nonzero of the same selection exactly (in
order), and the filtered candidate set must equal the oracle's valid set."""
import numpy as np
import pytest

import oracle
from paper_1706_01613_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU hosts, skipped there
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1706_01613_gb300 import hexval as hv  # noqa: E402


@pytest.fixture(scope="module")
def v():
    h = hv.Validator(precision="fp32", max_depth=8, queue_capacity=1 << 20, max_batch=1 << 24,
                     max_nodes=1 << 22, exact_capacity=1 << 12)
    yield h
    h.close()


@pytest.mark.parametrize("n", [0, 1, 31, 8191, 8192, 8193, 100_003, 3_000_007])
@pytest.mark.parametrize("verdicts", [(1,), (2,), (1, 2), (), (0, 1, 2, 3, 4, 5, 6, 7)])
def test_compaction_equals_nonzero(v, n, verdicts):
    rng = np.random.default_rng(n + 7 * len(verdicts))
    flags = rng.integers(0, 256, size=n).astype(np.uint8)
    ids, count = v.compact(torch.from_numpy(flags).cuda(), verdicts)
    c = int(count.item())
    want = np.nonzero(np.isin(flags & 7, verdicts))[0]
    assert c == len(want)
    assert np.array_equal(ids[:c].cpu().numpy(), want.astype(np.int32))


def test_unaligned_flags(v):
    flags = np.random.default_rng(3).integers(0, 5, size=50_001).astype(np.uint8)
    buf = torch.from_numpy(np.concatenate([[0], flags]).astype(np.uint8)).cuda()
    ids, count = v.compact(buf[1:], (1,))
    want = np.nonzero((flags & 7) == 1)[0]
    c = int(count.item())
    assert c == len(want) and np.array_equal(ids[:c].cpu().numpy(), want)


def test_candidate_filtering_matches_the_oracle(v):
    nodes, conn, _, _ = synth.hex_candidates(24, 10, sigma=0.25, seed=31)
    got = v.filter_valid(torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda())
    assert v.status() == 0
    f, _, _ = oracle.check_indexed(nodes, conn, max_depth=8, threads=oracle.max_threads())
    want = np.nonzero((f & 7) == oracle.VALID)[0]
    assert np.array_equal(got.cpu().numpy(), want)
    assert 0.3 < len(want) / len(conn) < 0.6  # about half are reflections


def test_full_candidate_set_sampled(v):
    """The benchmark's candidate set (65^3 nodes, 40 candidates per node):
    the compaction is consistent with the flags, and a sample of the flags
    matches the oracle."""
    nodes, conn, _, _ = synth.hex_candidates()
    N, C = torch.from_numpy(nodes).cuda(), torch.from_numpy(conn).cuda()
    flags, _, _ = v.check_indexed(N, C)
    ids, count = v.compact(flags, (1,))
    f = flags.cpu().numpy()
    c = int(count.item())
    assert np.array_equal(ids[:c].cpu().numpy(), np.nonzero((f & 7) == 1)[0])
    sample = np.random.default_rng(5).choice(len(conn), 20_000, replace=False)
    wf, _, _ = oracle.check_indexed(nodes, conn[sample], max_depth=8, threads=oracle.max_threads())
    assert np.array_equal(f[sample] & 0x7F, wf & 0x7F)
