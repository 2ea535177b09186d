"""Serving on the GPU: continuous batching of requests of very different
sizes; every request's result in the concurrent mix is identical to the same
request run alone, and matches the oracle on sampled elements."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1706_01613_gb300 import hexval as hv  # noqa: E402
from paper_1706_01613_gb300 import serve  # noqa: E402


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_mix_equals_alone(precision):
    pool = serve.Pool(200_000, seed=321)
    reqs = serve.poisson_stream(pool, 40, rate=3000.0, seed=654, size_max=200_000)
    caps = dict(queue_capacity=1 << 20, max_batch=1 << 20, max_nodes=1 << 22,
                exact_capacity=1 << 12)
    ex = serve.GpuExecutor(4, precision=precision, **caps)
    sched = serve.run_stream(reqs, ex, slots=4, budget_bytes=40 << 30)
    assert not sched.rejected
    assert all(s == 0 for s in ex.status())
    overlap = sum(1 for a in reqs for b in reqs
                  if a.id < b.id and b.admitted is not None and a.admitted <= b.admitted < a.done)
    assert overlap > 0  # requests really ran concurrently
    alone = hv.Validator(precision=precision, max_depth=8, **caps)
    rng = np.random.default_rng(5)
    for r in reqs:
        host = r.host_arrays()
        dev = [a.cuda() for a in host]
        got = (alone.check_soa(dev[0]) if r.kind == "soa" else alone.check_indexed(*dev))
        got = [t.cpu().numpy() for t in got]
        for x, y in zip(r.result, got):
            assert np.array_equal(x, y, equal_nan=True), r.id
        k = min(r.n, 200)
        idx = np.sort(rng.choice(r.n, size=k, replace=False))
        if r.kind == "soa":
            X = host[0].numpy()
            want = oracle.check_soa(np.ascontiguousarray(X[:, :, idx]), max_depth=8)
        else:
            want = oracle.check_indexed(host[0].numpy(), host[1].numpy()[idx], max_depth=8)
        assert np.array_equal(r.result[0][idx] & 0x7F, want[0] & 0x7F)
    s = serve.latency_summary(reqs)
    print(precision, s)
    assert s["p99_ms"] >= s["p50_ms"] > 0
    alone.close()
    ex.close()
