"""Serving: each request's solution is the same when it is solved alone and
when it is solved while other requests run beside it on other streams (the
kernels reduce in a fixed order and every request has its own context), and
every request reaches the 1e-8 FP64 residual."""
import numpy as np
import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_results_same_alone_and_in_the_mix():
    from paper_1805_11930_gb300 import serve
    kw = dict(n_range=(4, 9), p_range=(2, 5), seed=77)
    runner = serve.DeviceRunner(keep_solutions=True)
    mix = serve.make_trace(8, None, **kw)
    srv = serve.SolveServer(runner, slots=4)
    srv.run(mix)
    srv.close()
    assert srv.max_concurrent == 4
    alone = serve.make_trace(8, None, **kw)
    one = serve.SolveServer(runner, slots=1)
    for r in alone:
        one.run([r])
    one.close()
    for a, b in zip(mix, alone):
        assert a.error is None and b.error is None, (a.error, b.error)
        assert a.stats["converged"] == 1 and a.stats["rel_residual"] <= 1e-8
        assert (a.n, a.p) == (b.n, b.p)
        assert np.array_equal(a.solution, b.solution), f"request {a.rid} differs"


def test_evicted_request_resumes_on_the_gpu():
    """A request solved in chunks of 3 outer iterations, evicted after its
    first chunk, re-queued and resumed from its iterate, reaches the same
    1e-8 residual (relative to ||f||) as the uninterrupted solve, and its
    solution agrees with that one to the accuracy the residual allows."""
    from paper_1805_11930_gb300 import serve

    class EvictOnce(serve.DeviceRunner):
        def on_chunk(self, req, iterations, rel_residual):
            if req.evictions == 0:
                req.evict_requested = True

    kw = dict(n_range=(6, 8), p_range=(3, 4), seed=91)
    a = serve.make_trace(3, None, **kw)
    srv = serve.SolveServer(EvictOnce(keep_solutions=True, chunk=3), slots=2)
    srv.run(a)
    srv.close()
    b = serve.make_trace(3, None, **kw)
    one = serve.SolveServer(serve.DeviceRunner(keep_solutions=True), slots=1)
    one.run(b)
    one.close()
    for x, y in zip(a, b):
        assert x.error is None and x.evictions == 1 and 0 < x.checkpoint.iterations
        assert x.stats["converged"] == 1 and x.stats["rel_residual"] <= 1e-8 * (1 + 1e-9)
        assert x.stats["iterations"] >= y.stats["iterations"]
        d = np.linalg.norm(x.solution - y.solution) / np.linalg.norm(y.solution)
        assert d < 1e-5, (x.rid, d)
    assert serve.summarize(a)["evictions"] == 3


def test_batched_server_same_alone_and_in_the_mix():
    """The batched server (one batch per order, several requests per launch):
    each request's solution is bit for bit the one it gets alone in its batch,
    and every request reaches the 1e-8 FP64 residual."""
    from paper_1805_11930_gb300 import serve
    kw = dict(n_range=(4, 9), p_range=(2, 4), seed=78)
    mix = serve.make_trace(12, None, **kw)
    srv = serve.BatchedServer(serve.BatchBackend(keep_solutions=True), setup_workers=3, step=3)
    srv.run(mix)
    srv.close()
    assert srv.max_members_seen >= 2
    alone = serve.make_trace(12, None, **kw)
    one = serve.BatchedServer(serve.BatchBackend(keep_solutions=True), setup_workers=1, step=3, max_members=1)
    for r in alone:
        one.run([r])
    one.close()
    for a, b in zip(mix, alone):
        assert a.error is None and b.error is None, (a.error, b.error)
        assert a.stats["converged"] == 1 and a.stats["rel_residual"] <= 1e-8
        assert a.stats["iterations"] == b.stats["iterations"]
        assert np.array_equal(a.solution, b.solution), f"request {a.rid} differs"
