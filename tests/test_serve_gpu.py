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
