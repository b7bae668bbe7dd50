"""Host logic of the serving loop on CPU, with a fake runner: arrival order,
slot limit, HBM budget (a request waits until enough running ones finish),
per-request latency accounting."""
import threading
import time

from paper_1805_11930_gb300 import serve


class FakeRunner:
    def __init__(self, service=0.05):
        self.service = service
        self.lock = threading.Lock()
        self.running = 0
        self.peak = 0
        self.order = []

    def __call__(self, req):
        with self.lock:
            self.running += 1
            self.peak = max(self.peak, self.running)
            self.order.append(req.rid)
        time.sleep(self.service)
        with self.lock:
            self.running -= 1
        return {"converged": 1, "rel_residual": 1e-9}, None


def test_slots_fifo_and_latency():
    trace = serve.make_trace(12, None, n_range=(8, 10), p_range=(2, 2))
    r = FakeRunner()
    srv = serve.SolveServer(r, slots=3)
    srv.run(trace)
    srv.close()
    assert r.peak == 3 and srv.max_concurrent == 3
    assert r.order[:3] == sorted(r.order[:3]) and set(r.order) == set(range(12))
    s = serve.summarize(trace)
    assert s["completed"] == 12 and s["converged"] == 12
    assert s["p50_latency_s"] >= 0.05 and s["p99_latency_s"] >= s["p50_latency_s"]


def test_budget_limits_concurrency():
    trace = serve.make_trace(6, None, n_range=(8, 8), p_range=(3, 3))
    fp = trace[0].footprint
    r = FakeRunner()
    srv = serve.SolveServer(r, slots=6, hbm_budget=2 * fp)      # room for two at a time
    srv.run(trace)
    srv.close()
    assert r.peak == 2 and srv.max_used <= 2 * fp


def test_poisson_arrivals_are_seeded():
    a = [x.arrival for x in serve.make_trace(50, 10.0)]
    b = [x.arrival for x in serve.make_trace(50, 10.0)]
    assert a == b and a[0] == 0.0 and all(y >= x for x, y in zip(a, a[1:]))
    assert 2.5 < a[-1] < 8.0      # 49 gaps of mean 0.1 s


class FailingRunner(FakeRunner):
    """Raises for some requests, as a runner does when the library returns an
    error status (a failed allocation, a rejected argument)."""

    def __init__(self, bad, **kw):
        super().__init__(**kw)
        self.bad = set(bad)

    def __call__(self, req):
        if req.rid in self.bad:
            raise RuntimeError(f"request {req.rid}: DGMG_ERR_OOM")
        return super().__call__(req)


def test_failed_requests_are_reported_and_release_their_slot():
    trace = serve.make_trace(10, None, n_range=(8, 9), p_range=(2, 3))
    srv = serve.SolveServer(FailingRunner({2, 7}, service=0.01), slots=2, hbm_budget=2 * trace[0].footprint)
    srv.run(trace)
    srv.close()
    s = serve.summarize(trace)
    assert s["errors"] == 2 and s["completed"] == 8
    assert [r.rid for r in trace if r.error] == [2, 7] and all("DGMG_ERR_OOM" in trace[i].error for i in (2, 7))
    assert srv._used == 0 and srv._idle == 2      # the failed requests gave back slot and memory


class TrackingRunner(FakeRunner):
    """Records, for every request, how many requests were running with it."""

    def __init__(self, **kw):
        super().__init__(**kw)
        self.seen = {}

    def __call__(self, req):
        with self.lock:
            self.running += 1
            self.peak = max(self.peak, self.running)
            self.order.append(req.rid)
            self.seen[req.rid] = max(self.seen.get(req.rid, 0), self.running)
        time.sleep(self.service)
        with self.lock:
            self.seen[req.rid] = max(self.seen[req.rid], self.running)
            self.running -= 1
        return {"converged": 1, "rel_residual": 1e-9}, None


def test_exclusive_requests_run_alone_in_fifo_order():
    """exclusive_dofs: a request that large runs with nothing beside it, the
    smaller ones share the slots, and the arrival order is kept."""
    trace = serve.make_trace(24, None, n_range=(8, 40), p_range=(2, 6), seed=5)
    limit = sorted(r.ndof for r in trace)[16]          # about a third of the requests are large
    r = TrackingRunner(service=0.01)
    srv = serve.SolveServer(r, slots=4, exclusive_dofs=limit)
    srv.run(trace)
    srv.close()
    large = [q for q in trace if q.ndof >= limit]
    assert large and all(r.seen[q.rid] == 1 for q in large)
    assert r.peak > 1                                   # the small ones did share
    adm = [q.t_admit for q in sorted(trace, key=lambda q: q.rid)]
    assert adm == sorted(adm)                           # FIFO admission
    assert serve.summarize(trace)["completed"] == 24


class ChunkRunner:
    """A solve of `work` chunks that checks the request's flags between
    chunks, as DeviceRunner does between library calls; the checkpoint holds
    the chunks done."""

    def __init__(self, work=20, chunk_s=0.01):
        self.work, self.chunk_s = work, chunk_s
        self.lock = threading.Lock()
        self.calls = []          # rid per call, in call order
        self.chunks = {}         # rid -> chunks executed in total

    def __call__(self, req):
        with self.lock:
            self.calls.append(req.rid)
        done = 0 if req.checkpoint is None else req.checkpoint.iterations
        while done < self.work:
            if req.cancel_requested:
                raise serve.Cancelled()
            if req.evict_requested:
                raise serve.Evicted(serve.Checkpoint(None, float(self.work - done), done))
            time.sleep(self.chunk_s)
            done += 1
            with self.lock:
                self.chunks[req.rid] = self.chunks.get(req.rid, 0) + 1
        return {"converged": 1, "rel_residual": 1e-9, "iterations": done}, None


def _serve_in_thread(srv, trace):
    t = threading.Thread(target=srv.run, args=(trace,))
    t.start()
    return t


def test_cancel_waiting_request_never_runs():
    trace = serve.make_trace(4, None, n_range=(8, 8), p_range=(2, 2))
    r = FakeRunner(service=0.05)
    srv = serve.SolveServer(r, slots=1)
    t = _serve_in_thread(srv, trace)
    time.sleep(0.02)
    assert srv.cancel(3)
    t.join()
    srv.close()
    assert trace[3].cancelled and 3 not in r.order and r.order == [0, 1, 2]
    s = serve.summarize(trace)
    assert s["cancelled"] == 1 and s["completed"] == 3
    assert not srv.cancel(0)                       # finished requests cannot be cancelled


def test_cancel_running_request_stops_at_a_checkpoint():
    trace = serve.make_trace(2, None, n_range=(8, 8), p_range=(2, 2))
    r = ChunkRunner(work=30)
    srv = serve.SolveServer(r, slots=1)
    t = _serve_in_thread(srv, trace)
    time.sleep(0.08)
    assert srv.cancel(0)
    t.join()
    srv.close()
    assert trace[0].cancelled and trace[0].stats is None and r.chunks[0] < 30
    assert not trace[1].cancelled and r.chunks[1] == 30
    assert srv._used == 0 and srv._idle == 1


def test_evicted_request_resumes_from_its_checkpoint_at_the_head():
    """An evicted request loses no work (the resumed run starts from the
    checkpoint) and is re-admitted before the requests queued behind it."""
    trace = serve.make_trace(3, None, n_range=(8, 8), p_range=(2, 2))
    r = ChunkRunner(work=40)
    srv = serve.SolveServer(r, slots=1)
    t = _serve_in_thread(srv, trace)
    time.sleep(0.06)
    assert srv.evict(0)
    assert not srv.evict(2)                        # waiting, not running
    t.join()
    srv.close()
    assert r.calls == [0, 0, 1, 2]
    assert trace[0].evictions == 1 and trace[0].stats["iterations"] == 40 and r.chunks[0] == 40
    assert 0 < trace[0].checkpoint.iterations < 40
    s = serve.summarize(trace)
    assert s["completed"] == 3 and s["evictions"] == 1 and s["cancelled"] == 0


class OomOnceRunner(TrackingRunner):
    """Fails request `rid` with DGMG_ERR_OOM when it shares the GPU."""

    def __init__(self, rid, **kw):
        super().__init__(**kw)
        self.rid = rid
        self.failed = 0

    def __call__(self, req):
        if req.rid == self.rid and not req.alone:
            self.failed += 1
            time.sleep(self.service)
            raise RuntimeError(f"request {req.rid}: DGMG_ERR_OOM")
        return super().__call__(req)


def test_failed_allocation_is_retried_alone():
    trace = serve.make_trace(8, None, n_range=(8, 9), p_range=(2, 3))
    r = OomOnceRunner(3, service=0.03)
    srv = serve.SolveServer(r, slots=3)
    srv.run(trace)
    srv.close()
    assert r.failed == 1 and trace[3].retries == 1 and trace[3].error is None
    assert r.seen[3] == 1                          # the retry ran with nothing beside it
    s = serve.summarize(trace)
    assert s["completed"] == 8 and s["errors"] == 0 and s["retries"] == 1


class FakeCtx:
    """Stands in for a library context: a stationary iteration that reduces
    the residual by `rate` per outer iteration, reported the way dgmg_solve
    reports it (rel_residual relative to the call's own initial residual,
    status NOT_CONVERGED at maxit)."""

    def __init__(self, rate=0.5):
        self.rate = rate
        self.calls = []

    def solve(self, f, u, opts, check=False):
        import math
        import torch
        r0 = float(torch.linalg.vector_norm(f - u))
        need = math.ceil(math.log(opts.rtol) / math.log(self.rate))
        its = min(need, opts.maxit)
        u.add_((f - u) * (1 - self.rate ** its))      # residual f - u shrinks by rate^its
        self.calls.append((opts.rtol, opts.maxit, its))
        rel = float(torch.linalg.vector_norm(f - u)) / r0
        return {"status": "DGMG_OK" if its == need else "DGMG_ERR_NOT_CONVERGED", "iterations": its,
                "rel_residual": rel, "converged": int(its == need), "inner_mean": 0.0, "inner_max": 0}


def test_chunked_solve_keeps_the_stopping_test_relative_to_f():
    """DeviceRunner's chunked form: each call's tolerance is rescaled so that
    the overall stop is ||r|| <= rtol ||f||, iterations add up, and a resumed
    request continues from its checkpoint with the same total work as an
    uninterrupted one."""
    pytest = __import__("pytest")
    torch = pytest.importorskip("torch")
    from paper_1805_11930_gb300 import build, dgmg
    if not build.up_to_date():
        try:
            build.build()
        except RuntimeError as e:       # no nvcc: the options struct comes from the library
            pytest.skip(str(e))
    dgmg.load()
    f = torch.linspace(1.0, 2.0, 50, dtype=torch.float64)
    req = serve.make_trace(1, None)[0]
    runner = serve.DeviceRunner(chunk=4, rtol=1e-8)
    ctx = FakeCtx(0.5)
    u, st = runner._chunked(ctx, f, req, {})
    assert st["iterations"] == 27 and st["converged"] == 1      # 0.5^27 < 1e-8 < 0.5^26
    assert st["rel_residual"] <= 1e-8 and len(ctx.calls) == 7   # 6 chunks of 4, then 3
    assert all(m == 4 for _, m, _ in ctx.calls)
    # stopped after the second chunk, then resumed from the checkpoint
    hits = []

    class Stop(serve.DeviceRunner):
        def on_chunk(self, req, iterations, rel_residual):
            hits.append((iterations, rel_residual))
            if iterations == 8:
                req.evict_requested = True

    req2 = serve.make_trace(1, None)[0]
    with pytest.raises(serve.Evicted) as ev:
        Stop(chunk=4, rtol=1e-8)._chunked(FakeCtx(0.5), f, req2, {})
    cp = ev.value.checkpoint
    assert cp.iterations == 8 and abs(cp.res_abs / float(torch.linalg.vector_norm(f)) - 0.5 ** 8) < 1e-12
    req2.checkpoint, req2.evict_requested = cp, False
    u2, st2 = serve.DeviceRunner(chunk=4, rtol=1e-8)._chunked(FakeCtx(0.5), f, req2, {})
    assert st2["iterations"] == 27 and st2["converged"] == 1
    assert float(torch.linalg.vector_norm(u2 - u)) < 1e-12 * float(torch.linalg.vector_norm(u))


# ------------------------------------------------------------- batched server
class FakeBatch:
    """A batch whose members stop after as many steps as their order; records
    the largest membership and the orders it saw."""

    def __init__(self, p, log):
        self.p, self.log = p, log
        self.members = {}
        self.next = 0

    def add(self, item):
        if item.get("fail_add"):
            raise RuntimeError("DGMG_ERR_OOM")
        slot = self.next
        self.next += 1
        self.members[slot] = [item, 0]
        self.log["orders"].add(self.p)
        self.log["peak"] = max(self.log["peak"], len(self.members))
        return slot

    def step(self, k):
        time.sleep(0.002)
        for m in self.members.values():
            m[1] += k
        return sum(1 for m in self.members.values() if m[1] < m[0]["steps"])

    def poll(self, slot):
        item, done = self.members[slot]
        if done < item["steps"]:
            return None
        return {"converged": 1, "rel_residual": 1e-9, "iterations": done, "status": "DGMG_OK"}

    def remove(self, slot):
        del self.members[slot]

    def close(self):
        self.log["closed"] += 1


class FakeBackend:
    def __init__(self, fail=()):
        self.fail = set(fail)
        self.log = {"orders": set(), "peak": 0, "closed": 0, "prepared": []}
        self.lock = threading.Lock()

    def prepare(self, req):
        if req.rid in self.fail:
            raise RuntimeError("set-up failed")
        with self.lock:
            self.log["prepared"].append(req.rid)
        time.sleep(0.001)
        return {"steps": 4 * req.p}

    def new_batch(self, p):
        return FakeBatch(p, self.log)

    def finish(self, item, stats):
        return stats, None


def test_batched_server_completes_every_request_per_order():
    trace = serve.make_trace(40, None, n_range=(8, 10), p_range=(2, 6), seed=3)
    be = FakeBackend()
    srv = serve.BatchedServer(be, setup_workers=3, step=4, max_members=5)
    srv.run(trace)
    srv.close()
    s = serve.summarize(trace)
    assert s["completed"] == 40 and s["converged"] == 40 and s["errors"] == 0
    assert be.log["orders"] == {r.p for r in trace}
    assert be.log["peak"] <= 5 and srv.max_members_seen <= 5
    assert be.log["closed"] == len(be.log["orders"])
    for r in trace:
        assert r.stats["iterations"] >= 4 * r.p and r.t_done >= r.t_start >= r.t_admit >= r.arrival


def test_batched_server_budget_and_failures():
    trace = serve.make_trace(10, None, n_range=(8, 8), p_range=(3, 3), seed=4)
    fp = trace[0].footprint
    be = FakeBackend(fail={2, 5})
    srv = serve.BatchedServer(be, setup_workers=2, hbm_budget=2 * fp, step=2)
    srv.run(trace)
    srv.close()
    assert srv.max_used <= 2 * fp and be.log["peak"] <= 2
    s = serve.summarize(trace)
    assert s["errors"] == 2 and s["completed"] == 8
    assert all(trace[i].error for i in (2, 5))
