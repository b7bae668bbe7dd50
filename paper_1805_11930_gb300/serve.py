"""Continuous-batching solve server for a stream of DG diffusion problems.

Requests (mesh N^3, order p, log-normal K with its own sigma and seed,
Gaussian source, homogeneous Dirichlet) arrive over time.  The server keeps
`slots` workers; each worker is a host thread with its own CUDA stream and its
own library context (re-used across requests).  A request is admitted, in
arrival order, as soon as a worker is idle and its HBM footprint
(footprint.library_bytes) fits into what the running requests leave of the
budget; its set-up and solve then run on that worker's stream, overlapping on
the device with the other workers' solves.  Each worker's V-cycle is
captured into a CUDA graph on its second use and replayed (opts.graph), which
removes most of the per-kernel launch cost of small requests.  The library's
kernels reduce in a fixed order, so a request's result does not depend on
what runs beside it.

    python -m paper_1805_11930_gb300.serve [--requests 512] [--slots 4] [--rates 0.5,0.8,1.0,1.2]

measures the single-stream capacity (requests served back to back on one
worker, mixed precision) and, on the same requests, the plain FP64 solve
(FP64 smoother and CG) as the reference point, then for each rate
multiplier replays a seeded Poisson arrival trace at that multiple of the
capacity and prints solves/s and p50 / p99 latency (arrival to completion) as
one JSON line per rate.

A request can be cancelled (`SolveServer.cancel`): if it has not been
admitted it never runs; if it runs, the runner stops at its next checkpoint.
A running request can be evicted (`SolveServer.evict`): the runner stops at
its next checkpoint, hands back its iterate u and residual norm, and the
request goes back to the head of the queue; when it is admitted again the
solve restarts from that u (the outer Krylov space is rebuilt, the stopping
test stays relative to the first residual).  A request whose runner fails
with DGMG_ERR_OOM while others ran beside it is re-queued once and then
runs alone.
"""
import argparse
import collections
import json
import queue
import statistics
import threading
import time

import numpy as np

from . import footprint

SEED = 1805


class Checkpoint:
    """What a stopped solve hands back: its iterate u (host FP64), the FP64
    residual norm ||f - A u||_2 and the outer iterations done so far."""

    def __init__(self, u, res_abs, iterations):
        self.u, self.res_abs, self.iterations = u, res_abs, iterations


class Evicted(Exception):
    """Raised by a runner that stopped a request on request of the server."""

    def __init__(self, checkpoint):
        super().__init__("evicted")
        self.checkpoint = checkpoint


class Cancelled(Exception):
    """Raised by a runner that stopped a cancelled request."""


class Request:
    def __init__(self, rid, arrival, n, p, sigma, seed):
        self.rid, self.arrival, self.n, self.p, self.sigma, self.seed = rid, arrival, n, p, sigma, seed
        self.ndof = n ** 3 * (p + 1) ** 3
        self.t_admit = self.t_start = self.t_done = None
        self.stats = None
        self.solution = None
        self.error = None
        self.footprint = footprint.library_bytes((n, n, n), p, krylov="fcg")
        self.checkpoint = None          # set when the request was evicted
        self.evictions = 0
        self.retries = 0                # re-admissions after a failed allocation
        self.alone = False              # admit only when nothing else runs
        self.cancel_requested = False
        self.evict_requested = False
        self.cancelled = False

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.arrival


def make_trace(n_requests, rate, seed=SEED, n_range=(8, 48), p_range=(2, 6), sigma_range=(0.0, 2.0)):
    """Seeded Poisson arrivals (rate requests/s; rate None = all at t = 0)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, n_requests) if rate else np.zeros(n_requests)
    arrivals = np.cumsum(gaps) - (gaps[0] if rate else 0.0)
    ns = rng.integers(n_range[0], n_range[1] + 1, n_requests)
    ps = rng.integers(p_range[0], p_range[1] + 1, n_requests)
    sig = rng.uniform(*sigma_range, n_requests)
    seeds = rng.integers(0, 2 ** 31, n_requests)
    return [Request(i, float(arrivals[i]), int(ns[i]), int(ps[i]), float(sig[i]), int(seeds[i]))
            for i in range(n_requests)]


def request_inputs(req):
    """Coefficients and source of a request: K_T = exp(sigma N(0,1)) per cell;
    f the Gaussian of the diffusion experiments (centre (0.75, 0.5, 0.3),
    width 0.1) taken at each cell centre for all of the cell's quadrature
    points."""
    n, p = req.n, req.p
    rng = np.random.default_rng(req.seed)
    K = np.exp(req.sigma * rng.normal(size=n ** 3))
    c = (np.arange(n) + 0.5) / n
    cz, cy, cx = np.meshgrid(c, c, c, indexing="ij")
    fc = np.exp(-((cx - 0.75) ** 2 + (cy - 0.5) ** 2 + (cz - 0.3) ** 2) / (2 * 0.1 ** 2)).reshape(-1)
    return K, np.repeat(fc, (p + 1) ** 3)


class DeviceRunner:
    """Runs one request on one worker: its own stream and context.

    chunk: outer iterations per library call; between calls the runner
    checks the request's cancel and evict flags (None: one call, no
    checkpoints).  Each call restarts the Krylov method from the current u
    with its tolerance rescaled so that the stop stays ||r||_2 <= rtol ||f||_2
    (u = 0 at the start)."""

    def __init__(self, device=0, keep_solutions=False, chunk=None, rtol=1e-8, maxit=500, **opts):
        self.device = device
        self.keep = keep_solutions
        self.chunk = chunk
        self.rtol = rtol
        self.maxit = maxit
        self.opts = dict(opts)
        self._local = threading.local()

    def _worker_state(self):
        st = getattr(self._local, "state", None)
        if st is None:
            import torch
            from . import dgmg
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(self.device)
            ctx = dgmg.Context(self.device, stream=stream)
            st = self._local.state = (stream, ctx)
        return st

    def __call__(self, req):
        import torch
        from . import dgmg
        stream, ctx = self._worker_state()
        K, f_qp = request_inputs(req)
        with torch.cuda.stream(stream):
            ctx.set_mesh(req.n, req.n, req.n, 1.0, 1.0, 1.0, req.p, [0] * 6)
            ctx.set_coefficients(K)
            nd = ctx.sizes()["ndof"]
            f = torch.empty(nd, dtype=torch.float64, device=f"cuda:{self.device}")
            ctx.assemble_rhs(f_qp, f)
            kw = dict(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG, graph=1)
            kw.update(self.opts)
            if self.chunk is None and req.checkpoint is None:
                u = torch.zeros_like(f)
                stats = ctx.solve(f, u, dgmg.default_opts(rtol=self.rtol, maxit=self.maxit, **kw), check=False)
            else:
                u, stats = self._chunked(ctx, f, req, kw)
            sol = u.cpu().numpy() if self.keep else None
        stream.synchronize()
        return stats, sol

    def on_chunk(self, req, iterations, rel_residual):
        """Called on the worker's thread after each library call of a chunked
        solve (progress reporting; a subclass may set the request's flags)."""

    def _chunked(self, ctx, f, req, kw):
        import torch
        from . import dgmg
        fnorm = float(torch.linalg.vector_norm(f))
        target = self.rtol * fnorm
        cp = req.checkpoint
        if cp is None:
            u, res, its = torch.zeros_like(f), fnorm, 0
        else:
            u, res, its = torch.as_tensor(cp.u, device=f.device).clone(), cp.res_abs, cp.iterations
        stats = None
        while True:
            if res <= target or fnorm == 0.0:
                break
            if req.cancel_requested:
                raise Cancelled()
            if req.evict_requested:
                raise Evicted(Checkpoint(u.cpu().numpy(), res, its))
            step = min(self.chunk or self.maxit, self.maxit - its)
            if step <= 0:
                break
            stats = ctx.solve(f, u, dgmg.default_opts(rtol=target / res, maxit=step, **kw), check=False)
            its += stats["iterations"]
            res *= stats["rel_residual"]
            if stats["status"] not in ("DGMG_OK", "DGMG_ERR_NOT_CONVERGED"):
                raise RuntimeError(f"request {req.rid}: {stats['status']}")
            self.on_chunk(req, its, res / fnorm)
        out = dict(stats or {"status": "DGMG_OK", "inner_mean": 0.0, "inner_max": 0})
        out.update(iterations=its, rel_residual=res / fnorm if fnorm > 0 else 0.0,
                   converged=int(res <= target * (1 + 1e-12)))
        return u, out


class SolveServer:
    """Continuous batching over `slots` persistent workers with an HBM budget
    (bytes).  The runner is called on the worker's own thread, so per-worker
    state (stream, context) lives as long as the server.

    exclusive_dofs: requests with at least this many dofs run alone (they are
    admitted once nothing else runs, and nothing is admitted beside them): a
    solve that large fills the GPU by itself, and sharing the SMs and L2 with
    others only slows everyone down; smaller requests share the slots."""

    def __init__(self, runner, slots=4, hbm_budget=None, exclusive_dofs=None):
        self.runner = runner
        self.slots = slots
        self.budget = hbm_budget
        self.exclusive_dofs = exclusive_dofs
        self._exclusive_running = False
        self._lock = threading.Condition()
        self._jobs = queue.Queue()
        self._pending = collections.deque()
        self._requests = {}
        self._used = 0
        self._idle = slots
        self.max_concurrent = 0
        self.max_used = 0
        self._clock0 = None
        self._workers = [threading.Thread(target=self._loop, daemon=True) for _ in range(slots)]
        for t in self._workers:
            t.start()

    def _loop(self):
        while True:
            req = self._jobs.get()
            if req is None:
                return
            if req.t_start is None:
                req.t_start = time.perf_counter() - self._clock0
            requeue = False
            try:
                req.stats, req.solution = self.runner(req)
            except Evicted as e:     # back to the head of the queue with its iterate
                req.checkpoint = e.checkpoint
                req.evictions += 1
                requeue = True
            except Cancelled:
                req.cancelled = True
            except Exception as e:   # reported per request, the server keeps going
                if "DGMG_ERR_OOM" in str(e) and not req.alone and req.retries == 0:
                    req.retries += 1  # others held memory: try once more, alone
                    req.alone = True
                    requeue = True
                else:
                    req.error = repr(e)
            with self._lock:
                req.evict_requested = False
                if not requeue:
                    req.t_done = time.perf_counter() - self._clock0
                self._used -= req.footprint
                self._idle += 1
                if self._is_exclusive(req):
                    self._exclusive_running = False
                if requeue:
                    self._pending.appendleft(req)
                self._lock.notify_all()

    def _is_exclusive(self, req):
        return req.alone or (self.exclusive_dofs is not None and req.ndof >= self.exclusive_dofs)

    def cancel(self, rid):
        """Cancel request rid: dropped if it waits, stopped at its runner's
        next checkpoint if it runs.  Returns False for an unknown or finished
        request."""
        with self._lock:
            req = self._requests.get(rid)
            if req is None or req.t_done is not None:
                return False
            req.cancel_requested = True
            self._lock.notify_all()
            return True

    def evict(self, rid):
        """Ask the runner of request rid to stop at its next checkpoint and
        re-queue it at the head of the queue with its iterate.  Returns False
        unless the request is running."""
        with self._lock:
            req = self._requests.get(rid)
            if req is None or req.t_done is not None or req.t_admit is None or req in self._pending:
                return False
            req.evict_requested = True
            return True

    def run(self, trace):
        """Serve the trace; returns when every request has completed, failed
        or been cancelled."""
        self._clock0 = time.perf_counter()
        with self._lock:
            self._pending = pending = collections.deque(sorted(trace, key=lambda r: r.arrival))
            self._requests = {r.rid: r for r in trace}
            while pending or self._idle < self.slots:
                if not pending:
                    self._lock.wait(timeout=0.05)
                    continue
                head = pending[0]
                now = time.perf_counter() - self._clock0
                if head.cancel_requested:        # never admitted (again)
                    pending.popleft()
                    head.cancelled = True
                    head.t_done = now
                    continue
                if head.arrival > now:
                    self._lock.wait(timeout=head.arrival - now)
                    continue
                fits = self.budget is None or self._used + head.footprint <= self.budget or self._used == 0
                alone_ok = not self._is_exclusive(head) or self._idle == self.slots
                if self._idle == 0 or not fits or self._exclusive_running or not alone_ok:
                    self._lock.wait(timeout=0.05)
                    continue
                pending.popleft()
                if head.t_admit is None:
                    head.t_admit = now
                self._idle -= 1
                self._used += head.footprint
                if self._is_exclusive(head):
                    self._exclusive_running = True
                self.max_concurrent = max(self.max_concurrent, self.slots - self._idle)
                self.max_used = max(self.max_used, self._used)
                self._jobs.put(head)
        return trace

    def close(self):
        for _ in self._workers:
            self._jobs.put(None)
        for t in self._workers:
            t.join()


class BatchBackend:
    """Device side of the batched server.

    prepare(req) runs on a set-up worker thread: it takes a library context
    from that worker's pool (or creates one on the worker's stream), sets the
    request's mesh and coefficients, assembles its right-hand side, computes
    the initial Krylov state (dgmg_batch_prime: residual, first V-cycle) and
    returns the prepared item (context, f, u = 0).  new_batch(p) runs on the lane
    thread of order p and returns a dgmg.Batch on a stream of its own.
    finish(item, stats) copies the solution back if asked to, returns the
    context to its pool and drops the request's vectors."""

    def __init__(self, device=0, keep_solutions=False, rtol=1e-8, maxit=500, **opts):
        self.device = device
        self.keep = keep_solutions
        self.rtol = rtol
        self.maxit = maxit
        self.opts = dict(opts)
        self._local = threading.local()

    def solve_opts(self):
        from . import dgmg
        kw = dict(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG)
        kw.update(self.opts)
        return dgmg.default_opts(rtol=self.rtol, maxit=self.maxit, **kw)

    def _worker(self):
        st = getattr(self._local, "state", None)
        if st is None:
            import torch
            torch.cuda.set_device(self.device)
            st = self._local.state = (torch.cuda.Stream(self.device), [])
        return st

    def prepare(self, req):
        import torch
        from . import dgmg
        stream, pool = self._worker()
        ctx = pool.pop() if pool else dgmg.Context(self.device, stream=stream)
        K, f_qp = request_inputs(req)
        with torch.cuda.stream(stream):
            ctx.set_mesh(req.n, req.n, req.n, 1.0, 1.0, 1.0, req.p, [0] * 6)
            ctx.set_coefficients(K)
            f = torch.empty(ctx.sizes()["ndof"], dtype=torch.float64, device=f"cuda:{self.device}")
            ctx.assemble_rhs(f_qp, f)
            u = torch.zeros_like(f)
            ctx.batch_prime(f, u, self.solve_opts())   # the initial V-cycle on this worker's stream
        stream.synchronize()
        return {"ctx": ctx, "f": f, "u": u, "pool": pool}

    def new_batch(self, p):
        import torch
        from . import dgmg
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream(self.device)
        return _DeviceBatch(dgmg.Batch(self.device, stream=stream, opts=self.solve_opts()), self)

    def finish(self, item, stats):
        sol = item["u"].cpu().numpy() if self.keep else None
        item["pool"].append(item["ctx"])
        item["f"] = item["u"] = None
        return stats, sol


class _DeviceBatch:
    def __init__(self, batch, backend):
        self.b, self.backend = batch, backend

    def add(self, item):
        return self.b.add(item["ctx"], item["f"], item["u"], rtol=self.backend.rtol, maxit=self.backend.maxit)

    def step(self, k):
        return self.b.step(k)

    def poll(self, slot):
        return self.b.poll(slot)

    def remove(self, slot):
        self.b.remove(slot)

    def close(self):
        self.b.close()


class BatchedServer:
    """Continuous batching with one batch per polynomial order.

    Requests are admitted in arrival order while their HBM footprint fits the
    budget; `setup_workers` host threads prepare admitted requests (mesh,
    coefficients, right-hand side: host work that overlaps with the device);
    a prepared request joins the batch of its order at the next step
    boundary.  One lane thread per order drives its batch: `step` outer
    iterations of all its members per call (one kernel launch per step of the
    iteration for all of them, replayed from a CUDA graph), then retires the
    members that stopped (statistics, solution, latency) and frees their
    memory, which lets waiting requests in.  Lanes of different orders run on
    their own streams, so their work overlaps on the device.  A request's
    arithmetic is its own (see dgmg_batch_add): its result does not depend on
    what runs beside it.

    backend: an object with prepare(req), new_batch(p) and finish(item,
    stats) (BatchBackend, or a fake for host tests)."""

    def __init__(self, backend, setup_workers=4, hbm_budget=None, step=4, max_members=16):
        self.backend = backend
        self.budget = hbm_budget
        self.step = step
        self.max_members = max_members
        self._lock = threading.Condition()
        self._setup = queue.Queue()
        self._ready = {}
        self._lanes = {}
        self._used = 0
        self._open = 0            # admitted, not finished
        self.max_used = 0
        self.max_members_seen = 0
        self._clock0 = None
        self._stop = False
        self._workers = [threading.Thread(target=self._setup_loop, daemon=True) for _ in range(setup_workers)]
        for t in self._workers:
            t.start()

    def _now(self):
        return time.perf_counter() - self._clock0

    def _release(self, req):
        with self._lock:
            req.t_done = self._now()
            self._used -= req.footprint
            self._open -= 1
            self._lock.notify_all()

    def _setup_loop(self):
        while True:
            req = self._setup.get()
            if req is None:
                return
            try:
                item = self.backend.prepare(req)
            except Exception as e:       # reported per request, the server keeps going
                req.error = repr(e)
                self._release(req)
                continue
            self._lane_queue(req.p).put((req, item))

    def _lane_queue(self, p):
        with self._lock:
            if p not in self._ready:
                self._ready[p] = queue.Queue()
                t = threading.Thread(target=self._lane_loop, args=(p, self._ready[p]), daemon=True)
                self._lanes[p] = t
                t.start()
            return self._ready[p]

    def _lane_loop(self, p, q):
        batch = self.backend.new_batch(p)
        members = {}
        closing = False
        while True:
            while len(members) < self.max_members and not closing:
                try:
                    got = q.get(timeout=0.02) if not members else q.get_nowait()
                except queue.Empty:
                    break
                if got is None:
                    closing = True
                    break
                req, item = got
                try:
                    slot = batch.add(item)
                except Exception as e:
                    req.error = repr(e)
                    self._release(req)
                    continue
                req.t_start = self._now()
                members[slot] = (req, item)
            self.max_members_seen = max(self.max_members_seen, len(members))
            if not members:
                if closing:
                    batch.close()
                    return
                continue
            batch.step(self.step)
            for slot, (req, item) in list(members.items()):
                st = batch.poll(slot)
                if st is None:
                    continue
                batch.remove(slot)
                del members[slot]
                req.stats, req.solution = self.backend.finish(item, st)
                if st.get("status") not in ("DGMG_OK", None):
                    req.error = st["status"]
                self._release(req)

    def run(self, trace):
        """Serve the trace; returns when every request has completed or failed."""
        self._clock0 = time.perf_counter()
        pending = collections.deque(sorted(trace, key=lambda r: r.arrival))
        with self._lock:
            while pending or self._open > 0:
                if not pending:
                    self._lock.wait(timeout=0.05)
                    continue
                head = pending[0]
                now = self._now()
                if head.arrival > now:
                    self._lock.wait(timeout=head.arrival - now)
                    continue
                fits = self.budget is None or self._used + head.footprint <= self.budget or self._used == 0
                if not fits:
                    self._lock.wait(timeout=0.05)
                    continue
                pending.popleft()
                head.t_admit = now
                self._used += head.footprint
                self._open += 1
                self.max_used = max(self.max_used, self._used)
                self._setup.put(head)
        return trace

    def close(self):
        for _ in self._workers:
            self._setup.put(None)
        for t in self._workers:
            t.join()
        for p, q in list(self._ready.items()):
            q.put(None)
        for t in self._lanes.values():
            t.join()


def summarize(reqs):
    done = [r for r in reqs if r.t_done is not None and r.error is None and not r.cancelled]
    lat = sorted(r.latency for r in done)
    span = max(r.t_done for r in done) - min(r.arrival for r in reqs)
    conv = sum(1 for r in done if r.stats and r.stats["converged"])

    def pct(q):
        return lat[min(len(lat) - 1, int(np.ceil(q * len(lat))) - 1)]

    return {"requests": len(reqs), "completed": len(done), "converged": conv,
            "errors": sum(1 for r in reqs if r.error), "cancelled": sum(1 for r in reqs if r.cancelled),
            "evictions": sum(r.evictions for r in reqs), "retries": sum(r.retries for r in reqs),
            "solves_per_s": round(len(done) / span, 4),
            "p50_latency_s": round(pct(0.50), 4), "p99_latency_s": round(pct(0.99), 4),
            "mean_service_s": round(statistics.mean(r.t_done - r.t_start for r in done), 4),
            "makespan_s": round(span, 3)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--rates", default="0.5,0.8,1.0,1.2")
    ap.add_argument("--capacity-requests", type=int, default=16)
    ap.add_argument("--nmax", type=int, default=48)
    ap.add_argument("--budget-gb", type=float, default=200.0)
    ap.add_argument("--exclusive-mdofs", type=float, default=0.0,
                    help="requests with at least this many million dofs run alone (0: off)")
    ap.add_argument("--mode", default="batched", choices=["batched", "slots"],
                    help="batched: per-order batches (BatchedServer); slots: one context and stream per slot")
    ap.add_argument("--setup-workers", type=int, default=4)
    ap.add_argument("--step", type=int, default=4, help="outer iterations per batch step")
    args = ap.parse_args()
    runner = DeviceRunner()
    budget = args.budget_gb * 1e9
    rng_kw = dict(n_range=(8, args.nmax))
    # single-stream capacity: one worker, requests back to back (after warm-up)
    one = SolveServer(runner, slots=1, hbm_budget=budget)
    one.run(make_trace(2, None, seed=SEED + 7, **rng_kw))
    cap_trace = make_trace(args.capacity_requests, None, seed=SEED + 1, **rng_kw)
    one.run(cap_trace)
    one.close()
    cap = summarize(cap_trace)
    capacity = 1.0 / cap["mean_service_s"]
    # the plain FP64 solve of the same requests, back to back
    fp64 = SolveServer(DeviceRunner(smoother_prec=0, krylov=0, graph=0), slots=1, hbm_budget=budget)
    fp64_trace = make_trace(args.capacity_requests, None, seed=SEED + 1, **rng_kw)
    fp64.run(fp64_trace)
    fp64.close()
    print(json.dumps({"single_stream": cap, "capacity_req_per_s": round(capacity, 4),
                      "fp64_single_stream": summarize(fp64_trace)}), flush=True)
    for mult in [float(x) for x in args.rates.split(",")]:
        trace = make_trace(args.requests, mult * capacity, seed=SEED, **rng_kw)
        if args.mode == "batched":
            srv = BatchedServer(BatchBackend(), setup_workers=args.setup_workers, hbm_budget=budget, step=args.step)
            srv.run(make_trace(10, None, seed=SEED + 9, n_range=(8, 12)))    # warm the workers and lanes
            srv.max_used = srv.max_members_seen = 0
            srv.run(trace)
            srv.close()
            out = summarize(trace)
            out.update({"mode": "batched", "rate_multiplier": mult, "rate_req_per_s": round(mult * capacity, 4),
                        "setup_workers": args.setup_workers, "step": args.step,
                        "max_batch_members": srv.max_members_seen, "max_hbm_gb": round(srv.max_used / 1e9, 3)})
        else:
            excl = args.exclusive_mdofs * 1e6 if args.exclusive_mdofs > 0 else None
            srv = SolveServer(runner, slots=args.slots, hbm_budget=budget, exclusive_dofs=excl)
            srv.run(make_trace(args.slots, None, seed=SEED + 9, n_range=(8, 12)))    # warm the workers
            srv.max_concurrent = srv.max_used = 0
            srv.run(trace)
            srv.close()
            out = summarize(trace)
            out.update({"mode": "slots", "rate_multiplier": mult, "rate_req_per_s": round(mult * capacity, 4),
                        "slots": args.slots, "exclusive_mdofs": args.exclusive_mdofs,
                        "max_concurrent": srv.max_concurrent, "max_hbm_gb": round(srv.max_used / 1e9, 3)})
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
