"""Batched solves (dgmg_batch_*) against single solves and the oracle.

A batch runs the outer flexible CG (or CG) of several requests of one order
in lockstep, one launch per step over all members, with the Krylov scalars
on the device.  Per member the arithmetic is that of dgmg_solve with the same
options, so the checks are bitwise: a request's solution and iteration count
from a batch equal those of its single solve, alone in a batch and beside
other requests; the solution also solves the oracle's assembled system."""
import numpy as np
import pytest

from oracle import dg
from paper_1805_11930_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _request(nc, p, sigma, seed):
    """A log-normal diffusion request: K_T = exp(sigma N(0, 1)), Gaussian source."""
    rng = np.random.default_rng(seed)
    ncell = int(np.prod(nc))
    K = np.exp(sigma * rng.normal(size=ncell))
    return dict(nc=nc, p=p, K=K, L=(1.0, 1.0, 1.0))


def _prepare(req):
    from paper_1805_11930_gb300 import dgmg
    ctx = dgmg.Context(0)
    ctx.set_mesh(*req["nc"], *req["L"], req["p"], [0] * 6)
    ctx.set_coefficients(req["K"])
    vol, _ = ctx.quadrature_points()
    f = torch.empty(ctx.sizes()["ndof"], dtype=torch.float64, device="cuda")
    gauss = lambda x, y, z: np.exp(-((x - 0.75) ** 2 + (y - 0.5) ** 2 + (z - 0.3) ** 2) / (2 * 0.1 ** 2))
    ctx.assemble_rhs(inputs.evaluate(gauss, vol), f)
    return ctx, f


def _batch_solve(reqs, opts, rtol=1e-8, step=3, prime=False):
    from paper_1805_11930_gb300 import dgmg
    b = dgmg.Batch(0, stream=torch.cuda.Stream(0), opts=opts)
    items = []
    for r in reqs:
        ctx, f = _prepare(r)
        u = torch.zeros_like(f)
        if prime:
            ctx.batch_prime(f, u, opts)
        items.append((ctx, f, u, b.add(ctx, f, u, rtol=rtol, maxit=400)))
    out = [None] * len(items)
    for _ in range(1000):
        left = b.step(step)
        for i, (ctx, f, u, slot) in enumerate(items):
            if out[i] is None:
                st = b.poll(slot)
                if st is not None:
                    out[i] = (u.cpu().numpy(), st)
        if left == 0 and all(o is not None for o in out):
            break
    for ctx, f, u, slot in items:
        b.remove(slot)
    b.close()
    return out


REQS = [_request((6, 5, 7), 3, 1.0, 1), _request((9, 7, 5), 3, 0.5, 2), _request((11, 10, 9), 3, 2.0, 3)]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_batch_equals_single_solves_bit_for_bit(prec):
    """Three requests of order 3 with different meshes and contrasts: each
    member's solution and iteration count equal its dgmg_solve exactly
    (mixed: FP32 V-cycle and flexible CG; fp64: FP64 V-cycle and CG)."""
    from paper_1805_11930_gb300 import dgmg
    opts = (dgmg.default_opts(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG) if prec == "mixed"
            else dgmg.default_opts())
    batched = _batch_solve(REQS, opts)
    for r, (ub, st) in zip(REQS, batched):
        ctx, f = _prepare(r)
        u = torch.zeros_like(f)
        ss = ctx.solve(f, u, opts)
        assert st["status"] == "DGMG_OK" and st["converged"] == 1
        assert st["iterations"] == ss["iterations"]
        assert np.array_equal(ub, u.cpu().numpy())
        assert st["rel_residual"] == ss["rel_residual"] <= 1e-8


def test_batch_result_same_alone_and_in_the_mix():
    """A request solved alone in a batch and beside two others (members that
    stop at other iterations) gives the same bits; its solution satisfies the
    oracle's assembled system to the stated tolerance."""
    from paper_1805_11930_gb300 import dgmg
    opts = dgmg.default_opts(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG)
    alone = _batch_solve([REQS[1]], opts)[0]
    mixed = _batch_solve([REQS[0], REQS[1], REQS[2]], opts)[1]
    assert alone[1]["iterations"] == mixed[1]["iterations"]
    assert np.array_equal(alone[0], mixed[0])
    r = REQS[1]
    P = dg.Problem(*r["nc"], *r["L"], r["p"], [0] * 6, r["K"])
    A = P.assemble()
    ctx, f = _prepare(r)
    F = f.cpu().numpy()
    assert np.linalg.norm(F - A @ alone[0]) <= 1e-8 * np.linalg.norm(F) * (1 + 1e-6)


def test_batch_rejects_mixed_orders_and_bad_arguments():
    from paper_1805_11930_gb300 import dgmg
    b = dgmg.Batch(0, opts=dgmg.default_opts(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG))
    c3, f3 = _prepare(_request((4, 4, 4), 3, 1.0, 5))
    c2, f2 = _prepare(_request((4, 4, 4), 2, 1.0, 6))
    u3, u2 = torch.zeros_like(f3), torch.zeros_like(f2)
    s = b.add(c3, f3, u3)
    with pytest.raises(dgmg.DgmgError):
        b.add(c2, f2, u2)          # another order
    with pytest.raises(dgmg.DgmgError):
        b.add(c3, f3, u3)          # already a member
    with pytest.raises(dgmg.DgmgError):
        b.add(c2, f2, f2)          # f and u alias
    b.remove(s)
    b.close()
    with pytest.raises(dgmg.DgmgError):
        dgmg.Batch(0, opts=dgmg.default_opts(inner=dgmg.INNER_GMRES))


def test_primed_members_give_the_same_bits():
    """dgmg_batch_prime computes a member's initial state on its context's own
    stream; the batched solve that starts from it equals the unprimed one."""
    from paper_1805_11930_gb300 import dgmg
    opts = dgmg.default_opts(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG)
    a = _batch_solve(REQS, opts)
    b = _batch_solve(REQS, opts, prime=True)
    for (ua, sa), (ub, sb) in zip(a, b):
        assert sa["iterations"] == sb["iterations"] and np.array_equal(ua, ub)
