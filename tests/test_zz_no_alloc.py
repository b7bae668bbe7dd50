"""dgmg_restrict_noalloc against dgmg_restrict.

Some callers cannot allocate device memory (code under CUDA-graph capture,
hosts that own all device memory through their own pool); for them the
restriction has a context-free entry point whose scratch is a fixed array
inside the library.  It must give the same vertex vector as the context-based
dgmg_restrict, on consecutive calls whose grids differ (the shared scratch
keeps the previous call's contents), and reject grids larger than its
scratch."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_restrict_noalloc_matches_restrict_on_two_calls():
    from paper_1805_11930_gb300 import dgmg, inputs
    cases = [((9, 7, 5), 3, torch.float64, 31), ((4, 6, 3), 2, torch.float32, 32)]
    for nc, p, dtype, seed in cases:
        ctx = dgmg.Context(0)
        ctx.set_mesh(*nc, 1.0, 0.7, 1.1, p, [0] * 6)
        ctx.set_coefficients(np.ones(int(np.prod(nc))))
        s = ctx.sizes()
        r = torch.tensor(inputs.random_dg_vector(s["ndof"], seed=seed), dtype=dtype, device="cuda")
        ref = torch.empty(s["nvert"], dtype=torch.float64, device="cuda")
        got = torch.full((s["nvert"],), float("nan"), dtype=torch.float64, device="cuda")
        ctx.restrict(r, ref)
        dgmg.restrict_noalloc(*nc, p, r, got)
        torch.cuda.synchronize()
        tol = 1e-13 if dtype == torch.float64 else 1e-5
        assert _rel(got, ref) < tol
        ctx.close()


def test_restrict_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1805_11930_gb300 import dgmg
    r = torch.zeros(8, dtype=torch.float64, device="cuda")
    rh = torch.zeros(8, dtype=torch.float64, device="cuda")
    assert 64 * 64 * 33 > dgmg.NOALLOC_MAX_CELLS
    with pytest.raises(dgmg.DgmgError):
        dgmg.restrict_noalloc(64, 64, 33, 1, r, rh)
