"""dgmg_restrict_noalloc, the restriction for callers that cannot allocate.

Some callers may not allocate device memory at all: a host application that
owns every byte of device memory through its own pool and forbids other
allocators, or a real-time loop that must not wait on cudaMalloc (which can
synchronise the device).  For them the DG -> Q1 restriction has an entry
point that takes no context and keeps its scratch in a fixed array inside
the library.  These tests check that

* its first calls in a fresh process, before any context exists on the
  device (so its own one-time set-up of the 1D tables is what the kernels
  read), equal the oracle's R r = P^T r, on two calls in a row with
  different grids, orders and precisions;
* after the other tests, on two calls in a row, it gives the same vertex
  vector, bit for bit, as the context-based dgmg_restrict, which launches
  the same kernels with the same launch shape and summation order (the
  shared scratch keeps the previous call's contents);
* a grid of exactly DGMG_NOALLOC_MAX_CELLS cells, which fills the whole
  scratch array, is restricted correctly, and one cell more is refused.

This file is collected last, so that a run that stops at the first failure
has run every other test already."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Two grids, orders and precisions, restricted by the entry point before any
# context exists in the process, then compared with the oracle on the host.
FRESH = r"""
import json, sys
import numpy as np
import torch
sys.path.insert(0, ROOT)
from paper_1805_11930_gb300 import dgmg, inputs
from oracle import dg, transfer
out = []
for nc, p, dtype, seed in [((9, 7, 5), 3, torch.float64, 31), ((4, 6, 3), 2, torch.float32, 32)]:
    ncell = nc[0] * nc[1] * nc[2]
    r = inputs.random_dg_vector(ncell * (p + 1) ** 3, seed=seed)
    rd = torch.tensor(r, dtype=dtype, device="cuda")
    nvert = (nc[0] + 1) * (nc[1] + 1) * (nc[2] + 1)
    got = torch.full((nvert,), float("nan"), dtype=torch.float64, device="cuda")
    dgmg.restrict_noalloc(*nc, p, rd, got)
    torch.cuda.synchronize()
    P = dg.Problem(*nc, 1.0, 0.7, 1.1, p, [0] * 6, np.ones(ncell))
    ref = transfer.prolongation(P).T @ rd.double().cpu().numpy()
    g = got.cpu().numpy()
    out.append({"p": p, "fp32": dtype == torch.float32, "finite": bool(np.isfinite(g).all()),
                "rel": float(np.linalg.norm(g - ref) / np.linalg.norm(ref)),
                "max": float(np.abs(g - ref).max() / np.abs(ref).max())})
print(json.dumps(out))
"""


def test_restrict_noalloc_first_call_in_a_fresh_process_matches_the_oracle():
    env = dict(os.environ)
    r = subprocess.run([sys.executable, "-c", FRESH.replace("ROOT", repr(ROOT))], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(res) == 2
    for case in res:
        tol = 1e-5 if case["fp32"] else 1e-13
        assert case["finite"], case
        assert case["rel"] < tol and case["max"] < tol, case


def test_restrict_noalloc_equals_restrict_on_two_calls():
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
        assert torch.equal(got, ref)
        ctx.close()


def test_restrict_noalloc_at_its_limit_and_one_cell_beyond():
    from paper_1805_11930_gb300 import dgmg, inputs
    nc, p = (64, 64, 32), 1
    assert nc[0] * nc[1] * nc[2] == dgmg.NOALLOC_MAX_CELLS
    ctx = dgmg.Context(0)
    ctx.set_mesh(*nc, 1.0, 1.0, 0.5, p, [0] * 6)
    ctx.set_coefficients(np.ones(int(np.prod(nc))))
    s = ctx.sizes()
    r = torch.tensor(inputs.random_dg_vector(s["ndof"], seed=33), dtype=torch.float64, device="cuda")
    ref = torch.empty(s["nvert"], dtype=torch.float64, device="cuda")
    got = torch.full((s["nvert"],), float("nan"), dtype=torch.float64, device="cuda")
    ctx.restrict(r, ref)
    dgmg.restrict_noalloc(*nc, p, r, got)
    torch.cuda.synchronize()
    assert torch.equal(got, ref)
    ctx.close()
    rr = torch.zeros(8 * 2, dtype=torch.float64, device="cuda")
    rh = torch.zeros(4 * 2 * 2, dtype=torch.float64, device="cuda")
    with pytest.raises(dgmg.DgmgError):
        dgmg.restrict_noalloc(dgmg.NOALLOC_MAX_CELLS + 1, 1, 1, p, rr, rh)
    with pytest.raises(dgmg.DgmgError):
        dgmg.restrict_noalloc(64, 64, 33, p, rr, rh)
