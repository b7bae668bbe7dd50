"""Shared set-up of the parity tests: one workload dict (from
paper_1805_11930_gb300.inputs) turned into an oracle Problem and a library
Context, each evaluating the analytic data at its own quadrature points."""
import numpy as np

from oracle import dg
from paper_1805_11930_gb300 import inputs


def oracle_problem(w):
    return dg.Problem(*w["nc"], *w["L"], w["p"], w["bc"], w["K"], b_vertex=w["b"], c_cell=w["c"])


def oracle_rhs(P, w):
    X = P.volume_points()
    fq = inputs.evaluate(w["f"], X)
    gq = jq = None
    pts = np.concatenate([xyz.reshape(-1, 3) for _, xyz in P.boundary_points()])
    if w["g"] is not None:
        gq = inputs.evaluate(w["g"], pts)
    if w["j"] is not None:
        jq = inputs.evaluate(w["j"], pts)
    return P.rhs(fq, g_qp=gq, j_qp=jq)


def gpu_context(w, device=0):
    from paper_1805_11930_gb300 import dgmg
    ctx = dgmg.Context(device)
    ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
    ctx.set_coefficients(w["K"], b_vertex=w["b"], c_cell=w["c"])
    return ctx


def gpu_rhs(ctx, w, torch):
    vol, face = ctx.quadrature_points()
    s = ctx.sizes()
    rhs = torch.empty(s["ndof"], dtype=torch.float64, device="cuda")
    ctx.assemble_rhs(inputs.evaluate(w["f"], vol), rhs,
                     g_qp=inputs.evaluate(w["g"], face), j_qp=inputs.evaluate(w["j"], face))
    return rhs


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def custom(nc, L, p, bc, K, b=None, c=None, f=None, g=None, j=None):
    return dict(name="custom", nc=tuple(nc), L=tuple(L), p=p, bc=list(bc), K=K, b=b, c=c,
                f=f if f is not None else (lambda x, y, z: np.ones_like(x)), g=g, j=j, exact=None)


def elem_errors(v, ref, A, u, nc, ndof_cell):
    """Largest element error of v against ref, scaled by ||A||_inf ||u||_inf,
    over all elements and separately over the elements of the corner, edge and
    face cells of the nc grid (cells with 3, 2 or 1 coordinates on the
    boundary): {class: error}.  A norm-wise check could hide one wrong
    boundary value; this one cannot."""
    import scipy.sparse as sp
    v = np.asarray(v, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = abs(sp.csr_matrix(A)).sum(axis=1).max() * np.abs(np.asarray(u, dtype=np.float64)).max()
    err = np.abs(v - ref).reshape(-1, ndof_cell).max(axis=1) / max(scale, 1e-300)
    nx, ny, nz = nc
    c = np.arange(nx * ny * nz)
    cx, cy, cz = c % nx, (c // nx) % ny, c // (nx * ny)
    onb = (((cx == 0) | (cx == nx - 1)).astype(int) + ((cy == 0) | (cy == ny - 1)).astype(int)
           + ((cz == 0) | (cz == nz - 1)).astype(int))
    out = {"all": float(err.max())}
    for k, name in ((3, "corner"), (2, "edge"), (1, "face")):
        if (onb == k).any():
            out[name] = float(err[onb == k].max())
    return out
