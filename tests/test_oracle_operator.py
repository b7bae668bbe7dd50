"""Pins for the oracle's DG operator and right-hand side (Sec. 2.1, eqs.
bilinear_form_split, rhs, linear_equation).

Each test checks the assembled matrix against something fixed by the
mathematics rather than by the code: closed-form values of a_h on
piecewise-constant or piecewise-linear functions, symmetry and definiteness,
conservation, exact reproduction of discrete (polynomial) solutions, and the
O(h^(p+1)) convergence rate.  A swapped weight, a dropped term or a wrong
sign in any part of a_h or l_h fails at least one of them.
"""
import numpy as np
import pytest

from oracle import dg

ALPHA = 1.25


def vertex_field(nc, L, fn):
    nx, ny, nz = nc
    out = []
    for vz in range(nz + 1):
        for vy in range(ny + 1):
            for vx in range(nx + 1):
                out.append(fn(vx * L[0] / nx, vy * L[1] / ny, vz * L[2] / nz))
    return np.array(out)


def boundary_values(P, fn):
    vals = []
    for cells, xyz in P.boundary_points():
        vals.append(fn(xyz[..., 0], xyz[..., 1], xyz[..., 2]).reshape(-1))
    return np.concatenate(vals)


def test_symmetric_positive_definite_without_advection():
    rng = np.random.default_rng(1805)
    nc = (3, 2, 2)
    K = np.exp(rng.normal(size=(12, 3)))
    c = rng.uniform(0.0, 2.0, size=12)
    P = dg.Problem(*nc, 1.0, 0.7, 1.3, 2, [0, 1, 0, 0, 1, 0], K, c_cell=c)
    A = P.assemble().toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    np.linalg.cholesky(A)          # SPD: raises if not


def test_neumann_kernel_and_conservation():
    """All-Neumann, c = 0: A 1 = 0 when b = 0 (constants have zero energy),
    and 1^T A = 0 for any b, since a_h(u, 1) has only the reaction term."""
    rng = np.random.default_rng(7)
    nc = (2, 2, 3)
    K = np.exp(rng.normal(size=12))
    P = dg.Problem(*nc, 1, 1, 1, 3, [1] * 6, K)
    A = P.assemble()
    assert np.abs(A @ np.ones(P.ndof)).max() < 1e-12 * abs(A).max()
    b = vertex_field(nc, (1, 1, 1), lambda x, y, z: np.array([1 + x, y - 0.5 * z, 0.3]))
    Pb = dg.Problem(*nc, 1, 1, 1, 3, [1] * 6, K, b_vertex=b)
    Ab = Pb.assemble()
    assert np.abs(Ab.T @ np.ones(P.ndof)).max() < 1e-12 * abs(Ab).max()


@pytest.mark.parametrize("p", [1, 2, 4])
def test_interior_penalty_closed_form(p):
    """u = 1 on cell 0 and 0 on cell 1 (Neumann elsewhere, b = 0): only the
    penalty term survives, u^T A u = gamma_F |F| with
    gamma_F = alpha p (p+2) <K0_xx, K1_xx> / h_x."""
    K = np.array([[2.0, 5.0, 7.0], [0.5, 3.0, 1.0]])
    P = dg.Problem(2, 1, 1, 1.0, 0.6, 0.3, p, [1] * 6, K)
    A = P.assemble().toarray()
    u = np.zeros(P.ndof)
    u[:P.N] = 1.0
    hx, hy, hz = 0.5, 0.6, 0.3
    harm = 2 * 2.0 * 0.5 / 2.5
    expected = ALPHA * p * (p + 2) * harm / hx * hy * hz
    assert abs(u @ A @ u - expected) < 1e-12 * expected


@pytest.mark.parametrize("p", [1, 3])
def test_dirichlet_penalty_closed_form(p):
    """One cell, all Dirichlet, u = 1, b = 0, c = 0: u^T A u = sum over the six
    faces of gamma_F |F| = sum_k 2 alpha p (p+2) K_kk |F_k| / h_k."""
    K = np.array([[2.0, 3.0, 0.5]])
    h = np.array([0.5, 0.25, 2.0])
    P = dg.Problem(1, 1, 1, *h, p, [0] * 6, K)
    A = P.assemble().toarray()
    u = np.ones(P.N)
    area = [h[1] * h[2], h[0] * h[2], h[0] * h[1]]
    expected = sum(2 * ALPHA * p * (p + 2) * K[0, k] * area[k] / h[k] for k in range(3))
    assert abs(u @ A @ u - expected) < 1e-12 * expected


@pytest.mark.parametrize("p", [1, 2, 3])
def test_weighted_average_closed_form(p):
    """u = x on cell 0, 0 on cell 1; v = 1 on cell 1 (Neumann, b = 0).
    a_h(u, v) = |F| K0 K1/(K0+K1) (1 - 2 alpha p (p+2)): the consistency term
    carries w^- K0 = K1 K0/(K0+K1), the penalty gamma_F [[u]] [[v]] with
    [[u]] = h_x, [[v]] = -1.  Swapping w^- and w^+ gives K0^2/(K0+K1)."""
    K0, K1 = 4.0, 0.25
    P = dg.Problem(2, 1, 1, 2.0, 1.0, 1.0, p, [1] * 6, np.array([K0, K1]))
    A = P.assemble().toarray()
    u = P.interpolate(lambda x, y, z: x)
    u[P.N:] = 0.0
    v = np.zeros(P.ndof)
    v[P.N:] = 1.0
    expected = K0 * K1 / (K0 + K1) * (1 - 2 * ALPHA * p * (p + 2))
    assert abs(v @ A @ u - expected) < 1e-12 * abs(expected)
    assert abs(u @ A @ v - expected) < 1e-12 * abs(expected)      # symmetry term


@pytest.mark.parametrize("p", [1, 3])
def test_volume_and_reaction_closed_form(p):
    """One cell, all Neumann, b = 0, so a_h(u, v) = (K grad u, grad v)_T +
    (c u, v)_T: u = 1 gives c |T|; u = x - h_x/2 gives K_xx |T| + c |T| h_x^2/12."""
    K = np.array([[2.0, 3.0, 0.5]])
    h = np.array([0.5, 0.25, 2.0])
    c = 0.7
    P = dg.Problem(1, 1, 1, *h, p, [1] * 6, K, c_cell=np.array([c]))
    A = P.assemble().toarray()
    T = np.prod(h)
    tol = 1e-14 * np.abs(A).sum()           # rounding of the cancelling stiffness entries
    one = np.ones(P.N)
    assert abs(one @ A @ one - c * T) < tol
    u = P.interpolate(lambda x, y, z: x - h[0] / 2)
    expected = K[0, 0] * T + c * T * h[0] ** 2 / 12
    assert abs(u @ A @ u - expected) < tol


@pytest.mark.parametrize("p", [1, 2])
def test_upwind_closed_form(p):
    """Piecewise constants a, beta on two cells, b = (bx, 0, 0): the
    advection part of u^T A u is the interior upwind flux |F| bx a (a - beta)
    (bx > 0, u^- = a) plus the Dirichlet outflow term |F| bx beta^2; the
    inflow face contributes nothing.  Downwinding would give bx beta (a - beta)."""
    nc = (2, 1, 1)
    K = np.ones(2) * 0.1
    for bx in (1.5, -0.75):
        b = vertex_field(nc, (2, 1, 1), lambda x, y, z: np.array([bx, 0.0, 0.0]))
        P0 = dg.Problem(*nc, 2, 1, 1, p, [0] * 6, K)
        Pb = dg.Problem(*nc, 2, 1, 1, p, [0] * 6, K, b_vertex=b)
        Aadv = Pb.assemble().toarray() - P0.assemble().toarray()
        a, beta = 0.8, -1.7
        u = np.concatenate([np.full(P0.N, a), np.full(P0.N, beta)])
        if bx > 0:
            expected = bx * a * (a - beta) + bx * beta ** 2
        else:   # flow towards -x: u^+ = beta is upwind; outflow through x = 0
            expected = bx * beta * (a - beta) + (-bx) * a ** 2
        assert abs(u @ Aadv @ u - expected) < 1e-12 * abs(expected)


def _poly_problem(p, bc, K, b=None):
    nc = (2, 3, 2)
    L = (1.0, 1.5, 0.8)
    bv = None if b is None else vertex_field(nc, L, b)
    return dg.Problem(*nc, *L, p, bc, K, b_vertex=bv)


@pytest.mark.parametrize("p", [2, 3])
def test_discrete_solution_reproduced(p):
    """u = 1 + x^2 + 2y^2 - 3z^2 + xy is in V_h for p >= 2; with anisotropic
    constant K, f = -(2K1 + 4K2 - 6K3), Dirichlet g = u and Neumann
    j = (b u - K grad u).nu, consistency of the method gives A u_I = F
    exactly (every integrand is integrated exactly by the Gauss rule)."""
    Kd = np.array([1.5, 0.5, 2.0])
    bc = [0, 1, 0, 0, 1, 0]
    P = _poly_problem(p, bc, np.tile(Kd, (12, 1)))
    ue = lambda x, y, z: 1 + x ** 2 + 2 * y ** 2 - 3 * z ** 2 + x * y
    grad = lambda x, y, z: (2 * x + y, 4 * y + x, -6 * z)
    f = lambda x, y, z: -(2 * Kd[0] + 4 * Kd[1] - 6 * Kd[2]) + 0 * x
    X = P.volume_points()
    g = boundary_values(P, ue)
    jv = []
    for k in range(3):
        for side in (0, 1):
            cells, xyz = P.boundary_points()[2 * k + side]
            gr = grad(xyz[..., 0], xyz[..., 1], xyz[..., 2])
            nu = 1.0 if side == 1 else -1.0
            jv.append((-Kd[k] * gr[k] * nu).reshape(-1))
    F = P.rhs(f(X[..., 0], X[..., 1], X[..., 2]), g_qp=g, j_qp=np.concatenate(jv))
    A = P.assemble()
    uI = P.interpolate(ue)
    assert np.abs(A @ uI - F).max() < 1e-12 * np.abs(F).max()


@pytest.mark.parametrize("p", [2, 3])
def test_advection_discrete_solution(p):
    """u = x(1-x) y(1-y) z(1-z) with the divergence-free linear field
    b = (2(1/2 - y), x - 1/2, 1/4), kappa = 1e-3, g = 0:
    f = -kappa lap u + b . grad u, and A u_I = F exactly (Sec. 4.3 uses this u)."""
    kap = 1e-3
    nc = (3, 2, 2)
    L = (1.0, 1.0, 1.0)
    bf = lambda x, y, z: np.array([2 * (0.5 - y), x - 0.5, 0.25 + 0 * x])
    P = dg.Problem(*nc, *L, p, [0] * 6, np.full(12, kap), b_vertex=vertex_field(nc, L, bf))
    u = lambda x, y, z: x * (1 - x) * y * (1 - y) * z * (1 - z)

    def f(x, y, z):
        lap = -2 * (y * (1 - y) * z * (1 - z) + x * (1 - x) * z * (1 - z) + x * (1 - x) * y * (1 - y))
        ux = (1 - 2 * x) * y * (1 - y) * z * (1 - z)
        uy = x * (1 - x) * (1 - 2 * y) * z * (1 - z)
        uz = x * (1 - x) * y * (1 - y) * (1 - 2 * z)
        b = bf(x, y, z)
        return -kap * lap + b[0] * ux + b[1] * uy + b[2] * uz

    X = P.volume_points()
    F = P.rhs(f(X[..., 0], X[..., 1], X[..., 2]), g_qp=boundary_values(P, lambda x, y, z: 0 * x))
    A = P.assemble()
    assert np.abs(A @ P.interpolate(u) - F).max() < 1e-12 * np.abs(F).max()


@pytest.mark.parametrize("p", [1, 2])
def test_convergence_order(p):
    """-lap u = 3 pi^2 prod sin(pi x_k), u = 0 on the boundary: L2 error
    O(h^(p+1)) over 2^3, 4^3, 8^3 meshes."""
    import scipy.sparse.linalg as spla
    u = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    errs = []
    for nx in (2, 4, 8):
        P = dg.Problem(nx, nx, nx, 1, 1, 1, p, [0] * 6, np.ones(nx ** 3))
        X = P.volume_points()
        F = P.rhs(3 * np.pi ** 2 * u(X[..., 0], X[..., 1], X[..., 2]),
                  g_qp=boundary_values(P, lambda x, y, z: 0 * x))
        uh = spla.spsolve(P.assemble().tocsc(), F)
        errs.append(P.l2_error(uh, u))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates[-1] > p + 1 - 0.25, (errs, rates)


def test_sampled_rows_match_assembly():
    rng = np.random.default_rng(3)
    nc = (3, 3, 2)
    K = np.exp(rng.normal(size=(18, 3)))
    b = vertex_field(nc, (1, 1, 1), lambda x, y, z: np.array([1 - y, x, 0.2]))
    P = dg.Problem(*nc, 1, 1, 1, 2, [0, 1, 0, 1, 0, 0], K, b_vertex=b, c_cell=rng.uniform(size=18))
    u = rng.uniform(-1, 1, P.ndof)
    v = P.assemble() @ u
    cells = [0, 4, 17, 9]
    vs = P.apply_rows(u, cells)
    for r, c in enumerate(cells):
        np.testing.assert_allclose(vs[r], v[c * P.N:(c + 1) * P.N], rtol=0, atol=1e-13 * np.abs(v).max())


def test_pointwise_coefficients_reduce_to_cellwise():
    """K and c given as functions that are constant on each cell give the same
    matrix and right-hand side as the per-cell coefficients (volume, interior
    and boundary faces, Dirichlet data), to rounding."""
    rng = np.random.default_rng(21)
    nc, L, p, bc = (3, 2, 2), (1.0, 0.8, 1.2), 2, [0, 1, 0, 0, 1, 0]
    ncell = int(np.prod(nc))
    Q = np.linalg.qr(rng.normal(size=(3, 3)))[0]
    K = np.stack([Q @ np.diag(rng.uniform(0.5, 3.0, 3)) @ Q.T for _ in range(ncell)])
    c = rng.uniform(0.1, 1.0, ncell)
    # a function of x cannot tell the two cells of a face apart, so the
    # per-cell case is compared on one cell, and on a mesh with one constant K
    P1 = dg.Problem(1, 1, 1, *L, p, [0] * 6, K[:1], c_cell=c[:1])
    P2 = dg.Problem(1, 1, 1, *L, p, [0] * 6, K[:1], K_fn=lambda x: np.broadcast_to(K[0], x.shape[:-1] + (3, 3)),
                    c_fn=lambda x: np.full(x.shape[:-1], c[0]))
    A1, A2 = P1.assemble().toarray(), P2.assemble().toarray()
    assert np.abs(A1 - A2).max() < 1e-13 * np.abs(A1).max()
    Kc = K[0]
    Pa = dg.Problem(*nc, *L, p, bc, np.broadcast_to(Kc, (ncell, 3, 3)).copy(), c_cell=np.full(ncell, c[0]))
    Pb = dg.Problem(*nc, *L, p, bc, np.broadcast_to(Kc, (ncell, 3, 3)).copy(),
                    K_fn=lambda x: np.broadcast_to(Kc, x.shape[:-1] + (3, 3)),
                    c_fn=lambda x: np.full(x.shape[:-1], c[0]))
    Aa, Ab = Pa.assemble().toarray(), Pb.assemble().toarray()
    assert np.abs(Aa - Ab).max() < 1e-13 * np.abs(Aa).max()
    pts = np.concatenate([xyz.reshape(-1, 3) for _, xyz in Pa.boundary_points()])
    g = np.sin(pts[:, 0]) + pts[:, 1] * pts[:, 2]
    fq = np.ones((ncell, Pa.m ** 3))
    Fa, Fb = Pa.rhs(fq, g_qp=g, j_qp=g), Pb.rhs(fq, g_qp=g, j_qp=g)
    assert np.abs(Fa - Fb).max() < 1e-13 * np.abs(Fa).max()


def test_variable_tensor_manufactured_convergence():
    """-div(K(x) grad u) + c(x) u = f with the paper's rotated, quadratic K(x)
    (Sec. 4.2), u = sin(pi x) sin(pi y) sin(pi z) + x y z, Dirichlet data
    g = u, Neumann data j = -(K grad u).n on x = 1: the L2 error falls by
    about 2^(p+1) per halving of h (p = 2: ratio > 6)."""
    sympy = pytest.importorskip("sympy")
    import scipy.sparse.linalg as spla
    from paper_1805_11930_gb300 import inputs
    X = sympy.symbols("x y z")
    us = sympy.sin(sympy.pi * X[0]) * sympy.sin(sympy.pi * X[1]) * sympy.sin(sympy.pi * X[2]) + X[0] * X[1] * X[2]
    nb = inputs.VARK_BASIS
    Ks = sympy.zeros(3, 3)
    for k in range(3):
        pk = inputs.VARK_P0[k] + inputs.VARK_P2[k] * X[k] ** 2
        n = sympy.Matrix(nb[k])
        Ks += pk * (n * n.T)
    grad = sympy.Matrix([sympy.diff(us, v) for v in X])
    flux = Ks * grad
    gamma = 0.5        # a visible reaction term (the paper's 1e-8 would not be tested)
    cs = gamma * (X[0] ** 2 + X[1] ** 2 + X[2] ** 2)
    fs = -sum(sympy.diff(flux[i], X[i]) for i in range(3)) + cs * us
    f_fn = sympy.lambdify(X, fs, "numpy")
    u_fn = sympy.lambdify(X, us, "numpy")
    jx_fn = sympy.lambdify(X, -flux[0], "numpy")      # outward normal +e_x on x = 1
    errs = []
    for n in (3, 6):
        P = dg.Problem(n, n, n, 1.0, 1.0, 1.0, 2, [0, 1, 0, 0, 0, 0], np.ones(n ** 3),
                       K_fn=inputs.vark_tensor, c_fn=lambda x: inputs.vark_reaction(x, gamma))
        Xq = P.volume_points()
        pts = np.concatenate([xyz.reshape(-1, 3) for _, xyz in P.boundary_points()])
        F = P.rhs(f_fn(Xq[..., 0], Xq[..., 1], Xq[..., 2]), g_qp=u_fn(pts[:, 0], pts[:, 1], pts[:, 2]),
                  j_qp=jx_fn(pts[:, 0], pts[:, 1], pts[:, 2]))
        A = P.assemble().tocsc()
        u = spla.spsolve(A, F)
        errs.append(P.l2_error(u, u_fn))
    assert errs[0] / errs[1] > 6.0, errs


@pytest.mark.parametrize("p", [1, 3])
def test_penalty_parameter_enters_only_the_jump_term(p):
    """a_h depends on alpha only through gamma_F [[u]][[v]], which is linear in
    alpha: A(alpha) = A_0 + alpha J with J symmetric positive semi-definite,
    J u = 0 for every continuous u that vanishes on the Dirichlet faces (no
    jumps), and u^T J u = p (p+2) sum_F <K>/h |F| [[u]]^2 for a unit jump."""
    rng = np.random.default_rng(23)
    nc = (3, 2, 2)
    K = np.exp(rng.normal(size=(12, 3)))
    bc = [0, 1, 1, 0, 1, 1]
    mk = lambda a: dg.Problem(*nc, 1.0, 0.8, 0.6, p, bc, K, c_cell=np.full(12, 0.3), alpha=a).assemble().toarray()
    A1, A2, A3 = mk(1.0), mk(2.0), mk(3.5)
    J = A2 - A1
    assert np.abs((A3 - A1) - 2.5 * J).max() < 1e-11 * np.abs(A1).max()
    assert np.abs(J - J.T).max() < 1e-12 * np.abs(J).max()
    assert np.linalg.eigvalsh(J).min() > -1e-10 * np.abs(J).max()
    # a continuous piecewise-trilinear field, zero on the Dirichlet planes
    # (bc[2k+s] is the plane x_k = s L_k: here x = 0 and y = L_y)
    from oracle import transfer
    P = dg.Problem(*nc, 1.0, 0.8, 0.6, p, bc, K, alpha=2.0)
    Pm = transfer.prolongation(P).toarray()
    nv = P.nv
    uh = rng.normal(size=P.nvert)
    v = np.arange(P.nvert)
    uh[v % nv[0] == 0] = 0.0
    uh[(v // nv[0]) % nv[1] == nv[1] - 1] = 0.0
    u = Pm @ uh
    assert np.abs(J @ u).max() < 1e-11 * np.abs(J).max() * np.abs(u).max()


def test_block_structure_matches_the_problem_size_count():
    """The assembled matrix has a block for every cell and two for every
    interior face, nothing else: ncell + 2 (interior faces) blocks of
    (p+1)^6 entries, which tends to Table 1's 7 blocks per cell (Sec. 4)."""
    nc = (4, 3, 2)
    P = dg.Problem(*nc, 1, 1, 1, 1, [0, 1, 0, 1, 1, 0], np.ones(24))
    A = P.assemble()
    nx, ny, nz = nc
    faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1)
    assert A.indices.size == 24 + 2 * faces
    cols = {c: set(A.indices[A.indptr[c]:A.indptr[c + 1]]) for c in range(24)}
    for c in range(24):
        cx, cy, cz = P.cell_coords(c)
        nb = {c}
        for k, (v, n) in enumerate(zip((cx, cy, cz), nc)):
            for s in (-1, 1):
                if 0 <= v + s < n:
                    q = [cx, cy, cz]
                    q[k] += s
                    nb.add(P.cell_index(*q))
        assert cols[c] == nb


def test_l2_error_and_interpolation_closed_forms():
    """The norm used by the convergence pins: ||0 - u||_L2 of
    u = sin(pi x) sin(pi y) sin(pi z) on [0,1] x [0,2] x [0,1] is exactly
    sqrt(1/8 * 2) = 1/2 (up to the rule's accuracy), and the nodal
    interpolant of a polynomial in Q_p has zero error."""
    P = dg.Problem(3, 4, 2, 1.0, 2.0, 1.0, 3, [0] * 6, np.ones(24))
    u = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)   # noqa: E731
    assert abs(P.l2_error(np.zeros(P.ndof), u, extra=4) - 0.5) < 1e-7
    poly = lambda x, y, z: 1 + x ** 3 - 2 * x * y ** 2 * z ** 3 + y * z                 # noqa: E731
    assert P.l2_error(P.interpolate(poly), poly) < 1e-13
