"""Pins for the oracle's Q1 transfer, coarse matrix, AMG, block smoother,
V-cycle (Algorithm 1) and Krylov solvers."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import amg, dg, solvers, transfer


def small_problem(p=2, nc=(3, 2, 3), bc=(0, 0, 1, 0, 0, 1), seed=5, advect=False, react=False):
    rng = np.random.default_rng(seed)
    ncell = int(np.prod(nc))
    K = np.exp(rng.normal(size=(ncell, 3)))
    bv = None
    if advect:
        nv = [n + 1 for n in nc]
        bv = rng.uniform(-1, 1, size=(int(np.prod(nv)), 3))
    c = rng.uniform(0, 1, size=ncell) if react else None
    return dg.Problem(*nc, 1.0, 0.8, 1.2, p, list(bc), K, b_vertex=bv, c_cell=c)


def test_prolongation_reproduces_trilinear_functions():
    """P is injection (Sec. 2.2.2): a trilinear function given by its vertex
    values is reproduced exactly at every GLL node."""
    P = small_problem(p=3)
    Pm = transfer.prolongation(P)
    q = lambda x, y, z: 1.0 + 2 * x - y + 0.5 * z + 3 * x * y - x * z + y * z - 2 * x * y * z
    nx, ny, nz = P.nc
    vals = np.zeros(P.nvert)
    for vz in range(nz + 1):
        for vy in range(ny + 1):
            for vx in range(nx + 1):
                vals[P.vertex_index(vx, vy, vz)] = q(vx * P.h[0], vy * P.h[1], vz * P.h[2])
    np.testing.assert_allclose(Pm @ vals, P.interpolate(q), atol=1e-13)
    np.testing.assert_allclose(Pm @ np.ones(P.nvert), 1.0, atol=1e-14)    # partition of unity


@pytest.mark.parametrize("advect,react", [(False, False), (True, True)])
def test_q1_rediscretisation_equals_galerkin_product(advect, react):
    """App. A.2: re-discretising in Q1 (Dirichlet terms with gamma from the DG
    degree p) gives exactly P^T A P."""
    P = small_problem(p=2, advect=advect, react=react)
    Pm = transfer.prolongation(P)
    G = (Pm.T @ P.assemble() @ Pm).toarray()
    Ah = transfer.q1_matrix(P).toarray()
    assert np.abs(G - Ah).max() < 1e-13 * np.abs(G).max()


def test_aggregation_shapes_and_galerkin():
    Pa, cd = amg.aggregation((9, 9, 9))
    assert cd == (5, 5, 5) and Pa.shape == (729, 125)
    np.testing.assert_array_equal(np.asarray(Pa.sum(axis=1)).ravel(), 1.0)
    Pa, cd = amg.aggregation((61, 221, 86))
    assert cd == (31, 111, 43)


def test_amg_symmetric_and_convergent():
    """For symmetric A_hat the V-cycle (equal pre/post Jacobi) is a symmetric
    operator, and as a stationary iteration it converges."""
    P = small_problem(p=2, nc=(7, 6, 5), bc=(0,) * 6)
    Ah = transfer.q1_matrix(P)
    am = amg.AggregationAMG(Ah, P.nv, coarse_size=20)
    assert am.nlevels >= 3
    rng = np.random.default_rng(0)
    x, y = rng.normal(size=P.nvert), rng.normal(size=P.nvert)
    assert abs(y @ am.vcycle(x) - x @ am.vcycle(y)) < 1e-12 * abs(y @ am.vcycle(x))
    b = rng.normal(size=P.nvert)
    u = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    for _ in range(30):
        u = u + am.vcycle(b - Ah @ u)
    assert np.linalg.norm(b - Ah @ u) < 1e-3 * r0
    full = amg.AggregationAMG(Ah, P.nv, coarse_size=10 ** 6)    # one level: exact solve
    assert np.abs(Ah @ full.vcycle(b) - b).max() < 1e-10 * np.abs(b).max()


def test_block_pcg_and_gmres():
    rng = np.random.default_rng(2)
    P = small_problem(p=3, nc=(2, 2, 2))
    D = P.diagonal_block(3)
    d = rng.normal(size=P.N)
    exact = np.linalg.solve(D, d)
    x, it = solvers.block_pcg(D, d, np.diag(D), 1e-14, P.N)
    assert np.abs(x - exact).max() < 1e-9 * np.abs(exact).max()
    x, it = solvers.block_pcg(D, d, np.diag(D), 1e-2, P.N)
    assert np.linalg.norm(d - D @ x) <= 1e-2 * np.linalg.norm(d) and it >= 1
    Pa = small_problem(p=3, nc=(2, 2, 2), advect=True)
    Da = Pa.diagonal_block(5)
    exact = np.linalg.solve(Da, d)
    x, it = solvers.block_gmres(Da, d, np.diag(Da), 1e-13, 10 * P.N, 12)
    assert np.abs(x - exact).max() < 1e-8 * np.abs(exact).max()
    x, it = solvers.block_gmres(Da, d, np.diag(Da), 1e-2, 10 * P.N, 12)
    assert np.linalg.norm(d - Da @ x) <= 1e-2 * np.linalg.norm(d) * (1 + 1e-12)


def test_block_jacobi_single_cell_is_exact():
    P = small_problem(p=2, nc=(1, 1, 1), bc=(0,) * 6)
    A = P.assemble()
    f = np.random.default_rng(1).normal(size=P.ndof)
    S = solvers.BlockJacobi(A, P.N, inner="lu")
    u = S(f, np.zeros_like(f), 1, 1.0)
    np.testing.assert_allclose(A @ u, f, atol=1e-12 * np.abs(f).max())


def _c1_like(nx=4, p=2):
    P = dg.Problem(nx, nx, nx, 1, 1, 1, p, [0] * 6, np.ones(nx ** 3))
    A = P.assemble()
    Pm = transfer.prolongation(P)
    Ah = transfer.q1_matrix(P)
    return P, A, Pm, Ah


def test_vcycle_symmetric_with_exact_blocks():
    """With exact block solves and n_pre = n_post, the V-cycle of Algorithm 1
    (zero initial guess) is a symmetric linear operator for symmetric A."""
    P, A, Pm, Ah = _c1_like()
    am = amg.AggregationAMG(Ah, P.nv, coarse_size=10 ** 6)
    V = solvers.HybridVCycle(A, Pm, solvers.BlockJacobi(A, P.N, inner="lu"), am.vcycle)
    rng = np.random.default_rng(4)
    x, y = rng.normal(size=P.ndof), rng.normal(size=P.ndof)
    assert abs(y @ V(x) - x @ V(y)) < 1e-11 * abs(y @ V(x))


def test_cg_vcycle_solves_poisson():
    """CG + hybrid V-cycle (block-Jacobi, inner PCG eps = 1e-2, Q1 + AMG)
    reaches 1e-8.  Smoke check of the inner iteration counts against Sec. 4.2
    (mean below 4, maximum 15 for Poisson on the paper's smooth RHS): with a
    random RHS the mean here is about 4.3, so the bound is mean < 5, max <= 15."""
    P, A, Pm, Ah = _c1_like(nx=4, p=2)
    am = amg.AggregationAMG(Ah, P.nv, coarse_size=30)
    S = solvers.BlockJacobi(A, P.N, inner="pcg", eps=1e-2)
    V = solvers.HybridVCycle(A, Pm, S, am.vcycle)
    f = np.random.default_rng(9).normal(size=P.ndof)
    x, it, hist = solvers.cg(lambda v: A @ v, f, V, rtol=1e-8)
    assert np.linalg.norm(f - A @ x) <= 1e-8 * np.linalg.norm(f) * 1.0001
    assert it < 40
    assert S.last_its.mean() < 5 and S.last_its.max() <= 15
    xf, itf, _ = solvers.cg(lambda v: A @ v, f, V, rtol=1e-8, flexible=True)
    assert np.linalg.norm(f - A @ xf) <= 1e-8 * np.linalg.norm(f) * 1.0001
    exact = spla.spsolve(A.tocsc(), f)
    assert np.abs(x - exact).max() < 1e-5 * np.abs(exact).max()


def test_fgmres_nonsymmetric():
    P = small_problem(p=2, nc=(3, 3, 2), bc=(0,) * 6, advect=True)
    A = P.assemble()
    Pm = transfer.prolongation(P)
    am = amg.AggregationAMG(transfer.q1_matrix(P), P.nv, coarse_size=10 ** 6)
    V = solvers.HybridVCycle(A, Pm, solvers.BlockJacobi(A, P.N, inner="lu"), am.vcycle)
    f = np.random.default_rng(8).normal(size=P.ndof)
    x, it, hist = solvers.fgmres(lambda v: A @ v, f, V, restart=30, rtol=1e-10)
    assert np.linalg.norm(f - A @ x) <= 1e-10 * np.linalg.norm(f) * 1.0001
    exact = spla.spsolve(A.tocsc(), f)
    assert np.abs(x - exact).max() < 1e-7 * np.abs(exact).max()


def test_multicolour_sor_properties():
    """Colour classes have no face neighbours (so a colour can be updated in
    parallel); with one cell per colour (2x2x2 mesh) a forward pass with exact
    blocks is block Gauss-Seidel in colour order, which converges for SPD A;
    the symmetric sweep makes the smoother operator symmetric."""
    P = small_problem(p=2, nc=(2, 2, 2), bc=(0,) * 6)
    A = P.assemble()
    S = solvers.MulticolourBlockSOR(A, P.N, P.nc, symmetric=True, inner="lu")
    for c in range(P.ncell):
        for k in range(3):
            cx = list(P.cell_coords(c))
            if cx[k] + 1 < P.nc[k]:
                cx[k] += 1
                assert S.colour[c] != S.colour[P.cell_index(*cx)]
    rng = np.random.default_rng(3)
    f = rng.normal(size=P.ndof)
    u = np.zeros_like(f)
    r0 = np.linalg.norm(f)
    for _ in range(20):
        u = S(f, u, 1, 1.0)
    assert np.linalg.norm(f - A @ u) < 1e-3 * r0
    x, y = rng.normal(size=P.ndof), rng.normal(size=P.ndof)
    Sx = S(x, np.zeros_like(x), 1, 1.0)
    Sy = S(y, np.zeros_like(y), 1, 1.0)
    assert abs(y @ Sx - x @ Sy) < 1e-10 * abs(y @ Sx)


def test_thomas_solve_brute_force():
    """The Thomas algorithm against a dense solve of the assembled tridiagonal
    matrix (non-symmetric, diagonally dominant, so no pivoting is needed)."""
    rng = np.random.default_rng(7)
    n = 9
    sub = np.concatenate(([0.0], rng.uniform(-1, 1, n - 1)))
    sup = np.concatenate((rng.uniform(-1, 1, n - 1), [0.0]))
    diag = 3.0 + rng.uniform(0, 1, n)
    T = np.diag(diag) + np.diag(sub[1:], -1) + np.diag(sup[:-1], 1)
    r = rng.normal(size=n)
    assert np.abs(solvers.thomas_solve(sub, diag, sup, r) - np.linalg.solve(T, r)).max() < 1e-14
    s2, d2, u2 = solvers.tridiagonal_part(T + np.triu(rng.normal(size=(n, n)), 2))
    assert np.array_equal(s2, sub) and np.array_equal(u2, sup) and np.array_equal(d2, diag)


def test_tridiagonal_preconditioner_exact_on_tridiagonal_block():
    """Right preconditioning by the exact inverse: one GMRES iteration solves a
    tridiagonal block (a transposed or shifted band would not)."""
    rng = np.random.default_rng(8)
    n = 27
    D = np.diag(4.0 + rng.uniform(size=n)) + np.diag(rng.uniform(-2, 0, n - 1), -1) + np.diag(rng.uniform(0, 1, n - 1), 1)
    d = rng.normal(size=n)
    tri = solvers.tridiagonal_part(D)
    x, it = solvers.block_gmres(D, d, np.diag(D), 1e-12, 50, 12, minv=lambda v: solvers.thomas_solve(*tri, v))
    assert it == 1 and np.linalg.norm(d - D @ x) <= 1e-12 * np.linalg.norm(d)


def test_tridiagonal_preconditioner_convection_dominated_block():
    """Sec. 4.3: at grid Peclet number 2000 with b = (1, 0, 0) the diagonal
    preconditioner does not bring the inner GMRES to eps = 1e-2 (here: not in
    200 iterations), the tridiagonal (Thomas) preconditioner does within 20."""
    from paper_1805_11930_gb300 import inputs
    nc, L, p = (4, 4, 4), (1.0, 1.0, 1.0), 3
    K = np.full(64, 0.25 / 2000)
    b = inputs.vertex_field(nc, L, lambda x, y, z: np.stack([np.ones_like(x), 0 * x, 0 * x], -1))
    P = dg.Problem(*nc, *L, p, [0] * 6, K, b_vertex=b)
    D = P.diagonal_block(21)
    d = np.random.default_rng(0).normal(size=P.N)
    x, it = solvers.block_gmres(D, d, np.diag(D), 1e-2, 200, 12)
    assert it == 200 and np.linalg.norm(d - D @ x) > 1e-2 * np.linalg.norm(d)
    tri = solvers.tridiagonal_part(D)
    x, it = solvers.block_gmres(D, d, np.diag(D), 1e-2, 200, 12, minv=lambda v: solvers.thomas_solve(*tri, v))
    assert it <= 20 and np.linalg.norm(d - D @ x) <= 1e-2 * np.linalg.norm(d) * (1 + 1e-12)


def _modified_fv(nc, L, p, bc, K, c=None, bconst=None, alpha=1.25):
    """The cell-centred finite-volume matrix of App. A.1 (central differences
    with the harmonic mean of K on interior faces, one-sided differences over
    the centre-to-face distance h/2 on Dirichlet faces, upwind convection with
    b at the face centre, c |T| on the diagonal), with its diffusion terms
    scaled as the P0 Galerkin product scales them: interior faces by
    alpha p (p + 2), Dirichlet faces by alpha p (p + 2) / 2 (relative to the
    true distance h/2; the appendix prints |F| / (2 |T|) for that inverse
    distance, i.e. 1/(2h) instead of 2/h, and hence the factor 2 alpha p (p+2))."""
    nx, ny, nz = nc
    h = np.array(L) / np.array(nc)
    vol = np.prod(h)
    n = nx * ny * nz
    M = np.zeros((n, n))
    s = alpha * p * (p + 2)
    idx = lambda x, y, z: x + nx * (y + ny * z)   # noqa: E731
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                i = idx(x, y, z)
                if c is not None:
                    M[i, i] += c[i] * vol
                for k in range(3):
                    area = vol / h[k]
                    for side, step in ((0, -1), (1, 1)):
                        q = [x, y, z]
                        q[k] += step
                        inside = 0 <= q[k] < nc[k]
                        bn = 0.0 if bconst is None else bconst[k] * step   # b . outward normal
                        if inside:
                            j = idx(*q)
                            Kh = 2 * K[i, k] * K[j, k] / (K[i, k] + K[j, k])
                            M[i, i] += s * Kh / h[k] * area
                            M[i, j] -= s * Kh / h[k] * area
                            M[i, i] += max(bn, 0.0) * area
                            M[i, j] += min(bn, 0.0) * area
                        elif bc[2 * k + side] == 0:
                            M[i, i] += 0.5 * s * K[i, k] / (h[k] / 2) * area
                            M[i, i] += max(bn, 0.0) * area
    return M


@pytest.mark.parametrize("advect", [False, True])
def test_p0_galerkin_matrix_is_modified_fv(advect):
    """App. A.1: on an equidistant axis-parallel grid with K, b and c constant
    per cell, P^T A P for the P0 subspace is the finite-volume matrix with the
    diffusion terms re-scaled (interior faces by alpha p (p+d-1))."""
    from paper_1805_11930_gb300 import inputs
    rng = np.random.default_rng(11)
    nc, L, p, bc = (3, 4, 2), (1.0, 0.8, 1.2), 3, [0, 1, 0, 0, 1, 0]
    ncell = int(np.prod(nc))
    K = np.exp(rng.normal(size=(ncell, 3)))
    c = rng.uniform(0.1, 1.0, size=ncell)
    bconst = np.array([0.7, -0.4, 0.2]) if advect else None
    bv = None
    if advect:
        bv = inputs.vertex_field(nc, L, lambda x, y, z: np.stack([0 * x + bconst[0], 0 * x + bconst[1],
                                                                  0 * x + bconst[2]], -1))
    P = dg.Problem(*nc, *L, p, bc, K, b_vertex=bv, c_cell=c)
    Ah = transfer.p0_matrix(P.assemble(), P).toarray()
    M = _modified_fv(nc, L, p, bc, K, c=c, bconst=bconst)
    assert np.abs(Ah - M).max() < 1e-12 * np.abs(M).max()


def test_p0_transfer_and_neumann_nullspace():
    """P0: P injects cell constants (R P = N I, N dofs per cell) and, with
    pure Neumann conditions, b = 0 and c = 0, the constants span the kernel
    of P^T A P (zero row sums)."""
    P = small_problem(p=2, nc=(3, 2, 2), bc=(1,) * 6)
    P0 = transfer.p0_prolongation(P)
    assert np.abs((P0.T @ P0).toarray() - P.N * np.eye(P.ncell)).max() == 0.0
    Ah = transfer.p0_matrix(P.assemble(), P)
    assert np.abs(Ah @ np.ones(P.ncell)).max() < 1e-12 * abs(Ah).max()


def test_energy_norm_estimate_identity():
    """Strakos-Tichy: in PCG, ||e_k||_A^2 - ||e_{k+d}||_A^2 equals
    sum_{j=k}^{k+d-1} alpha_j (r_j, z_j); checked against the dense solution
    (brute force) for every k, together with the lower-bound property of the
    delay-4 estimate, and the stopping rule on the returned iterate."""
    P = small_problem(p=2, nc=(3, 3, 2), bc=(0,) * 6)
    A = P.assemble().tocsr()
    b = np.random.default_rng(3).normal(size=P.ndof)
    xs = np.linalg.solve(A.toarray(), b)
    dinv = 1.0 / A.diagonal()
    xs_list, terms = [], []
    x = np.zeros_like(b)
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = r @ z
    for _ in range(120):
        xs_list.append(x.copy())
        q = A @ p
        alpha = rz / (p @ q)
        terms.append(alpha * rz)
        x = x + alpha * p
        r = r - alpha * q
        z = dinv * r
        rzn = r @ z
        p = z + rzn / rz * p
        rz = rzn
    xs_list.append(x.copy())
    eA = [(xs - xk) @ (A @ (xs - xk)) for xk in xs_list]
    d = 4
    for k in range(0, 26):
        nu = sum(terms[k:k + d])
        assert abs((eA[k] - eA[k + d]) - nu) <= 1e-8 * eA[k]
        assert nu <= eA[k] * (1 + 1e-10)
    xe, k, hist = solvers.cg(lambda v: A @ v, b, lambda v: dinv * v, rtol=1e-6, stop="energy", delay=4)
    assert hist[-1] <= 1e-6 < hist[-2] and k + d < len(xs_list)
    assert np.sqrt(eA[k] / (xs @ (A @ xs))) == pytest.approx(hist[-1], rel=0.5)
    assert np.abs(xe - xs_list[k + d]).max() <= 1e-12 * np.abs(xs).max()
    assert np.sqrt((xs - xe) @ (A @ (xs - xe)) / (xs @ (A @ xs))) <= 1e-6


def test_outer_iterations_nearly_independent_of_inner_tolerance():
    """Sec. 4.2 observes that the outer CG iteration count hardly depends on
    the inner tolerance eps: with inner PCG to eps = 1e-2 .. 1e-8 the count
    stays within two of the count with exact (LU) block solves."""
    from paper_1805_11930_gb300 import inputs
    w = inputs.lognormal(4, 2)
    P = dg.Problem(*w["nc"], *w["L"], w["p"], w["bc"], w["K"])
    A = P.assemble()
    F = P.rhs(inputs.evaluate(w["f"], P.volume_points()))
    Pm = transfer.prolongation(P)
    am = amg.AggregationAMG(transfer.q1_matrix(P), P.nv)

    def outer_its(**kw):
        V = solvers.HybridVCycle(A, Pm, solvers.BlockJacobi(A, P.N, **kw), am.vcycle, omega=0.8)
        x, it, hist = solvers.cg(lambda v: A @ v, F, V, rtol=1e-8)
        assert np.linalg.norm(F - A @ x) <= 1e-8 * np.linalg.norm(F) * 1.0001
        return it

    exact = outer_its(inner="lu")
    for eps in (1e-2, 1e-4, 1e-8):
        assert abs(outer_its(inner="pcg", eps=eps) - exact) <= 2


def test_fgmres_with_ssor_at_peclet_2000():
    """Sec. 4.3's set-up for the strongly convection-dominated problem (grid
    Peclet number 2000, b = (1, 0.5, 0.3)): FGMRES preconditioned by two
    block-SSOR sweeps with inner GMRES and the Thomas preconditioner reaches
    1e-8 within the 10-25 iterations the paper reports for its grids (fewer
    on this 4^3 mesh), and its solution is the discrete one."""
    from paper_1805_11930_gb300 import inputs
    w = inputs.convection_pe(4, 3)
    P = dg.Problem(*w["nc"], *w["L"], w["p"], w["bc"], w["K"], b_vertex=w["b"], c_cell=w["c"])
    A = P.assemble()
    F = P.rhs(inputs.evaluate(w["f"], P.volume_points()))
    S = solvers.MulticolourBlockSOR(A, P.N, P.nc, symmetric=True, inner="gmres", eps=1e-2, restart=12,
                                    precond="tridiag", maxit=200)
    x, it, hist = solvers.fgmres(lambda v: A @ v, F, lambda r: S(r, np.zeros_like(r), 2, 1.0), restart=30, rtol=1e-8)
    assert it <= 25 and np.linalg.norm(F - A @ x) <= 1e-8 * np.linalg.norm(F) * 1.0001
    exact = spla.spsolve(A.tocsc(), F)
    assert np.abs(x - exact).max() < 1e-6 * np.abs(exact).max()


def test_flexible_cg_equals_cg_for_a_fixed_preconditioner():
    """With a fixed SPD preconditioner z_{k+1}.r_k = 0, so the Polak-Ribiere
    beta of flexible CG equals the Fletcher-Reeves beta of CG: the two give
    the same iterates up to rounding."""
    P = small_problem(p=2, nc=(3, 3, 2), bc=(0,) * 6)
    A = P.assemble().tocsr()
    b = np.random.default_rng(12).normal(size=P.ndof)
    dinv = 1.0 / A.diagonal()
    x1, k1, h1 = solvers.cg(lambda v: A @ v, b, lambda v: dinv * v, rtol=1e-10)
    x2, k2, h2 = solvers.cg(lambda v: A @ v, b, lambda v: dinv * v, rtol=1e-10, flexible=True)
    assert abs(k1 - k2) <= 1
    assert np.abs(x1 - x2).max() < 1e-8 * np.abs(x1).max()
    assert np.allclose(h1[:20], h2[:20], rtol=1e-6)
