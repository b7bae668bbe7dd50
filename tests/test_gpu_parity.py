"""GPU parity: every step of the hot path through the C ABI against the CPU
oracle, element by element, on seeded inputs.

Tolerances: FP64 operators 1e-12 relative (norm-wise), FP32 operators 1e-5
relative; quantities that pass through an iterative inner solve get a bound
derived from the solve tolerance (stated at each test).  Mesh sizes span
several thread blocks and leave ragged tails (one warp owns
max(1, 32/(p+1)^2) cells, a block 4 warps)."""
import numpy as np
import pytest

from oracle import amg, dg, solvers, transfer
from paper_1805_11930_gb300 import inputs

from gpu_helpers import custom, elem_errors, gpu_context, gpu_rhs, oracle_problem, oracle_rhs, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = {
    # (nc, p, bc, advect, react, kdim)
    "p1_dir": ((5, 3, 3), 1, [0] * 6, False, False, 1),
    "p2_mixed": ((5, 3, 3), 2, [0, 1, 0, 0, 1, 0], False, True, 3),
    "p3_adv": ((4, 3, 3), 3, [0, 0, 1, 0, 0, 1], True, False, 3),
    "p4_full": ((3, 3, 3), 4, [0, 1, 0, 1, 0, 0], True, True, 3),
    "p5_dir": ((3, 2, 2), 5, [0] * 6, False, False, 1),
    "p6_adv": ((2, 2, 2), 6, [1, 0, 0, 0, 0, 0], True, True, 3),
    "p7_adv": ((2, 2, 1), 7, [0, 1, 0, 0, 1, 0], True, True, 3),
    "p8_dir": ((2, 1, 1), 8, [0] * 6, False, True, 3),
}


def make_case(name, seed=11):
    nc, p, bc, adv, react, kdim = CASES[name]
    rng = np.random.default_rng(seed)
    ncell = int(np.prod(nc))
    L = (1.0, 0.75, 1.25)
    K = np.exp(rng.normal(size=(ncell, kdim) if kdim == 3 else ncell))
    b = None
    if adv:
        b = inputs.vertex_field(nc, L, lambda x, y, z: np.stack([1 - 2 * y, x - 0.3, 0.25 + 0.5 * z], -1))
    c = rng.uniform(0.1, 2.0, size=ncell) if react else None
    return custom(nc, L, p, bc, K, b=b, c=c, g=lambda x, y, z: x + y * z, j=lambda x, y, z: np.cos(x))


_cache = {}


def oracle_matrix(name):
    if name not in _cache:
        w = make_case(name)
        P = oracle_problem(w)
        _cache[name] = (w, P, P.assemble())
    return _cache[name]


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda").contiguous()


@pytest.mark.parametrize("name", list(CASES))
def test_apply_fp64_and_fp32(name):
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    u = inputs.random_dg_vector(P.ndof, seed=3)
    ref = A @ u
    v = torch.empty(P.ndof, dtype=torch.float64, device="cuda")
    ctx.apply(dev(u), v)
    assert rel_err(v.cpu().numpy(), ref) < 1e-12
    # element by element on the corner, edge and face cells, against ||A|| ||u||
    errs = elem_errors(v.cpu().numpy(), ref, A, u, w["nc"], P.N)
    assert max(errs.values()) < 1e-13, errs
    u32 = dev(u, torch.float32)
    v32 = torch.empty(P.ndof, dtype=torch.float32, device="cuda")
    ctx.apply(u32, v32)
    ref32 = A @ u32.cpu().double().numpy()
    assert rel_err(v32.cpu().numpy(), ref32) < 1e-5
    errs = elem_errors(v32.cpu().numpy(), ref32, A, u32.cpu().double().numpy(), w["nc"], P.N)
    assert max(errs.values()) < 2e-6, errs


@pytest.mark.parametrize("name", list(CASES))
def test_block_apply_and_diagonal(name):
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    N = P.N
    Ab = A.tobsr(blocksize=(N, N))
    D = np.zeros((P.ncell, N, N))
    for c in range(P.ncell):
        for k in range(Ab.indptr[c], Ab.indptr[c + 1]):
            if Ab.indices[k] == c:
                D[c] = Ab.data[k]
    u = inputs.random_dg_vector(P.ndof, seed=4)
    ref = np.einsum('cij,cj->ci', D, u.reshape(P.ncell, N)).reshape(-1)
    v = torch.empty(P.ndof, dtype=torch.float64, device="cuda")
    ctx.block_apply(dev(u), v)
    assert rel_err(v.cpu().numpy(), ref) < 1e-12
    errs = elem_errors(v.cpu().numpy(), ref, A, u, w["nc"], N)
    assert max(errs.values()) < 1e-13, errs
    dg_ = torch.empty(P.ndof, dtype=torch.float64, device="cuda")
    ctx.block_diagonal(dg_)
    refd = np.einsum('cii->ci', D).reshape(-1)
    assert rel_err(dg_.cpu().numpy(), refd) < 1e-12


@pytest.mark.parametrize("name", ["p1_dir", "p2_mixed", "p3_adv", "p5_dir"])
def test_restrict_prolong_and_coarse_matrix(name):
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    Pm = transfer.prolongation(P)
    r = inputs.random_dg_vector(P.ndof, seed=5)
    rh = torch.empty(P.nvert, dtype=torch.float64, device="cuda")
    ctx.restrict(dev(r), rh)
    assert rel_err(rh.cpu().numpy(), Pm.T @ r) < 1e-13
    uh = inputs.random_dg_vector(P.nvert, seed=6)
    u = inputs.random_dg_vector(P.ndof, seed=7)
    ud = dev(u)
    ctx.prolong_add(dev(uh), ud)
    assert rel_err(ud.cpu().numpy(), u + Pm @ uh) < 1e-13
    # A_hat (27-point stencil) against the oracle's P^T A P
    G = (Pm.T @ A @ Pm).toarray()
    st = ctx.coarse_matrix()
    Ah = np.zeros_like(G)
    Vx, Vy, Vz = P.nv
    for v in range(P.nvert):
        ix, iy, iz = v % Vx, (v // Vx) % Vy, v // (Vx * Vy)
        for k in range(27):
            jx, jy, jz = ix + k % 3 - 1, iy + (k // 3) % 3 - 1, iz + k // 9 - 1
            if 0 <= jx < Vx and 0 <= jy < Vy and 0 <= jz < Vz:
                Ah[v, jx + Vx * (jy + Vy * jz)] = st[v, k]
            else:
                assert st[v, k] == 0.0
    assert np.abs(Ah - G).max() < 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("nc", [(7, 6, 5), (9, 8, 8)])
def test_coarse_amg_cycle(nc):
    """Device AMG V-cycle equals the oracle's AMG (same aggregation,
    Galerkin levels, damped Jacobi with the Gershgorin weight 4/(3G),
    dense coarsest solve)."""
    rng = np.random.default_rng(8)
    w = custom(nc, (1, 1, 1), 2, [0] * 6, np.exp(rng.normal(size=int(np.prod(nc)))))
    P = oracle_problem(w)
    Ah = transfer.q1_matrix(P)
    am = amg.AggregationAMG(Ah, P.nv, coarse_size=512)
    ctx = gpu_context(w)
    r = rng.normal(size=P.nvert)
    out = torch.empty(P.nvert, dtype=torch.float64, device="cuda")
    ctx.coarse_cycle(dev(r), out)
    assert rel_err(out.cpu().numpy(), am.vcycle(r)) < 1e-11


@pytest.mark.parametrize("name", ["p1_dir", "p2_mixed", "p4_full", "p5_dir"])
def test_block_smooth_exact_blocks(name):
    """eps = 1e-13: each block solve is exact to ~kappa(D_T) 1e-13, so two
    sweeps match the oracle's dense-LU block-Jacobi to 1e-9."""
    w, P, A = oracle_matrix(name)
    if w["b"] is not None:
        pytest.skip("PCG needs symmetric blocks")
    ctx = gpu_context(w)
    f = inputs.random_dg_vector(P.ndof, seed=9)
    u0 = inputs.random_dg_vector(P.ndof, seed=10)
    S = solvers.BlockJacobi(A, P.N, inner="lu")
    ref = S(f, u0, 2, 0.8)
    u = dev(u0)
    ctx.block_smooth(dev(f), u, nsweep=2, omega=0.8, eps=1e-13, maxit=10 * P.N)
    assert rel_err(u.cpu().numpy(), ref) < 1e-9


@pytest.mark.parametrize("name", ["p2_mixed", "p5_dir"])
def test_block_smooth_inexact_matches_oracle_pcg(name):
    """eps = 1e-2: same PCG on the same block from the same start; cells whose
    iteration count equals the oracle's match to 1e-10, and every cell meets
    its stopping test."""
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    f = inputs.random_dg_vector(P.ndof, seed=12)
    u0 = inputs.random_dg_vector(P.ndof, seed=13)
    S = solvers.BlockJacobi(A, P.N, inner="pcg", eps=1e-2)
    ref = S(f, u0, 1, 1.0)
    its = torch.zeros(P.ncell, dtype=torch.int32, device="cuda")
    u = dev(u0)
    ctx.block_smooth(dev(f), u, nsweep=1, omega=1.0, eps=1e-2, inner_its=its)
    got = u.cpu().numpy()
    its = its.cpu().numpy()
    same = its == S.last_its
    assert same.mean() > 0.9
    N = P.N
    d = f - A @ u0
    for c in range(P.ncell):
        sl = slice(c * N, (c + 1) * N)
        delta = got[sl] - u0[sl]
        D = S.D[c]
        assert np.linalg.norm(d[sl] - D @ delta) <= 1e-2 * np.linalg.norm(d[sl]) * (1 + 1e-9)
        if same[c]:
            assert rel_err(got[sl] - u0[sl], ref[sl] - u0[sl]) < 1e-10


def test_vcycle_matches_oracle():
    """One V-cycle (Algorithm 1) with near-exact block solves against the
    oracle's V-cycle with dense-LU blocks and the same AMG."""
    w = make_case("p2_mixed")
    P = oracle_problem(w)
    A = P.assemble()
    Pm = transfer.prolongation(P)
    am = amg.AggregationAMG(transfer.q1_matrix(P), P.nv, coarse_size=512)
    V = solvers.HybridVCycle(A, Pm, solvers.BlockJacobi(A, P.N, inner="lu"), am.vcycle, omega=0.8)
    f = inputs.random_dg_vector(P.ndof, seed=14)
    ref = V(f)
    from paper_1805_11930_gb300 import dgmg
    ctx = gpu_context(w)
    u = torch.zeros(P.ndof, dtype=torch.float64, device="cuda")
    ctx.vcycle(dev(f), u, dgmg.default_opts(omega=0.8, eps_inner=1e-13, maxit_inner=10 * P.N))
    assert rel_err(u.cpu().numpy(), ref) < 1e-9


def test_rhs_assembly():
    w = make_case("p3_adv")
    P = oracle_problem(w)
    ref = oracle_rhs(P, w)
    ctx = gpu_context(w)
    rhs = gpu_rhs(ctx, w, torch)
    assert rel_err(rhs.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("krylov", ["cg", "fcg"])
def test_solve_poisson_c1(krylov):
    """Poisson 8^3, Q2 (13,824 dofs): CG + V-cycle to 1e-8 (true FP64
    residual); the solution matches the oracle's direct solve to the
    accuracy the residual allows, and the discretisation error is O(h^3)-small."""
    import scipy.sparse.linalg as spla
    from paper_1805_11930_gb300 import dgmg
    w = inputs.poisson_sine(8, 2)
    P = oracle_problem(w)
    A = P.assemble()
    F = oracle_rhs(P, w)
    x = spla.spsolve(A.tocsc(), F)
    ctx = gpu_context(w)
    f = gpu_rhs(ctx, w, torch)
    assert rel_err(f.cpu().numpy(), F) < 1e-13
    u = torch.zeros_like(f)
    kry = dgmg.KRYLOV_CG if krylov == "cg" else dgmg.KRYLOV_FCG
    st = ctx.solve(f, u, dgmg.default_opts(krylov=kry))
    assert st["converged"] == 1 and st["rel_residual"] <= 1e-8
    assert st["iterations"] < 40
    assert st["inner_mean"] < 6 and st["inner_max"] <= 27
    uh = u.cpu().numpy()
    assert rel_err(uh, x) < 1e-6
    assert P.l2_error(uh, w["exact"]) < 2e-3


def test_solve_mixed_precision_same_residual():
    """FP32 smoother and V-cycle, FP64 outer flexible CG: same 1e-8 FP64
    residual; solution within 1e-6 of the FP64 GPU solution."""
    from paper_1805_11930_gb300 import dgmg
    w = inputs.lognormal(8, 3)
    ctx = gpu_context(w)
    f = gpu_rhs(ctx, w, torch)
    u64 = torch.zeros_like(f)
    s64 = ctx.solve(f, u64, dgmg.default_opts())
    u32 = torch.zeros_like(f)
    s32 = ctx.solve(f, u32, dgmg.default_opts(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG))
    assert s64["converged"] and s32["converged"]
    assert s32["rel_residual"] <= 1e-8
    assert rel_err(u32.cpu().numpy(), u64.cpu().numpy()) < 1e-6


def test_solve_fgmres_matches_cg():
    """Right-preconditioned flexible GMRES(30) reaches the same 1e-8 residual
    and the same solution as CG on a symmetric problem."""
    from paper_1805_11930_gb300 import dgmg
    w = inputs.lognormal(6, 2)
    ctx = gpu_context(w)
    f = gpu_rhs(ctx, w, torch)
    u = torch.zeros_like(f)
    st = ctx.solve(f, u, dgmg.default_opts(krylov=dgmg.KRYLOV_FGMRES, restart=30))
    assert st["converged"] and st["rel_residual"] <= 1e-8
    u2 = torch.zeros_like(f)
    ctx.solve(f, u2, dgmg.default_opts())
    assert rel_err(u.cpu().numpy(), u2.cpu().numpy()) < 1e-6


def test_full_size_sampled_apply_lognormal_32():
    """32^3, Q4 (4.1M dofs), the launch configuration the benchmark times:
    sampled cells (corners, edges, faces, interior) against the oracle's block
    rows."""
    w = inputs.lognormal(32, 4)
    P = oracle_problem(w)
    ctx = gpu_context(w)
    u = inputs.random_dg_vector(P.ndof, seed=15)
    v = torch.empty(P.ndof, dtype=torch.float64, device="cuda")
    ctx.apply(dev(u), v)
    n = 32
    picks = [P.cell_index(0, 0, 0), P.cell_index(n - 1, n - 1, n - 1), P.cell_index(0, n - 1, 5),
             P.cell_index(17, 0, n - 1), P.cell_index(16, 16, 16), P.cell_index(3, 29, 11)]
    picks += list(np.random.default_rng(16).integers(0, P.ncell, size=6))
    ref = P.apply_rows(u, picks)
    got = v.cpu().numpy().reshape(P.ncell, P.N)[picks]
    assert rel_err(got, ref) < 1e-12


def test_errors_are_reported():
    from paper_1805_11930_gb300 import dgmg
    w = make_case("p2_mixed")
    ctx = dgmg.Context(0)
    with pytest.raises(dgmg.DgmgError):
        ctx.set_mesh(2, 2, 2, 1, 1, 1, 9, [0] * 6)          # p out of range
    ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
    with pytest.raises(dgmg.DgmgError):
        ctx.apply(torch.zeros(10, dtype=torch.float64, device="cuda"),
                  torch.zeros(10, dtype=torch.float64, device="cuda"))   # no coefficients yet
    with pytest.raises(dgmg.DgmgError):
        ctx.set_coefficients(-np.ones(np.prod(w["nc"])))                  # K <= 0
    ctx.set_mesh(1, 1, 1, 1, 1, 1, 2, [0] * 6)
    with pytest.raises(dgmg.DgmgError):
        ctx.set_coefficients(np.full(1, np.nan))                        # K not finite
    with pytest.raises(dgmg.DgmgError):
        ctx.set_mesh(16384, 16384, 16384, 1, 1, 1, 8, [0] * 6)          # 2^42 cells x 729 dofs: too large
    with pytest.raises(dgmg.DgmgError):
        ctx.set_mesh(0, 4, 4, 1, 1, 1, 2, [0] * 6)                     # empty mesh
    with pytest.raises(dgmg.DgmgError):
        ctx.set_mesh(2, 2, 2, 1, -1, 1, 2, [0] * 6)                    # negative length
    ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
    ctx.set_coefficients(w["K"])
    x = torch.zeros(ctx.sizes()["ndof"], dtype=torch.float64, device="cuda")
    with pytest.raises(dgmg.DgmgError):
        ctx.apply(x, x)                                                 # aliasing u and v
    with pytest.raises(dgmg.DgmgError):
        ctx.solve(x, torch.zeros_like(x), dgmg.default_opts(rtol=0.0))  # rtol must be > 0


@pytest.mark.parametrize("name", ["p3_adv", "p4_full", "p6_adv"])
def test_block_smooth_gmres_exact_blocks(name):
    """Non-symmetric blocks (b != 0), inner GMRES(12) with eps = 1e-13: two
    sweeps match the oracle's dense-LU block-Jacobi to 1e-9."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    f = inputs.random_dg_vector(P.ndof, seed=21)
    u0 = inputs.random_dg_vector(P.ndof, seed=22)
    ref = solvers.BlockJacobi(A, P.N, inner="lu")(f, u0, 2, 0.8)
    u = dev(u0)
    ctx.block_smooth(dev(f), u, nsweep=2, omega=0.8, eps=1e-13, maxit=20 * P.N, inner=dgmg.INNER_GMRES,
                     inner_restart=12)
    assert rel_err(u.cpu().numpy(), ref) < 1e-9


@pytest.mark.parametrize("name", ["p3_adv", "p6_adv"])
def test_block_smooth_gmres_inexact_matches_oracle(name):
    """eps = 1e-2: the same GMRES(12) as the oracle's block_gmres; cells with
    equal iteration counts agree to 1e-10 and every cell meets its stopping
    test (FP64 and, to 1e-4, FP32)."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    f = inputs.random_dg_vector(P.ndof, seed=23)
    u0 = inputs.random_dg_vector(P.ndof, seed=24)
    S = solvers.BlockJacobi(A, P.N, inner="gmres", eps=1e-2, restart=12, maxit=10 * P.N)
    ref = S(f, u0, 1, 1.0)
    its = torch.zeros(P.ncell, dtype=torch.int32, device="cuda")
    u = dev(u0)
    ctx.block_smooth(dev(f), u, nsweep=1, omega=1.0, eps=1e-2, maxit=10 * P.N, inner=dgmg.INNER_GMRES,
                     inner_restart=12, inner_its=its)
    got = u.cpu().numpy()
    same = its.cpu().numpy() == S.last_its
    assert same.mean() > 0.9
    N = P.N
    d = f - A @ u0
    for c in range(P.ncell):
        sl = slice(c * N, (c + 1) * N)
        assert np.linalg.norm(d[sl] - S.D[c] @ (got[sl] - u0[sl])) <= 1e-2 * np.linalg.norm(d[sl]) * (1 + 1e-9)
        if same[c]:
            assert rel_err(got[sl] - u0[sl], ref[sl] - u0[sl]) < 1e-10
    u32 = dev(u0, torch.float32)
    ctx.block_smooth(dev(f, torch.float32), u32, nsweep=1, omega=1.0, eps=1e-2, maxit=10 * P.N,
                     inner=dgmg.INNER_GMRES, inner_restart=12)
    g32 = u32.cpu().double().numpy()
    for c in range(P.ncell):
        sl = slice(c * N, (c + 1) * N)
        assert np.linalg.norm(d[sl] - S.D[c] @ (g32[sl] - u0[sl])) <= 1.0001e-2 * np.linalg.norm(d[sl]) + 1e-4 * np.linalg.norm(d[sl])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_solve_convection_fgmres(prec):
    """Upwind DG advection-diffusion at grid Peclet number 16 (kappa = h/16,
    rotating b), Q3 on 8^3: FGMRES(30) + V-cycle with inner GMRES block solves
    reaches 1e-8 (FP64 outer residual), the solution matches the oracle's
    direct solve, and the error against the exact polynomial solution is
    at the level the residual allows."""
    import scipy.sparse.linalg as spla
    from paper_1805_11930_gb300 import dgmg
    w = inputs.convection(8, 3, kappa=0.125 / 16)
    P = oracle_problem(w)
    A = P.assemble()
    F = oracle_rhs(P, w)
    x = spla.spsolve(A.tocsc(), F)
    ctx = gpu_context(w)
    f = gpu_rhs(ctx, w, torch)
    u = torch.zeros_like(f)
    st = ctx.solve(f, u, dgmg.default_opts(krylov=dgmg.KRYLOV_FGMRES, restart=30, inner=dgmg.INNER_GMRES,
                                           smoother_prec=dgmg.FP32 if prec == "fp32" else dgmg.FP64,
                                           maxit=400))
    assert st["converged"] and st["rel_residual"] <= 1e-8
    assert rel_err(u.cpu().numpy(), x) < 1e-6
    assert np.abs(u.cpu().numpy() - P.interpolate(w["exact"])).max() < 1e-6


@pytest.mark.parametrize("name,symmetric", [("p2_mixed", True), ("p2_mixed", False), ("p5_dir", True),
                                            ("p3_adv", True), ("p4_full", False)])
def test_block_sor_matches_oracle(name, symmetric):
    """Multicolour block-SOR / SSOR (colour = parity class of the cell
    indices), exact block solves (eps = 1e-13; PCG for symmetric blocks,
    GMRES(12) with b != 0): one sweep matches the oracle's colour-ordered
    block Gauss-Seidel with dense LU blocks to 1e-9."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    f = inputs.random_dg_vector(P.ndof, seed=41)
    u0 = inputs.random_dg_vector(P.ndof, seed=42)
    ref = solvers.MulticolourBlockSOR(A, P.N, P.nc, symmetric=symmetric, inner="lu")(f, u0, 1, 0.9)
    u = dev(u0)
    inner = dgmg.INNER_GMRES if w["b"] is not None else dgmg.INNER_PCG
    ctx.block_sor(dev(f), u, nsweep=1, omega=0.9, eps=1e-13, maxit=20 * P.N, inner=inner, symmetric=symmetric)
    assert rel_err(u.cpu().numpy(), ref) < 1e-9


def test_solve_convection_ssor_beats_jacobi():
    """Convection (grid Peclet 16), preconditioner = smoother only (no coarse
    space, as in the paper's convection runs): multicolour block-SSOR reaches
    1e-8 in fewer FGMRES iterations than block-Jacobi."""
    from paper_1805_11930_gb300 import dgmg
    w = inputs.convection(8, 3, kappa=0.125 / 16)
    ctx = gpu_context(w)
    f = gpu_rhs(ctx, w, torch)
    res = {}
    for sm in (dgmg.SMOOTHER_JACOBI, dgmg.SMOOTHER_SSOR):
        u = torch.zeros_like(f)
        st = ctx.solve(f, u, dgmg.default_opts(krylov=dgmg.KRYLOV_FGMRES, inner=dgmg.INNER_GMRES,
                                               coarse=dgmg.COARSE_NONE, smoother=sm, maxit=600))
        assert st["converged"] and st["rel_residual"] <= 1e-8
        res[sm] = st["iterations"]
    assert res[dgmg.SMOOTHER_SSOR] < res[dgmg.SMOOTHER_JACOBI]


@pytest.mark.parametrize("name", ["p1_dir", "p2_mixed", "p5_dir"])
def test_apply_df64(name):
    """Double-float arithmetic on FP64 vectors meets the FP64 tolerance
    (1e-12 relative) for the full operator and the block diagonal."""
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    u = inputs.random_dg_vector(P.ndof, seed=51)
    v = torch.empty(P.ndof, dtype=torch.float64, device="cuda")
    ctx.apply(dev(u), v, df64=True)
    assert rel_err(v.cpu().numpy(), A @ u) < 1e-12
    N = P.N
    Ab = A.tobsr(blocksize=(N, N))
    ref = np.zeros(P.ndof)
    for c in range(P.ncell):
        for k in range(Ab.indptr[c], Ab.indptr[c + 1]):
            if Ab.indices[k] == c:
                ref[c * N:(c + 1) * N] = Ab.data[k] @ u[c * N:(c + 1) * N]
    ctx.block_apply(dev(u), v, df64=True)
    assert rel_err(v.cpu().numpy(), ref) < 1e-12


def test_df64_rejects_unsupported_cases():
    """Double-float kernels exist for b = 0, p <= 6; other cases raise."""
    from paper_1805_11930_gb300 import dgmg
    for name in ("p3_adv", "p8_dir"):
        w, P, A = oracle_matrix(name)
        ctx = gpu_context(w)
        u = dev(np.zeros(P.ndof))
        v = dev(np.zeros(P.ndof))
        with pytest.raises(dgmg.DgmgError):
            ctx.apply(u, v, df64=True)


@pytest.mark.parametrize("name", ["p2_mixed", "p5_dir"])
def test_block_smooth_df64_exact_blocks(name):
    """Double-float inner solves to eps = 1e-12 reproduce the dense-LU
    block-Jacobi sweep to 1e-8 (the inner solve stops near the double-float
    rounding level times the block condition number)."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    f = inputs.random_dg_vector(P.ndof, seed=52)
    u0 = inputs.random_dg_vector(P.ndof, seed=53)
    ref = solvers.BlockJacobi(A, P.N, inner="lu")(f, u0, 1, 0.8)
    u = dev(u0)
    inner = dgmg.INNER_GMRES if w["b"] is not None else dgmg.INNER_PCG
    ctx.block_smooth(dev(f), u, nsweep=1, omega=0.8, eps=1e-12, maxit=10 * P.N, inner=inner, df64=True)
    assert rel_err(u.cpu().numpy(), ref) < 1e-8


def test_solve_df64_poisson_c1():
    """The whole solve in double-float (V-cycle and outer operator): same 1e-8
    residual, recomputed in native FP64, and the FP64 solution to 1e-7."""
    from paper_1805_11930_gb300 import dgmg
    w = inputs.poisson_sine(8, 2)
    ctx = gpu_context(w)
    f = gpu_rhs(ctx, w, torch)
    u64 = torch.zeros_like(f)
    ctx.solve(f, u64, dgmg.default_opts())
    u = torch.zeros_like(f)
    st = ctx.solve(f, u, dgmg.default_opts(smoother_prec=dgmg.DF64, apply_prec=dgmg.DF64, krylov=dgmg.KRYLOV_FCG))
    assert st["converged"] and st["rel_residual"] <= 1e-8
    assert rel_err(u.cpu().numpy(), u64.cpu().numpy()) < 1e-7


def test_graph_captured_preconditioner_same_result():
    """Capturing the V-cycle into a CUDA graph and replaying it gives the same
    iterates, bit for bit, as launching its kernels one by one."""
    from paper_1805_11930_gb300 import dgmg
    w = inputs.lognormal(6, 3)
    stream = torch.cuda.Stream()
    ctx = dgmg.Context(0, stream=stream)
    ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
    ctx.set_coefficients(w["K"])
    with torch.cuda.stream(stream):
        f = gpu_rhs(ctx, w, torch)
        out = []
        for graph in (0, 1):
            u = torch.zeros_like(f)
            st = ctx.solve(f, u, dgmg.default_opts(graph=graph, smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG))
            out.append((u.cpu().numpy(), st))
    stream.synchronize()
    (u0, s0), (u1, s1) = out
    assert s1["converged"] and s0["iterations"] == s1["iterations"]
    assert np.array_equal(u0, u1)
    assert s0["kernel_launches"] == s1["kernel_launches"] and s0["sweeps"] == s1["sweeps"]


def _layouts(prec, p, advection=False):
    """The work layouts that exist for a precision and order."""
    from paper_1805_11930_gb300 import dgmg
    out = [dgmg.LAYOUT_LINE, dgmg.LAYOUT_ELEMENT]
    if prec == dgmg.FP32 and p <= 4 and not advection:
        out.append(dgmg.LAYOUT_PLANE)
    return out


@pytest.mark.parametrize("prec_name,p,adv", [("FP64", 3, False), ("FP32", 3, False), ("FP32", 4, False),
                                              ("DF64", 3, False), ("FP64", 3, True), ("FP32", 4, True)])
def test_launch_shape_does_not_change_results(prec_name, p, adv):
    """In every work layout each warp owns whole cells, so the warps per block
    of the operator and smoother kernels change no bit of their outputs
    (ragged last block included: 5^3 cells do not fill any of the shapes or
    the plane layout's cells per warp evenly); with advection for the line
    and element forms and the inner GMRES smoother."""
    from paper_1805_11930_gb300 import dgmg
    prec = getattr(dgmg, prec_name)
    w = inputs.convection(5, p, kappa=1e-2) if adv else inputs.lognormal(5, p)
    inner = dgmg.INNER_GMRES if adv else dgmg.INNER_PCG
    ctx = gpu_context(w)
    dt = torch.float32 if prec == dgmg.FP32 else torch.float64
    df64 = prec == dgmg.DF64
    s = ctx.sizes()
    x = torch.tensor(inputs.random_dg_vector(s["ndof"], seed=11), device="cuda").to(dt)
    f = torch.tensor(inputs.random_dg_vector(s["ndof"], seed=12), device="cuda").to(dt)
    for lay in _layouts(prec, p, advection=adv):
        ctx.set_layout(prec, lay, lay)
        assert ctx.get_layout(prec) == (lay, lay)
        outs = []
        for wpb in (0, 1, 2, 8):
            ctx.set_launch_shape(prec, wpb, wpb)
            v = torch.empty_like(x)
            ctx.apply(x, v, df64=df64)
            u = x.clone()
            ctx.block_smooth(f, u, nsweep=2, omega=0.8, eps=1e-2, df64=df64, inner=inner)
            outs.append((v.cpu().numpy(), u.cpu().numpy()))
        for v, u in outs[1:]:
            assert np.array_equal(v, outs[0][0]) and np.array_equal(u, outs[0][1]), lay


@pytest.mark.parametrize("name", ["p1_dir", "p2_mixed", "p5_dir", "p8_dir"])
def test_every_layout_matches_the_oracle(name):
    """Each work layout of the b = 0 kernels (line, element, and the FP32
    plane layout for p <= 4) against the oracle: the operator and the block
    D_T to 1e-12 (FP64) and 1e-5 (FP32), norm-wise and element by element on
    the corner, edge and face cells; two FP64 block-Jacobi sweeps with
    eps = 1e-13 equal dense-LU block-Jacobi to 1e-9; one FP32 sweep with
    eps = 1e-2 meets every cell's stopping test (measured in FP64 against the
    exact defect, 1e-4 of slack for the FP32 defect) and agrees to 1e-4 with
    the oracle's block PCG where the iteration counts agree."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    N = P.N
    Ab = A.tobsr(blocksize=(N, N))
    D = np.zeros((P.ncell, N, N))
    for c in range(P.ncell):
        for k in range(Ab.indptr[c], Ab.indptr[c + 1]):
            if Ab.indices[k] == c:
                D[c] = Ab.data[k]
    u = inputs.random_dg_vector(P.ndof, seed=3)
    f = inputs.random_dg_vector(P.ndof, seed=9)
    u0 = inputs.random_dg_vector(P.ndof, seed=10)
    S = solvers.BlockJacobi(A, N, inner="lu")
    ref_sm = S(f, u0, 2, 0.8)
    ctx = gpu_context(w)
    for prec, dt, tol, etol in ((dgmg.FP64, torch.float64, 1e-12, 1e-13), (dgmg.FP32, torch.float32, 1e-5, 2e-6)):
        for lay in _layouts(prec, w["p"]):
            ctx.set_layout(prec, lay, lay)
            x = dev(u, dt)
            xd = x.double().cpu().numpy()
            for full in (True, False):
                v = torch.empty_like(x)
                (ctx.apply if full else ctx.block_apply)(x, v)
                ref = A @ xd if full else np.einsum('cij,cj->ci', D, xd.reshape(P.ncell, N)).reshape(-1)
                got = v.double().cpu().numpy()
                assert rel_err(got, ref) < tol, (prec, lay, full)
                errs = elem_errors(got, ref, A, xd, w["nc"], N)
                assert max(errs.values()) < etol, (prec, lay, full, errs)
            if prec == dgmg.FP64:
                us = dev(u0)
                ctx.block_smooth(dev(f), us, nsweep=2, omega=0.8, eps=1e-13, maxit=10 * N)
                assert rel_err(us.cpu().numpy(), ref_sm) < 1e-9, lay
            else:
                its = torch.zeros(P.ncell, dtype=torch.int32, device="cuda")
                us = dev(u0, dt)
                fs = dev(f, dt)
                ctx.block_smooth(fs, us, nsweep=1, omega=1.0, eps=1e-2, maxit=10 * N, inner_its=its)
                f32 = fs.double().cpu().numpy()
                u32 = dev(u0, dt).double().cpu().numpy()
                d = f32 - A @ u32
                got = us.double().cpu().numpy()
                its = its.cpu().numpy()
                same = 0
                for c in range(P.ncell):
                    sl = slice(c * N, (c + 1) * N)
                    delta = got[sl] - u32[sl]
                    assert np.linalg.norm(d[sl] - D[c] @ delta) <= (1.0001e-2 + 1e-4) * np.linalg.norm(d[sl]), lay
                    x_or, it_or = solvers.block_pcg(D[c], d[sl], np.diag(D[c]), 1e-2, 10 * N)
                    if it_or == its[c]:
                        same += 1
                        assert rel_err(delta, x_or) < 1e-4, (lay, c)
                assert same >= 0.8 * P.ncell, lay
        ctx.set_layout(prec, dgmg.LAYOUT_AUTO, dgmg.LAYOUT_AUTO)


@pytest.mark.parametrize("name", ["p3_adv", "p4_full", "p6_adv", "p7_adv"])
def test_advection_layouts_match_the_oracle(name):
    """With advection the line layout (one thread per pencil) and the element
    layout (the Gauss-point form: interpolate, differentiate, weight, project
    back) both give the oracle's operator and block D_T: FP64 to 1e-12, FP32
    to 1e-5, element by element on the
    corner, edge and face cells; in FP64 each form's block-Jacobi sweeps with
    inner GMRES(12), eps = 1e-13, equal dense-LU block-Jacobi to 1e-9 (up to
    p = 6; at p = 7 the element form's faces run one direction at a time)."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    N = P.N
    Ab = A.tobsr(blocksize=(N, N))
    D = np.zeros((P.ncell, N, N))
    for c in range(P.ncell):
        for k in range(Ab.indptr[c], Ab.indptr[c + 1]):
            if Ab.indices[k] == c:
                D[c] = Ab.data[k]
    u = inputs.random_dg_vector(P.ndof, seed=31)
    f = inputs.random_dg_vector(P.ndof, seed=32)
    u0 = inputs.random_dg_vector(P.ndof, seed=33)
    ref_sm = solvers.BlockJacobi(A, N, inner="lu")(f, u0, 2, 0.8) if w["p"] <= 6 else None
    ctx = gpu_context(w)
    cases = ((dgmg.FP64, torch.float64, 1e-12, 1e-13), (dgmg.FP32, torch.float32, 1e-5, 2e-6))
    for prec, dt, tol, etol in cases:
        for lay in (dgmg.LAYOUT_LINE, dgmg.LAYOUT_ELEMENT):
            ctx.set_layout(prec, lay, lay)
            x = dev(u, dt)
            xd = x.double().cpu().numpy()
            for full in (True, False):
                v = torch.empty_like(x)
                (ctx.apply if full else ctx.block_apply)(x, v)
                ref = A @ xd if full else np.einsum('cij,cj->ci', D, xd.reshape(P.ncell, N)).reshape(-1)
                got = v.double().cpu().numpy()
                assert rel_err(got, ref) < tol, (prec, lay, full)
                errs = elem_errors(got, ref, A, xd, w["nc"], N)
                assert max(errs.values()) < etol, (prec, lay, full, errs)
            if prec == dgmg.FP64 and w["p"] <= 6:
                us = dev(u0)
                ctx.block_smooth(dev(f), us, nsweep=2, omega=0.8, eps=1e-13, maxit=20 * N,
                                 inner=dgmg.INNER_GMRES, inner_restart=12)
                assert rel_err(us.cpu().numpy(), ref_sm) < 1e-9, lay
        ctx.set_layout(prec, dgmg.LAYOUT_AUTO, dgmg.LAYOUT_AUTO)
    with pytest.raises(dgmg.DgmgError):
        ctx.set_layout(dgmg.FP32, dgmg.LAYOUT_PLANE, dgmg.LAYOUT_PLANE)   # no plane form with advection


def test_autotune_choices_and_bitwise_solve():
    """dgmg_autotune picks a layout and a shape for each kernel (warps per
    block from {1, 2, 4, 8}), rejects bad arguments, and a solve with the
    tuned layouts equals, bit for bit, the solve with the same layouts at the
    default shapes; the tuned solve converges."""
    from paper_1805_11930_gb300 import dgmg
    w = inputs.lognormal(8, 4)
    ctx = gpu_context(w)
    f = gpu_rhs(ctx, w, torch)
    opts = dgmg.default_opts(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG)
    for prec in (dgmg.FP64, dgmg.FP32, dgmg.DF64):
        a, s = ctx.autotune(prec, reps=2)
        assert a in (1, 2, 4, 8) and s in (1, 2, 4, 8)
        la, ls = ctx.get_layout(prec)
        assert la in _layouts(prec, 4) and ls in _layouts(prec, 4)
    u1 = torch.zeros_like(f)
    s1 = ctx.solve(f, u1, opts)
    assert s1["converged"]
    for prec in (dgmg.FP64, dgmg.FP32, dgmg.DF64):
        ctx.set_launch_shape(prec, 0, 0)
    u0 = torch.zeros_like(f)
    s0 = ctx.solve(f, u0, opts)
    assert s0["iterations"] == s1["iterations"] and np.array_equal(u0.cpu().numpy(), u1.cpu().numpy())
    with pytest.raises(dgmg.DgmgError):
        ctx.set_launch_shape(dgmg.FP64, 3, 0)
    with pytest.raises(dgmg.DgmgError):
        ctx.set_launch_shape(7, 4, 4)
    with pytest.raises(dgmg.DgmgError):
        ctx.set_layout(dgmg.FP64, dgmg.LAYOUT_PLANE, 0)
    with pytest.raises(dgmg.DgmgError):
        ctx.set_layout(dgmg.FP32, 9, 0)


# ------------------------------------------------------------- stored inverses
@pytest.mark.parametrize("name", ["p1_dir", "p2_mixed", "p3_adv", "p4_full", "p5_dir", "p6_adv", "p8_dir"])
def test_block_inverse_matches_oracle_blocks(name):
    """dgmg_block_inverse: every stored block times the oracle's assembled
    diagonal block D_T is the identity up to the rounding of the stored
    double-float pairs (64 units of 2^-48 times max |D_T^-1| |D_T|, about
    1e-13 here), and the FP32 copy is the same inverse rounded (1e-6
    relative per block); p >= 5 takes the panel-blocked elimination in
    global memory."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    nb = P.N
    out = torch.empty(P.ncell * nb * nb, dtype=torch.float64, device="cuda")
    ctx.block_inverse(dgmg.FP64, out)
    inv = out.cpu().numpy().reshape(P.ncell, nb, nb).transpose(0, 2, 1)    # column-major per block
    D = solvers.BlockJacobi(A, nb, inner="lu").D
    eye = np.eye(nb)
    for c in range(P.ncell):
        bound = 64 * 2.0 ** -48 * (np.abs(inv[c]) @ np.abs(D[c])).max()
        assert np.abs(inv[c] @ D[c] - eye).max() < bound
    out32 = torch.empty(P.ncell * nb * nb, dtype=torch.float32, device="cuda")
    ctx.block_inverse(dgmg.FP32, out32)
    inv32 = out32.cpu().numpy().astype(np.float64).reshape(P.ncell, nb, nb).transpose(0, 2, 1)
    for c in range(P.ncell):
        assert rel_err(inv32[c], inv[c]) < 1e-6


@pytest.mark.parametrize("name", ["p1_dir", "p2_mixed", "p3_adv", "p4_full", "p5_dir", "p6_adv", "p8_dir"])
def test_block_smooth_direct_matches_exact_block_jacobi(name):
    """inner = DIRECT (stored inverses): two block-Jacobi sweeps equal the
    oracle's dense-LU block-Jacobi to 1e-12 in FP64 and double-float (b = 0)
    and 1e-5 in FP32, every cell reporting 0 inner iterations."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    f = inputs.random_dg_vector(P.ndof, seed=31)
    u0 = inputs.random_dg_vector(P.ndof, seed=32)
    ref = solvers.BlockJacobi(A, P.N, inner="lu")(f, u0, 2, 0.8)
    its = torch.full((P.ncell,), 7, dtype=torch.int32, device="cuda")
    u = dev(u0)
    ctx.block_smooth(dev(f), u, nsweep=2, omega=0.8, inner=dgmg.INNER_DIRECT, inner_its=its)
    assert rel_err(u.cpu().numpy(), ref) < 1e-12
    assert int(its.abs().max()) == 0
    u32 = dev(u0).float()
    ctx.block_smooth(dev(f).float(), u32, nsweep=2, omega=0.8, inner=dgmg.INNER_DIRECT)
    assert rel_err(u32.double().cpu().numpy(), ref) < 1e-5
    if w["b"] is None and w["p"] <= 6:   # double-float defect and product (diffusion, p <= 6)
        udf = dev(u0)
        ctx.block_smooth(dev(f), udf, nsweep=2, omega=0.8, inner=dgmg.INNER_DIRECT, df64=True)
        assert rel_err(udf.cpu().numpy(), ref) < 1e-12


@pytest.mark.parametrize("name", ["p2_mixed", "p3_adv"])
def test_block_ssor_direct_matches_oracle(name):
    """Multicolour block-SSOR with exact block solves by the stored inverses
    against the oracle's colour-ordered SSOR with dense-LU blocks."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    f = inputs.random_dg_vector(P.ndof, seed=33)
    u0 = inputs.random_dg_vector(P.ndof, seed=34)
    ref = solvers.MulticolourBlockSOR(A, P.N, P.nc, symmetric=True, inner="lu")(f, u0, 1, 1.1)
    u = dev(u0)
    ctx.block_sor(dev(f), u, nsweep=1, omega=1.1, inner=dgmg.INNER_DIRECT, symmetric=True)
    assert rel_err(u.cpu().numpy(), ref) < 1e-12


def test_solve_direct_blocks_c1_and_rejections():
    """CG with a V-cycle whose smoother uses the stored inverses reaches 1e-8
    on the Poisson workload in no more iterations than inner PCG, also in
    FP32 and double-float; DF64 rejects inner GMRES; at p = 6 (blocks built
    by the panel-blocked elimination) the stored-inverse solve reaches 1e-8
    with no more iterations than inner PCG."""
    from paper_1805_11930_gb300 import dgmg
    w = inputs.poisson_sine(8, 2)
    ctx = gpu_context(w)
    f = gpu_rhs(ctx, w, torch)
    u0 = torch.zeros_like(f)
    s_pcg = ctx.solve(f, u0, dgmg.default_opts())
    u1 = torch.zeros_like(f)
    s_dir = ctx.solve(f, u1, dgmg.default_opts(inner=dgmg.INNER_DIRECT))
    assert s_dir["converged"] and s_dir["rel_residual"] <= 1e-8
    assert s_dir["iterations"] <= s_pcg["iterations"]
    assert rel_err(u1.cpu().numpy(), u0.cpu().numpy()) < 1e-6
    u2 = torch.zeros_like(f)
    s32 = ctx.solve(f, u2, dgmg.default_opts(inner=dgmg.INNER_DIRECT, smoother_prec=dgmg.FP32,
                                             krylov=dgmg.KRYLOV_FCG))
    assert s32["converged"] and s32["rel_residual"] <= 1e-8
    udf = torch.zeros_like(f)
    sdf = ctx.solve(f, udf, dgmg.default_opts(inner=dgmg.INNER_DIRECT, smoother_prec=dgmg.DF64,
                                              krylov=dgmg.KRYLOV_FCG))
    assert sdf["converged"] and sdf["rel_residual"] <= 1e-8
    with pytest.raises(dgmg.DgmgError):
        ctx.solve(f, torch.zeros_like(f), dgmg.default_opts(inner=dgmg.INNER_GMRES, smoother_prec=dgmg.DF64))
    w6 = inputs.lognormal(4, 6)
    ctx6 = gpu_context(w6)
    f6 = gpu_rhs(ctx6, w6, torch)
    s6p = ctx6.solve(f6, torch.zeros_like(f6), dgmg.default_opts())
    u6 = torch.zeros_like(f6)
    s6d = ctx6.solve(f6, u6, dgmg.default_opts(inner=dgmg.INNER_DIRECT))
    assert s6d["converged"] and s6d["rel_residual"] <= 1e-8 and s6d["iterations"] <= s6p["iterations"]


# ------------------------------------------------------------- tridiagonal inner preconditioner
@pytest.mark.parametrize("name", ["p3_adv", "p4_full"])
def test_block_smooth_gmres_tridiag_exact_blocks(name):
    """GMRES(12) preconditioned by the tridiagonal part of D_T (Thomas), eps =
    1e-13: two sweeps equal the oracle's dense-LU block-Jacobi to 1e-9."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    f = inputs.random_dg_vector(P.ndof, seed=41)
    u0 = inputs.random_dg_vector(P.ndof, seed=42)
    ref = solvers.BlockJacobi(A, P.N, inner="lu")(f, u0, 2, 0.8)
    u = dev(u0)
    ctx.block_smooth(dev(f), u, nsweep=2, omega=0.8, eps=1e-13, maxit=20 * P.N, inner=dgmg.INNER_GMRES_TRIDIAG,
                     inner_restart=12)
    assert rel_err(u.cpu().numpy(), ref) < 1e-9


@pytest.mark.parametrize("name", ["p2_mixed", "p3_adv"])
def test_block_smooth_gmres_tridiag_matches_oracle(name):
    """eps = 1e-2: the oracle's GMRES(12) with the Thomas preconditioner; cells
    with equal iteration counts agree to 1e-10, every cell meets its stopping
    test, in FP64 and (stopping test to 1e-4) in FP32."""
    from paper_1805_11930_gb300 import dgmg
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    f = inputs.random_dg_vector(P.ndof, seed=43)
    u0 = inputs.random_dg_vector(P.ndof, seed=44)
    S = solvers.BlockJacobi(A, P.N, inner="gmres", eps=1e-2, restart=12, maxit=10 * P.N, precond="tridiag")
    ref = S(f, u0, 1, 1.0)
    N = P.N
    d = f - A @ u0
    for dt, tol in ((torch.float64, 1e-2 * (1 + 1e-9)), (torch.float32, 1.0001e-2 + 1e-4)):
        its = torch.zeros(P.ncell, dtype=torch.int32, device="cuda")
        u = dev(u0).to(dt)
        ctx.block_smooth(dev(f).to(dt), u, nsweep=1, omega=1.0, eps=1e-2, maxit=10 * N,
                         inner=dgmg.INNER_GMRES_TRIDIAG, inner_restart=12, inner_its=its)
        got = u.double().cpu().numpy()
        its = its.cpu().numpy()
        same = its == S.last_its
        assert same.mean() > 0.9
        for c in range(P.ncell):
            sl = slice(c * N, (c + 1) * N)
            delta = got[sl] - u0[sl]
            assert np.linalg.norm(d[sl] - S.D[c] @ delta) <= tol * np.linalg.norm(d[sl])
            if dt == torch.float64 and same[c]:
                assert rel_err(delta, ref[sl] - u0[sl]) < 1e-10


def test_tridiag_preconditioner_convection_dominated_gpu():
    """Grid Peclet number 2000, b = (1, 0, 0), p = 3: with diag(D_T) the inner
    GMRES runs into its 200-iteration cap in most cells; with the Thomas
    preconditioner every cell stops within 30 iterations."""
    from paper_1805_11930_gb300 import dgmg
    nc, L = (4, 4, 4), (1.0, 1.0, 1.0)
    b = inputs.vertex_field(nc, L, lambda x, y, z: np.stack([np.ones_like(x), 0 * x, 0 * x], -1))
    w = custom(nc, L, 3, [0] * 6, np.full(64, 0.25 / 2000), b=b)
    ctx = gpu_context(w)
    nd = ctx.sizes()["ndof"]
    f = dev(inputs.random_dg_vector(nd, seed=45))
    res = {}
    for inner in (dgmg.INNER_GMRES, dgmg.INNER_GMRES_TRIDIAG):
        its = torch.zeros(64, dtype=torch.int32, device="cuda")
        u = torch.zeros(nd, dtype=torch.float64, device="cuda")
        ctx.block_smooth(f, u, nsweep=1, omega=1.0, eps=1e-2, maxit=200, inner=inner, inner_restart=12,
                         inner_its=its)
        res[inner] = its.cpu().numpy()
    assert (res[dgmg.INNER_GMRES] == 200).mean() > 0.5
    assert res[dgmg.INNER_GMRES_TRIDIAG].max() <= 30


# ------------------------------------------------------------- P0 coarse space
def _stencil_dense(st, dims):
    Vx, Vy, Vz = dims
    n = Vx * Vy * Vz
    out = np.zeros((n, n))
    for v in range(n):
        ix, iy, iz = v % Vx, (v // Vx) % Vy, v // (Vx * Vy)
        for k in range(27):
            jx, jy, jz = ix + k % 3 - 1, iy + (k // 3) % 3 - 1, iz + k // 9 - 1
            if 0 <= jx < Vx and 0 <= jy < Vy and 0 <= jz < Vz:
                out[v, jx + Vx * (jy + Vy * jz)] = st[v, k]
            else:
                assert st[v, k] == 0.0
    return out


@pytest.mark.parametrize("name", ["p1_dir", "p2_mixed", "p3_adv", "p6_adv"])
def test_p0_transfer_and_coarse_matrix(name):
    """P0 restriction (cell sums) and prolongation against P^T r and u + P u_hat
    (FP64 1e-14, FP32 1e-6), and the re-discretised P0 A_hat against the
    oracle's Galerkin product P^T A P to 1e-12."""
    w, P, A = oracle_matrix(name)
    ctx = gpu_context(w)
    P0 = transfer.p0_prolongation(P)
    r = inputs.random_dg_vector(P.ndof, seed=51)
    rh = torch.empty(P.ncell, dtype=torch.float64, device="cuda")
    ctx.restrict_p0(dev(r), rh)
    assert rel_err(rh.cpu().numpy(), P0.T @ r) < 1e-14
    ctx.restrict_p0(dev(r).float(), rh)
    assert rel_err(rh.cpu().numpy(), P0.T @ r) < 1e-6
    uh = inputs.random_dg_vector(P.ncell, seed=52)
    u = inputs.random_dg_vector(P.ndof, seed=53)
    ud = dev(u)
    ctx.prolong_add_p0(dev(uh), ud)
    assert rel_err(ud.cpu().numpy(), u + P0 @ uh) < 1e-14
    G = transfer.p0_matrix(A, P).toarray()
    Ah = _stencil_dense(ctx.coarse_matrix_p0(), P.nc)
    assert np.abs(Ah - G).max() < 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("nc", [(6, 5, 4), (12, 10, 9)])
def test_p0_amg_cycle(nc):
    """Device AMG V-cycle on the P0 matrix equals the oracle's AMG on
    P^T A P with the cell grid as its structured grid."""
    rng = np.random.default_rng(9)
    w = custom(nc, (1, 1, 1), 2, [0] * 6, np.exp(rng.normal(size=int(np.prod(nc)))))
    P = oracle_problem(w)
    am = amg.AggregationAMG(transfer.p0_matrix(P.assemble(), P), P.nc, coarse_size=512)
    ctx = gpu_context(w)
    r = rng.normal(size=P.ncell)
    out = torch.empty(P.ncell, dtype=torch.float64, device="cuda")
    ctx.coarse_cycle_p0(dev(r), out)
    assert rel_err(out.cpu().numpy(), am.vcycle(r)) < 1e-11


def test_vcycle_p0_matches_oracle_and_solve():
    """One V-cycle with the P0 coarse space (near-exact blocks) against the
    oracle's Algorithm 1 with P0, dense-LU blocks and the same AMG; then CG
    with that V-cycle reaches 1e-8 on the Poisson workload, FP64 and mixed."""
    from paper_1805_11930_gb300 import dgmg
    w = make_case("p2_mixed")
    P = oracle_problem(w)
    A = P.assemble()
    P0 = transfer.p0_prolongation(P)
    am = amg.AggregationAMG(transfer.p0_matrix(A, P), P.nc, coarse_size=512)
    V = solvers.HybridVCycle(A, P0, solvers.BlockJacobi(A, P.N, inner="lu"), am.vcycle, omega=0.8)
    f = inputs.random_dg_vector(P.ndof, seed=54)
    ref = V(f)
    ctx = gpu_context(w)
    u = torch.zeros(P.ndof, dtype=torch.float64, device="cuda")
    ctx.vcycle(dev(f), u, dgmg.default_opts(omega=0.8, eps_inner=1e-13, maxit_inner=10 * P.N,
                                            coarse=dgmg.COARSE_P0))
    assert rel_err(u.cpu().numpy(), ref) < 1e-9
    w1 = inputs.poisson_sine(8, 2)
    c1 = gpu_context(w1)
    f1 = gpu_rhs(c1, w1, torch)
    for prec, kry in ((dgmg.FP64, dgmg.KRYLOV_CG), (dgmg.FP32, dgmg.KRYLOV_FCG)):
        u1 = torch.zeros_like(f1)
        st = c1.solve(f1, u1, dgmg.default_opts(coarse=dgmg.COARSE_P0, smoother_prec=prec, krylov=kry))
        assert st["converged"] and st["rel_residual"] <= 1e-8


def test_solve_energy_norm_stopping():
    """stop = ENERGY (Strakos-Tichy estimate, error bandwidth 4, Sec. 4.4):
    the solve stops once the estimate is <= rtol, reports k and k + 4
    iterations, and the returned iterate's true relative energy error against
    the oracle's direct solution is below rtol; FGMRES rejects the rule."""
    import scipy.sparse.linalg as spla
    from paper_1805_11930_gb300 import dgmg
    rng = np.random.default_rng(61)
    w = custom((4, 4, 3), (1.0, 1.0, 0.75), 2, [0] * 6, np.exp(2.0 * rng.normal(size=48)))
    P = oracle_problem(w)
    A = P.assemble().tocsc()
    F = oracle_rhs(P, w)
    xs = spla.spsolve(A, F)
    ctx = gpu_context(w)
    f = dev(F)
    u = torch.zeros_like(f)
    st = ctx.solve(f, u, dgmg.default_opts(stop=dgmg.STOP_ENERGY, rtol=1e-6))
    assert st["converged"] and st["energy_estimate"] <= 1e-6
    assert st["iterations_run"] == st["iterations"] + 4
    e = u.cpu().numpy() - xs
    assert np.sqrt(e @ (A @ e) / (xs @ (A @ xs))) <= 1e-6
    with pytest.raises(dgmg.DgmgError):
        ctx.solve(f, torch.zeros_like(f), dgmg.default_opts(stop=dgmg.STOP_ENERGY, krylov=dgmg.KRYLOV_FGMRES))


# ------------------------------------------------------------- full sizes, sampled cells
def _picks(P, seed, extra=8):
    nx, ny, nz = P.nc
    picks = [P.cell_index(0, 0, 0), P.cell_index(nx - 1, ny - 1, nz - 1), P.cell_index(0, ny - 1, nz // 2),
             P.cell_index(nx // 2, 0, nz - 1), P.cell_index(nx // 2, ny // 2, nz // 2), P.cell_index(nx - 1, 1, 0)]
    return picks + [int(c) for c in np.random.default_rng(seed).integers(0, P.ncell, size=extra)]


@pytest.mark.parametrize("which", ["convection_64_q3", "reservoir_q2"])
def test_full_size_sampled_apply(which):
    """The full convection (64^3 Q3, 16.8 M dofs, advection) and reservoir
    (60x220x85 Q2, 30.3 M dofs, anisotropic K, mixed boundary) operators on
    sampled cells (corners, edges, faces, interior, random) against the
    oracle's block rows: FP64 1e-12, FP32 1e-5."""
    w = inputs.convection(64, 3) if which.startswith("convection") else inputs.reservoir()
    P = oracle_problem(w)
    ctx = gpu_context(w)
    u = inputs.random_dg_vector(P.ndof, seed=71)
    picks = _picks(P, 72)
    ref = P.apply_rows(u, picks)
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 1e-5)):
        x = dev(u).to(dt)
        v = torch.empty_like(x)
        ctx.apply(x, v)
        got = v.double().cpu().numpy().reshape(P.ncell, P.N)[picks]
        assert rel_err(got, ref) < tol, dt
        del x, v


def test_full_size_sampled_smoothers_lognormal_32():
    """The benchmark's mesh (32^3 Q4) and autotuned launch shapes: one sweep
    with stored inverses equals, on sampled cells, u_T + omega D_T^-1 d_T from
    the oracle's block row and dense solve (1e-12); one inner-PCG sweep
    (eps = 1e-2) equals the oracle's block PCG from the same defect on every
    sampled cell with the same iteration count (1e-10) and meets the stopping
    test on all of them."""
    from paper_1805_11930_gb300 import dgmg
    w = inputs.lognormal(32, 4)
    P = oracle_problem(w)
    ctx = gpu_context(w)
    ctx.autotune(dgmg.FP64)
    N = P.N
    f = inputs.random_dg_vector(P.ndof, seed=73)
    u0 = inputs.random_dg_vector(P.ndof, seed=74)
    picks = _picks(P, 75)
    d = f.reshape(P.ncell, N)[picks] - P.apply_rows(u0, picks)
    D = [P.diagonal_block(c) for c in picks]
    u = dev(u0)
    ctx.block_smooth(dev(f), u, nsweep=1, omega=0.8, inner=dgmg.INNER_DIRECT)
    got = u.cpu().numpy().reshape(P.ncell, N)[picks]
    ref = u0.reshape(P.ncell, N)[picks] + 0.8 * np.stack([np.linalg.solve(Dc, dc) for Dc, dc in zip(D, d)])
    assert rel_err(got, ref) < 1e-12
    its = torch.zeros(P.ncell, dtype=torch.int32, device="cuda")
    u = dev(u0)
    ctx.block_smooth(dev(f), u, nsweep=1, omega=1.0, eps=1e-2, inner_its=its)
    got = u.cpu().numpy().reshape(P.ncell, N)[picks] - u0.reshape(P.ncell, N)[picks]
    its = its.cpu().numpy()[picks]
    same = 0
    for r, (Dc, dc) in enumerate(zip(D, d)):
        assert np.linalg.norm(dc - Dc @ got[r]) <= 1e-2 * np.linalg.norm(dc) * (1 + 1e-9)
        x, it = solvers.block_pcg(Dc, dc, np.diag(Dc), 1e-2, N)
        if it == its[r]:
            same += 1
            assert rel_err(got[r], x) < 1e-10
    assert same >= len(picks) - 2


# ------------------------------------------------------------- K(x), c(x) varying inside cells
def _vark_problem(nc, L, p, bc, gamma):
    return dg.Problem(*nc, *L, p, bc, np.ones(int(np.prod(nc))), K_fn=inputs.vark_tensor,
                      c_fn=lambda x: inputs.vark_reaction(x, gamma))


def _vark_context(nc, L, p, bc, gamma):
    from paper_1805_11930_gb300 import dgmg
    ctx = dgmg.Context(0)
    ctx.set_mesh(*nc, *L, p, bc)
    ctx.set_variable_coefficients(inputs.VARK_BASIS, inputs.VARK_P0, inputs.VARK_P2, gamma)
    return ctx


@pytest.mark.parametrize("case", [((3, 2, 2), 2, [0, 1, 0, 0, 1, 0]), ((2, 3, 2), 3, [0] * 6),
                                  ((2, 2, 2), 4, [1, 0, 0, 1, 0, 0]), ((3, 2, 1), 6, [0, 0, 1, 0, 0, 0])])
def test_variable_operator_and_rhs_match_oracle(case):
    """The operator with K(x), c(x) evaluated at every quadrature point (the
    paper's rotated quadratic K, a visible reaction gamma = 0.5) against the
    oracle's assembled matrix (1e-12), and the right-hand side with K(x) in
    the Dirichlet terms (1e-13)."""
    nc, p, bc = case
    L = (1.0, 0.8, 1.2)
    P = _vark_problem(nc, L, p, bc, 0.5)
    A = P.assemble()
    ctx = _vark_context(nc, L, p, bc, 0.5)
    u = inputs.random_dg_vector(P.ndof, seed=81)
    v = torch.empty(P.ndof, dtype=torch.float64, device="cuda")
    ctx.apply(dev(u), v)
    assert rel_err(v.cpu().numpy(), A @ u) < 1e-12
    g = lambda x, y, z: np.exp(-((x - 0.2) ** 2 + (y - 0.5) ** 2) / 0.1) + z   # noqa: E731
    j = lambda x, y, z: np.cos(x + 2 * y) * z                                   # noqa: E731
    f = lambda x, y, z: np.sin(3 * x) * y + z * z                              # noqa: E731
    w = custom(nc, L, p, bc, np.ones(int(np.prod(nc))), f=f, g=g, j=j)
    ref = oracle_rhs(P, w)
    rhs = gpu_rhs(ctx, w, torch)
    assert rel_err(rhs.cpu().numpy(), ref) < 1e-13


def test_variable_solve_paper_setup():
    """The inhomogeneous test of Sec. 4.2 (8^3, Q3, Neumann on x = 1, Gaussian
    data, gamma = 1e-8): CG with the cell-centre V-cycle reaches 1e-8 in the
    exact operator's residual, in FP64 and mixed precision and with the
    energy-norm rule, and matches the oracle's direct solve to 1e-6."""
    import scipy.sparse.linalg as spla
    from paper_1805_11930_gb300 import dgmg
    w = inputs.variable_k(8, 3)
    P = dg.Problem(*w["nc"], *w["L"], w["p"], w["bc"], w["K"], K_fn=w["K_fn"], c_fn=w["c_fn"])
    xs = spla.spsolve(P.assemble().tocsc(), oracle_rhs(P, w))
    ctx = dgmg.Context(0)
    ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
    vk = w["vark"]
    ctx.set_variable_coefficients(vk["basis"], vk["p0"], vk["p2"], vk["gamma"])
    f = gpu_rhs(ctx, w, torch)
    for opts in (dgmg.default_opts(), dgmg.default_opts(smoother_prec=dgmg.FP32, krylov=dgmg.KRYLOV_FCG)):
        u = torch.zeros_like(f)
        st = ctx.solve(f, u, opts)
        assert st["converged"] and st["rel_residual"] <= 1e-8
        assert rel_err(u.cpu().numpy(), xs) < 1e-6
    u = torch.zeros_like(f)
    st = ctx.solve(f, u, dgmg.default_opts(stop=dgmg.STOP_ENERGY, rtol=1e-6))
    assert st["converged"]
    with pytest.raises(dgmg.DgmgError):
        ctx.apply(f.float(), torch.empty_like(f).float())


# ------------------------------------------------------------- degenerate sizes and inputs
@pytest.mark.parametrize("nc,p,bc,react", [((1, 1, 1), 1, [0] * 6, False), ((1, 1, 1), 8, [1] * 6, True),
                                           ((1, 1, 7), 2, [0, 1, 1, 0, 0, 1], False), ((5, 1, 1), 3, [1, 0] * 3, True),
                                           ((2, 7, 1), 5, [0] * 6, False)])
def test_degenerate_meshes(nc, p, bc, react):
    """One cell, slabs one cell thick, p = 1 and p = 8 (the smallest and
    largest orders), pure Neumann with a reaction term: operator (FP64 1e-12),
    exact block smoother against dense-LU block-Jacobi, and the Q1 transfer,
    all on ragged warp tails."""
    rng = np.random.default_rng(91)
    ncell = int(np.prod(nc))
    w = custom(nc, (0.7, 1.3, 0.9), p, bc, np.exp(rng.normal(size=(ncell, 3))),
               c=rng.uniform(0.5, 2.0, ncell) if react else None)
    P = oracle_problem(w)
    A = P.assemble()
    ctx = gpu_context(w)
    u = inputs.random_dg_vector(P.ndof, seed=92)
    v = torch.empty(P.ndof, dtype=torch.float64, device="cuda")
    ctx.apply(dev(u), v)
    assert rel_err(v.cpu().numpy(), A @ u) < 1e-12
    f = inputs.random_dg_vector(P.ndof, seed=93)
    ref = solvers.BlockJacobi(A, P.N, inner="lu")(f, u, 1, 0.8)
    x = dev(u)
    ctx.block_smooth(dev(f), x, nsweep=1, omega=0.8, eps=1e-14, maxit=20 * P.N)
    assert rel_err(x.cpu().numpy(), ref) < 1e-9
    Pm = transfer.prolongation(P)
    rh = torch.empty(P.nvert, dtype=torch.float64, device="cuda")
    ctx.restrict(dev(u), rh)
    assert rel_err(rh.cpu().numpy(), Pm.T @ u) < 1e-13


def test_zero_inputs():
    """Zero in, zero out, exactly: the operator, a smoother sweep from u = 0
    with f = 0 (no 0/0 in the per-cell normalisation), the V-cycle, and a
    solve with f = 0 (converged at once, u stays 0)."""
    from paper_1805_11930_gb300 import dgmg
    w = make_case("p2_mixed")
    ctx = gpu_context(w)
    nd = ctx.sizes()["ndof"]
    z = torch.zeros(nd, dtype=torch.float64, device="cuda")
    v = torch.full_like(z, 7.0)
    ctx.apply(z, v)
    assert torch.count_nonzero(v) == 0
    for inner in (dgmg.INNER_PCG, dgmg.INNER_GMRES, dgmg.INNER_DIRECT):
        u = torch.zeros_like(z)
        ctx.block_smooth(z, u, nsweep=2, omega=0.8, inner=inner)
        assert torch.count_nonzero(u) == 0 and bool(torch.isfinite(u).all())
    u = torch.zeros_like(z)
    ctx.vcycle(z, u)
    assert torch.count_nonzero(u) == 0
    st = ctx.solve(z, u)
    assert st["converged"] and st["iterations"] == 0 and torch.count_nonzero(u) == 0


def test_nan_rhs_is_reported_not_hung():
    """A NaN in the right-hand side ends the solve with an error status
    (Krylov breakdown: p^T A p is not > 0) instead of iterating to maxit, and
    the context stays usable for the next, finite solve."""
    from paper_1805_11930_gb300 import dgmg
    w = inputs.poisson_sine(6, 2)
    ctx = gpu_context(w)
    f = gpu_rhs(ctx, w, torch)
    bad = f.clone()
    bad[17] = float("nan")
    for kry in (dgmg.KRYLOV_CG, dgmg.KRYLOV_FCG, dgmg.KRYLOV_FGMRES):
        u0 = torch.zeros_like(f)
        st = ctx.solve(bad, u0, dgmg.default_opts(krylov=kry), check=False)
        assert st["status"] == "DGMG_ERR_ARG" and st["iterations"] == 0
        assert not bool(u0.any())
    u = torch.zeros_like(f)
    assert ctx.solve(f, u)["converged"] and bool(torch.isfinite(u).all())


@pytest.mark.parametrize("coarse", ["AMG", "P0"])
def test_component_timers_and_inner_statistics(coarse):
    """With opts.timing the solve reports device time per component; the
    components are disjoint parts of the solve, so they are non-negative and
    add up to the whole (the rest, the Krylov work, is the remainder).  The
    inner iteration statistics obey 0 <= std and std^2 <= (max - mean) mean
    (Bhatia-Davis, the counts lying in [0, max])."""
    from paper_1805_11930_gb300 import dgmg
    w = inputs.lognormal(8, 3)
    ctx = gpu_context(w)
    f = gpu_rhs(ctx, w, torch)
    u = torch.zeros_like(f)
    st = ctx.solve(f, u, dgmg.default_opts(timing=1, coarse=getattr(dgmg, "COARSE_" + coarse)))
    assert st["converged"]
    parts = [st[k] for k in ("ms_smooth", "ms_apply", "ms_transfer", "ms_coarse", "ms_krylov")]
    assert all(x > 0 for x in parts)
    assert sum(parts) == pytest.approx(st["ms_device"], rel=1e-6)
    assert st["ms_device"] <= st["ms_total"] * 1.01
    m, s, mx = st["inner_mean"], st["inner_std"], st["inner_max"]
    assert 0 < m <= mx and 0 <= s and s * s <= (mx - m) * m * (1 + 1e-12)
    # without timing the component times stay zero and the statistics agree
    u.zero_()
    st2 = ctx.solve(f, u, dgmg.default_opts(coarse=getattr(dgmg, "COARSE_" + coarse)))
    assert st2["ms_device"] == 0 and st2["ms_coarse"] == 0
    assert st2["inner_std"] == pytest.approx(s, rel=1e-12) and st2["inner_mean"] == pytest.approx(m, rel=1e-12)


@pytest.mark.parametrize("alpha", [0.6, 4.0])
def test_penalty_parameter(alpha):
    """dgmg_set_penalty: with alpha other than 1.25 the operator, diag(D_T),
    the Q1 and P0 coarse matrices and the right-hand side (Dirichlet penalty
    term) all match the oracle built with the same alpha."""
    from oracle import dg as odg
    w = make_case("p2_mixed")
    P = odg.Problem(*w["nc"], *w["L"], w["p"], w["bc"], w["K"], b_vertex=w["b"], c_cell=w["c"], alpha=alpha)
    A = P.assemble()
    from paper_1805_11930_gb300 import dgmg
    ctx = dgmg.Context(0)
    ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
    ctx.set_penalty(alpha)
    ctx.set_coefficients(w["K"], b_vertex=w["b"], c_cell=w["c"])
    u = inputs.random_dg_vector(P.ndof, seed=61)
    v = torch.empty(P.ndof, dtype=torch.float64, device="cuda")
    ctx.apply(dev(u), v)
    assert rel_err(v.cpu().numpy(), A @ u) < 1e-12
    d = torch.empty(P.ndof, dtype=torch.float64, device="cuda")
    ctx.block_diagonal(d)
    assert rel_err(d.cpu().numpy(), A.diagonal()) < 1e-12
    Pm = transfer.prolongation(P)
    G = (Pm.T @ A @ Pm).toarray()
    st = ctx.coarse_matrix()
    Vx, Vy, Vz = P.nv
    Ah = np.zeros_like(G)
    for vtx in range(P.nvert):
        ix, iy, iz = vtx % Vx, (vtx // Vx) % Vy, vtx // (Vx * Vy)
        for k in range(27):
            jx, jy, jz = ix + k % 3 - 1, iy + (k // 3) % 3 - 1, iz + k // 9 - 1
            if 0 <= jx < Vx and 0 <= jy < Vy and 0 <= jz < Vz:
                Ah[vtx, jx + Vx * (jy + Vy * jz)] = st[vtx, k]
    assert np.abs(Ah - G).max() < 1e-12 * np.abs(G).max()
    G0 = transfer.p0_matrix(A, P).toarray()
    assert np.abs(_stencil_dense(ctx.coarse_matrix_p0(), P.nc) - G0).max() < 1e-12 * np.abs(G0).max()
    rhs = gpu_rhs(ctx, w, torch)
    assert rel_err(rhs.cpu().numpy(), oracle_rhs(P, w)) < 1e-13
    # the penalty is fixed once the coefficients are set; the context keeps it for the next mesh
    with pytest.raises(dgmg.DgmgError):
        ctx.set_penalty(1.25)
    ctx.set_mesh(*w["nc"], *w["L"], w["p"], w["bc"])
    ctx.set_coefficients(w["K"], b_vertex=w["b"], c_cell=w["c"])
    ctx.apply(dev(u), v)
    assert rel_err(v.cpu().numpy(), A @ u) < 1e-12
