"""CPU parity of the library's host-side set-up code (csrc/setup_host.cpp)
against the oracle, through a test shim built with the host compiler alone:
the Q1 coarse matrix by re-discretisation (App. A.2) against P^T A P, the P0
coarse matrix (App. A.1) against P0^T A P0, one 2x2x2 Galerkin coarsening
of the AMG against the oracle's aggregation, the right-hand side l_h (eq.
rhs; also with K(x) in the Dirichlet terms, Sec. 4.2), the Gauss and
Gauss-Lobatto rules and the 1D tables the kernels read.  The same code runs on the GPU tier through the C ABI;
here it is checked without a GPU."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import amg, dg, quadrature, transfer
from paper_1805_11930_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_1805_11930_gb300", "csrc")
D = ctypes.POINTER(ctypes.c_double)
I = ctypes.POINTER(ctypes.c_int)


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    so = str(tmp_path_factory.mktemp("shim") / "libhostshim.so")
    subprocess.run([cxx, "-O3", "-std=c++17", "-shared", "-fPIC", os.path.join(HERE, "host_shim.cpp"),
                    os.path.join(CSRC, "setup_host.cpp"), "-I", CSRC, "-o", so], check=True)
    return ctypes.CDLL(so)


def _p(a, t=D):
    return None if a is None else a.ctypes.data_as(t)


def _mesh_args(nc, L, p, bc, K, b=None, c=None, alpha=1.25):
    K = np.ascontiguousarray(K, dtype=np.float64)
    kdim = 1 if K.ndim == 1 else K.shape[1]
    h = np.array(L, dtype=np.float64) / np.array(nc)
    bca = np.ascontiguousarray(bc, dtype=np.int32)
    b = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
    c = None if c is None else np.ascontiguousarray(c, dtype=np.float64)
    keep = (K, h, bca, b, c)
    return keep, [*nc, p, _p(h), _p(bca, I), _p(K), kdim, _p(b), _p(c), ctypes.c_double(alpha)]


def _dense(st, dims):
    vx, vy, vz = dims
    n = vx * vy * vz
    M = np.zeros((n, n))
    for v in range(n):
        ix, iy, iz = v % vx, (v // vx) % vy, v // (vx * vy)
        for k in range(27):
            jx, jy, jz = ix + k % 3 - 1, iy + (k // 3) % 3 - 1, iz + k // 9 - 1
            if 0 <= jx < vx and 0 <= jy < vy and 0 <= jz < vz:
                M[v, jx + vx * (jy + vy * jz)] = st[v, k]
            else:
                assert st[v, k] == 0.0
    return M


CASES = {
    "p1_diffusion": ((3, 2, 4), 1, [0, 1, 0, 0, 1, 0], False, False),
    "p2_reaction": ((4, 3, 2), 2, [0, 0, 1, 0, 0, 1], False, True),
    "p3_advection": ((3, 3, 2), 3, [0, 1, 0, 1, 0, 0], True, True),
    "p4_dirichlet": ((2, 2, 3), 4, [0] * 6, True, False),
}


def _case(name, seed=17):
    nc, p, bc, adv, react = CASES[name]
    rng = np.random.default_rng(seed)
    ncell = int(np.prod(nc))
    L = (1.0, 0.7, 1.3)
    K = np.exp(rng.normal(size=(ncell, 3)))
    b = inputs.vertex_field(nc, L, lambda x, y, z: np.stack([1 - 2 * y, x - 0.3, 0.25 + 0.5 * z], -1)) if adv else None
    c = rng.uniform(0.1, 2.0, size=ncell) if react else None
    return nc, L, p, bc, K, b, c


@pytest.mark.parametrize("name", list(CASES))
def test_q1_stencil_is_galerkin_product(shim, name):
    nc, L, p, bc, K, b, c = _case(name)
    P = dg.Problem(*nc, *L, p, bc, K, b_vertex=b, c_cell=c)
    Pm = transfer.prolongation(P)
    G = (Pm.T @ P.assemble() @ Pm).toarray()
    keep, args = _mesh_args(nc, L, p, bc, K, b, c)
    st = np.zeros((P.nvert, 27))
    shim.shim_q1_stencil(*args, _p(st))
    assert np.abs(_dense(st, P.nv) - G).max() < 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("name", list(CASES))
def test_p0_stencil_is_galerkin_product(shim, name):
    nc, L, p, bc, K, b, c = _case(name)
    P = dg.Problem(*nc, *L, p, bc, K, b_vertex=b, c_cell=c)
    G = transfer.p0_matrix(P.assemble(), P).toarray()
    keep, args = _mesh_args(nc, L, p, bc, K, b, c)
    st = np.zeros((P.ncell, 27))
    shim.shim_p0_stencil(*args, _p(st))
    assert np.abs(_dense(st, P.nc) - G).max() < 1e-12 * np.abs(G).max()


@pytest.mark.parametrize("dims", [(5, 4, 3), (8, 7, 6), (2, 2, 2)])
def test_coarsening_matches_the_oracle_aggregation(shim, dims):
    """One level of the AMG hierarchy: the 2x2x2 Galerkin coarsening of a
    27-point stencil equals Pa^T A Pa with the oracle's aggregates (ragged
    grids included)."""
    rng = np.random.default_rng(5)
    n = int(np.prod(dims))
    st = rng.normal(size=(n, 27))
    vx, vy, vz = dims
    for v in range(n):          # zero the entries that point outside the grid
        ix, iy, iz = v % vx, (v // vx) % vy, v // (vx * vy)
        for k in range(27):
            jx, jy, jz = ix + k % 3 - 1, iy + (k // 3) % 3 - 1, iz + k // 9 - 1
            if not (0 <= jx < vx and 0 <= jy < vy and 0 <= jz < vz):
                st[v, k] = 0.0
    A = _dense(st, dims)
    Pa, cdims = amg.aggregation(dims)
    G = (Pa.T @ A @ Pa)
    G = G.toarray() if hasattr(G, "toarray") else np.asarray(G)
    out = np.zeros(27 * n)
    cd = np.zeros(3, dtype=np.int32)
    shim.shim_coarsen(_p(np.ascontiguousarray(st)), vx, vy, vz, _p(out), _p(cd, I))
    assert tuple(cd) == tuple(cdims)
    nco = int(np.prod(cd))
    assert np.abs(_dense(out[:27 * nco].reshape(nco, 27), tuple(cd)) - G).max() < 1e-13 * np.abs(G).max()


def _points(shim, nc, L, p):
    P = dg.Problem(*nc, *L, p, [0] * 6, np.ones(int(np.prod(nc))))
    h = np.array(L, dtype=np.float64) / np.array(nc)
    m = p + 1
    nvol = P.ncell * m ** 3
    nx, ny, nz = nc
    nface = 2 * (ny * nz + nx * nz + nx * ny) * m * m
    vol = np.zeros((nvol, 3))
    face = np.zeros((nface, 3))
    shim.shim_quadrature_points(*nc, p, _p(h), _p(vol), _p(face))
    return vol, face


@pytest.mark.parametrize("name", list(CASES))
def test_rhs_matches_oracle(shim, name):
    nc, L, p, bc, K, b, c = _case(name)
    P = dg.Problem(*nc, *L, p, bc, K, b_vertex=b, c_cell=c)
    f = lambda x, y, z: np.sin(3 * x) * y + z * z                              # noqa: E731
    g = lambda x, y, z: np.exp(-((x - 0.2) ** 2 + (y - 0.5) ** 2) / 0.1) + z   # noqa: E731
    j = lambda x, y, z: np.cos(x + 2 * y) * z                                   # noqa: E731
    pts = np.concatenate([xyz.reshape(-1, 3) for _, xyz in P.boundary_points()])
    ref = P.rhs(inputs.evaluate(f, P.volume_points()), g_qp=inputs.evaluate(g, pts), j_qp=inputs.evaluate(j, pts))
    vol, face = _points(shim, nc, L, p)
    fq, gq, jq = (np.ascontiguousarray(inputs.evaluate(fn, xyz)) for fn, xyz in ((f, vol), (g, face), (j, face)))
    keep, args = _mesh_args(nc, L, p, bc, K, b, c)
    out = np.zeros(P.ndof)
    shim.shim_rhs(*args, None, _p(fq), _p(gq), _p(jq), _p(out))
    assert np.linalg.norm(out - ref) < 1e-13 * np.linalg.norm(ref)


def test_rhs_with_pointwise_tensor_matches_oracle(shim):
    """Sec. 4.2's K(x) (rotated, quadratic) in the Dirichlet consistency and
    penalty terms of l_h."""
    nc, L, p, bc = (3, 2, 2), (1.0, 0.8, 1.2), 3, [0, 1, 0, 0, 1, 0]
    gamma = 0.5
    P = dg.Problem(*nc, *L, p, bc, np.ones(12), K_fn=inputs.vark_tensor,
                   c_fn=lambda x: inputs.vark_reaction(x, gamma))
    g = lambda x, y, z: np.exp(-((x - 0.2) ** 2 + (y - 0.5) ** 2) / 0.1) + z   # noqa: E731
    f = lambda x, y, z: np.sin(3 * x) * y + z * z                              # noqa: E731
    pts = np.concatenate([xyz.reshape(-1, 3) for _, xyz in P.boundary_points()])
    ref = P.rhs(inputs.evaluate(f, P.volume_points()), g_qp=inputs.evaluate(g, pts))
    var = np.concatenate([np.asarray(inputs.VARK_BASIS).reshape(-1), inputs.VARK_P0, inputs.VARK_P2, [gamma]])
    h = np.array(L) / np.array(nc)
    zz, yy, xx = np.meshgrid(*[(np.arange(n) + 0.5) * hh for n, hh in zip(nc[::-1], h[::-1])], indexing="ij")
    centres = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], -1)     # cells x fastest
    Kc = np.ascontiguousarray(np.diagonal(inputs.vark_tensor(centres), axis1=-2, axis2=-1))
    vol, face = _points(shim, nc, L, p)
    fq, gq = (np.ascontiguousarray(inputs.evaluate(fn, xyz)) for fn, xyz in ((f, vol), (g, face)))
    keep, args = _mesh_args(nc, L, p, bc, Kc)
    args[-1] = ctypes.c_double(1.25)
    out = np.zeros(P.ndof)
    shim.shim_rhs(*args, _p(np.ascontiguousarray(var)), _p(fq), _p(gq), None, _p(out))
    assert np.linalg.norm(out - ref) < 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("n", range(2, 10))
def test_quadrature_rules_match_the_oracle(shim, n):
    x, w = np.zeros(n), np.zeros(n)
    shim.shim_gauss_legendre01(n, _p(x), _p(w))
    gx, gw = quadrature.gauss_legendre(n)
    assert np.abs(x - gx).max() < 1e-15 and np.abs(w - gw).max() < 1e-15
    shim.shim_gauss_lobatto01(n, _p(x), _p(w))
    lx, lw = quadrature.gauss_lobatto(n)
    assert np.abs(x - lx).max() < 1e-15 and np.abs(w - lw).max() < 1e-15


@pytest.mark.parametrize("alpha", [0.6, 4.0])
def test_coarse_matrices_follow_the_penalty_parameter(shim, alpha):
    nc, L, p, bc, K, b, c = _case("p3_advection")
    P = dg.Problem(*nc, *L, p, bc, K, b_vertex=b, c_cell=c, alpha=alpha)
    A = P.assemble()
    Pm = transfer.prolongation(P)
    keep, args = _mesh_args(nc, L, p, bc, K, b, c, alpha=alpha)
    st = np.zeros((P.nvert, 27))
    shim.shim_q1_stencil(*args, _p(st))
    G = (Pm.T @ A @ Pm).toarray()
    assert np.abs(_dense(st, P.nv) - G).max() < 1e-12 * np.abs(G).max()
    st0 = np.zeros((P.ncell, 27))
    shim.shim_p0_stencil(*args, _p(st0))
    G0 = transfer.p0_matrix(A, P).toarray()
    assert np.abs(_dense(st0, P.nc) - G0).max() < 1e-12 * np.abs(G0).max()


@pytest.mark.parametrize("n", range(2, 10))
def test_kernel_tables_match_the_oracle_basis(shim, n):
    """The 1D tables the kernels read (GLL basis and its derivative at the
    Gauss points, the Gauss collocation derivative, end-point derivatives,
    mass and stiffness matrices, Q1 hats, Gauss points and weights) against
    the oracle's basis functions, with the mass and stiffness matrices
    integrated by the oracle with a finer Gauss rule."""
    T = np.zeros(5 * n * n + 6 * n)
    shim.shim_build_tables(n, _p(T))
    gll, _ = quadrature.gauss_lobatto(n)
    gq, gw = quadrature.gauss_legendre(n)
    off = 0

    def take(k):
        nonlocal off
        out = T[off:off + k]
        off += k
        return out
    B, Dg, w, dl, M1, G, hat, g, S1 = (take(n * n), take(n * n), take(n), take(2 * n), take(n * n), take(n * n),
                                       take(2 * n), take(n), take(n * n))
    tol = 1e-12 * n ** 2
    assert np.abs(B.reshape(n, n) - quadrature.lagrange_values(gll, gq)).max() < tol
    assert np.abs(G.reshape(n, n) - quadrature.lagrange_derivatives(gll, gq)).max() < tol * n
    assert np.abs(Dg.reshape(n, n) - quadrature.lagrange_derivatives(gq, gq)).max() < tol * n
    assert np.abs(dl.reshape(2, n) - quadrature.lagrange_derivatives(gll, np.array([0.0, 1.0]))).max() < tol * n
    assert np.abs(w - gw).max() < 1e-15 and np.abs(g - gq).max() < 1e-15
    assert np.abs(hat.reshape(2, n) - np.stack([1 - gll, gll])).max() < 1e-15
    fx, fw = quadrature.gauss_legendre(n + 3)
    V, Vd = quadrature.lagrange_values(gll, fx), quadrature.lagrange_derivatives(gll, fx)
    assert np.abs(M1.reshape(n, n) - V.T @ (fw[:, None] * V)).max() < tol
    assert np.abs(S1.reshape(n, n) - Vd.T @ (fw[:, None] * Vd)).max() < tol * n * n


@pytest.mark.parametrize("n", [1, 7, 64])
def test_coarsest_dense_inverse(shim, n):
    rng = np.random.default_rng(n)
    A = rng.normal(size=(n, n)) + n * np.eye(n)
    Ai = np.ascontiguousarray(A.copy())
    assert shim.shim_dense_inverse(n, _p(Ai)) == 1
    assert np.abs(Ai @ A - np.eye(n)).max() < 1e-12
    S = np.ascontiguousarray(np.outer(np.arange(1.0, n + 1), np.ones(n)))   # rank one
    if n > 1:
        assert shim.shim_dense_inverse(n, _p(S)) == 0


def test_pointwise_tensor(shim):
    """K(x) = sum_k (p0_k + p2_k x_k^2) n_k n_k^T (Sec. 4.2) at a few points."""
    var = np.ascontiguousarray(np.concatenate([np.asarray(inputs.VARK_BASIS).reshape(-1), inputs.VARK_P0,
                                               inputs.VARK_P2, [1e-8]]))
    for x in ([0.1, 0.7, 0.3], [1.0, 0.0, 0.5], [0.25, 0.5, 0.75]):
        K6 = np.zeros(6)
        shim.shim_var_tensor(_p(var), _p(np.array(x, dtype=np.float64)), _p(K6))
        K = inputs.vark_tensor(np.array(x))
        ref = [K[0, 0], K[1, 1], K[2, 2], K[0, 1], K[0, 2], K[1, 2]]
        assert np.abs(K6 - ref).max() < 1e-14 * np.abs(K).max()


def test_rhs_volume_term_on_a_mesh_split_over_threads(shim):
    """A mesh large enough for the host right-hand side to split its cells
    over threads (32 x 32 x 4 cells, Q7: 2^21 volume points): every sampled
    cell, including the ones at the split, equals the definition
    f_T(i) = sum_q w_q |J| f(x_q) psi_i(x_q) with the oracle's basis."""
    nc, p = (32, 32, 4), 7
    n = p + 1
    ncell = int(np.prod(nc))
    L = (1.0, 1.0, 0.125)
    h = np.array(L) / np.array(nc)
    fq = np.ascontiguousarray(np.random.default_rng(3).normal(size=ncell * n ** 3))
    keep, args = _mesh_args(nc, L, p, [1] * 6, np.ones(ncell))
    out = np.zeros(ncell * n ** 3)
    shim.shim_rhs(*args, None, _p(fq), None, None, _p(out))
    gll, _ = quadrature.gauss_lobatto(n)
    gq, gw = quadrature.gauss_legendre(n)
    Bv = quadrature.lagrange_values(gll, gq)                      # [q, i]
    W3 = np.einsum("a,b,c->abc", gw, gw, gw) * np.prod(h)         # [qz, qy, qx]
    for c in (0, 1, ncell // 4, ncell // 2 - 1, ncell // 2, ncell // 2 + 1, 3 * ncell // 4, ncell - 1):
        F = fq[c * n ** 3:(c + 1) * n ** 3].reshape(n, n, n) * W3
        ref = np.einsum("zyx,xi,yj,zk->kji", F, Bv, Bv, Bv)
        got = out[c * n ** 3:(c + 1) * n ** 3].reshape(n, n, n)
        assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max(), c
