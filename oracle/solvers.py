"""Block smoothers, the hybrid V-cycle and the Krylov solvers.

Part of the CPU oracle (test infrastructure only, never called by the
library).  All matrices come from the explicit assembly in dg.py; this is the
paper's matrix-explicit (MX) design (Sec. 4.1) with exact or inexact block
inverses.

* Block-Jacobi smoother, W = omega^-1 D (Algorithm 2): defect, block solve,
  update.  Exact block solves use a dense LU with partial pivoting per block;
  inexact ones reduce the block residual two-norm by a factor eps with a
  Krylov method preconditioned by diag(D_T) (Sec. 2.2.1 and Sec. 3.2).
* Inner preconditioners: the diagonal of D_T (diffusion) or, for strongly
  convection-dominated blocks, the tridiagonal part of D_T in the cell's
  lexicographic dof order (x fastest) solved by the Thomas algorithm
  (Sec. 3.2 and Sec. 4.3, where the diagonal one fails to converge).
* Hybrid V-cycle (Algorithm 1).
* CG, flexible CG (Polak-Ribiere beta) and right-preconditioned flexible
  GMRES(restart) (Saad 1993) for the outer solve.

Readings (the paper does not state them): the inner solve starts from
delta = 0 and stops once ||d - D delta||_2 <= eps ||d||_2 or after maxit
iterations; the outer relative residual is the Euclidean norm of the
coefficient residual divided by that of the initial residual.
"""
import numpy as np
import scipy.linalg as sla


# ----------------------------------------------------------------- inner solves
def tridiagonal_part(D):
    """(sub, diag, sup) of a square matrix: sub[i] = D[i, i-1] (sub[0] = 0),
    sup[i] = D[i, i+1] (sup[-1] = 0)."""
    n = D.shape[0]
    sub = np.zeros(n)
    sup = np.zeros(n)
    sub[1:] = np.diagonal(D, -1)
    sup[:-1] = np.diagonal(D, 1)
    return sub, np.diagonal(D).copy(), sup


def thomas_solve(sub, diag, sup, r):
    """Solve the tridiagonal system (sub, diag, sup) x = r by the Thomas
    algorithm (Gaussian elimination without pivoting): forward sweep
    c'_0 = c_0 / b_0, c'_i = c_i / (b_i - a_i c'_{i-1}),
    d'_i = (r_i - a_i d'_{i-1}) / (b_i - a_i c'_{i-1}); back substitution
    x_{n-1} = d'_{n-1}, x_i = d'_i - c'_i x_{i+1}."""
    n = len(r)
    cp = np.zeros(n)
    dp = np.zeros(n)
    prev_c = 0.0
    prev_d = 0.0
    for i in range(n):
        den = diag[i] - sub[i] * prev_c
        cp[i] = sup[i] / den
        dp[i] = (r[i] - sub[i] * prev_d) / den
        prev_c, prev_d = cp[i], dp[i]
    x = np.zeros(n)
    x[n - 1] = dp[n - 1]
    for i in range(n - 2, -1, -1):
        x[i] = dp[i] - cp[i] * x[i + 1]
    return x


def block_pcg(D, d, dg, eps, maxit):
    """PCG on the dense block D with preconditioner 1/dg, from delta = 0.
    Returns (delta, iterations)."""
    x = np.zeros_like(d)
    r = d.copy()
    rr0 = r @ r
    if rr0 == 0.0:
        return x, 0
    z = r / dg
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        q = D @ p
        pq = p @ q
        if pq <= 0.0:
            break
        alpha = rz / pq
        x += alpha * p
        r -= alpha * q
        it += 1
        if r @ r <= eps * eps * rr0:
            break
        z = r / dg
        rz_new = r @ z
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return x, it


def block_gmres(D, d, dg, eps, maxit, restart, minv=None):
    """Right-preconditioned restarted GMRES on the dense block D with modified
    Gram-Schmidt and Givens rotations, from delta = 0.  The preconditioner is
    1/dg, or the map minv(v) = M^-1 v when given; with minv each cycle ends
    with x += M^-1 (V y) (Saad's right-preconditioned update).
    Returns (delta, iterations)."""
    x = np.zeros_like(d)
    target = eps * np.linalg.norm(d)
    r = d.copy()
    beta = np.linalg.norm(r)
    it = 0
    while it < maxit and beta > target and beta > 0.0:
        V = [r / beta]
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        j_done = 0
        for j in range(restart):
            w = D @ (V[j] / dg if minv is None else minv(V[j]))
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0.0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            if abs(g[j + 1]) <= target or it >= maxit:
                break
        y = sla.solve_triangular(H[:j_done, :j_done], g[:j_done])
        if minv is None:
            for i in range(j_done):
                x += y[i] * V[i] / dg
        else:
            x += minv(sum(y[i] * V[i] for i in range(j_done)))
        r = d - D @ x
        beta = np.linalg.norm(r)
    return x, it


# ----------------------------------------------------------------- smoother
class BlockJacobi:
    """Block-Jacobi smoother S(f, u; nsweep, omega) of Algorithm 2 on the
    assembled BSR matrix A."""

    def __init__(self, A, N, inner="lu", eps=1e-2, maxit=None, restart=12, precond="diag"):
        self.A = A.tocsr()
        self.precond = precond
        self.N = N
        self.ncell = A.shape[0] // N
        self.inner = inner
        self.eps = eps
        self.maxit = N if maxit is None else maxit
        self.restart = restart
        Ab = A.tobsr(blocksize=(N, N))
        self.D = [None] * self.ncell
        for c in range(self.ncell):
            for k in range(Ab.indptr[c], Ab.indptr[c + 1]):
                if Ab.indices[k] == c:
                    self.D[c] = Ab.data[k].copy()
        self._lu = None
        self.last_its = None

    def solve_block(self, c, d):
        if self.inner == "lu":
            if self._lu is None:
                self._lu = [sla.lu_factor(D) for D in self.D]
            return sla.lu_solve(self._lu[c], d), 0
        dg = np.diag(self.D[c])
        if self.inner == "pcg":
            return block_pcg(self.D[c], d, dg, self.eps, self.maxit)
        minv = None
        if self.precond == "tridiag":
            tri = tridiagonal_part(self.D[c])
            minv = lambda v: thomas_solve(*tri, v)   # noqa: E731
        return block_gmres(self.D[c], d, dg, self.eps, self.maxit, self.restart, minv=minv)

    def __call__(self, f, u, nsweep, omega):
        N = self.N
        u = u.copy()
        its = np.zeros(self.ncell, dtype=np.int64)
        for _ in range(nsweep):
            d = f - self.A @ u
            du = np.zeros_like(u)
            for c in range(self.ncell):
                du[c * N:(c + 1) * N], its[c] = self.solve_block(c, d[c * N:(c + 1) * N])
            u = u + omega * du
        self.last_its = its
        return u


class MulticolourBlockSOR(BlockJacobi):
    """Block-SOR / block-SSOR (Algorithm 3 and Sec. 2.2.1) with the cells taken
    colour by colour: colour(T) = (cx mod 2) + 2 (cy mod 2) + 4 (cz mod 2).
    Cells of one colour share no face, so within a colour the order does not
    matter; each cell's defect uses the current values of all other cells.
    A forward pass visits colours 0..7, the backward pass 7..0; symmetric
    sweeps do both.  Update: u_T <- u_T + omega D_T^-1 d_T (the correction
    form of Algorithm 2, read into Algorithm 3 whose printed update is
    inconsistent with it)."""

    def __init__(self, A, N, nc, symmetric=True, **kw):
        super().__init__(A, N, **kw)
        nx, ny, nz = nc
        c = np.arange(nx * ny * nz)
        cx, cy, cz = c % nx, (c // nx) % ny, c // (nx * ny)
        self.colour = (cx % 2) + 2 * (cy % 2) + 4 * (cz % 2)
        self.symmetric = symmetric

    def __call__(self, f, u, nsweep, omega):
        N = self.N
        u = u.copy()
        its = np.zeros(self.ncell, dtype=np.int64)
        order = list(range(8)) + (list(range(7, -1, -1)) if self.symmetric else [])
        for _ in range(nsweep):
            for k in order:
                d = f - self.A @ u
                for c in np.nonzero(self.colour == k)[0]:
                    du, its[c] = self.solve_block(c, d[c * N:(c + 1) * N])
                    u[c * N:(c + 1) * N] += omega * du
        self.last_its = its
        return u


# ----------------------------------------------------------------- V-cycle
class HybridVCycle:
    """One V-cycle of Algorithm 1: presmooth, residual, restrict, coarse
    correction, prolongate and add, postsmooth.  `coarse` maps a vertex
    vector r_hat to an approximation of A_hat^-1 r_hat."""

    def __init__(self, A, P, smoother, coarse, npre=1, npost=1, omega=1.0):
        self.A = A.tocsr()
        self.P = P.tocsr()
        self.R = P.T.tocsr()
        self.S = smoother
        self.coarse = coarse
        self.npre, self.npost, self.omega = npre, npost, omega

    def __call__(self, f, u0=None):
        u = np.zeros_like(f) if u0 is None else u0.copy()
        u = self.S(f, u, self.npre, self.omega)
        r = f - self.A @ u
        rh = self.R @ r
        uh = self.coarse(rh)
        u = u + self.P @ uh
        u = self.S(f, u, self.npost, self.omega)
        return u


# ----------------------------------------------------------------- outer Krylov
def cg(apply_A, b, precond, rtol=1e-8, maxit=1000, x0=None, flexible=False, stop="residual", delay=4):
    """Preconditioned CG; with flexible=True the Polak-Ribiere beta
    z_{k+1}.(r_{k+1} - r_k) / z_k.r_k.  Returns (x, iterations, history).

    stop="residual": ||r_k||_2 <= rtol ||r_0||_2; history holds the relative
    residuals.  stop="energy": the energy-norm error estimate of Strakos and
    Tichy (BIT 45, 2005, Sec. 3.1; used in the paper's Sec. 4.4 with an
    error bandwidth of 4): in PCG, ||e_k||_A^2 - ||e_{k+d}||_A^2 equals
    sum_{j=k}^{k+d-1} alpha_j (r_j, z_j), so after iteration k+d that sum
    estimates ||e_k||_A^2 from below, and sum_{j<k+d} estimates ||x - x_0||_A^2.
    The loop stops at the first k with sqrt(nu_k / total) <= rtol and returns
    x_{k+d}, the iteration count k (the d run-ahead iterations not counted)
    and the estimates as history."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x)
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    energy = stop == "energy"
    terms = []
    if energy:
        hist = []
    z = precond(r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = apply_A(p)
        alpha = rz / (p @ q)
        terms.append(alpha * rz)
        x = x + alpha * p
        r_old = r
        r = r - alpha * q
        rel = np.linalg.norm(r) / r0
        if energy:
            if it >= delay:
                k = it - delay
                nu = sum(terms[k:it])
                est = np.sqrt(nu / sum(terms[:it]))
                hist.append(est)
                if est <= rtol:
                    return x, k, hist
        else:
            hist.append(rel)
            if rel <= rtol:
                return x, it, hist
        z = precond(r)
        rz_new = z @ (r - r_old) if flexible else r @ z
        beta = rz_new / rz
        rz = r @ z
        p = z + beta * p
    return x, maxit, hist


def fgmres(apply_A, b, precond, restart=30, rtol=1e-8, maxit=1000, x0=None):
    """Right-preconditioned flexible GMRES(restart) with classical Gram-Schmidt
    applied twice (CGS2).  Returns (x, iterations, history)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - apply_A(x)
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    it = 0
    beta = r0
    while it < maxit:
        V = [r / beta]
        Z = []
        H = np.zeros((restart + 1, restart))
        g = np.zeros(restart + 1)
        g[0] = beta
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        k = 0
        for j in range(restart):
            z = precond(V[j])
            Z.append(z)
            w = apply_A(z)
            for _ in range(2):
                h = np.array([w @ v for v in V])
                for i, v in enumerate(V):
                    w = w - h[i] * v
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            V.append(w / H[j + 1, j])
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / r0)
            if abs(g[j + 1]) <= rtol * r0 or it >= maxit:
                break
        y = sla.solve_triangular(H[:k, :k], g[:k])
        for i in range(k):
            x = x + y[i] * Z[i]
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= rtol * r0:
            hist[-1] = beta / r0
            return x, it, hist
    return x, it, hist
