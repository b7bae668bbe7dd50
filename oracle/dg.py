"""Explicit assembly of the SIPG / upwind DG operator and right-hand side.

Part of the CPU oracle (test infrastructure only, never called by the
library).  Every quantity is computed from its definition in Sec. 2.1 of the
paper:

* the bilinear form a_h = a^v + a^if + a^bf  (eq. bilinear_form_split),
* jump [[v]] = v^- - v^+, weighted average {v}_w = w^- v^- + w^+ v^+,
  with v^{+-} the limit from either side along the face normal nu_F,
* Ern-Stephansen-Zunino weights w^{+-} = delta^{-+} / (delta^- + delta^+),
  delta = nu^T K nu,
* penalty gamma_F = alpha p (p+d-1) <delta^-, delta^+> |F| / min(|T^-|,|T^+|)
  on interior faces and alpha p (p+d-1) delta^- |F| / |T^-| on Dirichlet
  faces, <a, b> = 2ab/(a+b), alpha = 1.25,
* upwind flux Phi(u^-, u^+, b_nu) = b_nu u^- if b_nu >= 0 else b_nu u^+,
* the right-hand side functional l_h (eq. rhs),
* A_ij = a_h(psi_j, psi_i)  (eq. linear_equation).

Each block (T, T') is obtained by looping over quadrature points and basis
pairs (einsum over the point index); there is no sum factorisation here.

Readings of the paper used below:
* cells are the axis-aligned boxes of a uniform nx x ny x nz grid of
  [0,Lx]x[0,Ly]x[0,Lz]; cell (cx,cy,cz) has index cx + nx (cy + ny cz);
* the DG vector is cell-major; inside a cell dof (i1,i2,i3) has index
  i1 + n i2 + n^2 i3 (x fastest), n = p+1;
* on the face between cells i and i+1 along axis k, T^- = cell i, T^+ =
  cell i+1 and nu_F = +e_k; on boundary faces nu is the outward normal;
* all integrals use the tensor Gauss rule with m = p+1 points per direction;
* K is given per cell (scalar, diagonal or full symmetric 3x3), c per cell,
  and b as a continuous trilinear (Q1) vertex field; or K and c are
  functions of the position (K_fn, c_fn), evaluated at every quadrature
  point, as in the paper's inhomogeneous test K(x) = sum_k P_k(x_k) n_k n_k^T,
  c(x) = gamma |x|^2 (Sec. 4.2).  A function K is continuous, so both traces
  on a face take the same value K(x); delta, the weights and the penalty are
  then evaluated point by point.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from . import quadrature as quad

DIM = 3


def harmonic(a, b):
    """<a, b> = 2ab/(a+b) (Sec. 2.1, penalty definition)."""
    return 2.0 * a * b / (a + b)


class Problem:
    """Mesh, polynomial degree, boundary flags and coefficients.

    bc[2k+s] is the condition on the boundary plane x_k = s*L_k
    (0 = Dirichlet, 1 = Neumann), planes ordered -x, +x, -y, +y, -z, +z.
    K: (ncell,) scalar, (ncell, 3) diagonal or (ncell, 3, 3) full tensor.
    b_vertex: None or (nvert, 3) values of b at the grid vertices, vertex
    (vx,vy,vz) at index vx + (nx+1) (vy + (ny+1) vz).
    c_cell: None or (ncell,) reaction coefficient.
    """

    def __init__(self, nx, ny, nz, lx, ly, lz, p, bc, K, b_vertex=None,
                 c_cell=None, alpha=1.25, K_fn=None, c_fn=None):
        if p < 1:
            raise ValueError("p >= 1 required")
        self.nc = (int(nx), int(ny), int(nz))
        self.L = np.array([lx, ly, lz], dtype=np.float64)
        self.h = self.L / np.array(self.nc, dtype=np.float64)
        self.p = int(p)
        self.n = self.p + 1
        self.m = self.p + 1
        self.N = self.n ** 3
        self.bc = [int(x) for x in bc]
        self.alpha = float(alpha)
        self.ncell = nx * ny * nz
        self.ndof = self.ncell * self.N
        self.nv = (nx + 1, ny + 1, nz + 1)
        self.nvert = (nx + 1) * (ny + 1) * (nz + 1)
        K = np.asarray(K, dtype=np.float64)
        if K.ndim == 1:
            Kf = K[:, None, None] * np.eye(3)[None]
        elif K.ndim == 2:
            Kf = np.zeros((self.ncell, 3, 3))
            for k in range(3):
                Kf[:, k, k] = K[:, k]
        else:
            Kf = K.copy()
        assert Kf.shape == (self.ncell, 3, 3)
        self.K = Kf
        self.b = None if b_vertex is None else np.asarray(b_vertex, dtype=np.float64).reshape(self.nvert, 3)
        self.c = None if c_cell is None else np.asarray(c_cell, dtype=np.float64).reshape(self.ncell)
        self.K_fn, self.c_fn = K_fn, c_fn       # pointwise coefficients (replace K, c when given)
        self.gll, self.gll_w = quad.gauss_lobatto(self.n)
        self.gq, self.gw = quad.gauss_legendre(self.m)
        self._volume_tables()

    # ---------------------------------------------------------------- indexing
    def cell_index(self, cx, cy, cz):
        return cx + self.nc[0] * (cy + self.nc[1] * cz)

    def cell_coords(self, c):
        cx = c % self.nc[0]
        cy = (c // self.nc[0]) % self.nc[1]
        cz = c // (self.nc[0] * self.nc[1])
        return (cx, cy, cz)

    def vertex_index(self, vx, vy, vz):
        return vx + self.nv[0] * (vy + self.nv[1] * vz)

    def cell_origin(self, c):
        return np.array(self.cell_coords(c), dtype=np.float64) * self.h

    # ------------------------------------------------------------ basis tables
    def basis_at(self, xi):
        """Values (P, N) and reference gradients (P, N, 3) of the n^3 tensor
        GLL Lagrange basis functions at reference points xi (P, 3) in [0,1]^3."""
        xi = np.atleast_2d(xi)
        V = [quad.lagrange_values(self.gll, xi[:, k]) for k in range(3)]
        G = [quad.lagrange_derivatives(self.gll, xi[:, k]) for k in range(3)]
        P = xi.shape[0]
        n = self.n
        val = np.zeros((P, self.N))
        grad = np.zeros((P, self.N, 3))
        for i3, i2, i1 in itertools.product(range(n), range(n), range(n)):
            i = i1 + n * i2 + n * n * i3
            val[:, i] = V[0][:, i1] * V[1][:, i2] * V[2][:, i3]
            grad[:, i, 0] = G[0][:, i1] * V[1][:, i2] * V[2][:, i3]
            grad[:, i, 1] = V[0][:, i1] * G[1][:, i2] * V[2][:, i3]
            grad[:, i, 2] = V[0][:, i1] * V[1][:, i2] * G[2][:, i3]
        return val, grad

    def _volume_tables(self):
        m = self.m
        pts, wts = [], []
        for q3, q2, q1 in itertools.product(range(m), range(m), range(m)):
            pts.append((self.gq[q1], self.gq[q2], self.gq[q3]))
            wts.append(self.gw[q1] * self.gw[q2] * self.gw[q3])
        self.vol_xi = np.array(pts)                      # (Q, 3), q = q1 + m q2 + m^2 q3
        self.vol_w = np.array(wts) * np.prod(self.h)     # physical weights
        self.vol_val, gref = self.basis_at(self.vol_xi)
        self.vol_grad = gref / self.h[None, None, :]     # physical gradients

    @staticmethod
    def tangential_axes(k):
        return [a for a in range(3) if a != k]

    def face_xi(self, k, side):
        """Reference points (F, 3) and physical weights (F,) of the face
        x_k = side of the reference cell; face point f = qa + m qb over the
        two tangential axes a < b."""
        a, b = self.tangential_axes(k)
        m = self.m
        pts, wts = [], []
        for qb, qa in itertools.product(range(m), range(m)):
            x = np.zeros(3)
            x[k] = float(side)
            x[a] = self.gq[qa]
            x[b] = self.gq[qb]
            pts.append(x)
            wts.append(self.gw[qa] * self.gw[qb])
        return np.array(pts), np.array(wts) * self.h[a] * self.h[b]

    # ------------------------------------------------------------ coefficients
    def b_at(self, c, xi):
        """b at reference points xi (P, 3) of cell c by trilinear interpolation
        of the vertex field; zeros if there is no advection."""
        xi = np.atleast_2d(xi)
        if self.b is None:
            return np.zeros((xi.shape[0], 3))
        cx, cy, cz = self.cell_coords(c)
        out = np.zeros((xi.shape[0], 3))
        for ox, oy, oz in itertools.product((0, 1), (0, 1), (0, 1)):
            wgt = np.ones(xi.shape[0])
            for k, o in enumerate((ox, oy, oz)):
                wgt *= xi[:, k] if o == 1 else (1.0 - xi[:, k])
            out += wgt[:, None] * self.b[self.vertex_index(cx + ox, cy + oy, cz + oz)][None, :]
        return out

    def K_points(self, c, xi):
        """K at reference points xi (P, 3) of cell c: (P, 3, 3), from K_fn at
        the physical points, or the cell's constant K."""
        xi = np.atleast_2d(xi)
        if self.K_fn is None:
            return np.broadcast_to(self.K[c], (xi.shape[0], 3, 3))
        return np.asarray(self.K_fn(self.cell_origin(c)[None, :] + xi * self.h[None, :]), dtype=np.float64)

    def c_of(self, c):
        return 0.0 if self.c is None else float(self.c[c])

    def penalty_interior(self, dm, dp, k):
        """gamma_F on an interior face normal to axis k (uniform grid, so
        min(|T^-|,|T^+|) = |T| and |F|/|T| = 1/h_k)."""
        a, b = self.tangential_axes(k)
        area = self.h[a] * self.h[b]
        vol = np.prod(self.h)
        return self.alpha * self.p * (self.p + DIM - 1) * harmonic(dm, dp) * area / vol

    def penalty_boundary(self, dm, k):
        a, b = self.tangential_axes(k)
        area = self.h[a] * self.h[b]
        vol = np.prod(self.h)
        return self.alpha * self.p * (self.p + DIM - 1) * dm * area / vol

    # ------------------------------------------------------------ local blocks
    def volume_block(self, c):
        """(A^v_{T,T})_{ij} = a^v(psi_j, psi_i) on cell c:
        (K grad u - b u, grad v)_T + (c u, v)_T by Gauss quadrature."""
        w = self.vol_w
        val, g = self.vol_val, self.vol_grad
        bq = self.b_at(c, self.vol_xi)
        if self.K_fn is None:
            K = self.K[c]
            A = np.einsum('q,kl,qjl,qik->ij', w, K, g, g, optimize=True)
        else:
            Kq = self.K_points(c, self.vol_xi)
            A = np.einsum('q,qkl,qjl,qik->ij', w, Kq, g, g, optimize=True)
        A -= np.einsum('q,qk,qj,qik->ij', w, bq, val, g, optimize=True)
        if self.c_fn is not None:
            X = self.cell_origin(c)[None, :] + self.vol_xi * self.h[None, :]
            A += np.einsum('q,q,qj,qi->ij', w, self.c_fn(X), val, val, optimize=True)
        else:
            cc = self.c_of(c)
            if cc != 0.0:
                A += cc * np.einsum('q,qj,qi->ij', w, val, val, optimize=True)
        return A

    def interior_face_matrix(self, cm, k):
        """2N x 2N matrix of a^if(psi_J, psi_I) on the face between cell cm
        (T^-) and its neighbour cp = cm + e_k (T^+); indices 0..N-1 belong to
        T^-, N..2N-1 to T^+.  Returns (matrix, cp)."""
        cx = list(self.cell_coords(cm))
        cx[k] += 1
        cp = self.cell_index(*cx)
        N = self.N
        xm, w = self.face_xi(k, 1)        # face seen from T^-: xi_k = 1
        xp, _ = self.face_xi(k, 0)        # seen from T^+: xi_k = 0
        vm, gm = self.basis_at(xm)
        vp, gp = self.basis_at(xp)
        gm = gm / self.h[None, None, :]
        gp = gp / self.h[None, None, :]
        nu = np.zeros(3)
        nu[k] = 1.0
        F = len(w)
        VM = np.concatenate([vm, np.zeros((F, N))], axis=1)
        VP = np.concatenate([np.zeros((F, N)), vp], axis=1)
        jump = VM - VP
        bnu = self.b_at(cm, xm) @ nu
        Phi = np.where(bnu[:, None] >= 0.0, bnu[:, None] * VM, bnu[:, None] * VP)
        if self.K_fn is None:
            Km, Kp = self.K[cm], self.K[cp]
            dm, dp = nu @ Km @ nu, nu @ Kp @ nu
            wm, wp = dp / (dm + dp), dm / (dm + dp)
            FM = np.concatenate([np.einsum('l,qjl->qj', Km @ nu, gm), np.zeros((F, N))], axis=1)
            FP = np.concatenate([np.zeros((F, N)), np.einsum('l,qjl->qj', Kp @ nu, gp)], axis=1)
            avg = wm * FM + wp * FP
            gamma = self.penalty_interior(dm, dp, k)
            A = np.einsum('q,qJ,qI->IJ', w, Phi, jump, optimize=True)
            A -= np.einsum('q,qJ,qI->IJ', w, avg, jump, optimize=True)
            A -= np.einsum('q,qI,qJ->IJ', w, avg, jump, optimize=True)
            A += gamma * np.einsum('q,qJ,qI->IJ', w, jump, jump, optimize=True)
            return A, cp
        # pointwise K (the same value from both sides): weights, delta and gamma per point
        Km, Kp = self.K_points(cm, xm), self.K_points(cp, xp)
        dm, dp = Km @ nu @ nu, Kp @ nu @ nu
        wm, wp = dp / (dm + dp), dm / (dm + dp)
        FM = np.concatenate([np.einsum('ql,qjl->qj', Km @ nu, gm), np.zeros((F, N))], axis=1)
        FP = np.concatenate([np.zeros((F, N)), np.einsum('ql,qjl->qj', Kp @ nu, gp)], axis=1)
        avg = wm[:, None] * FM + wp[:, None] * FP
        gamma = self.penalty_interior(dm, dp, k)
        A = np.einsum('q,qJ,qI->IJ', w, Phi, jump, optimize=True)
        A -= np.einsum('q,qJ,qI->IJ', w, avg, jump, optimize=True)
        A -= np.einsum('q,qI,qJ->IJ', w, avg, jump, optimize=True)
        A += np.einsum('q,q,qJ,qI->IJ', w, gamma, jump, jump, optimize=True)
        return A, cp

    def boundary_face_block(self, c, k, side):
        """N x N block a^bf(psi_j, psi_i) of a Dirichlet face x_k = side*L_k
        of cell c (outward normal +-e_k)."""
        xi, w = self.face_xi(k, side)
        v, g = self.basis_at(xi)
        g = g / self.h[None, None, :]
        nu = np.zeros(3)
        nu[k] = 1.0 if side == 1 else -1.0
        bnu = self.b_at(c, xi) @ nu
        Phi = np.where(bnu[:, None] >= 0.0, bnu[:, None] * v, 0.0)
        if self.K_fn is None:
            Kc = self.K[c]
            delta = nu @ Kc @ nu
            fl = np.einsum('l,qjl->qj', Kc @ nu, g)          # nu . K grad psi_j
            gamma = self.penalty_boundary(delta, k)
            A = np.einsum('q,qj,qi->ij', w, Phi, v, optimize=True)
            A -= np.einsum('q,qj,qi->ij', w, fl, v, optimize=True)
            A -= np.einsum('q,qi,qj->ij', w, fl, v, optimize=True)
            A += gamma * np.einsum('q,qj,qi->ij', w, v, v, optimize=True)
            return A
        Kq = self.K_points(c, xi)
        gamma = self.penalty_boundary(Kq @ nu @ nu, k)
        fl = np.einsum('ql,qjl->qj', Kq @ nu, g)
        A = np.einsum('q,qj,qi->ij', w, Phi, v, optimize=True)
        A -= np.einsum('q,qj,qi->ij', w, fl, v, optimize=True)
        A -= np.einsum('q,qi,qj->ij', w, fl, v, optimize=True)
        A += np.einsum('q,q,qj,qi->ij', w, gamma, v, v, optimize=True)
        return A

    def is_boundary(self, c, k, side):
        ck = self.cell_coords(c)[k]
        return (side == 0 and ck == 0) or (side == 1 and ck == self.nc[k] - 1)

    # ------------------------------------------------------------ assembly
    def block_row(self, c):
        """Dict {column cell: N x N block} of block row c of A."""
        N = self.N
        row = {c: self.volume_block(c)}
        for k in range(3):
            for side in (0, 1):
                if self.is_boundary(c, k, side):
                    if self.bc[2 * k + side] == 0:
                        row[c] = row[c] + self.boundary_face_block(c, k, side)
                    continue
                if side == 1:
                    AF, nb = self.interior_face_matrix(c, k)
                    row[c] = row[c] + AF[:N, :N]
                    row[nb] = row.get(nb, 0.0) + AF[:N, N:]
                else:
                    cx = list(self.cell_coords(c))
                    cx[k] -= 1
                    cm = self.cell_index(*cx)
                    AF, _ = self.interior_face_matrix(cm, k)
                    row[c] = row[c] + AF[N:, N:]
                    row[cm] = row.get(cm, 0.0) + AF[N:, :N]
        return row

    def assemble(self):
        """A as a scipy BSR matrix with (p+1)^3 x (p+1)^3 blocks (eq. block_ls)."""
        N = self.N
        indptr = [0]
        indices, data = [], []
        for c in range(self.ncell):
            row = self.block_row(c)
            for col in sorted(row):
                indices.append(col)
                data.append(row[col])
            indptr.append(len(indices))
        return sp.bsr_matrix((np.array(data), np.array(indices), np.array(indptr)),
                             shape=(self.ndof, self.ndof), blocksize=(N, N))

    def apply_rows(self, u, cells):
        """(A u) restricted to the given cells, from their block rows only
        (used to check sampled outputs at sizes too large to assemble)."""
        N = self.N
        out = np.zeros((len(cells), N))
        for r, c in enumerate(cells):
            for col, blk in self.block_row(int(c)).items():
                out[r] += blk @ u[col * N:(col + 1) * N]
        return out

    def diagonal_block(self, c):
        """D_T = A_{T,T} (volume plus the own-side face terms, eq. block_diag_apply)."""
        return self.block_row(c)[c]

    # ------------------------------------------------------------ quadrature points
    def volume_points(self):
        """Physical coordinates (ncell, m^3, 3) of the volume quadrature points,
        point q = q1 + m q2 + m^2 q3."""
        out = np.zeros((self.ncell, len(self.vol_w), 3))
        for c in range(self.ncell):
            out[c] = self.cell_origin(c)[None, :] + self.vol_xi * self.h[None, :]
        return out

    def boundary_cells(self, k, side):
        """Cells on plane x_k = side*L_k, ordered by (ca + n_a cb) over the
        tangential cell indices a < b."""
        a, b = self.tangential_axes(k)
        cells = []
        for cb in range(self.nc[b]):
            for ca in range(self.nc[a]):
                idx = [0, 0, 0]
                idx[k] = 0 if side == 0 else self.nc[k] - 1
                idx[a] = ca
                idx[b] = cb
                cells.append(self.cell_index(*idx))
        return cells

    def boundary_points(self):
        """Physical coordinates of boundary face quadrature points, planes in
        order -x,+x,-y,+y,-z,+z, cells as in boundary_cells, points f = qa + m qb.
        Returns a list of (cells, xyz (ncells_on_plane, m^2, 3))."""
        out = []
        for k in range(3):
            for side in (0, 1):
                xi, _ = self.face_xi(k, side)
                cells = self.boundary_cells(k, side)
                xyz = np.zeros((len(cells), len(xi), 3))
                for r, c in enumerate(cells):
                    xyz[r] = self.cell_origin(c)[None, :] + xi * self.h[None, :]
                out.append((cells, xyz))
        return out

    def rhs(self, f_qp, g_qp=None, j_qp=None):
        """f_i = l_h(psi_i) (eq. rhs) from values at quadrature points:
        f_qp (ncell, m^3); g_qp, j_qp flat arrays over all six planes in the
        boundary_points order (values on planes of the other kind unused)."""
        N = self.N
        F = np.zeros(self.ndof)
        f_qp = np.asarray(f_qp, dtype=np.float64).reshape(self.ncell, -1)
        for c in range(self.ncell):
            F[c * N:(c + 1) * N] += np.einsum('q,q,qi->i', self.vol_w, f_qp[c], self.vol_val, optimize=True)
        off = 0
        mm = self.m * self.m
        for k in range(3):
            for side in (0, 1):
                xi, w = self.face_xi(k, side)
                v, g = self.basis_at(xi)
                g = g / self.h[None, None, :]
                nu = np.zeros(3)
                nu[k] = 1.0 if side == 1 else -1.0
                cells = self.boundary_cells(k, side)
                for c in cells:
                    sl = slice(off, off + mm)
                    off += mm
                    if self.bc[2 * k + side] == 1:
                        if j_qp is not None:
                            jv = np.asarray(j_qp, dtype=np.float64)[sl]
                            F[c * N:(c + 1) * N] -= np.einsum('q,q,qi->i', w, jv, v, optimize=True)
                        continue
                    if g_qp is None:
                        continue
                    gv = np.asarray(g_qp, dtype=np.float64)[sl]
                    bnu = self.b_at(c, xi) @ nu
                    phi = np.where(bnu >= 0.0, 0.0, bnu * gv)       # Phi(0, g, b_nu)
                    F[c * N:(c + 1) * N] -= np.einsum('q,q,qi->i', w, phi, v, optimize=True)
                    if self.K_fn is None:
                        Kc = self.K[c]
                        delta = nu @ Kc @ nu
                        fl = np.einsum('l,qil->qi', Kc @ nu, g, optimize=True)
                        gamma = self.penalty_boundary(delta, k)
                        F[c * N:(c + 1) * N] -= np.einsum('q,q,qi->i', w, gv, fl, optimize=True)
                        F[c * N:(c + 1) * N] += gamma * np.einsum('q,q,qi->i', w, gv, v, optimize=True)
                    else:
                        Kq = self.K_points(c, xi)
                        fl = np.einsum('ql,qil->qi', Kq @ nu, g, optimize=True)
                        gamma = self.penalty_boundary(Kq @ nu @ nu, k)
                        F[c * N:(c + 1) * N] -= np.einsum('q,q,qi->i', w, gv, fl, optimize=True)
                        F[c * N:(c + 1) * N] += np.einsum('q,q,q,qi->i', w, gamma, gv, v, optimize=True)
        return F

    def interpolate(self, fn):
        """Nodal interpolant of fn(x, y, z) in V_h (values at the GLL nodes)."""
        n = self.n
        u = np.zeros(self.ndof)
        nodes = []
        for i3, i2, i1 in itertools.product(range(n), range(n), range(n)):
            nodes.append((self.gll[i1], self.gll[i2], self.gll[i3]))
        nodes = np.array(nodes)
        for c in range(self.ncell):
            x = self.cell_origin(c)[None, :] + nodes * self.h[None, :]
            u[c * self.N:(c + 1) * self.N] = fn(x[:, 0], x[:, 1], x[:, 2])
        return u

    def l2_error(self, u, fn, extra=2):
        """||u_h - fn||_{L2} with a Gauss rule of m + extra points per direction."""
        mq = self.m + extra
        g, w = quad.gauss_legendre(mq)
        pts, wts = [], []
        for q3, q2, q1 in itertools.product(range(mq), range(mq), range(mq)):
            pts.append((g[q1], g[q2], g[q3]))
            wts.append(w[q1] * w[q2] * w[q3])
        pts = np.array(pts)
        wts = np.array(wts) * np.prod(self.h)
        val, _ = self.basis_at(pts)
        err = 0.0
        for c in range(self.ncell):
            x = self.cell_origin(c)[None, :] + pts * self.h[None, :]
            uh = val @ u[c * self.N:(c + 1) * self.N]
            err += np.sum(wts * (uh - fn(x[:, 0], x[:, 1], x[:, 2])) ** 2)
        return np.sqrt(err)
