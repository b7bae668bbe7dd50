"""Intergrid operators and the Q1 coarse-space matrix.

Part of the CPU oracle (test infrastructure only, never called by the
library).

* Prolongation by injection of the conforming Q1 space into V_h^p, computed by
  evaluating the coarse basis at the nodal points: (P|_T)_{ij} =
  psi_hat_j(zeta_i) (Sec. 2.2.2, "Intergrid operators").
* Restriction R = P^T (same section).
* The piecewise-constant subspace P0 (Sec. 2.2.2; the coarse space of the
  paper's SPE10 runs, Sec. 4.4): P|_T = 1 (the nodal basis is a partition
  of unity), R = P^T sums a cell's values, and A_hat = P^T A P, the Galerkin
  product (App. A.1 defines A_hat this way and shows that it equals a
  re-scaled finite-volume matrix).
* Q1 matrix A_hat by re-discretisation (Sec. 2.2.3 and App. A.2): the
  conforming Q1 finite element matrix of the PDE plus the Dirichlet boundary
  terms of a_h, with the penalty gamma_F computed from the DG degree p.  Jump
  terms on interior faces vanish for continuous functions, so they are skipped.
  App. A.2 prints "+psi_hat_j psi_hat_i" where the reaction term
  c psi_hat_j psi_hat_i belongs and keeps a weight w^- that is 1 on the
  boundary; the oracle uses c and w^- = 1, so that A_hat equals P^T A P.
"""
import itertools

import numpy as np
import scipy.sparse as sp

from . import quadrature as quad


def hat(o, x):
    """1D Q1 hat functions on [0,1]: phi_0 = 1 - x, phi_1 = x."""
    return x if o == 1 else 1.0 - x


def hat_deriv(o):
    return 1.0 if o == 1 else -1.0


CORNERS = list(itertools.product((0, 1), (0, 1), (0, 1)))   # (ox, oy, oz), oz slowest


def corner_list():
    """The 8 corners of a cell as (ox, oy, oz), x fastest: corner c = ox + 2 oy + 4 oz."""
    return [(c & 1, (c >> 1) & 1, (c >> 2) & 1) for c in range(8)]


def prolongation(prob):
    """Sparse P (ndof x nvert): column j = vertex, row = DG dof; entries are the
    trilinear hat function of the vertex evaluated at the GLL nodes."""
    n, N = prob.n, prob.N
    rows, cols, vals = [], [], []
    z = prob.gll
    for c in range(prob.ncell):
        cx, cy, cz = prob.cell_coords(c)
        for (ox, oy, oz) in corner_list():
            v = prob.vertex_index(cx + ox, cy + oy, cz + oz)
            for i3, i2, i1 in itertools.product(range(n), range(n), range(n)):
                val = hat(ox, z[i1]) * hat(oy, z[i2]) * hat(oz, z[i3])
                if val != 0.0:
                    rows.append(c * N + i1 + n * i2 + n * n * i3)
                    cols.append(v)
                    vals.append(val)
    return sp.csr_matrix((vals, (rows, cols)), shape=(prob.ndof, prob.nvert))


def restriction(prob):
    """R = P^T."""
    return prolongation(prob).T.tocsr()


def p0_prolongation(prob):
    """Sparse P (ndof x ncell) of the P0 subspace: every dof of cell T takes
    the cell's coarse value."""
    rows = np.arange(prob.ndof)
    return sp.csr_matrix((np.ones(prob.ndof), (rows, rows // prob.N)), shape=(prob.ndof, prob.ncell))


def p0_matrix(A, prob):
    """A_hat = P^T A P for the P0 subspace (App. A.1), CSR (ncell x ncell),
    from the assembled DG matrix A."""
    P0 = p0_prolongation(prob)
    return sp.csr_matrix(P0.T @ A @ P0)


def _q1_basis(xi):
    """Values (P, 8) and reference gradients (P, 8, 3) of the 8 trilinear
    corner functions at reference points xi (P, 3)."""
    P = xi.shape[0]
    val = np.ones((P, 8))
    grad = np.ones((P, 8, 3))
    for ci, o in enumerate(corner_list()):
        for k in range(3):
            val[:, ci] *= hat(o[k], xi[:, k])
            for d in range(3):
                grad[:, ci, d] *= hat_deriv(o[k]) if d == k else hat(o[k], xi[:, k])
    return val, grad


def q1_matrix(prob):
    """A_hat by re-discretisation in Q1 (App. A.2), CSR (nvert x nvert)."""
    m = prob.m
    g, w1 = quad.gauss_legendre(m)
    pts, wts = [], []
    for q3, q2, q1 in itertools.product(range(m), range(m), range(m)):
        pts.append((g[q1], g[q2], g[q3]))
        wts.append(w1[q1] * w1[q2] * w1[q3])
    pts = np.array(pts)
    wv = np.array(wts) * np.prod(prob.h)
    val, gref = _q1_basis(pts)
    grad = gref / prob.h[None, None, :]
    rows, cols, vals = [], [], []

    def scatter(c, blk):
        cx, cy, cz = prob.cell_coords(c)
        ids = [prob.vertex_index(cx + o[0], cy + o[1], cz + o[2]) for o in corner_list()]
        for a in range(8):
            for b in range(8):
                rows.append(ids[a])
                cols.append(ids[b])
                vals.append(blk[a, b])

    for c in range(prob.ncell):
        K = prob.K[c]
        bq = prob.b_at(c, pts)
        blk = np.einsum('q,kl,qjl,qik->ij', wv, K, grad, grad, optimize=True)
        blk -= np.einsum('q,qk,qj,qik->ij', wv, bq, val, grad, optimize=True)
        cc = prob.c_of(c)
        if cc != 0.0:
            blk += cc * np.einsum('q,qj,qi->ij', wv, val, val, optimize=True)
        scatter(c, blk)
    # Dirichlet boundary terms of a^bf with gamma from the DG degree p.
    for k in range(3):
        for side in (0, 1):
            if prob.bc[2 * k + side] != 0:
                continue
            xi, wf = prob.face_xi(k, side)
            v, gr = _q1_basis(xi)
            gr = gr / prob.h[None, None, :]
            nu = np.zeros(3)
            nu[k] = 1.0 if side == 1 else -1.0
            for c in prob.boundary_cells(k, side):
                K = prob.K[c]
                delta = nu @ K @ nu
                fl = np.einsum('l,qjl->qj', K @ nu, gr, optimize=True)
                bnu = prob.b_at(c, xi) @ nu
                Phi = np.where(bnu[:, None] >= 0.0, bnu[:, None] * v, 0.0)
                gamma = prob.penalty_boundary(delta, k)
                blk = np.einsum('q,qj,qi->ij', wf, Phi, v, optimize=True)
                blk -= np.einsum('q,qj,qi->ij', wf, fl, v, optimize=True)
                blk -= np.einsum('q,qi,qj->ij', wf, fl, v, optimize=True)
                blk += gamma * np.einsum('q,qj,qi->ij', wf, v, v, optimize=True)
                scatter(c, blk)
    return sp.csr_matrix((vals, (rows, cols)), shape=(prob.nvert, prob.nvert))
