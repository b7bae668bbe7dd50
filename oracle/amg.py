"""Aggregation AMG on the Q1 coarse space.

Part of the CPU oracle (test infrastructure only, never called by the
library).

The paper uses the aggregation AMG of Blatt (DUNE-ISTL) for the subspace
correction (Algorithm 1, AMG step; Sec. 2.2) but gives none of its
parameters.  The reading taken here, fixed so that the CUDA path can be
compared with it exactly:

* aggregates are the 2x2x2 boxes of the structured vertex grid; vertex
  (vx, vy, vz) belongs to aggregate (vx//2, vy//2, vz//2);
* the tentative prolongation is piecewise constant (not smoothed);
* coarse matrices are Galerkin products A_{l+1} = P_l^T A_l P_l;
* one pre- and one post-smoothing sweep of damped Jacobi with the weight
  4 / (3 G), G = max_i sum_j |a_ij| / |a_ii| the Gershgorin bound of the
  spectrum of D^-1 A on that level (2/3 for the isotropic Q1 Laplacian,
  smaller where anisotropy or high contrast would make 2/3 unstable);
* coarsening stops once a level has at most 512 unknowns, which is solved
  exactly (dense LU);
* one V-cycle from a zero initial guess per use.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp


def aggregation(dims):
    """Piecewise-constant P (nfine x ncoarse) for 2x2x2 aggregates of a
    structured vertex grid with dims (Vx, Vy, Vz), x fastest."""
    Vx, Vy, Vz = dims
    Cx, Cy, Cz = (Vx + 1) // 2, (Vy + 1) // 2, (Vz + 1) // 2
    rows = np.arange(Vx * Vy * Vz)
    vx = rows % Vx
    vy = (rows // Vx) % Vy
    vz = rows // (Vx * Vy)
    cols = (vx // 2) + Cx * ((vy // 2) + Cy * (vz // 2))
    P = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(len(rows), Cx * Cy * Cz))
    return P, (Cx, Cy, Cz)


class AggregationAMG:
    def __init__(self, A, dims, coarse_size=512, max_levels=32):
        self.A = [sp.csr_matrix(A)]
        self.P = []
        self.dims = [tuple(dims)]
        while self.A[-1].shape[0] > coarse_size and len(self.A) < max_levels:
            P, cd = aggregation(self.dims[-1])
            self.P.append(P)
            self.A.append(sp.csr_matrix(P.T @ self.A[-1] @ P))
            self.dims.append(cd)
        self.dinv = [1.0 / Al.diagonal() for Al in self.A]
        self.omega = []
        for Al, dl in zip(self.A, self.dinv):
            G = np.max(np.asarray(abs(Al).sum(axis=1)).ravel() * np.abs(dl))
            self.omega.append(4.0 / (3.0 * G))
        self.coarse_lu = sla.lu_factor(self.A[-1].toarray())

    @property
    def nlevels(self):
        return len(self.A)

    def vcycle(self, b, level=0):
        """One V-cycle for A_level x = b from x = 0."""
        if level == len(self.A) - 1:
            return sla.lu_solve(self.coarse_lu, b)
        A, dinv, w = self.A[level], self.dinv[level], self.omega[level]
        x = np.zeros_like(b)
        x = x + w * dinv * (b - A @ x)                    # pre-smoothing
        r = b - A @ x
        xc = self.vcycle(self.P[level].T @ r, level + 1)  # coarse correction
        x = x + self.P[level] @ xc
        x = x + w * dinv * (b - A @ x)                    # post-smoothing
        return x
