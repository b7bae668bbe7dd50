"""1D quadrature rules and Lagrange bases on the unit interval [0, 1].

Part of the CPU oracle (test infrastructure only, never called by the
library).

* The DG basis is the tensor product of Lagrange polynomials whose nodes are
  the p+1 Gauss-Lobatto points (Sec. 2.1, "Gauss-Lobatto basis functions").
* Integrals use the tensor Gauss-Legendre rule with m = n = p+1 points per
  direction (Sec. 3.1, "typically m = n = p+1"); Gauss-Lobatto quadrature is
  mentioned only as future work (Sec. 5), so the current rule is Gauss.

Both rules come from numpy's Legendre routines (a library primitive); the
tests pin them to closed forms and exactness properties.
"""
import numpy as np
from numpy.polynomial import legendre as L


def gauss_legendre(m):
    """m-point Gauss-Legendre rule mapped to [0, 1]: (points, weights)."""
    x, w = L.leggauss(m)
    return 0.5 * (x + 1.0), 0.5 * w


def gauss_lobatto(n):
    """n-point Gauss-Lobatto-Legendre rule on [0, 1] (n >= 2).

    Nodes are the end points plus the roots of P'_{n-1}; weights on [-1, 1]
    are 2 / (n (n-1) P_{n-1}(x)^2), halved for [0, 1].
    """
    if n < 2:
        raise ValueError("Gauss-Lobatto needs n >= 2")
    c = np.zeros(n)
    c[-1] = 1.0                        # P_{n-1} in the Legendre basis
    interior = np.sort(np.real(L.legroots(L.legder(c)))) if n > 2 else np.zeros(0)
    x = np.concatenate(([-1.0], interior, [1.0]))
    pn = L.legval(x, c)
    w = 2.0 / (n * (n - 1) * pn ** 2)
    return 0.5 * (x + 1.0), 0.5 * w


def lagrange_values(nodes, x):
    """V[a, j] = l_j(x_a): Lagrange polynomial j of `nodes` at points x."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    V = np.ones((len(x), n))
    for j in range(n):
        for k in range(n):
            if k != j:
                V[:, j] *= (x - nodes[k]) / (nodes[j] - nodes[k])
    return V


def lagrange_derivatives(nodes, x):
    """G[a, j] = l_j'(x_a), from the product rule applied to the Lagrange
    product formula (a sum over the factor that is differentiated)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = len(nodes)
    G = np.zeros((len(x), n))
    for j in range(n):
        for l in range(n):
            if l == j:
                continue
            term = np.full(len(x), 1.0 / (nodes[j] - nodes[l]))
            for k in range(n):
                if k != j and k != l:
                    term *= (x - nodes[k]) / (nodes[j] - nodes[k])
            G[:, j] += term
    return G
