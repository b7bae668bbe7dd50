"""Seeded synthetic workloads shaped like the paper's experiments.

This module holds no arithmetic of the method: only coefficient fields,
analytic right-hand sides and boundary data, drawn with numpy's
default_rng(seed) (seed 1805 unless stated).  Both the CUDA path and the CPU
oracle receive these arrays and functions, and each side evaluates them at its
own quadrature points.

Workloads (the paper's data sets are not available, so these stand in for
them):
* poisson_sine   Poisson on the unit cube, K = 1, f = 3 pi^2 prod sin(pi x_k),
                 u = 0 on the boundary (exact u = prod sin(pi x_k)); 8^3, p = 2.
* lognormal      scalar K per cell, log K ~ N(0, 1); Gaussian source at
                 (0.75, 0.5, 0.3), width 0.1 (the source of Sec. 4.2);
                 homogeneous Dirichlet; 32^3, p = 4.
* convection     kappa = 1e-3, divergence-free rotating field
                 b = (2(1/2 - y), x - 1/2, 1/4), f such that
                 u = x(1-x) y(1-y) z(1-z) (the solution used in Sec. 4.3);
                 64^3, p = 3.
* reservoir      60 x 220 x 85 cells of 20 x 10 x 2 ft (the SPE10 grid of
                 Sec. 4.5, whose permeability data are not available);
                 diagonal K: top 35 layers log-normal per layer, bottom 50
                 layers a low-permeability background with 3-6 sinuous
                 high-permeability channels per layer, log10 K clipped to
                 [-3, 4], K_v = 0.1 K_h in channels and 1e-3 K_h elsewhere;
                 Dirichlet u = -y on the x and y planes, no-flow top/bottom;
                 p = 2.
"""
import numpy as np

SEED = 1805


def vertex_field(nc, L, fn):
    """Values of fn(x, y, z) -> (..., 3) at the grid vertices, vertex
    (vx, vy, vz) at vx + (nx+1)(vy + (ny+1) vz); shape (nvert, 3)."""
    nx, ny, nz = nc
    vz, vy, vx = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    x = vx.reshape(-1) * (L[0] / nx)
    y = vy.reshape(-1) * (L[1] / ny)
    z = vz.reshape(-1) * (L[2] / nz)
    return np.asarray(fn(x, y, z), dtype=np.float64).reshape(-1, 3)


def _zero(x, y, z):
    return np.zeros_like(x)


def poisson_sine(n=8, p=2):
    f = lambda x, y, z: 3 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    u = lambda x, y, z: np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    return dict(name=f"poisson_sine_{n}^3_p{p}", nc=(n, n, n), L=(1.0, 1.0, 1.0), p=p, bc=[0] * 6,
                K=np.ones(n ** 3), b=None, c=None, f=f, g=_zero, j=None, exact=u)


def lognormal(n=32, p=4, seed=SEED, sigma=1.0):
    rng = np.random.default_rng(seed)
    K = np.exp(sigma * rng.normal(size=n ** 3))
    f = lambda x, y, z: np.exp(-((x - 0.75) ** 2 + (y - 0.5) ** 2 + (z - 0.3) ** 2) / (2 * 0.1 ** 2))
    return dict(name=f"lognormal_{n}^3_p{p}", nc=(n, n, n), L=(1.0, 1.0, 1.0), p=p, bc=[0] * 6,
                K=K, b=None, c=None, f=f, g=_zero, j=None, exact=None)


def rotating_field(x, y, z):
    return np.stack([2 * (0.5 - y), x - 0.5, 0.25 + 0 * x], axis=-1)


def convection(n=64, p=3, kappa=1e-3):
    def u(x, y, z):
        return x * (1 - x) * y * (1 - y) * z * (1 - z)

    def f(x, y, z):
        lap = -2 * (y * (1 - y) * z * (1 - z) + x * (1 - x) * z * (1 - z) + x * (1 - x) * y * (1 - y))
        ux = (1 - 2 * x) * y * (1 - y) * z * (1 - z)
        uy = x * (1 - x) * (1 - 2 * y) * z * (1 - z)
        uz = x * (1 - x) * y * (1 - y) * (1 - 2 * z)
        b = rotating_field(x, y, z)
        return -kappa * lap + b[..., 0] * ux + b[..., 1] * uy + b[..., 2] * uz

    nc = (n, n, n)
    return dict(name=f"convection_{n}^3_p{p}", nc=nc, L=(1.0, 1.0, 1.0), p=p, bc=[0] * 6,
                K=np.full(n ** 3, kappa), b=vertex_field(nc, (1.0, 1.0, 1.0), rotating_field), c=None,
                f=f, g=_zero, j=None, exact=u)


def convection_pe(n=32, p=3, pe=2000.0, bvec=(1.0, 0.5, 0.3)):
    """Strongly convection-dominated flow of Sec. 4.3: constant b, kappa set by
    the grid Peclet number Pe = max_i |b_i| h / kappa, manufactured solution
    u = prod x_k (1 - x_k), homogeneous Dirichlet."""
    h = 1.0 / n
    kappa = max(abs(v) for v in bvec) * h / pe
    bx, by, bz = bvec

    def u(x, y, z):
        return x * (1 - x) * y * (1 - y) * z * (1 - z)

    def f(x, y, z):
        lap = -2 * (y * (1 - y) * z * (1 - z) + x * (1 - x) * z * (1 - z) + x * (1 - x) * y * (1 - y))
        ux = (1 - 2 * x) * y * (1 - y) * z * (1 - z)
        uy = x * (1 - x) * (1 - 2 * y) * z * (1 - z)
        uz = x * (1 - x) * y * (1 - y) * (1 - 2 * z)
        return -kappa * lap + bx * ux + by * uy + bz * uz

    nc = (n, n, n)
    bfield = vertex_field(nc, (1.0, 1.0, 1.0), lambda x, y, z: np.stack([0 * x + bx, 0 * x + by, 0 * x + bz], -1))
    return dict(name=f"convection_pe{int(pe)}_{n}^3_p{p}", nc=nc, L=(1.0, 1.0, 1.0), p=p, bc=[0] * 6,
                K=np.full(n ** 3, kappa), b=bfield, c=None, f=f, g=_zero, j=None, exact=u)


# Spatially varying diffusion of the paper's inhomogeneous test (Sec. 4.2):
# K(x) = sum_k P_k(x_k) n_k n_k^T with an orthonormal basis n_k and
# P_k(z) = p0_k + p2_k z^2 > 0; c(x) = gamma |x|^2 with gamma = 1e-8.
VARK_BASIS = None   # filled below: rows n_1, n_2, n_3
VARK_P0 = (1.0, 2.0, 0.5)
VARK_P2 = (3.0, 1.0, 4.0)
VARK_GAMMA = 1e-8


def _rotation(a, b, c):
    ca, sa, cb, sb, cc, sc = np.cos(a), np.sin(a), np.cos(b), np.sin(b), np.cos(c), np.sin(c)
    rz = np.array([[ca, -sa, 0], [sa, ca, 0], [0, 0, 1.0]])
    ry = np.array([[cb, 0, sb], [0, 1.0, 0], [-sb, 0, cb]])
    rx = np.array([[1.0, 0, 0], [0, cc, -sc], [0, sc, cc]])
    return rz @ ry @ rx


VARK_BASIS = _rotation(np.pi / 6, np.pi / 8, np.pi / 5).T     # rows are n_k


def vark_tensor(x, basis=None, p0=VARK_P0, p2=VARK_P2):
    """K(x) at points x (..., 3): (..., 3, 3)."""
    nb = VARK_BASIS if basis is None else np.asarray(basis)
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape[:-1] + (3, 3))
    for k in range(3):
        pk = p0[k] + p2[k] * x[..., k] ** 2
        out += pk[..., None, None] * np.outer(nb[k], nb[k])
    return out


def vark_reaction(x, gamma=VARK_GAMMA):
    x = np.asarray(x, dtype=np.float64)
    return gamma * np.sum(x * x, axis=-1)


def variable_k(n=16, p=3):
    """The inhomogeneous test of Sec. 4.2 on the unit cube: K(x), c(x) as
    above, Neumann on x = 1 with j a Gaussian at (1, 0.5, 0.5), Dirichlet
    elsewhere with g a Gaussian at (0, 0.5, 0.5) (widths 0.1), f the Gaussian
    at (0.75, 0.5, 0.3).  K_cell / c_cell: the coefficients at the cell
    centres (the diagonal of the tensor), which the preconditioner uses."""
    nc = (n, n, n)
    h = 1.0 / n
    ce = (np.arange(n) + 0.5) * h
    cz, cy, cx = np.meshgrid(ce, ce, ce, indexing="ij")
    centres = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], -1)
    Kc = vark_tensor(centres)
    gauss = lambda x0: (lambda x, y, z: np.exp(-((x - x0[0]) ** 2 + (y - x0[1]) ** 2 + (z - x0[2]) ** 2)  # noqa: E731
                                               / (2 * 0.1 ** 2)))
    return dict(name=f"variable_k_{n}^3_p{p}", nc=nc, L=(1.0, 1.0, 1.0), p=p, bc=[0, 1, 0, 0, 0, 0],
                K=np.stack([Kc[:, 0, 0], Kc[:, 1, 1], Kc[:, 2, 2]], -1), b=None, c=vark_reaction(centres),
                f=gauss((0.75, 0.5, 0.3)), g=gauss((0.0, 0.5, 0.5)), j=gauss((1.0, 0.5, 0.5)), exact=None,
                K_fn=vark_tensor, c_fn=vark_reaction,
                vark=dict(basis=VARK_BASIS, p0=VARK_P0, p2=VARK_P2, gamma=VARK_GAMMA))


def reservoir_permeability(nc=(60, 220, 85), seed=SEED):
    """Diagonal K (ncell, 3) of the channelised layered field."""
    nx, ny, nz = nc
    rng = np.random.default_rng(seed)
    logk = np.zeros((nz, ny, nx))
    chan = np.zeros((nz, ny, nx), dtype=bool)
    top = min(35, nz)
    for lz in range(nz):
        layer = nz - 1 - lz           # layer 0 is the top (largest z)
        if layer < top:
            mu = rng.uniform(-1.0, 3.0)
            logk[lz] = rng.normal(mu, 0.5, size=(ny, nx))
        else:
            logk[lz] = rng.normal(-1.5, 0.7, size=(ny, nx))
            yy = np.arange(ny)[:, None]
            xx = np.arange(nx)[None, :]
            for _ in range(rng.integers(3, 7)):
                x0 = rng.uniform(0, nx)
                amp = rng.uniform(3, 12)
                lam = rng.uniform(40, 160)
                ph = rng.uniform(0, 2 * np.pi)
                width = rng.uniform(3, 8)
                xc = x0 + amp * np.sin(2 * np.pi * yy / lam + ph)
                mask = np.abs(xx - xc) < width / 2
                logk[lz][mask] = rng.normal(3.0, 0.4, size=int(mask.sum()))
                chan[lz] |= mask
    logk = np.clip(logk, -3.0, 4.0)
    kh = 10.0 ** logk
    kv = np.where(chan, 0.1 * kh, 1e-3 * kh)
    K = np.stack([kh.reshape(-1), kh.reshape(-1), kv.reshape(-1)], axis=1)
    return K


def reservoir(nc=(60, 220, 85), p=2, seed=SEED):
    L = (20.0 * nc[0], 10.0 * nc[1], 2.0 * nc[2])
    return dict(name=f"reservoir_{nc[0]}x{nc[1]}x{nc[2]}_p{p}", nc=tuple(nc), L=L, p=p, bc=[0, 0, 0, 0, 1, 1],
                K=reservoir_permeability(nc, seed), b=None, c=None, f=_zero,
                g=lambda x, y, z: -y, j=_zero, exact=None)


def random_dg_vector(ndof, seed=SEED, low=-1.0, high=1.0):
    return np.random.default_rng(seed).uniform(low, high, size=ndof)


def evaluate(fn, xyz):
    """fn at an (..., 3) array of points; None -> None."""
    if fn is None:
        return None
    return np.asarray(fn(xyz[..., 0], xyz[..., 1], xyz[..., 2]), dtype=np.float64)
