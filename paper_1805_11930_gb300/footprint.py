"""Memory footprints.

paper_model: the storage estimates of the three implementations compared in
arXiv 1805.11930 (Sec. 4.4, eqs. memory_diffusion and memory_convection), in
doubles: with M_vec = N_cell (p+1)^d, M_mat = 7 N_cell (p+1)^(2d) and
M_blockdiag = N_cell (p+1)^(2d),
  diffusion   MX  M_mat + 6 M_vec + 30 N_cell
              PMF M_blockdiag + 7 M_vec + 30 N_cell
              MF  8 M_vec + 30 N_cell
  convection  MX  M_mat + (2 n_out + 4) M_vec
              PMF M_blockdiag + (2 n_out + 4) M_vec
              MF  (2 n_out + 7) M_vec + (n_blk + 1) (p+1)^d
(the MF block term is one solver's local Krylov basis, not per cell).

library_bytes: what this library allocates for one solve (used by the
serving loop to admit requests by HBM footprint).
"""

DOUBLE = 8


def paper_model(p, ncell, problem="diffusion", variant="MF", d=3, n_out=100, n_blk=100):
    """Doubles stored by the paper's MX / PMF / MF implementations."""
    vec = ncell * (p + 1) ** d
    blk = ncell * (p + 1) ** (2 * d)
    if problem == "diffusion":
        return {"MX": 7 * blk + 6 * vec + 30 * ncell,
                "PMF": blk + 7 * vec + 30 * ncell,
                "MF": 8 * vec + 30 * ncell}[variant]
    if problem == "convection":
        return {"MX": 7 * blk + (2 * n_out + 4) * vec,
                "PMF": blk + (2 * n_out + 4) * vec,
                "MF": (2 * n_out + 7) * vec + (n_blk + 1) * (p + 1) ** d}[variant]
    raise ValueError(problem)


def matrix_bytes(p, ncell, d=3):
    """Bytes of the assembled DG matrix counted as in the paper's problem-size
    table (Sec. 4): 7 blocks of (p+1)^(2d) doubles per cell (the cell and its
    2d face neighbours; boundary cells counted alike)."""
    return DOUBLE * 7 * ncell * (p + 1) ** (2 * d)


def library_bytes(nc, p, krylov="fcg", restart=30):
    """Device bytes of one context plus the caller's f and u: per dof the
    FP64/FP32 diagonals and inverses (24 B), FP64 and FP32 V-cycle work
    vectors (40 B), Krylov vectors (CG 4, flexible CG 5, FGMRES 2m+2 FP64),
    f and u (16 B); per cell the coefficient records and corner sums (256 B);
    per vertex the AMG levels (about 300 B); the coarsest dense inverse (2 MB)."""
    nx, ny, nz = nc
    ncell = nx * ny * nz
    ndof = ncell * (p + 1) ** 3
    nvert = (nx + 1) * (ny + 1) * (nz + 1)
    kvec = {"cg": 4, "fcg": 5, "fgmres": 2 * restart + 2}[krylov]
    per_dof = 24 + 40 + 8 * kvec + 16
    return ndof * per_dof + 256 * ncell + 300 * nvert + 2 * 1024 * 1024
