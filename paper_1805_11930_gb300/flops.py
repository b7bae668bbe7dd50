"""Algorithmic floating-point operation counts of the library's kernels
(diffusion operator, b = 0, c = 0), per cell, n = p+1.  An FMA counts as 2,
any other add, multiply or divide as 1.  These are the counts of the
sum-factorised algorithm as the kernels implement it:

volume (Sec. 3.1, Stages 1-3): six 1D contractions with the n x n matrices B
    and B^T (n^4 FMA each) and three fused derivative passes Dg, pointwise
    coefficient, Dg^T (2 n^4 FMA + 3 n^3 each)            -> 24 n^4 + 9 n^3
faces, per face node: own normal derivative (n FMA), the neighbour's (n FMA,
    full operator only), the face mass matrix M1 (x) M1 on two fields
    (4 n FMA), the scatter of the derivative term (n FMA), ~20 scalar
    operations; six faces of n^2 nodes
    full operator                                         -> 84 n^3 + 120 n^2
    block diagonal D_T                                    -> 72 n^3 + 100 n^2
inner PCG iteration: one D_T apply plus three dot products and three vector
    updates and the diagonal scaling                      -> F_block + 13 n^3
smoother sweep: the defect (one full apply, skipped when the sweep starts
    from zero), residual set-up and update                -> F_full + 8 n^3
"""


def apply_full(n):
    return 24 * n ** 4 + 9 * n ** 3 + 84 * n ** 3 + 120 * n ** 2


def apply_block(n):
    return 24 * n ** 4 + 9 * n ** 3 + 72 * n ** 3 + 100 * n ** 2


def pcg_iteration(n):
    return apply_block(n) + 13 * n ** 3


def smoother_total(n, ncell, sweeps, zero_sweeps, inner_its_total):
    """FP64 operations of `sweeps` smoother launches over ncell cells, of
    which `zero_sweeps` started from u = 0, with inner_its_total inner
    iterations summed over cells and sweeps."""
    per_sweep = 8 * n ** 3 * ncell
    defect = apply_full(n) * ncell * (sweeps - zero_sweeps)
    return per_sweep * sweeps + defect + pcg_iteration(n) * inner_its_total


def hbm_bytes_apply(n, ncell, word=8):
    """Compulsory HBM bytes of one operator application: read u, write v,
    read one K value per cell."""
    return 2 * word * n ** 3 * ncell + 8 * ncell
