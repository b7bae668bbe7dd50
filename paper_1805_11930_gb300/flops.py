"""Operation counts used for the roofline figures (n = p+1, per cell).

Algorithmic count (the roofline's "achieved" numerator): the sum-factorised
operator with the gradient-only volume term, face-centric faces, an FMA
counted as 2 flops,
    F(n) = 32 n^4 + 120 n^3
(16 contractions of 2 n^4 flops; 3 owned faces x 2 sides x 20 n^3), i.e.
216 / 248 / 280 / 312 / 344 flop per dof at p = 2..6 for diffusion, and 36 n^4
instead of 32 n^4 with advection or reaction.  A block-diagonal apply D_T is
counted like a full apply.  One smoother sweep over a cell costs one apply
for its defect (none when it starts from zero) plus one apply per inner
iteration.

Kernel count (what the kernels issue, b = 0): the FP64 and double-float
kernels apply the block in the factored form D_T = (M (x) M (x) M) o
sum_d (M^-1 A_d) x_d: one fused pass of 3 n multiply-adds per element and
three mass passes of n each, 12 n^4 per cell; the full operator adds the
neighbour face values (6 n^2 face points of n multiply-adds and 8 more
operations each, 12 n^3 + 48 n^2) and their injection before the mass
passes (12 multiply-adds per element, 24 n^3): 12 n^4 + 36 n^3 + 48 n^2.
Inner-iteration vector work 13 n^3.  With advection the volume term runs at
the Gauss points (24 n^4 + 9 n^3) and the faces add the upwind flux; the
FP32 kernels keep the eight-contraction Kronecker sequence (16 n^4 per
block apply).
"""


def algorithmic_apply(n, value_terms=False):
    return (36 if value_terms else 32) * n ** 4 + 120 * n ** 3


def algorithmic_smoother(n, ncell, sweeps, zero_sweeps, inner_its_total, value_terms=False):
    """Algorithmic flops of `sweeps` smoother launches over ncell cells, of
    which zero_sweeps start from u = 0, with inner_its_total inner iterations
    summed over cells and sweeps."""
    F = algorithmic_apply(n, value_terms)
    return F * (ncell * (sweeps - zero_sweeps) + inner_its_total)


def kernel_apply_full(n, advection=False, element=True):
    """Flops one cell of a full operator apply issues, counted from the
    kernel's loops.  b = 0: the factored form (element layout: 12 n^4 +
    36 n^3 + 48 n^2), else the Kronecker volume term and line-form faces
    (16 n^4 + 84 n^3 + 120 n^2).  Advection: the Gauss-point element form
    (six interpolation passes and six derivative passes, 24 n^4; the
    pointwise flux from the per-cell separable factors of b, 21 n^3, their
    tables 60 n^2; the six faces in element passes, 156 n^3 + 210 n^2), else
    the line form (24 n^4; the pointwise flux 18 n^3 and the reaction 4 n^3;
    the faces 84 n^3 + 120 n^2)."""
    if advection:
        if element:
            return 24 * n ** 4 + 177 * n ** 3 + 270 * n ** 2
        return 24 * n ** 4 + 22 * n ** 3 + 84 * n ** 3 + 120 * n ** 2
    if element:
        return 12 * n ** 4 + 36 * n ** 3 + 48 * n ** 2
    return 16 * n ** 4 + 84 * n ** 3 + 120 * n ** 2


def kernel_apply_block(n, advection=False, element=True):
    """The same for the block D_T (no neighbour values read)."""
    if advection:
        if element:
            return 24 * n ** 4 + 165 * n ** 3 + 270 * n ** 2
        return 24 * n ** 4 + 22 * n ** 3 + 72 * n ** 3 + 100 * n ** 2
    return 12 * n ** 4 if element else 16 * n ** 4


def kernel_smoother(n, ncell, sweeps, zero_sweeps, inner_its_total):
    """Flops the b = 0 inner-PCG smoother kernels issue (FP64, factored form)
    over `sweeps` launches: a full apply per defect, a block apply plus the
    vector work per inner iteration."""
    return (kernel_apply_full(n) * ncell * (sweeps - zero_sweeps)
            + (kernel_apply_block(n) + 13 * n ** 3) * inner_its_total)


def hbm_bytes_apply(n, ncell, word=8):
    """Compulsory HBM bytes of one operator application: read u, write v,
    read one K value per cell."""
    return 2 * word * n ** 3 * ncell + 8 * ncell
