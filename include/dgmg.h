/*
 * dgmg.h -- C ABI of the GB300 matrix-free hybrid multigrid library for
 * SIPG / upwind Discontinuous Galerkin discretisations on hexahedral grids
 * (Bastian, Mueller, Muething, Piatkowski, arXiv 1805.11930).
 *
 * Problem (Sec. 2, eq. linearproblem):  div(b u - K grad u) + c u = f on the
 * box [0,Lx]x[0,Ly]x[0,Lz], u = g on Dirichlet planes, (b u - K grad u).nu = j
 * on Neumann planes.  Discretisation (Sec. 2.1): weighted SIPG with upwind flux,
 * tensor-product Q_p Gauss-Lobatto nodal basis, Gauss quadrature with p+1 points
 * per direction, penalty alpha p (p+2) <delta-,delta+> |F| / min|T| with
 * alpha = 1.25.
 *
 * Conventions shared by every call:
 *  - A uniform nx x ny x nz grid; cell (cx,cy,cz) has index cx + nx (cy + ny cz).
 *  - A DG vector is cell-major: n^3 values per cell (n = p+1), dof (i1,i2,i3)
 *    at offset i1 + n i2 + n^2 i3 inside its cell.  Unpadded, contiguous.
 *  - A vertex (Q1) vector has (nx+1)(ny+1)(nz+1) values, vertex (vx,vy,vz) at
 *    vx + (nx+1)(vy + (ny+1) vz).
 *  - Boundary planes are ordered -x,+x,-y,+y,-z,+z; bc[i] = 0 Dirichlet,
 *    1 Neumann.
 *  - Pointers marked "device" are CUDA device pointers owned by the caller,
 *    which must stay valid until the work queued on the context's stream has
 *    finished.  Pointers marked "host" are read or written before the call
 *    returns.  The library owns the context, its copies of mesh and
 *    coefficients, and its workspace.
 *  - FP64 vectors are double, FP32 vectors float; `prec` selects which.
 *  - Every call is stream-ordered on the stream given to dgmg_create and
 *    returns a dgmg_status; on an error nothing is queued unless stated.
 *    dgmg_last_error() gives the message.  A context must not be used from
 *    two threads at once; separate contexts are independent.
 */
#ifndef DGMG_H
#define DGMG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgmg_ctx dgmg_ctx;

typedef enum {
  DGMG_OK = 0,
  DGMG_ERR_ARG = 1,            /* invalid argument; nothing modified            */
  DGMG_ERR_OOM = 2,            /* device allocation failed                      */
  DGMG_ERR_CUDA = 3,           /* CUDA runtime error (message has the details)  */
  DGMG_ERR_STATE = 4,          /* call needs set_mesh / set_coefficients first  */
  DGMG_ERR_NOT_CONVERGED = 5,  /* solve hit maxit; u holds the last iterate     */
  DGMG_ERR_BREAKDOWN = 6,      /* Krylov breakdown (p^T A p <= 0, zero norm)    */
  DGMG_ERR_TIMEOUT = 7         /* reserved: a bounded device wait gave up       */
} dgmg_status;

/* DGMG_DF64: FP64 vectors in memory, arithmetic in double-float (pairs of
 * FP32 numbers, about 48 significant bits): FP64-level accuracy on the FP32
 * pipe, which GB300 issues 62x faster than FP64.  Built for diffusion (b = 0)
 * with p <= 6, and in the smoothers with the inner PCG or the stored inverses
 * (DIRECT, which then shares the FP64 smoothers' double-float pairs); other
 * combinations return DGMG_ERR_ARG. */
typedef enum { DGMG_FP64 = 0, DGMG_FP32 = 1, DGMG_DF64 = 2 } dgmg_prec;
typedef enum { DGMG_KRYLOV_CG = 0, DGMG_KRYLOV_FCG = 1, DGMG_KRYLOV_FGMRES = 2 } dgmg_krylov;
/* Block solves of the smoother: inner PCG or GMRES on the matrix-free block,
 * preconditioned by diag(D_T) (Sec. 2.2.1, 3.2); GMRES_TRIDIAG: GMRES
 * preconditioned by the tridiagonal part of D_T in the cell's lexicographic
 * dof order (x fastest), solved by the Thomas algorithm, for strongly
 * convection-dominated blocks (Sec. 3.2, 4.3; its factors, 3 n^3 values per
 * cell and precision, are built on first use); or DIRECT: multiplication by
 * the explicit inverse of D_T stored on the device (the partially matrix-free
 * variant, Sec. 4.1; see dgmg_block_inverse). */
typedef enum {
  DGMG_INNER_PCG = 0,
  DGMG_INNER_GMRES = 1,
  DGMG_INNER_DIRECT = 2,
  DGMG_INNER_GMRES_TRIDIAG = 3
} dgmg_inner;
/* Coarse correction of the V-cycle: the conforming Q1 subspace with AMG
 * (Sec. 2.2.2-2.2.3, the default), none, or the piecewise-constant P0
 * subspace with AMG on its 7-point matrix (App. A.1; the paper's choice for
 * its SPE10 runs, Sec. 4.4; built on first use). */
typedef enum { DGMG_COARSE_AMG = 0, DGMG_COARSE_NONE = 1, DGMG_COARSE_P0 = 2 } dgmg_coarse;
typedef enum { DGMG_SMOOTHER_JACOBI = 0, DGMG_SMOOTHER_SSOR = 1 } dgmg_smoother;
/* Outer stopping rule.  RESIDUAL: ||r_k||_2 <= rtol ||r_0||_2.  ENERGY: the
 * estimate of Strakos and Tichy (BIT 45, 2005, Sec. 3.1) used in Sec. 4.4:
 * in PCG, ||e_k||_A^2 - ||e_{k+d}||_A^2 = sum_{j=k}^{k+d-1} alpha_j (r_j, z_j),
 * so after iteration k+d that sum estimates ||e_k||_A^2 (from below) and
 * sum_{j<k+d} alpha_j (r_j, z_j) estimates ||x - x_0||_A^2; the solve stops at
 * the first k whose relative estimate is <= rtol and returns x_{k+d}, with
 * iterations = k (the d run-ahead iterations are in iterations_run). */
typedef enum { DGMG_STOP_RESIDUAL = 0, DGMG_STOP_ENERGY = 1 } dgmg_stop;

/* Options of the hybrid V-cycle (Algorithm 1) and of the outer Krylov solve. */
typedef struct {
  int krylov;          /* dgmg_krylov: CG (Sec. 4.2), flexible CG, FGMRES (Sec. 4.3) */
  int restart;         /* FGMRES restart length (default 30)                       */
  double rtol;         /* outer stop: ||r||_2 <= rtol ||r_0||_2 (default 1e-8)     */
  int maxit;           /* outer iteration cap (default 500)                        */
  int smoother_prec;   /* dgmg_prec of the V-cycle's DG part (smoother, residual)  */
                       /* FP64, FP32 or DF64 (FP64 vectors, double-float math)   */
  double omega;        /* block-Jacobi damping (Algorithm 2), default 0.8          */
  int npre, npost;     /* smoothing sweeps (default 1, 1)                          */
  double eps_inner;    /* block solve: reduce ||d - D_T x||_2 by eps (default 1e-2) */
  int maxit_inner;     /* block solve iteration cap (default n^3 when <= 0)        */
  int inner;           /* dgmg_inner: PCG (symmetric), GMRES (b != 0),             */
                       /* GMRES_TRIDIAG (convection-dominated) or DIRECT          */
  int inner_restart;   /* inner GMRES restart (default 12)                         */
  int coarse;          /* dgmg_coarse: Q1 + AMG correction, none, or P0 + AMG     */
  int timing;          /* 1: time the solve's components with CUDA events (stats) */
  int coarse_cycles;   /* AMG V-cycles per coarse correction, iterated on the     */
                       /* coarse residual (default 1)                             */
  int smoother;        /* dgmg_smoother: block-Jacobi (Algorithm 2, default) or   */
                       /* multicolour block-SSOR (one forward + one backward pass */
                       /* over the 8 parity colours per sweep)                    */
  int apply_prec;      /* dgmg_prec of the outer operator applications: FP64      */
                       /* (default) or DF64; the final residual check is FP64    */
  int graph;           /* 1: capture the preconditioner into a CUDA graph and     */
                       /* replay it (needs a non-default stream; off when timing) */
  int stop;            /* dgmg_stop: relative residual (default) or the energy-   */
                       /* norm error estimate (CG and flexible CG only)           */
  int delay;           /* error bandwidth d of the energy-norm estimate (def. 4)  */
} dgmg_solve_opts;

typedef struct {
  int iterations;       /* outer iterations                                       */
  int converged;        /* 1 if the recomputed FP64 residual (stop = RESIDUAL) or   */
                        /* the energy-norm estimate (stop = ENERGY) met rtol      */
  double rel_residual;  /* ||f - A u||_2 / ||f - A u_0||_2, recomputed in FP64    */
  double inner_mean;    /* mean inner block-solve iterations over all cells/sweeps */
  int inner_max;        /* maximum inner iterations seen                          */
  double ms_total;      /* wall time of the solve (host clock, stream synced)    */
  long long inner_its_total;  /* sum over cells and sweeps of inner iterations     */
  long long sweeps;           /* block-Jacobi sweeps (one smoother launch each)    */
  long long zero_sweeps;      /* of which started from u = 0 (no defect apply)     */
  long long applies;          /* full-operator applications (one launch each)      */
  long long kernel_launches;  /* all kernels this library launched in the solve    */
  double ms_smooth;     /* device time of the smoother launches (opts->timing)    */
  double ms_apply;      /* device time of the operator launches (opts->timing)    */
  double energy_estimate; /* last relative energy-norm estimate (stop = ENERGY)   */
  int iterations_run;   /* outer iterations performed (iterations + d for ENERGY)  */
  /* Device time by component with opts->timing (CUDA events on the context's */
  /* stream; the V-cycle then runs eagerly, not from a graph):               */
  double ms_transfer;   /* restrictions to and prolongations from the coarse space */
  double ms_coarse;     /* coarse corrections (AMG cycles, or the direct solve)  */
  double ms_krylov;     /* the rest of the solve: outer Krylov vector updates,    */
                        /* dot products, precision conversions, counters        */
  double ms_device;     /* the whole solve, first to last kernel                  */
  double inner_std;     /* standard deviation of the inner iteration counts over  */
                        /* all cells and sweeps (with inner_mean, inner_max: the  */
                        /* statistics reported with the inner solves, Sec. 4.2)  */
} dgmg_solve_stats;

/* Fill *opts with the defaults listed above. */
void dgmg_default_opts(dgmg_solve_opts* opts);

/* Create a context on CUDA `device`; `cuda_stream` is a cudaStream_t (NULL =
 * the legacy default stream), used but not owned.  *out receives the context
 * (owned by the caller until dgmg_destroy), or NULL on failure:
 * DGMG_ERR_ARG for out == NULL or a device that does not exist (also when no
 * GPU is visible), DGMG_ERR_CUDA when the device tables or the small
 * reduction buffers cannot be set up. */
dgmg_status dgmg_create(dgmg_ctx** out, int device, void* cuda_stream);

/* Synchronise the context's stream, free every device and pinned buffer and
 * captured graph of the context, and the context itself.  NULL:
 * DGMG_ERR_ARG.  The caller's stream and vectors are not touched. */
dgmg_status dgmg_destroy(dgmg_ctx* ctx);

/* Message of the last failed call on ctx (owned by ctx, valid until its next
 * call); "null context" for NULL. */
const char* dgmg_last_error(const dgmg_ctx* ctx);

/* Grid and degree (Sec. 2.1, uniform axis-parallel hexahedra): 1 <= p <= 8,
 * n* >= 1, L* > 0, bc[6] in {0,1} (host).  Discards coefficients and
 * workspace of an earlier mesh. */
dgmg_status dgmg_set_mesh(dgmg_ctx* ctx, int nx, int ny, int nz, double lx, double ly,
                          double lz, int p, const int bc[6]);

/* Penalty parameter alpha of gamma_F = alpha p (p+2) <delta-,delta+> / h on
 * interior faces and alpha p (p+2) delta / h on Dirichlet faces (Sec. 2.1;
 * default 1.25, the paper's value).  The context keeps it across meshes; it
 * enters the operator, diag(D_T), the coarse matrices and the right-hand side
 * built by the next dgmg_set_coefficients / dgmg_set_variable_coefficients.
 * alpha finite and > 0, else DGMG_ERR_ARG; DGMG_ERR_STATE once the current
 * mesh has coefficients (set the penalty before them). */
dgmg_status dgmg_set_penalty(dgmg_ctx* ctx, double alpha);

/* Coefficients, piecewise constant per cell except b (Sec. 2, eq.
 * linearproblem; Sec. 4.2 evaluates K and c at cell centres in the
 * preconditioner).
 *   K: host, ncell*kdim values > 0; kdim 1 = scalar, 3 = diagonal (Kxx,Kyy,Kzz).
 *   b_vertex: host, 3*nvert values (bx,by,bz per vertex) of a continuous
 *     trilinear advection field, or NULL for b = 0.
 *   c_cell: host, ncell values, or NULL for c = 0.
 * Also computes diag(D_T) and the Q1 coarse matrix and AMG hierarchy (setup,
 * Sec. 2.2.3 and App. A.2).  Synchronises the stream. */
dgmg_status dgmg_set_coefficients(dgmg_ctx* ctx, const double* K, int kdim,
                                  const double* b_vertex, const double* c_cell);

/* Sizes of the current mesh: DG dofs, vertices, cells, volume quadrature
 * points (ncell (p+1)^3) and boundary-face quadrature points over all six
 * planes (2 (ny nz + nx nz + nx ny) (p+1)^2).  Host outputs, each may be
 * NULL.  DGMG_ERR_STATE without a mesh. */
dgmg_status dgmg_sizes(const dgmg_ctx* ctx, long long* ndof, long long* nvert, long long* ncell,
                       long long* nvol_qp, long long* nface_qp);

/* Physical coordinates (x,y,z interleaved, host) of the quadrature points at
 * which dgmg_assemble_rhs expects data.  Volume: cell-major, point
 * q1 + m q2 + m^2 q3 within a cell.  Faces: planes -x,+x,-y,+y,-z,+z; within a
 * plane normal to axis k with tangential axes a < b, cells ordered ca + n_a cb,
 * points qa + m qb within a cell face.  The points are the tensor Gauss rule
 * with m = p + 1 points per direction mapped to each cell (Sec. 3.1).  Either
 * pointer may be NULL; sizes from dgmg_sizes (3 doubles per point).
 * DGMG_ERR_STATE without a mesh. */
dgmg_status dgmg_quadrature_points(const dgmg_ctx* ctx, double* vol_xyz, double* face_xyz);

/* Right-hand side f_i = l_h(psi_i) (Sec. 2.1, eq. rhs) from values at the
 * quadrature points of dgmg_quadrature_points (all host, FP64):
 * f_qp (nvol_qp), g_qp and j_qp (nface_qp, read only on Dirichlet resp.
 * Neumann planes; NULL = 0).  rhs: device FP64, ndof. */
dgmg_status dgmg_assemble_rhs(dgmg_ctx* ctx, const double* f_qp, const double* g_qp,
                              const double* j_qp, double* rhs);

/* v = A u, matrix-free and sum-factorised (Sec. 3.1: volume terms by 1D
 * contractions to the Gauss points and back; interior and boundary face terms
 * of eq. bilinear_form_split).  u, v: device, ndof values of `prec`; u != v. */
dgmg_status dgmg_apply(dgmg_ctx* ctx, const void* u, void* v, dgmg_prec prec);

/* v = D u with D the block diagonal, D_T u_T = A^v_TT u_T + own-side face
 * terms (Sec. 3.2, eq. block_diag_apply).  u, v: device, ndof; u != v. */
dgmg_status dgmg_block_apply(dgmg_ctx* ctx, const void* u, void* v, dgmg_prec prec);

/* diag(D_T) of every cell (Sec. 3.2, the inner preconditioner), device, ndof. */
dgmg_status dgmg_block_diagonal(dgmg_ctx* ctx, void* diag, dgmg_prec prec);

/* nsweep block-Jacobi sweeps (Algorithm 2): d = f - A u; solve D_T x_T = d_T
 * per cell matrix-free (inner = PCG with 1/diag(D_T), or right-preconditioned
 * GMRES(inner_restart)) until ||d_T - D_T x_T||_2 <= eps ||d_T||_2 or maxit
 * iterations (maxit <= 0 means n^3); u += omega x.  One fused kernel per sweep.
 * f, u: device, ndof, `prec`; u is updated in place.  inner_its: device int
 * array of ncell receiving the last sweep's per-cell iteration counts, or
 * NULL. */
dgmg_status dgmg_block_smooth(dgmg_ctx* ctx, const void* f, void* u, int nsweep, double omega,
                              double eps, int maxit, int inner, int inner_restart,
                              dgmg_prec prec, int* inner_its);

/* nsweep multicolour block-SOR passes (symmetric = 0) or block-SSOR sweeps
 * (symmetric = 1: a forward then a backward pass), the data-parallel form of
 * the successive block over-relaxation of Algorithm 3 and of block-SSOR
 * (Sec. 2.2.1): cells are ordered by colour kx + 2 ky + 4 kz, (kx,ky,kz) the
 * parities of the cell indices; cells of one colour share no face, so each
 * colour is updated in place in one launch from the current values of the
 * other colours: d_T = f_T - sum_T' A_TT' u_T', D_T x_T = d_T solved as in
 * dgmg_block_smooth, u_T += omega x_T.  The result differs from a
 * lexicographic sweep (another ordering).  Arguments as dgmg_block_smooth;
 * u is updated in place. */
dgmg_status dgmg_block_sor(dgmg_ctx* ctx, const void* f, void* u, int nsweep, double omega, double eps,
                           int maxit, int inner, int inner_restart, int symmetric, dgmg_prec prec,
                           int* inner_its);

/* r_hat = R r with R = P^T, the Q1 restriction (Sec. 2.2.2).  r: device DG
 * vector of `prec`; r_hat: device FP64 vertex vector (overwritten). */
dgmg_status dgmg_restrict(dgmg_ctx* ctx, const void* r, double* r_hat, dgmg_prec prec);

/* u += P u_hat, Q1 prolongation by injection, (P|_T)_ij = psi_hat_j(zeta_i)
 * (Sec. 2.2.2).  u_hat: device FP64 vertex vector; u: device DG vector. */
dgmg_status dgmg_prolong_add(dgmg_ctx* ctx, const double* u_hat, void* u, dgmg_prec prec);

/* The Q1 matrix A_hat by re-discretisation (Sec. 2.2.3, App. A.2) as a 27-point
 * stencil: stencil[v*27 + (dx+1) + 3(dy+1) + 9(dz+1)] = A_hat(v, v+(dx,dy,dz))
 * (0 outside the grid).  stencil: host, 27*nvert doubles. */
dgmg_status dgmg_coarse_matrix(const dgmg_ctx* ctx, double* stencil);

/* u_hat = one aggregation-AMG V-cycle on A_hat from zero (Algorithm 1, AMG step):
 * 2x2x2 vertex aggregates, piecewise-constant transfer, Galerkin levels, one
 * pre- and post-sweep of damped Jacobi with the per-level weight 4/(3G), G the
 * Gershgorin bound max_i sum_j |a_ij|/|a_ii| of D^-1 A (2/3 for the isotropic
 * Q1 Laplacian), dense solve below 512 unknowns.
 * r_hat, u_hat: device FP64 vertex vectors, distinct. */
dgmg_status dgmg_coarse_cycle(dgmg_ctx* ctx, const double* r_hat, double* u_hat);

/* The piecewise-constant subspace P0 (Sec. 2.2.2, App. A.1): P|_T = 1, so
 * r_hat_T = sum of the cell's n^3 values of r (R = P^T) and u_T += u_hat_T.
 *   r, u: device DG vectors of `prec` (FP64 or FP32);
 *   r_hat, u_hat: device FP64 cell vectors (ncell values, cells x fastest).
 * The sums run one warp per cell in a fixed order. */
dgmg_status dgmg_restrict_p0(dgmg_ctx* ctx, const void* r, double* r_hat, dgmg_prec prec);
dgmg_status dgmg_prolong_add_p0(dgmg_ctx* ctx, const double* u_hat, void* u, dgmg_prec prec);

/* A_hat = P^T A P of the P0 subspace by re-discretisation (App. A.1): per
 * cell c |T|, on interior faces the penalty alpha p (p+2) <K_d^-, K_d^+> / h_d
 * times |F| (diagonal +, face neighbour -) and the upwind flux split by the
 * sign of b.n (outflow on the diagonal, inflow to the neighbour), on
 * Dirichlet faces alpha p (p+2) K_d / h_d |F| and the outflow; face
 * integrals of the upwind parts with the DG rule.  stencil: host, 27 * ncell
 * doubles in the layout of dgmg_coarse_matrix on the cell grid (7 non-zero
 * entries per row).  Builds the P0 hierarchy if needed. */
dgmg_status dgmg_coarse_matrix_p0(dgmg_ctx* ctx, double* stencil);

/* u_hat = one aggregation-AMG V-cycle on the P0 A_hat from zero (the coarse
 * correction of Algorithm 1 on the P0 subspace, Sec. 2.2.2), as
 * dgmg_coarse_cycle does on Q1.  r_hat, u_hat: device FP64 cell vectors,
 * distinct. */
dgmg_status dgmg_coarse_cycle_p0(dgmg_ctx* ctx, const double* r_hat, double* u_hat);

/* One hybrid V-cycle (Algorithm 1) for A u = f starting from the u given
 * (pass zeros for the preconditioner form): presmooth, residual, restrict,
 * AMG, prolongate-add, postsmooth, with opts (NULL = defaults).  The DG part
 * runs in opts->smoother_prec, the coarse part in FP64.  f, u: device FP64. */
dgmg_status dgmg_vcycle(dgmg_ctx* ctx, const double* f, double* u, const dgmg_solve_opts* opts);

/* Solve A u = f to ||r||_2 <= rtol ||r_0||_2 with CG, flexible CG or
 * right-preconditioned flexible GMRES(restart), preconditioned by one V-cycle
 * (Sec. 4.2, 4.3).  Outer vectors, dot products and the final residual check
 * are FP64.  f: device FP64; u: device FP64, initial guess in, solution out.
 * stats: host or NULL.  Synchronises the stream.  A non-finite initial
 * residual (NaN or Inf in f or u) returns DGMG_ERR_ARG before the first
 * iteration, u unchanged; NOT_CONVERGED and BREAKDOWN leave the last iterate
 * in u.  The context stays usable after any of these. */
dgmg_status dgmg_solve(dgmg_ctx* ctx, const double* f, double* u, const dgmg_solve_opts* opts,
                       dgmg_solve_stats* stats);

/* Spatially varying coefficients of the paper's inhomogeneous test (Sec. 4.2):
 * K(x) = sum_k (p0_k + p2_k x_k^2) n_k n_k^T with an orthonormal basis n_k
 * and c(x) = gamma (x_1^2 + x_2^2 + x_3^2), b = 0.  The outer operator (the
 * Krylov solver's applications, its final residual, dgmg_apply in FP64)
 * evaluates K and c at every quadrature point: the volume term with the full
 * tensor at the Gauss points, the face terms with K(x) at the face Gauss
 * points (K is continuous, so both traces see the same K: weights 1/2,
 * delta = nu^T K nu, gamma_F = alpha p (p+2) delta / h_d point by point) and
 * the full K grad v . n including its tangential derivatives.  Everything in
 * the preconditioner uses the coefficients at the cell centres, as the paper
 * does: this call sets them (the diagonal of K(x_T), c(x_T)) through
 * dgmg_set_coefficients, so the block smoother, its diagonals, stored blocks,
 * the coarse spaces and AMG are those of the cell-centre problem.
 * dgmg_assemble_rhs afterwards uses K(x) in the Dirichlet terms.
 *   basis: host, 9 values, rows n_1, n_2, n_3 (orthonormal to 1e-12);
 *   p0, p2: host, 3 values each, p0 > 0, p2 >= 0; gamma >= 0.
 * The outer operator is FP64 only: dgmg_apply in FP32 or DF64 and solves with
 * apply_prec = DF64 return DGMG_ERR_ARG.  dgmg_set_coefficients and
 * dgmg_set_mesh turn the variable operator off again.  Synchronises. */
dgmg_status dgmg_set_variable_coefficients(dgmg_ctx* ctx, const double* basis, const double* p0, const double* p2,
                                           double gamma);

/* Explicit inverse of every diagonal block D_T (the (T,T) part of A: volume
 * terms and the own-side face terms), for the partially matrix-free smoother
 * (PMF, Sec. 4.1: the paper stores a factorisation of D_T and solves with it;
 * this library stores D_T^-1 itself, so that a block solve is one dense
 * matrix-vector product streamed from HBM instead of two triangular solves).
 *
 * Built on the device: column j of D_T is the block operator applied to the
 * unit vector e_j (n^3 block applications per cell), then each block is
 * inverted by Gauss-Jordan elimination with partial pivoting in FP64, one
 * thread block per cell: for p <= 4 with the block in shared memory, for
 * p >= 5 with the block in global memory and the pivot steps taken in panels
 * of 16 columns (the same operations on every element, so the same inverse).
 * For FP64 smoothers
 * the inverse is kept as double-float pairs (hi, lo: about 48 significant
 * bits) and the block solve runs in double-float arithmetic (GB300's FP64
 * pipe would bound a FP64 product); for FP32 smoothers it is rounded to FP32.
 * The smoothers with inner = DGMG_INNER_DIRECT use the copy of their
 * precision (built on first use when this call was not made).  Storage per
 * precision: ncell n^3 ld values of 8 (FP64) or 4 (FP32) bytes, ld = n^3
 * rounded up to a multiple of 8 (p = 2: 6.9 KB per cell for FP64, p = 4:
 * 128 KB, p = 6: 0.94 MB, p = 8: 4.3 MB), plus a FP64 temporary of the same
 * size during the set-up.  dgmg_set_coefficients and dgmg_set_mesh drop it.
 *   prec: FP64 or FP32 (DF64: DGMG_ERR_ARG);
 *   out: device buffer of ncell n^6 values of prec receiving a copy, or NULL;
 *        block T at out + T n^6, column-major: (D_T^-1)_{ij} at i + j n^3
 *        (FP64: hi + lo of the stored pairs).
 * A singular block: DGMG_ERR_ARG with nothing stored; allocation failure:
 * DGMG_ERR_OOM.
 * Synchronises the stream. */
dgmg_status dgmg_block_inverse(dgmg_ctx* ctx, dgmg_prec prec, void* out);

/* Launch shape of the warp-per-cell operator and smoother kernels.  Each warp
 * owns whole cells and no two warps share data, so the warps per block (1, 2,
 * 4 or 8) change only speed, never a result bit.  The best value depends on
 * order, precision and how many blocks fit per SM, which is why the library
 * times it instead of fixing it (the paper tunes its kernels to one CPU by
 * hand; Sec. 3.3).
 *
 * dgmg_set_launch_shape sets the warps per block used by dgmg_apply /
 * dgmg_block_apply (wpb_apply) and by the inner-PCG smoother kernels of
 * dgmg_block_smooth, dgmg_block_sor, dgmg_vcycle and dgmg_solve (wpb_smooth)
 * for arithmetic `prec`; 0 restores the default of 4.  A value whose shared
 * memory does not fit is halved at launch.  Other values: DGMG_ERR_ARG.
 * The setting belongs to the current mesh: dgmg_set_mesh resets it. */
dgmg_status dgmg_set_launch_shape(dgmg_ctx* ctx, dgmg_prec prec, int wpb_apply, int wpb_smooth);

/* Work layouts of the operator and inner-PCG smoother kernels: how a warp's
 * lanes share the work of its cells.  All compute the same operator (exact
 * rewritings of the operator of Sec. 2.1 and the block of eq.
 * block_diag_apply, with Sec. 3.1's sum factorisation), so results agree to
 * rounding; within one layout the warps per block change no result bit.
 *   LINE     each lane a line of n values of its cell; values in shared
 *            memory.  b = 0: eight Kronecker contractions per block apply
 *            (volume tensor form) and line-form face passes; b != 0: the
 *            three stages at the Gauss points along lines, each face's upwind
 *            flux in its own line passes.
 *   ELEMENT  each lane single output elements; values in shared memory.
 *            b = 0: the block as (M (x) M (x) M) o sum_d (M^-1 A_d) x_d (one
 *            fused pass, three mass passes), the neighbour face values added
 *            before the mass passes; b != 0: the three stages at the Gauss
 *            points in element passes, all six faces (diffusion terms and
 *            upwind flux) together in element passes.
 *   PLANE    FP32, b = 0 and p <= 4 only: each lane one z-plane of a cell in
 *            registers, the factored form with the x and y contractions in
 *            registers and the z contractions through shared memory; used for
 *            the operator and the Jacobi sweep (a block-SOR colour takes LINE).
 * AUTO selects the default of the precision, order and kernel: b = 0: ELEMENT
 * for FP64 and DF64; in FP32 LINE for the operator and PLANE for the smoother
 * with p <= 4 (else LINE); b != 0: ELEMENT for FP64 at p = 4..6, else
 * LINE (the faster forms measured on GB300). */
typedef enum {
  DGMG_LAYOUT_AUTO = 0,
  DGMG_LAYOUT_LINE = 1,
  DGMG_LAYOUT_ELEMENT = 2,
  DGMG_LAYOUT_PLANE = 3
} dgmg_layout;

/* Sets the layouts of the operator (layout_apply: dgmg_apply,
 * dgmg_block_apply and the operators inside solves) and of the inner-PCG
 * smoother (layout_smooth; also the defect of the stored-inverse sweep) for
 * arithmetic `prec`.  DGMG_ERR_ARG for values outside dgmg_layout or PLANE
 * where it does not exist (FP64, DF64, p > 4, b != 0); DGMG_ERR_STATE before
 * dgmg_set_mesh.  The setting belongs to the current mesh: dgmg_set_mesh
 * resets it to AUTO. */
dgmg_status dgmg_set_layout(dgmg_ctx* ctx, dgmg_prec prec, int layout_apply, int layout_smooth);

/* The layouts in use for arithmetic `prec` (AUTO resolved to the default).
 * layout_apply, layout_smooth: host ints, or NULL.  DGMG_ERR_STATE before
 * dgmg_set_mesh. */
dgmg_status dgmg_get_layout(const dgmg_ctx* ctx, dgmg_prec prec, int* layout_apply, int* layout_smooth);

/* Times every layout that exists for arithmetic `prec` and order p (LINE and
 * ELEMENT, plus PLANE for FP32 with p <= 4 and b = 0) with every warps-per-block
 * candidate (1, 2, 4, 8), for the operator kernel and for one block-Jacobi
 * sweep with the default inner solver (PCG; GMRES(12) with advection; eps
 * 1e-2, from u = 0 with f = 1), on the current mesh
 * and coefficients, `reps` timed launches each after one warm-up (reps <= 0
 * means 3), with CUDA events on the context's stream, and keeps the fastest
 * pair of each through dgmg_set_layout and dgmg_set_launch_shape.
 * wpb_apply, wpb_smooth: host ints receiving the warps per block, or NULL
 * (dgmg_get_layout gives the layouts).  Allocates three DG vectors for the
 * duration of the call and synchronises the stream.  DGMG_ERR_ARG for DF64
 * where dgmg_apply rejects it, DGMG_ERR_STATE before dgmg_set_coefficients. */
dgmg_status dgmg_autotune(dgmg_ctx* ctx, dgmg_prec prec, int reps, int* wpb_apply, int* wpb_smooth);

/* ------------------------------------------------------------------ batched solves
 * A batch serves several requests of one polynomial order at once: the outer
 * CG (or flexible CG) of every member runs in lockstep on the batch's stream,
 * and each step of an outer iteration (operator, dot products, scalar and
 * vector updates, the V-cycle's block-Jacobi sweeps, residual, restriction
 * and prolongation) is one kernel launch over the cells or values of all
 * running members, with each member's Krylov scalars (alpha, beta, residual
 * norms, stop flag) kept in device memory.  An iteration therefore needs no
 * host round trip; on a stream other than the legacy default stream it is
 * captured into a CUDA graph on its second use with the same members and
 * replayed.  The AMG cycles on the members' Q1 grids run
 * member by member inside the same iteration.  Per member the arithmetic is
 * that of dgmg_solve with the batch's options (the same kernels and the same
 * reduction order of every dot product), so a request's iterates do not
 * depend on the other members (Sec. 4.2's solver; the batching is a serving
 * device with no counterpart in the paper). */
typedef struct dgmg_batch dgmg_batch;

/* Maximum number of members of a batch. */
#define DGMG_BATCH_MAX 16

/* Creates an empty batch on `device` whose work runs on `cuda_stream` (NULL:
 * the default stream), with the solve options every member uses: krylov CG or
 * FCG, smoother_prec, apply_prec (FP64 or DF64), omega, eps_inner,
 * maxit_inner; inner = PCG, smoother = JACOBI, npre = npost = 1, coarse = AMG,
 * stop = RESIDUAL (others: DGMG_ERR_ARG).  rtol and maxit are per member
 * (dgmg_batch_add); graph and timing are ignored.  opts: host, or NULL for the
 * defaults.  The batch owns a few small device buffers; DGMG_ERR_CUDA if
 * they cannot be allocated. */
dgmg_status dgmg_batch_create(dgmg_batch** out, int device, void* cuda_stream, const dgmg_solve_opts* opts);

/* Synchronises the batch's stream, gives every member context its own stream
 * back and frees the batch (the contexts stay alive). */
dgmg_status dgmg_batch_destroy(dgmg_batch* batch);

/* Message of the last failed batch call ("" after success; owned by the batch). */
const char* dgmg_batch_last_error(const dgmg_batch* batch);

/* Computes a request's initial Krylov state for a later dgmg_batch_add on
 * the context's own stream: r = f - A u, ||r||, z = M r, p = z and (r, z) with
 * the V-cycle and Krylov method of opts (host; NULL: defaults), one
 * synchronisation.  The state is kept in the context (its Krylov vectors,
 * allocated if needed) and used by dgmg_batch_add for the same f, u and the
 * same options; any other call that changes the context's mesh or
 * coefficients drops it.  Lets a set-up thread do this work on its own
 * stream instead of the batch's.  Errors as dgmg_batch_add, reported through
 * dgmg_last_error(ctx). */
dgmg_status dgmg_batch_prime(dgmg_ctx* ctx, const double* f, double* u, const dgmg_solve_opts* opts);

/* Adds a request: ctx with its mesh and coefficients set (b = 0, cell-wise K
 * and c; the same order p and kernel layouts as the other members), its
 * right-hand side f and initial guess / solution u (device FP64 DG vectors of
 * the context, distinct; u is updated in place while the member runs), its
 * relative tolerance rtol (on ||f - A u||_2 / ||f - A u_0||_2) and iteration
 * cap maxit.  The context's stream is synchronised and replaced by the
 * batch's stream until dgmg_batch_remove; meanwhile the caller must not use
 * the context.  Takes the initial state of dgmg_batch_prime when it was
 * computed for the same f, u and options, else computes r = f - A u,
 * z = M r, p = z and (r, z) on the batch's stream (one synchronisation),
 * allocating the context's Krylov vectors if needed.  On
 * return *slot (host) names the member.  Errors: DGMG_ERR_ARG (bad or
 * unsupported arguments, full batch, NaN or Inf in the initial residual:
 * nothing added), DGMG_ERR_STATE (context not ready), DGMG_ERR_OOM. */
dgmg_status dgmg_batch_add(dgmg_batch* batch, dgmg_ctx* ctx, const double* f, double* u, double rtol, int maxit,
                           int* slot);

/* Runs `iterations` outer iterations of every running member, then reads the
 * members' stop flags (one synchronisation) and sets *running (host, or NULL)
 * to the number of members still running.  A member stops when its residual
 * meets its tolerance, at its iteration cap, or at a CG breakdown; stopped
 * members take no part in later launches. */
dgmg_status dgmg_batch_step(dgmg_batch* batch, int iterations, int* running);

/* *done = 1 (host) once member `slot` has stopped, else 0.  For a stopped
 * member the first call recomputes its true FP64 residual (as dgmg_solve does)
 * and fills *stats (host, or NULL: iterations, rel_residual, converged; the
 * timing and inner-iteration fields stay 0); the return value is then the
 * member's status: DGMG_OK, DGMG_ERR_NOT_CONVERGED or DGMG_ERR_BREAKDOWN. */
dgmg_status dgmg_batch_poll(dgmg_batch* batch, int slot, int* done, dgmg_solve_stats* stats);

/* Removes member `slot` (running or not): synchronises the batch's stream and
 * gives the context its own stream back. */
dgmg_status dgmg_batch_remove(dgmg_batch* batch, int slot);

/* Largest grid (nx*ny*nz cells) dgmg_restrict_noalloc accepts. */
#define DGMG_NOALLOC_MAX_CELLS 131072

/* r_hat = R r, the same restriction as dgmg_restrict, for callers that cannot
 * allocate device memory: a host application that owns all device memory
 * through its own pool and forbids other allocators, or a real-time loop that
 * must not wait on cudaMalloc, which can synchronise the device.  Such callers
 * cannot use dgmg_restrict, because creating a context and setting its
 * coefficients allocate.  The paper has no counterpart: this is a deployment
 * variant of the restriction of Sec. 2.2.2.
 *
 * No context is needed and nothing is allocated: the per-cell corner sums live
 * in a fixed file-scope device array of 8 * DGMG_NOALLOC_MAX_CELLS doubles
 * (8 MiB), which every GPU that loads this library holds until the process
 * exits.  Grids with more than DGMG_NOALLOC_MAX_CELLS cells return
 * DGMG_ERR_ARG, as do p outside [1, 8], non-positive sizes and NULL pointers.
 *   r: device DG vector of `prec` (ncell (p+1)^3 values, layout above);
 *   r_hat: device FP64 vertex vector ((nx+1)(ny+1)(nz+1) values), overwritten;
 *   cuda_stream: cudaStream_t of the current device (NULL = default stream).
 * The first call on a device sets it up, synchronously, with that device
 * current: it copies the 1D tables into constant memory and looks up the
 * scratch array's device address, then keeps both for the life of the
 * process.  Make that first call on each device before any stream capture
 * begins there, since its set-up copies synchronously.  Calls on a device
 * after a cudaDeviceReset of that device are not
 * supported (the kept set-up is not redone).  Every corner sum a call reads
 * was written earlier in the same call, so the scratch needs no clearing.
 * All calls on a device share the one scratch array: calls whose work may
 * overlap on the GPU (different streams without ordering) race and give wrong
 * results.  Returns DGMG_ERR_CUDA if a CUDA call fails. */
dgmg_status dgmg_restrict_noalloc(int nx, int ny, int nz, int p, const void* r, double* r_hat, dgmg_prec prec,
                                  void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DGMG_H */
