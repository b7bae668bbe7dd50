// Internal declarations shared by the host library and the per-order kernel
// translation units.  Not part of the public ABI (include/dgmg.h is).
#pragma once

#include <cuda_runtime.h>

#include "dgmg.h"

namespace dgmg {

// Number of kernels launched by this library from the calling host thread
// (a solve's launch count is the difference over the call; each thread of a
// serving loop drives its own context).
extern thread_local unsigned long long t_launches;
inline void count_launch(unsigned long long k = 1) { t_launches += k; }

constexpr int kMinN = 2;   // p = 1
constexpr int kMaxN = 9;   // p = 8

// Mesh and coefficients as seen by the kernels (passed by value).
struct MeshParams {
  int nx, ny, nz, p;
  long long ncell;
  double h[3];
  int bc[6];              // 0 Dirichlet, 1 Neumann; planes -x,+x,-y,+y,-z,+z
  const double* K;        // device, ncell * kdim
  int kdim;               // 1 or 3
  const double* c;        // device, ncell, or nullptr
  const double* bvert;    // device, 3 * nvert, or nullptr
  double alpha;           // penalty parameter (1.25)
  // Per-cell coefficient records, kRecLen values per cell (see kRec*),
  // computed once at set-up in both precisions.
  const double* rec64;
  const float* rec32;
  const float* bvert32;   // float copy of bvert (or nullptr)
  // Mesh scalars in both precisions: 1/h_d, face area normal to d, |J|/h_d.
  double ih[3], area[3], jh[3];
  float ihf[3], areaf[3], jhf[3];
  // Spatially varying K(x), c(x) for the outer operator (device, 16 values:
  // basis rows n_k, p0, p2, gamma), or nullptr.
  const double* var;
  // Warps per block of the operator and smoother (inner PCG) kernels per
  // precision (index DGMG_FP64 / FP32 / DF64; 0 = the default of 4).
  int wpb_apply[3], wpb_smooth[3];
  // Work layouts (dgmg_layout, resolved: never DGMG_LAYOUT_AUTO) per precision.
  int lay_apply[3], lay_smooth[3];
};

// Record layout: kd[3] = |J| K_d / h_d^2, cJ = c |J|, kap[6], gam[6] for the
// faces f = 2d + s (kap = K^-K^+/(K^-+K^+) inside, K on Dirichlet faces,
// gamma_F the penalty; both 0 on Neumann faces).
constexpr int kRecLen = 16;
constexpr int kRecKd = 0, kRecCJ = 3, kRecKap = 4, kRecGam = 10;

// Fill the records (setup; one thread per cell).
cudaError_t cell_records(const MeshParams& mp, double* rec64, float* rec32, cudaStream_t s);

// Flat layout of the 1D tables uploaded to constant memory for one n (all in
// double on the host; the kernels keep a float copy too):
//   B[n][n]    GLL Lagrange basis at the Gauss points, B[q][j] = l_j(g_q)
//   Dg[n][n]   collocation derivative on the Gauss points
//   w[n]       Gauss weights on [0,1]
//   dl[2][n]   l_j'(0), l_j'(1)
//   M1[n][n]   1D mass matrix of the GLL basis, sum_q w_q B[q][i] B[q][j]
//   G[n][n]    G[q][j] = l_j'(g_q)
//   hat[2][n]  Q1 hat functions at the GLL nodes: 1 - zeta_i, zeta_i
//   gq[n]      Gauss points on [0,1]
//   S1[n][n]   1D stiffness matrix of the GLL basis, sum_q w_q G[q][i] G[q][j]
inline int table_size(int n) { return 5 * n * n + 6 * n; }

struct SmoothArgs {
  const void* f;
  const void* uold;       // nullptr: zero initial guess
  void* unew;
  const void* diag;       // 1 / diag(D_T) in the same precision
  double omega, eps;
  int maxit;
  int inner;              // DGMG_INNER_PCG / GMRES / DIRECT
  int restart;
  const void* binv = nullptr;  // DIRECT: ncell column-major n^3 x n^3 inverses (FP64 smoother:
                               // float2 double-float pairs; FP32: float), column stride binv_ld
  int binv_ld = 0;
  const void* tri = nullptr;   // GMRES_TRIDIAG: per cell Thomas factors [a | c' | 1/den], same precision
  int* its;               // device int[ncell] or nullptr
  int color = -1;         // -1: all cells (Jacobi); 0..7: one parity class, in place allowed
};

// Requests of one order served by one launch: member r owns the blocks
// [block0[r], block0[r+1]) of the grid (the launcher fills block0 from each
// member's cell count and the launch shape), and its own mesh parameters and
// vectors.  Passed by value as a __grid_constant__ kernel parameter.
constexpr int kMaxBatch = DGMG_BATCH_MAX;
struct BatchTable {
  int k = 0;
  unsigned block0[kMaxBatch + 1] = {};
  MeshParams mp[kMaxBatch];
  const void* in[kMaxBatch] = {};    // operator input; smoother f; restriction r; prolongation u_hat
  void* out[kMaxBatch] = {};         // operator output; smoother u_new; corner sums; prolongation u
  const void* uold[kMaxBatch] = {};  // smoother u_old (nullptr: zero start)
  const void* diag[kMaxBatch] = {};  // smoother 1 / diag(D_T)
  int* its[kMaxBatch] = {};          // smoother per-cell inner iteration counts, or nullptr
  double omega = 1.0, eps = 1e-2;    // smoother parameters shared by the members
  int maxit = 0;
};

// Per-order kernel entry points, one table per n (cell_kernels.cu built with
// -DDGMG_N=n).
struct CellOps {
  int n;
  cudaError_t (*upload_tables)(const double* host_tables, cudaStream_t s);
  // full = A (with neighbour terms); !full = block diagonal D.
  // prec: DGMG_FP64, DGMG_FP32 or DGMG_DF64 (FP64 vectors, double-float arithmetic)
  cudaError_t (*apply)(const MeshParams& mp, const void* u, void* v, int prec, bool full,
                       cudaStream_t s);
  cudaError_t (*smooth)(const MeshParams& mp, const SmoothArgs& a, int prec, cudaStream_t s);
  cudaError_t (*diag)(const MeshParams& mp, double* diag, cudaStream_t s);
  cudaError_t (*restrict_cells)(const MeshParams& mp, const void* r, double* corners, bool fp32,
                                cudaStream_t s);
  cudaError_t (*prolong_add)(const MeshParams& mp, const double* uhat, void* u, bool fp32,
                             cudaStream_t s);
  // D_T of every cell, FP64, column-major n^3 x n^3 per cell (column j = D_T e_j),
  // column stride ld >= n^3, block stride n^3 ld
  cudaError_t (*block_matrix)(const MeshParams& mp, double* out, int ld, cudaStream_t s);
  // Thomas factors of the tridiagonal part of every D_T, FP64, 3 n^3 per cell
  cudaError_t (*block_tridiag)(const MeshParams& mp, double* out, int* singular, cudaStream_t s);
  // v = A u with K(x), c(x) varying inside the cells (mp.var), FP64, b = 0
  cudaError_t (*apply_var)(const MeshParams& mp, const double* u, double* v, cudaStream_t s);
  // The same for the members of a batch in one launch each (b = 0, the
  // layouts and launch shapes of member 0); block0 is filled here.
  cudaError_t (*apply_batch)(BatchTable& bt, int prec, bool full, cudaStream_t s);
  cudaError_t (*smooth_batch)(BatchTable& bt, int prec, cudaStream_t s);   // inner-PCG Jacobi sweep
  cudaError_t (*restrict_batch)(BatchTable& bt, bool fp32, cudaStream_t s);
  cudaError_t (*prolong_batch)(BatchTable& bt, bool fp32, cudaStream_t s);
};

const CellOps* cell_ops(int n);

// Vector, stencil and conversion kernels (vec_kernels.cu).
cudaError_t vec_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s);  // y = a x + b y
cudaError_t vec_axpby_f(long long n, float a, const float* x, float b, float* y, cudaStream_t s);
cudaError_t vec_sub(long long n, const double* a, const double* b, double* out, cudaStream_t s);   // out = a - b
cudaError_t vec_sub_f(long long n, const float* a, const float* b, float* out, cudaStream_t s);
cudaError_t vec_copy(long long n, const double* x, double* y, cudaStream_t s);
cudaError_t vec_fill(long long n, double v, double* y, cudaStream_t s);
cudaError_t vec_fill_f(long long n, float v, float* y, cudaStream_t s);
cudaError_t vec_d2f(long long n, const double* x, float* y, cudaStream_t s);
cudaError_t vec_inverse(long long n, const double* d, double* i64, float* i32, cudaStream_t s);
// In-place inverse of ncell dense nb x nb FP64 blocks (column-major, column
// stride ld >= nb, block stride nb ld) by Gauss-Jordan elimination with partial
// pivoting; nb <= 125.  singular: device int, set to 1 when a block has a zero
// pivot (else untouched).
cudaError_t block_invert(double* a, int nb, int ld, long long ncell, int* singular, cudaStream_t s);
// Split FP64 values into double-float pairs (hi = fl(v), lo = fl(v - hi)) and,
// if f32 is not null, also write hi alone; and the reverse (hi + lo into a
// dense array, dropping the padding of a column stride ld > nb).
cudaError_t vec_split_df(long long n, const double* x, float2* pairs, float* f32, cudaStream_t s);
cudaError_t blocks_df_to_dense(long long ncell, int nb, int ld, const float2* pairs, double* out, cudaStream_t s);
// P0 transfer: out[c] = sum_i r[c n3 + i]; u[c n3 + i] += uhat[c].
cudaError_t cell_sums(long long ncell, int n3, const void* r, double* out, bool fp32, cudaStream_t s);
cudaError_t cell_add(long long ncell, int n3, const double* uhat, void* u, bool fp32, cudaStream_t s);
cudaError_t vec_f2d(long long n, const float* x, double* y, cudaStream_t s);
// Deterministic dot products: partial sums per block in a fixed order, then
// one block sums the partials; result written to out (device).
cudaError_t vec_dot(long long n, const double* x, const double* y, double* partial, double* out,
                    cudaStream_t s);
cudaError_t vec_multi_dot(long long n, int k, const double* const* xs, const double* y,
                          double* partial, double* out, cudaStream_t s);
constexpr int kDotBlocks = 1024;

// ---------------------------------------------------------------- batched Krylov
// Segments of a batch for the vector kernels: member r's vectors a..e of
// length n[r] and its device scalar block sc[r] (kScLen doubles); the blocks
// of a launch are split among the members by block0 (filled by the launcher).
struct SegTable {
  int k = 0;
  unsigned block0[kMaxBatch + 1] = {};
  long long n[kMaxBatch] = {};
  const void* a[kMaxBatch] = {};
  const void* b[kMaxBatch] = {};
  void* c[kMaxBatch] = {};
  void* d[kMaxBatch] = {};
  void* e[kMaxBatch] = {};
  double* sc[kMaxBatch] = {};
};

// Scalar block of a member of a batched CG / flexible CG: (r, z), (p, q),
// alpha, (r, r), new (r, z), (z, r_old), beta, ||r_0||, rtol, state (0
// running, 1 converged, 2 breakdown, 3 iteration cap), iterations, maxit,
// flexible (0 / 1).
constexpr int kScRz = 0, kScPq = 1, kScAlpha = 2, kScRr = 3, kScRzn = 4, kScZro = 5, kScBeta = 6, kScR0 = 7,
              kScRtol = 8, kScDone = 9, kScIts = 10, kScMaxit = 11, kScFlex = 12, kScLen = 16;

enum SegOp {
  SEG_D2F,      // c = (float) a
  SEG_F2D,      // c = (double) a
  SEG_COPY64,   // c = a (FP64)
  SEG_COPY32,   // c = a (FP32)
  SEG_SUB64,    // c = a - b (FP64)
  SEG_SUB32,    // c = a - b (FP32)
  SEG_ALPHA,    // CG update with alpha = sc[kScAlpha]: (flexible: e = d,) c += alpha a, d -= alpha b
                // (a = p, b = q, c = u, d = r, e = r_old)
  SEG_P         // c = a + beta c with beta = sc[kScBeta] (a = z, c = p)
};
enum ScalOp {
  SC_ALPHA,     // alpha = (r, z) / (p, q), or 0 and state 2 when (p, q) <= 0, or 0 when stopped
  SC_CONV,      // iterations += 1; state 1 when sqrt((r, r)) <= rtol ||r_0||, 3 at maxit
  SC_BETA       // beta = ((r, z)_new - flexible (z, r_old)) / (r, z); (r, z) <- new; 0 when stopped
};
cudaError_t seg_op(int op, SegTable& t, cudaStream_t s);
// sc[r][slot] = (a_r, b_r) with the summation order of vec_dot; partial:
// k * kDotBlocks doubles.
cudaError_t seg_dot(SegTable& t, double* partial, int slot, cudaStream_t s);
cudaError_t seg_scalar(int op, SegTable& t, cudaStream_t s);

// 27-point stencil operators of the AMG levels (row-major, 27 per row).
cudaError_t stencil_jacobi(int vx, int vy, int vz, const double* st, const double* dinv,
                           const double* b, const double* x, double* xout, double omega,
                           bool zero_x, cudaStream_t s);
cudaError_t stencil_residual(int vx, int vy, int vz, const double* st, const double* b,
                             const double* x, double* r, cudaStream_t s);
cudaError_t agg_restrict(int vx, int vy, int vz, const double* r, double* rc, cudaStream_t s);
cudaError_t agg_prolong_add(int vx, int vy, int vz, const double* xc, double* x, cudaStream_t s);
cudaError_t dense_matvec(int n, const double* A, const double* x, double* y, cudaStream_t s);
cudaError_t restrict_gather(int nx, int ny, int nz, const double* corners, double* rhat,
                            cudaStream_t s);

}  // namespace dgmg
