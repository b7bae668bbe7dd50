// Host-side setup of the library: 1D quadrature tables, the Q1 coarse matrix
// by re-discretisation, the aggregation-AMG hierarchy and the right-hand side.
#pragma once

#include <vector>

namespace dgmg {

constexpr int kMaxTableN = 9;   // largest n = p + 1 of the tables

// Gauss-Legendre (m points) and Gauss-Lobatto-Legendre (n >= 2 points) rules on
// [0, 1] by Newton iteration on the Legendre polynomials.
void gauss_legendre01(int m, std::vector<double>& x, std::vector<double>& w);
void gauss_lobatto01(int n, std::vector<double>& x, std::vector<double>& w);
void gauss_legendre01(int m, double* x, double* w);
void gauss_lobatto01(int n, double* x, double* w);
// l_j(x) and l_j'(x) of the Lagrange basis on `nodes`.
void lagrange(const std::vector<double>& nodes, double x, double* val, double* der);
void lagrange(const double* nodes, int n, double x, double* val, double* der);

// All per-order tables in the flat layout of dgmg_internal.h; the _into form
// writes table_size(n) doubles to T and uses no heap memory.
std::vector<double> build_tables(int n);
void build_tables_into(int n, double* T);

struct HostMesh {
  int nx, ny, nz, p;
  double h[3];
  int bc[6];
  const double* K;      // host ncell * kdim
  int kdim;
  const double* b;      // host 3 * nvert or nullptr
  const double* c;      // host ncell or nullptr
  double alpha;
  // K(x), c(x) varying inside the cells (basis rows n_k, p0, p2, gamma; 16
  // values) or nullptr; the right-hand side then uses K(x) on Dirichlet faces.
  const double* var = nullptr;
};

// K(x) = sum_k (p0_k + p2_k x_k^2) n_k n_k^T at a point: (xx, yy, zz, xy, xz, yz).
void var_tensor(const double* var, const double x[3], double K[6]);

// A_hat (App. A.2) as a 27-point stencil on the (nx+1)(ny+1)(nz+1) vertices.
std::vector<double> q1_stencil(const HostMesh& m);

// A_hat = P^T A P of the piecewise-constant subspace (App. A.1) as a 27-point
// stencil on the nx*ny*nz cell grid (7 non-zero entries per row).
std::vector<double> p0_stencil(const HostMesh& m);

// Galerkin coarsening of a 27-point stencil with 2x2x2 piecewise-constant
// aggregates; returns the coarse stencil and its grid dims.
std::vector<double> coarsen_stencil(const std::vector<double>& st, int vx, int vy, int vz, int& cx, int& cy, int& cz);

// Dense matrix of a stencil operator (row-major) and its inverse by LU with
// partial pivoting; false if singular.
std::vector<double> stencil_dense(const std::vector<double>& st, int vx, int vy, int vz);
bool dense_inverse(int n, std::vector<double>& A);

// l_h(psi_i) (eq. rhs) on the host, sum-factorised with the tables.
void assemble_rhs_host(const HostMesh& m, const double* f_qp, const double* g_qp, const double* j_qp, double* rhs);

// Quadrature point coordinates (see dgmg_quadrature_points).
void quadrature_points_host(const HostMesh& m, double* vol_xyz, double* face_xyz);

}  // namespace dgmg
