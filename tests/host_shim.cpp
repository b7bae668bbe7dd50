// Test shim: C entry points around the library's host-side set-up code
// (setup_host.cpp), built with the host compiler alone, so that the CPU test
// tier can compare the Q1 and P0 coarse matrices, the AMG coarsening, the
// right-hand side and the quadrature rules with the oracle without a GPU.
// Not part of the library; only tests/test_host_setup.py builds and loads it.
#include <cstring>
#include <vector>

#include "setup_host.h"

namespace {

dgmg::HostMesh mesh(int nx, int ny, int nz, int p, const double* h, const int* bc, const double* K, int kdim,
                    const double* b, const double* c, double alpha, const double* var) {
  dgmg::HostMesh m;
  m.nx = nx;
  m.ny = ny;
  m.nz = nz;
  m.p = p;
  for (int d = 0; d < 3; ++d) m.h[d] = h[d];
  for (int i = 0; i < 6; ++i) m.bc[i] = bc[i];
  m.K = K;
  m.kdim = kdim;
  m.b = b;
  m.c = c;
  m.alpha = alpha;
  m.var = var;
  return m;
}

}  // namespace

extern "C" {

// out: 27 * (nx+1)(ny+1)(nz+1) doubles.
void shim_q1_stencil(int nx, int ny, int nz, int p, const double* h, const int* bc, const double* K, int kdim,
                     const double* b, const double* c, double alpha, double* out) {
  const std::vector<double> st = dgmg::q1_stencil(mesh(nx, ny, nz, p, h, bc, K, kdim, b, c, alpha, nullptr));
  std::memcpy(out, st.data(), st.size() * sizeof(double));
}

// out: 27 * nx ny nz doubles.
void shim_p0_stencil(int nx, int ny, int nz, int p, const double* h, const int* bc, const double* K, int kdim,
                     const double* b, const double* c, double alpha, double* out) {
  const std::vector<double> st = dgmg::p0_stencil(mesh(nx, ny, nz, p, h, bc, K, kdim, b, c, alpha, nullptr));
  std::memcpy(out, st.data(), st.size() * sizeof(double));
}

// Galerkin 2x2x2 coarsening of a 27-point stencil on a vx*vy*vz grid; out
// receives 27 * cx cy cz doubles (at most 27 * vx vy vz), dims the coarse grid.
void shim_coarsen(const double* st, int vx, int vy, int vz, double* out, int* dims) {
  std::vector<double> s(st, st + 27LL * vx * vy * vz);
  int cx = 0, cy = 0, cz = 0;
  const std::vector<double> c = dgmg::coarsen_stencil(s, vx, vy, vz, cx, cy, cz);
  std::memcpy(out, c.data(), c.size() * sizeof(double));
  dims[0] = cx;
  dims[1] = cy;
  dims[2] = cz;
}

// rhs: ncell (p+1)^3 doubles; var: 16 values of K(x), c(x) or NULL.
void shim_rhs(int nx, int ny, int nz, int p, const double* h, const int* bc, const double* K, int kdim,
              const double* b, const double* c, double alpha, const double* var, const double* f_qp,
              const double* g_qp, const double* j_qp, double* rhs) {
  dgmg::assemble_rhs_host(mesh(nx, ny, nz, p, h, bc, K, kdim, b, c, alpha, var), f_qp, g_qp, j_qp, rhs);
}

void shim_quadrature_points(int nx, int ny, int nz, int p, const double* h, double* vol, double* face) {
  const int bc[6] = {0, 0, 0, 0, 0, 0};
  const double one = 1.0;
  dgmg::quadrature_points_host(mesh(nx, ny, nz, p, h, bc, &one, 1, nullptr, nullptr, 1.25, nullptr), vol, face);
}

// In-place inverse of the n x n row-major A (the coarsest AMG solve);
// returns 0 if A is singular.
int shim_dense_inverse(int n, double* A) {
  std::vector<double> a(A, A + (long long)n * n);
  if (!dgmg::dense_inverse(n, a)) return 0;
  std::memcpy(A, a.data(), a.size() * sizeof(double));
  return 1;
}

// K(x) of the pointwise tensor at one point: (xx, yy, zz, xy, xz, yz).
void shim_var_tensor(const double* var, const double* x, double* K) { dgmg::var_tensor(var, x, K); }

// The per-order 1D tables the kernels read (5 n^2 + 6 n doubles).
void shim_build_tables(int n, double* T) { dgmg::build_tables_into(n, T); }

void shim_gauss_legendre01(int m, double* x, double* w) { dgmg::gauss_legendre01(m, x, w); }
void shim_gauss_lobatto01(int n, double* x, double* w) { dgmg::gauss_lobatto01(n, x, w); }

}  // extern "C"
