// Host-side setup: quadrature tables, Q1 re-discretisation (App. A.2), AMG
// coarsening and the right-hand side l_h (Sec. 2.1, eq. rhs).
#include "setup_host.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

namespace dgmg {

namespace {

// P_k(x) and P_{k-1}(x) by the three-term recurrence.
void legendre(int k, double x, double& pk, double& pkm1) {
  double p0 = 1.0, p1 = x;
  if (k == 0) {
    pk = 1.0;
    pkm1 = 0.0;
    return;
  }
  for (int j = 1; j < k; ++j) {
    const double p2 = ((2.0 * j + 1.0) * x * p1 - j * p0) / (j + 1.0);
    p0 = p1;
    p1 = p2;
  }
  pk = p1;
  pkm1 = p0;
}

const double kPi = 3.14159265358979323846;

}  // namespace

void gauss_legendre01(int m, double* x, double* w) {
  for (int i = 0; i < m; ++i) {
    double t = std::cos(kPi * (i + 0.75) / (m + 0.5));
    double pm = 0, pm1 = 0, dp = 0;
    for (int it = 0; it < 100; ++it) {
      legendre(m, t, pm, pm1);
      dp = m * (t * pm - pm1) / (t * t - 1.0);
      const double dt = pm / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    legendre(m, t, pm, pm1);
    dp = m * (t * pm - pm1) / (t * t - 1.0);
    // descending t -> ascending x
    x[m - 1 - i] = 0.5 * (t + 1.0);
    w[m - 1 - i] = 0.5 * 2.0 / ((1.0 - t * t) * dp * dp);
  }
}

void gauss_legendre01(int m, std::vector<double>& x, std::vector<double>& w) {
  x.assign(m, 0.0);
  w.assign(m, 0.0);
  gauss_legendre01(m, x.data(), w.data());
}

void gauss_lobatto01(int n, double* x, double* w) {
  const int N = n - 1;
  double t[kMaxTableN];
  t[0] = -1.0;
  t[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double s = -std::cos(kPi * i / N);
    for (int it = 0; it < 100; ++it) {
      double pn, pn1;
      legendre(N, s, pn, pn1);
      const double d1 = N * (pn1 - s * pn) / (1.0 - s * s);                  // P_N'
      const double d2 = (2.0 * s * d1 - N * (N + 1.0) * pn) / (1.0 - s * s);  // P_N''
      const double ds = d1 / d2;
      s -= ds;
      if (std::fabs(ds) < 1e-16) break;
    }
    t[i] = s;
  }
  for (int i = 0; i < n; ++i) {
    double pn, pn1;
    legendre(N, t[i], pn, pn1);
    x[i] = 0.5 * (t[i] + 1.0);
    w[i] = 0.5 * 2.0 / (N * (N + 1.0) * pn * pn);
  }
}

void gauss_lobatto01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  gauss_lobatto01(n, x.data(), w.data());
}

void lagrange(const std::vector<double>& z, double x, double* val, double* der) {
  lagrange(z.data(), (int)z.size(), x, val, der);
}

void lagrange(const double* z, int n, double x, double* val, double* der) {
  for (int j = 0; j < n; ++j) {
    double v = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) v *= (x - z[k]) / (z[j] - z[k]);
    if (val) val[j] = v;
    if (der) {
      double d = 0.0;
      for (int l = 0; l < n; ++l) {
        if (l == j) continue;
        double term = 1.0 / (z[j] - z[l]);
        for (int k = 0; k < n; ++k)
          if (k != j && k != l) term *= (x - z[k]) / (z[j] - z[k]);
        d += term;
      }
      der[j] = d;
    }
  }
}

std::vector<double> build_tables(int n) {
  std::vector<double> T(5 * n * n + 6 * n, 0.0);
  build_tables_into(n, T.data());
  return T;
}

void build_tables_into(int n, double* T) {
  double gll[kMaxTableN], gllw[kMaxTableN], gq[kMaxTableN], gw[kMaxTableN];
  gauss_lobatto01(n, gll, gllw);
  gauss_legendre01(n, gq, gw);
  for (int i = 0; i < 5 * n * n + 6 * n; ++i) T[i] = 0.0;
  double* B = T;
  double* Dg = B + n * n;
  double* W = Dg + n * n;
  double* dl = W + n;
  double* M1 = dl + 2 * n;
  double* G = M1 + n * n;
  double* hat = G + n * n;
  double* GQ = hat + 2 * n;
  double* S1 = GQ + n;
  for (int q = 0; q < n; ++q) {
    lagrange(gll, n, gq[q], B + q * n, G + q * n);
    lagrange(gq, n, gq[q], nullptr, Dg + q * n);
    W[q] = gw[q];
    GQ[q] = gq[q];
  }
  lagrange(gll, n, 0.0, nullptr, dl);
  lagrange(gll, n, 1.0, nullptr, dl + n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s += gw[q] * B[q * n + i] * B[q * n + j];
      M1[i * n + j] = s;
    }
  for (int i = 0; i < n; ++i) {
    hat[i] = 1.0 - gll[i];
    hat[n + i] = gll[i];
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int q = 0; q < n; ++q) s += gw[q] * G[q * n + i] * G[q * n + j];
      S1[i * n + j] = s;
    }
}

namespace {

inline double kval(const HostMesh& m, long long c, int d) { return m.K[c * m.kdim + (m.kdim == 3 ? d : 0)]; }

inline double q1phi(int k, const double xi[3]) {
  double v = 1.0;
  for (int d = 0; d < 3; ++d) v *= ((k >> d) & 1) ? xi[d] : 1.0 - xi[d];
  return v;
}

inline double q1grad(int k, const double xi[3], int d, const double h[3]) {
  double v = (((k >> d) & 1) ? 1.0 : -1.0) / h[d];
  for (int e = 0; e < 3; ++e)
    if (e != d) v *= ((k >> e) & 1) ? xi[e] : 1.0 - xi[e];
  return v;
}

inline long long vid(const HostMesh& m, int vx, int vy, int vz) {
  return vx + (long long)(m.nx + 1) * (vy + (long long)(m.ny + 1) * vz);
}

void b_at(const HostMesh& m, int cx, int cy, int cz, const double xi[3], double out[3]) {
  out[0] = out[1] = out[2] = 0.0;
  if (!m.b) return;
  for (int k = 0; k < 8; ++k) {
    const long long v = vid(m, cx + (k & 1), cy + ((k >> 1) & 1), cz + (k >> 2));
    const double wk = q1phi(k, xi);
    for (int d = 0; d < 3; ++d) out[d] += wk * m.b[3 * v + d];
  }
}

}  // namespace

std::vector<double> q1_stencil(const HostMesh& m) {
  const long long nvert = (long long)(m.nx + 1) * (m.ny + 1) * (m.nz + 1);
  std::vector<double> st(27 * nvert, 0.0);
  // The DG rule (p+1 Gauss points per direction): with it A_hat equals P^T A P
  // exactly, also where the upwind term max(b.n, 0) has a kink inside a face.
  const int nq = m.p + 1;
  std::vector<double> g2, w2, gf2, wf2;
  gauss_legendre01(nq, g2, w2);
  gauss_legendre01(2, gf2, wf2);
  const double J = m.h[0] * m.h[1] * m.h[2];
  const double pen = m.alpha * m.p * (m.p + 2);
  auto scatter = [&](int cx, int cy, int cz, const double Ae[8][8]) {
    for (int a = 0; a < 8; ++a) {
      const long long va = vid(m, cx + (a & 1), cy + ((a >> 1) & 1), cz + (a >> 2));
      for (int b = 0; b < 8; ++b) {
        const int dx = (b & 1) - (a & 1), dy = ((b >> 1) & 1) - ((a >> 1) & 1), dz = (b >> 2) - (a >> 2);
        st[27 * va + (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] += Ae[a][b];
      }
    }
  };
  // The volume part of the element matrix from reference integrals over one
  // cell, taken once with the same rule (exact for these Q1 integrands):
  // R_d[a][b] = int d_d phi_b d_d phi_a, R_m[a][b] = int phi_b phi_a and, for
  // the trilinear advection field b = sum_v b_v phi_v, T_d[v][a][b] =
  // int phi_v phi_b d_d phi_a; then A_e = sum_d K_d R_d + c R_m -
  // sum_d sum_v b_{v,d} T_d[v].
  double Rd[3][8][8], Rm[8][8];
  std::memset(Rd, 0, sizeof(Rd));
  std::memset(Rm, 0, sizeof(Rm));
  std::vector<double> Tb(m.b ? 3 * 8 * 64 : 0, 0.0);
  for (int q3 = 0; q3 < nq; ++q3)
    for (int q2 = 0; q2 < nq; ++q2)
      for (int q1 = 0; q1 < nq; ++q1) {
        const double xi[3] = {g2[q1], g2[q2], g2[q3]};
        const double w = w2[q1] * w2[q2] * w2[q3] * J;
        double phi[8], gr[8][3];
        for (int k = 0; k < 8; ++k) {
          phi[k] = q1phi(k, xi);
          for (int d = 0; d < 3; ++d) gr[k][d] = q1grad(k, xi, d, m.h);
        }
        for (int a = 0; a < 8; ++a)
          for (int b = 0; b < 8; ++b) {
            Rm[a][b] += w * phi[b] * phi[a];
            for (int d = 0; d < 3; ++d) Rd[d][a][b] += w * gr[b][d] * gr[a][d];
          }
        if (m.b)
          for (int d = 0; d < 3; ++d)
            for (int v = 0; v < 8; ++v)
              for (int a = 0; a < 8; ++a)
                for (int b = 0; b < 8; ++b) Tb[((d * 8 + v) * 8 + a) * 8 + b] += w * phi[v] * phi[b] * gr[a][d];
      }
  for (int cz = 0; cz < m.nz; ++cz)
    for (int cy = 0; cy < m.ny; ++cy)
      for (int cx = 0; cx < m.nx; ++cx) {
        const long long c = cx + (long long)m.nx * (cy + (long long)m.ny * cz);
        const double K[3] = {kval(m, c, 0), kval(m, c, 1), kval(m, c, 2)};
        const double cc = m.c ? m.c[c] : 0.0;
        double Ae[8][8];
        for (int a = 0; a < 8; ++a)
          for (int b = 0; b < 8; ++b)
            Ae[a][b] = K[0] * Rd[0][a][b] + K[1] * Rd[1][a][b] + K[2] * Rd[2][a][b] + cc * Rm[a][b];
        if (m.b)
          for (int v = 0; v < 8; ++v) {
            const double* bv = m.b + 3 * vid(m, cx + (v & 1), cy + ((v >> 1) & 1), cz + (v >> 2));
            for (int d = 0; d < 3; ++d) {
              const double* T = &Tb[(d * 8 + v) * 64];
              for (int ab = 0; ab < 64; ++ab) Ae[ab >> 3][ab & 7] -= bv[d] * T[ab];
            }
          }
        // Dirichlet faces of boundary cells (gamma from the DG degree p); the
        // DG rule where the upwind term can have a kink inside the face, two
        // points per direction (exact for these Q1 products) without advection.
        const int cc3[3] = {cx, cy, cz};
        const int nn3[3] = {m.nx, m.ny, m.nz};
        for (int d = 0; d < 3; ++d)
          for (int s = 0; s < 2; ++s) {
            if (cc3[d] != (s ? nn3[d] - 1 : 0) || m.bc[2 * d + s] != 0) continue;
            const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
            const double area = m.h[ta] * m.h[tb];
            const double sgn = s ? 1.0 : -1.0;
            const double gam = pen * K[d] / m.h[d];
            const int nf = m.b ? nq : 2;
            const std::vector<double>& gf = m.b ? g2 : gf2;
            const std::vector<double>& wf = m.b ? w2 : wf2;
            for (int qb = 0; qb < nf; ++qb)
              for (int qa = 0; qa < nf; ++qa) {
                double xi[3];
                xi[d] = s;
                xi[ta] = gf[qa];
                xi[tb] = gf[qb];
                const double w = wf[qa] * wf[qb] * area;
                double bq[3];
                b_at(m, cx, cy, cz, xi, bq);
                const double bn = sgn * bq[d];
                double phi[8], dn[8];
                for (int k = 0; k < 8; ++k) {
                  phi[k] = q1phi(k, xi);
                  dn[k] = sgn * q1grad(k, xi, d, m.h);
                }
                for (int a = 0; a < 8; ++a)
                  for (int b = 0; b < 8; ++b) {
                    const double up = bn >= 0.0 ? bn * phi[b] : 0.0;
                    Ae[a][b] += w * (up * phi[a] - K[d] * dn[b] * phi[a] - K[d] * dn[a] * phi[b] + gam * phi[b] * phi[a]);
                  }
              }
          }
        scatter(cx, cy, cz, Ae);
      }
  return st;
}

// A_hat of the piecewise-constant subspace (App. A.1) on the cell grid.  For
// P0 functions the gradient terms vanish; what remains of a_h is, per row T:
// c |T| on the diagonal; on each interior face the penalty gamma_F |F| with
// gamma_F = alpha p (p+2) <K_d^-, K_d^+> / h_d (diagonal +, neighbour -) and
// the upwind flux split by the sign of b.n_out (n_out the outward normal of
// T): int max(b.n_out, 0) on the diagonal, int min(b.n_out, 0) for the
// neighbour; on Dirichlet faces gamma_F |F| with K_d^- alone and the outflow
// part int max(b.n_out, 0).  Face integrals of the upwind parts use the DG
// rule (p+1 Gauss points per direction), so that A_hat equals P^T A P also
// where b.n changes sign inside a face.
std::vector<double> p0_stencil(const HostMesh& m) {
  const long long ncell = (long long)m.nx * m.ny * m.nz;
  std::vector<double> st(27 * ncell, 0.0);
  const int nq = m.p + 1;
  std::vector<double> g, w;
  gauss_legendre01(nq, g, w);
  const double J = m.h[0] * m.h[1] * m.h[2];
  const double pen = m.alpha * m.p * (m.p + 2);
  const int nc[3] = {m.nx, m.ny, m.nz};
  for (int cz = 0; cz < m.nz; ++cz)
    for (int cy = 0; cy < m.ny; ++cy)
      for (int cx = 0; cx < m.nx; ++cx) {
        const long long c = cx + (long long)m.nx * (cy + (long long)m.ny * cz);
        double* row = &st[27 * c];
        if (m.c) row[13] += m.c[c] * J;
        const int cc[3] = {cx, cy, cz};
        for (int d = 0; d < 3; ++d) {
          const double area = J / m.h[d];
          const int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;
          for (int side = 0; side < 2; ++side) {
            const int step = side ? 1 : -1;
            const bool inside = cc[d] + step >= 0 && cc[d] + step < nc[d];
            if (!inside && m.bc[2 * d + side] != 0) continue;   // Neumann: nothing
            // upwind parts: int max(b.n_out, 0) and int min(b.n_out, 0) over the face
            double fout = 0.0, fin = 0.0;
            if (m.b) {
              for (int q2 = 0; q2 < nq; ++q2)
                for (int q1 = 0; q1 < nq; ++q1) {
                  double xi[3];
                  xi[d] = side ? 1.0 : 0.0;
                  xi[a] = g[q1];
                  xi[b] = g[q2];
                  double bv[3];
                  b_at(m, cx, cy, cz, xi, bv);
                  const double bn = step * bv[d];
                  const double wq = w[q1] * w[q2] * area;
                  if (bn >= 0.0)
                    fout += wq * bn;
                  else
                    fin += wq * bn;
                }
            }
            const double Km = kval(m, c, d);
            int off[3] = {0, 0, 0};
            off[d] = step;
            const int nb = (off[0] + 1) + 3 * (off[1] + 1) + 9 * (off[2] + 1);
            if (inside) {
              const long long cn = c + (d == 0 ? step : d == 1 ? step * (long long)m.nx : step * (long long)m.nx * m.ny);
              const double Kp = kval(m, cn, d);
              const double gam = pen * (2.0 * Km * Kp / (Km + Kp)) / m.h[d];
              row[13] += gam * area + fout;
              row[nb] += -gam * area + fin;
            } else {
              row[13] += pen * Km / m.h[d] * area + fout;
            }
          }
        }
      }
  return st;
}

std::vector<double> coarsen_stencil(const std::vector<double>& st, int vx, int vy, int vz, int& cx, int& cy,
                                    int& cz) {
  cx = (vx + 1) / 2;
  cy = (vy + 1) / 2;
  cz = (vz + 1) / 2;
  std::vector<double> sc(27 * (size_t)cx * cy * cz, 0.0);
  // Offset of stencil entry k = (dx+1) + 3 (dy+1) + 9 (dz+1) along each axis.
  static const int DX[27] = {-1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1, -1, 0, 1};
  static const int DY[27] = {-1, -1, -1, 0, 0, 0, 1, 1, 1, -1, -1, -1, 0, 0, 0, 1, 1, 1, -1, -1, -1, 0, 0, 0, 1, 1, 1};
  static const int DZ[27] = {-1, -1, -1, -1, -1, -1, -1, -1, -1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 1, 1, 1, 1, 1, 1, 1, 1};
  for (int iz = 0; iz < vz; ++iz)
    for (int iy = 0; iy < vy; ++iy)
      for (int ix = 0; ix < vx; ++ix) {
        const long long i = ix + (long long)vx * (iy + (long long)vy * iz);
        const long long I = ix / 2 + (long long)cx * (iy / 2 + (long long)cy * (iz / 2));
        const double* row = &st[27 * i];
        double* out = &sc[27 * I];
        for (int k = 0; k < 27; ++k) {
          const double a = row[k];
          if (a == 0.0) continue;
          const int jx = ix + DX[k], jy = iy + DY[k], jz = iz + DZ[k];
          if (jx < 0 || jy < 0 || jz < 0 || jx >= vx || jy >= vy || jz >= vz) continue;
          const int ox = (jx >> 1) - (ix >> 1), oy = (jy >> 1) - (iy >> 1), oz = (jz >> 1) - (iz >> 1);
          out[(ox + 1) + 3 * (oy + 1) + 9 * (oz + 1)] += a;
        }
      }
  return sc;
}

std::vector<double> stencil_dense(const std::vector<double>& st, int vx, int vy, int vz) {
  const long long n = (long long)vx * vy * vz;
  std::vector<double> A(n * n, 0.0);
  for (int iz = 0; iz < vz; ++iz)
    for (int iy = 0; iy < vy; ++iy)
      for (int ix = 0; ix < vx; ++ix) {
        const long long i = ix + (long long)vx * (iy + (long long)vy * iz);
        for (int k = 0; k < 27; ++k) {
          const int jx = ix + k % 3 - 1, jy = iy + (k / 3) % 3 - 1, jz = iz + k / 9 - 1;
          if (jx < 0 || jy < 0 || jz < 0 || jx >= vx || jy >= vy || jz >= vz) continue;
          A[i * n + jx + (long long)vx * (jy + (long long)vy * jz)] += st[27 * i + k];
        }
      }
  return A;
}

bool dense_inverse(int n, std::vector<double>& A) {
  // Gauss-Jordan elimination with partial pivoting on [A | I].
  std::vector<double> I((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
  for (int col = 0; col < n; ++col) {
    int piv = col;
    double best = std::fabs(A[(size_t)col * n + col]);
    for (int r = col + 1; r < n; ++r)
      if (std::fabs(A[(size_t)r * n + col]) > best) {
        best = std::fabs(A[(size_t)r * n + col]);
        piv = r;
      }
    if (best == 0.0) return false;
    if (piv != col)
      for (int j = 0; j < n; ++j) {
        std::swap(A[(size_t)piv * n + j], A[(size_t)col * n + j]);
        std::swap(I[(size_t)piv * n + j], I[(size_t)col * n + j]);
      }
    const double d = 1.0 / A[(size_t)col * n + col];
    for (int j = 0; j < n; ++j) {
      A[(size_t)col * n + j] *= d;
      I[(size_t)col * n + j] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == col) continue;
      const double f = A[(size_t)r * n + col];
      if (f == 0.0) continue;
      // columns left of col are already eliminated in the pivot row of A
      for (int j = col; j < n; ++j) A[(size_t)r * n + j] -= f * A[(size_t)col * n + j];
      for (int j = 0; j < n; ++j) I[(size_t)r * n + j] -= f * I[(size_t)col * n + j];
    }
  }
  A.swap(I);
  return true;
}

void var_tensor(const double* vp, const double x[3], double K[6]) {
  for (int i = 0; i < 6; ++i) K[i] = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double pk = vp[9 + k] + vp[12 + k] * x[k] * x[k];
    const double a = vp[3 * k], b = vp[3 * k + 1], e = vp[3 * k + 2];
    K[0] += pk * a * a;
    K[1] += pk * b * b;
    K[2] += pk * e * e;
    K[3] += pk * a * b;
    K[4] += pk * a * e;
    K[5] += pk * b * e;
  }
}

namespace {
inline double kent_host(const double K[6], int i, int j) {
  if (i == j) return K[i];
  const int s = i + j;
  return K[s == 1 ? 3 : (s == 2 ? 4 : 5)];
}
}  // namespace

void assemble_rhs_host(const HostMesh& m, const double* f_qp, const double* g_qp, const double* j_qp, double* rhs) {
  const int n = m.p + 1, n2 = n * n, n3 = n2 * n;
  const std::vector<double> T = build_tables(n);
  const double* B = T.data();
  const double* W = B + 2 * n * n;
  const double* dl = W + n;
  const double J = m.h[0] * m.h[1] * m.h[2];
  const long long ncell = (long long)m.nx * m.ny * m.nz;
  // Volume term, cell by cell; the cells are independent, so large meshes
  // are split over host threads (each cell's arithmetic is the same either way).
  auto volume = [&](long long c0, long long c1) {
    std::vector<double> t0(n3), t1(n3);
    for (long long c = c0; c < c1; ++c) {
      double* out = rhs + c * n3;
      const double* fc = f_qp ? f_qp + c * n3 : nullptr;
      for (int z = 0, q = 0; z < n; ++z)
        for (int y = 0; y < n; ++y)
          for (int x = 0; x < n; ++x, ++q) t0[q] = (fc ? fc[q] : 0.0) * W[x] * W[y] * W[z] * J;
      // B^T along x, y, z (quadrature point -> dof index); each output sums its
      // terms in quadrature-point order, with the output index innermost so
      // that the loops vectorise
      std::fill(t1.begin(), t1.end(), 0.0);
      for (int r = 0; r < n2; ++r)                   // rows (y, z)
        for (int q = 0; q < n; ++q) {
          const double a = t0[q + n * r];
          for (int i = 0; i < n; ++i) t1[i + n * r] += B[q * n + i] * a;
        }
      std::fill(t0.begin(), t0.end(), 0.0);
      for (int z = 0; z < n; ++z)
        for (int i = 0; i < n; ++i)
          for (int q = 0; q < n; ++q) {
            const double b = B[q * n + i];
            for (int x = 0; x < n; ++x) t0[x + n * i + n2 * z] += b * t1[x + n * q + n2 * z];
          }
      for (int k = 0; k < n3; ++k) out[k] = 0.0;
      for (int i = 0; i < n; ++i)
        for (int q = 0; q < n; ++q) {
          const double b = B[q * n + i];
          for (int xy = 0; xy < n2; ++xy) out[xy + n2 * i] += b * t0[xy + n2 * q];
        }
    }
  };
  const long long work = ncell * n3;
  const unsigned hw = std::thread::hardware_concurrency();
  const int nthreads = (int)std::max<long long>(1, std::min<long long>({(long long)(hw ? hw : 1), 8LL, work / (1LL << 20)}));
  if (nthreads == 1) {
    volume(0, ncell);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t) {
      const long long c0 = ncell * t / nthreads, c1 = ncell * (t + 1) / nthreads;
      try {
        pool.emplace_back(volume, c0, c1);
      } catch (...) {   // no thread to be had: this range runs here
        volume(c0, c1);
      }
    }
    for (auto& th : pool) th.join();
  }
  // boundary faces
  const double pen = m.alpha * m.p * (m.p + 2);
  const int nn3[3] = {m.nx, m.ny, m.nz};
  long long off = 0;
  std::vector<double> val(n2), der(n2), tv(n2), td(n2);
  std::vector<double> dera(n2), derb(n2), ta_(n2), tb_(n2);   // tangential parts (K(x) only)
  const double* G = B + 3 * n * n + 3 * n;   // layout: B, Dg, W, dl[2], M1, G, ...
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) {
      const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
      const double area = m.h[ta] * m.h[tb];
      const double sgn = s ? 1.0 : -1.0;
      const bool dir = m.bc[2 * d + s] == 0;
      for (int cb = 0; cb < nn3[tb]; ++cb)
        for (int ca = 0; ca < nn3[ta]; ++ca) {
          int idx[3];
          idx[d] = s ? nn3[d] - 1 : 0;
          idx[ta] = ca;
          idx[tb] = cb;
          const long long c = idx[0] + (long long)m.nx * (idx[1] + (long long)m.ny * idx[2]);
          const double* gv = g_qp ? g_qp + off : nullptr;
          const double* jv = j_qp ? j_qp + off : nullptr;
          off += n2;
          if (dir && !gv) continue;
          if (!dir && !jv) continue;
          const double Kd = kval(m, c, d);
          const double gam = pen * Kd / m.h[d];
          for (int qb = 0; qb < n; ++qb)
            for (int qa = 0; qa < n; ++qa) {
              const int f = qa + n * qb;
              const double w = W[qa] * W[qb] * area;
              dera[f] = derb[f] = 0.0;
              if (!dir) {
                val[f] = -w * jv[f];
                der[f] = 0.0;
                continue;
              }
              double xi[3];
              xi[d] = s;
              xi[ta] = T[4 * n * n + 5 * n + qa];   // gq
              xi[tb] = T[4 * n * n + 5 * n + qb];
              double bq[3];
              b_at(m, idx[0], idx[1], idx[2], xi, bq);
              const double bn = sgn * bq[d];
              if (m.var) {
                // K(x) at the face point: gamma from nu^T K nu, and the test
                // function's full K grad v . n (normal and tangential parts)
                double x[3], K[6];
                for (int e = 0; e < 3; ++e) x[e] = (idx[e] + xi[e]) * m.h[e];
                var_tensor(m.var, x, K);
                const double gx = pen * K[d] / m.h[d];
                val[f] = w * (gx * gv[f] - (bn < 0.0 ? bn * gv[f] : 0.0));
                der[f] = -w * gv[f] * sgn * kent_host(K, d, d) / m.h[d];
                dera[f] = -w * gv[f] * sgn * kent_host(K, ta, d) / m.h[ta];
                derb[f] = -w * gv[f] * sgn * kent_host(K, tb, d) / m.h[tb];
                continue;
              }
              val[f] = w * (gam * gv[f] - (bn < 0.0 ? bn * gv[f] : 0.0));
              der[f] = -w * Kd * gv[f] * sgn / m.h[d];
            }
          if (m.var && dir) {
            // tangential parts: (G_a^T (x) B_b^T) dera + (B_a^T (x) G_b^T) derb into the face layer
            for (int qb = 0; qb < n; ++qb)
              for (int ia = 0; ia < n; ++ia) {
                double sa = 0.0, sb = 0.0;
                for (int qa = 0; qa < n; ++qa) {
                  sa += G[qa * n + ia] * dera[qa + n * qb];
                  sb += B[qa * n + ia] * derb[qa + n * qb];
                }
                ta_[ia + n * qb] = sa;
                tb_[ia + n * qb] = sb;
              }
            for (int ib = 0; ib < n; ++ib)
              for (int ia = 0; ia < n; ++ia) {
                double sv = 0.0;
                for (int qb = 0; qb < n; ++qb)
                  sv += B[qb * n + ib] * ta_[ia + n * qb] + G[qb * n + ib] * tb_[ia + n * qb];
                int ii[3];
                ii[ta] = ia;
                ii[tb] = ib;
                ii[d] = s ? n - 1 : 0;
                rhs[c * n3 + ii[0] + n * ii[1] + n2 * ii[2]] += sv;
              }
          }
          // B^T along a then b
          for (int qb = 0; qb < n; ++qb)
            for (int ia = 0; ia < n; ++ia) {
              double sv = 0.0, sd = 0.0;
              for (int qa = 0; qa < n; ++qa) {
                sv += B[qa * n + ia] * val[qa + n * qb];
                sd += B[qa * n + ia] * der[qa + n * qb];
              }
              tv[ia + n * qb] = sv;
              td[ia + n * qb] = sd;
            }
          for (int ib = 0; ib < n; ++ib)
            for (int ia = 0; ia < n; ++ia) {
              double sv = 0.0, sd = 0.0;
              for (int qb = 0; qb < n; ++qb) {
                sv += B[qb * n + ib] * tv[ia + n * qb];
                sd += B[qb * n + ib] * td[ia + n * qb];
              }
              // dof with tangential indices (ia, ib), normal index k
              int ii[3];
              ii[ta] = ia;
              ii[tb] = ib;
              ii[d] = s ? n - 1 : 0;
              rhs[c * n3 + ii[0] + n * ii[1] + n2 * ii[2]] += sv;
              for (int k = 0; k < n; ++k) {
                ii[d] = k;
                rhs[c * n3 + ii[0] + n * ii[1] + n2 * ii[2]] += dl[s * n + k] * sd;
              }
            }
        }
    }
}

void quadrature_points_host(const HostMesh& m, double* vol, double* face) {
  const int n = m.p + 1, n2 = n * n, n3 = n2 * n;
  std::vector<double> gq, gw;
  gauss_legendre01(n, gq, gw);
  const long long ncell = (long long)m.nx * m.ny * m.nz;
  if (vol) {
    for (long long c = 0; c < ncell; ++c) {
      const int cx = (int)(c % m.nx), cy = (int)((c / m.nx) % m.ny), cz = (int)(c / ((long long)m.nx * m.ny));
      for (int q = 0; q < n3; ++q) {
        double* o = vol + 3 * (c * n3 + q);
        o[0] = (cx + gq[q % n]) * m.h[0];
        o[1] = (cy + gq[(q / n) % n]) * m.h[1];
        o[2] = (cz + gq[q / n2]) * m.h[2];
      }
    }
  }
  if (face) {
    const int nn3[3] = {m.nx, m.ny, m.nz};
    long long off = 0;
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
        for (int cb = 0; cb < nn3[tb]; ++cb)
          for (int ca = 0; ca < nn3[ta]; ++ca)
            for (int qb = 0; qb < n; ++qb)
              for (int qa = 0; qa < n; ++qa) {
                double* o = face + 3 * off++;
                o[d] = s ? nn3[d] * m.h[d] : 0.0;
                o[ta] = (ca + gq[qa]) * m.h[ta];
                o[tb] = (cb + gq[qb]) * m.h[tb];
              }
      }
  }
}

}  // namespace dgmg
