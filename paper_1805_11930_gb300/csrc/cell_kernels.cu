// Per-order kernels of the matrix-free DG operator, the block-diagonal apply,
// the fused block-Jacobi smoother and the DG <-> Q1 transfer.
//
// Built once per n = p+1 with -DDGMG_N=n.  One warp owns CPW = max(1, 32/n^2)
// whole cells; there is no block-level synchronisation, so every warp runs
// independently (cells whose inner solves take different iteration counts do
// not wait for each other beyond their own warp).  A cell's data live in
// shared memory as n x n x n arrays (x fastest).  A 1D contraction along axis
// d is done by "lines": the n^2 lines of a cell parallel to d are spread over
// the lanes, each lane loads its line into registers, multiplies it by an
// n x n matrix from constant memory and writes it back.  The same line
// decomposition gives the face node grid of the two faces normal to d.
//
// Operator (arXiv 1805.11930, Sec. 2.1, eq. bilinear_form_split):
//  volume  (K grad u - b u, grad v)_T + (c u, v)_T, evaluated by sum
//          factorisation (Sec. 3.1, Stages 1-3): u to the Gauss points by three
//          contractions with B, derivatives there by the Gauss collocation
//          derivative Dg, pointwise coefficients, Dg^T and B^T back;
//  faces   cell-centric: each cell adds the test-function side of the six face
//          integrals it touches.  With diagonal K constant per cell,
//          w^- K^- = w^+ K^+ = K^-K^+/(K^-+K^+) =: kap, so the consistency and
//          symmetry terms and the penalty reduce, per face node, to
//              qv  = gamma [[u]] - kap (dn u_in + dn u_out),   qdv = -kap [[u]],
//          integrated exactly with the 1D face mass matrix M1 (x) M1; the upwind
//          term is integrated at the face Gauss points (b varies on the face).
//  block   D_T: the same with the neighbour's trace set to zero
//          (Sec. 3.2, eq. block_diag_apply).
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "dfloat.cuh"
#include "dgmg_internal.h"

#ifndef DGMG_N
#error "compile with -DDGMG_N=<p+1>"
#endif

namespace dgmg {
namespace {

constexpr int N = DGMG_N;
constexpr int N2 = N * N;
constexpr int N3 = N * N * N;
constexpr int CPW = (N2 <= 32) ? (32 / N2) : 1;       // cells per warp
constexpr int LINES = CPW * N2;                        // lines per axis per warp
constexpr int LPL = (LINES + 31) / 32;                 // lines per lane
constexpr int VEC = CPW * N3;                          // values per warp vector
constexpr int WPB = 4;                                 // warps per block
constexpr unsigned FULLMASK = 0xffffffffu;

template <typename T>
struct Tab {
  T B[N][N];
  T Dg[N][N];
  T w[N];
  T dl[2][N];
  T M1[N][N];
  T G[N][N];
  T hat[2][N];
  T gq[N];
  T S1[N][N];
  // Derived on the host from M1, S1, dl for the factored operator (below):
  T MIS[N][N];    // M^-1 S
  T mie[2][N];    // M^-1 e_0, M^-1 e_{n-1} (columns 0 and n-1 of M^-1)
  T midl[2][N];   // M^-1 dl_0, M^-1 dl_1
};

__constant__ Tab<double> c_tab_d;
__constant__ Tab<float> c_tab_f;
__constant__ Tab<df> c_tab_df;

template <typename T>
__device__ __forceinline__ const Tab<T>& tab();
template <>
__device__ __forceinline__ const Tab<double>& tab<double>() { return c_tab_d; }
template <>
__device__ __forceinline__ const Tab<float>& tab<float>() { return c_tab_f; }
template <>
__device__ __forceinline__ const Tab<df>& tab<df>() { return c_tab_df; }

// Mesh scalars and coefficient records in the kernel's precision (no
// double arithmetic in the float kernels: the FP64 pipe is 1/64 of FP32).
template <typename T> struct Prec;
template <> struct Prec<double> {
  static __device__ __forceinline__ double ih(const MeshParams& m, int d) { return m.ih[d]; }
  static __device__ __forceinline__ double area(const MeshParams& m, int d) { return m.area[d]; }
  static __device__ __forceinline__ double jh(const MeshParams& m, int d) { return m.jh[d]; }
  static __device__ __forceinline__ double rec(const MeshParams& m, long long i) { return m.rec64[i]; }
  static __device__ __forceinline__ double bv(const MeshParams& m, long long i) { return __ldg(m.bvert + i); }
};
template <> struct Prec<float> {
  static __device__ __forceinline__ float ih(const MeshParams& m, int d) { return m.ihf[d]; }
  static __device__ __forceinline__ float area(const MeshParams& m, int d) { return m.areaf[d]; }
  static __device__ __forceinline__ float jh(const MeshParams& m, int d) { return m.jhf[d]; }
  static __device__ __forceinline__ float rec(const MeshParams& m, long long i) { return m.rec32[i]; }
  static __device__ __forceinline__ float bv(const MeshParams& m, long long i) { return __ldg(m.bvert32 + i); }
};
// double-float: the FP64 values split once per use (few per cell)
template <> struct Prec<df> {
  static __device__ __forceinline__ df ih(const MeshParams& m, int d) { return df(m.ih[d]); }
  static __device__ __forceinline__ df area(const MeshParams& m, int d) { return df(m.area[d]); }
  static __device__ __forceinline__ df jh(const MeshParams& m, int d) { return df(m.jh[d]); }
  static __device__ __forceinline__ df rec(const MeshParams& m, long long i) { return df(m.rec64[i]); }
  static __device__ __forceinline__ df bv(const MeshParams& m, long long i) { return df(__ldg(m.bvert + i)); }
};

// Values in global memory (G) and in the kernel's arithmetic (T): the same
// type, except double-float arithmetic on FP64 vectors.
template <typename T> struct Store { using type = T; };
template <> struct Store<df> { using type = double; };

__device__ __forceinline__ float shfl_x(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_x(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df shfl_x(df v, int o) { return shfl_xor(v, o); }
__device__ __forceinline__ float shfl_i(float v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ double shfl_i(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
__device__ __forceinline__ df shfl_i(df v, int src) {
  return df(__shfl_sync(0xffffffffu, v.h, src), __shfl_sync(0xffffffffu, v.l, src));
}

// Per-cell coefficients and face data staged in shared memory (computed
// once per cell; faces f = 2d + s, s = 0 low side, 1 high side).
template <typename T>
struct CellInfo {
  long long nb[6];  // neighbour cell across face f (interior faces)
  T kd[3];          // |J| K_d / h_d^2
  T cJ;             // c |J|
  T jh[3];          // |J| / h_d
  T bc[3][8];       // b_d at the 8 corners, corner = ox + 2 oy + 4 oz
  T kap[6];         // K^-K^+/(K^-+K^+) (interior) or K (Dirichlet)
  T gam[6];         // penalty gamma_F
  int kind[6];      // 0 interior, 1 Dirichlet, 2 Neumann
  int pad[2];
};

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Geometry of line L along axis D: owning cell slot cw, first element,
// stride, and the two tangential coordinates (a < b in axis order).
template <int D>
__device__ __forceinline__ void line_geom(int L, int& cw, int& base, int& st, int& a, int& b) {
  cw = L / N2;
  const int r = L - cw * N2;
  a = r % N;
  b = r / N;
  if (D == 0) {
    base = cw * N3 + N * a + N2 * b;
    st = 1;
  } else if (D == 1) {
    base = cw * N3 + a + N2 * b;
    st = N;
  } else {
    base = cw * N3 + a + N * b;
    st = N2;
  }
}

__device__ __forceinline__ void cell_xyz(const MeshParams& mp, long long c, int& cx, int& cy, int& cz) {
  cx = (int)(c % mp.nx);
  long long t = c / mp.nx;
  cy = (int)(t % mp.ny);
  cz = (int)(t / mp.ny);
}

__device__ __forceinline__ double kcoef(const MeshParams& mp, long long c, int d) {
  return __ldg(mp.K + c * mp.kdim + (mp.kdim == 3 ? d : 0));
}

// 0 = interior (nb set), 1 = Dirichlet, 2 = Neumann.
__device__ __forceinline__ int face_kind(const MeshParams& mp, long long c, int d, int s, long long& nb) {
  int cx, cy, cz;
  cell_xyz(mp, c, cx, cy, cz);
  const int ci = d == 0 ? cx : (d == 1 ? cy : cz);
  const int nd = d == 0 ? mp.nx : (d == 1 ? mp.ny : mp.nz);
  const long long stride = d == 0 ? 1LL : (d == 1 ? (long long)mp.nx : (long long)mp.nx * mp.ny);
  if ((s == 0 && ci == 0) || (s == 1 && ci == nd - 1)) return mp.bc[2 * d + s] == 0 ? 1 : 2;
  nb = s ? c + stride : c - stride;
  return 0;
}

// out = A in (or A^T in) along axis D for all lines of active cells.
template <int D, bool TR, bool ACC, typename T>
__device__ __forceinline__ void contract(const T* __restrict__ in, T* __restrict__ out,
                                         const T (&A)[N][N], int lane, const unsigned char* act) {
  for (int L = lane; L < LINES; L += 32) {
    int cw, base, st, a, b;
    line_geom<D>(L, cw, base, st, a, b);
    if (!act[cw]) continue;
    T x[N];
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = in[base + j * st];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T s;
      if constexpr (std::is_same<T, df>::value) {
        df_acc acc;
#pragma unroll
        for (int j = 0; j < N; ++j) acc.add_prod(TR ? A[j][i] : A[i][j], x[j]);
        s = acc.value();
      } else {
        s = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(TR ? A[j][i] : A[i][j], x[j], s);
      }
      if (ACC)
        out[base + i * st] += s;
      else
        out[base + i * st] = s;
    }
  }
}

// Stage 2 along axis D, fused with the derivative and its transpose:
// Y(+)= Dg^T [ w|J| (K_D/h_D^2) Dg U - w |J|/h_D b_D U ]  (+ w c|J| U for D = 0).
template <int D, bool ACC, bool ADV, bool REACT, typename T>
__device__ __forceinline__ void grad_pass(const T* __restrict__ U, T* __restrict__ Y, int lane,
                                          const CellInfo<T>* ci, const unsigned char* act) {
  const Tab<T>& t = tab<T>();
  for (int L = lane; L < LINES; L += 32) {
    int cw, base, st, a, b;
    line_geom<D>(L, cw, base, st, a, b);
    if (!act[cw]) continue;
    T u[N];
#pragma unroll
    for (int j = 0; j < N; ++j) u[j] = U[base + j * st];
    const T wab = t.w[a] * t.w[b];
    const T kd = ci[cw].kd[D] * wab;
    T lo = T(0), hi = T(0);
    if (ADV) {
      // b_D along the line is linear in xi_D: bilinear interpolation of the
      // corner values on the faces xi_D = 0 and xi_D = 1.
      const T xa = t.gq[a], xb = t.gq[b];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
        const int ka = D == 0 ? 1 : 0, kb = D == 2 ? 1 : 2;
        const T wa = o[ka] ? xa : T(1) - xa;
        const T wb = o[kb] ? xb : T(1) - xb;
        const T v = ci[cw].bc[D][c] * wa * wb;
        if (o[D])
          hi += v;
        else
          lo += v;
      }
      lo *= ci[cw].jh[D] * wab;
      hi *= ci[cw].jh[D] * wab;
    }
    const T dh = hi - lo;
    T q[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T g = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) g = fma(t.Dg[i][j], u[j], g);
      // w_i (kd g - b u), the weight applied once
      T v = kd * g;
      if (ADV) v = fma(-fma(dh, t.gq[i], lo), u[i], v);
      q[i] = t.w[i] * v;
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
      T s = T(0);
#pragma unroll
      for (int i = 0; i < N; ++i) s = fma(t.Dg[i][r], q[i], s);
      if (REACT && D == 0) s = fma(ci[cw].cJ * wab * t.w[r], u[r], s);
      if (ACC)
        Y[base + r * st] += s;
      else
        Y[base + r * st] = s;
    }
  }
}

// out (+)= scale_cw * (A in) along axis D; scale = kd[SEL] (SEL < 3) or cJ.
template <int D, bool ACC, int SEL, typename T>
__device__ __forceinline__ void contract_scaled(const T* __restrict__ in, T* __restrict__ out, const T (&A)[N][N],
                                                int lane, const unsigned char* act, const CellInfo<T>* ci) {
  for (int L = lane; L < LINES; L += 32) {
    int cw, base, st, a, b;
    line_geom<D>(L, cw, base, st, a, b);
    if (!act[cw]) continue;
    const T sc = SEL < 3 ? ci[cw].kd[SEL < 3 ? SEL : 0] : ci[cw].cJ;
    T x[N];
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = in[base + j * st];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T s;
      if constexpr (std::is_same<T, df>::value) {
        df_acc acc;
#pragma unroll
        for (int j = 0; j < N; ++j) acc.add_prod(A[i][j], x[j]);
        s = acc.value();
      } else {
        s = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(A[i][j], x[j], s);
      }
      if (ACC)
        out[base + i * st] = fma(sc, s, out[base + i * st]);
      else
        out[base + i * st] = sc * s;
    }
  }
}

// out (+)= A_cw in along axis D with a per-cell n x n matrix: A_cw at
// Am + (3 cw + D) n^2, row-major (A[i][j] multiplies in_j into out_i).
template <int D, bool ACC, typename T>
__device__ __forceinline__ void contract_cell(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ Am,
                                              int lane, const unsigned char* act) {
  for (int L = lane; L < LINES; L += 32) {
    int cw, base, st, a, b;
    line_geom<D>(L, cw, base, st, a, b);
    if (!act[cw]) continue;
    const T* A = Am + (3 * cw + D) * N2;
    T x[N];
#pragma unroll
    for (int j = 0; j < N; ++j) x[j] = in[base + j * st];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T s;
      if constexpr (std::is_same<T, df>::value) {
        df_acc acc;
#pragma unroll
        for (int j = 0; j < N; ++j) acc.add_prod(A[i * N + j], x[j]);
        s = acc.value();
      } else {
        s = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(A[i * N + j], x[j], s);
      }
      if (ACC)
        out[base + i * st] += s;
      else
        out[base + i * st] = s;
    }
  }
}

// The 1D matrices of the block D_T for b = 0: with K diagonal and constant on
// the affine cell, the volume term and the own-side parts of the face terms
// (consistency, symmetry, penalty, integrated exactly with the face mass
// M (x) M) are Kronecker products, so D_T = A_x (x) M (x) M + M (x) A_y (x) M
// + M (x) M (x) A_z with
//   A_d = |J| K_d / h_d^2 S + sum over the non-Neumann faces s of d of
//         |F| [ -kap sg / h_d (e_e dl_s^T + dl_s e_e^T) + gamma e_e e_e^T ],
// e = end node of side s, sg = +-1 its outward sign, kap = w K (K on
// Dirichlet faces), plus c |J| M in A_z.  Written to Am (3 n^2 per cell).
// FACES = false: the volume term alone (A_d = |J| K_d / h_d^2 S, c |J| M in A_z).
template <bool FACES = true, typename T>
__device__ __forceinline__ void block_matrices(const MeshParams& mp, T* Am, const CellInfo<T>* ci,
                                               const unsigned char* act, int lane) {
  const Tab<T>& t = tab<T>();
  for (int k = lane; k < CPW * 3 * N2; k += 32) {
    const int cw = k / (3 * N2), r = k - cw * 3 * N2, d = r / N2, i = (r % N2) / N, j = r % N;
    if (!act[cw]) continue;
    T a = ci[cw].kd[d] * t.S1[i][j];
    if (d == 2) a = fma(ci[cw].cJ, t.M1[i][j], a);
    const T ih = Prec<T>::ih(mp, d);
    for (int s = 0; s < 2 && FACES; ++s) {
      const int f = 2 * d + s;
      if (ci[cw].kind[f] == 2) continue;
      const int e = s ? N - 1 : 0;
      const T ks = (s ? -ci[cw].kap[f] : ci[cw].kap[f]) * ih;   // -kap sg / h_d
      T fv = T(0);
      if (i == e) fv = fma(ks, t.dl[s][j], fv);
      if (j == e) fv = fma(ks, t.dl[s][i], fv);
      if (i == e && j == e) fv = fv + ci[cw].gam[f];
      a = fma(ci[cw].jh[d], fv, a);
    }
    Am[k] = a;
  }
  __syncwarp();
}

// Element-per-lane contraction (FP64 and double-float kernels): lane work
// items are the outputs (cell, line, i) instead of whole lines, so that all 32
// lanes stay busy when n^2 lines per cell do not fill the warp (n = 5: 25
// lines -> 78 % of the lanes, 125 outputs -> 98 %).  Each output reads its
// line (n shared-memory loads) and a row of A from shared memory; that costs
// more load instructions than the line form, which the FP64 pipe can afford
// (it is the bound) but the FP32 kernels cannot (they are bound by
// shared-memory instructions), so FP32 keeps the line form.
template <int D, bool ACC, typename T>
__device__ __forceinline__ void contract_e(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ Am,
                                           int cstride, int lane, const unsigned char* act) {
  constexpr int st = D == 0 ? 1 : (D == 1 ? N : N2);
  for (int e = lane; e < VEC; e += 32) {
    const int cw = e / N3;
    if (!act[cw]) continue;
    const int r = e - cw * N3;
    const int i = D == 0 ? r % N : (D == 1 ? (r / N) % N : r / N2);
    const int base = e - i * st;
    const T* A = Am + cw * cstride + i * N;
    T s;
    if constexpr (std::is_same<T, df>::value) {
      df_acc acc;
#pragma unroll
      for (int j = 0; j < N; ++j) acc.add_prod(A[j], in[base + j * st]);
      s = acc.value();
    } else {
      s = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) s = fma(A[j], in[base + j * st], s);
    }
    if (ACC)
      out[e] += s;
    else
      out[e] = s;
  }
}

// Q = D_T P for b = 0 by the Kronecker form above: 8 contractions, no face
// passes (the face terms are inside A_d).
template <typename T>
__device__ __forceinline__ void block_kron(const T* X, T* Y, T* S0, T* S1, const T* Am, int lane,
                                           const unsigned char* act) {
  const Tab<T>& t = tab<T>();
  contract<2, false, false>(X, S0, t.M1, lane, act);   // a = M_z u
  __syncwarp();
  contract<1, false, false>(S0, S1, t.M1, lane, act);  // b = M_y a
  __syncwarp();
  contract_cell<0, false>(S1, Y, Am, lane, act);       // Y = A_x b
  __syncwarp();
  contract<0, false, false>(S0, S1, t.M1, lane, act);  // c = M_x a
  __syncwarp();
  contract_cell<1, true>(S1, Y, Am, lane, act);        // Y += A_y c
  __syncwarp();
  contract<0, false, false>(X, S0, t.M1, lane, act);   // e = M_x u
  __syncwarp();
  contract<1, false, false>(S0, S1, t.M1, lane, act);  // f = M_y e
  __syncwarp();
  contract_cell<2, true>(S1, Y, Am, lane, act);        // Y += A_z f
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Factored form of the b = 0 operator (FP64 and double-float kernels).
//
// With K diagonal and constant per affine axis-aligned cell, the block is a
// sum of Kronecker products D_T = sum_d A_d (x)_d M (x) M (reading of the
// block matrices above), and M (the 1D mass matrix of the GLL basis under the
// Gauss rule) is symmetric positive definite, so
//     D_T = (M (x) M (x) M) o sum_d (M^-1 A_d) x_d ,
// with x_d the 1D product along axis d.  One fused pass applies the three
// per-cell matrices Ah_d = M^-1 A_d to every element (3n multiply-adds), then
// three passes apply M along z, y, x (3n): 6 n^4 multiply-adds per cell
// instead of 8 n^4 for the eight-contraction sequence.  The neighbour terms of
// the full operator enter the same way: a face term e_e (x) (M (x) M) q (or
// dl_s (x) (M (x) M) q) equals (M (x) M (x) M)((M^-1 e_e) (x) q), so the
// neighbour's face values are added before the mass passes, weighted by the
// tabulated vectors M^-1 e_e and M^-1 dl_s, and need no contraction of their
// own.  Same operator up to rounding (M has condition number below 20 for
// n <= 9).

// Mass matrix and the vectors M^-1 e_e, M^-1 dl_s in shared memory (their
// index varies across the lanes, which constant memory would serialise):
// M1s[i N + j] = M[i][j]; MVs = [mie_0 | mie_1 | midl_0 | midl_1].
template <typename T>
__device__ __forceinline__ void factor_tables(T* M1s, T* MVs, int lane) {
  const Tab<T>& t = tab<T>();
  for (int k = lane; k < N2; k += 32) M1s[k] = t.M1[k / N][k % N];
  for (int k = lane; k < 4 * N; k += 32) {
    const int q = k / N, i = k % N;
    MVs[k] = q < 2 ? t.mie[q][i] : t.midl[q - 2][i];
  }
}

// Per cell slot and face f = 2d + s, the factors the face terms share (kept
// in FC, 4 values per face, computed once per cell so that the per-entry and
// per-node work is one product less each):
//   FC[0] = -|F| gamma,  FC[1] = -|F| kap sg / h_d,  FC[2] = |J|/h_d ks,
//   FC[3] = |J|/h_d gamma,  ks = -kap sg / h_d, sg = +-1 the outward sign.
template <typename T, int C = CPW>
__device__ __forceinline__ void face_consts(T* FC, const MeshParams& mp, const CellInfo<T>* ci,
                                            const unsigned char* act, int lane) {
  for (int it = lane; it < C * 6; it += 32) {
    const int cw = it / 6, f = it - cw * 6, d = f >> 1, S = f & 1;
    if (!act[cw]) continue;
    const T ih = Prec<T>::ih(mp, d), area = Prec<T>::area(mp, d);
    const T kap = ci[cw].kap[f], gam = ci[cw].gam[f], jh = ci[cw].jh[d];
    const T skap = S ? -kap : kap;
    T* q = FC + it * 4;
    q[0] = -area * gam;
    q[1] = skap * (area * ih);
    q[2] = jh * (skap * ih);
    q[3] = jh * gam;
  }
}

// Ah_d = M^-1 A_d of every staged cell, 3 n^2 per cell (row-major; Ah_d[i][j]
// multiplies x_j into z_i):
//   M^-1 A_d = |J| K_d / h_d^2 M^-1 S + [d = 2] c |J| I
//            + sum over the non-Neumann faces s of d of
//              |F| [ ks ((M^-1 e_e) dl_s^T + (M^-1 dl_s) e_e^T) + gamma (M^-1 e_e) e_e^T ],
// ks = -kap sg / h_d, e = end node of side s, sg = +-1 its outward sign
// (|F| = |J| / h_d on these cells); fc: the cell's face factors.
template <typename T>
__device__ __forceinline__ T hat_entry(const CellInfo<T>& c, const T* fc, int d, int i, int j) {
  const Tab<T>& t = tab<T>();
  T a = c.kd[d] * t.MIS[i][j];
  if (d == 2 && i == j) a = a + c.cJ;
  for (int s = 0; s < 2; ++s) {
    const int f = 2 * d + s;
    if (c.kind[f] == 2) continue;
    const T* q = fc + f * 4;
    const T me = t.mie[s][i];
    a = fma(q[2] * me, t.dl[s][j], a);
    if (j == (s ? N - 1 : 0)) a = fma(q[2], t.midl[s][i], fma(q[3], me, a));
  }
  return a;
}

template <typename T>
__device__ __forceinline__ void hat_matrices(T* Ah, const T* FC, const CellInfo<T>* ci, const unsigned char* act,
                                             int lane) {
  for (int k = lane; k < CPW * 3 * N2; k += 32) {
    const int cw = k / (3 * N2), r = k - cw * 3 * N2, d = r / N2, i = (r % N2) / N, j = r % N;
    if (!act[cw]) continue;
    Ah[k] = hat_entry(ci[cw], FC + cw * 24, d, i, j);
  }
}

// The neighbour side of the interior faces, for the full operator: at face
// point L of face f = 2d + s of cell slot cw, from the neighbour's trace
// u_o = u_nb(end 1-s) and normal derivative dn_o = sg / h_d sum_j dl_{1-s}[j] u_nb(j),
//   FS[cw][f][0][L] = |F| (-gamma u_o - kap dn_o),   FS[cw][f][1][L] = sg |F| / h_d kap u_o,
// (zero on boundary faces): the parts of qv = gamma [[u]] - kap (dn + dn_o),
// qdv = -kap [[u]] that the block D_T leaves out.  12 n^2 values per cell;
// FC the face factors of face_consts.
template <typename T, typename G, int C = CPW>
__device__ __forceinline__ void neighbour_faces(T* FS, const T* FC, const G* __restrict__ gu, int lane,
                                                const unsigned char* act, const CellInfo<T>* ci) {
  const Tab<T>& t = tab<T>();
  for (int it = lane; it < C * 6 * N2; it += 32) {
    const int cw = it / (6 * N2), r = it - cw * 6 * N2, f = r / N2, L = r - f * N2;
    const int d = f >> 1, S = f & 1;
    T qv = T(0), qd = T(0);
    if (act[cw] && ci[cw].kind[f] == 0) {
      const int a = L % N, b = L / N;
      const int st = d == 0 ? 1 : (d == 1 ? N : N2);
      const int base = d == 0 ? N * a + N2 * b : (d == 1 ? a + N2 * b : a + N * b);
      const G* xo = gu + ci[cw].nb[f] * N3 + base;
      const T tout = T(xo[(S ? 0 : N - 1) * st]);
      T dno;
      if constexpr (std::is_same<T, df>::value) {
        df_acc acc;
#pragma unroll
        for (int j = 0; j < N; ++j) acc.add_prod(t.dl[1 - S][j], T(xo[j * st]));
        dno = acc.value();
      } else {
        dno = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) dno = fma(t.dl[1 - S][j], T(xo[j * st]), dno);
      }
      const T* q = FC + (cw * 6 + f) * 4;
      qv = fma(q[0], tout, q[1] * dno);
      qd = -q[1] * tout;
    }
    T* fs = FS + (cw * 6 + f) * 2 * N2;
    fs[L] = qv;
    fs[N2 + L] = qd;
  }
}

// Z = sum_d Ah_d x_d X for the active cells, plus (FULL) the neighbour face
// values weighted by M^-1 e_e and M^-1 dl_s along each face normal.
template <bool FULL, typename T>
__device__ __forceinline__ void hat_pass(const T* X, T* Z, const T* Ah, const T* MVs, const T* FS, int lane,
                                         const unsigned char* act) {
  for (int e = lane; e < VEC; e += 32) {
    const int cw = e / N3;
    if (!act[cw]) continue;
    const int r = e - cw * N3;
    const int i0 = r % N, i1 = (r / N) % N, i2 = r / N2;
    const T* x = X + cw * N3;
    const T* ax = Ah + cw * 3 * N2 + i0 * N;
    const T* ay = Ah + cw * 3 * N2 + N2 + i1 * N;
    const T* az = Ah + cw * 3 * N2 + 2 * N2 + i2 * N;
    const int bx = r - i0, by = r - i1 * N, bz = r - i2 * N2;
    const T* fs = FS + cw * 12 * N2;
    const int L0 = i1 + N * i2, L1 = i0 + N * i2, L2 = i0 + N * i1;
    T s;
    if constexpr (std::is_same<T, df>::value) {
      df_acc acc;
#pragma unroll
      for (int j = 0; j < N; ++j) acc.add_prod(ax[j], x[bx + j]);
#pragma unroll
      for (int j = 0; j < N; ++j) acc.add_prod(ay[j], x[by + j * N]);
#pragma unroll
      for (int j = 0; j < N; ++j) acc.add_prod(az[j], x[bz + j * N2]);
      if (FULL) {
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          acc.add_prod(MVs[sd * N + i0], fs[(0 + sd) * 2 * N2 + L0]);
          acc.add_prod(MVs[2 * N + sd * N + i0], fs[(0 + sd) * 2 * N2 + N2 + L0]);
          acc.add_prod(MVs[sd * N + i1], fs[(2 + sd) * 2 * N2 + L1]);
          acc.add_prod(MVs[2 * N + sd * N + i1], fs[(2 + sd) * 2 * N2 + N2 + L1]);
          acc.add_prod(MVs[sd * N + i2], fs[(4 + sd) * 2 * N2 + L2]);
          acc.add_prod(MVs[2 * N + sd * N + i2], fs[(4 + sd) * 2 * N2 + N2 + L2]);
        }
      }
      s = acc.value();
    } else {
      s = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) s = fma(ax[j], x[bx + j], s);
#pragma unroll
      for (int j = 0; j < N; ++j) s = fma(ay[j], x[by + j * N], s);
#pragma unroll
      for (int j = 0; j < N; ++j) s = fma(az[j], x[bz + j * N2], s);
      if (FULL) {
#pragma unroll
        for (int sd = 0; sd < 2; ++sd) {
          s = fma(MVs[sd * N + i0], fs[(0 + sd) * 2 * N2 + L0], s);
          s = fma(MVs[2 * N + sd * N + i0], fs[(0 + sd) * 2 * N2 + N2 + L0], s);
          s = fma(MVs[sd * N + i1], fs[(2 + sd) * 2 * N2 + L1], s);
          s = fma(MVs[2 * N + sd * N + i1], fs[(2 + sd) * 2 * N2 + N2 + L1], s);
          s = fma(MVs[sd * N + i2], fs[(4 + sd) * 2 * N2 + L2], s);
          s = fma(MVs[2 * N + sd * N + i2], fs[(4 + sd) * 2 * N2 + N2 + L2], s);
        }
      }
    }
    Z[e] = s;
  }
}

// Y = A X (FULL, neighbour values from gu) or D_T X in the factored form;
// S0, S1 scratch vectors, Ah, M1s, MVs, FS as above, the face factors FC
// (face_consts) right after FS.  X and Y distinct from S0 and S1.
template <bool FULL, typename T, typename G>
__device__ __forceinline__ void factored_apply(const T* X, T* Y, T* S0, T* S1, const T* Ah, const T* M1s,
                                               const T* MVs, T* FS, const G* gu, int lane,
                                               const unsigned char* act, const CellInfo<T>* ci) {
  if (FULL) {
    neighbour_faces(FS, FS + 12 * CPW * N2, gu, lane, act, ci);
    __syncwarp();
  }
  hat_pass<FULL>(X, S0, Ah, MVs, FS, lane, act);
  __syncwarp();
  contract_e<2, false>(S0, S1, M1s, 0, lane, act);
  __syncwarp();
  contract_e<1, false>(S1, S0, M1s, 0, lane, act);
  __syncwarp();
  contract_e<0, false>(S0, Y, M1s, 0, lane, act);
  __syncwarp();
}

// Shared values per warp of the factored form: Ah (3 CPW n^2), M1s (n^2),
// MVs (4 n), FS (12 CPW n^2), FC (24 CPW).
constexpr int kFactorExtra = 3 * CPW * N2 + N2 + 4 * N + 12 * CPW * N2 + 24 * CPW;

// The per-cell matrices and the tables of the factored form (Ah, M1s, MVs as
// above; FC = FS + 12 CPW n^2 receives the face factors first).
template <typename T>
__device__ __forceinline__ void factor_setup(T* Ah, T* M1s, T* MVs, T* FS, const MeshParams& mp,
                                             const CellInfo<T>* ci, const unsigned char* act, int lane) {
  T* FC = FS + 12 * CPW * N2;
  face_consts(FC, mp, ci, act, lane);
  factor_tables(M1s, MVs, lane);
  __syncwarp();
  hat_matrices(Ah, FC, ci, act, lane);
  __syncwarp();
}


// Y = A^v X for the warp's cells.  S0, S1 scratch.
//  b = 0: K and c are constant per cell and the cell affine, so the volume
//   matrix is exactly sum_d |J| K_d / h_d^2 (S (x) M (x) M)_d + c |J| M (x) M (x) M
//   with the 1D stiffness S = G^T W G and mass M = B^T W B of the GLL basis
//   under the Gauss rule: 8 contractions (9 with c), no pointwise work.
//  b != 0: the three stages of Sec. 3.1 at the Gauss points (B, fused
//   Dg / coefficients / Dg^T, B^T), since b varies inside the cell.
template <bool ADV, typename T>
__device__ __forceinline__ void volume(const T* X, T* Y, T* S0, T* S1, int lane, const CellInfo<T>* ci,
                                       const unsigned char* act, bool react) {
  const Tab<T>& t = tab<T>();
  if (!ADV) {
    contract<2, false, false>(X, S0, t.M1, lane, act);          // a = M_z u
    __syncwarp();
    contract<1, false, false>(S0, S1, t.M1, lane, act);         // b = M_y a
    __syncwarp();
    contract_scaled<0, false, 0>(S1, Y, t.S1, lane, act, ci);   // Y = kx S_x b
    __syncwarp();
    contract<0, false, false>(S0, S1, t.M1, lane, act);         // c = M_x a
    __syncwarp();
    contract_scaled<1, true, 1>(S1, Y, t.S1, lane, act, ci);    // Y += ky S_y c
    __syncwarp();
    contract<0, false, false>(X, S0, t.M1, lane, act);          // e = M_x u
    __syncwarp();
    contract<1, false, false>(S0, S1, t.M1, lane, act);         // f = M_y e
    __syncwarp();
    contract_scaled<2, true, 2>(S1, Y, t.S1, lane, act, ci);    // Y += kz S_z f
    if (react) {
      __syncwarp();
      contract_scaled<2, true, 3>(S1, Y, t.M1, lane, act, ci);  // Y += c|J| M_z f
    }
    __syncwarp();
    return;
  }
  contract<0, false, false>(X, S0, t.B, lane, act);
  __syncwarp();
  contract<1, false, false>(S0, S1, t.B, lane, act);
  __syncwarp();
  contract<2, false, false>(S1, S0, t.B, lane, act);   // S0 = u at the Gauss points
  __syncwarp();
  grad_pass<0, false, ADV, true>(S0, S1, lane, ci, act);   // c|J| = 0 without reaction
  __syncwarp();
  grad_pass<1, true, ADV, false>(S0, S1, lane, ci, act);
  __syncwarp();
  grad_pass<2, true, ADV, false>(S0, S1, lane, ci, act);
  __syncwarp();
  contract<2, true, false>(S1, S0, t.B, lane, act);
  __syncwarp();
  contract<1, true, false>(S0, S1, t.B, lane, act);
  __syncwarp();
  contract<0, true, false>(S1, Y, t.B, lane, act);
  __syncwarp();
}

// Diffusion and penalty terms of both faces normal to axis D (s = 0, 1) of
// every active cell, added to Y.  The lines along D give both faces' node
// grids, so each own line is loaded once for the two faces.  F points to
// 4 * LINES scratch values (qv, qdv of face 0, then of face 1).
template <int D, bool FULL, typename T, typename G>
__device__ __forceinline__ void faces_diffusion_dir(const T* X, T* Y, T* F, const G* __restrict__ gu,
                                                    const MeshParams& mp, int lane, const unsigned char* act,
                                                    const CellInfo<T>* ci) {
  const Tab<T>& t = tab<T>();
  const T ih = Prec<T>::ih(mp, D);
  const T area = Prec<T>::area(mp, D);
  // phase 1: qv, qdv of both faces at the face nodes
  for (int L = lane; L < LINES; L += 32) {
    int cw, base, st, a, b;
    line_geom<D>(L, cw, base, st, a, b);
    T q[4] = {T(0), T(0), T(0), T(0)};
    if (act[cw]) {
      T x[N];
#pragma unroll
      for (int j = 0; j < N; ++j) x[j] = X[base + j * st];
#pragma unroll
      for (int S = 0; S < 2; ++S) {
        const int f = 2 * D + S;
        const int kind = ci[cw].kind[f];
        if (kind == 2) continue;
        const T sgn = S ? T(1) : T(-1);
        const T xin = x[S ? N - 1 : 0];
        T dn = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) dn = fma(t.dl[S][j], x[j], dn);
        dn *= sgn * ih;
        const T kap = ci[cw].kap[f];
        const T gam = ci[cw].gam[f];
        T tout = T(0), dno = T(0);
        if (FULL && kind == 0) {
          const G* xo = gu + ci[cw].nb[f] * N3 + (base - cw * N3);
          T y[N];
#pragma unroll
          for (int j = 0; j < N; ++j) y[j] = T(xo[j * st]);
          tout = y[S ? 0 : N - 1];
#pragma unroll
          for (int j = 0; j < N; ++j) dno = fma(t.dl[1 - S][j], y[j], dno);
          dno *= sgn * ih;
        }
        const T jmp = xin - tout;
        q[2 * S] = gam * jmp - kap * (dn + dno);
        q[2 * S + 1] = -kap * jmp;
      }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) F[k * LINES + L] = q[k];
  }
  __syncwarp();
  // phase 2: M1 along the first tangential axis, four fields
  T r[4][LPL];
#pragma unroll
  for (int k = 0; k < LPL; ++k) {
    const int L = lane + 32 * k;
#pragma unroll
    for (int fld = 0; fld < 4; ++fld) r[fld][k] = T(0);
    if (L < LINES) {
      const int cw = L / N2, rr = L - cw * N2, a = rr % N, b = rr / N;
      const int row = cw * N2 + N * b;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const T m = t.M1[a][j];
#pragma unroll
        for (int fld = 0; fld < 4; ++fld) r[fld][k] = fma(m, F[fld * LINES + row + j], r[fld][k]);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < LPL; ++k) {
    const int L = lane + 32 * k;
    if (L < LINES)
#pragma unroll
      for (int fld = 0; fld < 4; ++fld) F[fld * LINES + L] = r[fld][k];
  }
  __syncwarp();
  // phase 3: M1 along the second tangential axis, then scatter both faces
  for (int L = lane; L < LINES; L += 32) {
    int cw, base, st, a, b;
    line_geom<D>(L, cw, base, st, a, b);
    if (!act[cw]) continue;
    const int col = cw * N2 + a;
    T m[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const T mm = t.M1[b][j];
#pragma unroll
      for (int fld = 0; fld < 4; ++fld) m[fld] = fma(mm, F[fld * LINES + col + N * j], m[fld]);
    }
    const T d0 = -area * ih * m[1];   // sgn = -1 on face 0
    const T d1 = area * ih * m[3];
    Y[base] = fma(area, m[0], Y[base]);
    Y[base + (N - 1) * st] = fma(area, m[2], Y[base + (N - 1) * st]);
#pragma unroll
    for (int j = 0; j < N; ++j)
      Y[base + j * st] = fma(t.dl[0][j], d0, fma(t.dl[1][j], d1, Y[base + j * st]));
  }
  __syncwarp();
}

// Upwind term of face (D, S): int_F Phi(u_in, u_out, b.n) v_in at the face
// Gauss points (b.n from the bilinear interpolation of the face corners).
template <int D, int S, bool FULL, typename T, typename G>
__device__ __forceinline__ void face_upwind(const T* X, T* Y, T* F0, T* F1, const G* __restrict__ gu,
                                            const MeshParams& mp, long long cell0, int lane,
                                            const unsigned char* act, const CellInfo<T>* ci) {
  const Tab<T>& t = tab<T>();
  constexpr int lin = S ? N - 1 : 0;
  constexpr int lout = S ? 0 : N - 1;
  const int ta = D == 0 ? 1 : 0, tb = D == 2 ? 1 : 2;
  const T area = Prec<T>::area(mp, D);
  const T sgn = S ? T(1) : T(-1);
  // phase 1: traces at the face nodes
  for (int L = lane; L < LINES; L += 32) {
    int cw, base, st, a, b;
    line_geom<D>(L, cw, base, st, a, b);
    T tin = T(0), tout = T(0);
    const int kind = act[cw] ? ci[cw].kind[2 * D + S] : 2;
    if (kind != 2) {
      tin = X[base + lin * st];
      if (kind == 0 && FULL) tout = T(gu[ci[cw].nb[2 * D + S] * N3 + (base - cw * N3) + lout * st]);
    }
    F0[L] = tin;
    F1[L] = tout;
  }
  __syncwarp();
  // phase 2: B along the first tangential axis (nodes -> Gauss points)
  T r0[LPL], r1[LPL];
#pragma unroll
  for (int k = 0; k < LPL; ++k) {
    const int L = lane + 32 * k;
    r0[k] = T(0);
    r1[k] = T(0);
    if (L < LINES) {
      const int cw = L / N2, r = L - cw * N2, a = r % N, b = r / N;
      const int row = cw * N2 + N * b;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        r0[k] = fma(t.B[a][j], F0[row + j], r0[k]);
        r1[k] = fma(t.B[a][j], F1[row + j], r1[k]);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < LPL; ++k) {
    const int L = lane + 32 * k;
    if (L < LINES) {
      F0[L] = r0[k];
      F1[L] = r1[k];
    }
  }
  __syncwarp();
  // phase 3: B along the second axis, flux at the Gauss point (qa, qb)
#pragma unroll
  for (int k = 0; k < LPL; ++k) {
    const int L = lane + 32 * k;
    r0[k] = T(0);
    if (L < LINES) {
      const int cw = L / N2, r = L - cw * N2, qa = r % N, qb = r / N;
      if (act[cw]) {
        const int col = cw * N2 + qa;
        T ti = T(0), to = T(0);
#pragma unroll
        for (int j = 0; j < N; ++j) {
          ti = fma(t.B[qb][j], F0[col + N * j], ti);
          to = fma(t.B[qb][j], F1[col + N * j], to);
        }
        const T xa = t.gq[qa], xb = t.gq[qb];
        T bn = T(0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
          if (o[D] != S) continue;
          const T wa = o[ta] ? xa : T(1) - xa;
          const T wb = o[tb] ? xb : T(1) - xb;
          bn = fma(ci[cw].bc[D][c], wa * wb, bn);
        }
        bn *= sgn;
        r0[k] = t.w[qa] * t.w[qb] * area * bn * (bn >= T(0) ? ti : to);
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < LPL; ++k) {
    const int L = lane + 32 * k;
    if (L < LINES) F0[L] = r0[k];
  }
  __syncwarp();
  // phase 4: B^T along the second axis
#pragma unroll
  for (int k = 0; k < LPL; ++k) {
    const int L = lane + 32 * k;
    r0[k] = T(0);
    if (L < LINES) {
      const int cw = L / N2, r = L - cw * N2, a = r % N, b = r / N;
      const int col = cw * N2 + a;
#pragma unroll
      for (int j = 0; j < N; ++j) r0[k] = fma(t.B[j][b], F0[col + N * j], r0[k]);
    }
  }
  __syncwarp();
#pragma unroll
  for (int k = 0; k < LPL; ++k) {
    const int L = lane + 32 * k;
    if (L < LINES) F0[L] = r0[k];
  }
  __syncwarp();
  // phase 5: B^T along the first axis, add to the face layer of Y
  for (int L = lane; L < LINES; L += 32) {
    int cw, base, st, a, b;
    line_geom<D>(L, cw, base, st, a, b);
    if (!act[cw]) continue;
    const int row = cw * N2 + N * b;
    T s = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) s = fma(t.B[j][a], F0[row + j], s);
    Y[base + lin * st] += s;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Element form of the operator with advection (b != 0): the lane work items
// are single outputs, as in the factored form, so that all 32 lanes stay busy
// at every order (the line form leaves 7 of 32 lanes idle at n = 5 and takes
// five synchronised phases per face).
//
// Tables in shared memory (their index varies across the lanes, which
// constant memory would serialise):
// AT = [B | B^T | Dg | Dg^T | M | W2], n^2 each, row-major, W2[i + n j] =
// w_i w_j; then [w | gq | dl_0 | dl_1], n each.
constexpr int kAdvTab = 6 * N2 + 4 * N;

template <typename T>
__device__ __forceinline__ void adv_tables(T* AT, int lane) {
  const Tab<T>& t = tab<T>();
  for (int k = lane; k < N2; k += 32) {
    const int i = k / N, j = k % N;
    AT[k] = t.B[i][j];
    AT[N2 + k] = t.B[j][i];
    AT[2 * N2 + k] = t.Dg[i][j];
    AT[3 * N2 + k] = t.Dg[j][i];
    AT[4 * N2 + k] = t.M1[i][j];
    AT[5 * N2 + k] = t.w[j] * t.w[i];
  }
  for (int k = lane; k < N; k += 32) {
    AT[6 * N2 + k] = t.w[k];
    AT[6 * N2 + N + k] = t.gq[k];
    AT[6 * N2 + 2 * N + k] = t.dl[0][k];
    AT[6 * N2 + 3 * N + k] = t.dl[1][k];
  }
}

// Per cell slot and direction D the separable factors of the pointwise
// volume coefficients at the Gauss points.  b_D is trilinear on the cell, so
// b_D(x, y, z) = c0(x, y) + z c1(x, y) with c0 the bilinear blend of the
// z = 0 corners and c1 that of the z = 1 corners minus c0:
//   BT[(cw 3 + D) 3 n^2 + {0, 1, 2} n^2 + i0 + n i1]
//     = |J|/h_D w_i0 w_i1 {c0, c1} (gq_i0, gq_i1),  |J| K_D / h_D^2 w_i0 w_i1,
// so that at Gauss point (i0, i1, i2) w3 |J|/h_D b_D = w_i2 (c0' + gq_i2 c1')
// and w3 |J| K_D / h_D^2 = w_i2 k': the flux is w_i2 (k' g - (c0' + gq_i2 c1') u).
template <typename T>
__device__ __forceinline__ void adv_point_tables(T* BT, const T* AT, int lane, const CellInfo<T>* ci,
                                                 const unsigned char* act) {
  const Tab<T>& t = tab<T>();
  for (int it = lane; it < CPW * 3 * N2; it += 32) {
    const int cw = it / (3 * N2), r = it - cw * 3 * N2, D = r / N2, L = r - D * N2;
    if (!act[cw]) continue;
    const int i0 = L % N, i1 = L / N;
    const T x = t.gq[i0], y = t.gq[i1];
    const T* b = ci[cw].bc[D];
    const T b00 = fma(x, b[1] - b[0], b[0]), b10 = fma(x, b[3] - b[2], b[2]);
    const T b01 = fma(x, b[5] - b[4], b[4]), b11 = fma(x, b[7] - b[6], b[6]);
    const T c0 = fma(y, b10 - b00, b00), c1 = fma(y, b11 - b01, b01) - c0;
    const T w2 = AT[5 * N2 + L];
    T* bt = BT + (cw * 3 + D) * 3 * N2;
    bt[L] = ci[cw].jh[D] * w2 * c0;
    bt[N2 + L] = ci[cw].jh[D] * w2 * c1;
    bt[2 * N2 + L] = ci[cw].kd[D] * w2;
  }
}

// Y = A^v X with advection at the Gauss points (Sec. 3.1's three stages):
// U = (B (x) B (x) B) X; per direction D the pointwise flux
// Q = w (|J| K_D / h_D^2 Dg_D U - |J| / h_D b_D U) and E (+)= Dg_D^T Q, with the
// reaction c |J| w U added once; Y = (B^T (x) B^T (x) B^T) E.  Element passes;
// S0, S1, E scratch vectors; AT the shared tables; BT scratch for the point
// factors of adv_point_tables (9 n^2 values per cell slot).
template <typename T>
__device__ __forceinline__ void volume_adv_e(const T* X, T* Y, T* S0, T* S1, T* E, const T* AT, T* BT, int lane,
                                             const CellInfo<T>* ci, const unsigned char* act) {
  const T* Bs = AT;
  const T* Bts = AT + N2;
  const T* Ds = AT + 2 * N2;
  const T* Dts = AT + 3 * N2;
  contract_e<0, false>(X, S1, Bs, 0, lane, act);
  __syncwarp();
  contract_e<1, false>(S1, S0, Bs, 0, lane, act);
  __syncwarp();
  contract_e<2, false>(S0, S1, Bs, 0, lane, act);   // S1 = u at the Gauss points
  adv_point_tables(BT, AT, lane, ci, act);
  __syncwarp();
  const T* W2 = AT + 5 * N2;
  const T* Wq = AT + 6 * N2;
#pragma unroll
  for (int D = 0; D < 3; ++D) {
    const int st = D == 0 ? 1 : (D == 1 ? N : N2);
    for (int e = lane; e < VEC; e += 32) {
      const int cw = e / N3;
      if (!act[cw]) continue;
      const int r = e - cw * N3;
      const int i0 = r % N, i1 = (r / N) % N, i2 = r / N2;
      const int id = D == 0 ? i0 : (D == 1 ? i1 : i2);
      const T* line = S1 + (e - id * st);
      const T* dr = Ds + id * N;
      T g = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) g = fma(dr[j], line[j * st], g);
      const T* bt = BT + (cw * 3 + D) * 3 * N2 + i0 + N * i1;
      const T bq = fma(Wq[N + i2], bt[N2], bt[0]);   // w3 |J|/h_D b_D / w_i2
      S0[e] = Wq[i2] * fma(bt[2 * N2], g, -bq * S1[e]);
    }
    __syncwarp();
    for (int e = lane; e < VEC; e += 32) {
      const int cw = e / N3;
      if (!act[cw]) continue;
      const int r = e - cw * N3;
      const int i0 = r % N, i1 = (r / N) % N, i2 = r / N2;
      const int id = D == 0 ? i0 : (D == 1 ? i1 : i2);
      const T* line = S0 + (e - id * st);
      const T* dr = Dts + id * N;
      T acc;
      if (D == 0)
        acc = ci[cw].cJ * (W2[i0 + N * i1] * Wq[i2]) * S1[e];
      else
        acc = E[e];
#pragma unroll
      for (int j = 0; j < N; ++j) acc = fma(dr[j], line[j * st], acc);
      E[e] = acc;
    }
    __syncwarp();
  }
  contract_e<2, false>(E, S0, Bts, 0, lane, act);
  __syncwarp();
  contract_e<1, false>(S0, S1, Bts, 0, lane, act);
  __syncwarp();
  contract_e<0, false>(S1, Y, Bts, 0, lane, act);
  __syncwarp();
}

// The face terms with advection, element passes, for the faces FB ..
// FB + kAdvNF - 1 (FULL: with the neighbours' values from gu; else the block
// D_T, neighbour values 0):
//  1. per (face, node): qv = gamma [[u]] - kap (dn u + dn u_nb), qdv = -kap [[u]]
//     (consistency, symmetry and penalty, as in faces_diffusion_dir) and the
//     traces u_in, u_out;
//  2. along the first tangential axis: M for qv, qdv; B (nodes to Gauss
//     points) for the traces;
//  3. along the second: M for qv, qdv; B for the traces and, at the face
//     Gauss point, the upwind flux w |F| b.n (b.n >= 0 ? u_in : u_out);
//  4, 5. B^T along the second, then the first tangential axis (the flux's
//     test functions at the face nodes);
//  6. per element: the face-layer values and the normal-derivative test
//     functions of the group's faces added to Y.
// Faces per group: all six at once, or for n >= 7 the two of one direction
// at a time, so that the face scratch fits where the volume term keeps its
// Gauss-point accumulator and more warps fit on an SM (measured on GB300 in
// FP64: 2.09 against 1.59 GDOF/s at n = 7, 2.19 against 2.35 at n = 6).
// FS: kAdvFace values per cell slot (two areas of 4 fields per face); AT the
// shared tables.
constexpr int kAdvNF = N >= 7 ? 2 : 6;
constexpr int kAdvFace = 8 * kAdvNF * N2;

template <bool FULL, int FB, typename T, typename G>
__device__ void faces_adv_e(const T* X, T* Y, T* FS, const T* AT, const G* __restrict__ gu, const MeshParams& mp,
                            int lane, const unsigned char* act, const CellInfo<T>* ci) {
  constexpr int NF = kAdvNF;
  const Tab<T>& t = tab<T>();
  const T* Bs = AT;
  const T* Ms = AT + 4 * N2;
  const T* DL = AT + 6 * N2 + 2 * N;   // dl_0, dl_1
  auto A0 = [&](int cw, int fl, int fld) { return FS + ((cw * 2 + 0) * 4 * NF + fl * 4 + fld) * N2; };
  auto A1 = [&](int cw, int fl, int fld) { return FS + ((cw * 2 + 1) * 4 * NF + fl * 4 + fld) * N2; };
  // 1. face-node values
  for (int it = lane; it < CPW * NF * N2; it += 32) {
    const int cw = it / (NF * N2), r = it - cw * NF * N2, fl = r / N2, L = r - fl * N2;
    const int f = FB + fl, d = f >> 1, S = f & 1;
    T qv = T(0), qdv = T(0), tin = T(0), tout = T(0);
    if (act[cw] && ci[cw].kind[f] != 2) {
      const int a = L % N, b = L / N;
      const int st = d == 0 ? 1 : (d == 1 ? N : N2);
      const int base = cw * N3 + (d == 0 ? N * a + N2 * b : (d == 1 ? a + N2 * b : a + N * b));
      const T ih = Prec<T>::ih(mp, d);
      const T sgn = S ? T(1) : T(-1);
      T dn = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) dn = fma(t.dl[S][j], X[base + j * st], dn);
      dn = dn * sgn * ih;
      tin = X[base + (S ? N - 1 : 0) * st];
      T dno = T(0);
      if (FULL && ci[cw].kind[f] == 0) {
        const G* xo = gu + ci[cw].nb[f] * N3 + (base - cw * N3);
        tout = T(xo[(S ? 0 : N - 1) * st]);
#pragma unroll
        for (int j = 0; j < N; ++j) dno = fma(t.dl[1 - S][j], T(xo[j * st]), dno);
        dno = dno * sgn * ih;
      }
      const T kap = ci[cw].kap[f];
      const T jmp = tin - tout;
      qv = ci[cw].gam[f] * jmp - kap * (dn + dno);
      qdv = -kap * jmp;
    }
    A0(cw, fl, 0)[L] = qv;
    A0(cw, fl, 1)[L] = qdv;
    A0(cw, fl, 2)[L] = tin;
    A0(cw, fl, 3)[L] = tout;
  }
  __syncwarp();
  // 2. first tangential axis: A1[L = a + N b] = sum_j Mat[a][j] A0[j + N b]
  for (int it = lane; it < CPW * 4 * NF * N2; it += 32) {
    const int cw = it / (4 * NF * N2), r = it - cw * 4 * NF * N2, ff = r / N2, L = r - ff * N2;
    const int fl = ff >> 2, fld = ff & 3, a = L % N, b = L / N;
    const T* src = A0(cw, fl, fld) + N * b;
    const T* m = (fld < 2 ? Ms : Bs) + a * N;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) acc = fma(m[j], src[j], acc);
    A1(cw, fl, fld)[L] = acc;
  }
  __syncwarp();
  // 3. second tangential axis: qv, qdv by M into A0; the traces by B and the
  //    upwind flux at the face Gauss point (qa, qb) into A0[..][2]
  for (int it = lane; it < CPW * 3 * NF * N2; it += 32) {
    const int cw = it / (3 * NF * N2), r = it - cw * 3 * NF * N2;
    if (r < 2 * NF * N2) {
      const int ff = r / N2, L = r - ff * N2, fl = ff >> 1, fld = ff & 1, a = L % N, b = L / N;
      const int f = FB + fl;
      const T* src = A1(cw, fl, fld) + a;
      const T* m = Ms + b * N;
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) acc = fma(m[j], src[j * N], acc);
      // the face measure, and for the normal-derivative test functions the
      // outward 1/h, applied here once per face node
      const int d = f >> 1;
      const T area = Prec<T>::area(mp, d);
      const T ah = (f & 1) ? area * Prec<T>::ih(mp, d) : -(area * Prec<T>::ih(mp, d));
      A0(cw, fl, fld)[L] = acc * (fld == 0 ? area : ah);
    } else {
      const int rr = r - 2 * NF * N2, fl = rr / N2, L = rr - fl * N2, qa = L % N, qb = L / N;
      const int f = FB + fl, d = f >> 1, S = f & 1;
      const T* si = A1(cw, fl, 2) + qa;
      const T* so = A1(cw, fl, 3) + qa;
      const T* m = Bs + qb * N;
      T ti = T(0), to = T(0);
#pragma unroll
      for (int j = 0; j < N; ++j) {
        ti = fma(m[j], si[j * N], ti);
        to = fma(m[j], so[j * N], to);
      }
      T phi = T(0);
      if (act[cw] && ci[cw].kind[f] != 2) {
        const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
        const T xa = t.gq[qa], xb = t.gq[qb];
        T bn = T(0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const int o[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
          if (o[d] != S) continue;
          const T wa = o[ta] ? xa : T(1) - xa;
          const T wb = o[tb] ? xb : T(1) - xb;
          bn = fma(ci[cw].bc[d][c], wa * wb, bn);
        }
        bn = S ? bn : -bn;
        phi = AT[5 * N2 + qa + N * qb] * Prec<T>::area(mp, d) * bn * (bn >= T(0) ? ti : to);
      }
      A0(cw, fl, 2)[L] = phi;
    }
  }
  __syncwarp();
  // 4. B^T along the second axis: A1[.][3][qa + N b] = sum_qb B[qb][b] phi[qa + N qb]
  for (int it = lane; it < CPW * NF * N2; it += 32) {
    const int cw = it / (NF * N2), r = it - cw * NF * N2, fl = r / N2, L = r - fl * N2, qa = L % N, b = L / N;
    const T* src = A0(cw, fl, 2) + qa;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) acc = fma(Bs[j * N + b], src[j * N], acc);
    A1(cw, fl, 3)[L] = acc;
  }
  __syncwarp();
  // 5. B^T along the first axis: A0[.][3][a + N b] = sum_qa B[qa][a] A1[.][3][qa + N b]
  for (int it = lane; it < CPW * NF * N2; it += 32) {
    const int cw = it / (NF * N2), r = it - cw * NF * N2, fl = r / N2, L = r - fl * N2, a = L % N, b = L / N;
    const T* src = A1(cw, fl, 3) + N * b;
    T acc = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) acc = fma(Bs[j * N + a], src[j], acc);
    A0(cw, fl, 3)[L] = acc;
  }
  __syncwarp();
  // 6. scatter per element
  for (int e = lane; e < VEC; e += 32) {
    const int cw = e / N3;
    if (!act[cw]) continue;
    const int r = e - cw * N3;
    const int i0 = r % N, i1 = (r / N) % N, i2 = r / N2;
    T y = Y[e];
#pragma unroll
    for (int d = FB / 2; d < (FB + NF) / 2; ++d) {
      const int j = d == 0 ? i0 : (d == 1 ? i1 : i2);
      const int L = d == 0 ? i1 + N * i2 : (d == 1 ? i0 + N * i2 : i0 + N * i1);
#pragma unroll
      for (int S = 0; S < 2; ++S) {
        const int fl = 2 * d + S - FB;
        y = fma(DL[S * N + j], A0(cw, fl, 1)[L], y);
        if (j == (S ? N - 1 : 0)) y += A0(cw, fl, 0)[L] + A0(cw, fl, 3)[L];
      }
    }
    Y[e] = y;
  }
  __syncwarp();
}

// Shared values per warp of the element-form advection operator: the tables
// AT, then one region that holds the Gauss-point accumulator E (one vector)
// and the point factors BT (9 n^2 per cell slot) during the volume term and
// the face scratch during the faces.
constexpr int kAdvVol = VEC + 9 * CPW * N2;
constexpr int kAdvRegion = kAdvVol > CPW * kAdvFace ? kAdvVol : CPW * kAdvFace;
constexpr int kAdvExtra = kAdvTab + kAdvRegion;

// Y = A X (FULL, neighbour values from gu) or D_T X with advection in element
// form; Xt: the kAdvExtra region, its tables filled by adv_tables(Xt).
template <bool FULL, typename T, typename G>
__device__ __forceinline__ void adv_apply_e(const T* X, T* Y, T* S0, T* S1, T* Xt, const G* gu,
                                            const MeshParams& mp, int lane, const unsigned char* act,
                                            const CellInfo<T>* ci) {
  const T* AT = Xt;
  T* E = Xt + kAdvTab;
  volume_adv_e(X, Y, S0, S1, E, AT, E + VEC, lane, ci, act);
  if constexpr (kAdvNF == 6) {
    faces_adv_e<FULL, 0>(X, Y, E, AT, gu, mp, lane, act, ci);
  } else {
    faces_adv_e<FULL, 0>(X, Y, E, AT, gu, mp, lane, act, ci);
    faces_adv_e<FULL, 2>(X, Y, E, AT, gu, mp, lane, act, ci);
    faces_adv_e<FULL, 4>(X, Y, E, AT, gu, mp, lane, act, ci);
  }
}

// F0 must be followed by 4 * LINES values of scratch (F0, F1 and the
// reduction area are contiguous in every kernel's shared-memory carve).
template <bool FULL, bool ADV, typename T, typename G>
__device__ __forceinline__ void all_faces(const T* X, T* Y, T* F0, T* F1, const G* gu, const MeshParams& mp,
                                          long long cell0, int lane, const unsigned char* act,
                                          const CellInfo<T>* ci) {
  faces_diffusion_dir<0, FULL>(X, Y, F0, gu, mp, lane, act, ci);
  faces_diffusion_dir<1, FULL>(X, Y, F0, gu, mp, lane, act, ci);
  faces_diffusion_dir<2, FULL>(X, Y, F0, gu, mp, lane, act, ci);
  if (ADV) {
    face_upwind<0, 0, FULL>(X, Y, F0, F1, gu, mp, cell0, lane, act, ci);
    face_upwind<0, 1, FULL>(X, Y, F0, F1, gu, mp, cell0, lane, act, ci);
    face_upwind<1, 0, FULL>(X, Y, F0, F1, gu, mp, cell0, lane, act, ci);
    face_upwind<1, 1, FULL>(X, Y, F0, F1, gu, mp, cell0, lane, act, ci);
    face_upwind<2, 0, FULL>(X, Y, F0, F1, gu, mp, cell0, lane, act, ci);
    face_upwind<2, 1, FULL>(X, Y, F0, F1, gu, mp, cell0, lane, act, ci);
  }
}

// Stage the per-cell coefficients of the warp's cells; act[cw] = cell exists.
// Global cell of each slot of a warp: the CPW consecutive cells from cell0, or
// (color >= 0) the cells of one parity class (cx, cy, cz) = (kx, ky, kz) mod 2,
// color = kx + 2 ky + 4 kz, enumerated x fastest.  -1 = no cell.
__device__ __forceinline__ long long colored_cell(const MeshParams& mp, int color, long long j) {
  const int kx = color & 1, ky = (color >> 1) & 1, kz = color >> 2;
  const long long mx = (mp.nx - kx + 1) / 2, my = (mp.ny - ky + 1) / 2;
  const long long jx = j % mx, t = j / mx, jy = t % my, jz = t / my;
  return (2 * jx + kx) + (long long)mp.nx * ((2 * jy + ky) + (long long)mp.ny * (2 * jz + kz));
}

__device__ __forceinline__ long long color_count(const MeshParams& mp, int color) {
  if (color < 0) return mp.ncell;
  const int kx = color & 1, ky = (color >> 1) & 1, kz = color >> 2;
  return (long long)((mp.nx - kx + 1) / 2) * ((mp.ny - ky + 1) / 2) * ((mp.nz - kz + 1) / 2);
}

__device__ __forceinline__ void slot_cells(const MeshParams& mp, int color, long long s0, int lane, long long* cid) {
  if (lane < CPW) {
    const long long j = s0 + lane;
    const long long total = color_count(mp, color);
    cid[lane] = j < total ? (color < 0 ? j : colored_cell(mp, color, j)) : -1;
  }
  __syncwarp();
}

template <typename T, int C = CPW>
__device__ __forceinline__ void stage_cells(const MeshParams& mp, long long cell0, int lane, CellInfo<T>* ci,
                                            unsigned char* act, const long long* cid = nullptr) {
  if (lane < C) {
    const long long c = cid ? cid[lane] : cell0 + lane;
    const bool ok = c >= 0 && c < mp.ncell;
    act[lane] = ok ? 1 : 0;
    if (ok) {
      const long long r = c * kRecLen;
      for (int d = 0; d < 3; ++d) {
        ci[lane].kd[d] = Prec<T>::rec(mp, r + kRecKd + d);
        ci[lane].jh[d] = Prec<T>::jh(mp, d);
      }
      ci[lane].cJ = Prec<T>::rec(mp, r + kRecCJ);
      for (int f = 0; f < 6; ++f) {
        long long nb = -1;
        ci[lane].kind[f] = face_kind(mp, c, f >> 1, f & 1, nb);
        ci[lane].nb[f] = nb;
        ci[lane].kap[f] = Prec<T>::rec(mp, r + kRecKap + f);
        ci[lane].gam[f] = Prec<T>::rec(mp, r + kRecGam + f);
      }
      if (mp.bvert) {
        int cx, cy, cz;
        cell_xyz(mp, c, cx, cy, cz);
        const long long vx = mp.nx + 1, vxy = (long long)(mp.nx + 1) * (mp.ny + 1);
        for (int k = 0; k < 8; ++k) {
          const long long v = (cx + (k & 1)) + vx * (cy + ((k >> 1) & 1)) + vxy * (cz + (k >> 2));
          for (int d = 0; d < 3; ++d) ci[lane].bc[d][k] = Prec<T>::bv(mp, 3 * v + d);
        }
      }
    }
  }
  __syncwarp();
}

// Shared-memory carve-up of one warp.
template <typename T>
struct WarpMem {
  // nvec vectors of VEC values, face / reduction scratch, `extra` more values
  static __host__ __device__ constexpr size_t bytes(int nvec, int extra = 0) {
    return align16((size_t)(nvec * VEC + 5 * LINES + extra) * sizeof(T)) + align16(CPW * sizeof(CellInfo<T>)) +
           16 + align16(CPW * sizeof(long long));
  }
};

template <typename T>
__device__ __forceinline__ void carve(unsigned char* raw, int nvec, T** vec, T** F0, T** F1, T** red,
                                      CellInfo<T>** ci, unsigned char** act, long long** cid = nullptr,
                                      int extra = 0, T** xtra = nullptr) {
  T* p = reinterpret_cast<T*>(raw);
  for (int k = 0; k < nvec; ++k) vec[k] = p + k * VEC;
  *F0 = p + nvec * VEC;
  *F1 = *F0 + LINES;
  *red = *F1 + LINES;     // 3 * LINES spare (reductions)
  if (xtra) *xtra = *red + 3 * LINES;
  unsigned char* tail = raw + align16((size_t)(nvec * VEC + 5 * LINES + extra) * sizeof(T));
  *ci = reinterpret_cast<CellInfo<T>*>(tail);
  *act = tail + align16(CPW * sizeof(CellInfo<T>));
  if (cid) *cid = reinterpret_cast<long long*>(*act + 16);
}

template <typename T, bool FULL, bool ADV, bool FAC, typename G>
__device__ __forceinline__ void apply_body(const MeshParams& mp, const G* __restrict__ u, G* __restrict__ v,
                                           unsigned bid) {
  const bool react = mp.c != nullptr;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long cell0 = ((long long)bid * (blockDim.x >> 5) + warp) * CPW;
  if (cell0 >= mp.ncell) return;
  T* vec[4];
  T *F0, *F1, *red;
  CellInfo<T>* ci;
  unsigned char* act;
  // FAC: element work items: for b = 0 the factored form (per-cell matrices,
  // mass matrix, neighbour face values in the extra region), with advection
  // the Gauss-point form (its accumulator, tables and face scratch there);
  // else the line form
  constexpr int XT = FAC ? (ADV ? kAdvExtra : kFactorExtra) : 0;
  T* Xt = nullptr;
  carve(smem + warp * WarpMem<T>::bytes(4, XT), 4, vec, &F0, &F1, &red, &ci, &act, nullptr, XT, &Xt);
  T *X = vec[0], *Y = vec[1], *S0 = vec[2], *S1 = vec[3];
  stage_cells(mp, cell0, lane, ci, act);
  const long long nval = (mp.ncell - cell0) * N3 < VEC ? (mp.ncell - cell0) * N3 : VEC;
  const G* ug = u + cell0 * N3;
  for (int e = lane; e < VEC; e += 32) X[e] = e < nval ? T(ug[e]) : T(0);
  if constexpr (FAC && !ADV) {
    T* Ah = Xt;
    T* M1s = Ah + 3 * CPW * N2;
    T* MVs = M1s + N2;
    T* FS = MVs + 4 * N;
    factor_setup(Ah, M1s, MVs, FS, mp, ci, act, lane);
    factored_apply<FULL>(X, Y, S0, S1, Ah, M1s, MVs, FS, u, lane, act, ci);
  } else if constexpr (FAC && ADV) {
    adv_tables(Xt, lane);
    __syncwarp();
    adv_apply_e<FULL>(X, Y, S0, S1, Xt, u, mp, lane, act, ci);
  } else {
    __syncwarp();
    volume<ADV>(X, Y, S0, S1, lane, ci, act, react);
    all_faces<FULL, ADV>(X, Y, F0, F1, u, mp, cell0, lane, act, ci);
  }
  G* vg = v + cell0 * N3;
  for (int e = lane; e < nval; e += 32) vg[e] = static_cast<G>(Y[e]);
}

template <typename T, bool FULL, bool ADV, bool FAC, typename G = typename Store<T>::type>
__global__ void __launch_bounds__(256) k_apply(const __grid_constant__ MeshParams mp, const G* __restrict__ u,
                                               G* __restrict__ v) {
  apply_body<T, FULL, ADV, FAC, G>(mp, u, v, blockIdx.x);
}

// Member of a batch that owns block bid (block0 ascending, block0[0] = 0).
__device__ __forceinline__ int batch_member(const BatchTable& bt, unsigned bid) {
  int r = 0;
  while (r + 1 < bt.k && bid >= bt.block0[r + 1]) ++r;
  return r;
}

template <typename T, bool FULL, bool ADV, bool FAC, typename G = typename Store<T>::type>
__global__ void __launch_bounds__(256) k_apply_batch(const __grid_constant__ BatchTable bt) {
  const int r = batch_member(bt, blockIdx.x);
  apply_body<T, FULL, ADV, FAC, G>(bt.mp[r], (const G*)bt.in[r], (G*)bt.out[r], blockIdx.x - bt.block0[r]);
}

// Sum over the lanes that own lines of the same cell; every lane of that cell
// gets the same value (fixed summation order).
template <typename T>
__device__ __forceinline__ T cell_sum(T part, int lane, T* red) {
  if (CPW == 1) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += shfl_x(part, o);
    return part;
  } else {
    red[lane] = part;
    __syncwarp();
    T s = T(0);
    if (lane < LINES) {
      const int c0 = (lane / N2) * N2;
#pragma unroll
      for (int k = 0; k < N2; ++k) s += red[c0 + k];
    }
    __syncwarp();
    return s;
  }
}

// Two cell sums at once (the same summation order as cell_sum for each).
// One cell per warp: after the first level the lower half-warp carries the
// partial sums of a and the upper half those of b, so the remaining levels
// reduce one value per lane; each sum is added in the same tree as in
// cell_sum (the same bits, half the adds).
template <typename T>
__device__ __forceinline__ void cell_sum2(T& a, T& b, int lane, T* red) {
  if (CPW == 1) {
    const bool hi = (lane & 16) != 0;
    T v = (hi ? b : a) + shfl_x(hi ? a : b, 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += shfl_x(v, o);
    a = shfl_i(v, 0);
    b = shfl_i(v, 16);
  } else {
    red[lane] = a;
    red[LINES + lane] = b;
    __syncwarp();
    T sa = T(0), sb = T(0);
    if (lane < LINES) {
      const int c0 = (lane / N2) * N2;
#pragma unroll
      for (int k = 0; k < N2; ++k) {
        sa += red[c0 + k];
        sb += red[LINES + c0 + k];
      }
    }
    __syncwarp();
    a = sa;
    b = sb;
  }
}

// a / b of a cell (the same on its lanes), computed on the cell's first lane
// and broadcast, so that the division's instructions run once per cell
// instead of on every lane; `on` as on the cell's lanes.
template <typename T>
__device__ __forceinline__ T cell_div(T a, T b, int lane, bool on) {
  const int src = CPW == 1 ? 0 : (lane < LINES ? (lane / N2) * N2 : lane);
  T q = T(0);
  if (on && lane == src) q = a / b;
  return shfl_i(q, src);
}

// Extra shared values per warp of the inner-PCG smoother: the factored form's
// region (FP64, double-float, b = 0), the per-cell 1D matrices of D_T (FP32,
// b = 0), nothing with advection.
template <bool ADV, bool FAC>
__host__ __device__ constexpr int smooth_extra() {
  return FAC ? (ADV ? kAdvExtra : kFactorExtra) : (ADV ? 0 : 3 * CPW * N2);
}

// Block-Jacobi sweep with inner PCG (Algorithm 2; inner solve Sec. 2.2.1).
// Per cell: the defect d = f - A u_old (skipped from u = 0), PCG on D_T delta = d
// with the preconditioner 1/diag(D_T) from delta_0 = 0, u_new = u_old + omega delta.
// The block is applied in the factored form (FP64, double-float, b = 0), by
// the eight Kronecker contractions (FP32, b = 0), or at the Gauss points
// (advection).  With several cells per warp each lane owns one z-line of its
// cell for the pointwise vector operations; with one cell per warp every lane
// takes elements lane, lane + 32, ... (all 32 lanes busy).
template <typename T, bool ADV, bool FAC, typename G>
__device__ __forceinline__ void smooth_pcg_body(const MeshParams& mp, const G* __restrict__ f, const G* uold, G* unew,
                                                const G* __restrict__ diag, T omega, T eps, int maxit,
                                                int* __restrict__ its, int color, unsigned bid) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s0 = ((long long)bid * (blockDim.x >> 5) + warp) * CPW;
  if (s0 >= color_count(mp, color)) return;
  T *F0, *F1, *red;
  CellInfo<T>* ci;
  unsigned char* act;
  long long* cid;
  constexpr int XT = smooth_extra<ADV, FAC>();
  T* vec[6];
  T* Xt = nullptr;
  carve(smem + warp * WarpMem<T>::bytes(6, XT), 6, vec, &F0, &F1, &red, &ci, &act, &cid, XT, &Xt);
  T *P = vec[0], *Q = vec[1], *S0 = vec[2], *S1 = vec[3], *R = vec[4], *DL = vec[5];
  const bool react = mp.c != nullptr;
  const bool zero = uold == nullptr;   // first sweep from u = 0: no defect apply
  slot_cells(mp, color, s0, lane, cid);
  stage_cells(mp, 0, lane, ci, act, cid);
  const long long cell0 = cid[0];
  T* Ah = Xt;                     // FAC: M^-1 A_d; FP32: A_d (3 n^2 per cell)
  T* M1s = Ah + 3 * CPW * N2;     // FAC only: mass matrix, M^-1 e_e, M^-1 dl_s, face values
  T* MVs = M1s + N2;
  T* FS = MVs + 4 * N;
  if constexpr (FAC && !ADV) {
    factor_setup(Ah, M1s, MVs, FS, mp, ci, act, lane);
  } else if constexpr (FAC && ADV) {
    adv_tables(Xt, lane);
    __syncwarp();
  } else if constexpr (!ADV) {
    block_matrices(mp, Ah, ci, act, lane);
  }
  const int mycw = CPW == 1 ? 0 : (lane < LINES ? lane / N2 : -1);
  const bool mine = mycw >= 0 && act[mycw];
  const bool lead = CPW == 1 ? lane == 0 : (lane < LINES && lane % N2 == 0);
  auto my_elems = [&](auto&& fn) {
    if constexpr (CPW == 1) {
      for (int e = lane; e < N3; e += 32) fn(e);
    } else if (lane < LINES) {
      int cw, base, st, a, b;
      line_geom<2>(lane, cw, base, st, a, b);
#pragma unroll
      for (int i = 0; i < N; ++i) fn(base + i * N2);
    }
  };
  const long long gb = mycw >= 0 ? cid[mycw] * N3 - mycw * N3 : 0;   // global index = gb + e
  // defect d = f - A u_old
  if (!zero) {
    for (int e = lane; e < VEC; e += 32) {
      const int cw = e / N3;
      P[e] = act[cw] ? T(uold[cid[cw] * N3 + (e - cw * N3)]) : T(0);
    }
    __syncwarp();
    if constexpr (FAC && !ADV) {
      factored_apply<true>(P, Q, S0, S1, Ah, M1s, MVs, FS, uold, lane, act, ci);
    } else if constexpr (FAC && ADV) {
      adv_apply_e<true>(P, Q, S0, S1, Xt, uold, mp, lane, act, ci);
    } else {
      volume<ADV>(P, Q, S0, S1, lane, ci, act, react);
      all_faces<true, ADV>(P, Q, F0, F1, uold, mp, cell0, lane, act, ci);
    }
  }
  T prr = T(0), prz = T(0);
  if (mine)
    my_elems([&](int e) {
      const T r = T(f[gb + e]) - (zero ? T(0) : Q[e]);
      const T z = r * T(diag[gb + e]);
      R[e] = r;
      P[e] = z;
      DL[e] = T(0);
      prr = fma(r, r, prr);
      prz = fma(r, z, prz);
    });
  cell_sum2(prr, prz, lane, red);
  const T rr0 = prr;
  T rz = prz;
  // The inner solve works on d / ||d|| (and scales the correction back):
  // FP32 products of a tiny defect would otherwise lose precision in the
  // subnormal range.  The stopping test ||r|| <= eps ||d|| becomes
  // (r, r) <= eps^2, safe in every precision since (r_0, r_0) = 1.
  const T dnorm = sqrt(rr0);
  const T isc = rr0 > T(0) ? T(1) / dnorm : T(0);
  if (mine)
    my_elems([&](int e) {
      R[e] = R[e] * isc;
      P[e] = P[e] * isc;
    });
  rz = rz * isc * isc;
  const T thr2 = eps * eps;
  bool live = mine && rr0 > T(0);
  int it = 0;
  while (__any_sync(FULLMASK, live && it < maxit)) {
    if (mycw >= 0) act[mycw] = (live && it < maxit) ? 1 : 0;
    __syncwarp();
    const bool run = live && it < maxit;
    // Q = D_T P
    if constexpr (ADV && FAC) {
      adv_apply_e<false>(P, Q, S0, S1, Xt, (const G*)nullptr, mp, lane, act, ci);
    } else if constexpr (ADV) {
      volume<ADV>(P, Q, S0, S1, lane, ci, act, react);
      all_faces<false, ADV>(P, Q, F0, F1, (const G*)nullptr, mp, cell0, lane, act, ci);
    } else if constexpr (FAC) {
      factored_apply<false>(P, Q, S0, S1, Ah, M1s, MVs, FS, (const G*)nullptr, lane, act, ci);
    } else {
      block_kron(P, Q, S0, S1, Ah, lane, act);
    }
    T ppq = T(0);
    if (run) my_elems([&](int e) { ppq = fma(P[e], Q[e], ppq); });
    const T pq = cell_sum(ppq, lane, red);
    bool upd = run && pq > T(0);
    if (run && !upd) live = false;   // breakdown: stop this cell
    // delta += alpha p, r -= alpha q, and with the new r both (r, r) and
    // (r, z), z = r / diag (kept in S0 for the direction update)
    T prr2 = T(0), prz2 = T(0);
    const T alpha = cell_div(rz, pq, lane, upd);
    if (upd) {
      my_elems([&](int e) {
        DL[e] = fma(alpha, P[e], DL[e]);
        const T r = fma(-alpha, Q[e], R[e]);
        R[e] = r;
        prr2 = fma(r, r, prr2);
        const T z = r * T(diag[gb + e]);
        S0[e] = z;
        prz2 = fma(r, z, prz2);
      });
      ++it;
    }
    cell_sum2(prr2, prz2, lane, red);
    if (upd && prr2 <= thr2) {
      live = false;
      upd = false;
    }
    if (upd && it >= maxit) upd = false;
    const T beta = cell_div(prz2, rz, lane, upd);
    if (upd) {
      rz = prz2;
      my_elems([&](int e) { P[e] = fma(beta, P[e], S0[e]); });
    }
    __syncwarp();
  }
  // u_new = u_old + omega delta (in place is allowed: a launch touches only its
  // own cells' values, and reads neighbours only of other colours)
  if (mycw >= 0 && cid[mycw] >= 0)
    my_elems([&](int e) {
      const long long g = gb + e;
      const T dl = DL[e] * dnorm;
      unew[g] = static_cast<G>(zero ? omega * dl : fma(omega, dl, T(uold[g])));
    });
  if (its && lead && mycw >= 0 && cid[mycw] >= 0) its[cid[mycw]] = it;
}

template <typename T, bool ADV, bool FAC, typename G = typename Store<T>::type>
__global__ void __launch_bounds__(256) k_smooth_pcg(const __grid_constant__ MeshParams mp, const G* __restrict__ f,
                                                    const G* uold, G* unew, const G* __restrict__ diag, T omega,
                                                    T eps, int maxit, int* __restrict__ its, int color) {
  smooth_pcg_body<T, ADV, FAC, G>(mp, f, uold, unew, diag, omega, eps, maxit, its, color, blockIdx.x);
}

template <typename T, bool ADV, bool FAC, typename G = typename Store<T>::type>
__global__ void __launch_bounds__(256) k_smooth_pcg_batch(const __grid_constant__ BatchTable bt) {
  const int r = batch_member(bt, blockIdx.x);
  smooth_pcg_body<T, ADV, FAC, G>(bt.mp[r], (const G*)bt.in[r], (const G*)bt.uold[r], (G*)bt.out[r],
                                  (const G*)bt.diag[r], T(bt.omega), T(bt.eps), bt.maxit, bt.its[r], -1,
                                  blockIdx.x - bt.block0[r]);
}

// D_T of each cell column by column: column j is the block operator (volume
// terms and own-side face terms) applied to the unit vector e_j.  FP64;
// output column-major with column stride ld >= n^3 (block stride n^3 ld).
// Set-up of the stored inverses.
template <bool ADV>
__global__ void __launch_bounds__(256) k_block_matrix(MeshParams mp, double* __restrict__ out, int ld) {
  using T = double;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s0 = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * CPW;
  if (s0 >= mp.ncell) return;
  T* vec[4];
  T *F0, *F1, *red;
  CellInfo<T>* ci;
  unsigned char* act;
  long long* cid;
  carve(smem + warp * WarpMem<T>::bytes(4), 4, vec, &F0, &F1, &red, &ci, &act, &cid);
  T *P = vec[0], *Q = vec[1], *S0 = vec[2], *S1 = vec[3];
  const bool react = mp.c != nullptr;
  slot_cells(mp, -1, s0, lane, cid);
  stage_cells(mp, 0, lane, ci, act, cid);
  const long long cell0 = cid[0];
  for (int j = 0; j < N3; ++j) {
    for (int e = lane; e < VEC; e += 32) P[e] = (e % N3 == j) ? T(1) : T(0);
    __syncwarp();
    volume<ADV>(P, Q, S0, S1, lane, ci, act, react);
    all_faces<false, ADV>(P, Q, F0, F1, (const double*)nullptr, mp, cell0, lane, act, ci);
    __syncwarp();
    for (int e = lane; e < VEC; e += 32) {
      const int cw = e / N3;
      if (act[cw]) out[cid[cw] * (long long)(N3 * ld) + (long long)j * ld + (e - cw * N3)] = Q[e];
    }
    __syncwarp();
  }
}

// Block-Jacobi (color < 0) or one colour of block-SOR with exact block solves
// by the stored inverses (the partially matrix-free smoother): per cell
// d = f - A u_old (skipped from u = 0), delta = D_T^-1 d as a dense
// matrix-vector product whose columns (stride ld, a multiple of 8 values, so
// that a warp's reads of one column start on 32-byte sectors) are read
// coalesced from HBM, u_new = u_old + omega delta.  FP64 smoothers keep the
// inverse as double-float pairs (hi, lo) and form the product in double-float
// arithmetic: a FP64 product would make this kernel FP64-pipe bound
// (2 flop per 8-byte entry is above GB300's FP64 ridge of 0.18 flop/B);
// pairs keep ~48 significant bits at FP32 issue rates.  FP32 smoothers keep
// FP32 entries and FP32 arithmetic.
template <typename T> struct InvEntry { using type = T; };
template <> struct InvEntry<double> { using type = float2; };
template <> struct InvEntry<df> { using type = float2; };

template <typename T, bool ADV, bool FAC, typename G = typename Store<T>::type,
          typename M = typename InvEntry<T>::type>
__global__ void __launch_bounds__(256) k_smooth_inv(MeshParams mp, const G* __restrict__ f, const G* uold, G* unew,
                                                    const M* __restrict__ binv, int ld, T omega,
                                                    int* __restrict__ its, int color) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s0 = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * CPW;
  if (s0 >= color_count(mp, color)) return;
  T* vec[4];
  T *F0, *F1, *red;
  CellInfo<T>* ci;
  unsigned char* act;
  long long* cid;
  constexpr int XT = FAC ? (ADV ? kAdvExtra : kFactorExtra) : 0;
  T* Xt = nullptr;
  carve(smem + warp * WarpMem<T>::bytes(4, XT), 4, vec, &F0, &F1, &red, &ci, &act, &cid, XT, &Xt);
  T *P = vec[0], *Q = vec[1], *S0 = vec[2], *S1 = vec[3];
  const bool react = mp.c != nullptr;
  const bool zero = uold == nullptr;
  slot_cells(mp, color, s0, lane, cid);
  stage_cells(mp, 0, lane, ci, act, cid);
  const long long cell0 = cid[0];
  if (!zero) {
    for (int e = lane; e < VEC; e += 32) {
      const int cw = e / N3;
      P[e] = act[cw] ? T(uold[cid[cw] * N3 + (e - cw * N3)]) : T(0);
    }
    if constexpr (FAC && !ADV) {   // the defect's operator in the factored form
      T* Ah = Xt;
      T* M1s = Ah + 3 * CPW * N2;
      T* MVs = M1s + N2;
      factor_setup(Ah, M1s, MVs, MVs + 4 * N, mp, ci, act, lane);
      factored_apply<true>(P, Q, S0, S1, Ah, M1s, MVs, MVs + 4 * N, uold, lane, act, ci);
    } else if constexpr (FAC && ADV) {
      adv_tables(Xt, lane);
      __syncwarp();
      adv_apply_e<true>(P, Q, S0, S1, Xt, uold, mp, lane, act, ci);
    } else {
      __syncwarp();
      volume<ADV>(P, Q, S0, S1, lane, ci, act, react);
      all_faces<true, ADV>(P, Q, F0, F1, uold, mp, cell0, lane, act, ci);
      __syncwarp();
    }
  }
  // the defect goes to P (no longer needed); FP64: also as double-float pairs in S0
  df* D2 = reinterpret_cast<df*>(S0);
  for (int e = lane; e < VEC; e += 32) {
    const int cw = e / N3;
    const T dv = act[cw] ? T(f[cid[cw] * N3 + (e - cw * N3)]) - (zero ? T(0) : Q[e]) : T(0);
    P[e] = dv;
    if constexpr (std::is_same<T, double>::value) D2[e] = df(dv);
    if constexpr (std::is_same<T, df>::value) D2[e] = dv;
  }
  __syncwarp();
  for (int e = lane; e < VEC; e += 32) {
    const int cw = e / N3;
    if (!act[cw]) continue;
    const int i = e - cw * N3;
    const M* col = binv + cid[cw] * (long long)N3 * ld + i;
    T acc;
    if constexpr (!std::is_same<T, float>::value) {   // FP64 and double-float smoothers
      const df* d = D2 + cw * N3;
      df_acc a;
#pragma unroll 8
      for (int j = 0; j < N3; ++j) {
        const float2 m = __ldg(col + (long long)j * ld);
        a.add_prod(df(m.x, m.y), d[j]);
      }
      if constexpr (std::is_same<T, double>::value)
        acc = double(a.value());
      else
        acc = a.value();
    } else {
      const T* d = P + cw * N3;
      acc = T(0);
#pragma unroll 8
      for (int j = 0; j < N3; ++j) acc = fma(__ldg(col + (long long)j * ld), d[j], acc);
    }
    const long long g = cid[cw] * N3 + i;
    unew[g] = static_cast<G>(zero ? omega * acc : fma(omega, acc, T(uold[g])));
  }
  if (its && lane < CPW && cid[lane] >= 0) its[cid[lane]] = 0;
}

// Tridiagonal part of D_T in the cell's lexicographic dof order (x fastest)
// and its Thomas factors, per cell [a | c' | 1/den] (3 n^3 values):
// a_i = D[i][i-1] (a_0 = 0), den_i = D[i][i] - a_i c'_{i-1},
// c'_i = D[i][i+1] / den_i (c'_{n^3-1} = 0).  Columns of D_T come from block
// applications to unit vectors, as for the stored inverses.  FP64 set-up;
// a zero or non-finite den sets *singular.  (The inner preconditioner the
// paper uses for strongly convection-dominated blocks, Sec. 3.2 and 4.3.)
template <bool ADV>
__global__ void __launch_bounds__(256) k_block_tridiag(MeshParams mp, double* __restrict__ out,
                                                       int* __restrict__ singular) {
  using T = double;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s0 = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * CPW;
  if (s0 >= mp.ncell) return;
  T* vec[7];
  T *F0, *F1, *red;
  CellInfo<T>* ci;
  unsigned char* act;
  long long* cid;
  carve(smem + warp * WarpMem<T>::bytes(7), 7, vec, &F0, &F1, &red, &ci, &act, &cid);
  T *P = vec[0], *Q = vec[1], *S0 = vec[2], *S1 = vec[3], *TA = vec[4], *TB = vec[5], *TC = vec[6];
  const bool react = mp.c != nullptr;
  slot_cells(mp, -1, s0, lane, cid);
  stage_cells(mp, 0, lane, ci, act, cid);
  const long long cell0 = cid[0];
  for (int j = 0; j < N3; ++j) {
    for (int e = lane; e < VEC; e += 32) P[e] = (e % N3 == j) ? T(1) : T(0);
    __syncwarp();
    volume<ADV>(P, Q, S0, S1, lane, ci, act, react);
    all_faces<false, ADV>(P, Q, F0, F1, (const double*)nullptr, mp, cell0, lane, act, ci);
    __syncwarp();
    for (int e = lane; e < VEC; e += 32) {
      const int i = e % N3;
      if (i == j) TB[e] = Q[e];
      else if (i == j + 1) TA[e] = Q[e];
      else if (i + 1 == j) TC[e] = Q[e];
    }
    __syncwarp();
  }
  if (lane < CPW && act[lane]) {
    double* o = out + cid[lane] * (3LL * N3);
    const int b = lane * N3;
    T pc = T(0);
    bool bad = false;
    for (int i = 0; i < N3; ++i) {
      const T a = i > 0 ? TA[b + i] : T(0);
      const T c = i + 1 < N3 ? TC[b + i] : T(0);
      const T den = TB[b + i] - a * pc;
      if (den == T(0) || !isfinite(den)) bad = true;
      const T id = T(1) / den;
      pc = c * id;
      o[i] = a;
      o[N3 + i] = pc;
      o[2 * N3 + i] = id;
    }
    if (bad) *singular = 1;
  }
}

// dst = M^-1 src for the cells with act set, M the tridiagonal part of D_T
// given by its Thomas factors: forward d'_i = (r_i - a_i d'_{i-1}) / den_i,
// back x_i = d'_i - c'_i x_{i+1}.  One lane per cell (the recurrence is
// sequential); called by the whole warp.
template <typename T>
__device__ __forceinline__ void thomas_apply(const T* __restrict__ tri, const long long* cid,
                                             const unsigned char* act, const T* src, T* dst, int lane) {
  if (lane < CPW && act[lane]) {
    const T* fa = tri + cid[lane] * (3LL * N3);
    const T* fc = fa + N3;
    const T* fi = fc + N3;
    const T* r = src + lane * N3;
    T* x = dst + lane * N3;
    T prev = T(0);
    for (int i = 0; i < N3; ++i) {
      prev = (r[i] - fa[i] * prev) * fi[i];
      x[i] = prev;
    }
    for (int i = N3 - 2; i >= 0; --i) x[i] = fma(-fc[i], x[i + 1], x[i]);
  }
  __syncwarp();
}

// ----------------------------------------------------------------- variable coefficients
// K(x) = sum_k (p0_k + p2_k x_k^2) n_k n_k^T and c(x) = gamma |x|^2 at a
// physical point (the paper's inhomogeneous test, Sec. 4.2); vp holds the
// rows n_k (9 values), p0 (3), p2 (3), gamma.  K as (xx, yy, zz, xy, xz, yz).
__device__ __forceinline__ void var_coef(const double* __restrict__ vp, const double x[3], double K[6], double& c) {
#pragma unroll
  for (int i = 0; i < 6; ++i) K[i] = 0.0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double pk = fma(vp[12 + k] * x[k], x[k], vp[9 + k]);
    const double a = vp[3 * k], b = vp[3 * k + 1], e = vp[3 * k + 2];
    K[0] = fma(pk * a, a, K[0]);
    K[1] = fma(pk * b, b, K[1]);
    K[2] = fma(pk * e, e, K[2]);
    K[3] = fma(pk * a, b, K[3]);
    K[4] = fma(pk * a, e, K[4]);
    K[5] = fma(pk * b, e, K[5]);
  }
  c = vp[15] * (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
}

__device__ __forceinline__ double kent(const double K[6], int i, int j) {
  if (i == j) return K[i];
  const int s = i + j;   // (0,1) -> 3, (0,2) -> 4, (1,2) -> 5
  return K[s == 1 ? 3 : (s == 2 ? 4 : 5)];
}

// Index of dof (normal index id, tangential ia, ib) for faces normal to axis D.
template <int D>
__device__ __forceinline__ int fidx(int id, int ia, int ib) {
  if (D == 0) return id + N * ia + N2 * ib;
  if (D == 1) return ia + N * id + N2 * ib;
  return ia + N * ib + N2 * id;
}

// Own-row terms of the faces normal to axis D on side s (SIPG with K(x) at the
// face Gauss points; a continuous K gives both traces the same value, so the
// weights are 1/2 and <delta^-, delta^+> = delta = nu^T K nu):
//   -int {K grad u}.n v - int w (K grad v . n) [[u]] + int gamma [[u]] v,
// with n the outward normal of the cell, [[u]] = u_T - u_nb (u_nb = 0 and
// w = 1 on Dirichlet faces, nothing on Neumann faces).  Traces and normal
// derivatives come from the nodal values (GLL end points), tangential
// derivatives from the Gauss-point derivative table G.  FS: scratch of at
// least 18 CPW n^2 values.  Accumulates into Y.
template <int D>
__device__ void faces_var(const MeshParams& mp, const double* __restrict__ u, const double* X, double* Y,
                          double* FS, int s, int lane, const CellInfo<double>* ci, const unsigned char* act,
                          const long long* cid) {
  const Tab<double>& t = c_tab_d;
  constexpr int A = D == 0 ? 1 : 0, Bx = D == 2 ? 1 : 2;
  const int f = 2 * D + s;
  const int end = s ? N - 1 : 0, endn = s ? 0 : N - 1;
  const double ihd = mp.ih[D], iha = mp.ih[A], ihb = mp.ih[Bx];
  auto arr = [&](int k, int cw) { return FS + (k * CPW + cw) * N2; };
  // 1: traces and normal derivatives, own (0, 1) and neighbour (2, 3)
  for (int it = lane; it < CPW * N2; it += 32) {
    const int cw = it / N2, r = it - cw * N2, ia = r % N, ib = r / N;
    if (!act[cw] || ci[cw].kind[f] == 2) continue;
    const double* xc = X + cw * N3;
    double nd = 0.0;
#pragma unroll
    for (int k = 0; k < N; ++k) nd = fma(t.dl[s][k], xc[fidx<D>(k, ia, ib)], nd);
    arr(0, cw)[r] = xc[fidx<D>(end, ia, ib)];
    arr(1, cw)[r] = nd * ihd;
    double tn = 0.0, ndn = 0.0;
    if (ci[cw].kind[f] == 0) {
      const double* un = u + ci[cw].nb[f] * N3;
      tn = __ldg(un + fidx<D>(endn, ia, ib));
#pragma unroll
      for (int k = 0; k < N; ++k) ndn = fma(t.dl[1 - s][k], __ldg(un + fidx<D>(k, ia, ib)), ndn);
    }
    arr(2, cw)[r] = tn;
    arr(3, cw)[r] = ndn * ihd;
  }
  __syncwarp();
  // 2a: along a: B trace, G trace, B normal derivative (own 4..6, neighbour 7..9); index qa + N ib
  for (int it = lane; it < CPW * N2; it += 32) {
    const int cw = it / N2, r = it - cw * N2, qa = r % N, ib = r / N;
    if (!act[cw] || ci[cw].kind[f] == 2) continue;
    double v[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int ia = 0; ia < N; ++ia) {
      const double bq = t.B[qa][ia], gq = t.G[qa][ia];
      const int k = ia + N * ib;
      v[0] = fma(bq, arr(0, cw)[k], v[0]);
      v[1] = fma(gq, arr(0, cw)[k], v[1]);
      v[2] = fma(bq, arr(1, cw)[k], v[2]);
      v[3] = fma(bq, arr(2, cw)[k], v[3]);
      v[4] = fma(gq, arr(2, cw)[k], v[4]);
      v[5] = fma(bq, arr(3, cw)[k], v[5]);
    }
#pragma unroll
    for (int j = 0; j < 6; ++j) arr(4 + j, cw)[r] = v[j];
  }
  __syncwarp();
  // 2b: at the face Gauss points (qa, qb): the flux terms, weighted (10..13)
  for (int it = lane; it < CPW * N2; it += 32) {
    const int cw = it / N2, r = it - cw * N2, qa = r % N, qb = r / N;
    if (!act[cw] || ci[cw].kind[f] == 2) continue;
    double uT = 0, aT = 0, bT = 0, dT = 0, uN = 0, aN = 0, bN = 0, dN = 0;
#pragma unroll
    for (int ib = 0; ib < N; ++ib) {
      const double bq = t.B[qb][ib], gq = t.G[qb][ib];
      const int k = qa + N * ib;
      uT = fma(bq, arr(4, cw)[k], uT);
      aT = fma(bq, arr(5, cw)[k], aT);
      bT = fma(gq, arr(4, cw)[k], bT);
      dT = fma(bq, arr(6, cw)[k], dT);
      uN = fma(bq, arr(7, cw)[k], uN);
      aN = fma(bq, arr(8, cw)[k], aN);
      bN = fma(gq, arr(7, cw)[k], bN);
      dN = fma(bq, arr(9, cw)[k], dN);
    }
    int cx, cy, cz;
    cell_xyz(mp, cid[cw], cx, cy, cz);
    const int cc[3] = {cx, cy, cz};
    double x[3];
    x[D] = (cc[D] + s) * mp.h[D];
    x[A] = (cc[A] + t.gq[qa]) * mp.h[A];
    x[Bx] = (cc[Bx] + t.gq[qb]) * mp.h[Bx];
    double K[6], cdum;
    var_coef(mp.var, x, K, cdum);
    const double sg = s ? 1.0 : -1.0;
    const double knd = sg * kent(K, D, D), kna = sg * kent(K, A, D), knb = sg * kent(K, Bx, D);
    const double fT = knd * dT + kna * aT * iha + knb * bT * ihb;
    const double fN = knd * dN + kna * aN * iha + knb * bN * ihb;
    const double gam = mp.alpha * mp.p * (mp.p + 2) * kent(K, D, D) * ihd;
    const double wf = t.w[qa] * t.w[qb] * mp.area[D];
    double av, bv;
    if (ci[cw].kind[f] == 0) {
      av = -0.5 * (fT + fN) + gam * (uT - uN);
      bv = -0.5 * (uT - uN);
    } else {
      av = -fT + gam * uT;
      bv = -uT;
    }
    arr(10, cw)[r] = wf * av;
    arr(11, cw)[r] = wf * bv * kna;
    arr(12, cw)[r] = wf * bv * knb;
    arr(13, cw)[r] = wf * bv * knd;
  }
  __syncwarp();
  // 3a: transposed along b (14..17); index qa + N ib
  for (int it = lane; it < CPW * N2; it += 32) {
    const int cw = it / N2, r = it - cw * N2, qa = r % N, ib = r / N;
    if (!act[cw] || ci[cw].kind[f] == 2) continue;
    double v0 = 0, v1 = 0, v2 = 0, v3 = 0;
#pragma unroll
    for (int qb = 0; qb < N; ++qb) {
      const double bq = t.B[qb][ib], gq = t.G[qb][ib];
      const int k = qa + N * qb;
      v0 = fma(bq, arr(10, cw)[k], v0);
      v1 = fma(bq, arr(11, cw)[k], v1);
      v2 = fma(gq, arr(12, cw)[k], v2);
      v3 = fma(bq, arr(13, cw)[k], v3);
    }
    arr(14, cw)[r] = v0;
    arr(15, cw)[r] = v1;
    arr(16, cw)[r] = v2;
    arr(17, cw)[r] = v3;
  }
  __syncwarp();
  // 3b: transposed along a, into the face layer (values, tangential
  // derivatives) and along all layers (normal derivative)
  for (int it = lane; it < CPW * N2; it += 32) {
    const int cw = it / N2, r = it - cw * N2, ia = r % N, ib = r / N;
    if (!act[cw] || ci[cw].kind[f] == 2) continue;
    double lv = 0, nv = 0;
#pragma unroll
    for (int qa = 0; qa < N; ++qa) {
      const double bq = t.B[qa][ia], gq = t.G[qa][ia];
      const int k = qa + N * ib;
      lv = fma(bq, arr(14, cw)[k], lv);
      lv = fma(gq * iha, arr(15, cw)[k], lv);
      lv = fma(bq * ihb, arr(16, cw)[k], lv);
      nv = fma(bq, arr(17, cw)[k], nv);
    }
    nv *= ihd;
    double* yc = Y + cw * N3;
    yc[fidx<D>(end, ia, ib)] += lv;
#pragma unroll
    for (int k = 0; k < N; ++k) yc[fidx<D>(k, ia, ib)] = fma(t.dl[s][k], nv, yc[fidx<D>(k, ia, ib)]);
  }
  __syncwarp();
}

// v = A u for K(x), c(x) varying inside the cells (b = 0), FP64: volume
// terms at the Gauss points (u, grad u by B and the Gauss derivative Dg;
// pointwise flux |J| w K(x) grad u and |J| w c(x) u; transposed derivatives
// and B^T), then the six faces as in faces_var.
__global__ void __launch_bounds__(256) k_apply_var(MeshParams mp, const double* __restrict__ u, double* __restrict__ v) {
  using T = double;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long s0 = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * CPW;
  if (s0 >= mp.ncell) return;
  T* vec[11];
  T *F0, *F1, *red;
  CellInfo<T>* ci;
  unsigned char* act;
  long long* cid;
  carve(smem + warp * WarpMem<T>::bytes(11), 11, vec, &F0, &F1, &red, &ci, &act, &cid);
  T *X = vec[0], *Y = vec[1], *S0 = vec[2], *S1 = vec[3], *G0 = vec[4], *G1 = vec[5], *G2 = vec[6];
  const Tab<double>& t = c_tab_d;
  slot_cells(mp, -1, s0, lane, cid);
  stage_cells(mp, 0, lane, ci, act, cid);
  for (int e = lane; e < VEC; e += 32) {
    const int cw = e / N3;
    X[e] = act[cw] ? u[cid[cw] * N3 + (e - cw * N3)] : 0.0;
  }
  __syncwarp();
  contract<0, false, false>(X, S0, t.B, lane, act);
  __syncwarp();
  contract<1, false, false>(S0, S1, t.B, lane, act);
  __syncwarp();
  contract<2, false, false>(S1, S0, t.B, lane, act);   // S0 = u at the Gauss points
  __syncwarp();
  contract<0, false, false>(S0, G0, t.Dg, lane, act);
  contract<1, false, false>(S0, G1, t.Dg, lane, act);
  contract<2, false, false>(S0, G2, t.Dg, lane, act);
  __syncwarp();
  const double J = mp.h[0] * mp.h[1] * mp.h[2];
  for (int e = lane; e < VEC; e += 32) {
    const int cw = e / N3;
    if (!act[cw]) continue;
    const int q = e - cw * N3, qx = q % N, qy = (q / N) % N, qz = q / N2;
    int cx, cy, cz;
    cell_xyz(mp, cid[cw], cx, cy, cz);
    const double x[3] = {(cx + t.gq[qx]) * mp.h[0], (cy + t.gq[qy]) * mp.h[1], (cz + t.gq[qz]) * mp.h[2]};
    double K[6], c;
    var_coef(mp.var, x, K, c);
    const double wq = J * t.w[qx] * t.w[qy] * t.w[qz];
    const double g0 = G0[e] * mp.ih[0], g1 = G1[e] * mp.ih[1], g2 = G2[e] * mp.ih[2];
    G0[e] = wq * (K[0] * g0 + K[3] * g1 + K[4] * g2) * mp.ih[0];
    G1[e] = wq * (K[3] * g0 + K[1] * g1 + K[5] * g2) * mp.ih[1];
    G2[e] = wq * (K[4] * g0 + K[5] * g1 + K[2] * g2) * mp.ih[2];
    S0[e] = wq * c * S0[e];
  }
  __syncwarp();
  contract<0, true, true>(G0, S0, t.Dg, lane, act);
  __syncwarp();
  contract<1, true, true>(G1, S0, t.Dg, lane, act);
  __syncwarp();
  contract<2, true, true>(G2, S0, t.Dg, lane, act);
  __syncwarp();
  contract<2, true, false>(S0, S1, t.B, lane, act);
  __syncwarp();
  contract<1, true, false>(S1, S0, t.B, lane, act);
  __syncwarp();
  contract<0, true, false>(S0, Y, t.B, lane, act);
  __syncwarp();
  // faces (scratch: the 9 vectors after Y, contiguous)
  for (int sd = 0; sd < 2; ++sd) {
    faces_var<0>(mp, u, X, Y, S0, sd, lane, ci, act, cid);
    faces_var<1>(mp, u, X, Y, S0, sd, lane, ci, act, cid);
    faces_var<2>(mp, u, X, Y, S0, sd, lane, ci, act, cid);
  }
  for (int e = lane; e < VEC; e += 32) {
    const int cw = e / N3;
    if (act[cw]) v[cid[cw] * N3 + (e - cw * N3)] = Y[e];
  }
}

// Per-cell scalars of the inner GMRES(m): Hessenberg (m+1) x m, g, Givens
// cosines and sines, and the small solve y.
__host__ __device__ constexpr int gmres_scalars(int m) { return (m + 1) * m + 4 * m + 1; }

// Block-Jacobi sweep with inner right-preconditioned GMRES(m) (Algorithm 2;
// the inner solve of Sec. 2.2.1 for non-symmetric blocks, b != 0): per cell,
// V_0 = r / |r|; for j: w = D_T (V_j / diag), modified Gram-Schmidt, Givens
// rotations on the Hessenberg column, stop once the residual estimate
// |g_{j+1}| <= eps ||d|| or after maxit iterations; x += sum_i y_i V_i / diag;
// restart from the recomputed residual d - D_T x.  The warp count per block is
// blockDim.x / 32 (the basis needs (m+1) vectors per warp).
template <typename T, bool ADV, bool ELEM, typename G = typename Store<T>::type>
__global__ void __launch_bounds__(128) k_smooth_gmres(MeshParams mp, const G* __restrict__ f, const G* uold,
                                                      G* unew, const G* __restrict__ diag, T omega, T eps,
                                                      int maxit, int m, int* __restrict__ its, int color,
                                                      const T* __restrict__ tri) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  const long long s0 = ((long long)blockIdx.x * wpb + warp) * CPW;
  if (s0 >= color_count(mp, color)) return;
  const int nvec = m + 7;
  // advection: the element-form operator's region after the scalars
  constexpr int XA = (ADV && ELEM) ? kAdvExtra : 0;
  const size_t tbytes = align16((size_t)(nvec * VEC + 5 * LINES + CPW * gmres_scalars(m) + XA) * sizeof(T));
  const size_t wbytes = tbytes + align16(CPW * sizeof(CellInfo<T>)) + 16 + align16(CPW * sizeof(long long));
  unsigned char* base = smem + warp * wbytes;
  T* p = reinterpret_cast<T*>(base);
  T* V = p;                      // m+1 basis vectors
  T* Z = p + (m + 1) * VEC;      // preconditioned vector / block-apply input
  T* Q = Z + VEC;                // block-apply output
  T* S0 = Q + VEC;
  T* S1 = S0 + VEC;
  const bool react = mp.c != nullptr;
  const bool zero = uold == nullptr;
  T* DD = S1 + VEC;              // defect d
  T* X = DD + VEC;               // accumulated correction
  T* F0 = X + VEC;
  T* F1 = F0 + LINES;
  T* red = F1 + LINES;
  T* sc = red + 3 * LINES;       // CPW * gmres_scalars(m)
  T* Xa = sc + CPW * gmres_scalars(m);   // XA values (advection)
  CellInfo<T>* ci = reinterpret_cast<CellInfo<T>*>(base + tbytes);
  unsigned char* act = base + tbytes + align16(CPW * sizeof(CellInfo<T>));
  long long* cid = reinterpret_cast<long long*>(act + 16);
  slot_cells(mp, color, s0, lane, cid);
  stage_cells(mp, 0, lane, ci, act, cid);
  const long long cell0 = cid[0];
  if constexpr (ADV && ELEM) {
    adv_tables(Xa, lane);
    __syncwarp();
  }
  const int mycw = lane < LINES ? lane / N2 : -1;
  const bool mine = mycw >= 0 && act[mycw];
  const bool lead = lane < LINES && (lane % N2) == 0;    // writes the cell's scalars
  T* H = sc + (mycw >= 0 ? mycw : 0) * gmres_scalars(m);
  T* gv = H + (m + 1) * m;
  T* cs = gv + (m + 1);
  T* sn = cs + m;
  T* yv = sn + m;
  // defect d = f - A u_old
  if (!zero) {
    for (int e = lane; e < VEC; e += 32) {
      const int cw = e / N3;
      Z[e] = act[cw] ? T(uold[cid[cw] * N3 + (e - cw * N3)]) : T(0);
    }
    __syncwarp();
    if constexpr (ADV && ELEM) {
      adv_apply_e<true>(Z, Q, S0, S1, Xa, uold, mp, lane, act, ci);
    } else {
      volume<ADV>(Z, Q, S0, S1, lane, ci, act, react);
      all_faces<true, ADV>(Z, Q, F0, F1, uold, mp, cell0, lane, act, ci);
    }
  }
  T pdd = T(0);
  for (int L = lane; L < LINES; L += 32) {
    int cw, b0, st, a, b;
    line_geom<2>(L, cw, b0, st, a, b);
    if (!act[cw]) continue;
    const long long gb = cid[cw] * N3 - cw * N3;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const int e = b0 + i * N2;
      const T d = T(f[gb + e]) - (zero ? T(0) : Q[e]);
      DD[e] = d;
      X[e] = T(0);
      pdd = fma(d, d, pdd);
    }
  }
  // Work on d / ||d|| (subnormal FP32 products otherwise); the correction is
  // scaled back at the end, and the target eps ||d|| becomes eps.
  const T dnorm = sqrt(cell_sum(pdd, lane, red));
  const T isc = dnorm > T(0) ? T(1) / dnorm : T(0);
  for (int L = lane; L < LINES; L += 32) {
    int cw, b0, st, a, b;
    line_geom<2>(L, cw, b0, st, a, b);
    if (!act[cw]) continue;
#pragma unroll
    for (int i = 0; i < N; ++i) DD[b0 + i * N2] = DD[b0 + i * N2] * isc;
  }
  T beta = dnorm > T(0) ? T(1) : T(0);
  const T target = eps;
  bool live = mine && dnorm > T(0) && beta > target;
  int it = 0;
  // residual vector for the first cycle is d itself
  T* Rsrc = DD;
  while (__any_sync(FULLMASK, live && it < maxit)) {
    bool cyc = live && it < maxit;
    // V_0 = r / beta
    const T ibeta = cyc ? T(1) / beta : T(0);
    for (int L = lane; L < LINES; L += 32) {
      int cw, b0, st, a, b;
      line_geom<2>(L, cw, b0, st, a, b);
#pragma unroll
      for (int i = 0; i < N; ++i) {
        const int e = b0 + i * N2;
        if (cyc) V[e] = Rsrc[e] * ibeta;
      }
    }
    if (lead && cyc) {
      for (int k = 0; k <= m; ++k) gv[k] = T(0);
      gv[0] = beta;
    }
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      if (!__any_sync(FULLMASK, cyc)) break;
      if (lane < LINES) act[mycw] = cyc ? 1 : 0;
      __syncwarp();
      T* Vj = V + j * VEC;
      // Z = M^-1 V_j (M = diag(D_T), or its tridiagonal part); Q = D_T Z
      if (tri) {
        thomas_apply(tri, cid, act, Vj, Z, lane);
      } else {
        for (int L = lane; L < LINES; L += 32) {
          int cw, b0, st, a, b;
          line_geom<2>(L, cw, b0, st, a, b);
          if (!cyc) continue;
          const long long gb = cid[cw] * N3 - cw * N3;
#pragma unroll
          for (int i = 0; i < N; ++i) {
            const int e = b0 + i * N2;
            Z[e] = Vj[e] * T(diag[gb + e]);
          }
        }
      }
      __syncwarp();
      if constexpr (ADV && ELEM) {
        adv_apply_e<false>(Z, Q, S0, S1, Xa, (const G*)nullptr, mp, lane, act, ci);
      } else {
        volume<ADV>(Z, Q, S0, S1, lane, ci, act, react);
        all_faces<false, ADV>(Z, Q, F0, F1, (const G*)nullptr, mp, cell0, lane, act, ci);
      }
      // modified Gram-Schmidt
      for (int i = 0; i <= j; ++i) {
        const T* Vi = V + i * VEC;
        T ph = T(0);
        if (cyc) {
          for (int L = lane; L < LINES; L += 32) {
            int cw, b0, st, a, b;
            line_geom<2>(L, cw, b0, st, a, b);
#pragma unroll
            for (int k = 0; k < N; ++k) ph = fma(Q[b0 + k * N2], Vi[b0 + k * N2], ph);
          }
        }
        const T h = cell_sum(ph, lane, red);
        if (cyc) {
          for (int L = lane; L < LINES; L += 32) {
            int cw, b0, st, a, b;
            line_geom<2>(L, cw, b0, st, a, b);
#pragma unroll
            for (int k = 0; k < N; ++k) Q[b0 + k * N2] = fma(-h, Vi[b0 + k * N2], Q[b0 + k * N2]);
          }
          if (lead) H[i * m + j] = h;
        }
        __syncwarp();
      }
      T pw = T(0);
      if (cyc) {
        for (int L = lane; L < LINES; L += 32) {
          int cw, b0, st, a, b;
          line_geom<2>(L, cw, b0, st, a, b);
#pragma unroll
          for (int k = 0; k < N; ++k) pw = fma(Q[b0 + k * N2], Q[b0 + k * N2], pw);
        }
      }
      const T hn = sqrt(cell_sum(pw, lane, red));
      if (cyc) {
        T* Vn = V + (j + 1) * VEC;
        const T inv = hn != T(0) ? T(1) / hn : T(1);
        for (int L = lane; L < LINES; L += 32) {
          int cw, b0, st, a, b;
          line_geom<2>(L, cw, b0, st, a, b);
#pragma unroll
          for (int k = 0; k < N; ++k) Vn[b0 + k * N2] = hn != T(0) ? Q[b0 + k * N2] * inv : Q[b0 + k * N2];
        }
        if (lead) {
          H[(j + 1) * m + j] = hn;
          for (int i = 0; i < j; ++i) {
            const T t0 = cs[i] * H[i * m + j] + sn[i] * H[(i + 1) * m + j];
            H[(i + 1) * m + j] = -sn[i] * H[i * m + j] + cs[i] * H[(i + 1) * m + j];
            H[i * m + j] = t0;
          }
          const T den = hypot(H[j * m + j], H[(j + 1) * m + j]);
          cs[j] = H[j * m + j] / den;
          sn[j] = H[(j + 1) * m + j] / den;
          H[j * m + j] = den;
          H[(j + 1) * m + j] = T(0);
          gv[j + 1] = -sn[j] * gv[j];
          gv[j] = cs[j] * gv[j];
        }
      }
      __syncwarp();
      if (cyc) {
        ++it;
        jdone = j + 1;
        if (fabs(gv[j + 1]) <= target || it >= maxit) cyc = false;
      }
      __syncwarp();
    }
    // y = H^-1 g (upper triangular, size jdone), then X += sum_i y_i V_i / diag
    const bool ran = live && jdone > 0;
    if (lead && ran) {
      for (int i = jdone - 1; i >= 0; --i) {
        T s = gv[i];
        for (int l = i + 1; l < jdone; ++l) s = s - H[i * m + l] * yv[l];
        yv[i] = s / H[i * m + i];
      }
    }
    __syncwarp();
    if (tri) {
      // X += M^-1 (V y)
      if (lane < LINES) act[mycw] = ran ? 1 : 0;
      if (ran) {
        for (int L = lane; L < LINES; L += 32) {
          int cw, b0, st, a, b;
          line_geom<2>(L, cw, b0, st, a, b);
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const int e = b0 + k * N2;
            T s = T(0);
            for (int i = 0; i < jdone; ++i) s = fma(yv[i], V[i * VEC + e], s);
            Z[e] = s;
          }
        }
      }
      __syncwarp();
      thomas_apply(tri, cid, act, Z, S0, lane);
      if (ran) {
        for (int L = lane; L < LINES; L += 32) {
          int cw, b0, st, a, b;
          line_geom<2>(L, cw, b0, st, a, b);
#pragma unroll
          for (int k = 0; k < N; ++k) X[b0 + k * N2] += S0[b0 + k * N2];
        }
      }
    } else if (ran) {
      for (int L = lane; L < LINES; L += 32) {
        int cw, b0, st, a, b;
        line_geom<2>(L, cw, b0, st, a, b);
        const long long gb = cid[cw] * N3 - cw * N3;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const int e = b0 + k * N2;
          T s = T(0);
          for (int i = 0; i < jdone; ++i) s = fma(yv[i], V[i * VEC + e], s);
          X[e] = fma(s, T(diag[gb + e]), X[e]);
        }
      }
    }
    // r = d - D_T x; beta = ||r||
    if (lane < LINES) act[mycw] = ran ? 1 : 0;
    __syncwarp();
    if constexpr (ADV && ELEM) {
      adv_apply_e<false>(X, Q, S0, S1, Xa, (const G*)nullptr, mp, lane, act, ci);
    } else {
      volume<ADV>(X, Q, S0, S1, lane, ci, act, react);
      all_faces<false, ADV>(X, Q, F0, F1, (const G*)nullptr, mp, cell0, lane, act, ci);
    }
    T pr = T(0);
    if (ran) {
      for (int L = lane; L < LINES; L += 32) {
        int cw, b0, st, a, b;
        line_geom<2>(L, cw, b0, st, a, b);
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const int e = b0 + k * N2;
          const T r = DD[e] - Q[e];
          Q[e] = r;
          pr = fma(r, r, pr);
        }
      }
    }
    const T bn = sqrt(cell_sum(pr, lane, red));
    if (ran) {
      beta = bn;
      if (!(beta > target)) live = false;
    }
    Rsrc = Q;
    __syncwarp();
  }
  for (int L = lane; L < LINES; L += 32) {
    int cw, b0, st, a, b;
    line_geom<2>(L, cw, b0, st, a, b);
    if (cid[cw] < 0) continue;
    const long long gb = cid[cw] * N3 - cw * N3;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      const long long gi = gb + b0 + i * N2;
      const T x = X[b0 + i * N2] * dnorm;
      unew[gi] = static_cast<G>(zero ? omega * x : fma(omega, x, T(uold[gi])));
    }
  }
  if (its && lead && cid[mycw] >= 0) its[cid[mycw]] = it;
}

// diag(D_T) by direct quadrature per dof (setup; FP64).
template <bool ADV>
__global__ void k_diag(MeshParams mp, double* __restrict__ diag) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= mp.ncell * N3) return;
  const long long c = gid / N3;
  const int i = (int)(gid - c * N3);
  const int ii[3] = {i % N, (i / N) % N, i / N2};
  const Tab<double>& t = c_tab_d;
  const double J = mp.h[0] * mp.h[1] * mp.h[2];
  const double K[3] = {kcoef(mp, c, 0), kcoef(mp, c, 1), kcoef(mp, c, 2)};
  const double cc = mp.c ? mp.c[c] : 0.0;
  double bc[3][8];
  if (ADV) {
    int cx, cy, cz;
    cell_xyz(mp, c, cx, cy, cz);
    const long long vx = mp.nx + 1, vxy = (long long)(mp.nx + 1) * (mp.ny + 1);
    for (int k = 0; k < 8; ++k) {
      const long long v = (cx + (k & 1)) + vx * (cy + ((k >> 1) & 1)) + vxy * (cz + (k >> 2));
      for (int d = 0; d < 3; ++d) bc[d][k] = mp.bvert[3 * v + d];
    }
  }
  double acc = 0.0;
  for (int q3 = 0; q3 < N; ++q3)
    for (int q2 = 0; q2 < N; ++q2)
      for (int q1 = 0; q1 < N; ++q1) {
        const int q[3] = {q1, q2, q3};
        const double w = t.w[q1] * t.w[q2] * t.w[q3] * J;
        double val = 1.0, g[3];
        for (int d = 0; d < 3; ++d) val *= t.B[q[d]][ii[d]];
        for (int d = 0; d < 3; ++d) {
          g[d] = t.G[q[d]][ii[d]] / mp.h[d];
          for (int e = 0; e < 3; ++e)
            if (e != d) g[d] *= t.B[q[e]][ii[e]];
        }
        acc += w * (K[0] * g[0] * g[0] + K[1] * g[1] * g[1] + K[2] * g[2] * g[2] + cc * val * val);
        if (ADV) {
          double b[3] = {0, 0, 0};
          for (int k = 0; k < 8; ++k) {
            double wk = 1.0;
            for (int d = 0; d < 3; ++d) wk *= ((k >> d) & 1) ? t.gq[q[d]] : 1.0 - t.gq[q[d]];
            for (int d = 0; d < 3; ++d) b[d] += wk * bc[d][k];
          }
          acc -= w * val * (b[0] * g[0] + b[1] * g[1] + b[2] * g[2]);
        }
      }
  const double pen = mp.alpha * mp.p * (mp.p + 2);
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) {
      if (ii[d] != (s ? N - 1 : 0)) continue;
      long long nb;
      const int kind = face_kind(mp, c, d, s, nb);
      if (kind == 2) continue;
      const int ta = d == 0 ? 1 : 0, tb = d == 2 ? 1 : 2;
      const double area = mp.h[ta] * mp.h[tb];
      const double mass = area * t.M1[ii[ta]][ii[ta]] * t.M1[ii[tb]][ii[tb]];
      const double sgn = s ? 1.0 : -1.0;
      const double dterm = sgn / mp.h[d] * t.dl[s][ii[d]] * mass;
      double kap, gam;
      if (kind == 0) {
        const double ko = kcoef(mp, nb, d);
        kap = K[d] * ko / (K[d] + ko);
        gam = 2.0 * pen * kap / mp.h[d];
      } else {
        kap = K[d];
        gam = pen * kap / mp.h[d];
      }
      acc += gam * mass - 2.0 * kap * dterm;
      if (ADV) {
        for (int qb = 0; qb < N; ++qb)
          for (int qa = 0; qa < N; ++qa) {
            double bn = 0.0;
            for (int k = 0; k < 8; ++k) {
              const int o[3] = {k & 1, (k >> 1) & 1, (k >> 2) & 1};
              if (o[d] != s) continue;
              const double wa = o[ta] ? t.gq[qa] : 1.0 - t.gq[qa];
              const double wb = o[tb] ? t.gq[qb] : 1.0 - t.gq[qb];
              bn += bc[d][k] * wa * wb;
            }
            bn *= sgn;
            if (bn > 0.0) {
              const double ph = t.B[qa][ii[ta]] * t.B[qb][ii[tb]];
              acc += t.w[qa] * t.w[qb] * area * bn * ph * ph;
            }
          }
      }
    }
  diag[gid] = acc;
}

// diag(D_T) for b = 0 from the Kronecker form of the block on affine
// axis-aligned cells with K diagonal and constant per cell,
// D_T = A_x (x) M (x) M + M (x) A_y (x) M + M (x) M (x) A_z:
//   diag(D_T)(i0, i1, i2) = a_x(i0) m(i1) m(i2) + m(i0) a_y(i1) m(i2) + m(i0) m(i1) a_z(i2),
// m = diag(M), a_d = diag(A_d) = |J| K_d / h_d^2 S_ii (+ c |J| M_ii for d = 2)
// + on each non-Neumann face s of d, at its end node e: |F| (2 ks dl_s(e) + gamma),
// ks = -kap sg / h_d (the diagonal of the per-cell matrices of block_matrices).
// n^3 work per cell instead of the n^6 of the quadrature in k_diag.
__global__ void k_diag_kron(MeshParams mp, double* __restrict__ diag) {
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= mp.ncell * N3) return;
  const long long c = gid / N3;
  const int i = (int)(gid - c * N3);
  const int ii[3] = {i % N, (i / N) % N, i / N2};
  const Tab<double>& t = c_tab_d;
  const double* rec = mp.rec64 + c * kRecLen;
  double a[3];
  for (int d = 0; d < 3; ++d) {
    const int k = ii[d];
    double v = rec[kRecKd + d] * t.S1[k][k];
    if (d == 2) v = fma(rec[kRecCJ], t.M1[k][k], v);
    for (int s = 0; s < 2; ++s) {
      if (k != (s ? N - 1 : 0)) continue;
      long long nb;
      if (face_kind(mp, c, d, s, nb) == 2) continue;
      const double kap = rec[kRecKap + 2 * d + s], gam = rec[kRecGam + 2 * d + s];
      const double ks = (s ? -kap : kap) * mp.ih[d];
      v = fma(mp.jh[d], 2.0 * ks * t.dl[s][k] + gam, v);
    }
    a[d] = v;
  }
  const double m0 = t.M1[ii[0]][ii[0]], m1 = t.M1[ii[1]][ii[1]], m2 = t.M1[ii[2]][ii[2]];
  diag[gid] = a[0] * m1 * m2 + m0 * a[1] * m2 + m0 * m1 * a[2];
}

// Lanes per cell of the transfer kernels (at least 8: one per corner) and
// cells per warp: a lane per z-line (i, j) of the cell, n^2 lines.
constexpr int kTG = N2 <= 8 ? 8 : (N2 <= 16 ? 16 : 32);
constexpr int kTCells = 32 / kTG;

// Corner sums r_hat_c(T) = sum_i prod_k phi_{c_k}(zeta_{i_k}) r_T(i) (the cell
// part of R = P^T), in the separable order: each lane sums its z-line with
// the two z hats (coalesced loads: the lanes' lines are adjacent), weights
// the two sums with the four products of x and y hats of its line, and a
// fixed-order reduction over the cell's lanes gives the 8 corners (kernel
// precision; 4 flops per dof).  The reduction is transposed: at each of the
// first three levels a lane keeps half of its values and adds its partner's
// matching half, so that 8 values over kTG lanes take log2(kTG) + 4
// shuffle-adds per lane instead of 8 log2(kTG) (the FP64 adds of the plain
// tree cost more than the sums themselves).
template <typename T>
__device__ __forceinline__ void restrict_cells_body(long long ncell, const T* __restrict__ r,
                                                    double* __restrict__ corners, unsigned bid) {
  const int lane = threadIdx.x & 31;
  const long long c0 = (((long long)bid * blockDim.x + threadIdx.x) >> 5) * kTCells;
  if (c0 >= ncell) return;   // the whole warp
  const long long c = c0 + lane / kTG;
  const int g = lane % kTG;
  const bool on = c < ncell;
  const Tab<T>& t = tab<T>();
  T acc[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) acc[k] = T(0);
  if (on) {
    const T* rc = r + c * N3;
    for (int L = g; L < N2; L += kTG) {
      T s0 = T(0), s1 = T(0);
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T v = rc[L + N2 * k];
        s0 = fma(t.hat[0][k], v, s0);
        s1 = fma(t.hat[1][k], v, s1);
      }
      const int i = L % N, j = L / N;
      const T x0y0 = t.hat[0][i] * t.hat[0][j], x1y0 = t.hat[1][i] * t.hat[0][j];
      const T x0y1 = t.hat[0][i] * t.hat[1][j], x1y1 = t.hat[1][i] * t.hat[1][j];
      acc[0] = fma(x0y0, s0, acc[0]);
      acc[1] = fma(x1y0, s0, acc[1]);
      acc[2] = fma(x0y1, s0, acc[2]);
      acc[3] = fma(x1y1, s0, acc[3]);
      acc[4] = fma(x0y0, s1, acc[4]);
      acc[5] = fma(x1y0, s1, acc[5]);
      acc[6] = fma(x0y1, s1, acc[6]);
      acc[7] = fma(x1y1, s1, acc[7]);
    }
  }
  // xor offsets below kTG stay within the cell's lanes.  Levels with offsets
  // kTG/2, kTG/4, kTG/8: the lower lane of a pair keeps values [0, h), the
  // upper one [h, 2h), each adding the partner's copy of what it keeps; then
  // the lane holds corner g / (kTG / 8), summed over the remaining offsets.
#pragma unroll
  for (int h = 4, o = kTG / 2; h >= 1; h >>= 1, o >>= 1) {
    const bool upper = (g & o) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const T send = upper ? acc[k] : acc[k + h];
      const T keep = upper ? acc[k + h] : acc[k];
      acc[k] = keep + __shfl_xor_sync(FULLMASK, send, o);
    }
  }
#pragma unroll
  for (int o = kTG / 16; o > 0; o >>= 1) acc[0] += __shfl_xor_sync(FULLMASK, acc[0], o);
  constexpr int kSpan = kTG / 8;   // lanes per corner
  if (on && g % kSpan == 0) corners[c * 8 + g / kSpan] = (double)acc[0];
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_cells(long long ncell, const T* __restrict__ r,
                                                        double* __restrict__ corners) {
  restrict_cells_body<T>(ncell, r, corners, blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_cells_batch(const __grid_constant__ BatchTable bt) {
  const int m = batch_member(bt, blockIdx.x);
  restrict_cells_body<T>(bt.mp[m].ncell, (const T*)bt.in[m], (double*)bt.out[m], blockIdx.x - bt.block0[m]);
}

// u_T(i) += sum_c u_hat(vertex(T, c)) prod_k phi_{c_k}(zeta_{i_k}), separable:
// the cell's first 8 lanes load its corner values and broadcast them; each
// lane blends them bilinearly in x and y for its z-line (i, j), once for the
// z = 0 and once for the z = 1 corners, and adds the linear blend in z to the
// n values of the line (coalesced across the lanes; two FMAs per dof).
template <typename T>
__device__ __forceinline__ void prolong_add_body(const MeshParams& mp, const double* __restrict__ uhat,
                                                 T* __restrict__ u, unsigned bid) {
  const int lane = threadIdx.x & 31;
  const long long c0 = (((long long)bid * blockDim.x + threadIdx.x) >> 5) * kTCells;
  if (c0 >= mp.ncell) return;   // the whole warp
  const long long c = c0 + lane / kTG;
  const int g = lane % kTG;
  const bool on = c < mp.ncell;
  T cv = T(0);
  if (on && g < 8) {
    int cx, cy, cz;
    cell_xyz(mp, c, cx, cy, cz);
    const long long vx = mp.nx + 1, vxy = (long long)(mp.nx + 1) * (mp.ny + 1);
    const long long v = (cx + (g & 1)) + vx * (cy + ((g >> 1) & 1)) + vxy * (cz + (g >> 2));
    cv = (T)uhat[v];
  }
  T cor[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) cor[k] = __shfl_sync(FULLMASK, cv, lane - g + k);
  if (!on) return;
  const Tab<T>& t = tab<T>();
  T* uc = u + c * N3;
  for (int L = g; L < N2; L += kTG) {
    const int i = L % N, j = L / N;
    const T x0 = t.hat[0][i], x1 = t.hat[1][i], y0 = t.hat[0][j], y1 = t.hat[1][j];
    const T g0 = fma(y1, fma(x1, cor[3], x0 * cor[2]), y0 * fma(x1, cor[1], x0 * cor[0]));
    const T g1 = fma(y1, fma(x1, cor[7], x0 * cor[6]), y0 * fma(x1, cor[5], x0 * cor[4]));
#pragma unroll
    for (int k = 0; k < N; ++k) uc[L + N2 * k] = fma(t.hat[1][k], g1, fma(t.hat[0][k], g0, uc[L + N2 * k]));
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(const __grid_constant__ MeshParams mp,
                                                     const double* __restrict__ uhat, T* __restrict__ u) {
  prolong_add_body<T>(mp, uhat, u, blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add_batch(const __grid_constant__ BatchTable bt) {
  const int m = batch_member(bt, blockIdx.x);
  prolong_add_body<T>(bt.mp[m], (const double*)bt.in[m], (T*)bt.out[m], blockIdx.x - bt.block0[m]);
}

#include "plane_kernels.cuh"

// ---------------------------------------------------------------- launchers
// Synchronous copies: the staging struct lives on the host stack.
template <typename T>
cudaError_t upload_one(const double* h) {
  Tab<T> tb;
  const double* p = h;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) tb.B[i][j] = T(p[i * N + j]);
  p += N2;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) tb.Dg[i][j] = T(p[i * N + j]);
  p += N2;
  for (int i = 0; i < N; ++i) tb.w[i] = T(p[i]);
  p += N;
  for (int s2 = 0; s2 < 2; ++s2)
    for (int i = 0; i < N; ++i) tb.dl[s2][i] = T(p[s2 * N + i]);
  p += 2 * N;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) tb.M1[i][j] = T(p[i * N + j]);
  p += N2;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) tb.G[i][j] = T(p[i * N + j]);
  p += N2;
  for (int s2 = 0; s2 < 2; ++s2)
    for (int i = 0; i < N; ++i) tb.hat[s2][i] = T(p[s2 * N + i]);
  p += 2 * N;
  for (int i = 0; i < N; ++i) tb.gq[i] = T(p[i]);
  p += N;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) tb.S1[i][j] = T(p[i * N + j]);
  // M^-1 by Gauss-Jordan elimination with partial pivoting in long double
  // (M is symmetric positive definite with condition number below 20 for
  // n <= 9), then M^-1 S, M^-1 e_0, M^-1 e_{n-1}, M^-1 dl_s
  const double* M1 = h + 2 * N2 + 3 * N;
  const double* S1 = p;
  const double* dl = h + 2 * N2 + N;
  long double a[N][2 * N];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < 2 * N; ++j) a[i][j] = j < N ? (long double)M1[i * N + j] : (j - N == i ? 1.0L : 0.0L);
  for (int c = 0; c < N; ++c) {
    int piv = c;
    for (int r = c + 1; r < N; ++r)
      if (fabsl(a[r][c]) > fabsl(a[piv][c])) piv = r;
    for (int j = 0; j < 2 * N; ++j) {
      const long double tmp = a[c][j];
      a[c][j] = a[piv][j];
      a[piv][j] = tmp;
    }
    const long double ip = 1.0L / a[c][c];
    for (int j = 0; j < 2 * N; ++j) a[c][j] *= ip;
    for (int r = 0; r < N; ++r) {
      if (r == c) continue;
      const long double m = a[r][c];
      for (int j = 0; j < 2 * N; ++j) a[r][j] -= m * a[c][j];
    }
  }
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < N; ++j) {
      long double v = 0.0L;
      for (int k = 0; k < N; ++k) v += a[i][N + k] * (long double)S1[k * N + j];
      tb.MIS[i][j] = T((double)v);
    }
    tb.mie[0][i] = T((double)a[i][N]);
    tb.mie[1][i] = T((double)a[i][2 * N - 1]);
    for (int s2 = 0; s2 < 2; ++s2) {
      long double v = 0.0L;
      for (int k = 0; k < N; ++k) v += a[i][N + k] * (long double)dl[s2 * N + k];
      tb.midl[s2][i] = T((double)v);
    }
  }
  if (std::is_same<T, double>::value) return cudaMemcpyToSymbol(c_tab_d, &tb, sizeof(tb));
  if (std::is_same<T, df>::value) return cudaMemcpyToSymbol(c_tab_df, &tb, sizeof(tb));
  return cudaMemcpyToSymbol(c_tab_f, &tb, sizeof(tb));
}

cudaError_t upload_tables(const double* h, cudaStream_t) {
  cudaError_t e = upload_one<double>(h);
  if (e != cudaSuccess) return e;
  e = upload_one<float>(h);
  if (e != cudaSuccess) return e;
  return upload_one<df>(h);
}

inline long long host_color_count(const MeshParams& mp, int color) {
  const int kx = color & 1, ky = (color >> 1) & 1, kz = color >> 2;
  return (long long)((mp.nx - kx + 1) / 2) * ((mp.ny - ky + 1) / 2) * ((mp.nz - kz + 1) / 2);
}

inline unsigned grid_for(long long ncell, int wpb) {
  const long long groups = (ncell + CPW - 1) / CPW;
  return (unsigned)((groups + wpb - 1) / wpb);
}

// Warps per block of a launch: the tuned value if it fits in shared memory,
// else the largest power of two <= 4 that does.
inline int pick_wpb(int tuned, size_t per_warp) {
  int w = (tuned >= 1 && tuned <= 8) ? tuned : WPB;
  while (w > 1 && (size_t)w * per_warp > 200 * 1024) w >>= 1;
  return w;
}

template <typename T> constexpr int prec_index() { return DGMG_FP64; }
template <> constexpr int prec_index<float>() { return DGMG_FP32; }
template <> constexpr int prec_index<df>() { return DGMG_DF64; }

template <typename KernelT>
cudaError_t set_smem(KernelT k, size_t bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  return cudaSuccess;
}

// Warps per block, at most wmax (the kernel's launch bound / 32).
[[maybe_unused]] inline int pick_wpb_max(int tuned, size_t per_warp, int wmax) {
  int w = pick_wpb(tuned, per_warp);
  while (w > wmax) w >>= 1;
  return w;
}

template <typename T, bool FULL, bool ADV, bool FAC>
cudaError_t launch_apply_form(const MeshParams& mp, const void* u, void* v, cudaStream_t s) {
  using G = typename Store<T>::type;
  constexpr int XT = FAC ? (ADV ? kAdvExtra : kFactorExtra) : 0;
  const int wpb = pick_wpb(mp.wpb_apply[prec_index<T>()], WarpMem<T>::bytes(4, XT));
  const size_t sm = wpb * WarpMem<T>::bytes(4, XT);
  auto k = k_apply<T, FULL, ADV, FAC>;
  cudaError_t e = set_smem(k, sm);
  if (e != cudaSuccess) return e;
  k<<<grid_for(mp.ncell, wpb), wpb * 32, sm, s>>>(mp, (const G*)u, (G*)v);
  count_launch();
  return cudaGetLastError();
}

#if DGMG_N <= 5
template <bool FULL>
cudaError_t launch_apply_plane(const MeshParams& mp, const void* u, void* v, cudaStream_t s) {
  const size_t per = pl::warp_bytes(FULL);
  const int wpb = pick_wpb_max(mp.wpb_apply[DGMG_FP32], per, 8);
  const size_t sm = wpb * per;
  auto k = k_apply_plane<FULL>;
  cudaError_t e = set_smem(k, sm);
  if (e != cudaSuccess) return e;
  const long long groups = (mp.ncell + pl::PC - 1) / pl::PC;
  k<<<(unsigned)((groups + wpb - 1) / wpb), wpb * 32, sm, s>>>(mp, (const float*)u, (float*)v);
  count_launch();
  return cudaGetLastError();
}
#endif

// Operator launch in the layout the mesh parameters select for this
// precision (advection: the line form at the Gauss points).
template <typename T, bool FULL, bool ADV>
cudaError_t launch_apply(const MeshParams& mp, const void* u, void* v, cudaStream_t s) {
  if constexpr (ADV) {
    if (mp.lay_apply[prec_index<T>()] == DGMG_LAYOUT_ELEMENT) return launch_apply_form<T, FULL, true, true>(mp, u, v, s);
    return launch_apply_form<T, FULL, true, false>(mp, u, v, s);
  } else {
    const int lay = mp.lay_apply[prec_index<T>()];
#if DGMG_N <= 5
    if constexpr (std::is_same<T, float>::value)
      if (lay == DGMG_LAYOUT_PLANE) return launch_apply_plane<FULL>(mp, u, v, s);
#endif
    if (lay == DGMG_LAYOUT_LINE) return launch_apply_form<T, FULL, false, false>(mp, u, v, s);
    return launch_apply_form<T, FULL, false, true>(mp, u, v, s);
  }
}

template <typename T, bool FULL>
cudaError_t apply_t(const MeshParams& mp, const void* u, void* v, cudaStream_t s) {
  return mp.bvert ? launch_apply<T, FULL, true>(mp, u, v, s) : launch_apply<T, FULL, false>(mp, u, v, s);
}

cudaError_t apply(const MeshParams& mp, const void* u, void* v, int prec, bool full, cudaStream_t s) {
  if (mp.ncell == 0) return cudaSuccess;
  if (prec == DGMG_FP32) return full ? apply_t<float, true>(mp, u, v, s) : apply_t<float, false>(mp, u, v, s);
  if (prec == DGMG_DF64) {
    // double-float kernels: diffusion operators (b = 0), p <= 6
#if DGMG_N <= 7
    if (mp.bvert) return cudaErrorNotSupported;
    return full ? launch_apply<df, true, false>(mp, u, v, s) : launch_apply<df, false, false>(mp, u, v, s);
#else
    return cudaErrorNotSupported;
#endif
  }
  return full ? apply_t<double, true>(mp, u, v, s) : apply_t<double, false>(mp, u, v, s);
}

template <typename T, bool ADV, bool FAC>
cudaError_t launch_smooth_form(const MeshParams& mp, const SmoothArgs& a, cudaStream_t s) {
  using G = typename Store<T>::type;
  constexpr int XT = smooth_extra<ADV, FAC>();
  const int wpb = pick_wpb(mp.wpb_smooth[prec_index<T>()], WarpMem<T>::bytes(6, XT));
  const size_t sm = wpb * WarpMem<T>::bytes(6, XT);
  auto k = k_smooth_pcg<T, ADV, FAC>;
  cudaError_t e = set_smem(k, sm);
  if (e != cudaSuccess) return e;
  const long long cells = a.color < 0 ? mp.ncell : host_color_count(mp, a.color);
  k<<<grid_for(cells, wpb), wpb * 32, sm, s>>>(mp, (const G*)a.f, (const G*)a.uold, (G*)a.unew, (const G*)a.diag,
                                          T(a.omega), T(a.eps), a.maxit, a.its, a.color);
  count_launch();
  return cudaGetLastError();
}

// Inner-PCG sweep in the selected layout; the plane form covers the Jacobi
// sweep over all cells (a colour of block-SOR takes the line form).
template <typename T, bool ADV>
cudaError_t launch_smooth(const MeshParams& mp, const SmoothArgs& a, cudaStream_t s) {
  if constexpr (ADV) {
    if (mp.lay_smooth[prec_index<T>()] == DGMG_LAYOUT_ELEMENT) return launch_smooth_form<T, true, true>(mp, a, s);
    return launch_smooth_form<T, true, false>(mp, a, s);
  } else {
    const int lay = mp.lay_smooth[prec_index<T>()];
#if DGMG_N <= 5
    if constexpr (std::is_same<T, float>::value) {
      if (lay == DGMG_LAYOUT_PLANE) {
        if (a.color >= 0) return launch_smooth_form<float, false, false>(mp, a, s);
        const size_t per = pl::warp_bytes(true);
        const int wpb = pick_wpb_max(mp.wpb_smooth[DGMG_FP32], per, 4);
        const size_t sm = wpb * per;
        cudaError_t e = set_smem(k_smooth_plane, sm);
        if (e != cudaSuccess) return e;
        const long long groups = (mp.ncell + pl::PC - 1) / pl::PC;
        k_smooth_plane<<<(unsigned)((groups + wpb - 1) / wpb), wpb * 32, sm, s>>>(
            mp, (const float*)a.f, (const float*)a.uold, (float*)a.unew, (const float*)a.diag, float(a.omega),
            float(a.eps), a.maxit, a.its);
        count_launch();
        return cudaGetLastError();
      }
    }
#endif
    if (lay == DGMG_LAYOUT_LINE || lay == DGMG_LAYOUT_PLANE) return launch_smooth_form<T, false, false>(mp, a, s);
    return launch_smooth_form<T, false, true>(mp, a, s);
  }
}

template <typename T, bool ADV, bool FAC>
cudaError_t launch_inv_form(const MeshParams& mp, const SmoothArgs& a, cudaStream_t s) {
  using G = typename Store<T>::type;
  constexpr int XT = FAC ? (ADV ? kAdvExtra : kFactorExtra) : 0;
  const int wpb = pick_wpb(mp.wpb_apply[prec_index<T>()], WarpMem<T>::bytes(4, XT));
  const size_t sm = wpb * WarpMem<T>::bytes(4, XT);
  auto k = k_smooth_inv<T, ADV, FAC>;
  cudaError_t e = set_smem(k, sm);
  if (e != cudaSuccess) return e;
  const long long cells = a.color < 0 ? mp.ncell : host_color_count(mp, a.color);
  using M = typename InvEntry<T>::type;
  k<<<grid_for(cells, wpb), wpb * 32, sm, s>>>(mp, (const G*)a.f, (const G*)a.uold, (G*)a.unew, (const M*)a.binv,
                                          a.binv_ld, T(a.omega), a.its, a.color);
  count_launch();
  return cudaGetLastError();
}

// Stored-inverse sweep; its defect takes the factored form where the
// smoother layout is the factored one.
template <typename T, bool ADV>
cudaError_t launch_inv(const MeshParams& mp, const SmoothArgs& a, cudaStream_t s) {
  if (!a.binv) return cudaErrorInvalidValue;
  if constexpr (ADV) {
    if (mp.lay_smooth[prec_index<T>()] == DGMG_LAYOUT_ELEMENT) return launch_inv_form<T, true, true>(mp, a, s);
    return launch_inv_form<T, true, false>(mp, a, s);
  } else {
    if (mp.lay_smooth[prec_index<T>()] == DGMG_LAYOUT_ELEMENT) return launch_inv_form<T, false, true>(mp, a, s);
    return launch_inv_form<T, false, false>(mp, a, s);
  }
}

template <bool ADV>
cudaError_t launch_block_matrix(const MeshParams& mp, double* out, int ld, cudaStream_t s) {
  const int wpb = pick_wpb(0, WarpMem<double>::bytes(4));
  const size_t sm = wpb * WarpMem<double>::bytes(4);
  auto k = k_block_matrix<ADV>;
  cudaError_t e = set_smem(k, sm);
  if (e != cudaSuccess) return e;
  k<<<grid_for(mp.ncell, wpb), wpb * 32, sm, s>>>(mp, out, ld);
  count_launch();
  return cudaGetLastError();
}

template <bool ADV>
cudaError_t launch_block_tridiag(const MeshParams& mp, double* out, int* singular, cudaStream_t s) {
  const int wpb = pick_wpb(0, WarpMem<double>::bytes(7));
  const size_t sm = wpb * WarpMem<double>::bytes(7);
  auto k = k_block_tridiag<ADV>;
  cudaError_t e = set_smem(k, sm);
  if (e != cudaSuccess) return e;
  k<<<grid_for(mp.ncell, wpb), wpb * 32, sm, s>>>(mp, out, singular);
  count_launch();
  return cudaGetLastError();
}

cudaError_t apply_var(const MeshParams& mp, const double* u, double* v, cudaStream_t s) {
  if (mp.ncell == 0) return cudaSuccess;
  if (!mp.var || mp.bvert) return cudaErrorInvalidValue;
  const int wpb = pick_wpb(mp.wpb_apply[DGMG_FP64], WarpMem<double>::bytes(11));
  const size_t sm = wpb * WarpMem<double>::bytes(11);
  cudaError_t e = set_smem(k_apply_var, sm);
  if (e != cudaSuccess) return e;
  k_apply_var<<<grid_for(mp.ncell, wpb), wpb * 32, sm, s>>>(mp, u, v);
  count_launch();
  return cudaGetLastError();
}

cudaError_t block_tridiag(const MeshParams& mp, double* out, int* singular, cudaStream_t s) {
  if (mp.ncell == 0) return cudaSuccess;
  return mp.bvert ? launch_block_tridiag<true>(mp, out, singular, s)
                  : launch_block_tridiag<false>(mp, out, singular, s);
}

cudaError_t block_matrix(const MeshParams& mp, double* out, int ld, cudaStream_t s) {
  if (mp.ncell == 0) return cudaSuccess;
  if (ld < N3) return cudaErrorInvalidValue;
  return mp.bvert ? launch_block_matrix<true>(mp, out, ld, s) : launch_block_matrix<false>(mp, out, ld, s);
}

template <typename T, bool ADV, bool ELEM>
cudaError_t launch_gmres_form(const MeshParams& mp, const SmoothArgs& a, cudaStream_t s) {
  using G = typename Store<T>::type;
  const int m = a.restart;
  constexpr int XA = (ADV && ELEM) ? kAdvExtra : 0;
  const size_t wbytes =
      align16((size_t)((m + 7) * VEC + 5 * LINES + CPW * gmres_scalars(m) + XA) * sizeof(T)) +
      align16(CPW * sizeof(CellInfo<T>)) + 16 + align16(CPW * sizeof(long long));
  int wpb = (int)((200 * 1024) / wbytes);
  if (wpb > 4) wpb = 4;
  if (wpb < 1) return cudaErrorInvalidValue;      // restart too large for shared memory
  const size_t sm = wpb * wbytes;
  auto k = k_smooth_gmres<T, ADV, ELEM>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long long cells = a.color < 0 ? mp.ncell : host_color_count(mp, a.color);
  const long long groups = (cells + CPW - 1) / CPW;
  const unsigned grid = (unsigned)((groups + wpb - 1) / wpb);
  k<<<grid, wpb * 32, sm, s>>>(mp, (const G*)a.f, (const G*)a.uold, (G*)a.unew, (const G*)a.diag, T(a.omega),
                               T(a.eps), a.maxit, m, a.its, a.color, (const T*)a.tri);
  count_launch();
  return cudaGetLastError();
}

// GMRES sweep; with advection the element or line form by the smoother layout.
template <typename T, bool ADV>
cudaError_t launch_gmres(const MeshParams& mp, const SmoothArgs& a, cudaStream_t s) {
  if constexpr (ADV) {
    if (mp.lay_smooth[prec_index<T>()] == DGMG_LAYOUT_ELEMENT) return launch_gmres_form<T, true, true>(mp, a, s);
    return launch_gmres_form<T, true, false>(mp, a, s);
  } else {
    return launch_gmres_form<T, false, false>(mp, a, s);
  }
}

template <typename T>
cudaError_t smooth_t(const MeshParams& mp, const SmoothArgs& a, cudaStream_t s) {
  const bool adv = mp.bvert != nullptr;
  if (a.inner == DGMG_INNER_GMRES || a.inner == DGMG_INNER_GMRES_TRIDIAG) {
    if ((a.inner == DGMG_INNER_GMRES_TRIDIAG) != (a.tri != nullptr)) return cudaErrorInvalidValue;
    return adv ? launch_gmres<T, true>(mp, a, s) : launch_gmres<T, false>(mp, a, s);
  }
  if (a.inner == DGMG_INNER_DIRECT) return adv ? launch_inv<T, true>(mp, a, s) : launch_inv<T, false>(mp, a, s);
  return adv ? launch_smooth<T, true>(mp, a, s) : launch_smooth<T, false>(mp, a, s);
}

cudaError_t smooth(const MeshParams& mp, const SmoothArgs& a, int prec, cudaStream_t s) {
  if (mp.ncell == 0) return cudaSuccess;
  if (prec == DGMG_FP32) return smooth_t<float>(mp, a, s);
  if (prec == DGMG_DF64) {
    // double-float smoother: block-Jacobi / SOR with inner PCG or stored
    // inverses, b = 0, p <= 6
#if DGMG_N <= 7
    if (mp.bvert) return cudaErrorNotSupported;
    if (a.inner == DGMG_INNER_DIRECT) return launch_inv<df, false>(mp, a, s);
    if (a.inner != DGMG_INNER_PCG) return cudaErrorNotSupported;
    return launch_smooth<df, false>(mp, a, s);
#else
    return cudaErrorNotSupported;
#endif
  }
  return smooth_t<double>(mp, a, s);
}

cudaError_t diag(const MeshParams& mp, double* d, cudaStream_t s) {
  const long long n = mp.ncell * N3;
  if (n == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((n + 127) / 128);
  if (mp.bvert)
    k_diag<true><<<grid, 128, 0, s>>>(mp, d);
  else
    k_diag_kron<<<grid, 128, 0, s>>>(mp, d);
  count_launch();
  return cudaGetLastError();
}

// kTCells cells per warp, 8 warps per block.
cudaError_t restrict_cells(const MeshParams& mp, const void* r, double* corners, bool fp32, cudaStream_t s) {
  if (mp.ncell == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((mp.ncell + 8 * kTCells - 1) / (8 * kTCells));
  if (fp32)
    k_restrict_cells<float><<<grid, 256, 0, s>>>(mp.ncell, (const float*)r, corners);
  else
    k_restrict_cells<double><<<grid, 256, 0, s>>>(mp.ncell, (const double*)r, corners);
  count_launch();
  return cudaGetLastError();
}

cudaError_t prolong_add(const MeshParams& mp, const double* uhat, void* u, bool fp32, cudaStream_t s) {
  if (mp.ncell == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((mp.ncell + 8 * kTCells - 1) / (8 * kTCells));
  if (fp32)
    k_prolong_add<float><<<grid, 256, 0, s>>>(mp, uhat, (float*)u);
  else
    k_prolong_add<double><<<grid, 256, 0, s>>>(mp, uhat, (double*)u);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- batched launchers
// One launch over the members of a batch (b = 0): member r gets
// ceil(ncell_r / cells per block) blocks; layouts and launch shapes of member 0.
inline void fill_blocks(BatchTable& bt, long long cells_per_block) {
  bt.block0[0] = 0;
  for (int r = 0; r < bt.k; ++r)
    bt.block0[r + 1] = bt.block0[r] + (unsigned)((bt.mp[r].ncell + cells_per_block - 1) / cells_per_block);
}

template <typename T, bool FULL, bool FAC>
cudaError_t launch_apply_batch_form(BatchTable& bt, cudaStream_t s) {
  constexpr int XT = FAC ? kFactorExtra : 0;
  const int wpb = pick_wpb(bt.mp[0].wpb_apply[prec_index<T>()], WarpMem<T>::bytes(4, XT));
  const size_t sm = wpb * WarpMem<T>::bytes(4, XT);
  auto k = k_apply_batch<T, FULL, false, FAC>;
  cudaError_t e = set_smem(k, sm);
  if (e != cudaSuccess) return e;
  fill_blocks(bt, (long long)wpb * CPW);
  if (bt.block0[bt.k] == 0) return cudaSuccess;
  k<<<bt.block0[bt.k], wpb * 32, sm, s>>>(bt);
  count_launch();
  return cudaGetLastError();
}

template <typename T, bool FULL>
cudaError_t apply_batch_t(BatchTable& bt, cudaStream_t s) {
  const int lay = bt.mp[0].lay_apply[prec_index<T>()];
#if DGMG_N <= 5
  if constexpr (std::is_same<T, float>::value) {
    if (lay == DGMG_LAYOUT_PLANE) {
      const size_t per = pl::warp_bytes(FULL);
      const int wpb = pick_wpb_max(bt.mp[0].wpb_apply[DGMG_FP32], per, 8);
      const size_t sm = wpb * per;
      auto k = k_apply_plane_batch<FULL>;
      cudaError_t e = set_smem(k, sm);
      if (e != cudaSuccess) return e;
      fill_blocks(bt, (long long)wpb * pl::PC);
      if (bt.block0[bt.k] == 0) return cudaSuccess;
      k<<<bt.block0[bt.k], wpb * 32, sm, s>>>(bt);
      count_launch();
      return cudaGetLastError();
    }
  }
#endif
  if (lay == DGMG_LAYOUT_LINE || lay == DGMG_LAYOUT_PLANE) return launch_apply_batch_form<T, FULL, false>(bt, s);
  return launch_apply_batch_form<T, FULL, true>(bt, s);
}

cudaError_t apply_batch(BatchTable& bt, int prec, bool full, cudaStream_t s) {
  if (bt.k <= 0) return cudaSuccess;
  for (int r = 0; r < bt.k; ++r)
    if (bt.mp[r].bvert) return cudaErrorNotSupported;
  if (prec == DGMG_FP32) return full ? apply_batch_t<float, true>(bt, s) : apply_batch_t<float, false>(bt, s);
  if (prec == DGMG_DF64) {
#if DGMG_N <= 7
    return full ? apply_batch_t<df, true>(bt, s) : apply_batch_t<df, false>(bt, s);
#else
    return cudaErrorNotSupported;
#endif
  }
  return full ? apply_batch_t<double, true>(bt, s) : apply_batch_t<double, false>(bt, s);
}

template <typename T, bool FAC>
cudaError_t launch_smooth_batch_form(BatchTable& bt, cudaStream_t s) {
  constexpr int XT = smooth_extra<false, FAC>();
  const int wpb = pick_wpb(bt.mp[0].wpb_smooth[prec_index<T>()], WarpMem<T>::bytes(6, XT));
  const size_t sm = wpb * WarpMem<T>::bytes(6, XT);
  auto k = k_smooth_pcg_batch<T, false, FAC>;
  cudaError_t e = set_smem(k, sm);
  if (e != cudaSuccess) return e;
  fill_blocks(bt, (long long)wpb * CPW);
  if (bt.block0[bt.k] == 0) return cudaSuccess;
  k<<<bt.block0[bt.k], wpb * 32, sm, s>>>(bt);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
cudaError_t smooth_batch_t(BatchTable& bt, cudaStream_t s) {
  const int lay = bt.mp[0].lay_smooth[prec_index<T>()];
#if DGMG_N <= 5
  if constexpr (std::is_same<T, float>::value) {
    if (lay == DGMG_LAYOUT_PLANE) {
      const size_t per = pl::warp_bytes(true);
      const int wpb = pick_wpb_max(bt.mp[0].wpb_smooth[DGMG_FP32], per, 4);
      const size_t sm = wpb * per;
      cudaError_t e = set_smem(k_smooth_plane_batch, sm);
      if (e != cudaSuccess) return e;
      fill_blocks(bt, (long long)wpb * pl::PC);
      if (bt.block0[bt.k] == 0) return cudaSuccess;
      k_smooth_plane_batch<<<bt.block0[bt.k], wpb * 32, sm, s>>>(bt);
      count_launch();
      return cudaGetLastError();
    }
  }
#endif
  if (lay == DGMG_LAYOUT_LINE || lay == DGMG_LAYOUT_PLANE) return launch_smooth_batch_form<T, false>(bt, s);
  return launch_smooth_batch_form<T, true>(bt, s);
}

cudaError_t smooth_batch(BatchTable& bt, int prec, cudaStream_t s) {
  if (bt.k <= 0) return cudaSuccess;
  for (int r = 0; r < bt.k; ++r)
    if (bt.mp[r].bvert) return cudaErrorNotSupported;
  if (prec == DGMG_FP32) return smooth_batch_t<float>(bt, s);
  if (prec == DGMG_DF64) {
#if DGMG_N <= 7
    return smooth_batch_t<df>(bt, s);
#else
    return cudaErrorNotSupported;
#endif
  }
  return smooth_batch_t<double>(bt, s);
}

cudaError_t restrict_batch(BatchTable& bt, bool fp32, cudaStream_t s) {
  if (bt.k <= 0) return cudaSuccess;
  fill_blocks(bt, 8 * kTCells);   // kTCells cells per warp, 8 warps per block
  if (bt.block0[bt.k] == 0) return cudaSuccess;
  if (fp32)
    k_restrict_cells_batch<float><<<bt.block0[bt.k], 256, 0, s>>>(bt);
  else
    k_restrict_cells_batch<double><<<bt.block0[bt.k], 256, 0, s>>>(bt);
  count_launch();
  return cudaGetLastError();
}

cudaError_t prolong_batch(BatchTable& bt, bool fp32, cudaStream_t s) {
  if (bt.k <= 0) return cudaSuccess;
  fill_blocks(bt, 8 * kTCells);
  if (bt.block0[bt.k] == 0) return cudaSuccess;
  if (fp32)
    k_prolong_add_batch<float><<<bt.block0[bt.k], 256, 0, s>>>(bt);
  else
    k_prolong_add_batch<double><<<bt.block0[bt.k], 256, 0, s>>>(bt);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

#define DGMG_CAT2(a, b) a##b
#define DGMG_CAT(a, b) DGMG_CAT2(a, b)

const CellOps* DGMG_CAT(cell_ops_n, DGMG_N)() {
  static const CellOps ops = {N, &upload_tables, &apply, &smooth, &diag, &restrict_cells, &prolong_add,
                              &block_matrix, &block_tridiag, &apply_var, &apply_batch, &smooth_batch,
                              &restrict_batch, &prolong_batch};
  return &ops;
}

}  // namespace dgmg
