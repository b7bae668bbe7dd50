// Vector kernels of the outer Krylov solvers (FP64 dots with a fixed
// reduction order, axpby, precision conversion) and the sparse kernels of the
// aggregation-AMG cycle on the Q1 coarse space: 27-point stencil residual and
// damped Jacobi, 2x2x2 aggregate restriction / prolongation, the dense
// coarsest-level solve, and the vertex gather of the DG -> Q1 restriction.
#include <cuda_runtime.h>

#include "dgmg_internal.h"

namespace dgmg {
namespace {

constexpr int kThreads = 256;

inline unsigned grid1(long long n, int per = kThreads) {
  long long g = (n + per - 1) / per;
  if (g > 152LL * 64) g = 152LL * 64;     // grid-stride beyond 64 blocks per SM
  return (unsigned)(g > 0 ? g : 1);
}

// a x + b y as fma(a, x, round(b y)) in every kernel that updates a Krylov
// vector, so batched and single solves agree bit for bit: the product b y is
// rounded on its own (__dmul_rn / __fmul_rn are never contracted), also where
// a is the constant 1 and the compiler could otherwise fuse b y with x.
__device__ __forceinline__ double axpby_op(double a, double x, double b, double y) {
  return fma(a, x, __dmul_rn(b, y));
}
__device__ __forceinline__ float axpby_op(float a, float x, float b, float y) {
  return fmaf(a, x, __fmul_rn(b, y));
}

template <typename T>
__global__ void k_axpby(long long n, T a, const T* __restrict__ x, T b, T* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = axpby_op(a, x[i], b, y[i]);
}

template <typename T>
__global__ void k_sub(long long n, const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

template <typename T>
__global__ void k_fill(long long n, T v, T* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = v;
}

template <typename A, typename B>
__global__ void k_convert(long long n, const A* __restrict__ x, B* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = (B)x[i];
}

// Block-level sum in a fixed tree order.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  return sh[0];
}

// Stage 1 of a dot: kDotBlocks blocks, block b sums indices b*chunk + ...
// in a fixed order independent of timing.  k vectors xs[0..k) against y.
__global__ void k_dot_partial(long long n, int k, const double* const* __restrict__ xs, const double* __restrict__ x1,
                              const double* __restrict__ y, double* __restrict__ partial) {
  __shared__ double sh[kThreads];
  const long long chunk = (n + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  for (int j = 0; j < k; ++j) {
    const double* x = xs ? xs[j] : x1;
    double s = 0.0;
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s = fma(x[i], y[i], s);
    const double tot = block_sum(s, sh);
    if (threadIdx.x == 0) partial[(long long)j * gridDim.x + blockIdx.x] = tot;
    __syncthreads();
  }
}

__global__ void k_dot_final(int nblocks, int k, const double* __restrict__ partial, double* __restrict__ out) {
  __shared__ double sh[kThreads];
  for (int j = 0; j < k; ++j) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) s += partial[(long long)j * nblocks + i];
    const double tot = block_sum(s, sh);
    if (threadIdx.x == 0) out[j] = tot;
    __syncthreads();
  }
}

// 27-point stencil helpers: row v of a (vx, vy, vz) vertex grid.
__device__ __forceinline__ double stencil_row(int vx, int vy, int vz, const double* __restrict__ st,
                                              const double* __restrict__ x, long long v) {
  const int ix = (int)(v % vx);
  const long long t = v / vx;
  const int iy = (int)(t % vy), iz = (int)(t / vy);
  const double* a = st + 27 * v;
  double s = 0.0;
  for (int dz = -1; dz <= 1; ++dz) {
    const int z = iz + dz;
    if (z < 0 || z >= vz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int y = iy + dy;
      if (y < 0 || y >= vy) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int xx = ix + dx;
        if (xx < 0 || xx >= vx) continue;
        s = fma(a[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)], x[xx + (long long)vx * (y + (long long)vy * z)], s);
      }
    }
  }
  return s;
}

__global__ void k_stencil_jacobi(int vx, int vy, int vz, const double* __restrict__ st, const double* __restrict__ dinv,
                                 const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ xo,
                                 double omega, bool zero_x) {
  const long long n = (long long)vx * vy * vz;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    if (zero_x)
      xo[v] = omega * dinv[v] * b[v];
    else
      xo[v] = x[v] + omega * dinv[v] * (b[v] - stencil_row(vx, vy, vz, st, x, v));
  }
}

__global__ void k_stencil_residual(int vx, int vy, int vz, const double* __restrict__ st, const double* __restrict__ b,
                                   const double* __restrict__ x, double* __restrict__ r) {
  const long long n = (long long)vx * vy * vz;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x)
    r[v] = b[v] - stencil_row(vx, vy, vz, st, x, v);
}

// rc[I] = sum of r over the (up to) 8 fine vertices of aggregate I, fixed order.
__global__ void k_agg_restrict(int vx, int vy, int vz, const double* __restrict__ r, double* __restrict__ rc) {
  const int cx = (vx + 1) / 2, cy = (vy + 1) / 2, cz = (vz + 1) / 2;
  const long long n = (long long)cx * cy * cz;
  for (long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x; I < n; I += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(I % cx);
    const long long t = I / cx;
    const int iy = (int)(t % cy), iz = (int)(t / cy);
    double s = 0.0;
    for (int oz = 0; oz < 2; ++oz) {
      const int z = 2 * iz + oz;
      if (z >= vz) continue;
      for (int oy = 0; oy < 2; ++oy) {
        const int y = 2 * iy + oy;
        if (y >= vy) continue;
        for (int ox = 0; ox < 2; ++ox) {
          const int x = 2 * ix + ox;
          if (x >= vx) continue;
          s += r[x + (long long)vx * (y + (long long)vy * z)];
        }
      }
    }
    rc[I] = s;
  }
}

__global__ void k_agg_prolong_add(int vx, int vy, int vz, const double* __restrict__ xc, double* __restrict__ x) {
  const int cx = (vx + 1) / 2, cy = (vy + 1) / 2;
  const long long n = (long long)vx * vy * vz;
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(v % vx);
    const long long t = v / vx;
    const int iy = (int)(t % vy), iz = (int)(t / vy);
    x[v] += xc[(ix / 2) + (long long)cx * ((iy / 2) + (long long)cy * (iz / 2))];
  }
}

// y = A x, A dense n x n row-major; one warp per row.
__global__ void k_dense_matvec(int n, const double* __restrict__ A, const double* __restrict__ x, double* __restrict__ y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  double s = 0.0;
  for (int j = lane; j < n; j += 32) s = fma(A[(long long)warp * n + j], x[j], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[warp] = s;
}

// r_hat(v) = sum over the cells around vertex v (fixed order) of their corner
// sums for the corner at v.
__global__ void k_restrict_gather(int nx, int ny, int nz, const double* __restrict__ corners, double* __restrict__ rhat) {
  const int vx = nx + 1, vy = ny + 1;
  const long long n = (long long)vx * vy * (nz + 1);
  for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n; v += (long long)gridDim.x * blockDim.x) {
    const int ix = (int)(v % vx);
    const long long t = v / vx;
    const int iy = (int)(t % vy), iz = (int)(t / vy);
    double s = 0.0;
    for (int az = 0; az < 2; ++az) {
      const int cz = iz - 1 + az;
      if (cz < 0 || cz >= nz) continue;
      for (int ay = 0; ay < 2; ++ay) {
        const int cy = iy - 1 + ay;
        if (cy < 0 || cy >= ny) continue;
        for (int ax = 0; ax < 2; ++ax) {
          const int cx = ix - 1 + ax;
          if (cx < 0 || cx >= nx) continue;
          const long long c = cx + (long long)nx * (cy + (long long)ny * cz);
          const int corner = (1 - ax) + 2 * (1 - ay) + 4 * (1 - az);
          s += corners[8 * c + corner];
        }
      }
    }
    rhat[v] = s;
  }
}

// ------------------------------------------------------------- batched Krylov kernels
__device__ __forceinline__ int seg_member(const SegTable& t, unsigned bid) {
  int r = 0;
  while (r + 1 < t.k && bid >= t.block0[r + 1]) ++r;
  return r;
}

template <int OP>
__global__ void k_seg(const __grid_constant__ SegTable t) {
  const int r = seg_member(t, blockIdx.x);
  const long long n = t.n[r];
  const long long stride = (long long)(t.block0[r + 1] - t.block0[r]) * blockDim.x;
  const long long i0 = (long long)(blockIdx.x - t.block0[r]) * blockDim.x + threadIdx.x;
  if (OP == SEG_ALPHA) {
    const double alpha = t.sc[r][kScAlpha];
    const bool flex = t.sc[r][kScFlex] != 0.0;
    const double* p = (const double*)t.a[r];
    const double* q = (const double*)t.b[r];
    double* u = (double*)t.c[r];
    double* rv = (double*)t.d[r];
    double* ro = (double*)t.e[r];
    for (long long i = i0; i < n; i += stride) {
      u[i] = axpby_op(alpha, p[i], 1.0, u[i]);
      if (flex) ro[i] = rv[i];
      rv[i] = axpby_op(-alpha, q[i], 1.0, rv[i]);
    }
  } else if (OP == SEG_P) {
    const double beta = t.sc[r][kScBeta];
    const double* z = (const double*)t.a[r];
    double* p = (double*)t.c[r];
    for (long long i = i0; i < n; i += stride) p[i] = axpby_op(1.0, z[i], beta, p[i]);
  } else {
    for (long long i = i0; i < n; i += stride) {
      if (OP == SEG_D2F) ((float*)t.c[r])[i] = (float)((const double*)t.a[r])[i];
      if (OP == SEG_F2D) ((double*)t.c[r])[i] = (double)((const float*)t.a[r])[i];
      if (OP == SEG_COPY64) ((double*)t.c[r])[i] = ((const double*)t.a[r])[i];
      if (OP == SEG_COPY32) ((float*)t.c[r])[i] = ((const float*)t.a[r])[i];
      if (OP == SEG_SUB64) ((double*)t.c[r])[i] = ((const double*)t.a[r])[i] - ((const double*)t.b[r])[i];
      if (OP == SEG_SUB32) ((float*)t.c[r])[i] = ((const float*)t.a[r])[i] - ((const float*)t.b[r])[i];
    }
  }
}

// Stage 1 of the members' dots: kDotBlocks blocks per member, block b of
// member r sums its chunk exactly as k_dot_partial does with kDotBlocks blocks.
__global__ void k_seg_dot_partial(const __grid_constant__ SegTable t, double* __restrict__ partial) {
  __shared__ double sh[kThreads];
  const int r = blockIdx.x / kDotBlocks;
  const int b = blockIdx.x - r * kDotBlocks;
  const long long n = t.n[r];
  const long long chunk = (n + kDotBlocks - 1) / kDotBlocks;
  const long long lo = b * chunk;
  const long long hi = lo + chunk < n ? lo + chunk : n;
  const double* x = (const double*)t.a[r];
  const double* y = (const double*)t.b[r];
  double s = 0.0;
  for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) s = fma(x[i], y[i], s);
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) partial[(long long)r * kDotBlocks + b] = tot;
}

__global__ void k_seg_dot_final(const __grid_constant__ SegTable t, const double* __restrict__ partial, int slot) {
  __shared__ double sh[kThreads];
  const int r = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < kDotBlocks; i += blockDim.x) s += partial[(long long)r * kDotBlocks + i];
  const double tot = block_sum(s, sh);
  if (threadIdx.x == 0) t.sc[r][slot] = tot;
}

// The scalar steps of the members' CG iterations (one thread per member), the
// same arithmetic as the host loop of the single solve.
template <int OP>
__global__ void k_seg_scalar(const __grid_constant__ SegTable t) {
  const int r = threadIdx.x;
  if (r >= t.k) return;
  double* c = t.sc[r];
  const bool stopped = c[kScDone] != 0.0;
  if (OP == SC_ALPHA) {
    if (stopped) {
      c[kScAlpha] = 0.0;
    } else if (!(c[kScPq] > 0.0)) {
      c[kScAlpha] = 0.0;
      c[kScDone] = 2.0;
    } else {
      c[kScAlpha] = c[kScRz] / c[kScPq];
    }
  } else if (OP == SC_CONV) {
    if (!stopped) {
      c[kScIts] += 1.0;
      if (sqrt(c[kScRr]) <= c[kScRtol] * c[kScR0])
        c[kScDone] = 1.0;
      else if (c[kScIts] >= c[kScMaxit])
        c[kScDone] = 3.0;
    }
  } else {
    if (stopped) {
      c[kScBeta] = 0.0;
    } else {
      const double num = c[kScFlex] != 0.0 ? c[kScRzn] - c[kScZro] : c[kScRzn];
      c[kScBeta] = num / c[kScRz];
      c[kScRz] = c[kScRzn];
    }
  }
}

// The same Gauss-Jordan elimination for blocks too large for shared memory
// (nb > kInvMaxN, p >= 5): the block stays in global memory (column-major,
// column stride ld) and the pivot steps are taken in panels of kPanel
// columns.  A panel's columns are eliminated in shared memory step by step
// (pivot search, row swap, scaling, elimination of every other row); the
// steps' pivot rows, reciprocal pivots and pivot columns are kept, and then
// every column outside the panel receives the same swaps and eliminations in
// the same order, one warp per column held in registers.  Each element sees
// the same sequence of operations as in k_block_invert, so the inverse is the
// same, while the block is read and written once per panel instead of once
// per pivot step.  One thread block per cell; nb <= kInvMaxBig.
constexpr int kPanel = 16;
constexpr int kInvMaxBig = 736;                 // n^3 up to p = 8 (729), rounded to 32
constexpr int kColRegs = kInvMaxBig / 32;

__global__ void __launch_bounds__(256) k_block_invert_big(double* __restrict__ a, int nb, int ld, long long ncell,
                                                           int* __restrict__ singular) {
  extern __shared__ __align__(16) double sm_big[];
  double* P = sm_big;                    // panel: nb x kPanel, column-major
  double* L = P + (size_t)nb * kPanel;   // pivot columns before elimination: kPanel x nb
  __shared__ double pinv_s[kPanel];
  __shared__ int prow_s[kPanel];
  __shared__ int perm[kInvMaxBig];
  __shared__ double wv[8];
  __shared__ int wi[8];
  __shared__ int bad;
  const long long c = blockIdx.x;
  if (c >= ncell) return;
  double* g = a + c * (long long)nb * ld;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  if (tid == 0) bad = 0;
  for (int k0 = 0; k0 < nb; k0 += kPanel) {
    const int kb = nb - k0 < kPanel ? nb - k0 : kPanel;
    for (int t = tid; t < nb * kb; t += nt) P[t] = g[(t % nb) + (long long)(k0 + t / nb) * ld];
    __syncthreads();
    for (int kk = 0; kk < kb; ++kk) {
      const int k = k0 + kk;
      double best = -1.0;
      int bi = nb;
      for (int i = k + tid; i < nb; i += nt) {
        const double v = fabs(P[i + kk * nb]);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        wv[warp] = best;
        wi[warp] = bi;
      }
      __syncthreads();
      if (tid == 0) {
        double b = wv[0];
        int r = wi[0];
        for (int w = 1; w < nw; ++w)
          if (wv[w] > b || (wv[w] == b && wi[w] < r)) {
            b = wv[w];
            r = wi[w];
          }
        if (r >= nb) r = k;
        prow_s[kk] = r;
        perm[k] = r;
      }
      __syncthreads();
      const int p = prow_s[kk];
      if (p != k)
        for (int j = tid; j < kb; j += nt) {
          const double t = P[k + j * nb];
          P[k + j * nb] = P[p + j * nb];
          P[p + j * nb] = t;
        }
      __syncthreads();
      const double piv = P[k + kk * nb];
      if (piv == 0.0 || !isfinite(piv)) {
        if (tid == 0) *singular = 1;
        return;
      }
      const double pv = 1.0 / piv;
      if (tid == 0) pinv_s[kk] = pv;
      for (int i = tid; i < nb; i += nt) L[kk * nb + i] = P[i + kk * nb];
      __syncthreads();
      for (int j = tid; j < kb; j += nt) P[k + j * nb] = (j == kk ? 1.0 : P[k + j * nb]) * pv;
      __syncthreads();
      for (int t = tid; t < nb * kb; t += nt) {
        const int i = t % nb, j = t / nb;
        if (i == k) continue;
        P[t] = fma(-L[kk * nb + i], P[k + j * nb], j == kk ? 0.0 : P[t]);
      }
      __syncthreads();
    }
    for (int t = tid; t < nb * kb; t += nt) g[(t % nb) + (long long)(k0 + t / nb) * ld] = P[t];
    // the panel's steps on every other column, one warp per column
    for (int j = warp; j < nb; j += nw) {
      if (j >= k0 && j < k0 + kb) continue;
      double* col = g + (long long)j * ld;
      double x[kColRegs];
#pragma unroll
      for (int r = 0; r < kColRegs; ++r) {
        const int i = lane + 32 * r;
        x[r] = i < nb ? col[i] : 0.0;
      }
      for (int kk = 0; kk < kb; ++kk) {
        const int k = k0 + kk, p = prow_s[kk];
        // values at rows k and p (each held by one lane), swapped
        double xk = 0.0, xp = 0.0;
#pragma unroll
        for (int r = 0; r < kColRegs; ++r) {
          if (lane + 32 * r == k) xk = x[r];
          if (lane + 32 * r == p) xp = x[r];
        }
        xk = __shfl_sync(0xffffffffu, xk, k & 31);
        xp = __shfl_sync(0xffffffffu, xp, p & 31);
        if (p != k) {
#pragma unroll
          for (int r = 0; r < kColRegs; ++r) {
            if (lane + 32 * r == k) x[r] = xp;
            if (lane + 32 * r == p) x[r] = xk;
          }
        }
        const double rk = xp * pinv_s[kk];   // row k after the swap, scaled
#pragma unroll
        for (int r = 0; r < kColRegs; ++r) {
          const int i = lane + 32 * r;
          if (i < nb) x[r] = i == k ? rk : fma(-L[kk * nb + i], rk, x[r]);
        }
      }
#pragma unroll
      for (int r = 0; r < kColRegs; ++r) {
        const int i = lane + 32 * r;
        if (i < nb) col[i] = x[r];
      }
    }
    __syncthreads();
  }
  for (int k = nb - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = tid; i < nb; i += nt) {
        const double t = g[i + (long long)k * ld];
        g[i + (long long)k * ld] = g[i + (long long)p * ld];
        g[i + (long long)p * ld] = t;
      }
    __syncthreads();
  }
}

// Per-cell coefficient records (setup): kd[3], cJ, kap[6], gam[6].
__global__ void k_cell_records(MeshParams mp, double* __restrict__ r64, float* __restrict__ r32) {
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c >= mp.ncell) return;
  const int cx = (int)(c % mp.nx);
  const int cy = (int)((c / mp.nx) % mp.ny);
  const int cz = (int)(c / ((long long)mp.nx * mp.ny));
  const int ci[3] = {cx, cy, cz};
  const int nn[3] = {mp.nx, mp.ny, mp.nz};
  const long long stride[3] = {1, mp.nx, (long long)mp.nx * mp.ny};
  const double J = mp.h[0] * mp.h[1] * mp.h[2];
  const double pen = mp.alpha * mp.p * (mp.p + 2);
  double rec[kRecLen];
  auto K = [&](long long cell, int d) { return mp.K[cell * mp.kdim + (mp.kdim == 3 ? d : 0)]; };
  for (int d = 0; d < 3; ++d) rec[kRecKd + d] = J * K(c, d) / (mp.h[d] * mp.h[d]);
  rec[kRecCJ] = mp.c ? J * mp.c[c] : 0.0;
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) {
      const bool bnd = (s == 0 && ci[d] == 0) || (s == 1 && ci[d] == nn[d] - 1);
      const double kin = K(c, d);
      double kap = 0.0, gam = 0.0;
      if (!bnd) {
        const double kout = K(s ? c + stride[d] : c - stride[d], d);
        kap = kin * kout / (kin + kout);
        gam = 2.0 * pen * kap / mp.h[d];
      } else if (mp.bc[2 * d + s] == 0) {
        kap = kin;
        gam = pen * kap / mp.h[d];
      }
      rec[kRecKap + 2 * d + s] = kap;
      rec[kRecGam + 2 * d + s] = gam;
    }
  for (int k = 0; k < kRecLen; ++k) {
    r64[c * kRecLen + k] = rec[k];
    r32[c * kRecLen + k] = (float)rec[k];
  }
}

__global__ void k_inverse(long long n, const double* __restrict__ d, double* __restrict__ i64, float* __restrict__ i32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = 1.0 / d[i];
    i64[i] = v;
    i32[i] = (float)v;
  }
}

// Gauss-Jordan inversion in place with partial pivoting, one thread block per
// dense block, the block held in shared memory (column-major M[i + j nb]).
// Step k: pick the row p >= k with the largest |M[p][k]| (ties: smallest p),
// swap rows k and p, scale row k by 1 / M[k][k] with M[k][k] <- 1 first, and
// for every other row i subtract M[i][k] times row k, with M[i][k] <- 0 first;
// column k then holds the k-th column of the inverse of the eliminated matrix.
// The row interchanges are undone at the end as column interchanges in reverse
// order.
constexpr int kInvMaxN = 128;


__global__ void __launch_bounds__(256) k_block_invert(double* __restrict__ a, int nb, int ld, long long ncell,
                                                       int* __restrict__ singular) {
  extern __shared__ __align__(16) double sm_inv[];
  __shared__ int perm[kInvMaxN];
  __shared__ double wv[8];
  __shared__ int wi[8];
  __shared__ int piv_row;
  const long long c = blockIdx.x;
  if (c >= ncell) return;
  double* M = sm_inv;
  double* colk = M + nb * nb;
  double* rowk = colk + nb;
  double* g = a + c * (long long)nb * ld;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  for (int t = tid; t < nb * nb; t += nt) M[t] = g[(t % nb) + (long long)(t / nb) * ld];
  __syncthreads();
  for (int k = 0; k < nb; ++k) {
    double best = -1.0;
    int bi = nb;
    for (int i = k + tid; i < nb; i += nt) {
      const double v = fabs(M[i + k * nb]);
      if (v > best) {
        best = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) {
        best = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      wv[warp] = best;
      wi[warp] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double b = wv[0];
      int r = wi[0];
      for (int w = 1; w < nt / 32; ++w)
        if (wv[w] > b || (wv[w] == b && wi[w] < r)) {
          b = wv[w];
          r = wi[w];
        }
      if (r >= nb) r = k;   // no finite candidate: the pivot test below rejects the block
      piv_row = r;
      perm[k] = r;
    }
    __syncthreads();
    const int p = piv_row;
    if (p != k)
      for (int j = tid; j < nb; j += nt) {
        const double t = M[k + j * nb];
        M[k + j * nb] = M[p + j * nb];
        M[p + j * nb] = t;
      }
    __syncthreads();
    const double piv = M[k + k * nb];
    if (piv == 0.0 || !isfinite(piv)) {   // the same shared value for every thread
      if (tid == 0) *singular = 1;
      return;
    }
    const double pinv = 1.0 / piv;
    for (int i = tid; i < nb; i += nt) colk[i] = M[i + k * nb];
    __syncthreads();
    for (int j = tid; j < nb; j += nt) {
      const double v = (j == k ? 1.0 : M[k + j * nb]) * pinv;
      M[k + j * nb] = v;
      rowk[j] = v;
    }
    __syncthreads();
    for (int t = tid; t < nb * nb; t += nt) {
      const int i = t % nb, j = t / nb;
      if (i == k) continue;
      M[t] = fma(-colk[i], rowk[j], j == k ? 0.0 : M[t]);
    }
    __syncthreads();
  }
  for (int k = nb - 1; k >= 0; --k) {
    const int p = perm[k];
    if (p != k)
      for (int i = tid; i < nb; i += nt) {
        const double t = M[i + k * nb];
        M[i + k * nb] = M[i + p * nb];
        M[i + p * nb] = t;
      }
    __syncthreads();
  }
  for (int t = tid; t < nb * nb; t += nt) g[(t % nb) + (long long)(t / nb) * ld] = M[t];
}

__global__ void k_split_df(long long n, const double* __restrict__ x, float2* __restrict__ pairs,
                           float* __restrict__ f32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double v = x[i];
    const float h = (float)v;
    pairs[i] = make_float2(h, (float)(v - (double)h));
    if (f32) f32[i] = h;
  }
}

__global__ void k_df_to_dense(long long ncell, int nb, int ld, const float2* __restrict__ pairs,
                              double* __restrict__ out) {
  const long long n = ncell * nb * nb;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    const long long col = t / nb;              // cell * nb + j
    const int i = (int)(t - col * nb);
    const float2 p = pairs[col * ld + i];
    out[t] = (double)p.x + (double)p.y;
  }
}

// P0 restriction: out[c] = sum of cell c's n3 values, one warp per cell, lanes
// stride the cell, then a fixed shuffle tree (deterministic order).
template <typename T>
__global__ void k_cell_sums(long long ncell, int n3, const T* __restrict__ r, double* __restrict__ out) {
  const long long c = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= ncell) return;
  const T* rc = r + c * n3;
  double s = 0.0;
  for (int i = lane; i < n3; i += 32) s += (double)rc[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[c] = s;
}

// P0 prolongation: u[c n3 + i] += uhat[c].
template <typename T>
__global__ void k_cell_add(long long ncell, int n3, const double* __restrict__ uhat, T* __restrict__ u) {
  const long long n = ncell * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    u[i] = (T)((double)u[i] + uhat[i / n3]);
}

}  // namespace

cudaError_t cell_records(const MeshParams& mp, double* rec64, float* rec32, cudaStream_t s) {
  if (mp.ncell == 0) return cudaSuccess;
  k_cell_records<<<(unsigned)((mp.ncell + 127) / 128), 128, 0, s>>>(mp, rec64, rec32);
  count_launch();
  return cudaGetLastError();
}

cudaError_t vec_inverse(long long n, const double* d, double* i64, float* i32, cudaStream_t s) {
  k_inverse<<<grid1(n), kThreads, 0, s>>>(n, d, i64, i32);
  count_launch();
  return cudaGetLastError();
}

cudaError_t cell_sums(long long ncell, int n3, const void* r, double* out, bool fp32, cudaStream_t s) {
  if (ncell == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((ncell * 32 + 255) / 256);
  if (fp32)
    k_cell_sums<float><<<grid, 256, 0, s>>>(ncell, n3, (const float*)r, out);
  else
    k_cell_sums<double><<<grid, 256, 0, s>>>(ncell, n3, (const double*)r, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t cell_add(long long ncell, int n3, const double* uhat, void* u, bool fp32, cudaStream_t s) {
  if (ncell == 0) return cudaSuccess;
  const long long n = ncell * n3;
  if (fp32)
    k_cell_add<float><<<grid1(n), kThreads, 0, s>>>(ncell, n3, uhat, (float*)u);
  else
    k_cell_add<double><<<grid1(n), kThreads, 0, s>>>(ncell, n3, uhat, (double*)u);
  count_launch();
  return cudaGetLastError();
}

cudaError_t vec_split_df(long long n, const double* x, float2* pairs, float* f32, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  k_split_df<<<grid1(n), kThreads, 0, s>>>(n, x, pairs, f32);
  count_launch();
  return cudaGetLastError();
}

cudaError_t blocks_df_to_dense(long long ncell, int nb, int ld, const float2* pairs, double* out, cudaStream_t s) {
  const long long n = ncell * nb * nb;
  if (n == 0) return cudaSuccess;
  k_df_to_dense<<<grid1(n), kThreads, 0, s>>>(ncell, nb, ld, pairs, out);
  count_launch();
  return cudaGetLastError();
}

cudaError_t block_invert(double* a, int nb, int ld, long long ncell, int* singular, cudaStream_t s) {
  if (ncell == 0) return cudaSuccess;
  if (nb > kInvMaxN && nb <= kInvMaxBig) {
    if (ncell > 0x7fffffffLL || ld < nb) return cudaErrorInvalidValue;
    const size_t smem = (size_t)2 * nb * kPanel * sizeof(double);
    if (smem > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k_block_invert_big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
    }
    k_block_invert_big<<<(unsigned)ncell, 256, smem, s>>>(a, nb, ld, ncell, singular);
    count_launch();
    return cudaGetLastError();
  }
  if (nb < 1 || nb > kInvMaxN) return cudaErrorInvalidValue;
  const size_t smem = ((size_t)nb * nb + 2 * nb) * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_block_invert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  if (ncell > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (ld < nb) return cudaErrorInvalidValue;
  k_block_invert<<<(unsigned)ncell, nb >= 64 ? 256 : 128, smem, s>>>(a, nb, ld, ncell, singular);
  count_launch();
  return cudaGetLastError();
}

cudaError_t vec_axpby(long long n, double a, const double* x, double b, double* y, cudaStream_t s) {
  k_axpby<double><<<grid1(n), kThreads, 0, s>>>(n, a, x, b, y);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_axpby_f(long long n, float a, const float* x, float b, float* y, cudaStream_t s) {
  k_axpby<float><<<grid1(n), kThreads, 0, s>>>(n, a, x, b, y);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_sub(long long n, const double* a, const double* b, double* out, cudaStream_t s) {
  k_sub<double><<<grid1(n), kThreads, 0, s>>>(n, a, b, out);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_sub_f(long long n, const float* a, const float* b, float* out, cudaStream_t s) {
  k_sub<float><<<grid1(n), kThreads, 0, s>>>(n, a, b, out);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_copy(long long n, const double* x, double* y, cudaStream_t s) {
  return cudaMemcpyAsync(y, x, n * sizeof(double), cudaMemcpyDeviceToDevice, s);
}
cudaError_t vec_fill(long long n, double v, double* y, cudaStream_t s) {
  k_fill<double><<<grid1(n), kThreads, 0, s>>>(n, v, y);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_fill_f(long long n, float v, float* y, cudaStream_t s) {
  k_fill<float><<<grid1(n), kThreads, 0, s>>>(n, v, y);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_d2f(long long n, const double* x, float* y, cudaStream_t s) {
  k_convert<double, float><<<grid1(n), kThreads, 0, s>>>(n, x, y);
  count_launch();
  return cudaGetLastError();
}
cudaError_t vec_f2d(long long n, const float* x, double* y, cudaStream_t s) {
  k_convert<float, double><<<grid1(n), kThreads, 0, s>>>(n, x, y);
  count_launch();
  return cudaGetLastError();
}
// Elementwise launches over the members: about a thread per element, at most
// 64 blocks per SM in all.
cudaError_t seg_op(int op, SegTable& t, cudaStream_t s) {
  if (t.k <= 0) return cudaSuccess;
  const long long cap = 152LL * 64;
  long long tb = 0;
  for (int r = 0; r < t.k; ++r) tb += (t.n[r] + kThreads - 1) / kThreads;
  t.block0[0] = 0;
  for (int r = 0; r < t.k; ++r) {
    long long b = (t.n[r] + kThreads - 1) / kThreads;
    if (tb > cap) b = b * cap / tb;
    if (b < 1) b = 1;
    t.block0[r + 1] = t.block0[r] + (unsigned)b;
  }
  const unsigned g = t.block0[t.k];
  switch (op) {
    case SEG_D2F: k_seg<SEG_D2F><<<g, kThreads, 0, s>>>(t); break;
    case SEG_F2D: k_seg<SEG_F2D><<<g, kThreads, 0, s>>>(t); break;
    case SEG_COPY64: k_seg<SEG_COPY64><<<g, kThreads, 0, s>>>(t); break;
    case SEG_COPY32: k_seg<SEG_COPY32><<<g, kThreads, 0, s>>>(t); break;
    case SEG_SUB64: k_seg<SEG_SUB64><<<g, kThreads, 0, s>>>(t); break;
    case SEG_SUB32: k_seg<SEG_SUB32><<<g, kThreads, 0, s>>>(t); break;
    case SEG_ALPHA: k_seg<SEG_ALPHA><<<g, kThreads, 0, s>>>(t); break;
    case SEG_P: k_seg<SEG_P><<<g, kThreads, 0, s>>>(t); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t seg_dot(SegTable& t, double* partial, int slot, cudaStream_t s) {
  if (t.k <= 0) return cudaSuccess;
  k_seg_dot_partial<<<t.k * kDotBlocks, kThreads, 0, s>>>(t, partial);
  k_seg_dot_final<<<t.k, kThreads, 0, s>>>(t, partial, slot);
  count_launch(2);
  return cudaGetLastError();
}

cudaError_t seg_scalar(int op, SegTable& t, cudaStream_t s) {
  if (t.k <= 0) return cudaSuccess;
  switch (op) {
    case SC_ALPHA: k_seg_scalar<SC_ALPHA><<<1, 32, 0, s>>>(t); break;
    case SC_CONV: k_seg_scalar<SC_CONV><<<1, 32, 0, s>>>(t); break;
    case SC_BETA: k_seg_scalar<SC_BETA><<<1, 32, 0, s>>>(t); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t vec_dot(long long n, const double* x, const double* y, double* partial, double* out, cudaStream_t s) {
  k_dot_partial<<<kDotBlocks, kThreads, 0, s>>>(n, 1, nullptr, x, y, partial);
  k_dot_final<<<1, kThreads, 0, s>>>(kDotBlocks, 1, partial, out);
  count_launch(2);
  return cudaGetLastError();
}
cudaError_t vec_multi_dot(long long n, int k, const double* const* xs, const double* y, double* partial, double* out,
                          cudaStream_t s) {
  k_dot_partial<<<kDotBlocks, kThreads, 0, s>>>(n, k, xs, nullptr, y, partial);
  k_dot_final<<<1, kThreads, 0, s>>>(kDotBlocks, k, partial, out);
  count_launch(2);
  return cudaGetLastError();
}
cudaError_t stencil_jacobi(int vx, int vy, int vz, const double* st, const double* dinv, const double* b,
                           const double* x, double* xout, double omega, bool zero_x, cudaStream_t s) {
  k_stencil_jacobi<<<grid1((long long)vx * vy * vz), kThreads, 0, s>>>(vx, vy, vz, st, dinv, b, x, xout, omega, zero_x);
  count_launch();
  return cudaGetLastError();
}
cudaError_t stencil_residual(int vx, int vy, int vz, const double* st, const double* b, const double* x, double* r,
                             cudaStream_t s) {
  k_stencil_residual<<<grid1((long long)vx * vy * vz), kThreads, 0, s>>>(vx, vy, vz, st, b, x, r);
  count_launch();
  return cudaGetLastError();
}
cudaError_t agg_restrict(int vx, int vy, int vz, const double* r, double* rc, cudaStream_t s) {
  const long long nc = (long long)((vx + 1) / 2) * ((vy + 1) / 2) * ((vz + 1) / 2);
  k_agg_restrict<<<grid1(nc), kThreads, 0, s>>>(vx, vy, vz, r, rc);
  count_launch();
  return cudaGetLastError();
}
cudaError_t agg_prolong_add(int vx, int vy, int vz, const double* xc, double* x, cudaStream_t s) {
  k_agg_prolong_add<<<grid1((long long)vx * vy * vz), kThreads, 0, s>>>(vx, vy, vz, xc, x);
  count_launch();
  return cudaGetLastError();
}
cudaError_t dense_matvec(int n, const double* A, const double* x, double* y, cudaStream_t s) {
  const int threads = 256;
  const unsigned blocks = (unsigned)(((long long)n * 32 + threads - 1) / threads);
  k_dense_matvec<<<blocks, threads, 0, s>>>(n, A, x, y);
  count_launch();
  return cudaGetLastError();
}
cudaError_t restrict_gather(int nx, int ny, int nz, const double* corners, double* rhat, cudaStream_t s) {
  k_restrict_gather<<<grid1((long long)(nx + 1) * (ny + 1) * (nz + 1)), kThreads, 0, s>>>(nx, ny, nz, corners, rhat);
  count_launch();
  return cudaGetLastError();
}

}  // namespace dgmg
