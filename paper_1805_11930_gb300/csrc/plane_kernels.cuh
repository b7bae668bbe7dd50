// Plane-per-lane FP32 kernels for n = p+1 <= 5 (b = 0): the operator and the
// block-Jacobi sweep with inner PCG.  Included by cell_kernels.cu inside its
// anonymous namespace (it uses the per-order tables and cell helpers there).
//
// The line form of cell_kernels.cu keeps a cell's vectors in shared memory
// and loads and stores one value per n multiply-adds of a 1D contraction; on
// GB300 that bounds the FP32 kernels by shared-memory instructions, with the
// FP32 pipe a quarter busy.  Here lane (cw, k) of a warp owns z-plane k of
// cell slot cw in registers (PC = 32 / n cells per warp).  The block is
// applied in the factored form (M symmetric positive definite, so
// D_T = sum_d A_d (x)_d M (x) M = (M (x) M (x) M) o sum_d (M^-1 A_d) x_d),
//     Q = M_x M_y M_z sum_d Ah_d x_d P,   Ah_d = M^-1 A_d,
// with the contractions along x and y in registers (the per-cell matrix rows
// come from shared memory in 16-byte loads, each row serving n lines) and
// those along z from a staging area in shared memory that holds the cell's n
// planes: a lane reads plane j as 16-byte chunks that the n lanes of its
// cell share (a broadcast), so each staged value feeds n multiply-adds per
// lane.  The PC cells of a warp are PC consecutive cells, so their values
// move between global and shared memory in coalesced passes over one
// contiguous range.  Only the Jacobi sweep (all cells) and the operator use
// this form; the colour-by-colour block-SOR keeps the line form.
#if DGMG_N <= 5
namespace pl {
constexpr int PC = 32 / N;                     // cells per warp
constexpr int PL = PC * N;                     // lanes that own a plane
constexpr int PP = (N2 + 3) / 4 * 4;           // plane pitch (floats, 16-byte multiple)
constexpr int Q4 = PP / 4;                     // 16-byte chunks per plane
constexpr int CS0 = N * Q4;
constexpr int CS = (CS0 % 2) ? CS0 : CS0 + 1;  // chunks per cell, odd: the PC cells' chunks of one
                                               // broadcast read fall in different bank groups
constexpr int CF = 4 * CS;                     // floats per cell of a staging area
constexpr int RP = (N + 3) / 4 * 4;            // row pitch of the per-cell matrices
constexpr int AM0 = 3 * N * RP / 4;
constexpr int AMC = (AM0 % 2) ? AM0 : AM0 + 1;
constexpr int AMF = 4 * AMC;                   // floats per cell of the matrices
constexpr int FSF = 12 * N2;                   // floats per cell of the neighbour face values
constexpr int FCF = 24;                        // floats per cell of the face factors

// Shared bytes per warp: staging area, per-cell matrices, face factors,
// (full operator) neighbour face values, cell records, cell flags.
__host__ __device__ constexpr size_t warp_bytes(bool full) {
  return (size_t)(PC * CF + PC * AMF + PC * FCF + (full ? PC * FSF : 0)) * 4 + align16(PC * sizeof(CellInfo<float>)) +
         16;
}

struct Mem {
  float* st;
  float* ah;
  float* fc;
  float* fs;
  CellInfo<float>* ci;
  unsigned char* act;
};

__device__ __forceinline__ Mem carve_plane(unsigned char* raw, bool full) {
  Mem m;
  m.st = reinterpret_cast<float*>(raw);
  m.ah = m.st + PC * CF;
  m.fc = m.ah + PC * AMF;
  m.fs = m.fc + PC * FCF;
  unsigned char* tail = raw + (size_t)(PC * CF + PC * AMF + PC * FCF + (full ? PC * FSF : 0)) * 4;
  m.ci = reinterpret_cast<CellInfo<float>*>(tail);
  m.act = tail + align16(PC * sizeof(CellInfo<float>));
  return m;
}

// The face factors and Ah_d of the warp's cells, rows padded to RP.
__device__ __forceinline__ void matrices(const MeshParams& mp, const Mem& m, int lane) {
  face_consts<float, PC>(m.fc, mp, m.ci, m.act, lane);
  __syncwarp();
  for (int it = lane; it < PC * 3 * N2; it += 32) {
    const int cw = it / (3 * N2), r = it - cw * 3 * N2, d = r / N2, i = (r % N2) / N, j = r % N;
    if (!m.act[cw]) continue;
    m.ah[cw * AMF + (d * N + i) * RP + j] = hat_entry(m.ci[cw], m.fc + cw * FCF, d, i, j);
  }
}

// Coalesced copy of the warp's cells (values g[cell0 N^3 ...], nval of them,
// zero beyond) into the staging area, and the reverse.
template <typename G>
__device__ __forceinline__ void load_cells(const G* __restrict__ g, long long cell0, long long nval, float* st,
                                           int lane) {
  const G* src = g + cell0 * N3;
  for (int e = lane; e < PC * N3; e += 32) {
    const int c = e / N3, r = e - c * N3, kk = r / N2, q = r - kk * N2;
    st[c * CF + kk * PP + q] = e < nval ? float(src[e]) : 0.f;
  }
}

__device__ __forceinline__ void store_cells(float* __restrict__ g, long long cell0, long long nval, const float* st,
                                            int lane) {
  float* dst = g + cell0 * N3;
  for (int e = lane; e < nval; e += 32) {
    const int c = e / N3, r = e - c * N3, kk = r / N2, q = r - kk * N2;
    dst[e] = st[c * CF + kk * PP + q];
  }
}

// The lane's plane from / to the staging area (16-byte accesses).
__device__ __forceinline__ void read_plane(const float* st, int cw, int k, float (&x)[N2]) {
  const float4* p = reinterpret_cast<const float4*>(st + cw * CF + k * PP);
#pragma unroll
  for (int q = 0; q < Q4; ++q) {
    const float4 v = p[q];
    if (4 * q + 0 < N2) x[4 * q + 0] = v.x;
    if (4 * q + 1 < N2) x[4 * q + 1] = v.y;
    if (4 * q + 2 < N2) x[4 * q + 2] = v.z;
    if (4 * q + 3 < N2) x[4 * q + 3] = v.w;
  }
}

__device__ __forceinline__ void write_plane(float* st, int cw, int k, const float (&x)[N2]) {
  float4* p = reinterpret_cast<float4*>(st + cw * CF + k * PP);
#pragma unroll
  for (int q = 0; q < Q4; ++q) {
    float4 v;
    v.x = 4 * q + 0 < N2 ? x[4 * q + 0] : 0.f;
    v.y = 4 * q + 1 < N2 ? x[4 * q + 1] : 0.f;
    v.z = 4 * q + 2 < N2 ? x[4 * q + 2] : 0.f;
    v.w = 4 * q + 3 < N2 ? x[4 * q + 3] : 0.f;
    p[q] = v;
  }
}

// acc += w * plane (the lane's cell, plane j of the staging area st).
__device__ __forceinline__ void axpy_plane(const float* st, int cw, int j, float w, float (&acc)[N2]) {
  const float4* p = reinterpret_cast<const float4*>(st + cw * CF + j * PP);
#pragma unroll
  for (int q = 0; q < Q4; ++q) {
    const float4 v = p[q];
    if (4 * q + 0 < N2) acc[4 * q + 0] = fmaf(w, v.x, acc[4 * q + 0]);
    if (4 * q + 1 < N2) acc[4 * q + 1] = fmaf(w, v.y, acc[4 * q + 1]);
    if (4 * q + 2 < N2) acc[4 * q + 2] = fmaf(w, v.z, acc[4 * q + 2]);
    if (4 * q + 3 < N2) acc[4 * q + 3] = fmaf(w, v.w, acc[4 * q + 3]);
  }
}

// Row i of the lane's cell matrix Ah_d.
__device__ __forceinline__ void matrix_row(const float* ah, int cw, int d, int i, float (&row)[RP]) {
  const float4* p = reinterpret_cast<const float4*>(ah + cw * AMF + (d * N + i) * RP);
#pragma unroll
  for (int q = 0; q < RP / 4; ++q) {
    const float4 v = p[q];
    row[4 * q + 0] = v.x;
    row[4 * q + 1] = v.y;
    row[4 * q + 2] = v.z;
    row[4 * q + 3] = v.w;
  }
}

// Per-lane constants: row k of M and, for the z faces, the weights
// M^-1 e_e(k) (sides 0, 1) and M^-1 dl_s(k).
struct LaneConst {
  float mk[N];
  float wz[4];
};

__device__ __forceinline__ LaneConst lane_const(int k) {
  const Tab<float>& t = c_tab_f;
  LaneConst c;
#pragma unroll
  for (int j = 0; j < N; ++j) c.mk[j] = t.M1[k][j];
  c.wz[0] = t.mie[0][k];
  c.wz[1] = t.mie[1][k];
  c.wz[2] = t.midl[0][k];
  c.wz[3] = t.midl[1][k];
  return c;
}

// Q = A P (FULL, neighbour face values in fs) or D_T P for the lane's plane.
// On entry the staging area holds the planes of P of every cell of the warp;
// on exit it holds the planes of M_x M_y Z.  Z: scratch.  All lanes call it
// (the lanes beyond PL work on cell slot 0 and store nothing).
template <bool FULL>
__device__ __forceinline__ void apply(const float (&P)[N2], float (&Q)[N2], float (&Z)[N2], const Mem& m, int cw, int k,
                                      bool on, const LaneConst& lc) {
  const Tab<float>& t = c_tab_f;
  float row[RP];
  // x: Z[y][i] = sum_j Ax[i][j] P[y][j]
#pragma unroll
  for (int i = 0; i < N; ++i) {
    matrix_row(m.ah, cw, 0, i, row);
#pragma unroll
    for (int y = 0; y < N; ++y) {
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) s = fmaf(row[j], P[y * N + j], s);
      Z[y * N + i] = s;
    }
  }
  // y: Z[y][x] += sum_j Ay[y][j] P[j][x]
#pragma unroll
  for (int y = 0; y < N; ++y) {
    matrix_row(m.ah, cw, 1, y, row);
#pragma unroll
    for (int x = 0; x < N; ++x) {
      float s = Z[y * N + x];
#pragma unroll
      for (int j = 0; j < N; ++j) s = fmaf(row[j], P[j * N + x], s);
      Z[y * N + x] = s;
    }
  }
  // z: Z += sum_j Az[k][j] (plane j of P)
  matrix_row(m.ah, cw, 2, k, row);
#pragma unroll
  for (int j = 0; j < N; ++j) axpy_plane(m.st, cw, j, row[j], Z);
  if (FULL) {
    // neighbour values, weighted by M^-1 e_e and M^-1 dl_s along each normal
    const float* fs = m.fs + cw * FSF;
#pragma unroll
    for (int sd = 0; sd < 2; ++sd) {
      const float* xv = fs + (0 + sd) * 2 * N2;   // x faces: point y + N k
      const float* yv = fs + (2 + sd) * 2 * N2;   // y faces: point x + N k
      const float* zv = fs + (4 + sd) * 2 * N2;   // z faces: point x + N y
#pragma unroll
      for (int y = 0; y < N; ++y) {
        const float qv = xv[y + N * k], qd = xv[N2 + y + N * k];
#pragma unroll
        for (int x = 0; x < N; ++x) Z[y * N + x] = fmaf(t.mie[sd][x], qv, fmaf(t.midl[sd][x], qd, Z[y * N + x]));
      }
#pragma unroll
      for (int x = 0; x < N; ++x) {
        const float qv = yv[x + N * k], qd = yv[N2 + x + N * k];
#pragma unroll
        for (int y = 0; y < N; ++y) Z[y * N + x] = fmaf(t.mie[sd][y], qv, fmaf(t.midl[sd][y], qd, Z[y * N + x]));
      }
      const float wv = lc.wz[sd], wd = lc.wz[2 + sd];
#pragma unroll
      for (int e = 0; e < N2; ++e) Z[e] = fmaf(wv, zv[e], fmaf(wd, zv[N2 + e], Z[e]));
    }
  }
  // mass along x then y in registers (Q as the intermediate)
#pragma unroll
  for (int y = 0; y < N; ++y)
#pragma unroll
    for (int i = 0; i < N; ++i) {
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) s = fmaf(t.M1[i][j], Z[y * N + j], s);
      Q[y * N + i] = s;
    }
#pragma unroll
  for (int y = 0; y < N; ++y)
#pragma unroll
    for (int x = 0; x < N; ++x) {
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < N; ++j) s = fmaf(t.M1[y][j], Q[j * N + x], s);
      Z[y * N + x] = s;
    }
  // mass along z through the staging area
  __syncwarp();   // every lane has read the planes of P
  if (on) write_plane(m.st, cw, k, Z);
  __syncwarp();
#pragma unroll
  for (int e = 0; e < N2; ++e) Q[e] = 0.f;
#pragma unroll
  for (int j = 0; j < N; ++j) axpy_plane(m.st, cw, j, lc.mk[j], Q);
}

// Sum of x over the N lanes of the lane's cell (the same order in every lane).
__device__ __forceinline__ float cell_sum(float x, int cw) {
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < N; ++j) s += __shfl_sync(0xffffffffu, x, cw * N + j);
  return s;
}

}  // namespace pl

// v = A u (FULL) or D_T u, FP32, b = 0, plane per lane.
template <bool FULL>
__device__ __forceinline__ void apply_plane_body(const MeshParams& mp, const float* __restrict__ u,
                                                 float* __restrict__ v, unsigned bid) {
  using namespace pl;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long cell0 = ((long long)bid * (blockDim.x >> 5) + warp) * PC;
  if (cell0 >= mp.ncell) return;
  const Mem m = carve_plane(smem + warp * warp_bytes(FULL), FULL);
  stage_cells<float, PC>(mp, cell0, lane, m.ci, m.act);
  const bool on = lane < PL;
  const int cw = on ? lane / N : 0, k = on ? lane % N : 0;
  const long long left = (mp.ncell - cell0) * N3;
  const long long nval = left < PC * N3 ? left : PC * N3;
  load_cells(u, cell0, nval, m.st, lane);
  matrices(mp, m, lane);
  if (FULL) neighbour_faces<float, float, PC>(m.fs, m.fc, u, lane, m.act, m.ci);
  __syncwarp();
  const LaneConst lc = lane_const(k);
  float P[N2], Q[N2], Z[N2];
  read_plane(m.st, cw, k, P);
  pl::apply<FULL>(P, Q, Z, m, cw, k, on, lc);
  __syncwarp();
  if (on) write_plane(m.st, cw, k, Q);
  __syncwarp();
  store_cells(v, cell0, nval, m.st, lane);
}

template <bool FULL>
__global__ void __launch_bounds__(256) k_apply_plane(const __grid_constant__ MeshParams mp,
                                                     const float* __restrict__ u, float* __restrict__ v) {
  apply_plane_body<FULL>(mp, u, v, blockIdx.x);
}

template <bool FULL>
__global__ void __launch_bounds__(256) k_apply_plane_batch(const __grid_constant__ BatchTable bt) {
  const int r = batch_member(bt, blockIdx.x);
  apply_plane_body<FULL>(bt.mp[r], (const float*)bt.in[r], (float*)bt.out[r], blockIdx.x - bt.block0[r]);
}

// Block-Jacobi sweep with inner PCG, FP32, b = 0, plane per lane (the same
// algorithm as k_smooth_pcg: defect, PCG on D_T with 1/diag(D_T) from 0 on
// d / ||d|| to ||r|| <= eps, u_new = u_old + omega delta).
__device__ __forceinline__ void smooth_plane_body(const MeshParams& mp, const float* __restrict__ f,
                                                  const float* uold, float* unew, const float* __restrict__ diag,
                                                  float omega, float eps, int maxit, int* __restrict__ its,
                                                  unsigned bid) {
  using namespace pl;
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long cell0 = ((long long)bid * (blockDim.x >> 5) + warp) * PC;
  if (cell0 >= mp.ncell) return;
  const Mem m = carve_plane(smem + warp * warp_bytes(true), true);
  stage_cells<float, PC>(mp, cell0, lane, m.ci, m.act);
  const bool on = lane < PL;
  const int cw = on ? lane / N : 0, k = on ? lane % N : 0;
  const bool mine = on && m.act[cw];
  const bool zero = uold == nullptr;
  const long long left = (mp.ncell - cell0) * N3;
  const long long nval = left < PC * N3 ? left : PC * N3;
  matrices(mp, m, lane);
  const LaneConst lc = lane_const(k);
  float R[N2], D[N2], P[N2], Q[N2], Z[N2], DL[N2];
  // f and 1/diag(D_T) through the staging area
  load_cells(f, cell0, nval, m.st, lane);
  __syncwarp();
  read_plane(m.st, cw, k, R);
  __syncwarp();
  load_cells(diag, cell0, nval, m.st, lane);
  __syncwarp();
  read_plane(m.st, cw, k, D);
  __syncwarp();
  // defect d = f - A u_old
  if (!zero) {
    load_cells(uold, cell0, nval, m.st, lane);
    neighbour_faces<float, float, PC>(m.fs, m.fc, uold, lane, m.act, m.ci);
    __syncwarp();
    read_plane(m.st, cw, k, P);
    pl::apply<true>(P, Q, Z, m, cw, k, on, lc);
#pragma unroll
    for (int e = 0; e < N2; ++e) R[e] -= Q[e];
  }
  float prr = 0.f, prz = 0.f;
#pragma unroll
  for (int e = 0; e < N2; ++e) {
    const float z = R[e] * D[e];
    P[e] = z;
    DL[e] = 0.f;
    prr = fmaf(R[e], R[e], prr);
    prz = fmaf(R[e], z, prz);
  }
  const float rr0 = cell_sum(prr, cw);
  float rz = cell_sum(prz, cw);
  // work on d / ||d|| (see k_smooth_pcg)
  const float dnorm = sqrtf(rr0);
  const float isc = rr0 > 0.f ? 1.f / dnorm : 0.f;
#pragma unroll
  for (int e = 0; e < N2; ++e) {
    R[e] *= isc;
    P[e] *= isc;
  }
  rz = rz * isc * isc;
  const float thr2 = eps * eps;
  bool live = mine && rr0 > 0.f;
  int it = 0;
  while (__any_sync(0xffffffffu, live && it < maxit)) {
    const bool run = live && it < maxit;
    __syncwarp();   // the staging area is free
    if (on) write_plane(m.st, cw, k, P);
    __syncwarp();
    pl::apply<false>(P, Q, Z, m, cw, k, on, lc);
    float ppq = 0.f;
#pragma unroll
    for (int e = 0; e < N2; ++e) ppq = fmaf(P[e], Q[e], ppq);
    const float pq = cell_sum(ppq, cw);
    bool upd = run && pq > 0.f;
    if (run && !upd) live = false;   // breakdown: stop this cell
    float prr2 = 0.f, prz2 = 0.f;
    if (upd) {
      const float alpha = rz / pq;
#pragma unroll
      for (int e = 0; e < N2; ++e) {
        DL[e] = fmaf(alpha, P[e], DL[e]);
        const float r = fmaf(-alpha, Q[e], R[e]);
        R[e] = r;
        prr2 = fmaf(r, r, prr2);
        const float z = r * D[e];
        Z[e] = z;
        prz2 = fmaf(r, z, prz2);
      }
      ++it;
    }
    prr2 = cell_sum(prr2, cw);
    prz2 = cell_sum(prz2, cw);
    if (upd && prr2 <= thr2) {
      live = false;
      upd = false;
    }
    if (upd && it >= maxit) upd = false;
    if (upd) {
      const float beta = prz2 / rz;
      rz = prz2;
#pragma unroll
      for (int e = 0; e < N2; ++e) P[e] = fmaf(beta, P[e], Z[e]);
    }
  }
  // u_new = u_old + omega delta
  __syncwarp();
  if (!zero) {
    load_cells(uold, cell0, nval, m.st, lane);
    __syncwarp();
    read_plane(m.st, cw, k, P);
    __syncwarp();
  }
#pragma unroll
  for (int e = 0; e < N2; ++e) {
    const float dl = DL[e] * dnorm;
    Q[e] = zero ? omega * dl : fmaf(omega, dl, P[e]);
  }
  if (on) write_plane(m.st, cw, k, Q);
  __syncwarp();
  store_cells(unew, cell0, nval, m.st, lane);
  if (its && on && k == 0 && m.act[cw]) its[cell0 + cw] = it;
}

__global__ void __launch_bounds__(128) k_smooth_plane(const __grid_constant__ MeshParams mp,
                                                      const float* __restrict__ f, const float* uold, float* unew,
                                                      const float* __restrict__ diag, float omega, float eps,
                                                      int maxit, int* __restrict__ its) {
  smooth_plane_body(mp, f, uold, unew, diag, omega, eps, maxit, its, blockIdx.x);
}

__global__ void __launch_bounds__(128) k_smooth_plane_batch(const __grid_constant__ BatchTable bt) {
  const int r = batch_member(bt, blockIdx.x);
  smooth_plane_body(bt.mp[r], (const float*)bt.in[r], (const float*)bt.uold[r], (float*)bt.out[r],
                    (const float*)bt.diag[r], float(bt.omega), float(bt.eps), bt.maxit, bt.its[r],
                    blockIdx.x - bt.block0[r]);
}
#endif
