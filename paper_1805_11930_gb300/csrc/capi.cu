// The C ABI of include/dgmg.h: context, mesh and coefficient setup, the
// matrix-free operator and smoother entry points, the hybrid V-cycle
// (Algorithm 1 of arXiv 1805.11930) and the outer Krylov drivers.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "dgmg.h"
#include "dgmg_internal.h"
#include "setup_host.h"

namespace dgmg {
thread_local unsigned long long t_launches = 0;

const CellOps* cell_ops_n2();
const CellOps* cell_ops_n3();
const CellOps* cell_ops_n4();
const CellOps* cell_ops_n5();
const CellOps* cell_ops_n6();
const CellOps* cell_ops_n7();
const CellOps* cell_ops_n8();
const CellOps* cell_ops_n9();

const CellOps* cell_ops(int n) {
  switch (n) {
    case 2: return cell_ops_n2();
    case 3: return cell_ops_n3();
    case 4: return cell_ops_n4();
    case 5: return cell_ops_n5();
    case 6: return cell_ops_n6();
    case 7: return cell_ops_n7();
    case 8: return cell_ops_n8();
    case 9: return cell_ops_n9();
    default: return nullptr;
  }
}

namespace {
// Adds the per-cell inner iteration counts of one sweep to a running sum and
// maximum (integer atomics once per block; the result is order independent).
// sum[0] += sum of its, sum[1] += sum of its^2, *mx = max(*mx, its).
__global__ void k_its_acc(long long n, const int* __restrict__ its, unsigned long long* sum, int* mx) {
  __shared__ unsigned long long ssum[256], ssq[256];
  __shared__ int smax[256];
  unsigned long long s = 0, q = 0;
  int m = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long v = (unsigned long long)its[i];
    s += v;
    q += v * v;
    m = its[i] > m ? its[i] : m;
  }
  ssum[threadIdx.x] = s;
  ssq[threadIdx.x] = q;
  smax[threadIdx.x] = m;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      ssum[threadIdx.x] += ssum[threadIdx.x + o];
      ssq[threadIdx.x] += ssq[threadIdx.x + o];
      smax[threadIdx.x] = smax[threadIdx.x] > smax[threadIdx.x + o] ? smax[threadIdx.x] : smax[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    atomicAdd(sum, ssum[0]);
    atomicAdd(sum + 1, ssq[0]);
    atomicMax(mx, smax[0]);
  }
}
}  // namespace
}  // namespace dgmg

using namespace dgmg;

struct AmgLevel {
  int vx, vy, vz;
  long long n;
  // damped-Jacobi weight, set by build_hier to 4 / (3 G), G the Gershgorin
  // bound of D^-1 A (the initial value is never used)
  double omega = 2.0 / 3.0;
  double* st = nullptr;
  double* dinv = nullptr;
  double* b = nullptr;
  double* x = nullptr;
  double* xt = nullptr;
  double* r = nullptr;
};

// One aggregation-AMG hierarchy on a structured grid: the Q1 vertices, or the
// cells for the P0 subspace.  Level 0 holds A_hat as a 27-point stencil.
struct Hier {
  std::vector<AmgLevel> lv;
  double* coarse_inv = nullptr;   // dense inverse of the coarsest level
  int coarse_n = 0;
  double* rhat = nullptr;         // restricted residual / coarse correction
  double* uhat = nullptr;
  std::vector<double> st;         // host copy of the level-0 stencil
  bool built = false;
};

struct dgmg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  bool has_mesh = false, has_coef = false;
  int nx = 0, ny = 0, nz = 0, p = 0, n = 0;
  double L[3] = {0, 0, 0}, h[3] = {0, 0, 0};
  double alpha = 1.25;           // interior penalty parameter
  int bc[6] = {0, 0, 0, 0, 0, 0};
  long long ncell = 0, ndof = 0, nvert = 0;
  const CellOps* ops = nullptr;
  int kdim = 1;
  std::vector<double> hK, hb, hc, q1;
  double *dK = nullptr, *dc = nullptr, *db = nullptr;
  double* diag64 = nullptr;
  float* diag32 = nullptr;
  double* dinv64 = nullptr;      // 1 / diag(D_T), used by the smoothers
  float* dinv32 = nullptr;
  double* rec64 = nullptr;       // per-cell coefficient records
  float* rec32 = nullptr;
  float* db32 = nullptr;         // float copy of b
  double* w64[3] = {nullptr, nullptr, nullptr};
  float* w32[4] = {nullptr, nullptr, nullptr, nullptr};
  double* corners = nullptr;
  int* its = nullptr;
  unsigned long long* itsum = nullptr;   // [sum of inner iterations, sum of their squares]
  int* itmax = nullptr;
  Hier q1h;   // Q1 coarse space (built with the coefficients)
  Hier p0h;   // P0 coarse space (built on first use)
  double* kry = nullptr;
  size_t kry_vecs = 0;
  double* dot_partial = nullptr;
  double* dot_out = nullptr;
  double* dot_host = nullptr;      // pinned
  const double** dot_ptrs = nullptr;  // device array of vector pointers
  bool track_its = false;
  long long sweeps_tracked = 0;
  // per-launch CUDA-event timing of the smoother and operator kernels
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
  std::vector<std::pair<size_t, size_t>> ev_smooth, ev_apply, ev_transfer, ev_coarse;
  long long n_apply = 0, n_sweep = 0, n_zero_sweep = 0;
  // Captured preconditioner graphs, keyed by (input, output, V-cycle options).
  struct PrecGraph {
    const double* in;
    double* out;
    dgmg_solve_opts opts;
    cudaGraphExec_t exec;
    long long d_sweep, d_zero, d_apply, d_tracked;
    unsigned long long d_launches;
  };
  std::vector<PrecGraph> graphs;
  std::vector<void*> mesh_allocs;  // freed on a new mesh
  // warps per block of the operator / smoother kernels per precision (0 = 4)
  int wpb_apply[3] = {0, 0, 0}, wpb_smooth[3] = {0, 0, 0};
  // work layouts per precision (dgmg_layout; AUTO = the default)
  int lay_apply[3] = {0, 0, 0}, lay_smooth[3] = {0, 0, 0};
  // stored inverses of the diagonal blocks (DGMG_INNER_DIRECT), built on demand
  float2* binv_df = nullptr;    // for FP64 smoothers: double-float pairs
  float* binv32 = nullptr;      // for FP32 smoothers
  int binv_ld = 0;              // column stride (n^3 rounded up to a multiple of 8)
  // K(x), c(x) of the outer operator (dgmg_set_variable_coefficients)
  bool var_on = false;
  std::vector<double> hvar;     // 16 values: basis rows, p0, p2, gamma
  double* dvar = nullptr;
  // Thomas factors of the tridiagonal part of D_T (DGMG_INNER_GMRES_TRIDIAG)
  double* tri64 = nullptr;
  float* tri32 = nullptr;
  // Initial Krylov state of a batched solve computed by dgmg_batch_prime:
  // r, z, p in kry, ||r_0|| and (r, z), for (f, u) and the V-cycle options.
  bool primed = false;
  const double* prime_f = nullptr;
  double* prime_u = nullptr;
  double prime_r0 = 0.0, prime_rz = 0.0;
  dgmg_solve_opts prime_key;
};

namespace {

// NVTX range around a host-side phase (solve, V-cycle, smoother, operator,
// coarse correction, set-up), so that a profiler can select or attribute
// the kernels of each; costs a function call when no tool is attached.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

constexpr int kMaxDots = 72;

dgmg_status fail(dgmg_ctx* c, dgmg_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

size_t record_event(dgmg_ctx* ctx) {
  if (ctx->ev_used == ctx->ev.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    ctx->ev.push_back(e);
  }
  cudaEventRecord(ctx->ev[ctx->ev_used], ctx->stream);
  return ctx->ev_used++;
}

#define CK(expr)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, DGMG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));     \
  } while (0)

#define CS(expr)                      \
  do {                                \
    dgmg_status s_ = (expr);          \
    if (s_ != DGMG_OK) return s_;     \
  } while (0)

template <typename T>
dgmg_status dalloc(dgmg_ctx* ctx, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  // Stream-ordered allocation: no device-wide synchronisation, so contexts
  // on other streams (concurrent solves) keep running.
  cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, DGMG_ERR_OOM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  }
  ctx->mesh_allocs.push_back((void*)*p);
  return DGMG_OK;
}

void drop_graphs(dgmg_ctx* ctx) {
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
}

void free_mesh(dgmg_ctx* ctx) {
  ctx->primed = false;
  drop_graphs(ctx);
  for (void* q : ctx->mesh_allocs) cudaFreeAsync(q, ctx->stream);
  ctx->mesh_allocs.clear();
  ctx->dK = ctx->dc = ctx->db = ctx->diag64 = ctx->dinv64 = ctx->rec64 = nullptr;
  ctx->diag32 = ctx->dinv32 = ctx->rec32 = ctx->db32 = nullptr;
  for (auto& w : ctx->w64) w = nullptr;
  for (auto& w : ctx->w32) w = nullptr;
  ctx->corners = nullptr;
  ctx->its = nullptr;
  ctx->itsum = nullptr;
  ctx->itmax = nullptr;
  ctx->q1h = Hier();
  ctx->p0h = Hier();
  ctx->kry = nullptr;
  ctx->kry_vecs = 0;
  ctx->binv_df = nullptr;
  ctx->binv32 = nullptr;
  ctx->binv_ld = 0;
  ctx->var_on = false;
  ctx->dvar = nullptr;
  ctx->tri64 = nullptr;
  ctx->tri32 = nullptr;
  ctx->has_coef = false;
}

// Frees one allocation made by dalloc before the mesh changes.
void dfree(dgmg_ctx* ctx, void* q) {
  for (auto it = ctx->mesh_allocs.begin(); it != ctx->mesh_allocs.end(); ++it)
    if (*it == q) {
      ctx->mesh_allocs.erase(it);
      cudaFreeAsync(q, ctx->stream);
      return;
    }
}

// The layout a kernel uses for precision prec: AUTO is the default of the
// precision, order and kernel, the faster form measured on GB300.  b = 0:
// ELEMENT (the factored form) for FP64 and DF64; in FP32 LINE for the
// operator, PLANE for the smoother with p <= 4.  b != 0: ELEMENT for FP64 at
// p = 4..6, LINE otherwise (p = 7, 8 unmeasured: the line form).
int resolve_layout(const dgmg_ctx* ctx, int prec, int lay, bool smoother) {
  if (lay != DGMG_LAYOUT_AUTO) return lay;
  if (ctx->db) return prec == DGMG_FP64 && ctx->p >= 4 && ctx->p <= 6 ? DGMG_LAYOUT_ELEMENT : DGMG_LAYOUT_LINE;
  if (prec == DGMG_FP32) return smoother && ctx->p <= 4 ? DGMG_LAYOUT_PLANE : DGMG_LAYOUT_LINE;
  return DGMG_LAYOUT_ELEMENT;
}

bool layout_exists(const dgmg_ctx* ctx, int prec, int lay) {
  if (lay == DGMG_LAYOUT_AUTO || lay == DGMG_LAYOUT_LINE || lay == DGMG_LAYOUT_ELEMENT) return true;
  return lay == DGMG_LAYOUT_PLANE && prec == DGMG_FP32 && ctx->p <= 4 && !ctx->db;
}

MeshParams params(const dgmg_ctx* ctx) {
  MeshParams m;
  m.nx = ctx->nx;
  m.ny = ctx->ny;
  m.nz = ctx->nz;
  m.p = ctx->p;
  m.ncell = ctx->ncell;
  for (int d = 0; d < 3; ++d) m.h[d] = ctx->h[d];
  for (int i = 0; i < 6; ++i) m.bc[i] = ctx->bc[i];
  m.K = ctx->dK;
  m.kdim = ctx->kdim;
  m.c = ctx->dc;
  m.bvert = ctx->db;
  m.alpha = ctx->alpha;
  m.rec64 = ctx->rec64;
  m.rec32 = ctx->rec32;
  m.bvert32 = ctx->db32;
  m.var = ctx->var_on ? ctx->dvar : nullptr;
  for (int i = 0; i < 3; ++i) {
    m.wpb_apply[i] = ctx->wpb_apply[i];
    m.wpb_smooth[i] = ctx->wpb_smooth[i];
    m.lay_apply[i] = resolve_layout(ctx, i, ctx->lay_apply[i], false);
    m.lay_smooth[i] = resolve_layout(ctx, i, ctx->lay_smooth[i], true);
  }
  const double J = ctx->h[0] * ctx->h[1] * ctx->h[2];
  for (int d = 0; d < 3; ++d) {
    const int a = d == 0 ? 1 : 0, b = d == 2 ? 1 : 2;
    m.ih[d] = 1.0 / ctx->h[d];
    m.area[d] = ctx->h[a] * ctx->h[b];
    m.jh[d] = J / ctx->h[d];
    m.ihf[d] = (float)m.ih[d];
    m.areaf[d] = (float)m.area[d];
    m.jhf[d] = (float)m.jh[d];
  }
  return m;
}

HostMesh host_mesh(const dgmg_ctx* ctx) {
  HostMesh m;
  m.nx = ctx->nx;
  m.ny = ctx->ny;
  m.nz = ctx->nz;
  m.p = ctx->p;
  for (int d = 0; d < 3; ++d) m.h[d] = ctx->h[d];
  for (int i = 0; i < 6; ++i) m.bc[i] = ctx->bc[i];
  m.K = ctx->hK.data();
  m.kdim = ctx->kdim;
  m.b = ctx->hb.empty() ? nullptr : ctx->hb.data();
  m.c = ctx->hc.empty() ? nullptr : ctx->hc.data();
  m.alpha = ctx->alpha;
  m.var = ctx->var_on ? ctx->hvar.data() : nullptr;
  return m;
}

dgmg_status ready(dgmg_ctx* ctx) {
  if (!ctx) return DGMG_ERR_ARG;
  if (!ctx->has_mesh || !ctx->has_coef) return fail(ctx, DGMG_ERR_STATE, "set_mesh and set_coefficients first");
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return fail(ctx, DGMG_ERR_CUDA, cudaGetErrorString(e));
  return DGMG_OK;
}

// Double-float kernels exist for diffusion (b = 0) with p <= 6 and, in the
// smoothers, the inner PCG or the stored inverses.
dgmg_status check_df64(dgmg_ctx* ctx, int prec, int inner) {
  if (prec != DGMG_DF64) return DGMG_OK;
  if (ctx->p > 6) return fail(ctx, DGMG_ERR_ARG, "DF64 kernels are built for p <= 6");
  if (ctx->db) return fail(ctx, DGMG_ERR_ARG, "DF64 kernels are built for b = 0");
  if (inner != DGMG_INNER_PCG && inner != DGMG_INNER_DIRECT)
    return fail(ctx, DGMG_ERR_ARG, "DF64 smoothers use the inner PCG or stored inverses");
  return DGMG_OK;
}

// ------------------------------------------------------------------ dots
dgmg_status dot(dgmg_ctx* ctx, const double* x, const double* y, double& out) {
  CK(vec_dot(ctx->ndof, x, y, ctx->dot_partial, ctx->dot_out, ctx->stream));
  CK(cudaMemcpyAsync(ctx->dot_host, ctx->dot_out, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  out = ctx->dot_host[0];
  return DGMG_OK;
}

dgmg_status multi_dot(dgmg_ctx* ctx, int k, double* const* xs, const double* y, double* out) {
  CK(cudaMemcpyAsync(ctx->dot_ptrs, xs, k * sizeof(double*), cudaMemcpyHostToDevice, ctx->stream));
  CK(vec_multi_dot(ctx->ndof, k, ctx->dot_ptrs, y, ctx->dot_partial, ctx->dot_out, ctx->stream));
  CK(cudaMemcpyAsync(ctx->dot_host, ctx->dot_out, k * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < k; ++i) out[i] = ctx->dot_host[i];
  return DGMG_OK;
}

// ------------------------------------------------------------------ stored block inverses
// D_T^-1 of every cell: block matrices by unit-vector block applies and
// Gauss-Jordan per block in FP64 (a temporary), then kept as double-float
// pairs for FP64 smoothers or rounded to FP32 for FP32 smoothers, column
// stride ld = n^3 rounded up to a multiple of 8.
dgmg_status ensure_binv(dgmg_ctx* ctx, int prec) {
  Range range("dgmg block inverse set-up");
  if (prec != DGMG_FP64 && prec != DGMG_FP32)
    return fail(ctx, DGMG_ERR_ARG, "stored block inverses are FP64 or FP32");

  if (prec == DGMG_FP64 ? ctx->binv_df != nullptr : ctx->binv32 != nullptr) return DGMG_OK;
  if (ctx->stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(ctx, DGMG_ERR_STATE, "build the block inverses (dgmg_block_inverse) before stream capture");
  }
  const int nb = ctx->n * ctx->n * ctx->n;
  const int ld = (nb + 7) / 8 * 8;
  const size_t count = (size_t)ctx->ncell * nb * ld;
  double* m = nullptr;
  int* sing = nullptr;
  CS(dalloc(ctx, &m, count));
  dgmg_status st = dalloc(ctx, &sing, 1);
  if (st != DGMG_OK) {
    dfree(ctx, m);
    return st;
  }
  int h = 0;
  cudaError_t e = cudaMemsetAsync(sing, 0, sizeof(int), ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m, 0, count * sizeof(double), ctx->stream);
  if (e == cudaSuccess) e = ctx->ops->block_matrix(params(ctx), m, ld, ctx->stream);
  if (e == cudaSuccess) e = block_invert(m, nb, ld, ctx->ncell, sing, ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sing, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  dfree(ctx, sing);
  if (e != cudaSuccess || h) {
    dfree(ctx, m);
    if (e != cudaSuccess) return fail(ctx, DGMG_ERR_CUDA, std::string("block inverse: ") + cudaGetErrorString(e));
    return fail(ctx, DGMG_ERR_ARG, "a diagonal block is singular");
  }
  if (prec == DGMG_FP64) {
    float2* pairs = nullptr;
    st = dalloc(ctx, &pairs, count);
    if (st == DGMG_OK) {
      e = vec_split_df((long long)count, m, pairs, nullptr, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e == cudaSuccess) ctx->binv_df = pairs;
    }
  } else {
    float* m32 = nullptr;
    st = dalloc(ctx, &m32, count);
    if (st == DGMG_OK) {
      e = vec_d2f((long long)count, m, m32, ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e == cudaSuccess) ctx->binv32 = m32;
    }
  }
  dfree(ctx, m);
  if (st != DGMG_OK) return st;
  if (e != cudaSuccess) return fail(ctx, DGMG_ERR_CUDA, std::string("block inverse: ") + cudaGetErrorString(e));
  ctx->binv_ld = ld;
  return DGMG_OK;
}

// Thomas factors of the tridiagonal part of every D_T, FP64 (rounded to FP32
// when prec is FP32), for the GMRES_TRIDIAG inner solver.
dgmg_status ensure_tri(dgmg_ctx* ctx, int prec) {
  if (prec != DGMG_FP64 && prec != DGMG_FP32)
    return fail(ctx, DGMG_ERR_ARG, "the tridiagonal inner preconditioner is FP64 or FP32");
  if (prec == DGMG_FP64 ? ctx->tri64 != nullptr : ctx->tri32 != nullptr) return DGMG_OK;
  if (ctx->stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(ctx, DGMG_ERR_STATE, "run one uncaptured solve or sweep before stream capture");
  }
  const size_t count = (size_t)ctx->ncell * 3 * ctx->n * ctx->n * ctx->n;
  if (!ctx->tri64) {
    double* m = nullptr;
    int* sing = nullptr;
    CS(dalloc(ctx, &m, count));
    dgmg_status st = dalloc(ctx, &sing, 1);
    if (st != DGMG_OK) {
      dfree(ctx, m);
      return st;
    }
    int h = 0;
    cudaError_t e = cudaMemsetAsync(sing, 0, sizeof(int), ctx->stream);
    if (e == cudaSuccess) e = ctx->ops->block_tridiag(params(ctx), m, sing, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sing, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, sing);
    if (e != cudaSuccess || h) {
      dfree(ctx, m);
      if (e != cudaSuccess) return fail(ctx, DGMG_ERR_CUDA, std::string("tridiagonal factors: ") + cudaGetErrorString(e));
      return fail(ctx, DGMG_ERR_ARG, "the tridiagonal part of a diagonal block has a zero pivot");
    }
    ctx->tri64 = m;
  }
  if (prec == DGMG_FP32) {
    float* m32 = nullptr;
    CS(dalloc(ctx, &m32, count));
    CK(vec_d2f((long long)count, ctx->tri64, m32, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->tri32 = m32;
  }
  return DGMG_OK;
}

// Per-sweep arguments that depend on the inner solver: the stored inverses
// (DIRECT) or the Thomas factors (GMRES_TRIDIAG), built on first use.
dgmg_status inner_data(dgmg_ctx* ctx, int inner, int prec, const void** binv, const void** tri) {
  *binv = *tri = nullptr;
  const bool fp32 = prec == DGMG_FP32;
  if (inner == DGMG_INNER_DIRECT) {
    CS(ensure_binv(ctx, prec == DGMG_DF64 ? DGMG_FP64 : prec));   // DF64 shares the FP64 pairs
    *binv = fp32 ? (const void*)ctx->binv32 : (const void*)ctx->binv_df;
  } else if (inner == DGMG_INNER_GMRES_TRIDIAG) {
    CS(ensure_tri(ctx, prec));
    *tri = fp32 ? (const void*)ctx->tri32 : (const void*)ctx->tri64;
  }
  return DGMG_OK;
}

dgmg_status prepare_inner(dgmg_ctx* ctx, int inner, int prec) {
  const void *b, *t;
  return inner_data(ctx, inner, prec, &b, &t);
}

// ------------------------------------------------------------------ smoother
// nsweep block-Jacobi sweeps on u (in place) with ping-pong through tmp.
dgmg_status smooth_internal(dgmg_ctx* ctx, const void* f, void* u, void* tmp, int nsweep, double omega, double eps,
                            int maxit, int inner, int restart, int prec, bool zero_first, int* its) {
  Range range("dgmg smoother");
  const bool fp32 = prec == DGMG_FP32;
  if (nsweep <= 0) {
    if (zero_first) {
      if (fp32)
        CK(vec_fill_f(ctx->ndof, 0.f, (float*)u, ctx->stream));
      else
        CK(vec_fill(ctx->ndof, 0.0, (double*)u, ctx->stream));
    }
    return DGMG_OK;
  }
  if (maxit <= 0) maxit = ctx->n * ctx->n * ctx->n;
  if (inner < DGMG_INNER_PCG || inner > DGMG_INNER_GMRES_TRIDIAG) return fail(ctx, DGMG_ERR_ARG, "bad inner solver");
  if ((inner == DGMG_INNER_GMRES || inner == DGMG_INNER_GMRES_TRIDIAG) && (restart < 1 || restart > 64))
    return fail(ctx, DGMG_ERR_ARG, "inner_restart must be in [1, 64]");
  const void *binv = nullptr, *tri = nullptr;
  CS(inner_data(ctx, inner, prec, &binv, &tri));
  const MeshParams mp = params(ctx);
  void* src = u;
  void* dst = tmp;
  for (int k = 0; k < nsweep; ++k) {
    SmoothArgs a;
    a.f = f;
    a.uold = (k == 0 && zero_first) ? nullptr : src;
    a.unew = dst;
    a.diag = fp32 ? (const void*)ctx->dinv32 : (const void*)ctx->dinv64;
    a.omega = omega;
    a.eps = eps;
    a.maxit = maxit;
    a.inner = inner;
    a.restart = restart;
    a.binv = binv;
    a.binv_ld = ctx->binv_ld;
    a.tri = tri;
    a.its = (its || ctx->track_its) ? ctx->its : nullptr;
    const size_t e0 = ctx->timing ? record_event(ctx) : 0;
    CK(ctx->ops->smooth(mp, a, prec, ctx->stream));
    if (ctx->timing) ctx->ev_smooth.push_back({e0, record_event(ctx)});
    ++ctx->n_sweep;
    if (k == 0 && zero_first) ++ctx->n_zero_sweep;
    if (ctx->track_its) {
      k_its_acc<<<152, 256, 0, ctx->stream>>>(ctx->ncell, ctx->its, ctx->itsum, ctx->itmax);
      count_launch();
      CK(cudaGetLastError());
      ++ctx->sweeps_tracked;
    }
    void* t = src;
    src = dst;
    dst = t;
  }
  if (src != u) CK(cudaMemcpyAsync(u, src, ctx->ndof * (fp32 ? 4 : 8), cudaMemcpyDeviceToDevice, ctx->stream));
  if (its && its != ctx->its)
    CK(cudaMemcpyAsync(its, ctx->its, ctx->ncell * sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
  return DGMG_OK;
}

// nsweep multicolour block-SOR passes on u in place (NEXT to Algorithm 3):
// colours 0..7 (cells whose index parities (cx, cy, cz) give kx + 2ky + 4kz),
// each colour in one launch that reads the current values of the other
// colours; symmetric = forward colours then backward colours (block-SSOR).
dgmg_status sor_internal(dgmg_ctx* ctx, const void* f, void* u, int nsweep, double omega, double eps, int maxit,
                         int inner, int restart, int prec, bool zero_first, bool symmetric, int* its) {
  Range range("dgmg smoother (SSOR)");
  const bool fp32 = prec == DGMG_FP32;
  if (zero_first) {
    if (fp32)
      CK(vec_fill_f(ctx->ndof, 0.f, (float*)u, ctx->stream));
    else
      CK(vec_fill(ctx->ndof, 0.0, (double*)u, ctx->stream));
  }
  if (nsweep <= 0) return DGMG_OK;
  if (maxit <= 0) maxit = ctx->n * ctx->n * ctx->n;
  if (inner < DGMG_INNER_PCG || inner > DGMG_INNER_GMRES_TRIDIAG) return fail(ctx, DGMG_ERR_ARG, "bad inner solver");
  if ((inner == DGMG_INNER_GMRES || inner == DGMG_INNER_GMRES_TRIDIAG) && (restart < 1 || restart > 64))
    return fail(ctx, DGMG_ERR_ARG, "inner_restart must be in [1, 64]");
  const void *binv = nullptr, *tri = nullptr;
  CS(inner_data(ctx, inner, prec, &binv, &tri));
  const MeshParams mp = params(ctx);
  const int passes = symmetric ? 2 : 1;
  for (int k = 0; k < nsweep; ++k)
    for (int pass = 0; pass < passes; ++pass) {
      for (int c = 0; c < 8; ++c) {
        SmoothArgs a;
        a.f = f;
        a.uold = u;
        a.unew = u;
        a.diag = fp32 ? (const void*)ctx->dinv32 : (const void*)ctx->dinv64;
        a.omega = omega;
        a.eps = eps;
        a.maxit = maxit;
        a.inner = inner;
        a.restart = restart;
        a.binv = binv;
        a.binv_ld = ctx->binv_ld;
        a.tri = tri;
        a.its = (its || ctx->track_its) ? ctx->its : nullptr;
        a.color = pass == 0 ? c : 7 - c;
        const size_t e0 = ctx->timing ? record_event(ctx) : 0;
        CK(ctx->ops->smooth(mp, a, prec, ctx->stream));
        if (ctx->timing) ctx->ev_smooth.push_back({e0, record_event(ctx)});
      }
      ++ctx->n_sweep;
      if (ctx->track_its) {
        k_its_acc<<<152, 256, 0, ctx->stream>>>(ctx->ncell, ctx->its, ctx->itsum, ctx->itmax);
        count_launch();
        CK(cudaGetLastError());
        ++ctx->sweeps_tracked;
      }
    }
  if (its && its != ctx->its)
    CK(cudaMemcpyAsync(its, ctx->its, ctx->ncell * sizeof(int), cudaMemcpyDeviceToDevice, ctx->stream));
  return DGMG_OK;
}

// The smoother of the V-cycle: block-Jacobi (ping-pong) or multicolour
// block-SSOR (in place).
dgmg_status vcycle_smooth(dgmg_ctx* ctx, const dgmg_solve_opts& o, const void* F, void* U, void* T1, int nsweep,
                          int prec, bool zero) {
  if (o.smoother == DGMG_SMOOTHER_SSOR)
    return sor_internal(ctx, F, U, nsweep, o.omega, o.eps_inner, o.maxit_inner, o.inner, o.inner_restart, prec,
                        zero, true, nullptr);
  return smooth_internal(ctx, F, U, T1, nsweep, o.omega, o.eps_inner, o.maxit_inner, o.inner, o.inner_restart,
                         prec, zero, nullptr);
}

// ------------------------------------------------------------------ AMG
dgmg_status amg_cycle(dgmg_ctx* ctx, Hier& H, int l, const double* b, double* xout) {
  const int last = (int)H.lv.size() - 1;
  if (l == last) {
    CK(dense_matvec(H.coarse_n, H.coarse_inv, b, xout, ctx->stream));
    return DGMG_OK;
  }
  AmgLevel& L = H.lv[l];
  AmgLevel& C = H.lv[l + 1];
  const double w = L.omega;
  CK(stencil_jacobi(L.vx, L.vy, L.vz, L.st, L.dinv, b, nullptr, L.xt, w, true, ctx->stream));
  CK(stencil_residual(L.vx, L.vy, L.vz, L.st, b, L.xt, L.r, ctx->stream));
  CK(agg_restrict(L.vx, L.vy, L.vz, L.r, C.b, ctx->stream));
  CS(amg_cycle(ctx, H, l + 1, C.b, C.x));
  CK(agg_prolong_add(L.vx, L.vy, L.vz, C.x, L.xt, ctx->stream));
  CK(stencil_jacobi(L.vx, L.vy, L.vz, L.st, L.dinv, b, L.xt, xout, w, false, ctx->stream));
  return DGMG_OK;
}

// H.uhat ~ A_hat^-1 H.rhat by `cycles` AMG V-cycles: the first from zero, each
// further one on the current coarse residual (stationary iteration).
dgmg_status coarse_correction(dgmg_ctx* ctx, Hier& H, int cycles) {
  Range range("dgmg coarse AMG");
  CS(amg_cycle(ctx, H, 0, H.rhat, H.uhat));
  AmgLevel& L = H.lv[0];
  for (int k = 1; k < cycles && H.lv.size() > 1; ++k) {
    // r = r_hat - A_hat u_hat into L.b, correction into L.x, then u_hat += L.x
    CK(stencil_residual(L.vx, L.vy, L.vz, L.st, H.rhat, H.uhat, L.b, ctx->stream));
    CS(amg_cycle(ctx, H, 0, L.b, L.x));
    CK(vec_axpby(L.n, 1.0, L.x, 1.0, H.uhat, ctx->stream));
  }
  return DGMG_OK;
}

// Aggregation-AMG hierarchy from a level-0 stencil on a vx x vy x vz grid:
// Gershgorin-weighted Jacobi per level, 2x2x2 Galerkin coarsening down to at
// most 512 unknowns, dense inverse there (host set-up, device storage).
dgmg_status build_hier(dgmg_ctx* ctx, Hier& H, std::vector<double> st, int vx, int vy, int vz) {
  H = Hier();
  H.st = st;
  const long long n0 = (long long)vx * vy * vz;
  CS(dalloc(ctx, &H.rhat, n0));
  CS(dalloc(ctx, &H.uhat, n0));
  while (true) {
    AmgLevel L;
    L.vx = vx;
    L.vy = vy;
    L.vz = vz;
    L.n = (long long)vx * vy * vz;
    const bool coarsest = L.n <= 512;
    if (!coarsest) {
      std::vector<double> dinv(L.n);
      double gmax = 0.0;
      for (long long i = 0; i < L.n; ++i) {
        dinv[i] = 1.0 / st[27 * i + 13];
        double row = 0.0;
        for (int k = 0; k < 27; ++k) row += std::fabs(st[27 * i + k]);
        gmax = std::max(gmax, row * std::fabs(dinv[i]));
      }
      L.omega = 4.0 / (3.0 * gmax);
      CS(dalloc(ctx, &L.st, 27 * L.n));
      CS(dalloc(ctx, &L.dinv, L.n));
      CK(cudaMemcpyAsync(L.st, st.data(), 27 * L.n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      CK(cudaMemcpyAsync(L.dinv, dinv.data(), L.n * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      CS(dalloc(ctx, &L.xt, L.n));
      CS(dalloc(ctx, &L.r, L.n));
    }
    CS(dalloc(ctx, &L.b, L.n));
    CS(dalloc(ctx, &L.x, L.n));
    H.lv.push_back(L);
    if (coarsest) {
      std::vector<double> A = stencil_dense(st, vx, vy, vz);
      if (!dense_inverse((int)L.n, A)) return fail(ctx, DGMG_ERR_ARG, "coarse matrix is singular");
      H.coarse_n = (int)L.n;
      CS(dalloc(ctx, &H.coarse_inv, A.size()));
      CK(cudaMemcpyAsync(H.coarse_inv, A.data(), A.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      break;
    }
    int cx, cy, cz;
    st = coarsen_stencil(st, vx, vy, vz, cx, cy, cz);
    vx = cx;
    vy = cy;
    vz = cz;
  }
  CK(cudaStreamSynchronize(ctx->stream));   // the host stencils above must outlive their copies
  H.built = true;
  return DGMG_OK;
}

// The P0 hierarchy, built on first use (not under stream capture).
dgmg_status ensure_p0(dgmg_ctx* ctx) {
  if (ctx->p0h.built) return DGMG_OK;
  if (ctx->stream) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(ctx, DGMG_ERR_STATE, "run one uncaptured solve with the P0 coarse space before stream capture");
  }
  return build_hier(ctx, ctx->p0h, p0_stencil(host_mesh(ctx)), ctx->nx, ctx->ny, ctx->nz);
}

dgmg_status restrict_internal(dgmg_ctx* ctx, const void* r, double* rhat, bool fp32) {
  const MeshParams mp = params(ctx);
  CK(ctx->ops->restrict_cells(mp, r, ctx->corners, fp32, ctx->stream));
  CK(restrict_gather(ctx->nx, ctx->ny, ctx->nz, ctx->corners, rhat, ctx->stream));
  return DGMG_OK;
}

dgmg_status timed_apply(dgmg_ctx* ctx, const void* u, void* v, int prec, bool outer = false);

// ------------------------------------------------------------------ V-cycle
// One V-cycle of Algorithm 1 on FP64 f, u (u updated in place; zero: u == 0 on entry).
dgmg_status vcycle_internal(dgmg_ctx* ctx, const double* f, double* u, const dgmg_solve_opts& o, bool zero) {
  Range range("dgmg V-cycle");
  const int prec = o.smoother_prec;
  const bool fp32 = prec == DGMG_FP32;
  const MeshParams mp = params(ctx);
  const long long n = ctx->ndof;
  void *F, *U, *T1, *T2;
  if (fp32) {
    F = ctx->w32[0];
    U = ctx->w32[1];
    T1 = ctx->w32[2];
    T2 = ctx->w32[3];
    CK(vec_d2f(n, f, (float*)F, ctx->stream));
    if (!zero) CK(vec_d2f(n, u, (float*)U, ctx->stream));
  } else {
    F = (void*)f;
    U = u;
    T1 = ctx->w64[0];
    T2 = ctx->w64[1];
  }
  CS(vcycle_smooth(ctx, o, F, U, T1, o.npre, prec, zero));
  const bool u_zero = zero && o.npre <= 0;
  if (o.coarse == DGMG_COARSE_AMG || o.coarse == DGMG_COARSE_P0) {
    const bool p0 = o.coarse == DGMG_COARSE_P0;
    Hier& H = p0 ? ctx->p0h : ctx->q1h;
    // r = f - A u, restricted to the coarse space
    const void* R = F;
    if (!u_zero) {
      CS(timed_apply(ctx, U, T2, prec));
      if (fp32)
        CK(vec_sub_f(n, (const float*)F, (const float*)T2, (float*)T2, ctx->stream));
      else
        CK(vec_sub(n, (const double*)F, (const double*)T2, (double*)T2, ctx->stream));
      R = T2;
    }
    size_t e0 = ctx->timing ? record_event(ctx) : 0;
    if (p0)
      CK(cell_sums(ctx->ncell, ctx->n * ctx->n * ctx->n, R, H.rhat, fp32, ctx->stream));
    else
      CS(restrict_internal(ctx, R, H.rhat, fp32));
    if (ctx->timing) ctx->ev_transfer.push_back({e0, record_event(ctx)});
    e0 = ctx->timing ? record_event(ctx) : 0;
    CS(coarse_correction(ctx, H, o.coarse_cycles));
    if (ctx->timing) ctx->ev_coarse.push_back({e0, record_event(ctx)});
    e0 = ctx->timing ? record_event(ctx) : 0;
    if (p0)
      CK(cell_add(ctx->ncell, ctx->n * ctx->n * ctx->n, H.uhat, U, fp32, ctx->stream));
    else
      CK(ctx->ops->prolong_add(mp, H.uhat, U, fp32, ctx->stream));
    if (ctx->timing) ctx->ev_transfer.push_back({e0, record_event(ctx)});
    CS(vcycle_smooth(ctx, o, F, U, T1, o.npost, prec, false));
  } else {
    CS(vcycle_smooth(ctx, o, F, U, T1, o.npost, prec, u_zero));
  }
  if (fp32) CK(vec_f2d(n, (const float*)U, u, ctx->stream));
  return DGMG_OK;
}

dgmg_status timed_apply(dgmg_ctx* ctx, const void* u, void* v, int prec, bool outer) {
  Range range("dgmg operator");
  const MeshParams mp = params(ctx);
  const size_t e0 = ctx->timing ? record_event(ctx) : 0;
  if (outer && ctx->var_on)   // the operator with K(x), c(x); the preconditioner keeps cell values
    CK(ctx->ops->apply_var(mp, (const double*)u, (double*)v, ctx->stream));
  else
    CK(ctx->ops->apply(mp, u, v, prec, true, ctx->stream));
  if (ctx->timing) ctx->ev_apply.push_back({e0, record_event(ctx)});
  ++ctx->n_apply;
  return DGMG_OK;
}

dgmg_status ensure_krylov(dgmg_ctx* ctx, size_t nvec) {
  if (ctx->kry_vecs >= nvec) return DGMG_OK;
  if (ctx->kry) {
    for (auto it = ctx->mesh_allocs.begin(); it != ctx->mesh_allocs.end(); ++it)
      if (*it == (void*)ctx->kry) {
        ctx->mesh_allocs.erase(it);
        break;
      }
    cudaFreeAsync(ctx->kry, ctx->stream);
    ctx->kry = nullptr;
    ctx->kry_vecs = 0;
  }
  CS(dalloc(ctx, &ctx->kry, nvec * (size_t)ctx->ndof));
  ctx->kry_vecs = nvec;
  return DGMG_OK;
}

dgmg_status precond_eager(dgmg_ctx* ctx, const double* r, double* z, const dgmg_solve_opts& o) {
  CK(vec_fill(ctx->ndof, 0.0, z, ctx->stream));
  return vcycle_internal(ctx, r, z, o, true);
}

// The options the V-cycle reads.  The outer solver's fields (tolerance,
// iteration cap, Krylov method, stopping rule, operator precision, timing,
// graph) do not change the captured work and stay zero, so solves that
// differ only in those share a graph.
dgmg_solve_opts precond_key(const dgmg_solve_opts& o) {
  dgmg_solve_opts k;
  std::memset(&k, 0, sizeof(k));
  k.smoother_prec = o.smoother_prec;
  k.omega = o.omega;
  k.npre = o.npre;
  k.npost = o.npost;
  k.eps_inner = o.eps_inner;
  k.maxit_inner = o.maxit_inner;
  k.inner = o.inner;
  k.inner_restart = o.inner_restart;
  k.coarse = o.coarse;
  k.coarse_cycles = o.coarse_cycles;
  k.smoother = o.smoother;
  return k;
}

// z = M r.  With opts.graph the V-cycle (no host synchronisation inside) is
// captured into a CUDA graph on its second use with the same (r, z) and
// V-cycle options and replayed afterwards, removing the per-kernel launch
// cost; the launch and sweep counters of the captured work are added on each
// replay.
dgmg_status precond(dgmg_ctx* ctx, const double* r, double* z, const dgmg_solve_opts& o) {
  if (!o.graph || ctx->timing || !ctx->stream) return precond_eager(ctx, r, z, o);
  const dgmg_solve_opts key = precond_key(o);
  for (auto& g : ctx->graphs) {
    if (g.in == r && g.out == z && std::memcmp(&g.opts, &key, sizeof(key)) == 0) {
      if (!g.exec) {   // second use: capture
        const long long s0 = ctx->n_sweep, z0 = ctx->n_zero_sweep, a0 = ctx->n_apply, t0 = ctx->sweeps_tracked;
        const unsigned long long l0 = t_launches;
        CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        dgmg_status st = precond_eager(ctx, r, z, o);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
        if (st != DGMG_OK) {
          if (graph) cudaGraphDestroy(graph);
          return st;
        }
        if (e != cudaSuccess) return fail(ctx, DGMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return fail(ctx, DGMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        g.d_sweep = ctx->n_sweep - s0;
        g.d_zero = ctx->n_zero_sweep - z0;
        g.d_apply = ctx->n_apply - a0;
        g.d_tracked = ctx->sweeps_tracked - t0;
        g.d_launches = t_launches - l0;
        ctx->n_sweep = s0;
        ctx->n_zero_sweep = z0;
        ctx->n_apply = a0;
        ctx->sweeps_tracked = t0;
        t_launches = l0;
      }
      CK(cudaGraphLaunch(g.exec, ctx->stream));
      ctx->n_sweep += g.d_sweep;
      ctx->n_zero_sweep += g.d_zero;
      ctx->n_apply += g.d_apply;
      ctx->sweeps_tracked += g.d_tracked;
      t_launches += g.d_launches;
      return DGMG_OK;
    }
  }
  // first use: run eagerly (sets kernel attributes) and remember the key
  if (ctx->graphs.size() < 64) {
    dgmg_ctx::PrecGraph g = {};
    g.in = r;
    g.out = z;
    g.opts = key;
    g.exec = nullptr;
    ctx->graphs.push_back(g);
  }
  return precond_eager(ctx, r, z, o);
}

// Outer Krylov operator: FP64 vectors, FP64 or double-float arithmetic.
dgmg_status apply64(dgmg_ctx* ctx, const double* u, double* v, int prec = DGMG_FP64) {
  return timed_apply(ctx, u, v, prec == DGMG_DF64 ? DGMG_DF64 : DGMG_FP64, true);
}

dgmg_status solve_cg(dgmg_ctx* ctx, const double* f, double* u, const dgmg_solve_opts& o, dgmg_solve_stats& st) {
  const long long n = ctx->ndof;
  const bool flex = o.krylov == DGMG_KRYLOV_FCG;
  CS(ensure_krylov(ctx, flex ? 5 : 4));
  double* r = ctx->kry;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  double* ro = flex ? q + n : nullptr;
  CS(apply64(ctx, u, q));
  CK(vec_sub(n, f, q, r, ctx->stream));
  double rr;
  CS(dot(ctx, r, r, rr));
  const double r0 = std::sqrt(rr);
  st.iterations = 0;
  if (!std::isfinite(r0)) return fail(ctx, DGMG_ERR_ARG, "initial residual is not finite (NaN or Inf in f or u)");
  if (r0 == 0.0) {
    st.converged = 1;
    st.rel_residual = 0.0;
    return DGMG_OK;
  }
  CS(precond(ctx, r, z, o));
  CK(vec_copy(n, z, p, ctx->stream));
  double rz;
  CS(dot(ctx, r, z, rz));
  dgmg_status result = DGMG_ERR_NOT_CONVERGED;
  const bool energy = o.stop == DGMG_STOP_ENERGY;
  std::vector<double> terms;   // alpha_j (r_j, z_j), the energy-norm estimate's terms
  bool est_met = false;
  for (int it = 1; it <= o.maxit; ++it) {
    CS(apply64(ctx, p, q, o.apply_prec));
    double pq;
    CS(dot(ctx, p, q, pq));
    if (!(pq > 0.0)) {
      result = DGMG_ERR_BREAKDOWN;
      ctx->err = "CG breakdown: p^T A p <= 0";
      break;
    }
    const double alpha = rz / pq;
    terms.push_back(alpha * rz);
    CK(vec_axpby(n, alpha, p, 1.0, u, ctx->stream));
    if (flex) CK(vec_copy(n, r, ro, ctx->stream));
    CK(vec_axpby(n, -alpha, q, 1.0, r, ctx->stream));
    CS(dot(ctx, r, r, rr));
    st.iterations = it;
    st.iterations_run = it;
    if (energy) {
      if (it >= o.delay) {
        const int k = it - o.delay;
        double nu = 0.0, tot = 0.0;
        for (int j = k; j < it; ++j) nu += terms[j];
        for (int j = 0; j < it; ++j) tot += terms[j];
        st.energy_estimate = std::sqrt(nu / tot);
        st.iterations = k;
        if (st.energy_estimate <= o.rtol) {
          est_met = true;
          result = DGMG_OK;
          break;
        }
      }
    } else if (std::sqrt(rr) <= o.rtol * r0) {
      result = DGMG_OK;
      break;
    }
    CS(precond(ctx, r, z, o));
    double rzn;
    CS(dot(ctx, r, z, rzn));
    double num = rzn;
    if (flex) {
      double zro;
      CS(dot(ctx, z, ro, zro));
      num = rzn - zro;
    }
    const double beta = num / rz;
    rz = rzn;
    CK(vec_axpby(n, 1.0, z, beta, p, ctx->stream));
  }
  // true residual in FP64
  CS(apply64(ctx, u, q));
  CK(vec_sub(n, f, q, r, ctx->stream));
  CS(dot(ctx, r, r, rr));
  st.rel_residual = std::sqrt(rr) / r0;
  st.converged = (energy ? est_met : st.rel_residual <= o.rtol * (1.0 + 1e-6)) ? 1 : 0;
  if (result == DGMG_ERR_NOT_CONVERGED) ctx->err = "outer Krylov solve reached maxit";
  return result == DGMG_OK && !st.converged ? DGMG_ERR_NOT_CONVERGED : result;
}

dgmg_status solve_fgmres(dgmg_ctx* ctx, const double* f, double* u, const dgmg_solve_opts& o, dgmg_solve_stats& st) {
  const long long n = ctx->ndof;
  const int m = o.restart;
  if (m < 1 || m + 1 > kMaxDots) return fail(ctx, DGMG_ERR_ARG, "restart must be in [1, 71]");
  CS(ensure_krylov(ctx, 2 * (size_t)m + 2));
  double* r = ctx->kry;
  std::vector<double*> V(m + 1), Z(m);
  for (int i = 0; i <= m; ++i) V[i] = r + (size_t)(i + 1) * n;
  for (int i = 0; i < m; ++i) Z[i] = r + (size_t)(m + 2 + i) * n;
  CS(apply64(ctx, u, V[0]));
  CK(vec_sub(n, f, V[0], r, ctx->stream));
  double rr;
  CS(dot(ctx, r, r, rr));
  const double r0 = std::sqrt(rr);
  st.iterations = 0;
  if (!std::isfinite(r0)) return fail(ctx, DGMG_ERR_ARG, "initial residual is not finite (NaN or Inf in f or u)");
  if (r0 == 0.0) {
    st.converged = 1;
    st.rel_residual = 0.0;
    return DGMG_OK;
  }
  double beta = r0;
  int it = 0;
  dgmg_status result = DGMG_ERR_NOT_CONVERGED;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), h(m + 1), h2(m + 1), y(m);
  while (it < o.maxit) {
    CK(vec_axpby(n, 1.0 / beta, r, 0.0, V[0], ctx->stream));
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int k = 0;
    bool done = false;
    for (int j = 0; j < m; ++j) {
      CS(precond(ctx, V[j], Z[j], o));
      CS(apply64(ctx, Z[j], V[j + 1], o.apply_prec));
      CS(multi_dot(ctx, j + 1, V.data(), V[j + 1], h.data()));
      for (int i = 0; i <= j; ++i) CK(vec_axpby(n, -h[i], V[i], 1.0, V[j + 1], ctx->stream));
      CS(multi_dot(ctx, j + 1, V.data(), V[j + 1], h2.data()));
      for (int i = 0; i <= j; ++i) CK(vec_axpby(n, -h2[i], V[i], 1.0, V[j + 1], ctx->stream));
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = h[i] + h2[i];
      double ww;
      CS(dot(ctx, V[j + 1], V[j + 1], ww));
      const double hn = std::sqrt(ww);
      H[(size_t)(j + 1) * m + j] = hn;
      if (hn > 0.0) CK(vec_axpby(n, 0.0, V[j + 1], 1.0 / hn, V[j + 1], ctx->stream));
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * H[(size_t)i * m + j] + sn[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)(i + 1) * m + j] = -sn[i] * H[(size_t)i * m + j] + cs[i] * H[(size_t)(i + 1) * m + j];
        H[(size_t)i * m + j] = t;
      }
      const double den = std::hypot(H[(size_t)j * m + j], H[(size_t)(j + 1) * m + j]);
      if (den == 0.0) {
        result = DGMG_ERR_BREAKDOWN;
        ctx->err = "FGMRES breakdown";
        done = true;
        break;
      }
      cs[j] = H[(size_t)j * m + j] / den;
      sn[j] = H[(size_t)(j + 1) * m + j] / den;
      H[(size_t)j * m + j] = den;
      H[(size_t)(j + 1) * m + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++it;
      k = j + 1;
      if (std::fabs(g[j + 1]) <= o.rtol * r0 || it >= o.maxit) break;
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int l = i + 1; l < k; ++l) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    for (int i = 0; i < k; ++i) CK(vec_axpby(n, y[i], Z[i], 1.0, u, ctx->stream));
    CS(apply64(ctx, u, V[0]));
    CK(vec_sub(n, f, V[0], r, ctx->stream));
    CS(dot(ctx, r, r, rr));
    beta = std::sqrt(rr);
    st.iterations = it;
    if (beta <= o.rtol * r0) {
      result = DGMG_OK;
      break;
    }
    if (done) break;
  }
  st.rel_residual = beta / r0;
  st.converged = st.rel_residual <= o.rtol * (1.0 + 1e-6) ? 1 : 0;
  if (result == DGMG_ERR_NOT_CONVERGED) ctx->err = "outer Krylov solve reached maxit";
  return result;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

void dgmg_default_opts(dgmg_solve_opts* o) {
  if (!o) return;
  o->krylov = DGMG_KRYLOV_CG;
  o->restart = 30;
  o->rtol = 1e-8;
  o->maxit = 500;
  o->smoother_prec = DGMG_FP64;
  o->omega = 0.8;
  o->npre = 1;
  o->npost = 1;
  o->eps_inner = 1e-2;
  o->maxit_inner = 0;
  o->inner = DGMG_INNER_PCG;
  o->inner_restart = 12;
  o->coarse = DGMG_COARSE_AMG;
  o->timing = 0;
  o->coarse_cycles = 1;
  o->smoother = DGMG_SMOOTHER_JACOBI;
  o->apply_prec = DGMG_FP64;
  o->graph = 0;
  o->stop = DGMG_STOP_RESIDUAL;
  o->delay = 4;
}

dgmg_status dgmg_create(dgmg_ctx** out, int device, void* cuda_stream) {
  if (!out) return DGMG_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return DGMG_ERR_ARG;
  }
  dgmg_ctx* ctx = new dgmg_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) {
    for (int n = kMinN; n <= kMaxN && e == cudaSuccess; ++n) {
      const std::vector<double> t = build_tables(n);
      e = cell_ops(n)->upload_tables(t.data(), ctx->stream);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->dot_partial, sizeof(double) * kDotBlocks * kMaxDots);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->dot_out, sizeof(double) * kMaxDots);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->dot_ptrs, sizeof(double*) * kMaxDots);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->dot_host, sizeof(double) * kMaxDots);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return DGMG_ERR_CUDA;
  }
  *out = ctx;
  return DGMG_OK;
}

dgmg_status dgmg_destroy(dgmg_ctx* ctx) {
  if (!ctx) return DGMG_ERR_ARG;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  free_mesh(ctx);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
  drop_graphs(ctx);
  cudaFree(ctx->dot_partial);
  cudaFree(ctx->dot_out);
  cudaFree(ctx->dot_ptrs);
  cudaFreeHost(ctx->dot_host);
  delete ctx;
  return DGMG_OK;
}

const char* dgmg_last_error(const dgmg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

dgmg_status dgmg_set_mesh(dgmg_ctx* ctx, int nx, int ny, int nz, double lx, double ly, double lz, int p,
                          const int bc[6]) {
  if (!ctx) return DGMG_ERR_ARG;
  if (nx < 1 || ny < 1 || nz < 1) return fail(ctx, DGMG_ERR_ARG, "nx, ny, nz must be >= 1");
  if (!(lx > 0) || !(ly > 0) || !(lz > 0)) return fail(ctx, DGMG_ERR_ARG, "lengths must be > 0");
  if (p < kMinN - 1 || p > kMaxN - 1) return fail(ctx, DGMG_ERR_ARG, "p must be in [1, 8]");
  if (!bc) return fail(ctx, DGMG_ERR_ARG, "bc is NULL");
  for (int i = 0; i < 6; ++i)
    if (bc[i] != 0 && bc[i] != 1) return fail(ctx, DGMG_ERR_ARG, "bc values must be 0 or 1");
  const long long ncell = (long long)nx * ny * nz;
  const long long n3 = (long long)(p + 1) * (p + 1) * (p + 1);
  if (ncell * n3 > (1LL << 40)) return fail(ctx, DGMG_ERR_ARG, "mesh too large");
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  free_mesh(ctx);
  ctx->nx = nx;
  ctx->ny = ny;
  ctx->nz = nz;
  ctx->p = p;
  ctx->n = p + 1;
  ctx->L[0] = lx;
  ctx->L[1] = ly;
  ctx->L[2] = lz;
  ctx->h[0] = lx / nx;
  ctx->h[1] = ly / ny;
  ctx->h[2] = lz / nz;
  for (int i = 0; i < 6; ++i) ctx->bc[i] = bc[i];
  ctx->ncell = ncell;
  ctx->ndof = ncell * n3;
  ctx->nvert = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  ctx->ops = cell_ops(p + 1);
  for (int i = 0; i < 3; ++i) ctx->wpb_apply[i] = ctx->wpb_smooth[i] = ctx->lay_apply[i] = ctx->lay_smooth[i] = 0;
  ctx->has_mesh = true;
  ctx->has_coef = false;
  return DGMG_OK;
}

dgmg_status dgmg_set_penalty(dgmg_ctx* ctx, double alpha) {
  if (!ctx) return DGMG_ERR_ARG;
  if (!(alpha > 0.0) || !std::isfinite(alpha)) return fail(ctx, DGMG_ERR_ARG, "alpha must be finite and > 0");
  if (ctx->has_coef) return fail(ctx, DGMG_ERR_STATE, "set the penalty before the coefficients");
  ctx->alpha = alpha;
  return DGMG_OK;
}

dgmg_status dgmg_set_coefficients(dgmg_ctx* ctx, const double* K, int kdim, const double* b_vertex,
                                  const double* c_cell) {
  if (!ctx) return DGMG_ERR_ARG;
  if (!ctx->has_mesh) return fail(ctx, DGMG_ERR_STATE, "set_mesh first");
  if (!K || (kdim != 1 && kdim != 3)) return fail(ctx, DGMG_ERR_ARG, "K must be non-NULL with kdim 1 or 3");
  const long long nK = ctx->ncell * kdim;
  for (long long i = 0; i < nK; ++i)
    if (!(K[i] > 0.0) || !std::isfinite(K[i])) return fail(ctx, DGMG_ERR_ARG, "K must be finite and > 0");
  if (c_cell)
    for (long long i = 0; i < ctx->ncell; ++i)
      if (!std::isfinite(c_cell[i])) return fail(ctx, DGMG_ERR_ARG, "c must be finite");
  if (b_vertex)
    for (long long i = 0; i < 3 * ctx->nvert; ++i)
      if (!std::isfinite(b_vertex[i])) return fail(ctx, DGMG_ERR_ARG, "b must be finite");
  Range range("dgmg set-up");
  CK(cudaSetDevice(ctx->device));
  if (ctx->stream) CK(cudaStreamSynchronize(ctx->stream));
  free_mesh(ctx);
  ctx->kdim = kdim;
  ctx->hK.assign(K, K + nK);
  ctx->hb.assign(b_vertex ? b_vertex : K, b_vertex ? b_vertex + 3 * ctx->nvert : K);
  ctx->hc.assign(c_cell ? c_cell : K, c_cell ? c_cell + ctx->ncell : K);
  const long long n = ctx->ndof;
  CS(dalloc(ctx, &ctx->dK, nK));
  CK(cudaMemcpyAsync(ctx->dK, K, nK * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  if (b_vertex) {
    CS(dalloc(ctx, &ctx->db, 3 * ctx->nvert));
    CK(cudaMemcpyAsync(ctx->db, b_vertex, 3 * ctx->nvert * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    CS(dalloc(ctx, &ctx->db32, 3 * ctx->nvert));
    CK(vec_d2f(3 * ctx->nvert, ctx->db, ctx->db32, ctx->stream));
  }
  if (c_cell) {
    CS(dalloc(ctx, &ctx->dc, ctx->ncell));
    CK(cudaMemcpyAsync(ctx->dc, c_cell, ctx->ncell * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  }
  CS(dalloc(ctx, &ctx->diag64, n));
  CS(dalloc(ctx, &ctx->diag32, n));
  CS(dalloc(ctx, &ctx->dinv64, n));
  CS(dalloc(ctx, &ctx->dinv32, n));
  CS(dalloc(ctx, &ctx->rec64, kRecLen * ctx->ncell));
  CS(dalloc(ctx, &ctx->rec32, kRecLen * ctx->ncell));
  for (auto& w : ctx->w64) CS(dalloc(ctx, &w, n));
  for (auto& w : ctx->w32) CS(dalloc(ctx, &w, n));
  CS(dalloc(ctx, &ctx->corners, 8 * ctx->ncell));
  CS(dalloc(ctx, &ctx->its, ctx->ncell));
  CS(dalloc(ctx, &ctx->itsum, 2));
  CS(dalloc(ctx, &ctx->itmax, 1));
  const MeshParams mp = params(ctx);
  CK(cell_records(mp, ctx->rec64, ctx->rec32, ctx->stream));
  CK(ctx->ops->diag(mp, ctx->diag64, ctx->stream));
  CK(vec_d2f(n, ctx->diag64, ctx->diag32, ctx->stream));
  CK(vec_inverse(n, ctx->diag64, ctx->dinv64, ctx->dinv32, ctx->stream));
  // Q1 matrix and AMG hierarchy (host setup, device cycle)
  CS(build_hier(ctx, ctx->q1h, q1_stencil(host_mesh(ctx)), ctx->nx + 1, ctx->ny + 1, ctx->nz + 1));
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  ctx->has_coef = true;
  return DGMG_OK;
}

dgmg_status dgmg_sizes(const dgmg_ctx* ctx, long long* ndof, long long* nvert, long long* ncell, long long* nvol_qp,
                       long long* nface_qp) {
  if (!ctx || !ctx->has_mesh) return DGMG_ERR_STATE;
  const long long m2 = (long long)ctx->n * ctx->n;
  if (ndof) *ndof = ctx->ndof;
  if (nvert) *nvert = ctx->nvert;
  if (ncell) *ncell = ctx->ncell;
  if (nvol_qp) *nvol_qp = ctx->ncell * m2 * ctx->n;
  if (nface_qp)
    *nface_qp = 2 * ((long long)ctx->ny * ctx->nz + (long long)ctx->nx * ctx->nz + (long long)ctx->nx * ctx->ny) * m2;
  return DGMG_OK;
}

dgmg_status dgmg_quadrature_points(const dgmg_ctx* cctx, double* vol_xyz, double* face_xyz) {
  if (!cctx || !cctx->has_mesh) return DGMG_ERR_STATE;
  HostMesh hm;
  hm.nx = cctx->nx;
  hm.ny = cctx->ny;
  hm.nz = cctx->nz;
  hm.p = cctx->p;
  for (int d = 0; d < 3; ++d) hm.h[d] = cctx->h[d];
  quadrature_points_host(hm, vol_xyz, face_xyz);
  return DGMG_OK;
}

dgmg_status dgmg_assemble_rhs(dgmg_ctx* ctx, const double* f_qp, const double* g_qp, const double* j_qp,
                              double* rhs) {
  CS(ready(ctx));
  if (!rhs) return fail(ctx, DGMG_ERR_ARG, "rhs is NULL");
  std::vector<double> h((size_t)ctx->ndof, 0.0);
  assemble_rhs_host(host_mesh(ctx), f_qp, g_qp, j_qp, h.data());
  CK(cudaMemcpyAsync(rhs, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return DGMG_OK;
}

dgmg_status dgmg_apply(dgmg_ctx* ctx, const void* u, void* v, dgmg_prec prec) {
  CS(ready(ctx));
  if (!u || !v || u == v) return fail(ctx, DGMG_ERR_ARG, "u, v must be distinct non-NULL device pointers");
  if (prec != DGMG_FP64 && prec != DGMG_FP32 && prec != DGMG_DF64) return fail(ctx, DGMG_ERR_ARG, "bad precision");
  CS(check_df64(ctx, prec, DGMG_INNER_PCG));
  if (ctx->var_on) {
    if (prec != DGMG_FP64) return fail(ctx, DGMG_ERR_ARG, "the operator with K(x), c(x) is FP64");
    CK(ctx->ops->apply_var(params(ctx), (const double*)u, (double*)v, ctx->stream));
    return DGMG_OK;
  }
  CK(ctx->ops->apply(params(ctx), u, v, prec, true, ctx->stream));
  return DGMG_OK;
}

dgmg_status dgmg_block_apply(dgmg_ctx* ctx, const void* u, void* v, dgmg_prec prec) {
  CS(ready(ctx));
  if (!u || !v || u == v) return fail(ctx, DGMG_ERR_ARG, "u, v must be distinct non-NULL device pointers");
  if (prec != DGMG_FP64 && prec != DGMG_FP32 && prec != DGMG_DF64) return fail(ctx, DGMG_ERR_ARG, "bad precision");
  CS(check_df64(ctx, prec, DGMG_INNER_PCG));
  CK(ctx->ops->apply(params(ctx), u, v, prec, false, ctx->stream));
  return DGMG_OK;
}

dgmg_status dgmg_block_diagonal(dgmg_ctx* ctx, void* diag, dgmg_prec prec) {
  CS(ready(ctx));
  if (!diag) return fail(ctx, DGMG_ERR_ARG, "diag is NULL");
  const size_t bytes = ctx->ndof * (prec == DGMG_FP32 ? 4 : 8);
  CK(cudaMemcpyAsync(diag, prec == DGMG_FP32 ? (const void*)ctx->diag32 : (const void*)ctx->diag64, bytes,
                     cudaMemcpyDeviceToDevice, ctx->stream));
  return DGMG_OK;
}

dgmg_status dgmg_block_smooth(dgmg_ctx* ctx, const void* f, void* u, int nsweep, double omega, double eps, int maxit,
                              int inner, int inner_restart, dgmg_prec prec, int* inner_its) {
  CS(ready(ctx));
  if (!f || !u || f == u) return fail(ctx, DGMG_ERR_ARG, "f, u must be distinct non-NULL device pointers");
  if (nsweep < 0 || !(eps >= 0.0) || !std::isfinite(omega)) return fail(ctx, DGMG_ERR_ARG, "bad sweep arguments");
  if (prec != DGMG_FP64 && prec != DGMG_FP32 && prec != DGMG_DF64) return fail(ctx, DGMG_ERR_ARG, "bad precision");
  CS(check_df64(ctx, prec, inner));
  void* tmp = prec == DGMG_FP32 ? (void*)ctx->w32[3] : (void*)ctx->w64[2];
  return smooth_internal(ctx, f, u, tmp, nsweep, omega, eps, maxit, inner, inner_restart, prec, false, inner_its);
}

dgmg_status dgmg_block_sor(dgmg_ctx* ctx, const void* f, void* u, int nsweep, double omega, double eps, int maxit,
                           int inner, int inner_restart, int symmetric, dgmg_prec prec, int* inner_its) {
  CS(ready(ctx));
  if (!f || !u || f == u) return fail(ctx, DGMG_ERR_ARG, "f, u must be distinct non-NULL device pointers");
  if (nsweep < 0 || !(eps >= 0.0) || !std::isfinite(omega)) return fail(ctx, DGMG_ERR_ARG, "bad sweep arguments");
  if (prec != DGMG_FP64 && prec != DGMG_FP32 && prec != DGMG_DF64) return fail(ctx, DGMG_ERR_ARG, "bad precision");
  CS(check_df64(ctx, prec, inner));
  return sor_internal(ctx, f, u, nsweep, omega, eps, maxit, inner, inner_restart, prec, false, symmetric != 0,
                      inner_its);
}

dgmg_status dgmg_restrict(dgmg_ctx* ctx, const void* r, double* r_hat, dgmg_prec prec) {
  CS(ready(ctx));
  if (!r || !r_hat) return fail(ctx, DGMG_ERR_ARG, "NULL pointer");
  return restrict_internal(ctx, r, r_hat, prec == DGMG_FP32);
}

dgmg_status dgmg_prolong_add(dgmg_ctx* ctx, const double* u_hat, void* u, dgmg_prec prec) {
  CS(ready(ctx));
  if (!u || !u_hat) return fail(ctx, DGMG_ERR_ARG, "NULL pointer");
  CK(ctx->ops->prolong_add(params(ctx), u_hat, u, prec == DGMG_FP32, ctx->stream));
  return DGMG_OK;
}

dgmg_status dgmg_coarse_matrix(const dgmg_ctx* ctx, double* stencil) {
  if (!ctx || !ctx->has_coef) return DGMG_ERR_STATE;
  if (!stencil) return DGMG_ERR_ARG;
  std::memcpy(stencil, ctx->q1h.st.data(), ctx->q1h.st.size() * sizeof(double));
  return DGMG_OK;
}

dgmg_status dgmg_coarse_cycle(dgmg_ctx* ctx, const double* r_hat, double* u_hat) {
  CS(ready(ctx));
  if (!r_hat || !u_hat || r_hat == u_hat) return fail(ctx, DGMG_ERR_ARG, "r_hat, u_hat must be distinct");
  return amg_cycle(ctx, ctx->q1h, 0, r_hat, u_hat);
}

dgmg_status dgmg_restrict_p0(dgmg_ctx* ctx, const void* r, double* r_hat, dgmg_prec prec) {
  CS(ready(ctx));
  if (!r || !r_hat) return fail(ctx, DGMG_ERR_ARG, "NULL pointer");
  if (prec != DGMG_FP64 && prec != DGMG_FP32) return fail(ctx, DGMG_ERR_ARG, "bad precision");
  CK(cell_sums(ctx->ncell, ctx->n * ctx->n * ctx->n, r, r_hat, prec == DGMG_FP32, ctx->stream));
  return DGMG_OK;
}

dgmg_status dgmg_prolong_add_p0(dgmg_ctx* ctx, const double* u_hat, void* u, dgmg_prec prec) {
  CS(ready(ctx));
  if (!u || !u_hat) return fail(ctx, DGMG_ERR_ARG, "NULL pointer");
  if (prec != DGMG_FP64 && prec != DGMG_FP32) return fail(ctx, DGMG_ERR_ARG, "bad precision");
  CK(cell_add(ctx->ncell, ctx->n * ctx->n * ctx->n, u_hat, u, prec == DGMG_FP32, ctx->stream));
  return DGMG_OK;
}

dgmg_status dgmg_coarse_matrix_p0(dgmg_ctx* ctx, double* stencil) {
  CS(ready(ctx));
  if (!stencil) return fail(ctx, DGMG_ERR_ARG, "NULL pointer");
  CS(ensure_p0(ctx));
  std::memcpy(stencil, ctx->p0h.st.data(), ctx->p0h.st.size() * sizeof(double));
  return DGMG_OK;
}

dgmg_status dgmg_coarse_cycle_p0(dgmg_ctx* ctx, const double* r_hat, double* u_hat) {
  CS(ready(ctx));
  if (!r_hat || !u_hat || r_hat == u_hat) return fail(ctx, DGMG_ERR_ARG, "r_hat, u_hat must be distinct");
  CS(ensure_p0(ctx));
  return amg_cycle(ctx, ctx->p0h, 0, r_hat, u_hat);
}

dgmg_status dgmg_vcycle(dgmg_ctx* ctx, const double* f, double* u, const dgmg_solve_opts* opts) {
  CS(ready(ctx));
  if (!f || !u || f == u) return fail(ctx, DGMG_ERR_ARG, "f, u must be distinct non-NULL device pointers");
  dgmg_solve_opts o;
  dgmg_default_opts(&o);
  if (opts) o = *opts;
  if (o.npre < 0 || o.npost < 0) return fail(ctx, DGMG_ERR_ARG, "npre, npost must be >= 0");
  if (o.coarse < DGMG_COARSE_AMG || o.coarse > DGMG_COARSE_P0) return fail(ctx, DGMG_ERR_ARG, "bad coarse");
  CS(prepare_inner(ctx, o.inner, o.smoother_prec));
  if (o.coarse == DGMG_COARSE_P0) CS(ensure_p0(ctx));
  return vcycle_internal(ctx, f, u, o, false);
}

dgmg_status dgmg_solve(dgmg_ctx* ctx, const double* f, double* u, const dgmg_solve_opts* opts,
                       dgmg_solve_stats* stats) {
  CS(ready(ctx));
  if (!f || !u || f == u) return fail(ctx, DGMG_ERR_ARG, "f, u must be distinct non-NULL device pointers");
  dgmg_solve_opts o;
  dgmg_default_opts(&o);
  if (opts) o = *opts;
  if (!(o.rtol > 0.0) || o.maxit < 1) return fail(ctx, DGMG_ERR_ARG, "rtol > 0 and maxit >= 1 required");
  if (o.krylov < DGMG_KRYLOV_CG || o.krylov > DGMG_KRYLOV_FGMRES) return fail(ctx, DGMG_ERR_ARG, "bad krylov");
  if (o.smoother_prec < DGMG_FP64 || o.smoother_prec > DGMG_DF64) return fail(ctx, DGMG_ERR_ARG, "bad smoother_prec");
  CS(check_df64(ctx, o.smoother_prec, o.inner));
  CS(check_df64(ctx, o.apply_prec, DGMG_INNER_PCG));
  if (ctx->var_on && o.apply_prec == DGMG_DF64) return fail(ctx, DGMG_ERR_ARG, "the operator with K(x), c(x) is FP64");
  if (o.coarse < DGMG_COARSE_AMG || o.coarse > DGMG_COARSE_P0) return fail(ctx, DGMG_ERR_ARG, "bad coarse");
  if (o.stop != DGMG_STOP_RESIDUAL && o.stop != DGMG_STOP_ENERGY) return fail(ctx, DGMG_ERR_ARG, "bad stop");
  if (o.stop == DGMG_STOP_ENERGY && (o.krylov == DGMG_KRYLOV_FGMRES || o.delay < 1))
    return fail(ctx, DGMG_ERR_ARG, "the energy-norm estimate needs CG or flexible CG and delay >= 1");
  CS(prepare_inner(ctx, o.inner, o.smoother_prec));
  if (o.coarse == DGMG_COARSE_P0) CS(ensure_p0(ctx));
  Range range("dgmg solve");
  dgmg_solve_stats st;
  std::memset(&st, 0, sizeof(st));
  const auto t0 = std::chrono::steady_clock::now();
  ctx->track_its = stats != nullptr;
  ctx->sweeps_tracked = 0;
  ctx->timing = o.timing != 0;
  ctx->ev_used = 0;
  ctx->ev_smooth.clear();
  ctx->ev_apply.clear();
  ctx->ev_transfer.clear();
  ctx->ev_coarse.clear();
  ctx->n_apply = ctx->n_sweep = ctx->n_zero_sweep = 0;
  const unsigned long long launches0 = t_launches;
  const size_t ev_begin = ctx->timing ? record_event(ctx) : 0;
  if (ctx->track_its) {
    CK(cudaMemsetAsync(ctx->itsum, 0, 2 * sizeof(unsigned long long), ctx->stream));
    CK(cudaMemsetAsync(ctx->itmax, 0, sizeof(int), ctx->stream));
  }
  dgmg_status s = o.krylov == DGMG_KRYLOV_FGMRES ? solve_fgmres(ctx, f, u, o, st) : solve_cg(ctx, f, u, o, st);
  if (st.iterations_run == 0) st.iterations_run = st.iterations;
  const size_t ev_end = ctx->timing ? record_event(ctx) : 0;
  ctx->track_its = false;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fail(ctx, DGMG_ERR_CUDA, cudaGetErrorString(e));
  st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  st.kernel_launches = (long long)(t_launches - launches0);
  st.sweeps = ctx->n_sweep;
  st.zero_sweeps = ctx->n_zero_sweep;
  st.applies = ctx->n_apply;
  if (ctx->timing) {
    auto total = [ctx](const std::vector<std::pair<size_t, size_t>>& pairs) {
      double t = 0.0;
      float ms;
      for (auto& pr : pairs)
        if (cudaEventElapsedTime(&ms, ctx->ev[pr.first], ctx->ev[pr.second]) == cudaSuccess) t += ms;
      return t;
    };
    st.ms_smooth = total(ctx->ev_smooth);
    st.ms_apply = total(ctx->ev_apply);
    st.ms_transfer = total(ctx->ev_transfer);
    st.ms_coarse = total(ctx->ev_coarse);
    st.ms_device = total({{ev_begin, ev_end}});
    st.ms_krylov = std::max(0.0, st.ms_device - st.ms_smooth - st.ms_apply - st.ms_transfer - st.ms_coarse);
    ctx->timing = false;
  }
  if (stats) {
    unsigned long long sum[2] = {0, 0};
    int mx = 0;
    cudaMemcpyAsync(sum, ctx->itsum, sizeof(sum), cudaMemcpyDeviceToHost, ctx->stream);
    cudaMemcpyAsync(&mx, ctx->itmax, sizeof(mx), cudaMemcpyDeviceToHost, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    const long long sw = ctx->sweeps_tracked;
    const double cnt = (double)ctx->ncell * (double)sw;
    st.inner_mean = sw > 0 ? (double)sum[0] / cnt : 0.0;
    st.inner_std = sw > 0 ? std::sqrt(std::max(0.0, (double)sum[1] / cnt - st.inner_mean * st.inner_mean)) : 0.0;
    st.inner_its_total = (long long)sum[0];
    st.inner_max = mx;
    *stats = st;
  }
  return s;
}

dgmg_status dgmg_set_variable_coefficients(dgmg_ctx* ctx, const double* basis, const double* p0, const double* p2,
                                           double gamma) {
  if (!ctx) return DGMG_ERR_ARG;
  if (!ctx->has_mesh) return fail(ctx, DGMG_ERR_STATE, "set_mesh first");
  if (!basis || !p0 || !p2) return fail(ctx, DGMG_ERR_ARG, "NULL pointer");
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double d = 0.0;
      for (int k = 0; k < 3; ++k) d += basis[3 * i + k] * basis[3 * j + k];
      if (!(std::fabs(d - (i == j ? 1.0 : 0.0)) <= 1e-12)) return fail(ctx, DGMG_ERR_ARG, "basis rows must be orthonormal");
    }
  for (int k = 0; k < 3; ++k)
    if (!(p0[k] > 0.0) || !(p2[k] >= 0.0) || !std::isfinite(p0[k]) || !std::isfinite(p2[k]))
      return fail(ctx, DGMG_ERR_ARG, "p0 > 0 and p2 >= 0 required");
  if (!(gamma >= 0.0) || !std::isfinite(gamma)) return fail(ctx, DGMG_ERR_ARG, "gamma >= 0 required");
  std::vector<double> vp(16);
  for (int i = 0; i < 9; ++i) vp[i] = basis[i];
  for (int k = 0; k < 3; ++k) {
    vp[9 + k] = p0[k];
    vp[12 + k] = p2[k];
  }
  vp[15] = gamma;
  // the preconditioner's coefficients: K and c at the cell centres (the
  // diagonal of the tensor), as the paper evaluates them (Sec. 4.2)
  std::vector<double> Kc(3 * ctx->ncell), cc(ctx->ncell);
  for (long long c = 0; c < ctx->ncell; ++c) {
    const long long cx = c % ctx->nx, cy = (c / ctx->nx) % ctx->ny, cz = c / ((long long)ctx->nx * ctx->ny);
    const double x[3] = {(cx + 0.5) * ctx->h[0], (cy + 0.5) * ctx->h[1], (cz + 0.5) * ctx->h[2]};
    double K[6];
    var_tensor(vp.data(), x, K);
    for (int d = 0; d < 3; ++d) Kc[3 * c + d] = K[d];
    cc[c] = gamma * (x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  }
  CS(dgmg_set_coefficients(ctx, Kc.data(), 3, nullptr, gamma > 0.0 ? cc.data() : nullptr));
  CS(dalloc(ctx, &ctx->dvar, 16));
  CK(cudaMemcpyAsync(ctx->dvar, vp.data(), 16 * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->hvar = vp;
  ctx->var_on = true;
  return DGMG_OK;
}

dgmg_status dgmg_block_inverse(dgmg_ctx* ctx, dgmg_prec prec, void* out) {
  CS(ready(ctx));
  CS(ensure_binv(ctx, prec));
  if (out) {
    const int nb = ctx->n * ctx->n * ctx->n;
    if (prec == DGMG_FP32)
      CK(cudaMemcpy2DAsync(out, nb * sizeof(float), ctx->binv32, ctx->binv_ld * sizeof(float), nb * sizeof(float),
                           (size_t)ctx->ncell * nb, cudaMemcpyDeviceToDevice, ctx->stream));
    else
      CK(blocks_df_to_dense(ctx->ncell, nb, ctx->binv_ld, ctx->binv_df, (double*)out, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return DGMG_OK;
}

dgmg_status dgmg_set_launch_shape(dgmg_ctx* ctx, dgmg_prec prec, int wpb_apply, int wpb_smooth) {
  if (!ctx) return DGMG_ERR_ARG;
  if (!ctx->has_mesh) return fail(ctx, DGMG_ERR_STATE, "set_mesh first");
  if (prec != DGMG_FP64 && prec != DGMG_FP32 && prec != DGMG_DF64) return fail(ctx, DGMG_ERR_ARG, "bad precision");
  auto ok = [](int w) { return w == 0 || w == 1 || w == 2 || w == 4 || w == 8; };
  if (!ok(wpb_apply) || !ok(wpb_smooth)) return fail(ctx, DGMG_ERR_ARG, "warps per block must be 0, 1, 2, 4 or 8");
  drop_graphs(ctx);   // captured graphs hold the old launch shapes
  ctx->wpb_apply[prec] = wpb_apply;
  ctx->wpb_smooth[prec] = wpb_smooth;
  return DGMG_OK;
}

dgmg_status dgmg_set_layout(dgmg_ctx* ctx, dgmg_prec prec, int layout_apply, int layout_smooth) {
  if (!ctx) return DGMG_ERR_ARG;
  if (!ctx->has_mesh) return fail(ctx, DGMG_ERR_STATE, "set_mesh first");
  if (prec != DGMG_FP64 && prec != DGMG_FP32 && prec != DGMG_DF64) return fail(ctx, DGMG_ERR_ARG, "bad precision");
  if (!layout_exists(ctx, prec, layout_apply) || !layout_exists(ctx, prec, layout_smooth))
    return fail(ctx, DGMG_ERR_ARG, "no such layout for this precision and order");
  drop_graphs(ctx);   // captured graphs hold the old kernels
  ctx->lay_apply[prec] = layout_apply;
  ctx->lay_smooth[prec] = layout_smooth;
  return DGMG_OK;
}

dgmg_status dgmg_get_layout(const dgmg_ctx* cctx, dgmg_prec prec, int* layout_apply, int* layout_smooth) {
  if (!cctx) return DGMG_ERR_ARG;
  dgmg_ctx* ctx = const_cast<dgmg_ctx*>(cctx);
  if (!ctx->has_mesh) return fail(ctx, DGMG_ERR_STATE, "set_mesh first");
  if (prec != DGMG_FP64 && prec != DGMG_FP32 && prec != DGMG_DF64) return fail(ctx, DGMG_ERR_ARG, "bad precision");
  if (layout_apply) *layout_apply = resolve_layout(ctx, prec, ctx->lay_apply[prec], false);
  if (layout_smooth) *layout_smooth = resolve_layout(ctx, prec, ctx->lay_smooth[prec], true);
  return DGMG_OK;
}

dgmg_status dgmg_autotune(dgmg_ctx* ctx, dgmg_prec prec, int reps, int* wpb_apply, int* wpb_smooth) {
  if (!ctx) return DGMG_ERR_ARG;
  CS(ready(ctx));
  if (prec != DGMG_FP64 && prec != DGMG_FP32 && prec != DGMG_DF64) return fail(ctx, DGMG_ERR_ARG, "bad precision");
  CS(check_df64(ctx, prec, DGMG_INNER_PCG));
  if (reps <= 0) reps = 3;
  cudaSetDevice(ctx->device);
  const size_t es = prec == DGMG_FP32 ? 4 : 8;
  void* buf = nullptr;
  CK(cudaMallocAsync(&buf, 3 * ctx->ndof * es, ctx->stream));
  char* f = (char*)buf;
  char* u = f + ctx->ndof * es;
  char* t = u + ctx->ndof * es;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  dgmg_status st = DGMG_OK;
  const int cand[4] = {1, 2, 4, 8};
  std::vector<int> lays = {DGMG_LAYOUT_LINE, DGMG_LAYOUT_ELEMENT};
  if (layout_exists(ctx, prec, DGMG_LAYOUT_PLANE)) lays.push_back(DGMG_LAYOUT_PLANE);

  int best[2] = {0, 0}, best_lay[2] = {0, 0};
  const int saved_a = ctx->wpb_apply[prec], saved_s = ctx->wpb_smooth[prec];
  const int saved_la = ctx->lay_apply[prec], saved_ls = ctx->lay_smooth[prec];
  const bool saved_track = ctx->track_its, saved_timing = ctx->timing;
  ctx->track_its = false;
  ctx->timing = false;
  auto run = [&]() -> dgmg_status {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
      return fail(ctx, DGMG_ERR_CUDA, "event create");
    if (prec == DGMG_FP32)
      CK(vec_fill_f(ctx->ndof, 1.f, (float*)f, ctx->stream));
    else
      CK(vec_fill(ctx->ndof, 1.0, (double*)f, ctx->stream));
    for (int kind = 0; kind < 2; ++kind) {
      float best_ms = 0.f;
      for (int lay : lays) {
        for (int w : cand) {
          if (kind == 0) {
            ctx->wpb_apply[prec] = w;
            ctx->lay_apply[prec] = lay;
          } else {
            ctx->wpb_smooth[prec] = w;
            ctx->lay_smooth[prec] = lay;
          }
          const MeshParams mp = params(ctx);
          float total = 0.f;
          for (int r = 0; r <= reps; ++r) {
            CK(cudaEventRecord(e0, ctx->stream));
            if (kind == 0) {
              CK(ctx->ops->apply(mp, f, u, prec, true, ctx->stream));
            } else {
              // the inner solver a solve takes by default: PCG, GMRES(12) with advection
              CS(smooth_internal(ctx, f, u, t, 1, 1.0, 1e-2, 0, ctx->db ? DGMG_INNER_GMRES : DGMG_INNER_PCG,
                                 12, prec, true, nullptr));
            }
            CK(cudaEventRecord(e1, ctx->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            if (r > 0) total += ms;   // r = 0 is the warm-up
          }
          if (best[kind] == 0 || total < best_ms) {
            best[kind] = w;
            best_lay[kind] = lay;
            best_ms = total;
          }
        }
      }
    }
    return DGMG_OK;
  };
  st = run();
  ctx->track_its = saved_track;
  ctx->timing = saved_timing;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(buf, ctx->stream);
  cudaStreamSynchronize(ctx->stream);
  if (st != DGMG_OK) {
    ctx->wpb_apply[prec] = saved_a;
    ctx->wpb_smooth[prec] = saved_s;
    ctx->lay_apply[prec] = saved_la;
    ctx->lay_smooth[prec] = saved_ls;
    return st;
  }
  drop_graphs(ctx);
  ctx->wpb_apply[prec] = best[0];
  ctx->wpb_smooth[prec] = best[1];
  ctx->lay_apply[prec] = best_lay[0];
  ctx->lay_smooth[prec] = best_lay[1];
  if (wpb_apply) *wpb_apply = best[0];
  if (wpb_smooth) *wpb_smooth = best[1];
  return DGMG_OK;
}

}  // extern "C"

// ====================================================================== batched solves
// A batch runs the outer CG / flexible CG of up to kMaxBatch prepared requests
// of one order in lockstep on one stream: every step of an iteration (the
// operator, the dots, the scalar updates, the vector updates, the V-cycle's
// smoothers, residual, transfers) is one launch over the cells or values of
// all running members, reading each member's scalars from device memory, so
// an iteration needs no host round trip and is replayed from a CUDA graph
// while the membership stays the same.  Only the AMG cycles on the members'
// coarse grids run member by member.  Per member the arithmetic is that of
// dgmg_solve with the same options (the same kernels, the same reduction
// order of every dot), so a request's result does not depend on the others.
struct dgmg_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  dgmg_solve_opts opts;
  struct Member {
    bool used = false;
    bool running = false;     // in the launches of the next step
    bool finished = false;    // stopped (converged, breakdown or iteration cap)
    bool final_done = false;  // final true residual computed
    dgmg_ctx* ctx = nullptr;
    cudaStream_t saved_stream = nullptr;
    const double* f = nullptr;
    double* u = nullptr;
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *ro = nullptr;
    double r0 = 0.0, rtol = 1e-8;
    dgmg_solve_stats st;
    dgmg_status status = DGMG_OK;
  };
  Member m[kMaxBatch];
  double* sc = nullptr;        // kMaxBatch * kScLen device scalars
  double* sc_host = nullptr;   // pinned copy
  double* partial = nullptr;   // kMaxBatch * kDotBlocks dot partials
  std::vector<int> order;      // running slots, in launch order
  bool order_valid = false;
  cudaGraphExec_t graph = nullptr;
  int graph_state = 0;         // 0: run eagerly once, 1: capture on the next iteration, 2: replay
};

namespace {

dgmg_status fail_b(dgmg_batch* b, dgmg_status s, const std::string& msg) {
  b->err = msg;
  return s;
}

#define BK(expr)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail_b(b, DGMG_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// A member's context call; its message becomes the batch's.
#define BS(ctx, expr)                                 \
  do {                                                \
    dgmg_status s_ = (expr);                          \
    if (s_ != DGMG_OK) return fail_b(b, s_, (ctx)->err); \
  } while (0)

void batch_invalidate(dgmg_batch* b) {
  b->order_valid = false;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_state = 0;
}

void batch_order(dgmg_batch* b) {
  if (b->order_valid) return;
  b->order.clear();
  for (int i = 0; i < kMaxBatch; ++i)
    if (b->m[i].used && b->m[i].running) b->order.push_back(i);
  b->order_valid = true;
}

// Segment table over the running members: vectors picked by `pick`.
template <typename F>
SegTable seg_table(dgmg_batch* b, long long len_scale, F pick) {
  SegTable t;
  t.k = (int)b->order.size();
  for (int i = 0; i < t.k; ++i) {
    dgmg_batch::Member& mb = b->m[b->order[i]];
    t.n[i] = mb.ctx->ndof * len_scale;
    t.sc[i] = b->sc + (size_t)b->order[i] * kScLen;
    pick(mb, t, i);
  }
  return t;
}

BatchTable cell_table(dgmg_batch* b) {
  BatchTable t;
  t.k = (int)b->order.size();
  for (int i = 0; i < t.k; ++i) t.mp[i] = params(b->m[b->order[i]].ctx);
  return t;
}

// z = V(r) for every running member (Algorithm 1 with one pre- and one
// post-sweep of block-Jacobi, inner PCG, Q1 + AMG): the steps of
// vcycle_internal from a zero initial guess, each as one launch over the
// members except the AMG cycles.
dgmg_status batch_vcycle(dgmg_batch* b) {
  const dgmg_solve_opts& o = b->opts;
  const int prec = o.smoother_prec;
  const bool fp32 = prec == DGMG_FP32;
  const CellOps* ops = b->m[b->order[0]].ctx->ops;
  const int K = (int)b->order.size();
  auto F = [&](dgmg_batch::Member& mb) -> void* { return fp32 ? (void*)mb.ctx->w32[0] : (void*)mb.r; };
  auto U = [&](dgmg_batch::Member& mb) -> void* { return fp32 ? (void*)mb.ctx->w32[1] : (void*)mb.z; };
  auto T1 = [&](dgmg_batch::Member& mb) -> void* { return fp32 ? (void*)mb.ctx->w32[2] : (void*)mb.ctx->w64[0]; };
  auto T2 = [&](dgmg_batch::Member& mb) -> void* { return fp32 ? (void*)mb.ctx->w32[3] : (void*)mb.ctx->w64[1]; };
  const int n3 = b->m[b->order[0]].ctx->n * b->m[b->order[0]].ctx->n * b->m[b->order[0]].ctx->n;
  const int maxit = o.maxit_inner > 0 ? o.maxit_inner : n3;
  if (fp32) {
    SegTable t = seg_table(b, 1, [&](dgmg_batch::Member& mb, SegTable& s, int i) {
      s.a[i] = mb.r;
      s.c[i] = F(mb);
    });
    BK(seg_op(SEG_D2F, t, b->stream));
  }
  auto sweep = [&](bool zero) -> dgmg_status {
    BatchTable t = cell_table(b);
    for (int i = 0; i < K; ++i) {
      dgmg_batch::Member& mb = b->m[b->order[i]];
      t.in[i] = F(mb);
      t.uold[i] = zero ? nullptr : U(mb);
      t.out[i] = T1(mb);
      t.diag[i] = fp32 ? (const void*)mb.ctx->dinv32 : (const void*)mb.ctx->dinv64;
    }
    t.omega = o.omega;
    t.eps = o.eps_inner;
    t.maxit = maxit;
    BK(ops->smooth_batch(t, prec, b->stream));
    SegTable c = seg_table(b, 1, [&](dgmg_batch::Member& mb, SegTable& s, int i) {
      s.a[i] = T1(mb);
      s.c[i] = U(mb);
    });
    BK(seg_op(fp32 ? SEG_COPY32 : SEG_COPY64, c, b->stream));
    return DGMG_OK;
  };
  CS(sweep(true));
  {  // residual F - A U into T2
    BatchTable t = cell_table(b);
    for (int i = 0; i < K; ++i) {
      dgmg_batch::Member& mb = b->m[b->order[i]];
      t.in[i] = U(mb);
      t.out[i] = T2(mb);
    }
    BK(ops->apply_batch(t, prec, true, b->stream));
    SegTable s = seg_table(b, 1, [&](dgmg_batch::Member& mb, SegTable& st, int i) {
      st.a[i] = F(mb);
      st.b[i] = T2(mb);
      st.c[i] = T2(mb);
    });
    BK(seg_op(fp32 ? SEG_SUB32 : SEG_SUB64, s, b->stream));
  }
  {  // restriction to Q1, AMG per member, prolongation
    BatchTable t = cell_table(b);
    for (int i = 0; i < K; ++i) {
      dgmg_batch::Member& mb = b->m[b->order[i]];
      t.in[i] = T2(mb);
      t.out[i] = mb.ctx->corners;
    }
    BK(ops->restrict_batch(t, fp32, b->stream));
    for (int i = 0; i < K; ++i) {
      dgmg_ctx* ctx = b->m[b->order[i]].ctx;
      BK(restrict_gather(ctx->nx, ctx->ny, ctx->nz, ctx->corners, ctx->q1h.rhat, b->stream));
      BS(ctx, coarse_correction(ctx, ctx->q1h, o.coarse_cycles));
    }
    BatchTable pt = cell_table(b);
    for (int i = 0; i < K; ++i) {
      dgmg_batch::Member& mb = b->m[b->order[i]];
      pt.in[i] = mb.ctx->q1h.uhat;
      pt.out[i] = U(mb);
    }
    BK(ops->prolong_batch(pt, fp32, b->stream));
  }
  CS(sweep(false));
  if (fp32) {
    SegTable t = seg_table(b, 1, [&](dgmg_batch::Member& mb, SegTable& s, int i) {
      s.a[i] = U(mb);
      s.c[i] = mb.z;
    });
    BK(seg_op(SEG_F2D, t, b->stream));
  }
  return DGMG_OK;
}

// One outer iteration of every running member (the loop body of solve_cg).
dgmg_status batch_iteration(dgmg_batch* b) {
  const dgmg_solve_opts& o = b->opts;
  const CellOps* ops = b->m[b->order[0]].ctx->ops;
  const int K = (int)b->order.size();
  const bool flex = o.krylov == DGMG_KRYLOV_FCG;
  {  // q = A p
    BatchTable t = cell_table(b);
    for (int i = 0; i < K; ++i) {
      t.in[i] = b->m[b->order[i]].p;
      t.out[i] = b->m[b->order[i]].q;
    }
    BK(ops->apply_batch(t, o.apply_prec == DGMG_DF64 ? DGMG_DF64 : DGMG_FP64, true, b->stream));
  }
  SegTable pq = seg_table(b, 1, [&](dgmg_batch::Member& mb, SegTable& s, int i) {
    s.a[i] = mb.p;
    s.b[i] = mb.q;
  });
  BK(seg_dot(pq, b->partial, kScPq, b->stream));
  BK(seg_scalar(SC_ALPHA, pq, b->stream));
  SegTable up = seg_table(b, 1, [&](dgmg_batch::Member& mb, SegTable& s, int i) {
    s.a[i] = mb.p;
    s.b[i] = mb.q;
    s.c[i] = mb.u;
    s.d[i] = mb.r;
    s.e[i] = mb.ro;
  });
  BK(seg_op(SEG_ALPHA, up, b->stream));
  SegTable rr = seg_table(b, 1, [&](dgmg_batch::Member& mb, SegTable& s, int i) {
    s.a[i] = mb.r;
    s.b[i] = mb.r;
  });
  BK(seg_dot(rr, b->partial, kScRr, b->stream));
  BK(seg_scalar(SC_CONV, rr, b->stream));
  CS(batch_vcycle(b));
  SegTable rz = seg_table(b, 1, [&](dgmg_batch::Member& mb, SegTable& s, int i) {
    s.a[i] = mb.r;
    s.b[i] = mb.z;
  });
  BK(seg_dot(rz, b->partial, kScRzn, b->stream));
  if (flex) {
    SegTable zr = seg_table(b, 1, [&](dgmg_batch::Member& mb, SegTable& s, int i) {
      s.a[i] = mb.z;
      s.b[i] = mb.ro;
    });
    BK(seg_dot(zr, b->partial, kScZro, b->stream));
  }
  BK(seg_scalar(SC_BETA, rz, b->stream));
  SegTable pu = seg_table(b, 1, [&](dgmg_batch::Member& mb, SegTable& s, int i) {
    s.a[i] = mb.z;
    s.c[i] = mb.p;
  });
  BK(seg_op(SEG_P, pu, b->stream));
  return DGMG_OK;
}

// Final true residual of a stopped member and its statistics (as dgmg_solve).
dgmg_status batch_finish(dgmg_batch* b, dgmg_batch::Member& mb, const double* sc) {
  dgmg_ctx* ctx = mb.ctx;
  const long long n = ctx->ndof;
  std::memset(&mb.st, 0, sizeof(mb.st));
  if (mb.r0 == 0.0) {
    mb.st.converged = 1;
    mb.status = DGMG_OK;
    mb.final_done = true;
    return DGMG_OK;
  }
  const int state = (int)sc[kScDone];
  mb.st.iterations = (int)sc[kScIts];
  mb.st.iterations_run = mb.st.iterations;
  BS(ctx, apply64(ctx, mb.u, mb.q));
  BK(vec_sub(n, mb.f, mb.q, mb.r, b->stream));
  double rr = 0.0;
  BS(ctx, dot(ctx, mb.r, mb.r, rr));
  mb.st.rel_residual = std::sqrt(rr) / mb.r0;
  mb.st.converged = mb.st.rel_residual <= mb.rtol * (1.0 + 1e-6) ? 1 : 0;
  if (state == 2) {
    mb.status = DGMG_ERR_BREAKDOWN;
  } else {
    mb.status = mb.st.converged ? DGMG_OK : DGMG_ERR_NOT_CONVERGED;
  }
  mb.final_done = true;
  return DGMG_OK;
}

// The options that shape a batched member's iterates (its initial state
// included): the Krylov method and the V-cycle's.
dgmg_solve_opts batch_key(const dgmg_solve_opts& o) {
  dgmg_solve_opts k = precond_key(o);
  k.krylov = o.krylov;
  k.apply_prec = o.apply_prec;
  return k;
}

// r = f - A u, ||r||, z = M r, p = z, (r, z) on the context's stream: the
// steps of solve_cg before its loop, kept in the context for dgmg_batch_add.
dgmg_status prime_internal(dgmg_ctx* ctx, const double* f, double* u, const dgmg_solve_opts& o) {
  const bool flex = o.krylov == DGMG_KRYLOV_FCG;
  const long long n = ctx->ndof;
  ctx->primed = false;
  CS(ensure_krylov(ctx, flex ? 5 : 4));
  double* r = ctx->kry;
  double* z = r + n;
  double* p = z + n;
  double* q = p + n;
  CS(apply64(ctx, u, q));
  CK(vec_sub(n, f, q, r, ctx->stream));
  double rr = 0.0;
  CS(dot(ctx, r, r, rr));
  const double r0 = std::sqrt(rr);
  if (!std::isfinite(r0)) return fail(ctx, DGMG_ERR_ARG, "initial residual is not finite (NaN or Inf in f or u)");
  double rz = 0.0;
  if (r0 != 0.0) {
    dgmg_solve_opts po = o;
    po.graph = 0;
    po.timing = 0;
    CS(precond(ctx, r, z, po));
    CK(vec_copy(n, z, p, ctx->stream));
    CS(dot(ctx, r, z, rz));
  }
  ctx->prime_f = f;
  ctx->prime_u = u;
  ctx->prime_r0 = r0;
  ctx->prime_rz = rz;
  ctx->prime_key = batch_key(o);
  ctx->primed = true;
  return DGMG_OK;
}

}  // namespace

extern "C" {

dgmg_status dgmg_batch_create(dgmg_batch** out, int device, void* cuda_stream, const dgmg_solve_opts* opts) {
  if (!out) return DGMG_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return DGMG_ERR_ARG;
  }
  dgmg_solve_opts o;
  dgmg_default_opts(&o);
  if (opts) o = *opts;
  if (o.krylov != DGMG_KRYLOV_CG && o.krylov != DGMG_KRYLOV_FCG) return DGMG_ERR_ARG;
  if (o.smoother_prec < DGMG_FP64 || o.smoother_prec > DGMG_DF64) return DGMG_ERR_ARG;
  if (o.apply_prec != DGMG_FP64 && o.apply_prec != DGMG_DF64) return DGMG_ERR_ARG;
  if (o.inner != DGMG_INNER_PCG || o.smoother != DGMG_SMOOTHER_JACOBI || o.coarse != DGMG_COARSE_AMG ||
      o.npre != 1 || o.npost != 1 || o.stop != DGMG_STOP_RESIDUAL || o.coarse_cycles < 1)
    return DGMG_ERR_ARG;
  dgmg_batch* b = new dgmg_batch();
  b->device = device;
  b->stream = (cudaStream_t)cuda_stream;
  b->opts = o;
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->sc, sizeof(double) * kMaxBatch * kScLen);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->partial, sizeof(double) * kMaxBatch * kDotBlocks);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->sc_host, sizeof(double) * kMaxBatch * kScLen);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (b->sc) cudaFree(b->sc);
    if (b->partial) cudaFree(b->partial);
    delete b;
    return DGMG_ERR_CUDA;
  }
  *out = b;
  return DGMG_OK;
}

dgmg_status dgmg_batch_destroy(dgmg_batch* b) {
  if (!b) return DGMG_ERR_ARG;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  for (int i = 0; i < kMaxBatch; ++i)
    if (b->m[i].used) b->m[i].ctx->stream = b->m[i].saved_stream;
  batch_invalidate(b);
  cudaFree(b->sc);
  cudaFree(b->partial);
  cudaFreeHost(b->sc_host);
  delete b;
  return DGMG_OK;
}

const char* dgmg_batch_last_error(const dgmg_batch* b) { return b ? b->err.c_str() : "null batch"; }

dgmg_status dgmg_batch_prime(dgmg_ctx* ctx, const double* f, double* u, const dgmg_solve_opts* opts) {
  CS(ready(ctx));
  if (!f || !u || f == u) return fail(ctx, DGMG_ERR_ARG, "f, u must be distinct non-NULL device pointers");
  dgmg_solve_opts o;
  dgmg_default_opts(&o);
  if (opts) o = *opts;
  if (o.krylov != DGMG_KRYLOV_CG && o.krylov != DGMG_KRYLOV_FCG) return fail(ctx, DGMG_ERR_ARG, "CG or FCG only");
  CS(check_df64(ctx, o.smoother_prec, o.inner));
  CS(check_df64(ctx, o.apply_prec, DGMG_INNER_PCG));
  cudaSetDevice(ctx->device);
  return prime_internal(ctx, f, u, o);
}

dgmg_status dgmg_batch_add(dgmg_batch* b, dgmg_ctx* ctx, const double* f, double* u, double rtol, int maxit,
                           int* slot) {
  if (!b || !ctx || !slot) return DGMG_ERR_ARG;
  *slot = -1;
  if (ready(ctx) != DGMG_OK) return fail_b(b, DGMG_ERR_STATE, "the context needs a mesh and coefficients");
  if (!f || !u || f == u) return fail_b(b, DGMG_ERR_ARG, "f, u must be distinct non-NULL device pointers");
  if (!(rtol > 0.0) || maxit < 1) return fail_b(b, DGMG_ERR_ARG, "rtol > 0 and maxit >= 1 required");
  if (ctx->device != b->device) return fail_b(b, DGMG_ERR_ARG, "the context is on another device");
  if (ctx->db || ctx->var_on) return fail_b(b, DGMG_ERR_ARG, "batched solves cover b = 0 with cell-wise K, c");
  int free_slot = -1;
  for (int i = 0; i < kMaxBatch; ++i) {
    if (b->m[i].used) {
      if (b->m[i].ctx == ctx) return fail_b(b, DGMG_ERR_ARG, "the context is already in the batch");
      if (b->m[i].ctx->n != ctx->n) return fail_b(b, DGMG_ERR_ARG, "the members of a batch share the order p");
      const MeshParams a = params(b->m[i].ctx), c = params(ctx);
      for (int k = 0; k < 3; ++k)
        if (a.lay_apply[k] != c.lay_apply[k] || a.lay_smooth[k] != c.lay_smooth[k])
          return fail_b(b, DGMG_ERR_ARG, "the members of a batch share the kernel layouts");
    } else if (free_slot < 0) {
      free_slot = i;
    }
  }
  if (free_slot < 0) return fail_b(b, DGMG_ERR_ARG, "the batch is full");
  const dgmg_solve_opts& o = b->opts;
  if (check_df64(ctx, o.smoother_prec, o.inner) != DGMG_OK || check_df64(ctx, o.apply_prec, DGMG_INNER_PCG) != DGMG_OK)
    return fail_b(b, DGMG_ERR_ARG, ctx->err);
  cudaSetDevice(b->device);
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return fail_b(b, DGMG_ERR_CUDA, "context stream");
  dgmg_batch::Member& mb = b->m[free_slot];
  mb = dgmg_batch::Member();
  mb.used = true;
  mb.ctx = ctx;
  mb.saved_stream = ctx->stream;
  ctx->stream = b->stream;   // the member's work runs on the batch's stream while it belongs to it
  mb.f = f;
  mb.u = u;
  mb.rtol = rtol;
  auto undo = [&](dgmg_status s) {
    ctx->stream = mb.saved_stream;
    mb.used = false;
    return fail_b(b, s, ctx->err);
  };
  const bool flex = o.krylov == DGMG_KRYLOV_FCG;
  const long long n = ctx->ndof;
  const dgmg_solve_opts key = batch_key(o);
  const bool primed = ctx->primed && ctx->prime_f == f && ctx->prime_u == u &&
                      std::memcmp(&ctx->prime_key, &key, sizeof(key)) == 0;
  ctx->primed = false;
  if (!primed) {   // the initial state on the batch's stream
    dgmg_status s = prime_internal(ctx, f, u, o);
    if (s != DGMG_OK) return undo(s);
  }
  mb.r = ctx->kry;
  mb.z = mb.r + n;
  mb.p = mb.z + n;
  mb.q = mb.p + n;
  mb.ro = flex ? mb.q + n : nullptr;
  mb.r0 = ctx->prime_r0;
  double* sc = b->sc_host + (size_t)free_slot * kScLen;
  for (int k = 0; k < kScLen; ++k) sc[k] = 0.0;
  if (mb.r0 == 0.0) {
    mb.finished = true;
    mb.running = false;
  } else {
    sc[kScRz] = ctx->prime_rz;
    sc[kScR0] = mb.r0;
    sc[kScRtol] = rtol;
    sc[kScMaxit] = (double)maxit;
    sc[kScFlex] = flex ? 1.0 : 0.0;
    mb.running = true;
  }
  BK(cudaMemcpyAsync(b->sc + (size_t)free_slot * kScLen, sc, sizeof(double) * kScLen, cudaMemcpyHostToDevice,
                     b->stream));
  BK(cudaStreamSynchronize(b->stream));
  batch_invalidate(b);
  *slot = free_slot;
  return DGMG_OK;
}

dgmg_status dgmg_batch_step(dgmg_batch* b, int iterations, int* running) {
  if (!b || iterations < 0) return DGMG_ERR_ARG;
  cudaSetDevice(b->device);
  batch_order(b);
  if (!b->order.empty()) {
    for (int it = 0; it < iterations; ++it) {
      if (!b->stream) {   // the legacy default stream cannot be captured: eager launches
        CS(batch_iteration(b));
      } else if (b->graph_state == 2) {
        BK(cudaGraphLaunch(b->graph, b->stream));
      } else if (b->graph_state == 0) {   // first iteration of this membership: eager (sets kernel attributes)
        CS(batch_iteration(b));
        b->graph_state = 1;
      } else {
        BK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        dgmg_status s = batch_iteration(b);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (s != DGMG_OK) {
          if (g) cudaGraphDestroy(g);
          return s;
        }
        if (e != cudaSuccess) return fail_b(b, DGMG_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail_b(b, DGMG_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        b->graph_state = 2;
        BK(cudaGraphLaunch(b->graph, b->stream));
      }
    }
  }
  BK(cudaMemcpyAsync(b->sc_host, b->sc, sizeof(double) * kMaxBatch * kScLen, cudaMemcpyDeviceToHost, b->stream));
  BK(cudaStreamSynchronize(b->stream));
  int left = 0;
  for (int i : b->order) {
    if (b->sc_host[(size_t)i * kScLen + kScDone] != 0.0) {
      b->m[i].running = false;
      b->m[i].finished = true;
      batch_invalidate(b);
    } else {
      ++left;
    }
  }
  if (running) *running = left;
  return DGMG_OK;
}

dgmg_status dgmg_batch_poll(dgmg_batch* b, int slot, int* done, dgmg_solve_stats* stats) {
  if (!b || slot < 0 || slot >= kMaxBatch || !b->m[slot].used || !done) return DGMG_ERR_ARG;
  dgmg_batch::Member& mb = b->m[slot];
  *done = mb.finished ? 1 : 0;
  if (!mb.finished) return DGMG_OK;
  if (!mb.final_done) {
    cudaSetDevice(b->device);
    CS(batch_finish(b, mb, b->sc_host + (size_t)slot * kScLen));
  }
  if (stats) *stats = mb.st;
  return mb.status;
}

dgmg_status dgmg_batch_remove(dgmg_batch* b, int slot) {
  if (!b || slot < 0 || slot >= kMaxBatch || !b->m[slot].used) return DGMG_ERR_ARG;
  cudaSetDevice(b->device);
  BK(cudaStreamSynchronize(b->stream));
  dgmg_batch::Member& mb = b->m[slot];
  mb.ctx->stream = mb.saved_stream;
  mb = dgmg_batch::Member();
  batch_invalidate(b);
  return DGMG_OK;
}

}  // extern "C"
