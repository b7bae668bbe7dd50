// dgmg_restrict_noalloc: the DG -> Q1 restriction for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc at all: a host that manages all device
// memory through its own pool and forbids other allocators, or a real-time
// loop that must not wait on the allocator (cudaMalloc can synchronise the
// device).  dgmg_restrict needs a context, and creating a context (and
// setting its coefficients) allocates.  This entry point needs neither: the
// caller passes the input and output vectors and the grid size, and the
// per-cell corner sums live in a file-scope device array of fixed size that
// every GPU loading this library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "dgmg.h"
#include "dgmg_internal.h"
#include "setup_host.h"

namespace dgmg {
namespace {

// Eight corner sums per cell (FP64): 8 MiB for DGMG_NOALLOC_MAX_CELLS cells.
static __device__ __align__(256) double g_corner_scratch[8 * (size_t)DGMG_NOALLOC_MAX_CELLS];

constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

// Once per device, with that device current: upload the 1D tables of every
// order to the kernels' constant memory (a copy into fixed symbols, no
// allocation) and look up the device address of the scratch array (the
// host-side name g_corner_scratch is only a stand-in, not a device address).
cudaError_t setup_device(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev]) {
    *out = g_scratch_addr[dev];
    return cudaSuccess;
  }
  double tables[5 * kMaxTableN * kMaxTableN + 6 * kMaxTableN];
  for (int n = kMinN; n <= kMaxN; ++n) {
    build_tables_into(n, tables);
    cudaError_t e = cell_ops(n)->upload_tables(tables, nullptr);
    if (e != cudaSuccess) return e;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_corner_scratch);
  if (e != cudaSuccess) return e;
  g_scratch_addr[dev] = static_cast<double*>(p);
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace dgmg

extern "C" dgmg_status dgmg_restrict_noalloc(int nx, int ny, int nz, int p, const void* r, double* r_hat,
                                             dgmg_prec prec, void* cuda_stream) {
  using namespace dgmg;
  if (nx < 1 || ny < 1 || nz < 1 || p < kMinN - 1 || p > kMaxN - 1 || !r || !r_hat) return DGMG_ERR_ARG;
  if (prec != DGMG_FP64 && prec != DGMG_FP32) return DGMG_ERR_ARG;
  const long long ncell = (long long)nx * ny * nz;
  if (ncell > DGMG_NOALLOC_MAX_CELLS) return DGMG_ERR_ARG;   // beyond the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return DGMG_ERR_CUDA;
  }
  double* scratch = nullptr;
  if (setup_device(dev, &scratch) != cudaSuccess) {
    cudaGetLastError();
    return DGMG_ERR_CUDA;
  }
  MeshParams mp = {};
  mp.nx = nx;
  mp.ny = ny;
  mp.nz = nz;
  mp.p = p;
  mp.ncell = ncell;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // Every corner entry of the ncell cells is overwritten before it is read, so
  // the scratch left by an earlier call needs no clearing.
  if (cell_ops(p + 1)->restrict_cells(mp, r, scratch, prec == DGMG_FP32, s) != cudaSuccess ||
      restrict_gather(nx, ny, nz, scratch, r_hat, s) != cudaSuccess) {
    cudaGetLastError();
    return DGMG_ERR_CUDA;
  }
  return DGMG_OK;
}
