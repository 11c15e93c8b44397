// Constraint norms without any device allocation.
//
// lbnr_constraints() reduces through a per-context workspace that the library
// (or the caller, through lbnr_opts.dev_buffer) allocates. Some callers cannot
// make that allocation: a run that has given almost all of the GPU's memory
// to its distribution buffers (a lattice sized to fill HBM leaves no room, and
// an allocation attempted mid-run would fail with out-of-memory), or a host
// framework whose own allocator owns the device memory and forbids other
// allocations while its step runs. For them this file offers one entry point,
// lbnr_constraint_norms_noalloc(), that takes the corrected fields and the
// output already on the device and keeps its per-block partial sums in a
// fixed array compiled into the library.
//
// The array lives in every GPU that loads the library until the process
// exits. Its size bounds the lattice: at most kNoAllocMaxCells cells.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/lbnr.h"
#include "dispatch.h"
#include "kernels.cuh"

namespace lbnr {
namespace {

constexpr int64_t kNoAllocMaxCells = LBNR_NOALLOC_MAX_CELLS;
constexpr int kBlock = 128;  // block size of k_constraints64 below
constexpr int64_t kMaxBlocks = (kNoAllocMaxCells + kBlock - 1) / kBlock;
constexpr int kPartialStride = 22;  // k_constraints64 writes 6 values per block at this stride
constexpr int kMaxDevices = 64;

// Per-block partials of the constraint reduction: 16384 x 22 doubles
// (2.75 MiB). Shared by every call on a device; each call writes every slot
// it later reads, so nothing has to start at zero.
static __device__ __align__(256) double g_partials[kMaxBlocks * kPartialStride];

// Device address of g_partials, looked up once per device context (host code
// cannot use the symbol itself: on the host it is only a stand-in). The entry
// is keyed on the context's unique ID, so after a device reset (a new context,
// into which the module is loaded again and where the array may sit at another
// address) the next call looks the address up again instead of reusing a stale
// pointer.
struct SymbolSlot {
  unsigned long long ctx_id;
  void* addr;
};
SymbolSlot g_slot[kMaxDevices] = {};
std::mutex g_slot_mu;

typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

// Unique ID of the calling thread's current context; false when there is none
// yet (the runtime creates it on the first call that needs it) or the driver
// offers no way to ask.
bool current_ctx_id(unsigned long long* id) {
  static PfnCtxGetCurrent get_current = nullptr;
  static PfnCtxGetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<PfnCtxGetCurrent>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<PfnCtxGetId>(p);
  });
  if (!get_current || !get_id) return false;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

// Device address of g_partials in the current device's context.
cudaError_t partials_address(int dev, void** out) {
  unsigned long long id = 0;
  const bool have_id = current_ctx_id(&id);
  std::lock_guard<std::mutex> lock(g_slot_mu);
  if (have_id && g_slot[dev].addr && g_slot[dev].ctx_id == id) {
    *out = g_slot[dev].addr;
    return cudaSuccess;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
  if (e != cudaSuccess) return e;
  if (!p) return cudaErrorInvalidSymbol;
  // the lookup made the context current if it was not yet
  if (!current_ctx_id(&id)) id = 0;
  g_slot[dev].ctx_id = id;
  g_slot[dev].addr = id ? p : nullptr;  // without an ID, look it up every call
  *out = p;
  return cudaSuccess;
}

__global__ void k_noalloc_final(const double* __restrict__ partials, int64_t nblk, int64_t cells,
                                double* __restrict__ out) {
  __shared__ double red[kBlock / 32][6];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < 6; ++i) {
    const bool is_max = (i & 1) != 0;
    double x = 0;
    for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) {
      const double y = partials[b * kPartialStride + i];
      x = is_max ? fmax(x, y) : x + y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = is_max ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[warp][i] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int i = threadIdx.x;
    double x = 0;
    for (int w = 0; w < kBlock / 32; ++w) x = (i & 1) ? fmax(x, red[w][i]) : x + red[w][i];
    out[i] = (i & 1) ? x : sqrt(x / (double)cells);
  }
}

template <int Q>
cudaError_t launch_norms(const double* fields, const Grid& G, double dx, double* partials,
                         double* out, cudaStream_t st) {
  const int64_t nblk = (G.cells + kBlock - 1) / kBlock;
  k_constraints64<Q><<<(unsigned)nblk, kBlock, 0, st>>>(fields, G, 1.0 / (2.0 * dx),
                                                         1.0 / (4.0 * dx), partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_noalloc_final<<<1, kBlock, 0, st>>>(partials, nblk, G.cells, out);
  return cudaGetLastError();
}

int fail_na(int code, const char* msg) {
  set_thread_error(msg);  // readable through lbnr_last_error(NULL)
  return code;
}

}  // namespace
}  // namespace lbnr

extern "C" int lbnr_constraint_norms_noalloc(int vset, const lbnr_grid* grid, double dx,
                                              const double* d_fields, double* d_out,
                                              void* cuda_stream) {
  using namespace lbnr;
  if (!grid || !d_fields || !d_out) return fail_na(LBNR_EINVAL, "null argument");
  if (vset < LBNR_D1Q3 || vset > LBNR_D3Q19) return fail_na(LBNR_EINVAL, "unknown velocity set");
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return fail_na(LBNR_EINVAL, "empty lattice");
  if ((vset == LBNR_D1Q3 && (grid->ny != 1 || grid->nz != 1)) ||
      (vset == LBNR_D2Q9 && grid->nz != 1))
    return fail_na(LBNR_EINVAL, "lattice shape does not match the velocity set");
  if (!(dx > 0)) return fail_na(LBNR_EINVAL, "dx must be positive");
  // Each side first, then the product one factor at a time: every product
  // formed is at most 2^21 * 2^21, so none can overflow.
  const int64_t nx = grid->nx, ny = grid->ny, nz = grid->nz;
  if (nx > kNoAllocMaxCells || ny > kNoAllocMaxCells || nz > kNoAllocMaxCells ||
      nx * ny > kNoAllocMaxCells || nx * ny * nz > kNoAllocMaxCells)
    return fail_na(LBNR_EINVAL,
                   "lattice larger than LBNR_NOALLOC_MAX_CELLS (2^21 cells); use lbnr_constraints");
  const int64_t cells = nx * ny * nz;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail_na(LBNR_ECUDA, "no usable current device");
  void* addr = nullptr;
  e = partials_address(dev, &addr);
  if (e != cudaSuccess) return fail_na(LBNR_ECUDA, cudaGetErrorString(e));
  const Grid G = make_grid((int32_t)nx, (int32_t)ny, (int32_t)nz, cells, cells);
  double* partials = static_cast<double*>(addr);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  switch (vset) {
    case LBNR_D1Q3: e = launch_norms<3>(d_fields, G, dx, partials, d_out, st); break;
    case LBNR_D2Q9: e = launch_norms<9>(d_fields, G, dx, partials, d_out, st); break;
    default: e = launch_norms<19>(d_fields, G, dx, partials, d_out, st); break;
  }
  if (e != cudaSuccess) return fail_na(LBNR_ECUDA, cudaGetErrorString(e));
  return LBNR_OK;
}
