// C-ABI of the 37-field scheme (lbnr_ad_* in include/lbnr.h): context,
// device memory, the step loop and transfers. Kernels in ad.cuh; one
// instantiation unit per velocity set and storage (ad_q*_f*.cu).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>

#include "ad.cuh"

using namespace lbnr;

struct lbnr_ad_ctx {
  lbnr_grid grid;
  int vset = 0, Q = 0, slicing = 1, storage = LBNR_F64;
  double tau = 0, dx = 0, dt = 0;
  Grid G;
  ad::Table ops;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  void* f[2] = {nullptr, nullptr};
  double* macro = nullptr;  // [37][cells] FP64: fields in, moments out
  int* flag = nullptr;
  int64_t steps = 0;
  bool initialised = false;
  int form = 0;  // launch form of the collide kernel
  std::string err;
};

static thread_local std::string g_ad_err;

static int ad_fail(lbnr_ad_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  g_ad_err = buf;
  return code;
}

#define AD_TRY(ctx, call)                                                                       \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return ad_fail((ctx), LBNR_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),       \
                     __FILE__, __LINE__);                                                       \
  } while (0)

static int64_t ad_cells(const lbnr_ad_ctx* c) { return c->G.cells; }
static void* ad_state(const lbnr_ad_ctx* c) { return c->f[c->steps & 1]; }

extern "C" {

void lbnr_ad_destroy(lbnr_ad_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  if (c->f[0]) cudaFree(c->f[0]);
  if (c->f[1]) cudaFree(c->f[1]);
  if (c->macro) cudaFree(c->macro);
  if (c->flag) cudaFree(c->flag);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
}

int lbnr_ad_create(const lbnr_grid* grid, int vset, double tau, double dx, double dt, int slicing,
                   int storage, void* cuda_stream, lbnr_ad_ctx** out) {
  if (!out) return ad_fail(nullptr, LBNR_EINVAL, "null output pointer");
  *out = nullptr;
  if (!grid) return ad_fail(nullptr, LBNR_EINVAL, "null grid");
  const int Q = vset == LBNR_D1Q3 ? 3 : vset == LBNR_D2Q9 ? 9 : vset == LBNR_D3Q19 ? 19 : 0;
  if (!Q) return ad_fail(nullptr, LBNR_EINVAL, "unknown velocity set %d", vset);
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1)
    return ad_fail(nullptr, LBNR_EINVAL, "grid sizes must be positive");
  if (vset == LBNR_D1Q3 && (grid->ny != 1 || grid->nz != 1))
    return ad_fail(nullptr, LBNR_EINVAL, "D1Q3 needs ny = nz = 1");
  if (vset == LBNR_D2Q9 && grid->nz != 1) return ad_fail(nullptr, LBNR_EINVAL, "D2Q9 needs nz = 1");
  if (grid->nx > (1 << 30) || grid->ny > (1 << 30) || grid->nz > (1 << 30))
    return ad_fail(nullptr, LBNR_EINVAL, "grid side too large");
  const uint64_t cells = (uint64_t)grid->nx * grid->ny * grid->nz;
  const uint64_t ps = (cells + kTile - 1) / kTile * kTile;
  if (cells >= (1ull << 31) || (uint64_t)Q * ps >= (1ull << 32))
    return ad_fail(nullptr, LBNR_EINVAL, "lattice too large (%llu cells)", (unsigned long long)cells);
  if (storage != LBNR_F64 && storage != LBNR_F32)
    return ad_fail(nullptr, LBNR_EINVAL, "storage must be LBNR_F64 or LBNR_F32");
  if (slicing < 0 || slicing > 2) return ad_fail(nullptr, LBNR_EINVAL, "unknown slicing %d", slicing);
  if (!(tau > 0.5) || !(dx > 0) || !(dt > 0) || !std::isfinite(tau) || !std::isfinite(dx) ||
      !std::isfinite(dt))
    return ad_fail(nullptr, LBNR_EINVAL, "need tau > 1/2 and positive dx, dt");
  if (fabs(dt - dx) > 1e-12 * dx) return ad_fail(nullptr, LBNR_EINVAL, "dt must equal dx");
  lbnr_ad_ctx* c = new (std::nothrow) lbnr_ad_ctx;
  if (!c) return ad_fail(nullptr, LBNR_ENOMEM, "out of host memory");
  c->grid = *grid;
  c->vset = vset;
  c->Q = Q;
  c->slicing = slicing;
  c->storage = storage;
  c->tau = tau;
  c->dx = dx;
  c->dt = dt;
  c->G = make_grid(grid->nx, grid->ny, grid->nz, (int64_t)cells, (int64_t)ps);
  // the fastest forms on GB300: registers for 2 blocks per SM (FP64), the
  // staged form with one lane per cell (FP32)
  c->form = storage == LBNR_F64 ? 0 : 4;
  if (storage == LBNR_F64)
    c->ops = Q == 3 ? ad::table_q3_f64() : Q == 9 ? ad::table_q9_f64() : ad::table_q19_f64();
  else
    c->ops = Q == 3 ? ad::table_q3_f32() : Q == 9 ? ad::table_q9_f32() : ad::table_q19_f32();
  // the 37 fields padded to whole words (FP32: 40 slots, FP64: 37)
  const size_t fbytes = storage == LBNR_F64 ? (size_t)ad::kSlots<double> * Q * ps * 8
                                            : (size_t)ad::kSlots<float> * Q * ps * 4;
  cudaError_t e = cudaSuccess;
  if (cuda_stream) {
    c->st = static_cast<cudaStream_t>(cuda_stream);
  } else {
    e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
    c->own_stream = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = cudaMalloc(&c->f[0], fbytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->f[1], fbytes);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&c->macro), sizeof(double) * ad::kNFA * cells);
  if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&c->flag), 256);
  // the plane padding must hold finite values
  if (e == cudaSuccess) e = cudaMemsetAsync(c->f[0], 0, fbytes, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->f[1], 0, fbytes, c->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->flag, 0, 256, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    lbnr_ad_destroy(c);
    return ad_fail(nullptr, e == cudaErrorMemoryAllocation ? LBNR_ENOMEM : LBNR_ECUDA,
                   "create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return LBNR_OK;
}

int lbnr_ad_init(lbnr_ad_ctx* c, const double* fields, int nfields) {
  if (!c || !fields) return ad_fail(c, LBNR_EINVAL, "null context or fields");
  if (nfields != 16 && nfields != ad::kNFA)
    return ad_fail(c, LBNR_EINVAL, "nfields must be 16 or 37");
  const int64_t cells = ad_cells(c);
  for (int64_t i = 0; i < cells; ++i)
    if (!(fields[i] > 0)) return ad_fail(c, LBNR_EINVAL, "alpha must be positive (cell %lld)", (long long)i);
  AD_TRY(c, cudaMemcpyAsync(c->macro, fields, sizeof(double) * nfields * cells,
                            cudaMemcpyHostToDevice, c->st));
  AD_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int), c->st));
  AD_TRY(c, c->ops.init(c->G, c->macro, nfields, c->f[0], c->flag, c->dx, c->dt, c->slicing, c->st));
  AD_TRY(c, cudaStreamSynchronize(c->st));
  c->steps = 0;
  c->initialised = true;
  return LBNR_OK;
}

int lbnr_ad_step(lbnr_ad_ctx* c, int64_t n) {
  if (!c) return ad_fail(c, LBNR_EINVAL, "null context");
  if (!c->initialised) return ad_fail(c, LBNR_ESTATE, "step before init");
  if (n < 0) return ad_fail(c, LBNR_EINVAL, "negative step count");
  for (int64_t i = 0; i < n; ++i) {
    AD_TRY(c, c->ops.step[c->form](c->G, c->f[c->steps & 1], c->f[(c->steps + 1) & 1], c->flag,
                                   c->tau, c->dt, c->slicing, c->st));
    ++c->steps;
  }
  return LBNR_OK;
}

int lbnr_ad_step_timed(lbnr_ad_ctx* c, int64_t n, double* ms_out) {
  if (!c || !ms_out) return ad_fail(c, LBNR_EINVAL, "null context or output");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) e = cudaEventRecord(e0, c->st);
  int rc = e == cudaSuccess ? lbnr_ad_step(c, n) : LBNR_OK;
  if (e == cudaSuccess) e = cudaEventRecord(e1, c->st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess)
    return ad_fail(c, LBNR_ECUDA, "step_timed: %s", cudaGetErrorString(e));
  *ms_out = ms;
  return rc;
}

int lbnr_ad_status(lbnr_ad_ctx* c) {
  if (!c) return ad_fail(c, LBNR_EINVAL, "null context");
  int h = 0;
  AD_TRY(c, cudaMemcpyAsync(&h, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  AD_TRY(c, cudaStreamSynchronize(c->st));
  if (h & 6) return ad_fail(c, LBNR_ETIMEOUT, "a bounded device wait ran out (flag %d)", h);
  return h ? ad_fail(c, LBNR_ENONFINITE, "non-finite moment seen") : LBNR_OK;
}

int lbnr_ad_moments(lbnr_ad_ctx* c, double* out) {
  if (!c || !out) return ad_fail(c, LBNR_EINVAL, "null context or output");
  if (!c->initialised) return ad_fail(c, LBNR_ESTATE, "moments before init");
  AD_TRY(c, c->ops.moments(c->G, ad_state(c), c->macro, c->dt, c->slicing, c->st));
  AD_TRY(c, cudaMemcpyAsync(out, c->macro, sizeof(double) * ad::kNFA * ad_cells(c),
                            cudaMemcpyDeviceToHost, c->st));
  AD_TRY(c, cudaStreamSynchronize(c->st));
  return lbnr_ad_status(c);
}

int lbnr_ad_get_distributions(lbnr_ad_ctx* c, double* out) {
  if (!c || !out) return ad_fail(c, LBNR_EINVAL, "null context or output");
  const int64_t cells = ad_cells(c);
  for (int F = 0; F < ad::kNFA; ++F)
    for (int l = 0; l < c->Q; ++l) {
      AD_TRY(c, c->ops.get_plane(c->G, ad_state(c), F, l, c->macro, c->st));
      AD_TRY(c, cudaMemcpyAsync(out + ((int64_t)F * c->Q + l) * cells, c->macro,
                                sizeof(double) * cells, cudaMemcpyDeviceToHost, c->st));
    }
  AD_TRY(c, cudaStreamSynchronize(c->st));
  return LBNR_OK;
}

int lbnr_ad_set_distributions(lbnr_ad_ctx* c, const double* in) {
  if (!c || !in) return ad_fail(c, LBNR_EINVAL, "null context or input");
  const int64_t cells = ad_cells(c);
  for (int F = 0; F < ad::kNFA; ++F)
    for (int l = 0; l < c->Q; ++l) {
      AD_TRY(c, cudaMemcpyAsync(c->macro, in + ((int64_t)F * c->Q + l) * cells,
                                sizeof(double) * cells, cudaMemcpyHostToDevice, c->st));
      AD_TRY(c, c->ops.set_plane(c->G, ad_state(c), F, l, c->macro, c->st));
    }
  AD_TRY(c, cudaMemsetAsync(c->flag, 0, sizeof(int), c->st));
  AD_TRY(c, cudaStreamSynchronize(c->st));
  c->initialised = true;
  return LBNR_OK;
}

int64_t lbnr_ad_steps_done(const lbnr_ad_ctx* c) { return c ? c->steps : -1; }

int lbnr_ad_num_forms(void) { return ad::kForms; }

int lbnr_ad_form_blocks(int form) {
  return (form >= 0 && form < ad::kForms) ? ad::kFormBlocks[form] : -100;
}

int lbnr_ad_set_form(lbnr_ad_ctx* c, int form) {
  if (!c || form < 0 || form >= ad::kForms) return ad_fail(c, LBNR_EINVAL, "no launch form %d", form);
  c->form = form;
  return LBNR_OK;
}

const char* lbnr_ad_last_error(const lbnr_ad_ctx* c) { return c ? c->err.c_str() : g_ad_err.c_str(); }

}  // extern "C"
