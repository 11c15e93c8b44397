// C-ABI of the lbnr library (declared in include/lbnr.h): context set-up,
// device memory layout, the step loop (CUDA graphs of two-step cycles) and
// the FP64 monitoring calls.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "../../include/lbnr.h"
#include "dispatch.h"

namespace lbnr {

size_t storage_bytes(int storage) {
  switch (storage) {
    case LBNR_F64: return 8;
    case LBNR_F32:
    case LBNR_DEV_F32: return 4;
    case LBNR_DEV_BF16:
    case LBNR_DEV_F16: return 2;
    default: return 0;
  }
}
bool storage_is_fp64(int storage) { return storage == LBNR_F64; }

static int q_of(int vset) { return vset == LBNR_D1Q3 ? 3 : vset == LBNR_D2Q9 ? 9 : vset == LBNR_D3Q19 ? 19 : 0; }

static const Ops* ops_of(int vset, int storage) {
  typedef const Ops* (*Getter)();
  static const Getter table[3][5] = {
      {ops_q3_s0, ops_q3_s1, ops_q3_s2, ops_q3_s3, ops_q3_s4},
      {ops_q9_s0, ops_q9_s1, ops_q9_s2, ops_q9_s3, ops_q9_s4},
      {ops_q19_s0, ops_q19_s1, ops_q19_s2, ops_q19_s3, ops_q19_s4}};
  if (vset < 1 || vset > 3 || storage < 0 || storage > 4) return nullptr;
  return table[vset - 1][storage]();
}

// Final fixed-order reduction of per-block partials into out[22]:
// H_L2, H_inf, M_L2, M_inf, C_L2, C_inf, sum rho~_F (16).
static __global__ void __launch_bounds__(256) k_reduce_final(const double* __restrict__ partials,
                                                      int64_t nblk_c, int64_t nblk_s, int64_t cells,
                                                      double* out) {
  __shared__ double red[8][22];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = 0; i < 22; ++i) {
    const int64_t nb = i < 6 ? nblk_c : nblk_s;
    double x = 0;
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
      const double y = partials[b * 22 + i];
      x = (i < 6 && (i & 1)) ? fmax(x, y) : x + y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = (i < 6 && (i & 1)) ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[warp][i] = x;
  }
  __syncthreads();
  if (threadIdx.x < 22) {
    const int i = threadIdx.x;
    double x = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
      x = (i < 6 && (i & 1)) ? fmax(x, red[w][i]) : x + red[w][i];
    out[i] = (i < 6 && !(i & 1)) ? sqrt(x / (double)cells) : x;
  }
}


static cudaError_t reduce_final(const double* partials, int64_t nbc, int64_t nbs, int64_t cells,
                                double* out, cudaStream_t st) {
  k_reduce_final<<<1, 256, 0, st>>>(partials, nbc, nbs, cells, out);
  return cudaGetLastError();
}

}  // namespace lbnr

using namespace lbnr;

struct lbnr_ctx {
  lbnr_grid grid;
  int vset = 0, Q = 0;
  double tau = 0, dx = 0, dt = 0;
  lbnr_opts opts;
  int streaming = LBNR_STREAM_PINGPONG;
  const Ops* ops = nullptr;
  int variant = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  void* base = nullptr;  // device memory (owned when own_mem)
  bool own_mem = false;
  uint64_t bytes = 0;
  void* f[2] = {nullptr, nullptr};
  // LAG (reading R17): stencil planes of the current step ([steps & 1]) and
  // of the next, which the collide kernel writes; under R5 only [0] is used
  // and k_aux refills it every step.
  void* aux[2] = {nullptr, nullptr};
  LaunchCtx L;
  bool initialised = false;
  int64_t steps = 0;
  cudaGraphExec_t cycle[2] = {nullptr, nullptr};  // two-step cycle from even / odd step
  double fluid_rho0 = 0, fluid_w = 0, fluid_t0 = 1;  // perfect fluid (rho0 = 0: vacuum)
  double* beta_field = nullptr;  // static shift field [3][cells] (owned)
  std::string err;
};

// Advances the device step counter that the fluid's time is read from.
static __global__ void k_tick(int64_t* clock) { *clock += 1; }

// Fluid pressure at the current state's time t0 + steps dt (0 in vacuum).
static double fluid_pressure_now(const lbnr_ctx* c) {
  if (!c->L.clock) return 0.0;
  const double r = c->fluid_t0 / (c->fluid_t0 + (double)c->steps * c->dt);
  return c->fluid_w * c->fluid_rho0 * r * r;
}

static thread_local std::string g_err;

void lbnr::set_thread_error(const char* msg) { g_err = msg; }

static int fail(lbnr_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  g_err = buf;
  return code;
}

#define CUDA_TRY(ctx, call)                                                                   \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail((ctx), LBNR_ECUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                                  \
  } while (0)

namespace {

struct Layout {
  uint64_t f0, f1, aux, aux2, macro, aux64, partials, out22, flag, stage, total;
};

uint64_t align256(uint64_t x) { return (x + 255) & ~uint64_t(255); }

int validate(const lbnr_grid* g, int vset, const lbnr_opts* o) {
  if (!g || !o) return fail(nullptr, LBNR_EINVAL, "null grid or options");
  if (q_of(vset) == 0) return fail(nullptr, LBNR_EINVAL, "unknown velocity set %d", vset);
  if (g->nx < 1 || g->ny < 1 || g->nz < 1)
    return fail(nullptr, LBNR_EINVAL, "grid sizes must be positive");
  if (g->nx > (1 << 30) || g->ny > (1 << 30) || g->nz > (1 << 30))
    return fail(nullptr, LBNR_EINVAL, "grid side too large");
  {
    // 32-bit cell indices; a buffer of at most 2^32 values per field
    const uint64_t cells = (uint64_t)g->nx * g->ny * g->nz;
    const uint64_t ps = (cells + kTile - 1) / kTile * kTile;
    if (cells >= (1ull << 31) || (uint64_t)q_of(vset) * ps >= (1ull << 32))
      return fail(nullptr, LBNR_EINVAL, "lattice too large (%llu cells)", (unsigned long long)cells);
  }
  if (vset == LBNR_D1Q3 && (g->ny != 1 || g->nz != 1))
    return fail(nullptr, LBNR_EINVAL, "D1Q3 needs ny = nz = 1");
  if (vset == LBNR_D2Q9 && g->nz != 1) return fail(nullptr, LBNR_EINVAL, "D2Q9 needs nz = 1");
  if (storage_bytes(o->storage) == 0) return fail(nullptr, LBNR_EINVAL, "unknown storage %d", o->storage);
  if (o->slicing < 0 || o->slicing > 2) return fail(nullptr, LBNR_EINVAL, "unknown slicing %d", o->slicing);
  if (o->streaming < 0 || o->streaming > 2)
    return fail(nullptr, LBNR_EINVAL, "unknown streaming %d", o->streaming);
  if (o->deriv_mode != LBNR_DERIV_SYNC && o->deriv_mode != LBNR_DERIV_LAG)
    return fail(nullptr, LBNR_EINVAL, "unknown derivative mode %d", o->deriv_mode);
  return LBNR_OK;
}

Layout layout_for(const lbnr_grid* g, int vset, int storage, int streaming, int deriv_mode) {
  const int Q = q_of(vset);
  const uint64_t cells = (uint64_t)g->nx * g->ny * g->nz;
  const uint64_t ps = (cells + kTile - 1) / kTile * kTile;
  const uint64_t fbytes = align256(16ull * Q * ps * storage_bytes(storage));
  const uint64_t cb = storage_is_fp64(storage) ? 8 : 4;
  const uint64_t nblk = (cells + 127) / 128;
  Layout L;
  uint64_t off = 0;
  L.f0 = off;
  off += fbytes;
  L.f1 = off;
  if (streaming == LBNR_STREAM_PINGPONG) off += fbytes;
  L.aux = off;
  off += align256(7 * cells * cb);
  L.aux2 = off;
  if (deriv_mode == LBNR_DERIV_LAG) off += align256(7 * cells * cb);
  L.macro = off;
  off += align256(16 * cells * 8);
  L.aux64 = off;
  off += align256(7 * cells * 8);
  L.partials = off;
  off += align256(nblk * 22 * 8);
  L.out22 = off;
  off += 256;
  L.flag = off;
  off += 256;
  L.stage = off;
  off += kStageBytes;
  L.total = off;
  return L;
}

int layout_now(const lbnr_ctx* c) {
  if (c->streaming == LBNR_STREAM_PINGPONG) return 0;
  return (c->steps & 1) ? 2 : 1;
}
void* state_now(const lbnr_ctx* c) {
  return c->streaming == LBNR_STREAM_PINGPONG ? c->f[c->steps & 1] : c->f[0];
}

bool lagged(const lbnr_ctx* c) { return c->opts.deriv_mode == LBNR_DERIV_LAG; }

// The launch context of the step that starts from step count `parity`: under
// LAG the collide kernel reads the stencil planes of that step and writes
// those of the next (no moment pass).
LaunchCtx step_ctx(const lbnr_ctx* c, int64_t parity) {
  LaunchCtx L = c->L;
  if (lagged(c)) {
    L.aux = c->aux[parity & 1];
    L.aux_out = c->aux[(parity + 1) & 1];
  }
  return L;
}

// Enqueues one step starting from step parity `parity`.
cudaError_t enqueue_step(lbnr_ctx* c, int64_t parity) {
  int layout;
  void *fin, *fout;
  if (c->streaming == LBNR_STREAM_PINGPONG) {
    layout = 0;
    fin = c->f[parity & 1];
    fout = c->f[(parity + 1) & 1];
  } else {
    layout = (parity & 1) ? 2 : 1;
    fin = fout = c->f[0];
  }
  const LaunchCtx L = step_ctx(c, parity);
  cudaError_t e = cudaSuccess;
  if (!lagged(c)) e = c->ops->aux(L, layout, fin);
  if (e != cudaSuccess) return e;
  e = c->ops->step(L, layout, c->variant, fin, fout);
  if (e == cudaSuccess && c->L.clock) {
    k_tick<<<1, 1, 0, c->st>>>(const_cast<int64_t*>(c->L.clock));
    e = cudaGetLastError();
  }
  return e;
}

void drop_graphs(lbnr_ctx* c) {
  for (auto& g : c->cycle)
    if (g) {
      cudaGraphExecDestroy(g);
      g = nullptr;
    }
}

int build_cycle(lbnr_ctx* c, int parity) {
  cudaGraph_t graph = nullptr;
  CUDA_TRY(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
  cudaError_t e1 = enqueue_step(c, parity);
  cudaError_t e2 = e1 == cudaSuccess ? enqueue_step(c, parity + 1) : e1;
  cudaError_t e3 = cudaStreamEndCapture(c->st, &graph);
  if (e2 != cudaSuccess || e3 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return fail(c, LBNR_ECUDA, "graph capture failed: %s",
                cudaGetErrorString(e2 != cudaSuccess ? e2 : e3));
  }
  cudaError_t e4 = cudaGraphInstantiate(&c->cycle[parity], graph, 0);
  cudaGraphDestroy(graph);
  if (e4 != cudaSuccess) return fail(c, LBNR_ECUDA, "graph instantiate: %s", cudaGetErrorString(e4));
  return LBNR_OK;
}

int read_flag(lbnr_ctx* c, int* flag) {
  CUDA_TRY(c, cudaMemcpyAsync(flag, c->L.flag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return LBNR_OK;
}

// Device flag word: bit 0 non-finite moment, bit 1 a bounded wait gave up,
// bit 2 a launch-consistency check failed (work was skipped).
int flag_status(lbnr_ctx* c, int flag) {
  if (flag & 4) return fail(c, LBNR_ECUDA, "device consistency check failed (flag %d)", flag);
  if (flag & 2) return fail(c, LBNR_ETIMEOUT, "a device-side wait timed out");
  if (flag & 1) return fail(c, LBNR_ENONFINITE, "non-finite moment seen");
  return LBNR_OK;
}

}  // namespace

extern "C" {

void lbnr_default_opts(lbnr_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->slicing = LBNR_HARMONIC;
  o->storage = LBNR_F64;
  o->streaming = LBNR_STREAM_AUTO;
  o->sources_on = 1;
}

int lbnr_workspace_bytes(const lbnr_grid* grid, int vset, const lbnr_opts* opts, uint64_t* out) {
  int rc = validate(grid, vset, opts);
  if (rc) return rc;
  if (!out) return fail(nullptr, LBNR_EINVAL, "null output");
  if (opts->streaming == LBNR_STREAM_AUTO)
    return fail(nullptr, LBNR_EINVAL, "workspace size needs a fixed streaming pattern");
  *out = layout_for(grid, vset, opts->storage, opts->streaming, opts->deriv_mode).total;
  return LBNR_OK;
}

int lbnr_create(const lbnr_grid* grid, int vset, double tau, double dx, double dt,
                const lbnr_opts* opts, lbnr_ctx** out) {
  if (!out) return fail(nullptr, LBNR_EINVAL, "null output");
  *out = nullptr;
  int rc = validate(grid, vset, opts);
  if (rc) return rc;
  if (!(tau > 0.5)) return fail(nullptr, LBNR_EINVAL, "tau must exceed 1/2 (got %g)", tau);
  if (!(dx > 0) || !(dt > 0)) return fail(nullptr, LBNR_EINVAL, "dx and dt must be positive");
  if (fabs(dt - dx) > 1e-12 * dx) return fail(nullptr, LBNR_EINVAL, "dt must equal dx");
  const Ops* ops = ops_of(vset, opts->storage);
  if (!ops) return fail(nullptr, LBNR_EINVAL, "no kernels for this set and storage");

  lbnr_ctx* c = new (std::nothrow) lbnr_ctx();
  if (!c) return fail(nullptr, LBNR_ENOMEM, "host allocation failed");
  c->grid = *grid;
  c->vset = vset;
  c->Q = q_of(vset);
  c->tau = tau;
  c->dx = dx;
  c->dt = dt;
  c->opts = *opts;
  c->ops = ops;

  // streaming pattern
  int streaming = opts->streaming;
  lbnr_grid g = *grid;
  const uint64_t need_pp =
      layout_for(&g, vset, opts->storage, LBNR_STREAM_PINGPONG, opts->deriv_mode).total;
  if (streaming == LBNR_STREAM_AUTO) {
    if (opts->dev_buffer) {
      streaming = opts->dev_bytes >= need_pp ? LBNR_STREAM_PINGPONG : LBNR_STREAM_AA;
    } else {
      size_t freeb = 0, totalb = 0;
      cudaError_t e = cudaMemGetInfo(&freeb, &totalb);
      if (e != cudaSuccess) {
        delete c;
        return fail(nullptr, LBNR_ECUDA, "cudaMemGetInfo: %s", cudaGetErrorString(e));
      }
      streaming = (double)need_pp <= 0.9 * (double)freeb ? LBNR_STREAM_PINGPONG : LBNR_STREAM_AA;
    }
  }
  c->streaming = streaming;
  const Layout Ly = layout_for(&g, vset, opts->storage, streaming, opts->deriv_mode);
  c->bytes = Ly.total;
  if (opts->dev_buffer) {
    if (opts->dev_bytes < Ly.total) {
      delete c;
      return fail(nullptr, LBNR_ENOMEM, "device buffer has %llu bytes, needs %llu",
                  (unsigned long long)opts->dev_bytes, (unsigned long long)Ly.total);
    }
    if ((uintptr_t)opts->dev_buffer % 256) {
      delete c;
      return fail(nullptr, LBNR_EINVAL, "device buffer must be 256-byte aligned");
    }
    c->base = opts->dev_buffer;
  } else {
    cudaError_t e = cudaMalloc(&c->base, Ly.total);
    if (e != cudaSuccess) {
      delete c;
      return fail(nullptr, LBNR_ENOMEM, "cudaMalloc(%llu): %s", (unsigned long long)Ly.total,
                  cudaGetErrorString(e));
    }
    c->own_mem = true;
  }
  if (opts->cuda_stream) {
    c->st = static_cast<cudaStream_t>(opts->cuda_stream);
  } else {
    cudaError_t e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      lbnr_destroy(c);
      return fail(nullptr, LBNR_ECUDA, "stream: %s", cudaGetErrorString(e));
    }
    c->own_stream = true;
  }
  char* b = static_cast<char*>(c->base);
  c->f[0] = b + Ly.f0;
  c->f[1] = streaming == LBNR_STREAM_PINGPONG ? b + Ly.f1 : nullptr;
  LaunchCtx& L = c->L;
  L.nx = (int32_t)grid->nx;
  L.ny = (int32_t)grid->ny;
  L.nz = (int32_t)grid->nz;
  L.cells = grid->nx * grid->ny * grid->nz;
  L.pstride = (L.cells + kTile - 1) / kTile * kTile;
  L.dx = dx;
  L.dt = dt;
  L.tau = tau;
  L.slicing = opts->slicing;
  L.sources_on = opts->sources_on ? 1 : 0;
  L.aux = b + Ly.aux;
  L.aux_out = nullptr;
  c->aux[0] = b + Ly.aux;
  c->aux[1] = opts->deriv_mode == LBNR_DERIV_LAG ? b + Ly.aux2 : nullptr;
  L.macro = reinterpret_cast<double*>(b + Ly.macro);
  L.aux64 = reinterpret_cast<double*>(b + Ly.aux64);
  L.partials = reinterpret_cast<double*>(b + Ly.partials);
  L.out22 = reinterpret_cast<double*>(b + Ly.out22);
  L.flag = reinterpret_cast<int*>(b + Ly.flag);
  L.stage = b + Ly.stage;
  L.st = c->st;
  L.block = 128;
  L.clock = nullptr;
  L.fluid_P0 = L.fluid_t0 = L.fluid_P_now = 0;
  L.beta[0] = L.beta[1] = L.beta[2] = 0;
  L.shift_on = 0;
  L.beta_field = nullptr;
  // zero everything once: the padding cells of the last tile must hold finite values
  cudaError_t e = cudaMemsetAsync(c->base, 0, Ly.total, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  if (e != cudaSuccess) {
    lbnr_destroy(c);
    return fail(nullptr, LBNR_ECUDA, "memset: %s", cudaGetErrorString(e));
  }
  *out = c;
  return LBNR_OK;
}

int lbnr_init(lbnr_ctx* c, const double* fields) {
  if (!c || !fields) return fail(c, LBNR_EINVAL, "null argument");
  const size_t nb = sizeof(double) * 16 * (size_t)c->L.cells;
  CUDA_TRY(c, cudaMemcpyAsync(c->L.macro, fields, nb, cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, cudaMemsetAsync(c->L.flag, 0, sizeof(int), c->st));
  if (c->L.clock)
    CUDA_TRY(c, cudaMemsetAsync(const_cast<int64_t*>(c->L.clock), 0, sizeof(int64_t), c->st));
  CUDA_TRY(c, c->ops->init(c->L, c->f[0]));
  // LAG: the first step's derivatives come from the initial fields
  if (lagged(c)) CUDA_TRY(c, c->ops->lag_from64(c->L, c->aux[0]));
  // the host array may be released as soon as we return
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->steps = 0;
  c->initialised = true;
  return LBNR_OK;
}

int lbnr_step(lbnr_ctx* c, int64_t n) {
  if (!c) return fail(c, LBNR_EINVAL, "null context");
  if (n < 0) return fail(c, LBNR_EINVAL, "negative step count");
  if (!c->initialised) return fail(c, LBNR_ESTATE, "step before init");
  while (n > 0) {
    const int parity = (int)(c->steps & 1);
    if (n >= 2) {
      if (!c->cycle[parity]) {
        int rc = build_cycle(c, parity);
        if (rc) return rc;
      }
      CUDA_TRY(c, cudaGraphLaunch(c->cycle[parity], c->st));
      c->steps += 2;
      n -= 2;
    } else {
      CUDA_TRY(c, enqueue_step(c, c->steps));
      c->steps += 1;
      n -= 1;
    }
  }
  return LBNR_OK;
}

int lbnr_step_timed(lbnr_ctx* c, int64_t n, double* ms_out) {
  if (!c || !ms_out) return fail(c, LBNR_EINVAL, "null argument");
  if (n < 0) return fail(c, LBNR_EINVAL, "negative step count");
  if (!c->initialised) return fail(c, LBNR_ESTATE, "step before init");
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  for (auto& e : ev) {
    const cudaError_t ce = cudaEventCreate(&e);
    if (ce != cudaSuccess) {
      for (auto& d : ev)
        if (d) cudaEventDestroy(d);
      return fail(c, LBNR_ECUDA, "timed step: %s", cudaGetErrorString(ce));
    }
  }
  double t_aux = 0, t_col = 0;
  int rc = LBNR_OK;
  for (int64_t i = 0; i < n && rc == LBNR_OK; ++i) {
    const int64_t parity = c->steps;
    int layout;
    void *fin, *fout;
    if (c->streaming == LBNR_STREAM_PINGPONG) {
      layout = 0;
      fin = c->f[parity & 1];
      fout = c->f[(parity + 1) & 1];
    } else {
      layout = (parity & 1) ? 2 : 1;
      fin = fout = c->f[0];
    }
    const LaunchCtx L = step_ctx(c, parity);
    cudaError_t e = cudaEventRecord(ev[0], c->st);
    if (e == cudaSuccess && !lagged(c)) e = c->ops->aux(L, layout, fin);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], c->st);
    if (e == cudaSuccess) e = c->ops->step(L, layout, c->variant, fin, fout);
    if (e == cudaSuccess) e = cudaEventRecord(ev[2], c->st);
    if (e == cudaSuccess && c->L.clock) {
      k_tick<<<1, 1, 0, c->st>>>(const_cast<int64_t*>(c->L.clock));
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[2]);
    float a = 0, b = 0;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[0], ev[1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[1], ev[2]);
    if (e != cudaSuccess) {
      rc = fail(c, LBNR_ECUDA, "timed step: %s", cudaGetErrorString(e));
      break;
    }
    t_aux += a;
    t_col += b;
    c->steps += 1;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  ms_out[0] += t_aux;
  ms_out[1] += t_col;
  return rc;
}

int lbnr_moments(lbnr_ctx* c, double* out) {
  if (!c || !out) return fail(c, LBNR_EINVAL, "null argument");
  if (!c->initialised) return fail(c, LBNR_ESTATE, "moments before init");
  int64_t nb = 0;
  c->L.fluid_P_now = fluid_pressure_now(c);
  CUDA_TRY(c, c->ops->sum64(c->L, layout_now(c), state_now(c), &nb));
  if (lagged(c)) CUDA_TRY(c, c->ops->lag_to64(c->L, c->aux[c->steps & 1], nullptr));
  CUDA_TRY(c, c->ops->correct64(c->L));
  CUDA_TRY(c, cudaMemcpyAsync(out, c->L.macro, sizeof(double) * 16 * (size_t)c->L.cells,
                              cudaMemcpyDeviceToHost, c->st));
  int flag = 0;
  int rc = read_flag(c, &flag);
  if (rc) return rc;
  return flag_status(c, flag);
}

int lbnr_constraints(lbnr_ctx* c, double* out) {
  if (!c || !out) return fail(c, LBNR_EINVAL, "null argument");
  if (!c->initialised) return fail(c, LBNR_ESTATE, "constraints before init");
  int64_t nbs = 0, nbc = 0;
  c->L.fluid_P_now = fluid_pressure_now(c);
  CUDA_TRY(c, c->ops->sum64(c->L, layout_now(c), state_now(c), &nbs));
  if (lagged(c)) CUDA_TRY(c, c->ops->lag_to64(c->L, c->aux[c->steps & 1], nullptr));
  CUDA_TRY(c, c->ops->correct64(c->L));
  CUDA_TRY(c, c->ops->constraints64(c->L, &nbc));
  CUDA_TRY(c, reduce_final(c->L.partials, nbc, nbs, c->L.cells, c->L.out22, c->st));
  CUDA_TRY(c, cudaMemcpyAsync(out, c->L.out22, sizeof(double) * 22, cudaMemcpyDeviceToHost, c->st));
  int flag = 0;
  int rc = read_flag(c, &flag);
  if (rc) return rc;
  return flag_status(c, flag);
}

int lbnr_get_distributions(lbnr_ctx* c, double* out) {
  if (!c || !out) return fail(c, LBNR_EINVAL, "null argument");
  if (!c->initialised) return fail(c, LBNR_ESTATE, "no state before init");
  const size_t cells = (size_t)c->L.cells;
  for (int F = 0; F < 16; ++F)
    for (int l = 0; l < c->Q; ++l) {
      double* plane = c->L.macro + (size_t)((F * c->Q + l) % 16) * cells;
      CUDA_TRY(c, c->ops->get_plane(c->L, layout_now(c), state_now(c), F, l, plane));
      CUDA_TRY(c, cudaMemcpyAsync(out + (size_t)(F * c->Q + l) * cells, plane, sizeof(double) * cells,
                                  cudaMemcpyDeviceToHost, c->st));
    }
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return LBNR_OK;
}

int lbnr_get_cells(lbnr_ctx* c, int64_t n, const int64_t* cells, double* out) {
  if (!c || (n > 0 && (!cells || !out)) || n < 0) return fail(c, LBNR_EINVAL, "bad argument");
  if (!c->initialised) return fail(c, LBNR_ESTATE, "no state before init");
  for (int64_t i = 0; i < n; ++i)
    if (cells[i] < 0 || cells[i] >= c->L.cells)
      return fail(c, LBNR_EINVAL, "cell index %lld out of range", (long long)cells[i]);
  const int64_t per = 16 * c->Q;
  const int64_t chunk = (int64_t)(kStageBytes / (8 * (per + 1)));
  int64_t* didx = static_cast<int64_t*>(c->L.stage);
  double* dout = reinterpret_cast<double*>(didx + chunk);
  for (int64_t s = 0; s < n; s += chunk) {
    const int64_t m = n - s < chunk ? n - s : chunk;
    CUDA_TRY(c, cudaMemcpyAsync(didx, cells + s, sizeof(int64_t) * m, cudaMemcpyHostToDevice, c->st));
    CUDA_TRY(c, c->ops->get_cells(c->L, layout_now(c), state_now(c), m, didx, dout));
    CUDA_TRY(c, cudaMemcpyAsync(out + s * per, dout, sizeof(double) * m * per, cudaMemcpyDeviceToHost,
                                c->st));
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
  }
  return LBNR_OK;
}

int lbnr_set_distributions(lbnr_ctx* c, const double* in) {
  if (!c || !in) return fail(c, LBNR_EINVAL, "null argument");
  const size_t cells = (size_t)c->L.cells;
  for (int F = 0; F < 16; ++F)
    for (int l = 0; l < c->Q; ++l) {
      double* plane = c->L.macro + (size_t)((F * c->Q + l) % 16) * cells;
      CUDA_TRY(c, cudaMemcpyAsync(plane, in + (size_t)(F * c->Q + l) * cells, sizeof(double) * cells,
                                  cudaMemcpyHostToDevice, c->st));
      CUDA_TRY(c, c->ops->set_plane(c->L, layout_now(c), state_now(c), F, l, plane));
    }
  CUDA_TRY(c, cudaMemsetAsync(c->L.flag, 0, sizeof(int), c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->initialised = true;
  return LBNR_OK;
}

int lbnr_get_lagged(lbnr_ctx* c, double* out) {
  if (!c || !out) return fail(c, LBNR_EINVAL, "null argument");
  if (!lagged(c)) return fail(c, LBNR_ESTATE, "the context does not use lagged derivatives");
  if (!c->initialised) return fail(c, LBNR_ESTATE, "no state before init");
  // decoded into the FP64 field planes (alpha, gamma) on the device, then copied
  double* d = c->L.macro;
  CUDA_TRY(c, c->ops->lag_to64(c->L, c->aux[c->steps & 1], d));
  CUDA_TRY(c, cudaMemcpyAsync(out, d, sizeof(double) * 7 * (size_t)c->L.cells,
                              cudaMemcpyDeviceToHost, c->st));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return LBNR_OK;
}

int lbnr_set_lagged(lbnr_ctx* c, const double* in) {
  if (!c || !in) return fail(c, LBNR_EINVAL, "null argument");
  if (!lagged(c)) return fail(c, LBNR_ESTATE, "the context does not use lagged derivatives");
  for (int64_t i = 0; i < c->L.cells; ++i)
    if (!(in[i] > 0) || !std::isfinite(in[i])) return fail(c, LBNR_EINVAL, "lapse must be positive");
  CUDA_TRY(c, cudaMemcpyAsync(c->L.macro, in, sizeof(double) * 7 * (size_t)c->L.cells,
                              cudaMemcpyHostToDevice, c->st));
  CUDA_TRY(c, c->ops->lag_from64(c->L, c->aux[c->steps & 1]));
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  return LBNR_OK;
}

int lbnr_deriv_mode(const lbnr_ctx* c) { return c ? c->opts.deriv_mode : -1; }

int lbnr_status(lbnr_ctx* c) {
  if (!c) return fail(c, LBNR_EINVAL, "null context");
  int flag = 0;
  int rc = read_flag(c, &flag);
  if (rc) return rc;
  return flag_status(c, flag);
}

int lbnr_num_variants(const lbnr_ctx* c) { return c ? c->ops->nvariants : 0; }

const char* lbnr_variant_name(const lbnr_ctx* c, int v) {
  return (c && v >= 0 && v < c->ops->nvariants) ? c->ops->variant_name(v) : "";
}

int lbnr_set_fluid(lbnr_ctx* c, double rho0, double w, double t0) {
  if (!c) return fail(c, LBNR_EINVAL, "null context");
  if (!std::isfinite(rho0) || !std::isfinite(w) || !(t0 > 0) || !std::isfinite(t0) || rho0 < 0)
    return fail(c, LBNR_EINVAL, "fluid needs rho0 >= 0, finite w and t0 > 0");
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->fluid_rho0 = rho0;
  c->fluid_w = w;
  c->fluid_t0 = t0;
  if (rho0 == 0) {
    c->L.clock = nullptr;
  } else {
    int64_t* clock = reinterpret_cast<int64_t*>(reinterpret_cast<char*>(c->L.flag) + 64);
    const int64_t n = c->steps;
    CUDA_TRY(c, cudaMemcpy(clock, &n, sizeof(n), cudaMemcpyHostToDevice));
    c->L.clock = clock;
  }
  c->L.fluid_P0 = w * rho0;
  c->L.fluid_t0 = t0;
  drop_graphs(c);  // the captured steps carry the old parameters
  return LBNR_OK;
}

int lbnr_set_shift(lbnr_ctx* c, double bx, double by, double bz) {
  if (!c) return fail(c, LBNR_EINVAL, "null context");
  if (!std::isfinite(bx) || !std::isfinite(by) || !std::isfinite(bz))
    return fail(c, LBNR_EINVAL, "shift must be finite");
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  c->L.beta[0] = bx;
  c->L.beta[1] = by;
  c->L.beta[2] = bz;
  c->L.shift_on = (bx != 0.0 || by != 0.0 || bz != 0.0 || c->L.beta_field) ? 1 : 0;
  drop_graphs(c);  // the captured steps carry the old parameters
  return LBNR_OK;
}

int lbnr_set_shift_field(lbnr_ctx* c, const double* beta) {
  if (!c) return fail(c, LBNR_EINVAL, "null context");
  const int64_t cells = c->L.cells;
  if (beta) {
    for (int64_t i = 0; i < 3 * cells; ++i)
      if (!std::isfinite(beta[i])) return fail(c, LBNR_EINVAL, "shift field value %lld not finite", (long long)i);
  }
  CUDA_TRY(c, cudaStreamSynchronize(c->st));
  if (beta) {
    if (!c->beta_field)
      CUDA_TRY(c, cudaMalloc(reinterpret_cast<void**>(&c->beta_field), sizeof(double) * 3 * cells));
    CUDA_TRY(c, cudaMemcpy(c->beta_field, beta, sizeof(double) * 3 * cells, cudaMemcpyHostToDevice));
    c->L.beta_field = c->beta_field;
  } else {
    if (c->beta_field) cudaFree(c->beta_field);
    c->beta_field = nullptr;
    c->L.beta_field = nullptr;
  }
  const double* b = c->L.beta;
  c->L.shift_on = (b[0] != 0.0 || b[1] != 0.0 || b[2] != 0.0 || c->L.beta_field) ? 1 : 0;
  drop_graphs(c);
  return LBNR_OK;
}

int lbnr_set_variant(lbnr_ctx* c, int v) {
  if (!c || v < 0 || v >= c->ops->nvariants) return fail(c, LBNR_EINVAL, "no variant %d", v);
  if (v != c->variant) {
    CUDA_TRY(c, cudaStreamSynchronize(c->st));
    drop_graphs(c);
    c->variant = v;
  }
  return LBNR_OK;
}

int64_t lbnr_steps_done(const lbnr_ctx* c) { return c ? c->steps : -1; }
int lbnr_q(const lbnr_ctx* c) { return c ? c->Q : 0; }
int lbnr_streaming(const lbnr_ctx* c) { return c ? c->streaming : 0; }

void lbnr_destroy(lbnr_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  drop_graphs(c);
  if (c->own_mem && c->base) cudaFree(c->base);
  if (c->beta_field) cudaFree(c->beta_field);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  delete c;
}

const char* lbnr_last_error(const lbnr_ctx* c) { return c ? c->err.c_str() : g_err.c_str(); }

}  // extern "C"
