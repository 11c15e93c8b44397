// Batched ensemble: many independent lattices (each its own set, size, tau,
// slicing and step count) advanced by one persistent launch.
//
// Each run is the same lattice Boltzmann step as a single context (Eq. numlb
// with the equilibria and sources of Eqs. alfa-ekstsor): a moment pass for
// the derivative stencil, then the fused collide-and-stream pass.
//
// Plan (host): a run's cost is cells x steps x Q. With W resident CTAs and
// an even share L = total / W, a run costing more than L gets a team of
// ceil(cost / L) CTAs of its own; the other runs are packed onto the
// remaining CTAs, longest first onto the least-loaded CTA. Every CTA walks
// its list of (run, rank, team size) assignments.
//
// Kernel: for each step of a run the team's CTAs split the cells, run the
// moment pass, meet at a team barrier, run the collide pass, and meet again.
// A team barrier is a per-run counter: each CTA adds one and waits until
// the counter reaches the number of arrivals expected so far. The wait is
// bounded (globaltimer); on time-out the run's status gets bit 1 and its
// CTAs leave the run. The launch is cooperative, so the whole grid is
// resident and team members cannot wait on CTAs that never started.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <queue>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/lbnr.h"
#include "dispatch.h"
#include "kernels.cuh"

namespace lbnr {
namespace {

struct BatchRun {
  void* f[2];
  void* aux;
  Grid G;
  double tau, dx;
  int64_t steps;
  int q, slicing;
};

struct Assign {
  int run, rank, team;
};

struct BatchParams {
  const BatchRun* runs;
  const Assign* assign;
  const int* astart;  // CTA i walks assign[astart[i] .. astart[i+1])
  int64_t* done;      // steps taken so far, per run
  unsigned* bar;      // team barrier counters, zeroed before each launch
  int* status;        // per run: bit 0 non-finite, bit 1 wait timed out
  int* flag;          // any run: same bits
  int64_t max_steps;  // < 0: every run takes its own step count
  uint64_t wait_ns;
  int sources_on;
  int drop_run;  // test hook: rank 0 of this run's team skips its first arrival
};

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Team barrier number k (0-based) of a run with `team` CTAs. Returns false
// when the wait ran out.
__device__ bool team_sync(const BatchParams& p, const Assign& A, int k) {
  __syncthreads();
  if (A.team == 1) {
    __threadfence_block();
    return true;
  }
  __shared__ int ok;
  if (threadIdx.x == 0) {
    __threadfence();
    const bool drop = (A.run == p.drop_run && A.rank == 0 && k == 0);
    if (!drop) atomicAdd(&p.bar[A.run], 1u);
    const unsigned target = (unsigned)(k + 1) * (unsigned)A.team;
    ok = 1;
    const uint64_t t0 = now_ns();
    while (*((volatile unsigned*)&p.bar[A.run]) < target) {
      if (now_ns() - t0 > p.wait_ns) {
        ok = 0;
        atomicOr(&p.status[A.run], 2);
        atomicOr(p.flag, 2);
        break;
      }
      __nanosleep(256);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <int Q, class S, class C, int REP>
__device__ void run_steps(const BatchParams& p, const BatchRun& R, const Assign& A) {
  const int64_t want = p.max_steps < 0 ? R.steps : (p.max_steps < R.steps ? p.max_steps : R.steps);
  const int64_t start = p.done[A.run];
  StepArgs<S, C> a;
  a.aux = static_cast<const C*>(R.aux);
  a.flag = &p.status[A.run];
  a.G = R.G;
  a.inv2dx = C(1.0 / (2.0 * R.dx));
  a.inv4dx = C(1.0 / (4.0 * R.dx));
  a.half_dt = C(0.5 * R.dx);
  a.omega = C(1.0 / R.tau);
  a.omc = C(1.0 - 1.0 / R.tau);
  a.sigma = C(R.dx * (1.0 - 1.0 / (2.0 * R.tau)));
  a.slicing = R.slicing;
  a.sources_on = p.sources_on;
  const int64_t cells = R.G.cells;
  const int64_t B = blockDim.x;
  // A run that went non-finite or timed out in an earlier launch stays where
  // it stopped. Flags are raised only in the collide phase, between two team
  // barriers, so every block of the team reads the same value here and below.
  if (*((volatile int*)&p.status[A.run]) & 3) return;
  int k = 0;
  int64_t s = 0;
  while (s < want) {
    const int par = (int)((start + s) & 1);
    a.fin = static_cast<const S*>(R.f[par]);
    a.fout = static_cast<S*>(R.f[par ^ 1]);
    for (int64_t base = A.rank * B; base < cells; base += (int64_t)A.team * B) {
      const int64_t c = base + threadIdx.x;
      if (c < cells) aux_cell<Q, S, C, REP, kPingPong>(a.fin, static_cast<C*>(R.aux), R.G, c);
    }
    if (!team_sync(p, A, k++)) return;
    for (int64_t base = A.rank * B; base < cells; base += (int64_t)A.team * B) {
      const int64_t c = base + threadIdx.x;
      if (c < cells) collide_cell<Q, S, C, REP, kPingPong>(a, c);
    }
    if (!team_sync(p, A, k++)) return;
    ++s;
    // the step just taken read non-finite moments: the run stops here
    if (*((volatile int*)&p.status[A.run]) & 1) break;
  }
  if (A.rank == 0 && threadIdx.x == 0) {
    p.done[A.run] = start + s;
    if (p.status[A.run] & 1) atomicOr(p.flag, 1);
  }
}

template <class S, int REP>
__global__ void __launch_bounds__(256, sizeof(S) == 4 ? 2 : 1) k_batch(const BatchParams p) {
  using C = typename std::conditional<sizeof(S) == 8, double, float>::type;
  for (int e = p.astart[blockIdx.x]; e < p.astart[blockIdx.x + 1]; ++e) {
    const Assign A = p.assign[e];
    const BatchRun R = p.runs[A.run];
    if (R.q == 3)
      run_steps<3, S, C, REP>(p, R, A);
    else
      run_steps<9, S, C, REP>(p, R, A);
  }
}

void* batch_kernel(int storage) {
  switch (storage) {
    case LBNR_F64: return (void*)k_batch<double, kABS>;
    case LBNR_F32: return (void*)k_batch<float, kABS>;
    case LBNR_DEV_F32: return (void*)k_batch<float, kDEV>;
    case LBNR_DEV_BF16: return (void*)k_batch<__nv_bfloat16, kDEV>;
    case LBNR_DEV_F16: return (void*)k_batch<__half, kDEV>;
    default: return nullptr;
  }
}

int qv(int vset) { return vset == LBNR_D1Q3 ? 3 : vset == LBNR_D2Q9 ? 9 : 0; }

const Ops* ops_for_run(int vset, int s) {
  if (vset == LBNR_D1Q3)
    return s == 0 ? ops_q3_s0() : s == 1 ? ops_q3_s1() : s == 2 ? ops_q3_s2() : s == 3 ? ops_q3_s3() : ops_q3_s4();
  return s == 0 ? ops_q9_s0() : s == 1 ? ops_q9_s1() : s == 2 ? ops_q9_s2() : s == 3 ? ops_q9_s3() : ops_q9_s4();
}

}  // namespace
}  // namespace lbnr

using namespace lbnr;

struct lbnr_batch {
  std::vector<lbnr_run_desc> runs;
  lbnr_batch_opts opts;
  std::vector<BatchRun> hruns;
  std::vector<int64_t> done;  // host copy, valid after lbnr_batch_status
  cudaStream_t st = nullptr;
  bool own_stream = false;
  void* base = nullptr;
  size_t bytes = 0;
  BatchRun* d_runs = nullptr;
  Assign* d_assign = nullptr;
  int* d_astart = nullptr;
  int64_t* d_done = nullptr;
  unsigned* d_bar = nullptr;
  int* d_status = nullptr;
  int* d_flag = nullptr;
  double* d_stage = nullptr;  // 16 x max cells FP64 (init, transfers)
  int64_t max_cells = 0;
  int grid = 0, block = 256;
  std::vector<Assign> assign;
  std::vector<int> astart;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_steps = -2;
  bool graphed = true;  // false when the runtime refused to capture the launch
  std::string err;
};

namespace {

int bfail(lbnr_batch* b, int code, const char* msg) {
  if (b) b->err = msg;
  set_thread_error(msg);
  return code;
}

#define BTRY(b, call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) return bfail((b), LBNR_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

// Builds the CTA assignments for `workers` resident CTAs.
void make_plan(lbnr_batch* b, int workers) {
  const int R = (int)b->runs.size();
  std::vector<double> cost(R);
  double total = 0;
  for (int r = 0; r < R; ++r) {
    const lbnr_run_desc& d = b->runs[r];
    cost[r] = (double)(d.grid.nx * d.grid.ny * d.grid.nz) * (double)std::max<int64_t>(d.steps, 1) *
              qv(d.vset);
    total += cost[r];
  }
  const double share = total / std::max(workers, 1);
  std::vector<int> team(R, 1);
  int big = 0;
  bool any_small = false;
  for (int r = 0; r < R; ++r) {
    const int64_t cells = b->runs[r].grid.nx * b->runs[r].grid.ny * b->runs[r].grid.nz;
    const int64_t max_team = std::max<int64_t>(1, (cells + b->block - 1) / b->block);
    int t = (int)std::min<double>(std::ceil(cost[r] / std::max(share, 1.0)), (double)max_team);
    t = std::max(1, std::min(t, workers));
    team[r] = t;
    if (t > 1) big += t;
    else any_small = true;
  }
  // keep at least one CTA for the small runs
  while (big > workers - (any_small ? 1 : 0)) {
    int rmax = -1;
    for (int r = 0; r < R; ++r)
      if (team[r] > 1 && (rmax < 0 || team[r] > team[rmax])) rmax = r;
    if (rmax < 0) break;
    --team[rmax];
    --big;
    if (team[rmax] == 1) any_small = true;
  }
  std::vector<std::vector<Assign>> per(workers);
  int next = 0;
  for (int r = 0; r < R; ++r)
    if (team[r] > 1)
      for (int k = 0; k < team[r]; ++k) per[next++].push_back(Assign{r, k, team[r]});
  // longest first onto the least-loaded of the remaining CTAs
  std::vector<int> small;
  for (int r = 0; r < R; ++r)
    if (team[r] == 1) small.push_back(r);
  std::sort(small.begin(), small.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  typedef std::pair<double, int> Load;
  std::priority_queue<Load, std::vector<Load>, std::greater<Load>> heap;
  for (int w = next; w < workers; ++w) heap.push(Load(0.0, w));
  if (heap.empty() && !small.empty()) heap.push(Load(0.0, 0));
  for (int r : small) {
    Load l = heap.top();
    heap.pop();
    per[l.second].push_back(Assign{r, 0, 1});
    heap.push(Load(l.first + cost[r], l.second));
  }
  b->assign.clear();
  b->astart.assign(1, 0);
  for (int w = 0; w < workers; ++w) {
    for (const Assign& a : per[w]) b->assign.push_back(a);
    b->astart.push_back((int)b->assign.size());
  }
  b->grid = workers;
}

int upload_plan(lbnr_batch* b) {
  if (b->d_assign) cudaFree(b->d_assign);
  if (b->d_astart) cudaFree(b->d_astart);
  b->d_assign = nullptr;
  b->d_astart = nullptr;
  BTRY(b, cudaMalloc(&b->d_assign, sizeof(Assign) * std::max<size_t>(1, b->assign.size())));
  BTRY(b, cudaMalloc(&b->d_astart, sizeof(int) * b->astart.size()));
  BTRY(b, cudaMemcpy(b->d_assign, b->assign.data(), sizeof(Assign) * b->assign.size(),
                     cudaMemcpyHostToDevice));
  BTRY(b, cudaMemcpy(b->d_astart, b->astart.data(), sizeof(int) * b->astart.size(),
                     cudaMemcpyHostToDevice));
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return LBNR_OK;
}

int configure(lbnr_batch* b, int block, int ctas_per_sm) {
  if (block != 128 && block != 256) return bfail(b, LBNR_EINVAL, "block must be 128 or 256");
  void* kern = batch_kernel(b->opts.storage);
  int occ = 0;
  BTRY(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, 0));
  if (occ < 1) return bfail(b, LBNR_ECUDA, "batched kernel cannot be resident");
  int dev = 0, sms = 0;
  BTRY(b, cudaGetDevice(&dev));
  BTRY(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
  b->block = block;
  make_plan(b, sms * per_sm);
  return upload_plan(b);
}

// Barrier reset and the cooperative launch, on the batch's stream.
cudaError_t enqueue_batch(lbnr_batch* b, BatchParams& p) {
  cudaError_t e = cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned) * b->runs.size(), b->st);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)b->grid);
  cfg.blockDim = dim3((unsigned)b->block);
  cfg.stream = b->st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&p};
  return cudaLaunchKernelExC(&cfg, batch_kernel(b->opts.storage), args);
}

}  // namespace

extern "C" {

void lbnr_default_batch_opts(lbnr_batch_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->storage = LBNR_DEV_F32;
  o->block = 256;
  o->ctas_per_sm = 0;
  o->sources_on = 1;
  o->wait_limit_ns = 2000000000ll;
  o->test_drop_arrival_run = -1;
}

int lbnr_batch_create(int nruns, const lbnr_run_desc* runs, const lbnr_batch_opts* opts,
                      lbnr_batch** out) {
  if (!out || !runs || !opts || nruns < 1) return bfail(nullptr, LBNR_EINVAL, "bad argument");
  *out = nullptr;
  if (!batch_kernel(opts->storage)) return bfail(nullptr, LBNR_EINVAL, "unknown storage");
  for (int r = 0; r < nruns; ++r) {
    const lbnr_run_desc& d = runs[r];
    if (qv(d.vset) == 0) return bfail(nullptr, LBNR_EINVAL, "batched runs are D1Q3 or D2Q9");
    if (d.grid.nx < 1 || d.grid.ny < 1 || d.grid.nz != 1 ||
        (d.vset == LBNR_D1Q3 && d.grid.ny != 1))
      return bfail(nullptr, LBNR_EINVAL, "bad run lattice");
    if ((uint64_t)d.grid.nx * d.grid.ny >= (1ull << 28))
      return bfail(nullptr, LBNR_EINVAL, "run lattice too large");
    if (!(d.tau > 0.5) || !(d.dx > 0) || d.steps < 0 || d.slicing < 0 || d.slicing > 2)
      return bfail(nullptr, LBNR_EINVAL, "bad run parameters (tau > 1/2, dx > 0, steps >= 0)");
  }
  lbnr_batch* b = new (std::nothrow) lbnr_batch();
  if (!b) return bfail(nullptr, LBNR_ENOMEM, "host allocation failed");
  b->runs.assign(runs, runs + nruns);
  b->opts = *opts;
  if (b->opts.wait_limit_ns <= 0) b->opts.wait_limit_ns = 2000000000ll;
  const size_t sb = storage_bytes(opts->storage);
  const size_t cb = storage_is_fp64(opts->storage) ? 8 : 4;
  // lay out every run's two buffers and stencil planes in one allocation
  std::vector<size_t> off_f(nruns), off_aux(nruns);
  size_t off = 0;
  for (int r = 0; r < nruns; ++r) {
    const int64_t cells = runs[r].grid.nx * runs[r].grid.ny;
    const int64_t ps = (cells + kTile - 1) / kTile * kTile;
    b->max_cells = std::max(b->max_cells, cells);
    off_f[r] = off;
    off += ((size_t)2 * 16 * qv(runs[r].vset) * ps * sb + 255) & ~(size_t)255;
    off_aux[r] = off;
    off += ((size_t)7 * cells * cb + 255) & ~(size_t)255;
  }
  const size_t stage_off = off;
  off += ((size_t)16 * b->max_cells * 8 + 255) & ~(size_t)255;
  b->bytes = off;
  cudaError_t e = cudaMalloc(&b->base, off);
  if (e != cudaSuccess) {
    delete b;
    return bfail(nullptr, LBNR_ENOMEM, "device allocation for the batch failed");
  }
  e = cudaMemset(b->base, 0, off);
  char* base = static_cast<char*>(b->base);
  b->d_stage = reinterpret_cast<double*>(base + stage_off);
  b->hruns.resize(nruns);
  for (int r = 0; r < nruns; ++r) {
    const lbnr_run_desc& d = runs[r];
    const int64_t cells = d.grid.nx * d.grid.ny;
    const int64_t ps = (cells + kTile - 1) / kTile * kTile;
    BatchRun& h = b->hruns[r];
    h.f[0] = base + off_f[r];
    h.f[1] = base + off_f[r] + (size_t)16 * qv(d.vset) * ps * sb;
    h.aux = base + off_aux[r];
    h.G = make_grid((int32_t)d.grid.nx, (int32_t)d.grid.ny, 1, cells, ps);
    h.tau = d.tau;
    h.dx = d.dx;
    h.steps = d.steps;
    h.q = qv(d.vset);
    h.slicing = d.slicing;
  }
  b->done.assign(nruns, 0);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_runs, sizeof(BatchRun) * nruns);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_runs, b->hruns.data(), sizeof(BatchRun) * nruns, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_done, sizeof(int64_t) * nruns);
  if (e == cudaSuccess) e = cudaMemset(b->d_done, 0, sizeof(int64_t) * nruns);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_bar, sizeof(unsigned) * nruns);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int) * nruns);
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int) * nruns);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_flag, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_flag, 0, sizeof(int));
  if (e == cudaSuccess && opts->cuda_stream) {
    b->st = static_cast<cudaStream_t>(opts->cuda_stream);
  } else if (e == cudaSuccess) {
    e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    b->own_stream = e == cudaSuccess;
  }
  if (e != cudaSuccess) {
    lbnr_batch_destroy(b);
    return bfail(nullptr, LBNR_ECUDA, cudaGetErrorString(e));
  }
  int rc = configure(b, opts->block ? opts->block : 256, opts->ctas_per_sm);
  if (rc) {
    std::string m = b->err;
    lbnr_batch_destroy(b);
    return bfail(nullptr, rc, m.c_str());
  }
  *out = b;
  return LBNR_OK;
}

int lbnr_batch_configure(lbnr_batch* b, int block, int ctas_per_sm) {
  if (!b) return bfail(b, LBNR_EINVAL, "null batch");
  BTRY(b, cudaStreamSynchronize(b->st));
  return configure(b, block, ctas_per_sm);
}

int lbnr_batch_init(lbnr_batch* b, int run, const double* fields) {
  if (!b || !fields || run < 0 || run >= (int)b->runs.size())
    return bfail(b, LBNR_EINVAL, "bad argument");
  const BatchRun& h = b->hruns[run];
  const lbnr_run_desc& d = b->runs[run];
  const size_t cells = (size_t)h.G.cells;
  BTRY(b, cudaMemcpyAsync(b->d_stage, fields, sizeof(double) * 16 * cells,
                          cudaMemcpyHostToDevice, b->st));
  LaunchCtx L;
  memset(&L, 0, sizeof(L));
  L.nx = h.G.nx;
  L.ny = h.G.ny;
  L.nz = 1;
  L.cells = h.G.cells;
  L.pstride = h.G.pstride;
  L.dx = d.dx;
  L.dt = d.dx;
  L.tau = d.tau;
  L.slicing = d.slicing;
  L.sources_on = b->opts.sources_on ? 1 : 0;
  L.macro = b->d_stage;
  L.flag = b->d_status + run;
  L.st = b->st;
  const Ops* o = ops_for_run(d.vset, b->opts.storage);
  BTRY(b, cudaMemsetAsync(b->d_status + run, 0, sizeof(int), b->st));
  BTRY(b, o->init(L, h.f[0]));
  BTRY(b, cudaMemsetAsync(b->d_done + run, 0, sizeof(int64_t), b->st));
  BTRY(b, cudaStreamSynchronize(b->st));
  b->done[run] = 0;
  return LBNR_OK;
}

int lbnr_batch_run(lbnr_batch* b, int64_t max_steps) {
  if (!b) return bfail(b, LBNR_EINVAL, "null batch");
  if (max_steps < 0) max_steps = -1;
  BatchParams p;
  p.runs = b->d_runs;
  p.assign = b->d_assign;
  p.astart = b->d_astart;
  p.done = b->d_done;
  p.bar = b->d_bar;
  p.status = b->d_status;
  p.flag = b->d_flag;
  p.max_steps = max_steps;
  p.wait_ns = (uint64_t)b->opts.wait_limit_ns;
  p.sources_on = b->opts.sources_on ? 1 : 0;
  p.drop_run = b->opts.test_drop_arrival_run;
  if (b->graphed && (!b->graph || b->graph_steps != max_steps)) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    BTRY(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = enqueue_batch(b, p);
    cudaError_t e2 = cudaStreamEndCapture(b->st, &g);
    if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      // this runtime cannot capture the cooperative launch: launch directly
      (void)cudaGetLastError();
      b->graph = nullptr;
      b->graphed = false;
    } else {
      b->graph_steps = max_steps;
    }
  }
  if (b->graphed) {
    BTRY(b, cudaGraphLaunch(b->graph, b->st));
  } else {
    BTRY(b, enqueue_batch(b, p));
  }
  return LBNR_OK;
}

int lbnr_batch_status(lbnr_batch* b, int32_t* per_run) {
  if (!b) return bfail(b, LBNR_EINVAL, "null batch");
  std::vector<int> st(b->runs.size());
  BTRY(b, cudaMemcpyAsync(st.data(), b->d_status, sizeof(int) * st.size(), cudaMemcpyDeviceToHost,
                          b->st));
  BTRY(b, cudaMemcpyAsync(b->done.data(), b->d_done, sizeof(int64_t) * st.size(),
                          cudaMemcpyDeviceToHost, b->st));
  BTRY(b, cudaStreamSynchronize(b->st));
  int worst = LBNR_OK;
  for (size_t r = 0; r < st.size(); ++r) {
    const int code = (st[r] & 2) ? LBNR_ETIMEOUT : (st[r] & 1) ? LBNR_ENONFINITE : LBNR_OK;
    if (per_run) per_run[r] = code;
    if (code == LBNR_ETIMEOUT || (code == LBNR_ENONFINITE && worst == LBNR_OK)) worst = code;
  }
  return worst == LBNR_OK ? LBNR_OK : bfail(b, worst, "some runs reported an error");
}

int lbnr_batch_get_distributions(lbnr_batch* b, int run, double* out) {
  if (!b || !out || run < 0 || run >= (int)b->runs.size()) return bfail(b, LBNR_EINVAL, "bad argument");
  int64_t done = 0;
  BTRY(b, cudaMemcpyAsync(&done, b->d_done + run, sizeof(int64_t), cudaMemcpyDeviceToHost, b->st));
  BTRY(b, cudaStreamSynchronize(b->st));
  b->done[run] = done;
  const BatchRun& h = b->hruns[run];
  const lbnr_run_desc& d = b->runs[run];
  const Ops* o = ops_for_run(d.vset, b->opts.storage);
  LaunchCtx L;
  memset(&L, 0, sizeof(L));
  L.nx = h.G.nx;
  L.ny = h.G.ny;
  L.nz = 1;
  L.cells = h.G.cells;
  L.pstride = h.G.pstride;
  L.st = b->st;
  const size_t cells = (size_t)h.G.cells;
  for (int F = 0; F < 16; ++F)
    for (int l = 0; l < h.q; ++l) {
      double* plane = b->d_stage + (size_t)((F * h.q + l) % 16) * cells;
      BTRY(b, o->get_plane(L, 0, h.f[done & 1], F, l, plane));
      BTRY(b, cudaMemcpyAsync(out + (size_t)(F * h.q + l) * cells, plane, sizeof(double) * cells,
                              cudaMemcpyDeviceToHost, b->st));
    }
  BTRY(b, cudaStreamSynchronize(b->st));
  return LBNR_OK;
}

int lbnr_batch_plan(const lbnr_batch* b, int32_t* grid, int32_t* block, int32_t* graphed,
                    int32_t* team_of_run) {
  if (!b) return LBNR_EINVAL;
  if (grid) *grid = b->grid;
  if (block) *block = b->block;
  if (graphed) *graphed = b->graphed ? 1 : 0;
  if (team_of_run) {
    for (size_t r = 0; r < b->runs.size(); ++r) team_of_run[r] = 1;
    for (const Assign& a : b->assign) team_of_run[a.run] = a.team;
  }
  return LBNR_OK;
}

int64_t lbnr_batch_steps_done(const lbnr_batch* b, int run) {
  return (b && run >= 0 && run < (int)b->runs.size()) ? b->done[run] : -1;
}

void lbnr_batch_destroy(lbnr_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->d_assign);
  cudaFree(b->d_astart);
  cudaFree(b->d_runs);
  cudaFree(b->d_done);
  cudaFree(b->d_bar);
  cudaFree(b->d_status);
  cudaFree(b->d_flag);
  cudaFree(b->base);
  if (b->own_stream && b->st) cudaStreamDestroy(b->st);
  delete b;
}

const char* lbnr_batch_last_error(const lbnr_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
