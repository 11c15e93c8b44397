// Batched ensemble: many independent lattices (each its own set, size, tau,
// slicing and step count) advanced by one persistent launch.
//
// Each run is the same lattice Boltzmann step as a single context (Eq. numlb
// with the equilibria and sources of Eqs. alfa-ekstsor): a moment pass for
// the derivative stencil, then the fused collide-and-stream pass.
//
// Plan (host): a run's cost is cells x steps x Q. With W resident CTAs and
// an even share L = total / W, a run costing more than L gets a team of
// ceil(cost / L) CTAs of its own. The work list holds one entry per team
// member first, then every other run, longest first; each CTA claims the
// next entry with an atomic counter whenever it is free. Runs that stop
// early (non-finite) thus leave no CTA idle while work remains.
//
// Team members never wait on an entry nobody claims: the team entries come
// first and number at most W - 1 when other runs exist (W otherwise), every
// CTA makes its first claim when the launch starts, and a CTA can only claim
// again after finishing its entry, so the counter hands out all team entries
// while at least one CTA is free to claim.
//
// Kernel: for each step of a run the team's CTAs split the cells, run the
// moment pass, meet at a team barrier, run the collide pass, and meet again.
// With lagged derivatives (reading R17) a step is the collide pass alone,
// reading the stencil planes the previous step wrote and writing the next
// ones into the run's second plane set, and one team barrier.
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
  void* aux2;  // LAG: the second set of stencil planes (nullptr otherwise)
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
  const Assign* work;  // team entries, then single-CTA runs longest first
  const int* nwork;    // entries in `work` (device memory: re-planning
                       // rewrites the list without touching the graph)
  unsigned* head;      // next work entry, zeroed before each launch
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

template <int Q, class S, class C, int REP, bool LAG>
__device__ void run_steps(const BatchParams& p, const BatchRun& R, const Assign& A) {
  // every field read once into registers (a runtime index into a copy of the
  // descriptor would put it in local memory)
  const S* const f0 = static_cast<const S*>(R.f[0]);
  const S* const f1 = static_cast<const S*>(R.f[1]);
  const int64_t rsteps = R.steps;
  const int64_t want = p.max_steps < 0 ? rsteps : (p.max_steps < rsteps ? p.max_steps : rsteps);
  const int64_t start = p.done[A.run];
  StepArgs<S, C> a;
  a.aux = static_cast<const C*>(R.aux);
  a.flag = &p.status[A.run];
  a.G = R.G;
  const double dx = R.dx, tau = R.tau;
  a.inv2dx = C(1.0 / (2.0 * dx));
  a.inv4dx = C(1.0 / (4.0 * dx));
  a.half_dt = C(0.5 * dx);
  a.omega = C(1.0 / tau);
  a.omc = C(1.0 - 1.0 / tau);
  a.sigma = C(dx * (1.0 - 1.0 / (2.0 * tau)));
  a.slicing = R.slicing;
  a.sources_on = p.sources_on;
  a.clock = nullptr;  // batched runs are vacuum, zero shift
  a.fluid_P0 = a.fluid_t0 = a.fluid_dt = 0;
  a.beta[0] = a.beta[1] = a.beta[2] = C(0);
  a.beta_field = nullptr;
  C* const aux = static_cast<C*>(R.aux);
  C* const aux2 = static_cast<C*>(R.aux2);
  const int64_t cells = a.G.cells;
  const int64_t B = blockDim.x;
  // A run that went non-finite or timed out in an earlier launch stays where
  // it stopped. Flags are raised only in the collide phase, between two team
  // barriers, so every block of the team reads the same value here and below.
  if (*((volatile int*)&p.status[A.run]) & 3) return;
  int k = 0;
  int64_t s = 0;
  while (s < want) {
    const bool odd = ((start + s) & 1) != 0;
    a.fin = odd ? f1 : f0;
    a.fout = const_cast<S*>(odd ? f0 : f1);
    if (LAG) {
      // the stencil planes of this step (written by the previous one) and of
      // the next, alternating with the step parity like the distributions
      a.aux = odd ? aux2 : aux;
      a.aux_out = odd ? aux : aux2;
    } else {
      for (int64_t base = A.rank * B; base < cells; base += (int64_t)A.team * B) {
        const int64_t c = base + threadIdx.x;
        if (c < cells) aux_cell<Q, S, C, REP, kPingPong>(a.fin, aux, a.G, c);
      }
      if (!team_sync(p, A, k++)) return;
    }
    for (int64_t base = A.rank * B; base < cells; base += (int64_t)A.team * B) {
      const int64_t c = base + threadIdx.x;
      if (c < cells) collide_cell<Q, S, C, REP, kPingPong, LAG>(a, c);
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

// Launch bounds: form 0 takes blocks of 256 threads with up to 255
// registers a thread (one block per SM), form 1 blocks of 128 with up to 168
// (three per SM), form 2 blocks of 128 with up to 128 (four per SM).
template <int FORM>
struct BatchForm;
template <>
struct BatchForm<0> {
  static constexpr int kThreads = 256, kMinBlocks = 1;
};
template <>
struct BatchForm<1> {
  static constexpr int kThreads = 128, kMinBlocks = 3;
};
template <>
struct BatchForm<2> {
  static constexpr int kThreads = 128, kMinBlocks = 4;
};

template <class S, int REP, int FORM, bool LAG>
__global__ void __launch_bounds__(BatchForm<FORM>::kThreads, BatchForm<FORM>::kMinBlocks)
    k_batch(const BatchParams p) {
  using C = typename std::conditional<sizeof(S) == 8, double, float>::type;
  __shared__ int next;
  const int nwork = *p.nwork;
  for (;;) {
    if (threadIdx.x == 0) next = (int)atomicAdd(p.head, 1u);
    __syncthreads();
    const int i = next;
    __syncthreads();  // all have read `next` before thread 0 writes it again
    if (i >= nwork) break;
    const Assign A = p.work[i];
    const BatchRun& R = p.runs[A.run];
    if (R.q == 3)
      run_steps<3, S, C, REP, LAG>(p, R, A);
    else
      run_steps<9, S, C, REP, LAG>(p, R, A);
  }
}

template <int FORM, bool LAG>
void* batch_kernel_form(int storage) {
  switch (storage) {
    case LBNR_F64: return (void*)k_batch<double, kABS, FORM, LAG>;
    case LBNR_F32: return (void*)k_batch<float, kABS, FORM, LAG>;
    case LBNR_DEV_F32: return (void*)k_batch<float, kDEV, FORM, LAG>;
    case LBNR_DEV_BF16: return (void*)k_batch<__nv_bfloat16, kDEV, FORM, LAG>;
    case LBNR_DEV_F16: return (void*)k_batch<__half, kDEV, FORM, LAG>;
    default: return nullptr;
  }
}

// Form for a block size and a requested number of blocks per SM (0: the
// form's own maximum).
int form_for(int block, int per_sm) {
  if (block == 256) return 0;
  return per_sm == 4 ? 2 : 1;
}

template <bool LAG>
void* batch_kernel_mode(int storage, int form) {
  return form == 0 ? batch_kernel_form<0, LAG>(storage)
                   : form == 1 ? batch_kernel_form<1, LAG>(storage)
                               : batch_kernel_form<2, LAG>(storage);
}

void* batch_kernel(int storage, int form, int deriv_mode) {
  return deriv_mode == LBNR_DERIV_LAG ? batch_kernel_mode<true>(storage, form)
                                      : batch_kernel_mode<false>(storage, form);
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
  Assign* d_work = nullptr;  // work list (capacity work_cap)
  int64_t* d_done = nullptr;
  unsigned* d_bar = nullptr;
  int* d_status = nullptr;
  int* d_flag = nullptr;
  double* d_stage = nullptr;  // 16 x max cells FP64 (init, transfers)
  int64_t max_cells = 0;
  int grid = 0, block = 256, form = 0;
  std::vector<Assign> work;
  std::vector<int> team;   // blocks per run in the current plan (0: not stepped)
  size_t work_cap = 0;
  Assign* h_work = nullptr;  // pinned staging of the work list
  int* h_nwork = nullptr;
  int* d_nwork = nullptr;
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

// Builds the work list for `workers` resident CTAs over the runs marked
// live (all when `live` is empty).
void make_plan(lbnr_batch* b, int workers, const std::vector<char>& live) {
  const int R = (int)b->runs.size();
  std::vector<double> cost(R);
  double total = 0;
  for (int r = 0; r < R; ++r) {
    const lbnr_run_desc& d = b->runs[r];
    const bool on = live.empty() || live[r];
    cost[r] = on ? (double)(d.grid.nx * d.grid.ny * d.grid.nz) *
                       (double)std::max<int64_t>(d.steps, 1) * qv(d.vset)
                 : 0.0;
    total += cost[r];
  }
  const double share = total / std::max(workers, 1);
  std::vector<int> team(R, 1);
  int big = 0;
  bool any_small = false;
  for (int r = 0; r < R; ++r) {
    if (cost[r] == 0.0) {
      team[r] = 0;  // not stepped
      continue;
    }
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
  b->work.clear();
  for (int r = 0; r < R; ++r)
    if (team[r] > 1)
      for (int k = 0; k < team[r]; ++k) b->work.push_back(Assign{r, k, team[r]});
  std::vector<int> single;
  for (int r = 0; r < R; ++r)
    if (team[r] == 1) single.push_back(r);
  b->team = team;
  std::stable_sort(single.begin(), single.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  for (int r : single) b->work.push_back(Assign{r, 0, 1});
  b->grid = workers;
}

// Copies the work list and its length to the device (stream-ordered, from
// pinned staging; callers have synchronised the stream, so the staging is
// free).
int upload_plan(lbnr_batch* b) {
  const size_t n = b->work.size();
  if (n > b->work_cap) return bfail(b, LBNR_ECUDA, "work list larger than its buffer");
  memcpy(b->h_work, b->work.data(), sizeof(Assign) * n);
  *b->h_nwork = (int)n;
  if (n) BTRY(b, cudaMemcpyAsync(b->d_work, b->h_work, sizeof(Assign) * n, cudaMemcpyHostToDevice, b->st));
  BTRY(b, cudaMemcpyAsync(b->d_nwork, b->h_nwork, sizeof(int), cudaMemcpyHostToDevice, b->st));
  return LBNR_OK;
}

// Runs still to be stepped: neither non-finite nor timed out.
int live_runs(lbnr_batch* b, std::vector<char>& live) {
  std::vector<int> st(b->runs.size());
  BTRY(b, cudaMemcpyAsync(st.data(), b->d_status, sizeof(int) * st.size(), cudaMemcpyDeviceToHost,
                          b->st));
  BTRY(b, cudaStreamSynchronize(b->st));
  live.resize(st.size());
  for (size_t r = 0; r < st.size(); ++r) live[r] = (st[r] & 3) == 0;
  return LBNR_OK;
}

int configure(lbnr_batch* b, int block, int ctas_per_sm) {
  if (block != 128 && block != 256) return bfail(b, LBNR_EINVAL, "block must be 128 or 256");
  if (ctas_per_sm < 0 || ctas_per_sm > 4) return bfail(b, LBNR_EINVAL, "ctas_per_sm must be 0..4");
  const int form = form_for(block, ctas_per_sm);
  void* kern = batch_kernel(b->opts.storage, form, b->opts.deriv_mode);
  // the kernel uses no shared memory to speak of: give the SM's unified
  // cache to L1
  BTRY(b, cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0));
  int occ = 0;
  BTRY(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, block, 0));
  if (occ < 1) return bfail(b, LBNR_ECUDA, "batched kernel cannot be resident");
  int dev = 0, sms = 0;
  BTRY(b, cudaGetDevice(&dev));
  BTRY(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = ctas_per_sm > 0 ? std::min(ctas_per_sm, occ) : occ;
  const int workers = sms * per_sm;
  // work list buffers: at most one entry per CTA for team members plus one
  // per run
  const size_t cap = b->runs.size() + (size_t)workers;
  if (cap > b->work_cap) {
    cudaFree(b->d_work);
    cudaFreeHost(b->h_work);
    b->d_work = nullptr;
    b->h_work = nullptr;
    b->work_cap = 0;
    BTRY(b, cudaMalloc(&b->d_work, sizeof(Assign) * cap));
    BTRY(b, cudaMallocHost(&b->h_work, sizeof(Assign) * cap));
    b->work_cap = cap;
  }
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->block = block;
  b->form = form;
  std::vector<char> live;
  int rc = live_runs(b, live);
  if (rc) return rc;
  make_plan(b, workers, live);
  return upload_plan(b);
}

// Barrier reset and the cooperative launch, on the batch's stream.
cudaError_t enqueue_batch(lbnr_batch* b, BatchParams& p) {
  // team barrier counters and the work-list head
  cudaError_t e = cudaMemsetAsync(b->d_bar, 0, sizeof(unsigned) * (b->runs.size() + 1), b->st);
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
  return cudaLaunchKernelExC(&cfg, batch_kernel(b->opts.storage, b->form, b->opts.deriv_mode),
                             args);
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
  o->deriv_mode = LBNR_DERIV_SYNC;
}

int lbnr_batch_create(int nruns, const lbnr_run_desc* runs, const lbnr_batch_opts* opts,
                      lbnr_batch** out) {
  if (!out || !runs || !opts || nruns < 1) return bfail(nullptr, LBNR_EINVAL, "bad argument");
  *out = nullptr;
  if (!batch_kernel(opts->storage, 0, LBNR_DERIV_SYNC))
    return bfail(nullptr, LBNR_EINVAL, "unknown storage");
  if (opts->deriv_mode != LBNR_DERIV_SYNC && opts->deriv_mode != LBNR_DERIV_LAG)
    return bfail(nullptr, LBNR_EINVAL, "unknown derivative mode");
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
  const bool lag = opts->deriv_mode == LBNR_DERIV_LAG;
  std::vector<size_t> off_f(nruns), off_aux(nruns);
  size_t off = 0;
  for (int r = 0; r < nruns; ++r) {
    const int64_t cells = runs[r].grid.nx * runs[r].grid.ny;
    const int64_t ps = (cells + kTile - 1) / kTile * kTile;
    b->max_cells = std::max(b->max_cells, cells);
    off_f[r] = off;
    off += ((size_t)2 * 16 * qv(runs[r].vset) * ps * sb + 255) & ~(size_t)255;
    off_aux[r] = off;
    off += (((size_t)7 * cells * cb + 255) & ~(size_t)255) * (lag ? 2 : 1);
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
    h.aux2 = lag ? base + off_aux[r] + (((size_t)7 * cells * cb + 255) & ~(size_t)255) : nullptr;
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
  if (e == cudaSuccess) e = cudaMalloc(&b->d_bar, sizeof(unsigned) * (nruns + 1));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int) * nruns);
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int) * nruns);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_nwork, sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_nwork, sizeof(int));
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
  // LAG: the first step's derivatives come from the initial fields
  if (b->opts.deriv_mode == LBNR_DERIV_LAG) BTRY(b, o->lag_from64(L, h.aux));
  BTRY(b, cudaMemsetAsync(b->d_done + run, 0, sizeof(int64_t), b->st));
  BTRY(b, cudaStreamSynchronize(b->st));
  b->done[run] = 0;
  if (b->team[run] == 0) return lbnr_batch_replan(b);  // stopped run restarted
  return LBNR_OK;
}

int lbnr_batch_replan(lbnr_batch* b) {
  if (!b) return bfail(b, LBNR_EINVAL, "null batch");
  std::vector<char> live;
  int rc = live_runs(b, live);  // synchronises
  if (rc) return rc;
  make_plan(b, b->grid, live);
  return upload_plan(b);
}

int lbnr_batch_run(lbnr_batch* b, int64_t max_steps) {
  if (!b) return bfail(b, LBNR_EINVAL, "null batch");
  if (max_steps < 0) max_steps = -1;
  if (b->opts.replan) {
    int rc = lbnr_batch_replan(b);
    if (rc) return rc;
  }
  BatchParams p;
  p.runs = b->d_runs;
  p.work = b->d_work;
  p.nwork = b->d_nwork;
  p.head = b->d_bar + b->runs.size();
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
    for (size_t r = 0; r < b->runs.size(); ++r) team_of_run[r] = b->team[r];
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
  cudaFree(b->d_work);
  cudaFree(b->d_nwork);
  cudaFreeHost(b->h_work);
  cudaFreeHost(b->h_nwork);
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
