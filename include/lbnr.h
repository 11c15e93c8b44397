/*
 * lbnr: GB300 (sm_103a) library for the lattice Boltzmann model of the
 * Bona-Masso Einstein equations (Ilseven & Mendoza, "Lattice Boltzmann Model
 * for Numerical Relativity", arXiv:1505.02037).
 *
 * One context = one periodic lattice on one GPU. Each step is the paper's
 * forced BGK update (Eq. numlb) with the equilibria and source distributions
 * of Eqs. (alfa)-(ekstsor), the moment rule rho = sum_l f_l + dt S / 2
 * (Sec. "Lattice Boltzmann Model"), the Bona-Masso right-hand sides of
 * Sec. "Bona-Masso evolution equations" at zero shift in vacuum, and A_k,
 * D_kij formed from alpha and gamma by central differences (Sec. "First order
 * derivatives").
 *
 * Conventions used by every call:
 *  - Fields, 16 per cell, in this order: alpha; gamma_xx, gamma_xy, gamma_xz,
 *    gamma_yy, gamma_yz, gamma_zz; K_xx, K_xy, K_xz, K_yy, K_yz, K_zz;
 *    V_x, V_y, V_z.
 *  - Cells: index x + nx*(y + ny*z), x fastest; the lattice is periodic.
 *  - Host field arrays are float64 [16][nz][ny][nx]; distribution arrays are
 *    float64 [16][Q][nz][ny][nx] with the velocities in the paper's order
 *    (D2Q9 and D3Q19 as printed; D1Q3 is c = 0, +1, -1, w = 2/3, 1/6, 1/6, the
 *    x-marginal of both printed sets).
 *  - tau is the dimensionless relaxation time tau/dt of Eq. (lbe); dt must
 *    equal dx (Sec. "Gauge Wave": dt = dr).
 *  - All host pointers belong to the caller and are only read or written
 *    during the call. Every call that returns data to the host synchronises
 *    the context's stream; lbnr_init and lbnr_step only enqueue work.
 *  - Return value: LBNR_OK (0) or a negative LBNR_E* code; lbnr_last_error
 *    gives a message. A context is used from one host thread at a time.
 */
#ifndef LBNR_H
#define LBNR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lbnr_ctx lbnr_ctx;

/* Velocity sets (Sec. "Lattice Boltzmann Model"). */
enum { LBNR_D1Q3 = 1, LBNR_D2Q9 = 2, LBNR_D3Q19 = 3 };

/* Distribution storage. F64/F32 store f itself. The DEV_* forms store
 * (f_l / w_l - rho_flat) with rho_flat the flat-space value of the field
 * (alpha = 1, gamma = delta, K = V = 0), so small waves keep their relative
 * precision; all single-precision forms collide in FP32. */
enum { LBNR_F64 = 0, LBNR_F32 = 1, LBNR_DEV_F32 = 2, LBNR_DEV_BF16 = 3, LBNR_DEV_F16 = 4 };

/* Slicing condition (Sec. "Gauge choices"): Q = 0, Q = tr K, Q = tr K/alpha. */
enum { LBNR_GEODESIC = 0, LBNR_HARMONIC = 1, LBNR_ONE_PLUS_LOG = 2 };

/* Streaming: AUTO takes ping-pong buffers when two copies fit in free device
 * memory, else the in-place AA pattern (one copy). */
enum { LBNR_STREAM_AUTO = 0, LBNR_STREAM_PINGPONG = 1, LBNR_STREAM_AA = 2 };

/* Time level of A_k and D_kij, on which the paper is silent (Sec. "Lattice
 * Boltzmann Model", moment rule; Sec. "Bona-Masso evolution equations",
 * first-order derivatives). SYNC: central differences of this step's zeroth
 * moments of alpha and gamma (a moment pass over their distributions, then
 * the collide kernel). LAG: central differences of the previous step's
 * corrected alpha and gamma (the initial fields at the first step), which
 * the collide kernel itself writes for the next step: one kernel per step.
 * Both are first order in dt; they differ by O(dt) per step. */
enum { LBNR_DERIV_SYNC = 0, LBNR_DERIV_LAG = 1 };

enum {
  LBNR_OK = 0,
  LBNR_EINVAL = -1,     /* bad argument: sizes, tau <= 1/2, dt != dx, NULL */
  LBNR_ENOMEM = -2,     /* device memory or the given buffer is too small */
  LBNR_ECUDA = -3,      /* a CUDA call failed; see lbnr_last_error */
  LBNR_ENONFINITE = -4, /* a step produced a NaN or Inf moment */
  LBNR_ETIMEOUT = -5,   /* a bounded device-side wait ran out */
  LBNR_ESTATE = -6      /* call out of order (e.g. step before init) */
};

typedef struct {
  int64_t nx, ny, nz; /* D1Q3 needs ny = nz = 1, D2Q9 needs nz = 1 */
} lbnr_grid;

typedef struct {
  int32_t slicing;    /* LBNR_GEODESIC / LBNR_HARMONIC / LBNR_ONE_PLUS_LOG */
  int32_t storage;    /* LBNR_F64 ... LBNR_DEV_F16 */
  int32_t streaming;  /* LBNR_STREAM_* */
  int32_t sources_on; /* 1 normally; 0 drops every source (a test switch) */
  void* cuda_stream;  /* cudaStream_t for all work; NULL = default stream */
  void* dev_buffer;   /* optional caller-owned device memory of dev_bytes
                         (>= lbnr_workspace_bytes); it must outlive the
                         context. NULL: the library allocates its own. */
  uint64_t dev_bytes;
  int32_t deriv_mode; /* LBNR_DERIV_SYNC (default) or LBNR_DERIV_LAG */
  int32_t reserved;   /* 0 */
} lbnr_opts;

/* Fills o with the defaults: harmonic slicing, F64, AUTO, sources on, SYNC. */
void lbnr_default_opts(lbnr_opts* o);

/* Device bytes a context needs for this grid, set and options (the
 * streaming choice must not be AUTO). */
int lbnr_workspace_bytes(const lbnr_grid* grid, int vset, const lbnr_opts* opts,
                         uint64_t* out_bytes);

/* Creates a context: validates the arguments, fixes the streaming pattern and
 * lays out (or allocates) the device memory. Nothing is computed. */
int lbnr_create(const lbnr_grid* grid, int vset, double tau, double dx, double dt,
                const lbnr_opts* opts, lbnr_ctx** out);

/* Initial distributions from host fields [16][cells]: the shifted equilibrium
 * f = f_eq(rho0) - (dt/2) w_l S(rho0), with A, D taken from rho0 (the paper
 * does not state its initialisation). Resets the step count to 0. */
int lbnr_init(lbnr_ctx* ctx, const double* fields);

/* Enqueues n steps on the context's stream (graph-captured two-step cycles).
 * Returns without waiting; a NaN/Inf is reported by the next synchronising
 * call. */
int lbnr_step(lbnr_ctx* ctx, int64_t n);

/* Same work as lbnr_step(n), launched one kernel at a time with CUDA events
 * recorded around every launch on the context's stream; synchronises and
 * adds the elapsed milliseconds per kernel kind into ms_out[2]
 * (ms_out[0]: the moment pass feeding the derivative stencil, which LAG does
 * not run, ms_out[1]: the fused collide-and-stream kernel). For
 * measurement. */
int lbnr_step_timed(lbnr_ctx* ctx, int64_t n, double* ms_out);

/* Corrected macroscopic fields rho = sum_l f_l + dt S/2 (Sec. LBM), evaluated
 * in FP64 from the stored distributions, into host out[16][cells]. Under
 * LAG the sources take A and D from the lagged fields, as the step does. */
int lbnr_moments(lbnr_ctx* ctx, double* out);

/* Constraint monitor, FP64 on the device, into host out[22]:
 * H_L2, H_inf, M_L2, M_inf, C_L2, C_inf, then sum over cells of sum_l f_l for
 * each of the 16 fields. H = R - K_ij K^ij + (tr K)^2 and
 * M_i = D_j K^j_i - d_i tr K are the vacuum Hamiltonian and momentum
 * constraints (Sec. "3+1 ADM formalism"), C_k = V_k - (D_kr^r - D^r_rk) the
 * definition of V (Sec. "Bona-Masso formulation"), all at the corrected
 * fields with central differences; L2 = root mean square over cells of the
 * (vector) norm, inf = largest magnitude. */
int lbnr_constraints(lbnr_ctx* ctx, double* out);

/* Stored distributions decoded to FP64, host out[16][Q][cells] (standard
 * layout whatever the device layout and streaming pattern: on the device the
 * 16 Q values of each 32-cell tile form one block of words of several fields
 * each). For checks and checkpoints. */
int lbnr_get_distributions(lbnr_ctx* ctx, double* out);

/* Stored distributions of n selected cells, decoded to FP64, into host
 * out[n][16][Q] (standard layout). cells[] holds n cell indices in
 * [0, nx*ny*nz); an index outside that range gives LBNR_EINVAL. Used for
 * sampled checks of lattices too large to copy back whole. */
int lbnr_get_cells(lbnr_ctx* ctx, int64_t n, const int64_t* cells, double* out);

/* Replaces the distributions with host in[16][Q][cells] (encoded to the
 * storage type). With lbnr_get_distributions this gives checkpoint/resume.
 * Keeps the step count. */
int lbnr_set_distributions(lbnr_ctx* ctx, const double* in);

/* LAG only: the lagged fields the next step differentiates, the corrected
 * alpha and gamma_ij of the previous step (the initial fields before the
 * first step), host out[7][cells] FP64 (decoded from the stencil planes: ln
 * alpha and gamma, in the compute type). With lbnr_get_distributions this is
 * a LAG run's whole state. LBNR_ESTATE under SYNC or before init. */
int lbnr_get_lagged(lbnr_ctx* ctx, double* out);

/* LAG only: replaces the lagged fields with host in[7][cells] (alpha > 0,
 * gamma_ij), for checkpoint/resume with lbnr_set_distributions. LBNR_ESTATE
 * under SYNC, LBNR_EINVAL for a non-positive or non-finite lapse. */
int lbnr_set_lagged(lbnr_ctx* ctx, const double* in);

/* The context's LBNR_DERIV_* mode (-1 for NULL). */
int lbnr_deriv_mode(const lbnr_ctx* ctx);

/* Synchronises and returns LBNR_ENONFINITE if any step so far produced a
 * non-finite moment, else LBNR_OK. */
int lbnr_status(lbnr_ctx* ctx);

/* Matter (Sec. "Expansion of flat universe"): a homogeneous perfect fluid at
 * rest in the slice frame, energy density rho(t) = rho0 (t0 / t)^2 (the
 * density of a flat FLRW universe, for any equation of state) and pressure
 * P = w rho, prescribed rather than evolved, as in the paper's test. The
 * state after n steps is at t = t0 + n dt. It enters S_ij through
 * -R^(4)_ij + (gamma_ij / 4) 2 alpha^2 G^00 with G_ij = P gamma_ij and
 * alpha^2 G^00 = rho, which is (P / 2) gamma_ij; Omega_k is unchanged
 * (G^0_k = 0). rho0 = 0 returns to vacuum. Call before lbnr_init (which
 * evaluates the initial sources at t0); later calls take the current step
 * as n. Errors: LBNR_EINVAL for rho0 < 0, t0 <= 0 or non-finite values. */
int lbnr_set_fluid(lbnr_ctx* ctx, double rho0, double w, double t0);

/* Shift (Sec. "Bona-Masso evolution equations"): a constant, uniform shift
 * vector beta^i = (bx, by, bz) in lattice units of dr/dt, so B_k^i = 0 and
 * s_ij = 0. Adds alpha beta^r A_r to the lapse source and 2 beta^r D_rij to
 * the metric source, and the factor 1 - c_l.beta / c_s^2 to the equilibria
 * of K_ij and V_i (fluxes -beta^k K_ij and -beta^k V_i). The collide step
 * then runs in its one shift-carrying launch form (one thread per cell,
 * distributions re-read; any streaming pattern), whatever lbnr_set_variant
 * chose; (0, 0, 0) returns to the zero-shift forms. Call before lbnr_init
 * (the initial equilibria carry the shift); takes effect at the next step.
 * Errors: LBNR_EINVAL for a null context or non-finite values. */
int lbnr_set_shift(lbnr_ctx* ctx, double bx, double by, double bz);

/* Shift field (Sec. "Bona-Masso evolution equations"): a prescribed, static
 * beta^i(x), host beta[3][cells] (x fastest), added to the constant shift of
 * lbnr_set_shift; a gauge choice (the shift equation's Q_i is left free).
 * B_k^i = d_k beta^i / 2 comes from central differences of the field, and
 * the step gains every B term: s_ij = (B_ij + B_ji)/alpha in the metric
 * source, (2/alpha)(K_ir B_j^r + K_jr B_i^r - K_ij trB) in S_ij,
 * 2(B_k^r - delta_k^r trB)V_r + 2(D_rk^s - delta^s_k D^j_jr)B^r_s in Omega_k,
 * and B^r_k - B_k^r in the flux of V_k along r. The field is copied to a
 * device buffer of 24 bytes per cell that the context allocates on the first
 * call and owns (freed by lbnr_destroy or a call with beta = NULL, which
 * removes the field). The collide step then runs its shift-field launch form
 * (one thread per cell). Call before lbnr_init. Errors: LBNR_EINVAL for a
 * null context or a non-finite value, LBNR_ECUDA if the buffer cannot be
 * allocated. */
int lbnr_set_shift_field(lbnr_ctx* ctx, const double* beta);

/* Launch forms of the collide kernel available for this context's set and
 * storage (all give the same results within rounding; every form runs one
 * thread per cell): their number, a short name, and the selection (default
 * 0). Used by the autotuner. Names: "P1-hold" / "P1-reread" (distributions
 * held in registers between the moment and update passes, or read again),
 * with a suffix "-<t>x<b>" for blocks of t threads sized for b blocks per SM
 * (no suffix: 128 x 3); "tma-p1-nc<c>-k<k>-t32" (persistent, fed by bulk
 * copies of whole 32-cell tiles, c consumer warps with k stages each). The
 * bulk-copy-fed forms read each tile's own cells only; at the odd step of the
 * in-place pattern a register form runs in their place. */
int lbnr_num_variants(const lbnr_ctx* ctx);
const char* lbnr_variant_name(const lbnr_ctx* ctx, int variant);
int lbnr_set_variant(lbnr_ctx* ctx, int variant);

/* Steps taken since lbnr_init; Q of the velocity set; the streaming pattern
 * chosen (LBNR_STREAM_PINGPONG or LBNR_STREAM_AA). */
int64_t lbnr_steps_done(const lbnr_ctx* ctx);
int lbnr_q(const lbnr_ctx* ctx);
int lbnr_streaming(const lbnr_ctx* ctx);

/* The FP64 fused multiply-add rate the current device sustains, measured
 * on the given stream (cudaStream_t, NULL = default) by a kernel of
 * independent register-resident FMA chains at full occupancy, best of three
 * timed launches after one warm-up; *tflops in TFLOP/s (2 flops per FMA).
 * The FP64 lattice Boltzmann step is bound by that pipe, not by HBM, and its
 * roofline is quoted against this figure. Synchronises the stream. Errors:
 * LBNR_EINVAL (NULL output), LBNR_ECUDA; message in lbnr_last_error(NULL). */
int lbnr_fp64_fma_rate(void* cuda_stream, double* tflops);

/* Largest lattice lbnr_constraint_norms_noalloc accepts. */
#define LBNR_NOALLOC_MAX_CELLS 2097152

/* The first six values of lbnr_constraints (H_L2, H_inf, M_L2, M_inf, C_L2,
 * C_inf) for corrected fields that are already on the device, computed
 * without allocating any device memory. The paper has no counterpart: this
 * is for callers that must not allocate, such as a run that has handed
 * nearly all device memory to its lattice, or a host framework whose own
 * allocator owns the device memory during its step.
 *   d_fields: device float64 [16][cells], the corrected fields in the field
 *             order above (e.g. what lbnr_moments returns, copied back);
 *   d_out:    device float64 [6], written on the stream;
 *   cuda_stream: cudaStream_t (NULL = default stream). Returns after enqueue.
 * The per-block partial sums live in one fixed array compiled into the
 * library (LBNR_NOALLOC_MAX_CELLS / 128 blocks x 22 doubles, 2.75 MiB); every
 * GPU that loads the library keeps it until the process exits. Lattices of
 * more than LBNR_NOALLOC_MAX_CELLS cells (or with any side above it) give
 * LBNR_EINVAL. The first call on a device looks up the array's device
 * address (with that device current) and keeps it for that device's context;
 * after the context is reset (cudaDeviceReset) the next call looks it up
 * again. So make the first call on each device, and the first after a reset,
 * before any stream capture. d_fields, d_out and the stream must belong to
 * the current device. All calls share the array: calls whose work overlaps on
 * the GPU (different streams, or different host threads) race and must be
 * serialised by the caller. Errors are reported through
 * lbnr_last_error(NULL). */
int lbnr_constraint_norms_noalloc(int vset, const lbnr_grid* grid, double dx,
                                  const double* d_fields, double* d_out, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Batched ensemble: many independent periodic 1D (D1Q3) and 2D (D2Q9)
 * lattices, each with its own size, tau, slicing and step count, advanced by
 * one persistent cooperative kernel launch (captured in a CUDA graph). Every
 * run is the same step as a single context (Eq. numlb with the equilibria
 * and sources of Eqs. (alfa)-(ekstsor), ping-pong streaming); a run of many
 * cells is split over a team of thread blocks that meet at device-side
 * barriers between the moment pass and the collide pass; the other runs
 * wait in a queue, longest first, from which every block without (or done
 * with) a team run takes the next one. The paper runs one lattice at a
 * time; the batch is for parameter scans and convergence studies.
 * ------------------------------------------------------------------------ */
typedef struct lbnr_batch lbnr_batch;

typedef struct {
  int32_t vset;    /* LBNR_D1Q3 or LBNR_D2Q9 */
  int32_t slicing; /* LBNR_GEODESIC / LBNR_HARMONIC / LBNR_ONE_PLUS_LOG */
  lbnr_grid grid;  /* nz = 1; ny = 1 for D1Q3; nx * ny < 2^28 */
  double tau, dx;  /* tau > 1/2 (units of dt); dt = dx */
  int64_t steps;   /* steps this run takes per lbnr_batch_run call */
} lbnr_run_desc;

typedef struct {
  int32_t storage;      /* LBNR_F64 ... LBNR_DEV_F16, for every run */
  int32_t block;        /* threads per block: 128 or 256 (default 256) */
  int32_t ctas_per_sm;  /* resident blocks per SM; 0 = as many as fit */
  int32_t sources_on;   /* 1 normally; 0 drops every source */
  void* cuda_stream;    /* cudaStream_t; NULL = a stream of the batch's own */
  int64_t wait_limit_ns; /* bound of every device-side barrier wait (2 s) */
  int32_t test_drop_arrival_run; /* test hook, -1 normally: block 0 of this
                            run's team skips its first barrier arrival so the
                            run's waits time out */
  int32_t replan;       /* 1: every lbnr_batch_run first calls
                           lbnr_batch_replan (and so waits for the work
                           before it); 0 (default): plan once */
  int32_t deriv_mode;   /* LBNR_DERIV_SYNC (default): per step a moment pass,
                           a team barrier, the collide pass and a barrier;
                           LBNR_DERIV_LAG: the collide pass (it writes the
                           next step's stencil planes) and one barrier */
  int32_t reserved;     /* 0 */
} lbnr_batch_opts;

/* Fills o with the defaults: DEV_F32, 256 threads, all resident blocks,
 * sources on, 2 s wait limit, no dropped arrival, no re-planning, SYNC. */
void lbnr_default_batch_opts(lbnr_batch_opts* o);

/* Validates the runs, allocates every run's two distribution buffers and
 * stencil planes in one device allocation, and plans the block assignment
 * (resident blocks from the occupancy calculator). runs[] is copied. */
int lbnr_batch_create(int nruns, const lbnr_run_desc* runs, const lbnr_batch_opts* opts,
                      lbnr_batch** out);

/* Re-plans for another block size / blocks per SM (the autotuner's knobs). */
int lbnr_batch_configure(lbnr_batch* b, int block, int ctas_per_sm);

/* Synchronises and plans the work again over the runs that are still
 * stepped (not non-finite, not timed out), so that blocks freed by stopped
 * runs join the remaining ones. Keeps the block shape; the captured graph
 * stays valid (the plan lives in device memory). */
int lbnr_batch_replan(lbnr_batch* b);

/* Initial distributions of one run from host fields [16][cells] (same rule as
 * lbnr_init); resets the run's step count and status. Synchronises. */
int lbnr_batch_init(lbnr_batch* b, int run, const double* fields);

/* Enqueues one launch in which every run takes min(max_steps, its steps)
 * steps (max_steps < 0: its steps). A run whose moments turn non-finite
 * stops after the step that read them, and a run whose barrier wait timed
 * out stops where it was; neither is stepped again until lbnr_batch_init.
 * Returns without waiting. */
int lbnr_batch_run(lbnr_batch* b, int64_t max_steps);

/* Synchronises; per_run[r] (optional, nruns entries) receives LBNR_OK,
 * LBNR_ENONFINITE or LBNR_ETIMEOUT for each run; returns the worst. */
int lbnr_batch_status(lbnr_batch* b, int32_t* per_run);

/* Stored distributions of one run decoded to FP64, host out[16][Q][cells]
 * in the standard layout. Synchronises. */
int lbnr_batch_get_distributions(lbnr_batch* b, int run, double* out);

/* The current plan: blocks launched, threads per block, whether the launch is
 * replayed from a CUDA graph (1) or launched directly (0), and the team size
 * (blocks) of every run (team_of_run: nruns entries; 1 for a run stepped by
 * a single block, 0 for a run the plan leaves out because it stopped). Any
 * pointer may be NULL. */
int lbnr_batch_plan(const lbnr_batch* b, int32_t* grid, int32_t* block, int32_t* graphed,
                    int32_t* team_of_run);

/* Steps taken by one run since its lbnr_batch_init, as read back by the last
 * lbnr_batch_status or lbnr_batch_get_distributions; -1 for a bad index. */
int64_t lbnr_batch_steps_done(const lbnr_batch* b, int run);

/* Frees the batch (synchronises first). NULL is a no-op. */
void lbnr_batch_destroy(lbnr_batch* b);

/* Last error message of the batch. */
const char* lbnr_batch_last_error(const lbnr_batch* b);

/* Frees what the context allocated. NULL is a no-op. */
void lbnr_destroy(lbnr_ctx* ctx);

/* Last error message of ctx, or of the calling thread when ctx is NULL. */
const char* lbnr_last_error(const lbnr_ctx* ctx);

/* ------------------------------------------------------------------------
 * Independently evolved A_k and D_kij: the 37-field scheme
 * ------------------------------------------------------------------------
 * The original Bona-Masso formulation evolves A_k = d_k ln alpha and
 * D_kij = d_k gamma_ij / 2 as variables of their own; the paper mentions it
 * and reports that they then drift from the derivatives of alpha and gamma
 * (Sec. "Bona-Masso evolution equations", after the first-order derivatives).
 * This comparison variant evolves them, with zero shift, by
 *   d_t A_k + d_k(alpha Q) = 0,  d_t D_kij + d_k(alpha K_ij) = 0
 * (flux-only sets, equilibria w [A_k + c_k alpha Q / c_s^2] and
 * w [D_kij + c_k alpha K_ij / c_s^2], no sources), and the other 16 fields
 * take A and D from these moments: the step reads no neighbour's moments.
 * Fields: the 16 of lbnr_init, then A_x A_y A_z (16..18), then D_kij at
 * 19 + 6 k + pair(i, j) (pairs xx xy xz yy yz zz). Distributions
 * [37][Q][pstride] (pstride = cells rounded up to 32), ping-pong, FP64 or
 * FP32 storage (arithmetic in the storage type). The context owns its device
 * memory: 2 x 37 x Q x pstride values, plus 37 FP64 values per cell. */
typedef struct lbnr_ad_ctx lbnr_ad_ctx;

/* vset LBNR_D1Q3/D2Q9/D3Q19; tau the dimensionless tau/dt (> 1/2); dt must
 * equal dx; slicing LBNR_GEODESIC/HARMONIC/ONE_PLUS_LOG; storage LBNR_F64 or
 * LBNR_F32; cuda_stream a cudaStream_t or NULL (the context makes one).
 * Errors: LBNR_EINVAL, LBNR_ENOMEM (device memory), LBNR_ECUDA. */
int lbnr_ad_create(const lbnr_grid* grid, int vset, double tau, double dx, double dt,
                   int slicing, int storage, void* cuda_stream, lbnr_ad_ctx** out);

/* Host fields[nfields][cells], nfields 16 (A and D start as second-order
 * central differences of ln alpha and gamma / 2) or 37 (given). Initial
 * distributions f = f_eq - (dt/2) w S, as lbnr_init. Errors: LBNR_EINVAL
 * (NULL, nfields, alpha <= 0), LBNR_ECUDA. */
int lbnr_ad_init(lbnr_ad_ctx* ctx, const double* fields, int nfields);

/* n steps, enqueued on the context's stream (asynchronous). */
int lbnr_ad_step(lbnr_ad_ctx* ctx, int64_t n);

/* n steps timed with CUDA events on the context's stream; *ms_out the total. */
int lbnr_ad_step_timed(lbnr_ad_ctx* ctx, int64_t n, double* ms_out);

/* Corrected moments of the 37 fields into host out[37][cells] (FP64):
 * rho = sum f + dt S / 2 for the 16, the plain sums for A and D. Returns
 * LBNR_ENONFINITE (after the copy) if a step saw a non-finite moment. */
int lbnr_ad_moments(lbnr_ad_ctx* ctx, double* out);

/* LBNR_ENONFINITE if any step so far saw a non-finite moment, else LBNR_OK. */
int lbnr_ad_status(lbnr_ad_ctx* ctx);

/* Distributions to / from host [37][Q][cells] (FP64). */
int lbnr_ad_get_distributions(lbnr_ad_ctx* ctx, double* out);
int lbnr_ad_set_distributions(lbnr_ad_ctx* ctx, const double* in);

int64_t lbnr_ad_steps_done(const lbnr_ad_ctx* ctx);

/* Launch forms of the 37-field collide kernel: blocks of 128 threads with
 * registers sized for lbnr_ad_form_blocks(form) blocks per SM (2 to 5: more
 * warps in flight against more spilled values), and two shared-memory
 * staged forms (lbnr_ad_form_blocks 0: one lane per cell, -1: two lanes per
 * cell, each owning half the words): one persistent block per SM whose
 * producer warp copies each tile of 32 cells, its contiguous block of words,
 * into shared memory with one bulk copy, so every distribution is read from
 * HBM once; their waits are bounded and a timeout sets LBNR_ETIMEOUT in
 * lbnr_ad_status. All forms compute the same values. lbnr_ad_form_blocks
 * returns -100 for an unknown form, lbnr_ad_set_form LBNR_EINVAL. Defaults:
 * 2 blocks per SM with FP64 storage, the one-lane staged form with FP32. */
int lbnr_ad_num_forms(void);
int lbnr_ad_form_blocks(int form);
int lbnr_ad_set_form(lbnr_ad_ctx* ctx, int form);
void lbnr_ad_destroy(lbnr_ad_ctx* ctx);
/* Last error message of ctx (or of the calling thread when ctx is NULL). */
const char* lbnr_ad_last_error(const lbnr_ad_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* LBNR_H */
