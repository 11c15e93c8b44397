// Internal interface between the C-ABI (capi.cu) and the per-velocity-set
// translation units that instantiate the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbnr {

constexpr uint64_t kStageBytes = 1ull << 20;
constexpr int64_t kTile = 32;  // cells per tile of the tile-blocked distribution layout

struct LaunchCtx {
  int32_t nx, ny, nz;
  int64_t cells;
  int64_t pstride;  // cells rounded up to whole tiles (kTile)
  double dx, dt, tau;
  int slicing, sources_on;
  void* aux;        // 7 planes of the compute type (stencil input)
  void* aux_out;    // LAG (reading R17): the step writes its corrected lapse and
                    // metric here for the next step; nullptr under R5
  double* macro;    // 16 FP64 planes (fields, moments)
  double* aux64;    // 7 FP64 planes (stencil input of the FP64 kernels)
  double* partials; // per-block reduction partials, 22 doubles each
  double* out22;    // reduction result
  void* stage;      // staging area for sampled transfers (kStageBytes)
  int* flag;        // non-finite flag
  cudaStream_t st;
  int block;        // threads per block of the collide kernel
  // Matter (perfect fluid at rest): pressure P0 (t0/t)^2 at t = t0 + n dt;
  // clock points at the device step counter n (nullptr: vacuum), P_now is
  // the pressure at the state the FP64 moment calls read.
  const int64_t* clock;
  double fluid_P0, fluid_t0, fluid_P_now;
  // Shift: constant beta^i plus an optional static field [3][cells] (FP64,
  // nullptr: none); shift_on = 0 when both are absent or zero.
  double beta[3];
  int shift_on;
  const double* beta_field;
};

// layout: 0 ping-pong, 1 AA at even step, 2 AA at odd step
struct Ops {
  int nvariants;
  const char* (*variant_name)(int variant);
  cudaError_t (*step)(const LaunchCtx&, int layout, int variant, const void* fin, void* fout);
  cudaError_t (*aux)(const LaunchCtx&, int layout, const void* f);
  cudaError_t (*init)(const LaunchCtx&, void* f);  // from macro, standard layout
  cudaError_t (*sum64)(const LaunchCtx&, int layout, const void* f, int64_t* nblocks);
  cudaError_t (*correct64)(const LaunchCtx&);
  cudaError_t (*constraints64)(const LaunchCtx&, int64_t* nblocks);
  cudaError_t (*get_plane)(const LaunchCtx&, int layout, const void* f, int F, int l, double* out);
  cudaError_t (*set_plane)(const LaunchCtx&, int layout, void* f, int F, int l, const double* in);
  cudaError_t (*get_cells)(const LaunchCtx&, int layout, const void* f, int64_t n,
                           const int64_t* idx, double* out);
  // LAG: stencil planes `aux` from the FP64 fields in macro; and back to FP64
  // (aux64, plus the fields alpha and gamma into out when it is not null)
  cudaError_t (*lag_from64)(const LaunchCtx&, void* aux);
  cudaError_t (*lag_to64)(const LaunchCtx&, const void* aux, double* out);
};

// One getter per (velocity set, storage), each in its own translation unit
// so the kernels compile in parallel.
#define LBNR_DECLARE_OPS(q)                                                           \
  const Ops* ops_q##q##_s0();                                                         \
  const Ops* ops_q##q##_s1();                                                         \
  const Ops* ops_q##q##_s2();                                                         \
  const Ops* ops_q##q##_s3();                                                         \
  const Ops* ops_q##q##_s4();
LBNR_DECLARE_OPS(3)
LBNR_DECLARE_OPS(9)
LBNR_DECLARE_OPS(19)
#undef LBNR_DECLARE_OPS

size_t storage_bytes(int storage);
void set_thread_error(const char* msg);  // message for lbnr_last_error(NULL)
bool storage_is_fp64(int storage);

}  // namespace lbnr
