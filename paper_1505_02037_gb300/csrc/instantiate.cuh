// Launchers for one velocity set; included once per set by inst_q*.cu.
#pragma once

#include "dispatch.h"

#include "collide_tma.cuh"
#include "kernels.cuh"

namespace lbnr {

// Launch forms of the collide kernel, per velocity set and storage width.
// Every form runs one thread (lane) per cell, P = 1 (the P in the names).
// kind 0: blocks of 128 threads; HOLD keeps a thread's distributions in
//         registers between the moment pass and the update pass (else they
//         are read again, from cache). Any layout.
// kind 1: bulk-copy-fed persistent kernel (collide_tma.cuh) with NC consumer
//         warps and NC K shared-memory stages of one 32-cell tile; local
//         reads only, so at the odd AA step it hands over to the form named
//         by `fallback`.
struct VariantSpec {
  int kind, P;
  bool hold;
  int nc, k, tc;  // consumer warps, stages per warp, cells per tile (kind 1)
  int tpb, minb;  // kind 0, word forms: threads per block and the blocks per SM the
                  // registers are sized for (0: 128 and 3)
};

template <int Q, int SB>
struct VariantTable;
#define LBNR_VARIANTS(Q_, SB_, FALLBACK_, ...)              \
  template <>                                                \
  struct VariantTable<Q_, SB_> {                             \
    static constexpr VariantSpec v[] = {__VA_ARGS__};        \
    static constexpr int n = sizeof(v) / sizeof(v[0]);       \
    static_assert(n <= 8, "at most 8 launch forms");         \
    static constexpr int fallback = FALLBACK_;               \
  };
// FP64 storage (FP64 arithmetic)
LBNR_VARIANTS(3, 8, 0, {0, 1, true, 0, 0, 0}, {1, 1, false, 8, 1, 32})
LBNR_VARIANTS(9, 8, 0, {0, 1, false, 0, 0, 0}, {1, 1, false, 4, 1, 32})
LBNR_VARIANTS(19, 8, 0, {0, 1, false, 0, 0, 0}, {1, 1, false, 2, 1, 32})
// FP32 and 16-bit storage: one lane per cell, word by word. (Forms with two
// lanes per cell split a word's fields between the lanes; on the word
// layout they ran at half the speed and are not offered.) The re-read forms
// come in three block shapes: 128 threads x 3 blocks per SM (168 registers),
// 64 x 4 and 128 x 2 (255 registers, 8 warps per SM: fewer cells resident,
// so more of the update pass's re-read stays in L2).
LBNR_VARIANTS(3, 4, 1, {1, 1, false, 8, 4, 32}, {0, 1, true, 0, 0, 0}, {0, 1, false, 0, 0, 0},
              {0, 1, false, 0, 0, 0, 64, 4})
LBNR_VARIANTS(9, 4, 1, {1, 1, false, 4, 2, 32}, {0, 1, true, 0, 0, 0}, {0, 1, false, 0, 0, 0},
              {0, 1, false, 0, 0, 0, 64, 4})
LBNR_VARIANTS(19, 4, 2, {1, 1, false, 4, 1, 32}, {1, 1, false, 5, 1, 32}, {0, 1, false, 0, 0, 0},
              {0, 1, false, 0, 0, 0, 64, 4}, {0, 1, false, 0, 0, 0, 128, 2})
LBNR_VARIANTS(3, 2, 1, {1, 1, false, 8, 4, 32}, {0, 1, true, 0, 0, 0}, {0, 1, false, 0, 0, 0},
              {0, 1, false, 0, 0, 0, 64, 4})
LBNR_VARIANTS(9, 2, 1, {1, 1, false, 8, 2, 32}, {0, 1, true, 0, 0, 0}, {0, 1, false, 0, 0, 0},
              {0, 1, false, 0, 0, 0, 64, 4})
LBNR_VARIANTS(19, 2, 1, {1, 1, false, 8, 1, 32}, {0, 1, false, 0, 0, 0},
              {0, 1, false, 0, 0, 0, 64, 4}, {0, 1, false, 0, 0, 0, 128, 2})
#undef LBNR_VARIANTS

inline int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <class S>
struct ComputeOf {
  using type = float;
};
template <>
struct ComputeOf<double> {
  using type = double;
};

inline unsigned grid_for(int64_t threads, int block) {
  return (unsigned)((threads + block - 1) / block);
}

template <int Q, class S, int REP>
struct Impl {
  using C = typename ComputeOf<S>::type;
  using VT = VariantTable<Q, (int)sizeof(S)>;

  static const char* variant_name(int v) {
    static char buf[8][48];
    if (v < 0 || v >= VT::n || v >= 8) return "?";
    const VariantSpec& x = VT::v[v];
    if (x.kind == 0 && x.tpb > 0)
      snprintf(buf[v], sizeof(buf[v]), "P%d%s-%dx%d", x.P, x.hold ? "-hold" : "-reread", x.tpb,
               x.minb);
    else if (x.kind == 0)
      snprintf(buf[v], sizeof(buf[v]), "P%d%s", x.P, x.hold ? "-hold" : "-reread");
    else
      snprintf(buf[v], sizeof(buf[v]), "tma-p%d-nc%d-k%d-t%d", x.P, x.nc, x.k, x.tc);
    return buf[v];
  }

  template <int LAYOUT, int VI>
  static cudaError_t launch_generic(const LaunchCtx& L, const StepArgs<S, C>& a) {
    constexpr VariantSpec x = VT::v[VI];
    static_assert(x.P == 1, "one thread per cell");
    constexpr bool H = x.hold;
    const int block = 128;
    const int64_t threads = L.cells;
    if constexpr (Codec<S>::kV > 1) {
      // one thread per cell, word by word. The default shape, 128 threads
      // sized for 3 blocks per SM with or without the lagged-field writes,
      // takes 2 at the odd AA step, which holds a field group's Q words and
      // reads and writes at neighbours.
      constexpr int TPB = x.tpb > 0 ? x.tpb : 128;
      constexpr int WMINB = x.minb > 0 ? x.minb : (LAYOUT == kAAOdd ? 2 : 3);
      if (a.aux_out)
        k_collide_w<Q, S, C, REP, LAYOUT, H, WMINB, true, 0, TPB>
            <<<grid_for(threads, TPB), TPB, 0, L.st>>>(a);
      else
        k_collide_w<Q, S, C, REP, LAYOUT, H, WMINB, false, 0, TPB>
            <<<grid_for(threads, TPB), TPB, 0, L.st>>>(a);
    } else {
      // the lagged-field writes cost registers: sized for 2 blocks per SM
      if (a.aux_out)
        k_collide<Q, S, C, REP, LAYOUT, H, 0, 2, true>
            <<<grid_for(threads, block), block, 0, L.st>>>(a);
      else
        k_collide<Q, S, C, REP, LAYOUT, H><<<grid_for(threads, block), block, 0, L.st>>>(a);
    }
    return cudaGetLastError();
  }

  // Registers of the shift forms. FP64 (value by value): 3 blocks of 128
  // threads per SM (the FP64 step is bound by its arithmetic; 8.9 against
  // 9.3 ms at 128^3). FP32 and 16-bit storage (word by word): 3 blocks with
  // a constant shift, which fits 168 registers without spills outside the
  // odd AA step, else 2 (255 registers; 3 would spill).
  template <int LAYOUT, int SHIFT>
  static cudaError_t launch_shifted(const LaunchCtx& L, const StepArgs<S, C>& a) {
    constexpr int MINB = sizeof(C) == 8 ? 3 : 2;
    constexpr int WMINB = SHIFT == 1 && LAYOUT != kAAOdd ? 3 : 2;
    const int block = 128;
    if constexpr (Codec<S>::kV > 1) {
      if (a.aux_out)
        k_collide_w<Q, S, C, REP, LAYOUT, false, WMINB, true, SHIFT>
            <<<grid_for(L.cells, block), block, 0, L.st>>>(a);
      else
        k_collide_w<Q, S, C, REP, LAYOUT, false, WMINB, false, SHIFT>
            <<<grid_for(L.cells, block), block, 0, L.st>>>(a);
    } else {
      if (a.aux_out)
        k_collide<Q, S, C, REP, LAYOUT, false, SHIFT, MINB, true>
            <<<grid_for(L.cells, block), block, 0, L.st>>>(a);
      else
        k_collide<Q, S, C, REP, LAYOUT, false, SHIFT, MINB>
            <<<grid_for(L.cells, block), block, 0, L.st>>>(a);
    }
    return cudaGetLastError();
  }

  template <int LAYOUT, int VI>
  static cudaError_t launch_tma(const LaunchCtx& L, const StepArgs<S, C>& a) {
    constexpr VariantSpec x = VT::v[VI];
    constexpr int NC = x.nc > 0 ? x.nc : 1;
    constexpr int K = x.k > 0 ? x.k : 1;
    static_assert(x.P == 1, "one lane per cell");
    constexpr int TC = x.tc > 0 ? x.tc : kTileCells;
    constexpr int NS = NC * K;
    constexpr uint32_t smem = tma_smem_bytes(tma_stage_bytes<S>(Q, TC), NS);
    static_assert(smem <= 232448, "shared memory per block");
    auto kern = k_collide_tma<Q, S, C, REP, LAYOUT, NC, K, TC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t ntiles = L.pstride / TC;
    const int64_t grid = ntiles < sm_count() ? ntiles : sm_count();
    kern<<<(unsigned)grid, 32 * (NC + 1), smem, L.st>>>(a, ntiles);
    return cudaGetLastError();
  }

  template <int LAYOUT, int VI>
  static cudaError_t launch_variant(const LaunchCtx& L, const StepArgs<S, C>& a) {
    if constexpr (VT::v[VI].kind == 1) {
      if constexpr (LAYOUT == kAAOdd)
        return launch_generic<LAYOUT, VT::fallback>(L, a);
      else
        return launch_tma<LAYOUT, VI>(L, a);
    } else {
      return launch_generic<LAYOUT, VI>(L, a);
    }
  }

  template <int LAYOUT>
  static cudaError_t collide_layout(const LaunchCtx& L, int variant, const StepArgs<S, C>& a) {
    if constexpr (VT::n > 7) {
      if (variant == 7) return launch_variant<LAYOUT, 7>(L, a);
    }
    if constexpr (VT::n > 6) {
      if (variant == 6) return launch_variant<LAYOUT, 6>(L, a);
    }
    if constexpr (VT::n > 5) {
      if (variant == 5) return launch_variant<LAYOUT, 5>(L, a);
    }
    if constexpr (VT::n > 4) {
      if (variant == 4) return launch_variant<LAYOUT, 4>(L, a);
    }
    if constexpr (VT::n > 3) {
      if (variant == 3) return launch_variant<LAYOUT, 3>(L, a);
    }
    if constexpr (VT::n > 2) {
      if (variant == 2) return launch_variant<LAYOUT, 2>(L, a);
    }
    if constexpr (VT::n > 1) {
      if (variant == 1) return launch_variant<LAYOUT, 1>(L, a);
    }
    return launch_variant<LAYOUT, 0>(L, a);
  }

  static cudaError_t step(const LaunchCtx& L, int layout, int variant, const void* fin, void* fout) {
    StepArgs<S, C> a;
    a.fin = static_cast<const S*>(fin);
    a.fout = static_cast<S*>(fout);
    a.aux = static_cast<const C*>(L.aux);
    a.aux_out = static_cast<C*>(L.aux_out);
    a.flag = L.flag;
    a.G = make_grid(L.nx, L.ny, L.nz, L.cells, L.pstride);
    a.inv2dx = C(1.0 / (2.0 * L.dx));
    a.inv4dx = C(1.0 / (4.0 * L.dx));
    a.half_dt = C(0.5 * L.dt);
    a.omega = C(1.0 / L.tau);
    a.omc = C(1.0 - 1.0 / L.tau);
    a.sigma = C(L.dt * (1.0 - 1.0 / (2.0 * L.tau)));
    a.slicing = L.slicing;
    a.sources_on = L.sources_on;
    a.clock = L.clock;
    a.fluid_P0 = L.fluid_P0;
    a.fluid_t0 = L.fluid_t0;
    a.fluid_dt = L.dt;
    for (int k = 0; k < 3; ++k) a.beta[k] = C(L.beta[k]);
    a.beta_field = L.beta_field;
    if (L.beta_field) {
      // A shift field: its own form (B terms), P1-reread, any layout.
      if (layout == kPingPong) return launch_shifted<kPingPong, 2>(L, a);
      if (layout == kAAEven) return launch_shifted<kAAEven, 2>(L, a);
      return launch_shifted<kAAOdd, 2>(L, a);
    }
    if (L.shift_on) {
      // One launch form carries the constant shift: P1-reread, any layout.
      if (layout == kPingPong) return launch_shifted<kPingPong, 1>(L, a);
      if (layout == kAAEven) return launch_shifted<kAAEven, 1>(L, a);
      return launch_shifted<kAAOdd, 1>(L, a);
    }
    if (layout == kPingPong) return collide_layout<kPingPong>(L, variant, a);
    if (layout == kAAEven) return collide_layout<kAAEven>(L, variant, a);
    return collide_layout<kAAOdd>(L, variant, a);
  }

  static cudaError_t aux(const LaunchCtx& L, int layout, const void* f) {
    const Grid G = make_grid(L.nx, L.ny, L.nz, L.cells, L.pstride);
    const unsigned grid = grid_for(L.cells, 256);
    const S* fp = static_cast<const S*>(f);
    C* ap = static_cast<C*>(L.aux);
    if (layout == kPingPong) k_aux<Q, S, C, REP, kPingPong><<<grid, 256, 0, L.st>>>(fp, ap, G);
    else if (layout == kAAEven) k_aux<Q, S, C, REP, kAAEven><<<grid, 256, 0, L.st>>>(fp, ap, G);
    else k_aux<Q, S, C, REP, kAAOdd><<<grid, 256, 0, L.st>>>(fp, ap, G);
    return cudaGetLastError();
  }

  static cudaError_t init(const LaunchCtx& L, void* f) {
    Init64Args<S> a;
    a.fields = L.macro;
    a.f = static_cast<S*>(f);
    a.flag = L.flag;
    a.G = make_grid(L.nx, L.ny, L.nz, L.cells, L.pstride);
    a.inv2dx = 1.0 / (2.0 * L.dx);
    a.inv4dx = 1.0 / (4.0 * L.dx);
    a.half_dt = 0.5 * L.dt;
    a.slicing = L.slicing;
    a.sources_on = L.sources_on;
    a.fluidP = L.clock ? L.fluid_P0 : 0.0;  // the initial state is at t0
    for (int k = 0; k < 3; ++k) a.beta[k] = L.beta[k];
    a.shift_on = L.shift_on;
    a.beta_field = L.beta_field;
    k_init<Q, S, REP><<<grid_for(L.cells, 128), 128, 0, L.st>>>(a);
    return cudaGetLastError();
  }

  static cudaError_t sum64(const LaunchCtx& L, int layout, const void* f, int64_t* nblocks) {
    const Grid G = make_grid(L.nx, L.ny, L.nz, L.cells, L.pstride);
    const unsigned grid = grid_for(L.cells, 256);
    *nblocks = grid;
    const S* fp = static_cast<const S*>(f);
    if (layout == kPingPong)
      k_sum64<Q, S, REP, kPingPong><<<grid, 256, 0, L.st>>>(fp, L.macro, L.aux64, L.partials, G);
    else if (layout == kAAEven)
      k_sum64<Q, S, REP, kAAEven><<<grid, 256, 0, L.st>>>(fp, L.macro, L.aux64, L.partials, G);
    else
      k_sum64<Q, S, REP, kAAOdd><<<grid, 256, 0, L.st>>>(fp, L.macro, L.aux64, L.partials, G);
    return cudaGetLastError();
  }

  static cudaError_t correct64(const LaunchCtx& L) {
    const Grid G = make_grid(L.nx, L.ny, L.nz, L.cells, L.pstride);
    k_correct64<Q><<<grid_for(L.cells, 128), 128, 0, L.st>>>(
        L.macro, L.aux64, G, 1.0 / (2.0 * L.dx), 1.0 / (4.0 * L.dx), 0.5 * L.dt, L.slicing,
        L.sources_on, L.clock ? L.fluid_P_now : 0.0, L.shift_on ? L.beta[0] : 0.0,
        L.shift_on ? L.beta[1] : 0.0, L.shift_on ? L.beta[2] : 0.0, L.beta_field);
    return cudaGetLastError();
  }

  static cudaError_t constraints64(const LaunchCtx& L, int64_t* nblocks) {
    const Grid G = make_grid(L.nx, L.ny, L.nz, L.cells, L.pstride);
    const unsigned grid = grid_for(L.cells, 128);
    *nblocks = grid;
    k_constraints64<Q><<<grid, 128, 0, L.st>>>(L.macro, G, 1.0 / (2.0 * L.dx), 1.0 / (4.0 * L.dx),
                                               L.partials);
    return cudaGetLastError();
  }

  static cudaError_t get_plane(const LaunchCtx& L, int layout, const void* f, int F, int l,
                               double* out) {
    const Grid G = make_grid(L.nx, L.ny, L.nz, L.cells, L.pstride);
    const unsigned grid = grid_for(L.cells, 256);
    const S* fp = static_cast<const S*>(f);
    if (layout == kPingPong) k_get_plane<Q, S, REP, kPingPong><<<grid, 256, 0, L.st>>>(fp, out, G, F, l);
    else if (layout == kAAEven) k_get_plane<Q, S, REP, kAAEven><<<grid, 256, 0, L.st>>>(fp, out, G, F, l);
    else k_get_plane<Q, S, REP, kAAOdd><<<grid, 256, 0, L.st>>>(fp, out, G, F, l);
    return cudaGetLastError();
  }

  static cudaError_t set_plane(const LaunchCtx& L, int layout, void* f, int F, int l,
                               const double* in) {
    const Grid G = make_grid(L.nx, L.ny, L.nz, L.cells, L.pstride);
    const unsigned grid = grid_for(L.cells, 256);
    S* fp = static_cast<S*>(f);
    if (layout == kPingPong) k_set_plane<Q, S, REP, kPingPong><<<grid, 256, 0, L.st>>>(fp, in, G, F, l);
    else if (layout == kAAEven) k_set_plane<Q, S, REP, kAAEven><<<grid, 256, 0, L.st>>>(fp, in, G, F, l);
    else k_set_plane<Q, S, REP, kAAOdd><<<grid, 256, 0, L.st>>>(fp, in, G, F, l);
    return cudaGetLastError();
  }

  static cudaError_t get_cells(const LaunchCtx& L, int layout, const void* f, int64_t n,
                               const int64_t* idx, double* out) {
    const Grid G = make_grid(L.nx, L.ny, L.nz, L.cells, L.pstride);
    const unsigned grid = grid_for(n * kNF, 128);
    const S* fp = static_cast<const S*>(f);
    if (layout == kPingPong) k_get_cells<Q, S, REP, kPingPong><<<grid, 128, 0, L.st>>>(fp, idx, n, out, G);
    else if (layout == kAAEven) k_get_cells<Q, S, REP, kAAEven><<<grid, 128, 0, L.st>>>(fp, idx, n, out, G);
    else k_get_cells<Q, S, REP, kAAOdd><<<grid, 128, 0, L.st>>>(fp, idx, n, out, G);
    return cudaGetLastError();
  }

  static cudaError_t lag_from64(const LaunchCtx& L, void* aux) {
    k_lag_from64<C, REP><<<grid_for(L.cells, 256), 256, 0, L.st>>>(L.macro, static_cast<C*>(aux),
                                                                 L.cells);
    return cudaGetLastError();
  }

  static cudaError_t lag_to64(const LaunchCtx& L, const void* aux, double* out) {
    k_lag_to64<C, REP><<<grid_for(L.cells, 256), 256, 0, L.st>>>(static_cast<const C*>(aux),
                                                               L.aux64, out, L.cells);
    return cudaGetLastError();
  }

  static const Ops* ops() {
    static const Ops o = {VT::n,     &variant_name, &step,          &aux,       &init,
                          &sum64,    &correct64,    &constraints64, &get_plane, &set_plane,
                          &get_cells, &lag_from64,  &lag_to64};
    return &o;
  }
};

// storage codes as in lbnr.h: 0 F64, 1 F32, 2 DEV_F32, 3 DEV_BF16, 4 DEV_F16
template <int Q, int STORAGE>
const Ops* ops_for() {
  if constexpr (STORAGE == 0) return Impl<Q, double, kABS>::ops();
  else if constexpr (STORAGE == 1) return Impl<Q, float, kABS>::ops();
  else if constexpr (STORAGE == 2) return Impl<Q, float, kDEV>::ops();
  else if constexpr (STORAGE == 3) return Impl<Q, __nv_bfloat16, kDEV>::ops();
  else return Impl<Q, __half, kDEV>::ops();
}

}  // namespace lbnr
