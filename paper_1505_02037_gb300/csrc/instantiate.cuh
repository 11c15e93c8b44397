// Launchers for one velocity set; included once per set by inst_q*.cu.
#pragma once

#include "dispatch.h"
#include "kernels.cuh"

namespace lbnr {

// Thread-to-cell layouts of the collide kernel, per compute type and set:
// P threads per cell (1 or 2); HOLD keeps all of a thread's distributions in
// registers between the moment pass and the update pass (else they are read
// again, from cache).
template <int Q, class C>
struct Variants;
template <>
struct Variants<3, double> {
  static constexpr int n = 2;
  static constexpr int P[2] = {1, 1};
  static constexpr bool HOLD[2] = {true, false};
};
template <>
struct Variants<9, double> {
  static constexpr int n = 1;
  static constexpr int P[1] = {1};
  static constexpr bool HOLD[1] = {false};
};
template <>
struct Variants<19, double> {
  static constexpr int n = 1;
  static constexpr int P[1] = {1};
  static constexpr bool HOLD[1] = {false};
};
template <>
struct Variants<3, float> {
  static constexpr int n = 2;
  static constexpr int P[2] = {1, 1};
  static constexpr bool HOLD[2] = {true, false};
};
template <>
struct Variants<9, float> {
  static constexpr int n = 2;
  static constexpr int P[2] = {1, 2};
  static constexpr bool HOLD[2] = {true, true};
};
template <>
struct Variants<19, float> {
  static constexpr int n = 2;
  static constexpr int P[2] = {2, 1};
  static constexpr bool HOLD[2] = {true, false};
};

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
  using V = Variants<Q, C>;

  static const char* variant_name(int v) {
    static char buf[2][32];
    if (v < 0 || v >= V::n) return "?";
    snprintf(buf[v], sizeof(buf[v]), "P%d%s", V::P[v], V::HOLD[v] ? "-hold" : "-reread");
    return buf[v];
  }

  template <int LAYOUT, int VI>
  static cudaError_t launch_collide(const LaunchCtx& L, const StepArgs<S, C>& a) {
    constexpr int P = V::P[VI < V::n ? VI : 0];
    constexpr bool H = V::HOLD[VI < V::n ? VI : 0];
    const int block = 128;
    const int64_t threads = P == 2 ? ((L.cells + 15) / 16) * 32 : L.cells;
    k_collide<Q, S, C, REP, LAYOUT, P, H><<<grid_for(threads, block), block, 0, L.st>>>(a);
    return cudaGetLastError();
  }

  template <int LAYOUT>
  static cudaError_t collide_layout(const LaunchCtx& L, int variant, const StepArgs<S, C>& a) {
    if (variant == 1 && V::n > 1) return launch_collide<LAYOUT, 1>(L, a);
    return launch_collide<LAYOUT, 0>(L, a);
  }

  static cudaError_t step(const LaunchCtx& L, int layout, int variant, const void* fin, void* fout) {
    StepArgs<S, C> a;
    a.fin = static_cast<const S*>(fin);
    a.fout = static_cast<S*>(fout);
    a.aux = static_cast<const C*>(L.aux);
    a.flag = L.flag;
    a.G = Grid{L.nx, L.ny, L.nz, L.cells};
    a.inv2dx = C(1.0 / (2.0 * L.dx));
    a.inv4dx = C(1.0 / (4.0 * L.dx));
    a.half_dt = C(0.5 * L.dt);
    a.omega = C(1.0 / L.tau);
    a.omc = C(1.0 - 1.0 / L.tau);
    a.sigma = C(L.dt * (1.0 - 1.0 / (2.0 * L.tau)));
    a.slicing = L.slicing;
    a.sources_on = L.sources_on;
    if (layout == kPingPong) return collide_layout<kPingPong>(L, variant, a);
    if (layout == kAAEven) return collide_layout<kAAEven>(L, variant, a);
    return collide_layout<kAAOdd>(L, variant, a);
  }

  static cudaError_t aux(const LaunchCtx& L, int layout, const void* f) {
    const Grid G{L.nx, L.ny, L.nz, L.cells};
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
    a.G = Grid{L.nx, L.ny, L.nz, L.cells};
    a.inv2dx = 1.0 / (2.0 * L.dx);
    a.inv4dx = 1.0 / (4.0 * L.dx);
    a.half_dt = 0.5 * L.dt;
    a.slicing = L.slicing;
    a.sources_on = L.sources_on;
    k_init<Q, S, REP><<<grid_for(L.cells, 128), 128, 0, L.st>>>(a);
    return cudaGetLastError();
  }

  static cudaError_t sum64(const LaunchCtx& L, int layout, const void* f, int64_t* nblocks) {
    const Grid G{L.nx, L.ny, L.nz, L.cells};
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
    const Grid G{L.nx, L.ny, L.nz, L.cells};
    k_correct64<Q><<<grid_for(L.cells, 128), 128, 0, L.st>>>(
        L.macro, L.aux64, G, 1.0 / (2.0 * L.dx), 1.0 / (4.0 * L.dx), 0.5 * L.dt, L.slicing,
        L.sources_on);
    return cudaGetLastError();
  }

  static cudaError_t constraints64(const LaunchCtx& L, int64_t* nblocks) {
    const Grid G{L.nx, L.ny, L.nz, L.cells};
    const unsigned grid = grid_for(L.cells, 128);
    *nblocks = grid;
    k_constraints64<Q><<<grid, 128, 0, L.st>>>(L.macro, G, 1.0 / (2.0 * L.dx), 1.0 / (4.0 * L.dx),
                                               L.partials);
    return cudaGetLastError();
  }

  static cudaError_t get_plane(const LaunchCtx& L, int layout, const void* f, int F, int l,
                               double* out) {
    const Grid G{L.nx, L.ny, L.nz, L.cells};
    const unsigned grid = grid_for(L.cells, 256);
    const S* fp = static_cast<const S*>(f);
    if (layout == kPingPong) k_get_plane<Q, S, REP, kPingPong><<<grid, 256, 0, L.st>>>(fp, out, G, F, l);
    else if (layout == kAAEven) k_get_plane<Q, S, REP, kAAEven><<<grid, 256, 0, L.st>>>(fp, out, G, F, l);
    else k_get_plane<Q, S, REP, kAAOdd><<<grid, 256, 0, L.st>>>(fp, out, G, F, l);
    return cudaGetLastError();
  }

  static cudaError_t set_plane(const LaunchCtx& L, int layout, void* f, int F, int l,
                               const double* in) {
    const Grid G{L.nx, L.ny, L.nz, L.cells};
    const unsigned grid = grid_for(L.cells, 256);
    S* fp = static_cast<S*>(f);
    if (layout == kPingPong) k_set_plane<Q, S, REP, kPingPong><<<grid, 256, 0, L.st>>>(fp, in, G, F, l);
    else if (layout == kAAEven) k_set_plane<Q, S, REP, kAAEven><<<grid, 256, 0, L.st>>>(fp, in, G, F, l);
    else k_set_plane<Q, S, REP, kAAOdd><<<grid, 256, 0, L.st>>>(fp, in, G, F, l);
    return cudaGetLastError();
  }

  static cudaError_t get_cells(const LaunchCtx& L, int layout, const void* f, int64_t n,
                               const int64_t* idx, double* out) {
    const Grid G{L.nx, L.ny, L.nz, L.cells};
    const unsigned grid = grid_for(n * kNF, 128);
    const S* fp = static_cast<const S*>(f);
    if (layout == kPingPong) k_get_cells<Q, S, REP, kPingPong><<<grid, 128, 0, L.st>>>(fp, idx, n, out, G);
    else if (layout == kAAEven) k_get_cells<Q, S, REP, kAAEven><<<grid, 128, 0, L.st>>>(fp, idx, n, out, G);
    else k_get_cells<Q, S, REP, kAAOdd><<<grid, 128, 0, L.st>>>(fp, idx, n, out, G);
    return cudaGetLastError();
  }

  static const Ops* ops() {
    static const Ops o = {V::n,      &variant_name, &step,          &aux,       &init,
                          &sum64,    &correct64,    &constraints64, &get_plane, &set_plane,
                          &get_cells};
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
