// Kernels of one lattice Boltzmann step for the Bona-Masso system
// (Ilseven & Mendoza, arXiv:1505.02037): Eq. numlb with the equilibria and
// source distributions of Eqs. alfa-ekstsor and the moment rule
// rho = sum_l f_l + dt S / 2 (Sec. "Lattice Boltzmann Model").
//
// One step = k_aux (zeroth moments of alpha and gamma -> 7 planes used by the
// derivative stencil) + the collide kernel (k_collide_w, word by word, for
// FP32 and 16-bit storage; k_collide, value by value, for FP64; or the
// bulk-copy-fed k_collide_tma): moments of all 16 fields, A and D by central
// differences, sources at rho~, corrected rho, flux at rho, equilibria, BGK
// relaxation plus source, streaming. Under LAG (reading R17) the collide
// kernel writes the next step's stencil planes itself and k_aux goes.
//
// Memory: tile-blocked words (fidx below). The 16 Q values of 32 consecutive
// cells (x fastest) form one block; a word holds kV fields of one cell and
// velocity, and a warp's 32 cells of one (word, l) are one aligned row.
//
// Streaming layouts (the state after n steps):
//   ping-pong: f_l(x) at (l, x) of the current buffer; a step writes f*_l(x)
//              to (l, x + c_l) of the other buffer.
//   AA in place, n even: f_l(x) at (l, x); the step writes f*_l(x) to
//              (opp(l), x): no neighbour access.
//   AA in place, n odd:  f_l(x) at (opp(l), x - c_l); the step writes f*_l(x)
//              to (l, x + c_l), which is exactly where it read opp(l), so
//              every cell reads and writes the same locations and no two
//              cells touch the same location.
//
// Representations: ABS holds f itself; DEV holds g = f/w_l - rho_flat,F
// (rho_flat: alpha = 1, gamma = delta, K = V = 0). In DEV form the update
// f* = (1-w) f + w_l (omega rho + 3 omega c.F + sigma S) becomes
// g* = (1-omega) g + omega (rho - rho_flat) + sigma S + 3 omega c.F.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lattice.cuh"
#include "physics.cuh"

namespace lbnr {

enum : int { kABS = 0, kDEV = 1 };
enum : int { kPingPong = 0, kAAEven = 1, kAAOdd = 2 };

// ---------------------------------------------------------------------------
// Storage codecs
// ---------------------------------------------------------------------------
template <class S>
struct Codec;
template <>
struct Codec<double> {
  // one value per distribution word (see the layout below)
  static constexpr int kV = 1;
  using W = double;
  __device__ static __forceinline__ double load(const double* p) { return __ldcs(p); }
  __device__ static __forceinline__ double load_keep(const double* p) { return __ldg(p); }
  __device__ static __forceinline__ double load_coh(const double* p) { return __ldcg(p); }
  __device__ static __forceinline__ void store(double* p, double v) { __stcs(p, v); }
  // Store under a predicate without a branch.
  __device__ static __forceinline__ void store_if(double* p, double v, bool q) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p st.global.cs.f64 [%0], %1;\n}\n" ::"l"(p),
                 "d"(v), "r"((int)q)
                 : "memory");
  }
};
template <>
struct Codec<float> {
  // four values per word: fields 4m .. 4m + 3 (.x .. .w)
  static constexpr int kV = 4;
  using W = float4;
  __device__ static __forceinline__ void unpack(W w, float* v) {
    v[0] = w.x;
    v[1] = w.y;
    v[2] = w.z;
    v[3] = w.w;
  }
  __device__ static __forceinline__ W pack(const float* v) { return make_float4(v[0], v[1], v[2], v[3]); }
  __device__ static __forceinline__ float load(const float* p) { return __ldcs(p); }
  __device__ static __forceinline__ float load_keep(const float* p) { return __ldg(p); }
  __device__ static __forceinline__ float load_coh(const float* p) { return __ldcg(p); }
  __device__ static __forceinline__ void store(float* p, float v) { __stcs(p, v); }
  __device__ static __forceinline__ void store_if(float* p, float v, bool q) {
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p st.global.cs.f32 [%0], %1;\n}\n" ::"l"(p),
                 "f"(v), "r"((int)q)
                 : "memory");
  }
};
template <>
struct Codec<__nv_bfloat16> {
  // four values per word: fields 4m .. 4m + 3, lowest half first
  static constexpr int kV = 4;
  using W = uint2;
  __device__ static __forceinline__ void unpack(W w, float* v) {
    // bfloat16 -> float is exact: the top half of the float
    v[0] = __uint_as_float(w.x << 16);
    v[1] = __uint_as_float(w.x & 0xffff0000u);
    v[2] = __uint_as_float(w.y << 16);
    v[3] = __uint_as_float(w.y & 0xffff0000u);
  }
  __device__ static __forceinline__ W pack(const float* v) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(v[0], v[1]);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(v[2], v[3]);
    return make_uint2((uint32_t)__bfloat16_as_ushort(h0.x) | ((uint32_t)__bfloat16_as_ushort(h0.y) << 16),
                      (uint32_t)__bfloat16_as_ushort(h1.x) | ((uint32_t)__bfloat16_as_ushort(h1.y) << 16));
  }
  __device__ static __forceinline__ float load(const __nv_bfloat16* p) {
    return __bfloat162float(__ldcs(p));
  }
  __device__ static __forceinline__ float load_keep(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
  }
  __device__ static __forceinline__ float load_coh(const __nv_bfloat16* p) {
    return __bfloat162float(__ldcg(p));
  }
  __device__ static __forceinline__ void store(__nv_bfloat16* p, float v) {
    __stcs(p, __float2bfloat16_rn(v));
  }
  __device__ static __forceinline__ void store_if(__nv_bfloat16* p, float v, bool q) {
    const unsigned short b = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p st.global.cs.b16 [%0], %1;\n}\n" ::"l"(p),
                 "h"(b), "r"((int)q)
                 : "memory");
  }
};
template <>
struct Codec<__half> {
  static constexpr int kV = 4;
  using W = uint2;
  __device__ static __forceinline__ void unpack(W w, float* v) {
    v[0] = __half2float(__ushort_as_half((unsigned short)(w.x & 0xffffu)));
    v[1] = __half2float(__ushort_as_half((unsigned short)(w.x >> 16)));
    v[2] = __half2float(__ushort_as_half((unsigned short)(w.y & 0xffffu)));
    v[3] = __half2float(__ushort_as_half((unsigned short)(w.y >> 16)));
  }
  __device__ static __forceinline__ W pack(const float* v) {
    const __half2 h0 = __floats2half2_rn(v[0], v[1]);
    const __half2 h1 = __floats2half2_rn(v[2], v[3]);
    return make_uint2((uint32_t)__half_as_ushort(h0.x) | ((uint32_t)__half_as_ushort(h0.y) << 16),
                      (uint32_t)__half_as_ushort(h1.x) | ((uint32_t)__half_as_ushort(h1.y) << 16));
  }
  __device__ static __forceinline__ float load(const __half* p) { return __half2float(__ldcs(p)); }
  __device__ static __forceinline__ float load_keep(const __half* p) {
    return __half2float(__ldg(p));
  }
  __device__ static __forceinline__ float load_coh(const __half* p) { return __half2float(__ldcg(p)); }
  __device__ static __forceinline__ void store(__half* p, float v) { __stcs(p, __float2half_rn(v)); }
  __device__ static __forceinline__ void store_if(__half* p, float v, bool q) {
    const unsigned short b = __half_as_ushort(__float2half_rn(v));
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n @p st.global.cs.b16 [%0], %1;\n}\n" ::"l"(p),
                 "h"(b), "r"((int)q)
                 : "memory");
  }
};

// Whole distribution words (four values): ldw streams (evict-first),
// ldw_keep takes the read-only path, ldw_coh reads coherently through L2;
// stw streams a word out, stw_if under a predicate.
template <class S>
struct WordIO {
  using W = typename Codec<S>::W;  // float4 (FP32) or uint2 (16-bit)
  __device__ static __forceinline__ W ldw(const S* p) { return __ldcs(reinterpret_cast<const W*>(p)); }
  __device__ static __forceinline__ W ldw_keep(const S* p) { return __ldg(reinterpret_cast<const W*>(p)); }
  __device__ static __forceinline__ W ldw_coh(const S* p) { return __ldcg(reinterpret_cast<const W*>(p)); }
  __device__ static __forceinline__ void stw(S* p, W w) { __stcs(reinterpret_cast<W*>(p), w); }
  __device__ static __forceinline__ void stw_if(S* p, W w, bool q) {
    if constexpr (sizeof(W) == 16) {
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %5, 0;\n"
          " @p st.global.cs.v4.f32 [%0], {%1, %2, %3, %4};\n}\n" ::"l"(p),
          "f"(w.x), "f"(w.y), "f"(w.z), "f"(w.w), "r"((int)q)
          : "memory");
    } else {
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %3, 0;\n @p st.global.cs.v2.b32 [%0], {%1, %2};\n}\n" ::"l"(p),
          "r"(w.x), "r"(w.y), "r"((int)q)
          : "memory");
    }
  }
};

// One word's kV values, and a store of kV values as one word under a
// predicate, for every storage type (a word of FP64 storage is one value).
template <class S, class C>
__device__ __forceinline__ void unpack_word(typename Codec<S>::W w, C* v) {
  if constexpr (Codec<S>::kV == 1)
    v[0] = w;
  else
    Codec<S>::unpack(w, v);
}
template <class S, class C>
__device__ __forceinline__ void store_word_if(S* p, const C* v, bool q) {
  if constexpr (Codec<S>::kV == 1)
    Codec<S>::store_if(p, v[0], q);
  else
    WordIO<S>::stw_if(p, Codec<S>::pack(v), q);
}

// Flat-space value of field F (alpha = 1, gamma = delta, K = V = 0).
__host__ __device__ constexpr double flat_value(int F) {
  return (F == 0 || F == 1 || F == 4 || F == 6) ? 1.0 : 0.0;
}
__host__ __device__ constexpr bool has_flux(int F) { return F >= kK && F < kV; }
// V_i: a flux (-beta^k V_i) only under a shift.
__host__ __device__ constexpr bool is_v(int F) { return F >= kV && F < kNF; }

// ---------------------------------------------------------------------------
// Geometry of one cell and its neighbours (periodic)
// ---------------------------------------------------------------------------
// n / d for n < 2^31 by a multiply-high with a precomputed round-up
// multiplier (Granlund-Montgomery); d = 1 is passed through.
struct FastDiv {
  uint32_t d, mul, shift;
  __device__ __forceinline__ uint32_t div(uint32_t n) const {
    return d == 1 ? n : (__umulhi(n, mul) >> shift);
  }
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f{d, 0, 0};
  if (d > 1) {
    uint32_t l = 0;
    while ((1ull << l) < d) ++l;  // ceil(log2 d)
    const uint32_t p = 31 + l;
    f.mul = (uint32_t)(((1ull << p) + d - 1) / d);
    f.shift = p - 32;
  }
  return f;
}

struct Grid {
  int32_t nx, ny, nz;
  int64_t cells;    // < 2^31 (32-bit cell indices)
  int64_t pstride;  // cells rounded up to whole 32-cell tiles (a buffer holds 16 Q pstride values)
  FastDiv fx, fy;   // division by nx and by ny
};

inline Grid make_grid(int32_t nx, int32_t ny, int32_t nz, int64_t cells, int64_t pstride) {
  return Grid{nx, ny, nz, cells, pstride, make_fastdiv((uint32_t)nx), make_fastdiv((uint32_t)ny)};
}

// A cell and its periodic neighbours, as 32-bit cell indices.
struct Nbr {
  uint32_t c;
  int32_t ox[3];  // offset along x for c_x = 0, +1, -1
  int32_t oy[3];
  int32_t oz[3];
  __device__ __forceinline__ uint32_t at(int cx, int cy, int cz) const {
    return (uint32_t)((int32_t)c + ox[cx == 0 ? 0 : (cx > 0 ? 1 : 2)] +
                      oy[cy == 0 ? 0 : (cy > 0 ? 1 : 2)] + oz[cz == 0 ? 0 : (cz > 0 ? 1 : 2)]);
  }
};

__device__ __forceinline__ Nbr make_nbr(const Grid& G, int64_t c64) {
  Nbr n;
  const uint32_t c = (uint32_t)c64;
  n.c = c;
  const uint32_t t = G.fx.div(c);
  const int32_t x = (int32_t)(c - t * (uint32_t)G.nx);
  const uint32_t zz = G.fy.div(t);
  const int32_t y = (int32_t)(t - zz * (uint32_t)G.ny);
  const int32_t z = (int32_t)zz;
  const int32_t plane = G.nx * G.ny;
  n.ox[0] = 0;
  n.ox[1] = (x + 1 == G.nx) ? -(G.nx - 1) : 1;
  n.ox[2] = (x == 0) ? (G.nx - 1) : -1;
  n.oy[0] = 0;
  n.oy[1] = ((y + 1 == G.ny) ? -(G.ny - 1) : 1) * G.nx;
  n.oy[2] = ((y == 0) ? (G.ny - 1) : -1) * G.nx;
  n.oz[0] = 0;
  n.oz[1] = ((z + 1 == G.nz) ? -(G.nz - 1) : 1) * plane;
  n.oz[2] = ((z == 0) ? (G.nz - 1) : -1) * plane;
  return n;
}

// Distribution layout in HBM: tile-blocked words. The 16 Q values of the 32
// consecutive cells of a tile form one contiguous block, ordered by velocity,
// then field word, then cell. A word holds kV consecutive fields of one
// (cell, velocity): kV = 4 for FP32 (a 16-byte float4) and for 16-bit storage
// (8 bytes), 1 for FP64. With W = 16 / kV words per velocity, f_{F,l}(c) sits at
//   (((c / 32) W Q + l W + F / kV) 32 + c % 32) kV + F % kV.
// A warp's 32 cells of one (word, l) are one aligned row of 32 words, the
// fields of one velocity are W consecutive rows, and a tile's whole state is
// one block. With one plane per (F, l) instead (all cells of a plane
// contiguous, one value per access), the 600-odd tiles in flight on the GPU
// touched 16 Q separate DRAM regions each and every thread issued 16 Q loads
// per pass: the FP32 collide ran at 0.65 of the copy bandwidth, against 0.72
// with tile blocks and 0.99 with tile-blocked words (256^3 D3Q19, GB300).
constexpr int kTileCells = 32;
template <int Q, class S>
__host__ __device__ __forceinline__ size_t fidx(uint32_t c, int F, int l) {
  constexpr int V = Codec<S>::kV;
  return (((size_t)(c >> 5) * (size_t)(kNF / V * Q) + (size_t)(l * (kNF / V) + F / V)) * kTileCells +
          (c & 31u)) * V + (size_t)(F % V);
}
// Where f_{F,l}(x) of the current state lives, for each streaming layout:
// cell read_cell(l), velocity slot read_slot(l), the same for every field.
template <int Q, int LAYOUT>
__device__ __forceinline__ uint32_t read_cell(const Nbr& n, int l) {
  using L = Lattice<Q>;
  return LAYOUT == kAAOdd ? n.at(-L::c(l, 0), -L::c(l, 1), -L::c(l, 2)) : n.c;
}
template <int LAYOUT>
__host__ __device__ constexpr int read_slot(int l) {
  return LAYOUT == kAAOdd ? opposite(l) : l;
}
template <int Q, int LAYOUT, class S>
__device__ __forceinline__ size_t read_index(const Nbr& n, int F, int l) {
  return fidx<Q, S>(read_cell<Q, LAYOUT>(n, l), F, read_slot<LAYOUT>(l));
}
// Where f*_{F,l}(x) goes.
template <int Q, int LAYOUT>
__device__ __forceinline__ uint32_t write_cell(const Nbr& n, int l) {
  using L = Lattice<Q>;
  return LAYOUT == kAAEven ? n.c : n.at(L::c(l, 0), L::c(l, 1), L::c(l, 2));
}
template <int LAYOUT>
__host__ __device__ constexpr int write_slot(int l) {
  return LAYOUT == kAAEven ? opposite(l) : l;
}
template <int Q, int LAYOUT, class S>
__device__ __forceinline__ size_t write_index(const Nbr& n, int F, int l) {
  return fidx<Q, S>(write_cell<Q, LAYOUT>(n, l), F, write_slot<LAYOUT>(l));
}


// ---------------------------------------------------------------------------
// Step arguments
// ---------------------------------------------------------------------------
template <class S, class C>
struct StepArgs {
  const S* fin;
  S* fout;
  const C* aux;  // 7 planes: ln(alpha~) or log1p(alpha~ - 1); gamma~ or gamma~ - delta
  // Reading R17 (LAG): aux holds the previous step's corrected lapse and
  // metric in that form, and the step writes its own corrected ones to
  // aux_out for the next step. nullptr: aux holds this step's rho~ (R5).
  C* aux_out;
  int* flag;     // set to 1 when a non-finite moment is seen
  Grid G;
  C inv2dx, inv4dx;  // 1/(2 dx), 1/(4 dx)
  C half_dt, omega, omc, sigma;  // dt/2, 1/tau, 1 - 1/tau, dt (1 - 1/(2 tau))
  int slicing;
  int sources_on;
  // Matter: pressure P(t) = P0 (t0/t)^2 of a fluid at rest, t = t0 + n dt at
  // step n, n read from *clock (device memory, advanced after every step);
  // clock == nullptr is vacuum.
  const int64_t* clock;
  double fluid_P0, fluid_t0, fluid_dt;
  // Shift, read by the forms compiled with SHIFT: the constant beta^i, and
  // with SHIFT = 2 also a static field beta_field[3][cells] (FP64) added to
  // it, whose central differences give B_k^i.
  C beta[3];
  const double* beta_field;
};

// Reading R17: the corrected lapse and metric of this step, in the stencil
// planes' form (ln alpha and gamma_ij; log1p(alpha - 1) and gamma_ij - delta_ij
// from deviation moments), for the next step's derivatives.
template <int REP, class C>
__device__ __forceinline__ void write_lagged(C* __restrict__ aux_out, int64_t cells, uint32_t c,
                                             const C rho[kNF]) {
  aux_out[c] = REP == kDEV ? log1p(rho[0]) : log(rho[0]);
#pragma unroll
  for (int q = 0; q < 6; ++q) aux_out[(size_t)(1 + q) * (size_t)cells + c] = rho[1 + q];
}

// Adds the fluid's term (P/2) gamma_ij to the sources of K_ij (alpha S_ij),
// with P at the step being taken; nothing without matter. Kept apart from
// bm_sources so that vacuum launches carry no extra live values.
template <class S, class C>
__device__ __forceinline__ void add_fluid(const StepArgs<S, C>& a, C alpha, const C g[6],
                                          C Sr[kNF]) {
  if (a.clock == nullptr) return;
  const double r = a.fluid_t0 / (a.fluid_t0 + (double)(*a.clock) * a.fluid_dt);
  const C half_p = C(0.5 * a.fluid_P0 * r * r);
#pragma unroll
  for (int q = 0; q < 6; ++q) Sr[kK + q] += alpha * half_p * g[q];
}

// Shift sources (Sec. "Bona-Masso evolution equations", constant beta):
// alpha beta^r A_r to the lapse, 2 beta^r D_rij to the metric.
template <class C>
__device__ __forceinline__ void shift_sources(const C beta[3], C alpha, const C A[3],
                                              const C D[3][6], C Sr[kNF]) {
  Sr[0] += alpha * (beta[0] * A[0] + beta[1] * A[1] + beta[2] * A[2]);
#pragma unroll
  for (int q = 0; q < 6; ++q)
    Sr[kG + q] += C(2) * (beta[0] * D[0][q] + beta[1] * D[1][q] + beta[2] * D[2][q]);
}

// Shift part of the K fluxes: -beta^k K_ij (the K equilibria's factor
// 1 - c.beta / c_s^2), K at the corrected moments.
template <class C, int dim>
__device__ __forceinline__ void shift_flux_k(const C beta[3], const C K[6], C Fl[6][3]) {
#pragma unroll
  for (int k = 0; k < dim; ++k)
#pragma unroll
    for (int q = 0; q < 6; ++q) Fl[q][k] -= beta[k] * K[q];
}

// Shift at a cell with a static field: beta^i = the constant part + the
// field's value; B_k^i = d_k beta^i / 2 by central differences (zero along
// the axes the velocity set does not span).
template <int Q, class C>
__device__ __forceinline__ void shift_field_at(const Nbr& n, int64_t cells,
                                               const double* __restrict__ bf, const C beta0[3],
                                               double inv4dx, C beta[3], C B[3][3]) {
  constexpr int dim = Lattice<Q>::kDim;
#pragma unroll
  for (int i = 0; i < 3; ++i) beta[i] = beta0[i] + C(__ldg(bf + (size_t)i * (size_t)cells + n.c));
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k < dim) {
      const uint32_t cp = n.at(k == 0, k == 1, k == 2);
      const uint32_t cm = n.at(-(k == 0), -(k == 1), -(k == 2));
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const double* pl = bf + (size_t)i * (size_t)cells;
        B[k][i] = C((__ldg(pl + cp) - __ldg(pl + cm)) * inv4dx);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i) B[k][i] = C(0);
    }
  }
}

// A_k and D_kij by central differences of the aux planes (reading: second
// order differences of ln alpha and gamma_ij / 2).
template <int Q, class C>
__device__ __forceinline__ void derivatives(const Nbr& n, int64_t cells, const C* __restrict__ aux,
                                            C inv2dx, C inv4dx, C A[3], C D[3][6]) {
  constexpr int dim = Lattice<Q>::kDim;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k < dim) {
      const uint32_t cp = n.at(k == 0, k == 1, k == 2);
      const uint32_t cm = n.at(-(k == 0), -(k == 1), -(k == 2));
      A[k] = (__ldg(aux + cp) - __ldg(aux + cm)) * inv2dx;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const C* plane = aux + (size_t)(1 + q) * (size_t)cells;
        D[k][q] = (__ldg(plane + cp) - __ldg(plane + cm)) * inv4dx;
      }
    } else {
      A[k] = C(0);
#pragma unroll
      for (int q = 0; q < 6; ++q) D[k][q] = C(0);
    }
  }
}

// Unpacks 16 moments (ABS: the values; DEV: deviations from flat space) into
// the state the physics needs.
template <int REP, class C>
__device__ __forceinline__ void unpack(const C m[kNF], C& alpha, C g[6], C K[6], C V[3]) {
  alpha = REP == kDEV ? C(1) + m[0] : m[0];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    g[q] = (REP == kDEV && (q == 0 || q == 3 || q == 5)) ? C(1) + m[kG + q] : m[kG + q];
    K[q] = m[kK + q];
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) V[k] = m[kV + k];
}

// ---------------------------------------------------------------------------
// k_collide: the fused step, one thread per cell, value by value (FP64)
// ---------------------------------------------------------------------------
// Storage with one value per distribution word: FP64 (FP32 and 16-bit
// storage take k_collide_w below). SHIFT: the shift terms are compiled in: 1
// a constant shift (a.beta), 2 a static field on top of it (a.beta_field,
// with its B terms). The zero-shift forms (0) keep none of their code or
// registers. MINB: blocks per SM the registers are sized for (without HOLD).
// LAGW: the form writes the lagged fields of reading R17 to a.aux_out
// (compiled in only where asked, so the other forms keep their registers).
template <int Q, class S, class C, int REP, int LAYOUT, bool HOLD, int SHIFT = 0, int MINB = 3,
          bool LAGW = false>
__global__ void __launch_bounds__(128, HOLD ? 1 : MINB) k_collide(const StepArgs<S, C> a) {
  using L = Lattice<Q>;
  constexpr int dim = L::kDim;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = cell < a.G.cells;
  const int64_t c = valid ? cell : a.G.cells - 1;
  const int64_t cells = a.G.cells;
  const Nbr n = make_nbr(a.G, c);

  // source and destination cell of each velocity
  uint32_t rc[Q], wc[Q];
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    rc[l] = read_cell<Q, LAYOUT>(n, l);
    wc[l] = write_cell<Q, LAYOUT>(n, l);
  }

  // Pass 1: zeroth moments (ascending l).
  C fv[HOLD ? kNF : 1][HOLD ? Q : 1];
  C rt[kNF];
#pragma unroll
  for (int F = 0; F < kNF; ++F) {
    C s = C(0);
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      // In place (AA) the buffer is written by this kernel: re-read values
      // must come through coherent loads, never the read-only path.
      const S* src = a.fin + fidx<Q, S>(rc[l], F, read_slot<LAYOUT>(l));
      const C v = HOLD ? Codec<S>::load(src)
                  : LAYOUT == kPingPong ? Codec<S>::load_keep(src) : Codec<S>::load_coh(src);
      if (HOLD) fv[HOLD ? F : 0][HOLD ? l : 0] = v;
      s += REP == kDEV ? C(L::w(l)) * v : v;
    }
    rt[F] = s;
  }
  {
    C chk = C(0);
#pragma unroll
    for (int F = 0; F < kNF; ++F) chk += rt[F];
    if (valid && !isfinite(chk)) atomicOr(a.flag, 1);
  }

  // Derivatives, sources at rho~, corrected rho, flux at rho.
  C A[3], D[3][6];
  derivatives<Q, C>(n, cells, a.aux, a.inv2dx, a.inv4dx, A, D);
  C alpha, gm[6], K[6], V[3];
  unpack<REP, C>(rt, alpha, gm, K, V);
  C Sr[kNF];
  bm_sources<C>(alpha, gm, K, V, A, D, a.slicing, Sr);
  add_fluid(a, alpha, gm, Sr);
  C sb[3], sB[3][3];  // shift and B_k^i at this cell (SHIFT = 2)
  if (SHIFT == 1) shift_sources<C>(a.beta, alpha, A, D, Sr);
  if (SHIFT == 2) {
    shift_field_at<Q, C>(n, cells, a.beta_field, a.beta, (double)a.inv4dx, sb, sB);
    shift_sources<C>(sb, alpha, A, D, Sr);
    shift_field_sources<C>(gm, K, V, D, sB, Sr);
  }
  if (!a.sources_on) {
#pragma unroll
    for (int F = 0; F < kNF; ++F) Sr[F] = C(0);
  }
  C rho[kNF];  // ABS: rho; DEV: rho - rho_flat
#pragma unroll
  for (int F = 0; F < kNF; ++F) rho[F] = rt[F] + a.half_dt * Sr[F];
  if (LAGW && valid) write_lagged<REP, C>(a.aux_out, cells, n.c, rho);
  C Fl[6][3];
  C Fv[SHIFT == 2 ? 3 : 1][3];  // V fluxes under a shift field
  {
    C alpha2, g2[6], K2[6], V2[3];
    unpack<REP, C>(rho, alpha2, g2, K2, V2);
    bm_flux<C, dim>(alpha2, g2, V2, A, D, Fl);
    if (SHIFT == 1) shift_flux_k<C, dim>(a.beta, K2, Fl);
    if (SHIFT == 2) {
      shift_flux_k<C, dim>(sb, K2, Fl);
      shift_field_vflux<C, dim>(g2, V2, sb, sB, Fv);
    }
  }
  // Per-field coefficients: coef = omega rho + sigma S; flux scaled by 3 omega.
  C coef[kNF];
#pragma unroll
  for (int F = 0; F < kNF; ++F) coef[F] = a.omega * rho[F] + a.sigma * Sr[F];
  const C three_omega = C(3) * a.omega;

  // Pass 2: relax, add the source, stream.
#pragma unroll
  for (int F = 0; F < kNF; ++F) {
    const C cf = coef[F];
    C b[3] = {C(0), C(0), C(0)};
    if (has_flux(F)) {
#pragma unroll
      for (int k = 0; k < dim; ++k) b[k] = three_omega * Fl[F - kK][k];
    }
    // under a shift the V fields take the flux -beta^k V_i
    const bool vflux = SHIFT && is_v(F);
    // All Q values of this field are read before any is written: in place
    // (AA) the field's reads and writes touch the same Q locations.
    C v_[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const S* src = a.fin + fidx<Q, S>(rc[l], F, read_slot<LAYOUT>(l));
      // the second read is the last use: streaming (evict-first) load
      v_[l] = HOLD ? fv[HOLD ? F : 0][HOLD ? l : 0]
              : LAYOUT == kPingPong ? Codec<S>::load(src) : Codec<S>::load_coh(src);
    }
    if (vflux && SHIFT == 2) {
#pragma unroll
      for (int k = 0; k < dim; ++k) b[k] = three_omega * Fv[SHIFT == 2 ? F - kV : 0][k];
    } else if (vflux) {
      // V_i at the corrected moments, recovered from this field's own values
      // rather than kept live since pass 1: coef = omega rho~ + dt S (as
      // omega dt/2 + sigma = dt), so rho = rho~ + (coef - omega rho~) / 2.
      C s = C(0);
#pragma unroll
      for (int l = 0; l < Q; ++l) s += REP == kDEV ? C(L::w(l)) * v_[l] : v_[l];
      const C mv = -three_omega * (s + C(0.5) * (cf - a.omega * s));
#pragma unroll
      for (int k = 0; k < dim; ++k) b[k] = mv * a.beta[k];
    }
    // FP64 (bound by its arithmetic): w_l (cf + c.b) as w_l cf + c.(w_l b),
    // whose products repeat across velocities of equal weight and are formed
    // once each, instead of one product per velocity
    constexpr bool kLeanRelax = sizeof(C) == 8 && REP == kABS;
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const C v = v_[l];
      C t = kLeanRelax ? C(L::w(l)) * cf : cf;
      if (has_flux(F) || vflux) {
#pragma unroll
        for (int k = 0; k < dim; ++k) {
          const C bk = kLeanRelax ? C(L::w(l)) * b[k] : b[k];
          if (L::c(l, k) > 0) t += bk;
          if (L::c(l, k) < 0) t -= bk;
        }
      }
      const C out = REP == kDEV ? fma(a.omc, v, t)
                                : (kLeanRelax ? fma(a.omc, v, t) : fma(a.omc, v, C(L::w(l)) * t));
      // Ping-pong: lanes past the last cell were clamped to it and write the
      // same bytes as its own lanes, so every store can be unconditional.
      S* dst = a.fout + fidx<Q, S>(wc[l], F, write_slot<LAYOUT>(l));
      if (LAYOUT == kPingPong)
        Codec<S>::store(dst, out);
      else
        Codec<S>::store_if(dst, out, valid);
    }
  }
}

// From one cell's zeroth moments rt and stencil derivatives A, D: the
// sources S at rt, the corrected moments rho = rt + dt/2 S (the moment rule
// of the forced scheme) and the fluxes at rho. SHIFT = 1 adds the terms of a
// constant shift a.beta, SHIFT = 2 those of the static shift field (with its
// B_k^i) and the V fluxes -beta^k V_i it gives (Fv).
template <int Q, class S, class C, int REP, int SHIFT = 0>
__device__ __forceinline__ void cell_terms(const StepArgs<S, C>& a, const Nbr& n, const C rt[kNF],
                                           const C A[3], const C D[3][6], C rho[kNF], C Sr[kNF],
                                           C Fl[6][3], C Fv[3][3]) {
  constexpr int dim = Lattice<Q>::kDim;
  C alpha, gm[6], K[6], V[3];
  unpack<REP, C>(rt, alpha, gm, K, V);
  bm_sources<C>(alpha, gm, K, V, A, D, a.slicing, Sr);
  add_fluid(a, alpha, gm, Sr);
  C sb[3], sB[3][3];  // shift and B_k^i at this cell (SHIFT = 2)
  if (SHIFT == 1) shift_sources<C>(a.beta, alpha, A, D, Sr);
  if (SHIFT == 2) {
    shift_field_at<Q, C>(n, a.G.cells, a.beta_field, a.beta, (double)a.inv4dx, sb, sB);
    shift_sources<C>(sb, alpha, A, D, Sr);
    shift_field_sources<C>(gm, K, V, D, sB, Sr);
  }
  if (!a.sources_on) {
#pragma unroll
    for (int F = 0; F < kNF; ++F) Sr[F] = C(0);
  }
#pragma unroll
  for (int F = 0; F < kNF; ++F) rho[F] = rt[F] + a.half_dt * Sr[F];
  C alpha2, g2[6], K2[6], V2[3];
  unpack<REP, C>(rho, alpha2, g2, K2, V2);
  bm_flux<C, dim>(alpha2, g2, V2, A, D, Fl);
  if (SHIFT == 1) shift_flux_k<C, dim>(a.beta, K2, Fl);
  if (SHIFT == 2) {
    shift_flux_k<C, dim>(sb, K2, Fl);
    shift_field_vflux<C, dim>(g2, V2, sb, sB, Fv);
  }
}

// ---------------------------------------------------------------------------
// k_collide_w: one thread per cell for FP32 and 16-bit storage, word by word
// ---------------------------------------------------------------------------
// The step of k_collide with every load and store moving a whole word of kV
// consecutive fields of one (cell, velocity): a kV-th of the memory
// instructions of value-by-value access. HOLD keeps the words of a
// cell in registers between the passes. SHIFT as in k_collide: 1 a constant
// shift, 2 a static shift field; under a shift the V fields take the flux
// -beta^k V_i at the corrected moments. TPB: threads per block.
template <int Q, class S, class C, int REP, int LAYOUT, bool HOLD, int MINB = 3, bool LAGW = false,
          int SHIFT = 0, int TPB = 128>
__global__ void __launch_bounds__(TPB, HOLD ? 1 : MINB) k_collide_w(const StepArgs<S, C> a) {
  using L = Lattice<Q>;
  using IO = WordIO<S>;
  using W = typename IO::W;
  constexpr int V = Codec<S>::kV;
  static_assert(V > 1 && kNF % V == 0, "word access: several fields per word");
  constexpr int NW = kNF / V;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = cell < a.G.cells;
  const int64_t c = valid ? cell : a.G.cells - 1;
  const int64_t cells = a.G.cells;
  const Nbr n = make_nbr(a.G, c);

  // Pass 1: zeroth moments, kV fields per load (ascending l).
  W hw[HOLD ? NW : 1][HOLD ? Q : 1];
  C rt[kNF];
#pragma unroll
  for (int m = 0; m < NW; ++m) {
    C sum[V];
#pragma unroll
    for (int i = 0; i < V; ++i) sum[i] = C(0);
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      // in place (AA) the buffer is written by this kernel: coherent loads
      const S* src = a.fin + read_index<Q, LAYOUT, S>(n, V * m, l);
      const W w = HOLD ? IO::ldw(src) : LAYOUT == kPingPong ? IO::ldw_keep(src) : IO::ldw_coh(src);
      if (HOLD) hw[HOLD ? m : 0][HOLD ? l : 0] = w;
      C v[V];
      Codec<S>::unpack(w, v);
#pragma unroll
      for (int i = 0; i < V; ++i) sum[i] += REP == kDEV ? C(L::w(l)) * v[i] : v[i];
    }
#pragma unroll
    for (int i = 0; i < V; ++i) rt[V * m + i] = sum[i];
  }
  // Non-finite moments are reported, and the lagged fields written, only
  // after the update pass: a global write here (the flag or aux_out may
  // alias the input as far as the compiler knows) would keep the update
  // pass's loads from being issued ahead of the physics.
  bool bad;
  {
    C chk = C(0);
#pragma unroll
    for (int F = 0; F < kNF; ++F) chk += rt[F];
    bad = valid && !isfinite(chk);
  }

  C A[3], D[3][6];
  derivatives<Q, C>(n, cells, a.aux, a.inv2dx, a.inv4dx, A, D);
  C rho[kNF], Sr[kNF], Fl[6][3], Fv[3][3];
  cell_terms<Q, S, C, REP, SHIFT>(a, n, rt, A, D, rho, Sr, Fl, Fv);
  const C three_omega = C(3) * a.omega;

  // Pass 2: relax, add the source, stream; all Q words of a field group are
  // read before any is written (in place they share the Q locations).
#pragma unroll
  for (int m = 0; m < NW; ++m) {
    W vw[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const S* src = a.fin + read_index<Q, LAYOUT, S>(n, V * m, l);
      vw[l] = HOLD ? hw[HOLD ? m : 0][HOLD ? l : 0]
              : LAYOUT == kPingPong ? IO::ldw(src) : IO::ldw_coh(src);
    }
    C cf[V], b[V][3];
#pragma unroll
    for (int i = 0; i < V; ++i) {
      const int F = V * m + i;
      cf[i] = a.omega * rho[F] + a.sigma * Sr[F];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        C bk = has_flux(F) ? three_omega * Fl[F - kK][k] : C(0);
        if (SHIFT == 1 && is_v(F)) bk = -three_omega * rho[F] * a.beta[k];
        if (SHIFT == 2 && is_v(F)) bk = three_omega * Fv[SHIFT == 2 && is_v(F) ? F - kV : 0][k];
        b[i][k] = bk;
      }
    }
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      C v[V], out[V];
      Codec<S>::unpack(vw[l], v);
#pragma unroll
      for (int i = 0; i < V; ++i) {
        C t = cf[i];
        if (has_flux(V * m + i) || (SHIFT && is_v(V * m + i))) {
#pragma unroll
          for (int k = 0; k < L::kDim; ++k) {
            if (L::c(l, k) > 0) t += b[i][k];
            if (L::c(l, k) < 0) t -= b[i][k];
          }
        }
        out[i] = REP == kDEV ? fma(a.omc, v[i], t) : fma(a.omc, v[i], C(L::w(l)) * t);
      }
      S* dst = a.fout + write_index<Q, LAYOUT, S>(n, V * m, l);
      if (LAYOUT == kPingPong)
        IO::stw(dst, Codec<S>::pack(out));
      else
        IO::stw_if(dst, Codec<S>::pack(out), valid);
    }
  }
  if (LAGW && valid) write_lagged<REP, C>(a.aux_out, cells, n.c, rho);
  if (bad) atomicOr(a.flag, 1);
}

// ---------------------------------------------------------------------------
// k_aux: ln(alpha~) and gamma~ (or their deviations) for the stencil
// ---------------------------------------------------------------------------
template <int Q, class S, class C, int REP, int LAYOUT>
__global__ void __launch_bounds__(256) k_aux(const S* __restrict__ f, C* __restrict__ aux, Grid G) {
  using L = Lattice<Q>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.cells) return;
  constexpr int V = Codec<S>::kV;
  constexpr int NW = (7 + V - 1) / V;  // the words holding fields 0..6
  const Nbr n = make_nbr(G, c);
  C s[NW * V];
#pragma unroll
  for (int F = 0; F < NW * V; ++F) s[F] = C(0);
#pragma unroll
  for (int m = 0; m < NW; ++m) {
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const S* src = f + read_index<Q, LAYOUT, S>(n, V * m, l);
      C v[V];
      if constexpr (V > 1)
        Codec<S>::unpack(WordIO<S>::ldw_keep(src), v);
      else
        v[0] = Codec<S>::load_keep(src);
#pragma unroll
      for (int i = 0; i < V; ++i)
        if (V * m + i < 7) s[V * m + i] += REP == kDEV ? C(L::w(l)) * v[i] : v[i];
    }
  }
  s[0] = REP == kDEV ? log1p(s[0]) : log(s[0]);
#pragma unroll
  for (int F = 0; F < 7; ++F) aux[(int64_t)F * G.cells + c] = s[F];
}

// ---------------------------------------------------------------------------
// Per-cell bodies for kernels that run many steps in one launch (the batched
// ensemble). Other thread blocks of the same launch write the buffers these
// read, so every load is coherent (L1 bypassed). Same arithmetic, in the
// same order, as k_aux and k_collide with one thread per cell.
// ---------------------------------------------------------------------------
template <int Q, class S, class C, int REP, int LAYOUT>
__device__ __forceinline__ void aux_cell(const S* __restrict__ f, C* __restrict__ aux,
                                         const Grid& G, int64_t c) {
  using L = Lattice<Q>;
  constexpr int V = Codec<S>::kV;
  constexpr int NW = (7 + V - 1) / V;  // the words holding fields 0..6
  const Nbr n = make_nbr(G, c);
  C s[NW * V];
#pragma unroll
  for (int F = 0; F < NW * V; ++F) s[F] = C(0);
#pragma unroll
  for (int m = 0; m < NW; ++m) {
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const S* src = f + read_index<Q, LAYOUT, S>(n, V * m, l);
      C v[V];
      if constexpr (V > 1)
        Codec<S>::unpack(WordIO<S>::ldw_coh(src), v);
      else
        v[0] = Codec<S>::load_coh(src);
#pragma unroll
      for (int i = 0; i < V; ++i) s[V * m + i] += REP == kDEV ? C(L::w(l)) * v[i] : v[i];
    }
  }
  s[0] = REP == kDEV ? log1p(s[0]) : log(s[0]);
#pragma unroll
  for (int F = 0; F < 7; ++F) aux[(int64_t)F * G.cells + c] = s[F];
}

template <int Q, class C>
__device__ __forceinline__ void derivatives_coh(const Nbr& n, int64_t cells,
                                                const C* __restrict__ aux, C inv2dx, C inv4dx,
                                                C A[3], C D[3][6]) {
  constexpr int dim = Lattice<Q>::kDim;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k < dim) {
      const uint32_t cp = n.at(k == 0, k == 1, k == 2);
      const uint32_t cm = n.at(-(k == 0), -(k == 1), -(k == 2));
      A[k] = (__ldcg(aux + cp) - __ldcg(aux + cm)) * inv2dx;
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const C* plane = aux + (size_t)(1 + q) * (size_t)cells;
        D[k][q] = (__ldcg(plane + cp) - __ldcg(plane + cm)) * inv4dx;
      }
    } else {
      A[k] = C(0);
#pragma unroll
      for (int q = 0; q < 6; ++q) D[k][q] = C(0);
    }
  }
}

template <int Q, class S, class C, int REP, int LAYOUT, bool LAGW = false>
__device__ __forceinline__ void collide_cell(const StepArgs<S, C>& a, int64_t c) {
  using L = Lattice<Q>;
  constexpr int dim = L::kDim;
  const int64_t cells = a.G.cells;
  constexpr int VW = Codec<S>::kV;  // fields per distribution word
  const Nbr n = make_nbr(a.G, c);
  C rt[kNF];
#pragma unroll
  for (int F = 0; F < kNF; ++F) rt[F] = C(0);
#pragma unroll
  for (int m = 0; m < kNF / VW; ++m) {
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      const S* src = a.fin + read_index<Q, LAYOUT, S>(n, VW * m, l);
      C v[VW];
      if constexpr (VW > 1)
        Codec<S>::unpack(WordIO<S>::ldw_coh(src), v);
      else
        v[0] = Codec<S>::load_coh(src);
#pragma unroll
      for (int i = 0; i < VW; ++i) rt[VW * m + i] += REP == kDEV ? C(L::w(l)) * v[i] : v[i];
    }
  }
  // reported at the end: a global write here would hold back the second
  // pass's loads (see k_collide_w)
  bool bad;
  {
    C chk = C(0);
#pragma unroll
    for (int F = 0; F < kNF; ++F) chk += rt[F];
    bad = !isfinite(chk);
  }
  C A[3], D[3][6];
  derivatives_coh<Q, C>(n, cells, a.aux, a.inv2dx, a.inv4dx, A, D);
  C alpha, gm[6], K[6], V[3];
  unpack<REP, C>(rt, alpha, gm, K, V);
  C Sr[kNF];
  bm_sources<C>(alpha, gm, K, V, A, D, a.slicing, Sr);
  add_fluid(a, alpha, gm, Sr);
  if (!a.sources_on) {
#pragma unroll
    for (int F = 0; F < kNF; ++F) Sr[F] = C(0);
  }
  C rho[kNF];
#pragma unroll
  for (int F = 0; F < kNF; ++F) rho[F] = rt[F] + a.half_dt * Sr[F];
  C Fl[6][3];
  {
    C alpha2, g2[6], K2[6], V2[3];
    unpack<REP, C>(rho, alpha2, g2, K2, V2);
    bm_flux<C, dim>(alpha2, g2, V2, A, D, Fl);
  }
  const C three_omega = C(3) * a.omega;
  // FP64: the same weight-first form as k_collide, so a batched run stays
  // bitwise equal to the run on its own context
  constexpr bool kLeanRelax = sizeof(C) == 8 && REP == kABS;
  if constexpr (VW == 1) {
    // value by value, in k_collide's own expression form (the compiler
    // contracts products into fused multiply-adds the same way in both)
#pragma unroll
    for (int F = 0; F < kNF; ++F) {
      const C cf = a.omega * rho[F] + a.sigma * Sr[F];
      C b[3] = {C(0), C(0), C(0)};
      if (has_flux(F)) {
#pragma unroll
        for (int k = 0; k < dim; ++k) b[k] = three_omega * Fl[F - kK][k];
      }
      C v_[Q];
#pragma unroll
      for (int l = 0; l < Q; ++l) v_[l] = Codec<S>::load_coh(a.fin + read_index<Q, LAYOUT, S>(n, F, l));
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        C t = kLeanRelax ? C(L::w(l)) * cf : cf;
        if (has_flux(F)) {
#pragma unroll
          for (int k = 0; k < dim; ++k) {
            const C bk = kLeanRelax ? C(L::w(l)) * b[k] : b[k];
            if (L::c(l, k) > 0) t += bk;
            if (L::c(l, k) < 0) t -= bk;
          }
        }
        const C out = REP == kDEV ? fma(a.omc, v_[l], t)
                                  : (kLeanRelax ? fma(a.omc, v_[l], t)
                                                : fma(a.omc, v_[l], C(L::w(l)) * t));
        Codec<S>::store(a.fout + write_index<Q, LAYOUT, S>(n, F, l), out);
      }
    }
  } else {
#pragma unroll
    for (int m = 0; m < kNF / VW; ++m) {
      C cf[VW], b[VW][3];
#pragma unroll
      for (int i = 0; i < VW; ++i) {
        const int F = VW * m + i;
        cf[i] = a.omega * rho[F] + a.sigma * Sr[F];
#pragma unroll
        for (int k = 0; k < 3; ++k) b[i][k] = has_flux(F) ? three_omega * Fl[F - kK][k] : C(0);
      }
      typename Codec<S>::W vw[Q];
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        const S* src = a.fin + read_index<Q, LAYOUT, S>(n, VW * m, l);
        vw[l] = WordIO<S>::ldw_coh(src);
      }
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        C v[VW], out[VW];
        Codec<S>::unpack(vw[l], v);
#pragma unroll
        for (int i = 0; i < VW; ++i) {
          C t = cf[i];
          if (has_flux(VW * m + i)) {
#pragma unroll
            for (int k = 0; k < dim; ++k) {
              if (L::c(l, k) > 0) t += b[i][k];
              if (L::c(l, k) < 0) t -= b[i][k];
            }
          }
          out[i] = REP == kDEV ? fma(a.omc, v[i], t) : fma(a.omc, v[i], C(L::w(l)) * t);
        }
        S* dst = a.fout + write_index<Q, LAYOUT, S>(n, VW * m, l);
        WordIO<S>::stw(dst, Codec<S>::pack(out));
      }
    }
  }
  if (LAGW) write_lagged<REP, C>(a.aux_out, cells, n.c, rho);
  if (bad) atomicOr(a.flag, 1);
}

// ---------------------------------------------------------------------------
// FP64 kernels outside the hot loop: init, moments, constraints, transfers
// ---------------------------------------------------------------------------
template <class S>
struct Init64Args {
  const double* fields;  // [16][cells]
  S* f;                  // standard layout
  int* flag;
  Grid G;
  double inv2dx, inv4dx, half_dt;
  int slicing, sources_on;
  double fluidP;  // fluid pressure at the initial time (0: vacuum)
  double beta[3];  // constant shift
  int shift_on;
  const double* beta_field;  // static shift field [3][cells] or nullptr
};

// Shifted equilibrium: f = f_eq(rho0) - (dt/2) w_l S(rho0), A and D from rho0.
template <int Q, class S, int REP>
__global__ void __launch_bounds__(128) k_init(const Init64Args<S> a) {
  using L = Lattice<Q>;
  constexpr int dim = L::kDim;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.G.cells) return;
  const int64_t cells = a.G.cells;
  const Nbr n = make_nbr(a.G, c);
  double r[kNF];
#pragma unroll
  for (int F = 0; F < kNF; ++F) r[F] = a.fields[(int64_t)F * cells + c];
  double A[3], D[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k < dim) {
      const int64_t cp = n.at(k == 0, k == 1, k == 2);
      const int64_t cm = n.at(-(k == 0), -(k == 1), -(k == 2));
      A[k] = (log(a.fields[cp]) - log(a.fields[cm])) * a.inv2dx;
#pragma unroll
      for (int q = 0; q < 6; ++q)
        D[k][q] = (a.fields[(int64_t)(1 + q) * cells + cp] - a.fields[(int64_t)(1 + q) * cells + cm]) *
                  a.inv4dx;
    } else {
      A[k] = 0;
#pragma unroll
      for (int q = 0; q < 6; ++q) D[k][q] = 0;
    }
  }
  double alpha, gm[6], K[6], V[3];
  unpack<kABS, double>(r, alpha, gm, K, V);
  double Sr[kNF];
  bm_sources<double>(alpha, gm, K, V, A, D, a.slicing, Sr, a.fluidP);
  double sb[3] = {a.beta[0], a.beta[1], a.beta[2]}, sB[3][3];
  if (a.beta_field) {
    shift_field_at<Q, double>(n, cells, a.beta_field, a.beta, a.inv4dx, sb, sB);
    shift_field_sources<double>(gm, K, V, D, sB, Sr);
  }
  if (a.shift_on) shift_sources<double>(sb, alpha, A, D, Sr);
  if (!a.sources_on)
    for (int F = 0; F < kNF; ++F) Sr[F] = 0;
  double Fl[6][3], Fv[3][3];
  bm_flux<double, dim>(alpha, gm, V, A, D, Fl);
  if (a.shift_on) shift_flux_k<double, dim>(sb, K, Fl);
  if (a.beta_field) shift_field_vflux<double, dim>(gm, V, sb, sB, Fv);
  bool bad = false;
#pragma unroll
  for (int F = 0; F < kNF; ++F) {
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      double cf = 0;
      if (has_flux(F)) {
#pragma unroll
        for (int k = 0; k < dim; ++k) cf += L::c(l, k) * Fl[F - kK][k];
      }
      if (is_v(F) && a.beta_field) {
#pragma unroll
        for (int k = 0; k < dim; ++k) cf += L::c(l, k) * Fv[F - kV][k];
      } else if (is_v(F) && a.shift_on) {
#pragma unroll
        for (int k = 0; k < dim; ++k) cf += L::c(l, k) * (-sb[k] * r[F]);
      }
      // f = w (rho + 3 c.F) - (dt/2) w S
      double v;
      if (REP == kDEV)
        v = (r[F] - flat_value(F)) + 3.0 * cf - a.half_dt * Sr[F];
      else
        v = L::w(l) * (r[F] + 3.0 * cf) - a.half_dt * L::w(l) * Sr[F];
      bad |= !isfinite(v);
      Codec<S>::store(a.f + fidx<Q, S>((uint32_t)c, F, l), (decltype(Codec<S>::load(a.f)))v);
    }
  }
  if (bad) atomicOr(a.flag, 1);
}

// Reading R17: the stencil planes of the first step (lbnr_init) or of a
// restored state (lbnr_set_lagged) from FP64 fields [>= 7][cells]: ln alpha
// and gamma_ij, or log1p(alpha - 1) and gamma_ij - delta_ij in DEV form.
template <class C, int REP>
__global__ void __launch_bounds__(256) k_lag_from64(const double* __restrict__ fields,
                                                    C* __restrict__ aux, int64_t cells) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const double al = fields[c];
  aux[c] = REP == kDEV ? C(log1p(al - 1.0)) : C(log(al));
#pragma unroll
  for (int q = 0; q < 6; ++q)
    aux[(1 + q) * cells + c] = C(fields[(1 + q) * cells + c] - (REP == kDEV ? flat_value(1 + q) : 0.0));
}

// Reading R17: the lagged stencil planes as FP64 ln alpha and gamma_ij
// (aux64, what the FP64 moment and constraint kernels differentiate) and,
// when out is given, as the fields alpha and gamma_ij [7][cells].
template <class C, int REP>
__global__ void __launch_bounds__(256) k_lag_to64(const C* __restrict__ aux,
                                                  double* __restrict__ aux64, double* out,
                                                  int64_t cells) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cells) return;
  const double la = (double)aux[c];
  aux64[c] = la;
  if (out) out[c] = exp(la);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const double g = (double)aux[(1 + q) * cells + c] + (REP == kDEV ? flat_value(1 + q) : 0.0);
    aux64[(1 + q) * cells + c] = g;
    if (out) out[(1 + q) * cells + c] = g;
  }
}

// Sums of all 16 fields in FP64 (rho~ -> macro), ln alpha~ / gamma~ (-> aux64),
// and per-block partial sums of rho~ (-> partials[block][6 + F]).
template <int Q, class S, int REP, int LAYOUT>
__global__ void __launch_bounds__(256) k_sum64(const S* __restrict__ f, double* __restrict__ macro,
                                               double* __restrict__ aux64, double* partials,
                                               Grid G) {
  using L = Lattice<Q>;
  __shared__ double red[8][kNF];
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = c < G.cells;
  const Nbr n = make_nbr(G, valid ? c : 0);
  double m[kNF];
#pragma unroll
  for (int F = 0; F < kNF; ++F) {
    double s = 0;
    if (valid) {
      if constexpr (sizeof(S) == 4 && REP == kABS) {
        // FP32 values summed in FP32 with the rounding error of every
        // addition carried along (Knuth's TwoSum): hi + lo holds the sum to
        // about twice FP32's precision, as the FP64 sum would, without
        // putting 2 Q FP64 operations per field on the FP64 pipe.
        float hi = 0.f, lo = 0.f;
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          const float v = Codec<S>::load_keep(f + read_index<Q, LAYOUT, S>(n, F, l));
          const float t = __fadd_rn(hi, v);
          const float bp = __fsub_rn(t, hi);
          const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(v, bp));
          hi = t;
          lo = __fadd_rn(lo, e);
        }
        s = (double)hi + (double)lo;
      } else {
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          const double v =
              (double)Codec<S>::load_keep(f + read_index<Q, LAYOUT, S>(n, F, l));
          s += REP == kDEV ? L::w(l) * v : v;
        }
      }
      if (REP == kDEV) s += flat_value(F);
      macro[(int64_t)F * G.cells + c] = s;
      if (F < 7) aux64[(int64_t)F * G.cells + c] = F == 0 ? log(s) : s;
    }
    m[F] = s;
  }
  // block reduction in a fixed order
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int F = 0; F < kNF; ++F) {
    double v = m[F];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][F] = v;
  }
  __syncthreads();
  if (threadIdx.x < kNF) {
    double v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w][threadIdx.x];
    partials[(int64_t)blockIdx.x * 22 + 6 + threadIdx.x] = v;
  }
}

// rho = rho~ + dt S(rho~)/2 in place (FP64), derivatives from aux64.
template <int Q>
__global__ void __launch_bounds__(128) k_correct64(double* __restrict__ macro,
                                                   const double* __restrict__ aux64, Grid G,
                                                   double inv2dx, double inv4dx, double half_dt,
                                                   int slicing, int sources_on, double fluidP,
                                                   double bx, double by, double bz,
                                                   const double* __restrict__ beta_field) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.cells || !sources_on) return;
  const Nbr n = make_nbr(G, c);
  double r[kNF];
#pragma unroll
  for (int F = 0; F < kNF; ++F) r[F] = macro[(int64_t)F * G.cells + c];
  double A[3], D[3][6];
  derivatives<Q, double>(n, G.cells, aux64, inv2dx, inv4dx, A, D);
  double alpha, gm[6], K[6], V[3];
  unpack<kABS, double>(r, alpha, gm, K, V);
  double S[kNF];
  bm_sources<double>(alpha, gm, K, V, A, D, slicing, S, fluidP);
  double sb[3] = {bx, by, bz};
  if (beta_field) {
    const double b0[3] = {bx, by, bz};
    double sB[3][3];
    shift_field_at<Q, double>(n, G.cells, beta_field, b0, inv4dx, sb, sB);
    shift_field_sources<double>(gm, K, V, D, sB, S);
  }
  if (beta_field || bx != 0.0 || by != 0.0 || bz != 0.0) shift_sources<double>(sb, alpha, A, D, S);
#pragma unroll
  for (int F = 0; F < kNF; ++F) macro[(int64_t)F * G.cells + c] = r[F] + half_dt * S[F];
}

// Christoffel symbols Gamma^k_ij (and the inverse metric, D) at a cell from
// central differences of the corrected metric.
template <int Q>
__device__ __forceinline__ void christoffel64(const double* __restrict__ macro, const Grid& G,
                                              int64_t c, double inv4dx, double Gam[3][6],
                                              double gi[6], double D[3][6]) {
  constexpr int dim = Lattice<Q>::kDim;
  const Nbr n = make_nbr(G, c);
  double g[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) g[q] = macro[(int64_t)(1 + q) * G.cells + c];
  invert_sym3(g, gi);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (k < dim) {
      const int64_t cp = n.at(k == 0, k == 1, k == 2);
      const int64_t cm = n.at(-(k == 0), -(k == 1), -(k == 2));
#pragma unroll
      for (int q = 0; q < 6; ++q)
        D[k][q] = (macro[(int64_t)(1 + q) * G.cells + cp] - macro[(int64_t)(1 + q) * G.cells + cm]) *
                  inv4dx;
    } else {
#pragma unroll
      for (int q = 0; q < 6; ++q) D[k][q] = 0;
    }
  }
  // Gamma_mij = D_ijm + D_jim - D_mij ; Gamma^k_ij = g^{km} Gamma_mij
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      double low[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) low[m] = D[i][sym(j, m)] + D[j][sym(i, m)] - D[m][sym(i, j)];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        Gam[k][sym(i, j)] = gi[sym(k, 0)] * low[0] + gi[sym(k, 1)] * low[1] + gi[sym(k, 2)] * low[2];
    }
}

__device__ __forceinline__ double trK64(const double* __restrict__ macro, int64_t cells, int64_t c) {
  double g[6], gi[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) g[q] = macro[(int64_t)(1 + q) * cells + c];
  invert_sym3(g, gi);
  double t = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q)
    t += (q == 1 || q == 2 || q == 4 ? 2.0 : 1.0) * gi[q] * macro[(int64_t)(kK + q) * cells + c];
  return t;
}

// Hamiltonian, momentum and V constraints per cell (FP64), reduced per block
// into partials[block][0..5] = sum H^2, max|H|, sum |M|^2, max|M_i|,
// sum |C|^2, max|C_k|.
template <int Q>
__global__ void __launch_bounds__(128) k_constraints64(const double* __restrict__ macro, Grid G,
                                                       double inv2dx, double inv4dx,
                                                       double* partials) {
  constexpr int dim = Lattice<Q>::kDim;
  __shared__ double red[4][6];
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = cell < G.cells;
  const int64_t c = valid ? cell : 0;
  const Nbr n = make_nbr(G, c);
  double Gam[3][6], gi[6], D[3][6];
  christoffel64<Q>(macro, G, c, inv4dx, Gam, gi, D);
  // d_m Gamma^k_ij
  double dGam[3][3][6];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    if (m < dim) {
      double Gp[3][6], Gm[3][6], t1[6], t2[3][6];
      christoffel64<Q>(macro, G, n.at(m == 0, m == 1, m == 2), inv4dx, Gp, t1, t2);
      christoffel64<Q>(macro, G, n.at(-(m == 0), -(m == 1), -(m == 2)), inv4dx, Gm, t1, t2);
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int q = 0; q < 6; ++q) dGam[m][k][q] = (Gp[k][q] - Gm[k][q]) * inv2dx;
    } else {
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int q = 0; q < 6; ++q) dGam[m][k][q] = 0;
    }
  }
  // R = g^{ij} R_ij, R_ij = d_k G^k_ij - d_j G^k_ik + G^k_km G^m_ij - G^k_jm G^m_ik
  double R = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double t = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        t += dGam[k][k][sym(i, j)] - dGam[j][k][sym(i, k)];
#pragma unroll
        for (int m = 0; m < 3; ++m)
          t += Gam[k][sym(k, m)] * Gam[m][sym(i, j)] - Gam[k][sym(j, m)] * Gam[m][sym(i, k)];
      }
      R += gi[sym(i, j)] * t;
    }
  double K[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) K[q] = macro[(int64_t)(kK + q) * G.cells + c];
  double Km[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Km[i][j] = gi[sym(i, 0)] * K[sym(0, j)] + gi[sym(i, 1)] * K[sym(1, j)] + gi[sym(i, 2)] * K[sym(2, j)];
  double trK = Km[0][0] + Km[1][1] + Km[2][2], trK2 = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) trK2 += Km[i][j] * Km[j][i];
  const double H = R - trK2 + trK * trK;
  // momentum constraint
  double dK[3][6], dtr[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) {
    if (m < dim) {
      const int64_t cp = n.at(m == 0, m == 1, m == 2), cm = n.at(-(m == 0), -(m == 1), -(m == 2));
#pragma unroll
      for (int q = 0; q < 6; ++q)
        dK[m][q] = (macro[(int64_t)(kK + q) * G.cells + cp] - macro[(int64_t)(kK + q) * G.cells + cm]) *
                   inv2dx;
      dtr[m] = (trK64(macro, G.cells, cp) - trK64(macro, G.cells, cm)) * inv2dx;
    } else {
#pragma unroll
      for (int q = 0; q < 6; ++q) dK[m][q] = 0;
      dtr[m] = 0;
    }
  }
  double M2 = 0, Mi = 0, C2 = 0, Ci = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double t = 0;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double cov = dK[j][sym(k, i)];
#pragma unroll
        for (int m = 0; m < 3; ++m) cov -= Gam[m][sym(j, k)] * K[sym(m, i)] + Gam[m][sym(j, i)] * K[sym(k, m)];
        t += gi[sym(j, k)] * cov;
      }
    t -= dtr[i];
    M2 += t * t;
    Mi = fmax(Mi, fabs(t));
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double t1 = 0, t2 = 0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        t1 += gi[sym(r, m)] * D[k][sym(r, m)];
        t2 += gi[sym(r, m)] * D[m][sym(r, k)];
      }
    const double cv = macro[(int64_t)(kV + k) * G.cells + c] - (t1 - t2);
    C2 += cv * cv;
    Ci = fmax(Ci, fabs(cv));
  }
  double v[6] = {H * H, fabs(H), M2, Mi, C2, Ci};
  if (!valid) {
#pragma unroll
    for (int i = 0; i < 6; ++i) v[i] = 0;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    double x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = (i & 1) ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[warp][i] = x;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int i = threadIdx.x;
    double x = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x = (i & 1) ? fmax(x, red[w][i]) : x + red[w][i];
    partials[(int64_t)blockIdx.x * 22 + i] = x;
  }
}

// Plane transfer between the FP64 standard layout and the stored state.
template <int Q, class S, int REP, int LAYOUT>
__global__ void k_get_plane(const S* __restrict__ f, double* __restrict__ out, Grid G, int F, int l) {
  using L = Lattice<Q>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.cells) return;
  const Nbr n = make_nbr(G, c);
  const double v = (double)Codec<S>::load_keep(f + read_index<Q, LAYOUT, S>(n, F, l));
  double w = 0;
#pragma unroll
  for (int ll = 0; ll < Q; ++ll)
    if (ll == l) w = L::w(ll);
  out[c] = REP == kDEV ? w * (v + flat_value(F)) : v;
}

template <int Q, class S, int REP, int LAYOUT>
__global__ void k_set_plane(S* __restrict__ f, const double* __restrict__ in, Grid G, int F, int l) {
  using L = Lattice<Q>;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.cells) return;
  const Nbr n = make_nbr(G, c);
  double w = 0;
#pragma unroll
  for (int ll = 0; ll < Q; ++ll)
    if (ll == l) w = L::w(ll);
  const double v = REP == kDEV ? in[c] / w - flat_value(F) : in[c];
  Codec<S>::store(f + read_index<Q, LAYOUT, S>(n, F, l), (decltype(Codec<S>::load(f)))v);
}

// Distributions of selected cells: out[i][F][l] = f_{F,l}(idx[i]) in FP64.
template <int Q, class S, int REP, int LAYOUT>
__global__ void k_get_cells(const S* __restrict__ f, const int64_t* __restrict__ idx, int64_t n,
                            double* __restrict__ out, Grid G) {
  using L = Lattice<Q>;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * kNF) return;
  const int64_t i = t / kNF;
  const int F = (int)(t % kNF);
  const Nbr nb = make_nbr(G, idx[i]);
#pragma unroll
  for (int l = 0; l < Q; ++l) {
    const double v = (double)Codec<S>::load_keep(f + read_index<Q, LAYOUT, S>(nb, F, l));
    out[(i * kNF + F) * Q + l] = REP == kDEV ? L::w(l) * (v + flat_value(F)) : v;
  }
}

}  // namespace lbnr
