// Kernels and launchers of the 37-field scheme: the 16 Bona-Masso fields plus independently evolved
// A_k and D_kij, the original formulation that the paper mentions and sets
// aside (Sec. "Bona-Masso evolution equations", the remark after the
// first-order derivatives). With zero shift their equations follow from the
// definitions and the lapse and metric equations:
//   d_t A_k + d_k(alpha Q) = 0,   d_t D_kij + d_k(alpha K_ij) = 0,
// flux-only lattice Boltzmann sets with equilibria w [A_k + c_k alpha Q / c_s^2]
// and w [D_kij + c_k alpha K_ij / c_s^2]. The other 16 fields read A and D
// from these moments, so a cell's update needs no neighbour's moments: one
// kernel per step, no stencil pass. Ping-pong streaming; FP64 or FP32
// storage. C-ABI: lbnr_ad_* in include/lbnr.h.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "../../include/lbnr.h"

#include "collide_tma.cuh"
#include "dispatch.h"
#include "kernels.cuh"

namespace lbnr {
namespace ad {

constexpr int kNFA = 37;  // 16 fields, A_k (3), D_kij (3 x 6)
constexpr int kA = 16, kD = 19;

// alpha Q of the slicing (Sec. "Gauge choices": Q = 0, tr K, tr K / alpha).
template <class T>
__device__ __forceinline__ T alpha_q(int slicing, T alpha, const T g[6], const T K[6]) {
  if (slicing == 0) return T(0);
  T gi[6];
  invert_sym3(g, gi);
  const T trK = gi[0] * K[0] + gi[3] * K[3] + gi[5] * K[5] +
                T(2) * (gi[1] * K[1] + gi[2] * K[2] + gi[4] * K[4]);
  return slicing == 1 ? alpha * trK : trK;
}

template <class S, class C>
struct Args {
  const S* fin;
  S* fout;
  int* flag;
  Grid G;
  C half_dt, omega, omc, sigma;
  int slicing;
};

// Distribution layout: the tile-blocked words of the 16-field scheme, with
// the 37 fields padded to whole words. A word holds kV consecutive fields of
// one cell and velocity (four for FP32: 10 words per velocity, slots 37-39
// held at zero; one for FP64: 37 words). The values of the 32 cells of a tile
// form one contiguous block, ordered by velocity, then word, then cell.
template <class S>
constexpr int kWords = (kNFA + Codec<S>::kV - 1) / Codec<S>::kV;
template <class S>
constexpr int kSlots = kWords<S> * Codec<S>::kV;

template <int Q, class S>
__host__ __device__ __forceinline__ size_t ad_fidx(uint32_t c, int F, int l) {
  constexpr int V = Codec<S>::kV;
  constexpr int NW = kWords<S>;
  return (((size_t)(c >> 5) * (size_t)(NW * Q) + (size_t)(l * NW + F / V)) * lbnr::kTileCells +
          (c & 31u)) * V + (size_t)(F % V);
}

// Whole words: read-only path, streaming (last use) load, streaming store.
template <class S>
__device__ __forceinline__ typename Codec<S>::W ld_word_keep(const S* p) {
  if constexpr (Codec<S>::kV == 1)
    return Codec<S>::load_keep(p);
  else
    return WordIO<S>::ldw_keep(p);
}
template <class S>
__device__ __forceinline__ typename Codec<S>::W ld_word_last(const S* p) {
  if constexpr (Codec<S>::kV == 1)
    return Codec<S>::load(p);
  else
    return WordIO<S>::ldw(p);
}
template <class S, class C>
__device__ __forceinline__ void store_word(S* p, const C* v) {
  if constexpr (Codec<S>::kV == 1)
    Codec<S>::store(p, v[0]);
  else
    WordIO<S>::stw(p, Codec<S>::pack(v));
}

// Relaxation coefficient and flux of field F (compile-time F after
// unrolling): coef = omega rho + sigma S for the 16 fields, omega rho~ for A
// and D (no source); b[k] = 3 omega times the flux along k.
template <int dim, class C>
__device__ __forceinline__ void ad_field_terms(int F, const C rt[kNFA], const C rho[kNF],
                                               const C Sr[kNF], const C Fl[6][3], C aQ,
                                               const C aK[6], C omega, C sigma, C& cf, C b[3]) {
  const C three_omega = C(3) * omega;
  b[0] = b[1] = b[2] = C(0);
  if (F < kNF) {
    cf = omega * rho[F] + sigma * Sr[F];
    if (has_flux(F)) {
#pragma unroll
      for (int k = 0; k < dim; ++k) b[k] = three_omega * Fl[F - kK][k];
    }
  } else {
    cf = omega * rt[F];
    const int k = F < kD ? F - kA : (F - kD) / 6;
    const C fk = F < kD ? aQ : aK[(F - kD) % 6];
#pragma unroll
    for (int kk = 0; kk < dim; ++kk)
      if (kk == k) b[kk] = three_omega * fk;
  }
}
// The same for a word's slot F: zero for the padding slots (F >= 37).
template <int dim, class S, class C>
__device__ __forceinline__ void ad_word_terms(int F, const C rt[kNFA], const C rho[kNF],
                                              const C Sr[kNF], const C Fl[6][3], C aQ,
                                              const C aK[6], const Args<S, C>& a, C& cf, C b[3]) {
  if (F < kNFA) {
    ad_field_terms<dim, C>(F, rt, rho, Sr, Fl, aQ, aK, a.omega, a.sigma, cf, b);
  } else {
    cf = C(0);
    b[0] = b[1] = b[2] = C(0);
  }
}

// One step: moments, sources (A and D from the cell's own moments), the
// corrected moments, fluxes at them, relax, stream to x + c_l, one word
// (kV fields) per load and store. MINB: thread blocks of 128 per SM the
// registers are sized for (the launch forms trade occupancy against spills).
template <int Q, class S, class C, int MINB>
__global__ void __launch_bounds__(128, MINB) k_ad_collide(const Args<S, C> a) {
  using L = Lattice<Q>;
  using W = typename Codec<S>::W;
  constexpr int dim = L::kDim;
  constexpr int V = Codec<S>::kV;
  constexpr int NW = kWords<S>;
  const int64_t cell = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = cell < a.G.cells;
  const int64_t c = valid ? cell : a.G.cells - 1;
  const Nbr n = make_nbr(a.G, c);

  C rt[kNFA];
#pragma unroll
  for (int F = 0; F < kNFA; ++F) rt[F] = C(0);
#pragma unroll
  for (int m = 0; m < NW; ++m) {
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      C v[V];
      unpack_word<S>(ld_word_keep<S>(a.fin + ad_fidx<Q, S>(n.c, V * m, l)), v);
#pragma unroll
      for (int i = 0; i < V; ++i)
        if (V * m + i < kNFA) rt[V * m + i] += v[i];
    }
  }
  // reported after the update pass, so that no global write stands between
  // the two passes' loads
  bool bad;
  {
    C chk = C(0);
#pragma unroll
    for (int F = 0; F < kNFA; ++F) chk += rt[F];
    bad = valid && !isfinite(chk);
  }
  C A[3], D[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    A[k] = rt[kA + k];
#pragma unroll
    for (int q = 0; q < 6; ++q) D[k][q] = rt[kD + 6 * k + q];
  }
  C alpha, gm[6], K[6], Vv[3];
  unpack<kABS, C>(rt, alpha, gm, K, Vv);
  C Sr[kNF];
  bm_sources<C>(alpha, gm, K, Vv, A, D, a.slicing, Sr);
  C rho[kNF];
#pragma unroll
  for (int F = 0; F < kNF; ++F) rho[F] = rt[F] + a.half_dt * Sr[F];
  C Fl[6][3], aQ, aK[6];
  {
    C alpha2, g2[6], K2[6], V2[3];
    unpack<kABS, C>(rho, alpha2, g2, K2, V2);
    bm_flux<C, dim>(alpha2, g2, V2, A, D, Fl);
    aQ = alpha_q<C>(a.slicing, alpha2, g2, K2);
#pragma unroll
    for (int q = 0; q < 6; ++q) aK[q] = alpha2 * K2[q];
  }

#pragma unroll
  for (int m = 0; m < NW; ++m) {
    W vw[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) vw[l] = ld_word_last<S>(a.fin + ad_fidx<Q, S>(n.c, V * m, l));
    C cf[V], b[V][3];
#pragma unroll
    for (int i = 0; i < V; ++i) ad_word_terms<dim>(V * m + i, rt, rho, Sr, Fl, aQ, aK, a, cf[i], b[i]);
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      C v[V], out[V];
      unpack_word<S>(vw[l], v);
#pragma unroll
      for (int i = 0; i < V; ++i) {
        C t = cf[i];
#pragma unroll
        for (int k = 0; k < dim; ++k) {
          if (L::c(l, k) > 0) t += b[i][k];
          if (L::c(l, k) < 0) t -= b[i][k];
        }
        // padding slots stay zero
        out[i] = V * m + i < kNFA ? fma(a.omc, v[i], C(L::w(l)) * t) : C(0);
      }
      store_word<S>(a.fout + ad_fidx<Q, S>(n.at(L::c(l, 0), L::c(l, 1), L::c(l, 2)), V * m, l), out);
    }
  }
  if (bad) atomicOr(a.flag, 1);
}

// Initial distributions f = f_eq(v) - (dt/2) w S(v) from nf = 16 fields
// (A, D as central differences of ln alpha and gamma / 2) or nf = 37.
template <int Q, class S>
__global__ void __launch_bounds__(128) k_ad_init(const double* __restrict__ fields, int nf, S* f,
                                                  int* flag, Grid G, double inv2dx, double inv4dx,
                                                  double half_dt, int slicing) {
  using L = Lattice<Q>;
  constexpr int dim = L::kDim;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.cells) return;
  const int64_t cells = G.cells;
  const Nbr n = make_nbr(G, c);
  double v[kNFA];
#pragma unroll
  for (int F = 0; F < kNF; ++F) v[F] = fields[(int64_t)F * cells + c];
  if (nf == kNFA) {
#pragma unroll
    for (int F = kNF; F < kNFA; ++F) v[F] = fields[(int64_t)F * cells + c];
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k < dim) {
        const int64_t cp = n.at(k == 0, k == 1, k == 2);
        const int64_t cm = n.at(-(k == 0), -(k == 1), -(k == 2));
        v[kA + k] = (log(fields[cp]) - log(fields[cm])) * inv2dx;
#pragma unroll
        for (int q = 0; q < 6; ++q)
          v[kD + 6 * k + q] =
              (fields[(int64_t)(1 + q) * cells + cp] - fields[(int64_t)(1 + q) * cells + cm]) * inv4dx;
      } else {
        v[kA + k] = 0;
#pragma unroll
        for (int q = 0; q < 6; ++q) v[kD + 6 * k + q] = 0;
      }
    }
  }
  double A[3], D[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    A[k] = v[kA + k];
#pragma unroll
    for (int q = 0; q < 6; ++q) D[k][q] = v[kD + 6 * k + q];
  }
  double alpha, gm[6], K[6], V[3];
  unpack<kABS, double>(v, alpha, gm, K, V);
  double Sr[kNF], Fl[6][3];
  bm_sources<double>(alpha, gm, K, V, A, D, slicing, Sr);
  bm_flux<double, dim>(alpha, gm, V, A, D, Fl);
  const double aQ = alpha_q<double>(slicing, alpha, gm, K);
  bool bad = false;
#pragma unroll
  for (int F = 0; F < kNFA; ++F) {
#pragma unroll
    for (int l = 0; l < Q; ++l) {
      double cf = 0;
      if (has_flux(F)) {
#pragma unroll
        for (int k = 0; k < dim; ++k) cf += L::c(l, k) * Fl[F - kK][k];
      } else if (F >= kA) {
        const int k = F < kD ? F - kA : (F - kD) / 6;
        const double fk = F < kD ? aQ : alpha * K[(F - kD) % 6];
#pragma unroll
        for (int kk = 0; kk < dim; ++kk)
          if (kk == k) cf += L::c(l, kk) * fk;
      }
      const double s = F < kNF ? Sr[F] : 0.0;
      const double val = L::w(l) * (v[F] + 3.0 * cf) - half_dt * L::w(l) * s;
      bad |= !isfinite(val);
      Codec<S>::store(f + ad_fidx<Q, S>((uint32_t)c, F, l), (decltype(Codec<S>::load(f)))val);
    }
  }
  // padding slots of the last word
#pragma unroll
  for (int F = kNFA; F < kSlots<S>; ++F)
#pragma unroll
    for (int l = 0; l < Q; ++l) Codec<S>::store(f + ad_fidx<Q, S>((uint32_t)c, F, l), 0.0f);
  if (bad) atomicOr(flag, 1);
}

// Corrected moments of the 37 fields in FP64 ([37][cells]): rho = rho~ +
// dt S(rho~)/2 for the 16, the plain sums for A and D.
template <int Q, class S>
__global__ void __launch_bounds__(128) k_ad_moments(const S* __restrict__ f,
                                                     double* __restrict__ out, Grid G,
                                                     double half_dt, int slicing) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= G.cells) return;
  double rt[kNFA];
#pragma unroll
  for (int F = 0; F < kNFA; ++F) {
    double s = 0;
#pragma unroll
    for (int l = 0; l < Q; ++l) s += (double)Codec<S>::load_keep(f + ad_fidx<Q, S>((uint32_t)c, F, l));
    rt[F] = s;
  }
  double A[3], D[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    A[k] = rt[kA + k];
#pragma unroll
    for (int q = 0; q < 6; ++q) D[k][q] = rt[kD + 6 * k + q];
  }
  double alpha, gm[6], K[6], V[3];
  unpack<kABS, double>(rt, alpha, gm, K, V);
  double Sr[kNF];
  bm_sources<double>(alpha, gm, K, V, A, D, slicing, Sr);
#pragma unroll
  for (int F = 0; F < kNFA; ++F)
    out[(int64_t)F * G.cells + c] = F < kNF ? rt[F] + half_dt * Sr[F] : rt[F];
}

inline unsigned blocks_for(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ---------------------------------------------------------------------------
// Shared-memory staged form: every distribution is read from HBM once
// ---------------------------------------------------------------------------
// One persistent CTA per SM. Warp NC (the producer) copies each tile of 32
// consecutive cells, the contiguous block of its words, into one of NS
// shared-memory stages with one bulk copy (cp.async.bulk). Each stage belongs
// to a group of P consumer warps, which takes the CTA's tiles s, s + NS, ...
// With P = 2 two lanes share a cell: each sums the fields of half of the
// words from shared memory and the partner lanes swap them, both evaluate the
// cell's sources and fluxes, and each relaxes and stores its half of the
// words. The group then frees the stage. Every wait is bounded (~2 s, then
// bit 1 of the flag).
constexpr int kTileCells = 32;

template <class S>
__host__ __device__ constexpr uint32_t tma_stage(int Q) {
  return (uint32_t)(kSlots<S> * Q * kTileCells * sizeof(S));
}
// Stages that fit the 227 KB of shared memory (at most 4).
template <class S>
__host__ __device__ constexpr int tma_stages(int Q) {
  return (int)((232448u - 1024u) / tma_stage<S>(Q)) > 4 ? 4
                                                       : (int)((232448u - 1024u) / tma_stage<S>(Q));
}

template <int Q, class S, class C, int NS, int P>
__global__ void __launch_bounds__(32 * (NS * P + 1), 1)
    k_ad_collide_tma(const Args<S, C> a, int64_t ntiles) {
  static_assert(P == 1 || P == 2, "one or two lanes per cell");
  using L = Lattice<Q>;
  using W = typename Codec<S>::W;
  constexpr int dim = L::kDim;
  constexpr int T = kTileCells;
  constexpr int V = Codec<S>::kV;
  constexpr int NW = kWords<S>;
  constexpr int NC = NS * P;  // consumer warps
  constexpr uint32_t STAGEB = tma_stage<S>(Q);
  constexpr uint64_t kLimitNs = 2000000000ull;
  static_assert(STAGEB % 16 == 0, "bulk copies move multiples of 16 bytes");

  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);  // [0,NS) full, [NS,2NS) empty
  unsigned char* stages = smem + 1024;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[NS + s]), P);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t G = gridDim.x;
  const int64_t my = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / G + 1 : 0;

  if (warp == NC) {
    // ---------------- producer ----------------
    if (lane == 0) {
      int64_t issued = 0;
      for (int64_t j = 0; j < my; ++j) {
        const int s = (int)(j % NS);
        const int64_t r = j / NS;
        if (r >= 1 && !mbar_wait(smem_u32(&bars[NS + s]), (uint32_t)((r - 1) & 1), kLimitNs)) {
          atomicOr(a.flag, 2);
          break;
        }
        const int64_t tile = blockIdx.x + j * G;
        if ((tile + 1) * T > a.G.pstride) {  // never true for a consistent launch
          atomicOr(a.flag, 4);
          break;
        }
        const uint32_t fb = smem_u32(&bars[s]);
        mbar_expect_tx(fb, STAGEB);
        bulk_load(smem_u32(stages + (size_t)s * STAGEB),
                  a.fin + (size_t)tile * (size_t)(kSlots<S> * Q * T), STAGEB, fb);
        issued = j + 1;
      }
      // leave only when every copy started here has landed
      for (int64_t j = issued > NS ? issued - NS : 0; j < issued; ++j) {
        if (!mbar_wait(smem_u32(&bars[j % NS]), (uint32_t)((j / NS) & 1), kLimitNs)) {
          atomicOr(a.flag, 2);
          break;
        }
      }
    }
    return;
  }

  // ---------------- consumers ----------------
  const int s = warp / P;
  const int g = P == 2 ? (lane >> 4) : 0;  // which half of the words this lane owns
  const int ci = P == 2 ? (warp % P) * 16 + (lane & 15) : lane;
  const int64_t cells = a.G.cells;
  for (int64_t m = 0;; ++m) {
    const int64_t j = s + m * NS;
    if (j >= my) break;
    const int64_t tile = blockIdx.x + j * G;
    const int64_t cell = tile * T + ci;
    const bool valid = cell < cells;
    const int64_t c = valid ? cell : cells - 1;
    const Nbr n = make_nbr(a.G, c);
    if (!mbar_wait(smem_u32(&bars[s]), (uint32_t)(m & 1), kLimitNs)) {
      if (lane == 0) atomicOr(a.flag, 2);
      break;
    }
    const S* st = reinterpret_cast<const S*>(stages + (size_t)s * STAGEB);
    auto word = [&](int w, int l) -> W {
      return *reinterpret_cast<const W*>(st + ad_fidx<Q, S>((uint32_t)ci, V * w, l));
    };
    C rt[kNFA];
    if constexpr (P == 1) {
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        C sum[V];
#pragma unroll
        for (int i = 0; i < V; ++i) sum[i] = C(0);
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          C v[V];
          unpack_word<S>(word(w, l), v);
#pragma unroll
          for (int i = 0; i < V; ++i) sum[i] += v[i];
        }
#pragma unroll
        for (int i = 0; i < V; ++i)
          if (V * w + i < kNFA) rt[V * w + i] = sum[i];
      }
    } else {
      // words 2jj (lanes g = 0) and 2jj + 1 (g = 1), swapped between partner
      // lanes; with an odd word count both lanes sum the last word
#pragma unroll
      for (int jj = 0; jj < NW / 2; ++jj) {
        C sum[V];
#pragma unroll
        for (int i = 0; i < V; ++i) sum[i] = C(0);
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          C v[V];
          unpack_word<S>(word(2 * jj + g, l), v);
#pragma unroll
          for (int i = 0; i < V; ++i) sum[i] += v[i];
        }
#pragma unroll
        for (int i = 0; i < V; ++i) {
          const C other = __shfl_xor_sync(0xffffffffu, sum[i], 16);
          if (V * (2 * jj) + i < kNFA) rt[V * (2 * jj) + i] = g ? other : sum[i];
          if (V * (2 * jj + 1) + i < kNFA) rt[V * (2 * jj + 1) + i] = g ? sum[i] : other;
        }
      }
      if constexpr (NW % 2 == 1) {
        C sum[V];
#pragma unroll
        for (int i = 0; i < V; ++i) sum[i] = C(0);
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          C v[V];
          unpack_word<S>(word(NW - 1, l), v);
#pragma unroll
          for (int i = 0; i < V; ++i) sum[i] += v[i];
        }
#pragma unroll
        for (int i = 0; i < V; ++i)
          if (V * (NW - 1) + i < kNFA) rt[V * (NW - 1) + i] = sum[i];
      }
    }
    bool bad;
    {
      C chk = C(0);
#pragma unroll
      for (int F = 0; F < kNFA; ++F) chk += rt[F];
      bad = valid && g == 0 && !isfinite(chk);
    }
    C A[3], D[3][6];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      A[k] = rt[kA + k];
#pragma unroll
      for (int q = 0; q < 6; ++q) D[k][q] = rt[kD + 6 * k + q];
    }
    C alpha, gm[6], K[6], Vv[3];
    unpack<kABS, C>(rt, alpha, gm, K, Vv);
    C Sr[kNF];
    bm_sources<C>(alpha, gm, K, Vv, A, D, a.slicing, Sr);
    C rho[kNF];
#pragma unroll
    for (int F = 0; F < kNF; ++F) rho[F] = rt[F] + a.half_dt * Sr[F];
    C Fl[6][3], aQ, aK[6];
    {
      C alpha2, g2[6], K2[6], V2[3];
      unpack<kABS, C>(rho, alpha2, g2, K2, V2);
      bm_flux<C, dim>(alpha2, g2, V2, A, D, Fl);
      aQ = alpha_q<C>(a.slicing, alpha2, g2, K2);
#pragma unroll
      for (int q = 0; q < 6; ++q) aK[q] = alpha2 * K2[q];
    }

    // relax and store word w of this cell with coefficients cf and b
    auto relax = [&](int w, const C cf[V], const C b[V][3], bool store) {
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        C v[V], out[V];
        unpack_word<S>(word(w, l), v);
#pragma unroll
        for (int i = 0; i < V; ++i) {
          C t = cf[i];
#pragma unroll
          for (int k = 0; k < dim; ++k) {
            if (L::c(l, k) > 0) t += b[i][k];
            if (L::c(l, k) < 0) t -= b[i][k];
          }
          out[i] = fma(a.omc, v[i], C(L::w(l)) * t);
        }
        store_word_if<S>(a.fout + ad_fidx<Q, S>(n.at(L::c(l, 0), L::c(l, 1), L::c(l, 2)), V * w, l),
                         out, store);
      }
    };
    if constexpr (P == 1) {
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        C cf[V], b[V][3];
#pragma unroll
        for (int i = 0; i < V; ++i) ad_word_terms<dim>(V * w + i, rt, rho, Sr, Fl, aQ, aK, a, cf[i], b[i]);
        relax(w, cf, b, valid);
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < NW / 2; ++jj) {
        C cf0[V], b0[V][3], cf1[V], b1[V][3], cf[V], b[V][3];
#pragma unroll
        for (int i = 0; i < V; ++i) {
          ad_word_terms<dim>(V * (2 * jj) + i, rt, rho, Sr, Fl, aQ, aK, a, cf0[i], b0[i]);
          ad_word_terms<dim>(V * (2 * jj + 1) + i, rt, rho, Sr, Fl, aQ, aK, a, cf1[i], b1[i]);
          cf[i] = g ? cf1[i] : cf0[i];
#pragma unroll
          for (int k = 0; k < 3; ++k) b[i][k] = g ? b1[i][k] : b0[i][k];
        }
        relax(2 * jj + g, cf, b, valid);
      }
      if constexpr (NW % 2 == 1) {
        C cf[V], b[V][3];
#pragma unroll
        for (int i = 0; i < V; ++i) ad_word_terms<dim>(V * (NW - 1) + i, rt, rho, Sr, Fl, aQ, aK, a, cf[i], b[i]);
        relax(NW - 1, cf, b, valid && g == 0);
      }
    }
    if (bad) atomicOr(a.flag, 1);
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&bars[NS + s]));
  }
}

// One (F, l) of every cell of the 37-field state to FP64 and back.
template <int Q, class S>
__global__ void k_ad_get_plane(const S* __restrict__ f, double* __restrict__ out, int64_t cells,
                               int F, int l) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < cells) out[c] = (double)Codec<S>::load_keep(f + ad_fidx<Q, S>((uint32_t)c, F, l));
}
template <int Q, class S>
__global__ void k_ad_set_plane(S* __restrict__ f, const double* __restrict__ in, int64_t cells,
                               int F, int l) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < cells) Codec<S>::store(f + ad_fidx<Q, S>((uint32_t)c, F, l), (decltype(Codec<S>::load(f)))in[c]);
}

template <int Q, class S>
struct Ops {
  using C = typename std::conditional<sizeof(S) == 8, double, float>::type;
  template <int MINB>
  static cudaError_t step(const Grid& G, const void* fin, void* fout, int* flag, double tau,
                          double dt, int slicing, cudaStream_t st) {
    Args<S, C> a;
    a.fin = static_cast<const S*>(fin);
    a.fout = static_cast<S*>(fout);
    a.flag = flag;
    a.G = G;
    a.half_dt = C(0.5 * dt);
    a.omega = C(1.0 / tau);
    a.omc = C(1.0 - 1.0 / tau);
    a.sigma = C(dt * (1.0 - 1.0 / (2.0 * tau)));
    a.slicing = slicing;
    k_ad_collide<Q, S, C, MINB><<<blocks_for(G.cells, 128), 128, 0, st>>>(a);
    return cudaGetLastError();
  }
  template <int P>
  static cudaError_t step_tma(const Grid& G, const void* fin, void* fout, int* flag, double tau,
                              double dt, int slicing, cudaStream_t st) {
    constexpr int NS = tma_stages<S>(Q);
    static_assert(NS >= 1, "a stage must fit in shared memory");
    constexpr uint32_t smem = 1024u + NS * tma_stage<S>(Q);
    Args<S, C> a;
    a.fin = static_cast<const S*>(fin);
    a.fout = static_cast<S*>(fout);
    a.flag = flag;
    a.G = G;
    a.half_dt = C(0.5 * dt);
    a.omega = C(1.0 / tau);
    a.omc = C(1.0 - 1.0 / tau);
    a.sigma = C(dt * (1.0 - 1.0 / (2.0 * tau)));
    a.slicing = slicing;
    auto kern = k_ad_collide_tma<Q, S, C, NS, P>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = G.pstride / kTileCells;
    const int64_t grid = ntiles < sms ? ntiles : (sms > 0 ? sms : 1);
    kern<<<(unsigned)grid, 32 * (NS * P + 1), smem, st>>>(a, ntiles);
    return cudaGetLastError();
  }
  static cudaError_t init(const Grid& G, const double* fields, int nf, void* f, int* flag,
                          double dx, double dt, int slicing, cudaStream_t st) {
    k_ad_init<Q, S><<<blocks_for(G.cells, 128), 128, 0, st>>>(
        fields, nf, static_cast<S*>(f), flag, G, 1.0 / (2.0 * dx), 1.0 / (4.0 * dx), 0.5 * dt,
        slicing);
    return cudaGetLastError();
  }
  static cudaError_t moments(const Grid& G, const void* f, double* out, double dt, int slicing,
                             cudaStream_t st) {
    k_ad_moments<Q, S><<<blocks_for(G.cells, 128), 128, 0, st>>>(static_cast<const S*>(f), out,
                                                                 G, 0.5 * dt, slicing);
    return cudaGetLastError();
  }
  static cudaError_t get_plane(const Grid& G, const void* f, int F, int l, double* out,
                               cudaStream_t st) {
    k_ad_get_plane<Q, S><<<blocks_for(G.cells, 256), 256, 0, st>>>(static_cast<const S*>(f), out,
                                                                   G.cells, F, l);
    return cudaGetLastError();
  }
  static cudaError_t set_plane(const Grid& G, void* f, int F, int l, const double* in,
                               cudaStream_t st) {
    k_ad_set_plane<Q, S><<<blocks_for(G.cells, 256), 256, 0, st>>>(static_cast<S*>(f), in,
                                                                   G.cells, F, l);
    return cudaGetLastError();
  }
};

// Launch forms: blocks of 128 threads sized for 2 to 5 blocks per SM, and
// the shared-memory staged form with one or two lanes per cell (blocks per
// SM 0 and -1 mark them).
constexpr int kForms = 6;
constexpr int kFormBlocks[kForms] = {2, 3, 4, 5, 0, -1};

struct Table {
  cudaError_t (*step[kForms])(const Grid&, const void*, void*, int*, double, double, int,
                              cudaStream_t);
  cudaError_t (*init)(const Grid&, const double*, int, void*, int*, double, double, int,
                      cudaStream_t);
  cudaError_t (*moments)(const Grid&, const void*, double*, double, int, cudaStream_t);
  cudaError_t (*get_plane)(const Grid&, const void*, int, int, double*, cudaStream_t);
  cudaError_t (*set_plane)(const Grid&, void*, int, int, const double*, cudaStream_t);
};

template <int Q, class S>
Table make_table() {
  return Table{{&Ops<Q, S>::template step<2>, &Ops<Q, S>::template step<3>,
                &Ops<Q, S>::template step<4>, &Ops<Q, S>::template step<5>,
                &Ops<Q, S>::template step_tma<1>, &Ops<Q, S>::template step_tma<2>},
               &Ops<Q, S>::init, &Ops<Q, S>::moments, &Ops<Q, S>::get_plane,
               &Ops<Q, S>::set_plane};
}

// One translation unit per (Q, storage), compiled in parallel.
Table table_q3_f64();
Table table_q9_f64();
Table table_q19_f64();
Table table_q3_f32();
Table table_q9_f32();
Table table_q19_f32();

}  // namespace ad
}  // namespace lbnr

