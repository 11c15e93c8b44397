// TMA-fed, warp-specialised form of the fused collide-and-stream step
// (same arithmetic as k_collide in kernels.cuh: Eq. numlb with the
// equilibria and sources of Eqs. alfa-ekstsor and rho = sum f + dt S/2).
//
// One persistent CTA per SM. Warp NC (the producer) streams tiles of 32
// consecutive cells into a ring of NS shared-memory stages: in the
// tile-blocked layout a tile's 16 Q rows of 32 values are one contiguous
// block, and the whole stage arrives through one bulk copy (cp.async.bulk)
// that signals a "full" mbarrier. Consumer warps
// 0..NC-1 each take whole tiles: two lanes per cell, each lane owning 8 of
// the 16 fields. A consumer sums its moments from shared memory, swaps them
// with its partner lane, evaluates the Bona-Masso sources and fluxes, then
// relaxes and streams every value of the tile straight from shared memory to
// the destination buffer and releases the stage through an "empty" mbarrier.
// Registers only carry the physics, so occupancy no longer depends on the
// 304 distributions of a D3Q19 cell.
//
// Reads must be local (ping-pong, or AA at an even step): the stage holds
// the planes of the tile's own cells. Every wait is bounded: after ~2 s the
// kernel sets bit 1 of the flag word and leaves.
#pragma once

#include <cuda.h>

#include "kernels.cuh"

namespace lbnr {


__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      "  .reg .pred p;\n"
      "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "  selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits for the phase of the given parity to complete; false after limit_ns.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}
// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned)
// from global to shared memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

template <int Q>
struct TmaShape {
  static constexpr int kPlanes = kNF * Q;
};

template <class S>
__host__ __device__ constexpr uint32_t tma_stage_bytes(int Q, int TC) {
  return (uint32_t)(kNF * Q * TC * sizeof(S));
}
__host__ __device__ constexpr uint32_t tma_smem_bytes(uint32_t stage_bytes, int NS) {
  return 1024u + stage_bytes * (uint32_t)NS;
}

// TC = 32 cells per tile; P lanes per cell (P = 2: each lane owns 8
// fields and partner lanes swap moments; P = 1: one lane per cell, all 16
// fields). A tile is consumed by WPT = TC / (32/P) warps together (a group);
// there are NP = NC/WPT groups, and each group owns K
// consecutive stages of the ring (NS = NP*K). Tile j of this CTA goes to
// group j % NP as its m-th tile (m = j / NP) and lands in the group's stage
// m % K, round m / K. Every stage is therefore filled and consumed in round
// order by one group, so a parity wait can never mistake an older phase for
// the awaited one.
template <int Q, class S, class C, int REP, int LAYOUT, int NC, int K, int TC, int P>
__global__ void __launch_bounds__(32 * (NC + 1), 1)
    k_collide_tma(const StepArgs<S, C> a, int64_t ntiles) {
  static_assert(LAYOUT == kPingPong || LAYOUT == kAAEven, "reads must be local");
  static_assert(P == 1 || P == 2, "one or two lanes per cell");
  constexpr int CPW = 32 / P;    // cells per consumer warp
  constexpr int NJ = kNF / P;    // fields per lane
  constexpr int WPT = TC / CPW;  // warps per tile
  constexpr int NP = NC / WPT;
  constexpr int NS = NP * K;
  static_assert(TC == kTileCells, "a stage is one tile of the tile-blocked layout");
  static_assert(TC % CPW == 0, "a tile holds whole warps of cells");
  static_assert(NC % WPT == 0 && K >= 1, "whole warp groups per tile");
  using L = Lattice<Q>;
  using TS = TmaShape<Q>;
  // one lane per cell: whole words (kV fields) at a time
  constexpr int VW = Codec<S>::kV;  // fields per word
  constexpr bool WORDS = P == 1 && VW > 1;
  using W = typename Codec<S>::W;
  constexpr int T = TC;
  constexpr int dim = L::kDim;
  constexpr uint32_t ROWB = T * sizeof(S);
  constexpr uint32_t STAGEB = TS::kPlanes * ROWB;
  static_assert(STAGEB % 16 == 0, "bulk copies move multiples of 16 bytes");
  constexpr uint64_t kLimitNs = 2000000000ull;

  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem);  // [0,NS) full, [NS,2NS) empty
  unsigned char* stages = smem + 1024;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&bars[s]), 1);
      mbar_init(smem_u32(&bars[NS + s]), WPT);
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
        const int64_t m = j / NP;
        const int s = (int)(j % NP) * K + (int)(m % K);
        const int64_t r = m / K;
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
        bulk_load(smem_u32(stages + (size_t)s * STAGEB), a.fin + (size_t)tile * TS::kPlanes * T,
                  STAGEB, fb);
        issued = j + 1;
      }
      // Leave only when every copy this warp started has landed: the last
      // fill of each stage is among the last NS tiles issued.
      for (int64_t j = issued > NS ? issued - NS : 0; j < issued; ++j) {
        const int64_t m = j / NP;
        const int s = (int)(j % NP) * K + (int)(m % K);
        if (!mbar_wait(smem_u32(&bars[s]), (uint32_t)((m / K) & 1), kLimitNs)) {
          atomicOr(a.flag, 2);
          break;
        }
      }
    }
    return;
  }

  // ---------------- consumers ----------------
  const int g = P == 2 ? (lane >> 4) : 0;
  const int grp = warp / WPT;
  const int half = warp % WPT;
  const int ci = half * CPW + (P == 2 ? (lane & 15) : lane);
  const int64_t cells = a.G.cells;
  for (int64_t m = 0;; ++m) {
    const int64_t j = grp + m * NP;
    if (j >= my) break;
    const int s = grp * K + (int)(m % K);
    const uint32_t ph = (uint32_t)((m / K) & 1);
    const int64_t tile = blockIdx.x + j * G;
    const int64_t cell = tile * T + ci;
    const bool valid = cell < cells;
    const int64_t c = valid ? cell : cells - 1;
    const Nbr n = make_nbr(a.G, c);
    // stencil loads first: their latency overlaps the wait for the stage
    C A[3], D[3][6];
    derivatives<Q, C>(n, cells, a.aux, a.inv2dx, a.inv4dx, A, D);
    if (!mbar_wait(smem_u32(&bars[s]), ph, kLimitNs)) {
      if (lane == 0) atomicOr(a.flag, 2);
      break;
    }
    const S* st = reinterpret_cast<const S*>(stages + (size_t)s * STAGEB);

    // moments of this lane's fields
    C mine[NJ];
    if constexpr (WORDS) {
      // one word, kV fields, per shared-memory read
#pragma unroll
      for (int m = 0; m < NJ / VW; ++m) {
        C sum[VW];
#pragma unroll
        for (int i = 0; i < VW; ++i) sum[i] = C(0);
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          C v[VW];
          Codec<S>::unpack(*reinterpret_cast<const W*>(st + fidx<Q, S>((uint32_t)ci, VW * m, l)), v);
#pragma unroll
          for (int i = 0; i < VW; ++i) sum[i] += REP == kDEV ? C(L::w(l)) * v[i] : v[i];
        }
#pragma unroll
        for (int i = 0; i < VW; ++i) mine[VW * m + i] = sum[i];
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const int F = g ? field_of(P, 1, jj) : field_of(P, 0, jj);
        C sum = C(0);
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          const C v = (C)st[fidx<Q, S>((uint32_t)ci, F, l)];
          sum += REP == kDEV ? C(L::w(l)) * v : v;
        }
        mine[jj] = sum;
      }
    }
    C rt[kNF];
#pragma unroll
    for (int jj = 0; jj < NJ; ++jj) {
      if (P == 1) {
        rt[jj] = mine[jj];
      } else {
        const C other = __shfl_xor_sync(0xffffffffu, mine[jj], 16);
        rt[field_of(P, 0, jj)] = g ? other : mine[jj];
        rt[field_of(P, 1, jj)] = g ? mine[jj] : other;
      }
    }
    {
      C chk = C(0);
#pragma unroll
      for (int F = 0; F < kNF; ++F) chk += rt[F];
      if (valid && g == 0 && !isfinite(chk)) atomicOr(a.flag, 1);
    }

    C alpha, gm[6], Kf[6], V[3];
    unpack<REP, C>(rt, alpha, gm, Kf, V);
    C Sr[kNF];
    bm_sources<C>(alpha, gm, Kf, V, A, D, a.slicing, Sr);
    add_fluid(a, alpha, gm, Sr);
    if (!a.sources_on) {
#pragma unroll
      for (int F = 0; F < kNF; ++F) Sr[F] = C(0);
    }
    C rho[kNF];
#pragma unroll
    for (int F = 0; F < kNF; ++F) rho[F] = rt[F] + a.half_dt * Sr[F];
    if (a.aux_out && valid && g == 0) write_lagged<REP, C>(a.aux_out, cells, n.c, rho);
    C Fl[6][3];
    {
      C alpha2, g2[6], K2[6], V2[3];
      unpack<REP, C>(rho, alpha2, g2, K2, V2);
      bm_flux<C, dim>(alpha2, g2, V2, A, D, Fl);
    }
    const C three_omega = C(3) * a.omega;

    if constexpr (WORDS) {
#pragma unroll
      for (int m = 0; m < NJ / VW; ++m) {
        C cf[VW], b[VW][3];
#pragma unroll
        for (int i = 0; i < VW; ++i) {
          const int F = VW * m + i;
          cf[i] = a.omega * rho[F] + a.sigma * Sr[F];
#pragma unroll
          for (int k = 0; k < 3; ++k) b[i][k] = has_flux(F) ? three_omega * Fl[F - kK][k] : C(0);
        }
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          C v[VW], out[VW];
          Codec<S>::unpack(*reinterpret_cast<const W*>(st + fidx<Q, S>((uint32_t)ci, VW * m, l)), v);
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
          WordIO<S>::stw_if(a.fout + write_index<Q, LAYOUT, S>(n, VW * m, l), Codec<S>::pack(out),
                            valid);
        }
      }
    } else {
#pragma unroll
      for (int jj = 0; jj < NJ; ++jj) {
        const int F0 = field_of(P, 0, jj), F1 = field_of(P, 1, jj);
        const int F = g ? F1 : F0;
        const C cf = a.omega * (g ? rho[F1] : rho[F0]) + a.sigma * (g ? Sr[F1] : Sr[F0]);
        C b[3] = {C(0), C(0), C(0)};
        if (has_flux(F0)) {
#pragma unroll
          for (int k = 0; k < dim; ++k) b[k] = three_omega * (g ? Fl[F1 - kK][k] : Fl[F0 - kK][k]);
        }
#pragma unroll
        for (int l = 0; l < Q; ++l) {
          const C v = (C)st[fidx<Q, S>((uint32_t)ci, F, l)];
          C t = cf;
          if (has_flux(F0)) {
#pragma unroll
            for (int k = 0; k < dim; ++k) {
              if (L::c(l, k) > 0) t += b[k];
              if (L::c(l, k) < 0) t -= b[k];
            }
          }
          const C out = REP == kDEV ? fma(a.omc, v, t) : fma(a.omc, v, C(L::w(l)) * t);
          Codec<S>::store_if(a.fout + write_index<Q, LAYOUT, S>(n, F, l), out, valid);
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&bars[NS + s]));
  }
}

}  // namespace lbnr
