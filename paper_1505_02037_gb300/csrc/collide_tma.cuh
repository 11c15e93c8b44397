// Bulk-copy-fed, warp-specialised form of the fused collide-and-stream step
// (same arithmetic as k_collide_w in kernels.cuh: Eq. numlb with the
// equilibria and sources of Eqs. alfa-ekstsor and rho = sum f + dt S/2).
//
// One persistent CTA per SM. Warp NC (the producer) streams tiles of 32
// consecutive cells into a ring of NS shared-memory stages: in the
// tile-blocked layout a tile's 16 Q rows of 32 words are one contiguous
// block, and the whole stage arrives through one bulk copy (cp.async.bulk)
// that signals a "full" mbarrier. Consumer warps 0..NC-1 each take whole
// tiles, one lane per cell: a lane sums its cell's 16 moments from shared
// memory (one word of kV fields per read), evaluates the Bona-Masso sources
// and fluxes, then relaxes and streams every value of the cell straight from
// shared memory to the destination buffer; the warp then releases the stage
// through an "empty" mbarrier. Registers only carry the physics, so
// occupancy does not depend on the 16 Q distributions of a cell.
//
// Reads must be local (ping-pong, or AA at an even step): the stage holds
// the words of the tile's own cells. Every wait is bounded: after ~2 s the
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

// Values per cell: 16 fields times Q velocities (a tile's block holds 32
// cells of them).
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

// NC consumer warps, each owning K consecutive stages of the ring (NS =
// NC K); TC = 32 cells per tile. Tile j of this CTA goes to warp j % NC as
// its m-th tile (m = j / NC) and lands in the warp's stage m % K, round
// m / K. Every stage is therefore filled and consumed in round order by one
// warp, so a parity wait can never mistake an older phase for the awaited
// one.
template <int Q, class S, class C, int REP, int LAYOUT, int NC, int K, int TC>
__global__ void __launch_bounds__(32 * (NC + 1), 1)
    k_collide_tma(const StepArgs<S, C> a, int64_t ntiles) {
  static_assert(LAYOUT == kPingPong || LAYOUT == kAAEven, "reads must be local");
  static_assert(TC == kTileCells, "a stage is one tile of the tile-blocked layout");
  static_assert(K >= 1, "at least one stage per consumer warp");
  constexpr int NS = NC * K;
  using L = Lattice<Q>;
  using TS = TmaShape<Q>;
  constexpr int VW = Codec<S>::kV;  // fields per word
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
      mbar_init(smem_u32(&bars[NS + s]), 1);
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
        const int64_t m = j / NC;
        const int s = (int)(j % NC) * K + (int)(m % K);
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
        const int64_t m = j / NC;
        const int s = (int)(j % NC) * K + (int)(m % K);
        if (!mbar_wait(smem_u32(&bars[s]), (uint32_t)((m / K) & 1), kLimitNs)) {
          atomicOr(a.flag, 2);
          break;
        }
      }
    }
    return;
  }

  // ---------------- consumers: one lane per cell ----------------
  const int64_t cells = a.G.cells;
  for (int64_t m = 0;; ++m) {
    const int64_t j = warp + m * NC;
    if (j >= my) break;
    const int s = warp * K + (int)(m % K);
    const uint32_t ph = (uint32_t)((m / K) & 1);
    const int64_t tile = blockIdx.x + j * G;
    const int64_t cell = tile * T + lane;
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

    // zeroth moments, one word (kV fields) per shared-memory read
    C rt[kNF];
#pragma unroll
    for (int F = 0; F < kNF; ++F) rt[F] = C(0);
#pragma unroll
    for (int mw = 0; mw < kNF / VW; ++mw) {
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        C v[VW];
        unpack_word<S>(*reinterpret_cast<const W*>(st + fidx<Q, S>((uint32_t)lane, VW * mw, l)), v);
#pragma unroll
        for (int i = 0; i < VW; ++i) rt[VW * mw + i] += REP == kDEV ? C(L::w(l)) * v[i] : v[i];
      }
    }
    {
      C chk = C(0);
#pragma unroll
      for (int F = 0; F < kNF; ++F) chk += rt[F];
      if (valid && !isfinite(chk)) atomicOr(a.flag, 1);
    }

    C rho[kNF], Sr[kNF], Fl[6][3], Fv[3][3];
    cell_terms<Q, S, C, REP>(a, n, rt, A, D, rho, Sr, Fl, Fv);
    if (a.aux_out && valid) write_lagged<REP, C>(a.aux_out, cells, n.c, rho);
    const C three_omega = C(3) * a.omega;

#pragma unroll
    for (int mw = 0; mw < kNF / VW; ++mw) {
      C cf[VW], b[VW][3];
#pragma unroll
      for (int i = 0; i < VW; ++i) {
        const int F = VW * mw + i;
        cf[i] = a.omega * rho[F] + a.sigma * Sr[F];
#pragma unroll
        for (int k = 0; k < 3; ++k) b[i][k] = has_flux(F) ? three_omega * Fl[F - kK][k] : C(0);
      }
#pragma unroll
      for (int l = 0; l < Q; ++l) {
        C v[VW], out[VW];
        unpack_word<S>(*reinterpret_cast<const W*>(st + fidx<Q, S>((uint32_t)lane, VW * mw, l)), v);
#pragma unroll
        for (int i = 0; i < VW; ++i) {
          C t = cf[i];
          if (has_flux(VW * mw + i)) {
#pragma unroll
            for (int k = 0; k < dim; ++k) {
              if (L::c(l, k) > 0) t += b[i][k];
              if (L::c(l, k) < 0) t -= b[i][k];
            }
          }
          out[i] = REP == kDEV ? fma(a.omc, v[i], t) : fma(a.omc, v[i], C(L::w(l)) * t);
        }
        store_word_if<S>(a.fout + write_index<Q, LAYOUT, S>(n, VW * mw, l), out, valid);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(smem_u32(&bars[NS + s]));
  }
}

}  // namespace lbnr
