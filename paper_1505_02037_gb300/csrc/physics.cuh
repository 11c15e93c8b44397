// Pointwise Bona-Masso right-hand sides at zero shift in vacuum
// (Ilseven & Mendoza, arXiv:1505.02037, Sec. "Bona-Masso evolution
// equations"; Eq. alfan for the lapse, the three-metric equation, the
// extrinsic-curvature flux lambda^k_ij and source S_ij, and Eq. Vsor for
// Omega_k).
//
// Symmetric tensors are held as their 6 independent components
// (xx, xy, xz, yy, yz, zz); D_kij as D[k][6]. All loops are unrolled so
// every index is a compile-time constant and every array lives in registers.
//
// Index placement: raised indices use the inverse three-metric g^{ij};
// D_kr^r = g^{rm} D_krm, D^r_rk = g^{rm} D_mrk, D_k^{rs} = g^{ra} g^{sb} D_kab,
// D^k_ij = g^{km} D_mij. The second term of the gamma_ij/4 bracket of S_ij is
// taken as D_kr^r D^{ks}_s: with that placement the K equation equals the ADM
// evolution minus (alpha/4) gamma_ij times the Hamiltonian constraint, as the
// paper's "Einstein evolution system" requires.
#pragma once

namespace lbnr {

// Index of the stored component (i, j) of a symmetric tensor. Not recursive,
// so that every use with constant arguments folds to an immediate and the
// arrays it indexes stay in registers.
__host__ __device__ constexpr int sym(int i, int j) {
  return (i < j ? i : j) == 0 ? (i < j ? j : i) : ((i < j ? i : j) == 1 ? 2 + (i < j ? j : i) : 5);
}

template <class T>
__device__ __forceinline__ void invert_sym3(const T g[6], T gi[6]) {
  const T c00 = g[3] * g[5] - g[4] * g[4];
  const T c01 = g[2] * g[4] - g[1] * g[5];
  const T c02 = g[1] * g[4] - g[2] * g[3];
  const T det = g[0] * c00 + g[1] * c01 + g[2] * c02;
  const T inv = T(1) / det;
  gi[0] = c00 * inv;
  gi[1] = c01 * inv;
  gi[2] = c02 * inv;
  gi[3] = (g[0] * g[5] - g[2] * g[2]) * inv;
  gi[4] = (g[1] * g[2] - g[0] * g[4]) * inv;
  gi[5] = (g[0] * g[3] - g[1] * g[1]) * inv;
}

// The 16 field values in storage order: alpha, gamma(6), K(6), V(3).
enum : int { kAlpha = 0, kG = 1, kK = 7, kV = 13, kNF = 16 };

// Sources S_F of all 16 fields (d_t of each field less its flux divergence)
// at the state (alpha, gamma, K, V) with derivatives A_k, D_kij.
//
// Matter (Sec. "Expansion of flat universe"): a perfect fluid at rest in the
// slice frame, with energy density rho = alpha^2 G^00 and pressure P:
// G_ij = P gamma_ij, tr G = 3P, G^0_k = 0. S_ij gains -R^(4)_ij +
// (gamma_ij / 4) 2 alpha^2 G^00 with R^(4)_ij = G_ij - (gamma_ij / 2)
// (-alpha^2 G^00 + tr G) = (rho - P) gamma_ij / 2, so the sum is
// (P / 2) gamma_ij and rho drops out; Omega_k gains alpha^2 G^0_k = 0.
// fluidP = 0 is vacuum.
template <class T>
__device__ __forceinline__ void bm_sources(const T alpha, const T g[6], const T K[6],
                                           const T V[3], const T A[3], const T D[3][6],
                                           int slicing, T S[kNF], T fluidP = T(0)) {
  T gi[6];
  invert_sym3(g, gi);

  // K^i_j = g^{im} K_mj (not symmetric in general)
  T Km[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Km[i][j] = gi[sym(i, 0)] * K[sym(0, j)] + gi[sym(i, 1)] * K[sym(1, j)] +
                 gi[sym(i, 2)] * K[sym(2, j)];
  const T trK = Km[0][0] + Km[1][1] + Km[2][2];
  T trK2 = T(0);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) trK2 += Km[i][j] * Km[j][i];

  // D_ki^r = D_kim g^{mr}
  T Dl[3][3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int r = 0; r < 3; ++r)
        Dl[k][i][r] = D[k][sym(i, 0)] * gi[sym(0, r)] + D[k][sym(i, 1)] * gi[sym(1, r)] +
                      D[k][sym(i, 2)] * gi[sym(2, r)];
  // traces: D_kr^r and D^r_rk
  T tr1[3], tr2[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    tr1[k] = Dl[k][0][0] + Dl[k][1][1] + Dl[k][2][2];
    tr2[k] = Dl[0][k][0] + Dl[1][k][1] + Dl[2][k][2];
  }
  // raised vectors
  T Au[3], Vu[3], tr1u[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Au[k] = gi[sym(k, 0)] * A[0] + gi[sym(k, 1)] * A[1] + gi[sym(k, 2)] * A[2];
    Vu[k] = gi[sym(k, 0)] * V[0] + gi[sym(k, 1)] * V[1] + gi[sym(k, 2)] * V[2];
    tr1u[k] = gi[sym(k, 0)] * tr1[0] + gi[sym(k, 1)] * tr1[1] + gi[sym(k, 2)] * tr1[2];
  }
  // D^k_ij = g^{km} D_mij (symmetric in ij)
  T Du[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int q = 0; q < 6; ++q)
      Du[k][q] = gi[sym(k, 0)] * D[0][q] + gi[sym(k, 1)] * D[1][q] + gi[sym(k, 2)] * D[2][q];
  // Christoffel symbols Gamma^k_ij = D_ij^k + D_ji^k - D^k_ij
  T Gam[3][6];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) Gam[k][sym(i, j)] = Dl[i][j][k] + Dl[j][i][k] - Du[k][sym(i, j)];
  // Gamma^k_kr
  T Gc[3];
#pragma unroll
  for (int r = 0; r < 3; ++r)
    Gc[r] = Gam[0][sym(0, r)] + Gam[1][sym(1, r)] + Gam[2][sym(2, r)];
  // D_k^{kr} = g^{ka} D_ka^r
  T Dkk[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    T t = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int a = 0; a < 3; ++a) t += gi[sym(k, a)] * Dl[k][a][r];
    Dkk[r] = t;
  }
  // In FP64 (bound by its arithmetic) two sums are taken with fewer
  // operations: D_k^{rs} Gamma^k_rs over the six pairs r <= s (both factors
  // are symmetric in rs), and M_ij = D_ik^r D_rj^k once for all six S_ij. The
  // FP32 forms keep the plain sums, whose register allocation they are tuned to.
  constexpr bool kLean = sizeof(T) == 8;
  // D_k^{rs} Gamma^k_rs, with D_k^{rs} = g^{ra} D_ka^s
  T DG = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int s = kLean ? r : 0; s < 3; ++s) {
        const T Duu = gi[sym(r, 0)] * Dl[k][0][s] + gi[sym(r, 1)] * Dl[k][1][s] +
                      gi[sym(r, 2)] * Dl[k][2][s];
        DG += (kLean && r != s ? T(2) : T(1)) * Duu * Gam[k][sym(r, s)];
      }
  T Mdd[3][3];
  if (kLean) {
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        T t = T(0);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int r = 0; r < 3; ++r) t += Dl[i][k][r] * Dl[r][j][k];
        Mdd[i][j] = t;
      }
  }
  const T bracket = -DG + (tr1[0] * tr1u[0] + tr1[1] * tr1u[1] + tr1[2] * tr1u[2]) -
                    T(2) * (Vu[0] * A[0] + Vu[1] * A[1] + Vu[2] * A[2]) + trK2 - trK * trK;

  // S_ij
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int q = sym(i, j);
      // -2 K_ik K^k_j + trK K_ij
      T t = -T(2) * (K[sym(i, 0)] * Km[0][j] + K[sym(i, 1)] * Km[1][j] + K[sym(i, 2)] * Km[2][j]) +
            trK * K[q];
      // 2 D_ik^r D_rj^k + 2 D_jk^r D_ri^k ; Gamma^k_kr Gamma^r_ij - Gamma^k_ri Gamma^r_kj
      if (kLean) {
        t += T(2) * (Mdd[i][j] + Mdd[j][i]);
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int r = 0; r < 3; ++r) t -= Gam[k][sym(r, i)] * Gam[r][sym(k, j)];
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
          for (int r = 0; r < 3; ++r)
            t += T(2) * (Dl[i][k][r] * Dl[r][j][k] + Dl[j][k][r] * Dl[r][i][k]) -
                 Gam[k][sym(r, i)] * Gam[r][sym(k, j)];
      }
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        t += Gc[r] * Gam[r][q];
        // -(2 D_k^{kr} - A^r)(D_ijr + D_jir)
        t -= (T(2) * Dkk[r] - Au[r]) * (D[i][sym(j, r)] + D[j][sym(i, r)]);
        // - V^k D_kij
        t -= Vu[r] * D[r][q];
      }
      // A_i (V_j - D_jk^k / 2) + A_j (V_i - D_ik^k / 2)
      t += A[i] * (V[j] - T(0.5) * tr1[j]) + A[j] * (V[i] - T(0.5) * tr1[i]);
      t += T(0.25) * g[q] * bracket;
      t += T(0.5) * fluidP * g[q];
      S[kK + q] = alpha * t;
    }

  // Omega_k (Eq. Vsor at zero shift, vacuum)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T t = A[0] * Km[0][k] + A[1] * Km[1][k] + A[2] * Km[2][k] - trK * A[k];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
      for (int s = 0; s < 3; ++s) t += (Dl[k][r][s] - T(2) * Dl[r][k][s]) * Km[r][s];
      t -= Km[r][k] * (tr1[r] - T(2) * tr2[r]);
    }
    S[kV + k] = alpha * t;
  }

  // Lapse (Eq. alfan, beta = 0) and metric (beta = 0, s_ij = 0)
  const T Qg = slicing == 1 ? trK : (slicing == 2 ? trK / alpha : T(0));
  S[kAlpha] = -alpha * alpha * Qg;
#pragma unroll
  for (int q = 0; q < 6; ++q) S[kG + q] = -T(2) * alpha * K[q];
}

// Flux of K_ij along axis k: alpha lambda^k_ij, with
// lambda^k_ij = D^k_ij + 1/2 delta^k_i (A_j + 2 V_j - D_jr^r)
//             + 1/2 delta^k_j (A_i + 2 V_i - D_ir^r) - 1/2 V^k gamma_ij.
// Only the first `dim` axes are formed (the lattice has no other velocities).
template <class T, int dim>
__device__ __forceinline__ void bm_flux(const T alpha, const T g[6], const T V[3], const T A[3],
                                        const T D[3][6], T F[6][3]) {
  T gi[6];
  invert_sym3(g, gi);
  T tr1[3];
#pragma unroll
  for (int k = 0; k < 3; ++k)
    tr1[k] = gi[0] * D[k][0] + gi[3] * D[k][3] + gi[5] * D[k][5] +
             T(2) * (gi[1] * D[k][1] + gi[2] * D[k][2] + gi[4] * D[k][4]);
  T e[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) e[i] = T(0.5) * (A[i] + T(2) * V[i] - tr1[i]);
#pragma unroll
  for (int k = 0; k < dim; ++k) {
    const T Vu = gi[sym(k, 0)] * V[0] + gi[sym(k, 1)] * V[1] + gi[sym(k, 2)] * V[2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = i; j < 3; ++j) {
        const int q = sym(i, j);
        T l = gi[sym(k, 0)] * D[0][q] + gi[sym(k, 1)] * D[1][q] + gi[sym(k, 2)] * D[2][q] -
              T(0.5) * Vu * g[q];
        if (k == i) l += e[j];
        if (k == j) l += e[i];
        F[q][k] = alpha * l;
      }
  }
#pragma unroll
  for (int k = dim; k < 3; ++k)
#pragma unroll
    for (int q = 0; q < 6; ++q) F[q][k] = T(0);
}

// Shift-field terms (Sec. "Bona-Masso evolution equations"; B_k^i =
// d_k beta^i / 2, B[k][i]): added to the sources S (metric, K_ij: alpha S_ij,
// V: Omega_k) at the point, with B_ij = B_i^m gamma_mj, B^r_s = g^{rl} B_ls.
//   gamma_ij: 2 (B_ij + B_ji)
//   K_ij:     2 (K_ir B_j^r + K_jr B_i^r - K_ij tr B)
//   V_k:      2 (B_k^r - delta_k^r tr B) V_r + 2 (D_rk^s - delta^s_k D^j_jr) B^r_s
template <class T>
__device__ __forceinline__ void shift_field_sources(const T g[6], const T K[6], const T V[3],
                                                    const T D[3][6], const T B[3][3],
                                                    T S[16]) {
  T gi[6];
  invert_sym3(g, gi);
  T Bl[3][3], Bul[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Bl[i][j] = B[i][0] * g[sym(0, j)] + B[i][1] * g[sym(1, j)] + B[i][2] * g[sym(2, j)];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Bul[i][j] = gi[sym(i, 0)] * Bl[0][j] + gi[sym(i, 1)] * Bl[1][j] + gi[sym(i, 2)] * Bl[2][j];
  const T trB = B[0][0] + B[1][1] + B[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int q = sym(i, j);
      S[1 + q] += T(2) * (Bl[i][j] + Bl[j][i]);
      T t = -K[q] * trB;
#pragma unroll
      for (int r = 0; r < 3; ++r) t += K[sym(i, r)] * B[j][r] + K[sym(j, r)] * B[i][r];
      S[7 + q] += T(2) * t;
    }
  // D^j_jr = g^{ja} D_jar
  T Dt2[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    T t = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
      for (int a = 0; a < 3; ++a) t += gi[sym(j, a)] * D[j][sym(a, r)];
    Dt2[r] = t;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T t = T(0);
#pragma unroll
    for (int r = 0; r < 3; ++r) t += (B[k][r] - (k == r ? trB : T(0))) * V[r];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
#pragma unroll
      for (int s2 = 0; s2 < 3; ++s2) {
        // D_rk^s = g^{sm} D_rkm
        const T Drks = gi[sym(s2, 0)] * D[r][sym(k, 0)] + gi[sym(s2, 1)] * D[r][sym(k, 1)] +
                       gi[sym(s2, 2)] * D[r][sym(k, 2)];
        t += (Drks - (s2 == k ? Dt2[r] : T(0))) * Bul[r][s2];
      }
    }
    S[13 + k] += T(2) * t;
  }
}

// Flux of V_i along k under a shift field: -beta^k V_i + B^k_i - B_i^k
// (the V equation's flux; B^k_i = g^{kl} B_l^m gamma_mi).
template <class T, int dim>
__device__ __forceinline__ void shift_field_vflux(const T g[6], const T V[3], const T beta[3],
                                                  const T B[3][3], T Fv[3][3]) {
  T gi[6];
  invert_sym3(g, gi);
  T Bl[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Bl[i][j] = B[i][0] * g[sym(0, j)] + B[i][1] * g[sym(1, j)] + B[i][2] * g[sym(2, j)];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (k < dim) {
        const T Bki = gi[sym(k, 0)] * Bl[0][i] + gi[sym(k, 1)] * Bl[1][i] + gi[sym(k, 2)] * Bl[2][i];
        Fv[i][k] = -beta[k] * V[i] + Bki - B[i][k];
      } else {
        Fv[i][k] = T(0);
      }
    }
}

}  // namespace lbnr
