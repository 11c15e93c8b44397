/*
 * lbnr oracle: a plain, slow FP64 CPU implementation of the lattice
 * Boltzmann model for the Bona-Masso form of the Einstein equations
 * (Ilseven & Mendoza, "Lattice Boltzmann Model for Numerical Relativity",
 * arXiv:1505.02037).
 *
 * TEST INFRASTRUCTURE ONLY. This file exists to check the CUDA library.
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * may build, load or run it. The product library never calls it, and the two
 * share no code, header, table or helper.
 *
 * Everything is written with full 3x3 and 3x3x3 tensors and explicit index
 * loops so that each term can be read against the paper's equations.
 *
 * Storage conventions (shared with the callers only through plain arrays):
 *   fields F = 0..15 : alpha; g_xx g_xy g_xz g_yy g_yz g_zz;
 *                      K_xx K_xy K_xz K_yy K_yz K_zz; V_x V_y V_z
 *   cell index       : x + nx*(y + ny*z)
 *   distributions    : f[(F*Q + l)*cells + cell]
 *
 * Readings of places where the paper is silent or garbled (each one is used
 * below where it applies):
 *   R1  tau is the dimensionless relaxation time tau/dt of Eq. (lbe); the
 *       factors (1 - 1/(2 tau)) of the source distributions use the same tau.
 *   R2  dt = dr (Sec. "Gauge Wave": dt = dr = 0.00125).
 *   R3  D1Q3 (c = 0, +1, -1; w = 2/3, 1/6, 1/6; c_s^2 = 1/3) is the x-marginal
 *       of D2Q9 and D3Q19; the paper prints only the 2D and 3D sets.
 *   R4  A_k and D_kij are second-order central differences of ln(alpha) and
 *       gamma_ij built from the zeroth moments sum_l f_l (Sec. "First order
 *       derivatives": evolve alpha and gamma, then differentiate).
 *   R5  One explicit evaluation per step: the macroscopic sources are taken at
 *       the uncorrected moments rho~ = sum_l f_l with the R4 derivatives; the
 *       corrected moments are rho = rho~ + dt S/2; the equilibria (and the flux
 *       lambda inside them) use the corrected rho with the same derivatives.
 *   R6  Initial distributions: f = f_eq(rho0) - (dt/2) w_l S(rho0), so that the
 *       first step's corrected moments reproduce rho0 to O(dt^2).
 *   R7  Vacuum and zero shift unless a fluid (R13) or a shift (R14 constant,
 *       R15 static field) is set: G_ab = 0, beta = B = s = 0, R4_ij = 0.
 *   R8  Index placement of the contracted D terms: every raised index uses the
 *       inverse three-metric; D_kr^r = g^{rm} D_krm, D^r_rk = g^{rm} D_mrk,
 *       D_k^{rs} = g^{ra} g^{sb} D_kab, D^k_ij = g^{km} D_mij.
 *   R9  Slicing: 0 geodesic (Q = 0), 1 harmonic (Q = tr K), 2 "1+log"
 *       (Q = tr K / alpha); all with zero shift (Sec. "Gauge choices").
 *   R10 The second term of the gamma_ij/4 bracket of S_ij is read as
 *       D_kr^r D^{ks}_s (both D traces taken over the last index pair). As
 *       printed, D_kr^r D_s^{ks}, the K equation would differ from the ADM
 *       evolution by -(alpha/4) gamma_ij D_kr^r V^k, which is not a multiple
 *       of any constraint; with the reading it differs by exactly
 *       -(alpha/4) gamma_ij times the Hamiltonian constraint, which is how
 *       the paper describes the Einstein evolution system.
 *   R17 Time level of the derivatives, variant LAG (deriv_mode 1): the
 *       paper is silent on it. A_k and D_kij come from central differences
 *       of the previous step's corrected alpha and gamma_ij (the initial
 *       fields at the first step) instead of this step's rho~. Everything
 *       else is R5. The state of a LAG run is the distributions plus those
 *       7 corrected fields ("prev"), which each step returns for the next.
 *   R18 Variant FIXED (deriv_mode 2), for measuring how much the explicit
 *       evaluation of R5 matters: the moment rule rho = rho~ + dt S(rho)/2
 *       taken as an equation and solved by fixed-point iteration over the
 *       whole lattice, with A and D from the iterate's alpha and gamma, to a
 *       relative change of 1e-15. The collision then uses S(rho), the flux
 *       at rho and the equilibria at rho, all with those A and D.
 *   R16 Independently evolved A_k and D_kij (the original formulation the
 *       paper mentions and sets aside): with zero shift their equations
 *       follow from the definitions and the lapse and metric equations,
 *       d_t A_k + d_k(alpha Q) = 0 and d_t D_kij + d_k(alpha K_ij) = 0, with
 *       equilibria w_l [A_k + c_lk alpha Q / c_s^2] and
 *       w_l [D_kij + c_lk alpha K_ij / c_s^2] and no sources. The other 16
 *       fields then take A and D from these moments instead of a stencil.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NF 16
#define ORC_QMAX 19

typedef struct {
  int32_t vset;       /* 1 = D1Q3, 2 = D2Q9, 3 = D3Q19 */
  int32_t slicing;    /* R9 */
  int32_t sources_on; /* 1 normally; 0 switches every source off (test flag) */
  int32_t deriv_mode; /* 0 SYNC (R5), 1 LAG (R17), 2 FIXED (R18) */
  int64_t nx, ny, nz;
  double dx, dt, tau;
  /* Matter (Sec. "Expansion of flat universe"): a perfect fluid at rest in
   * the slice frame with energy density rho(t) = fluid_rho0 (fluid_t0/t)^2
   * and pressure P = fluid_w rho, prescribed, not evolved. t is the time of
   * the state a call reads (the caller advances it). fluid_on = 0: vacuum. */
  double t;
  int32_t fluid_on;
  int32_t pad2;
  double fluid_rho0, fluid_w, fluid_t0;
  /* Shift (Sec. "Bona-Masso evolution equations"): a constant, uniform
   * beta^i, so B_k^i = d_k beta^i / 2 = 0, s_ij = 0, and with Q_i = 0 beta
   * stays constant. Zero: the zero-shift system of the paper's tests. */
  double beta[3];
  /* Shift field (reading R15): a prescribed, static beta^i(x), [3][cells],
   * added to beta; B_k^i = d_k beta^i / 2 from its central differences.
   * NULL: no field. */
  const double* beta_field;
} orc_params;

/* ------------------------------------------------------------------------ */
/* Velocity sets (Sec. "Lattice Boltzmann Model")                            */
/* ------------------------------------------------------------------------ */

/* D2Q9, paper ordering: c0; c1,2 = (+-1,0); c3,4 = (0,+-1); c5,6 = (+-1,-+1);
 * c7,8 = (+-1,+-1); w0 = 4/9, w1..4 = 1/9, w5..8 = 1/36. */
static const int d2q9_c[9][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
    {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},  {-1, -1, 0}};
static const double d2q9_w[9] = {4.0 / 9,  1.0 / 9,  1.0 / 9,  1.0 / 9, 1.0 / 9,
                                 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* D3Q19, paper ordering: columns of the printed 3x19 matrix, w0 = 1/3,
 * w1..6 = 1/18, w7..18 = 1/36. */
static const int d3q19_c[19][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
    {0, 0, 1},  {0, 0, -1}, {1, -1, 0}, {-1, 1, 0}, {1, 1, 0},
    {-1, -1, 0}, {1, 0, -1}, {-1, 0, 1}, {1, 0, 1},  {-1, 0, -1},
    {0, 1, -1}, {0, -1, 1}, {0, 1, 1},  {0, -1, -1}};
static const double d3q19_w[19] = {
    1.0 / 3,  1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18, 1.0 / 18,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36,
    1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};

/* D1Q3 (reading R3). */
static const int d1q3_c[3][3] = {{0, 0, 0}, {1, 0, 0}, {-1, 0, 0}};
static const double d1q3_w[3] = {2.0 / 3, 1.0 / 6, 1.0 / 6};

static const double CS2 = 1.0 / 3.0; /* c_s^2, both printed sets */

typedef struct {
  int Q;
  int c[ORC_QMAX][3];
  double w[ORC_QMAX];
} vset_t;

static int get_vset(int v, vset_t* out) {
  const int(*c)[3];
  const double* w;
  int Q;
  if (v == 1) { Q = 3; c = d1q3_c; w = d1q3_w; }
  else if (v == 2) { Q = 9; c = d2q9_c; w = d2q9_w; }
  else if (v == 3) { Q = 19; c = d3q19_c; w = d3q19_w; }
  else return -1;
  out->Q = Q;
  for (int l = 0; l < Q; ++l) {
    for (int a = 0; a < 3; ++a) out->c[l][a] = c[l][a];
    out->w[l] = w[l];
  }
  return 0;
}

/* Exported so the tests can check the tables against the paper's matrices. */
int orc_vset(int v, int* c_out, double* w_out) {
  vset_t vs;
  if (get_vset(v, &vs)) return -1;
  for (int l = 0; l < vs.Q; ++l) {
    for (int a = 0; a < 3; ++a) c_out[3 * l + a] = vs.c[l][a];
    w_out[l] = vs.w[l];
  }
  return vs.Q;
}

/* ------------------------------------------------------------------------ */
/* Symmetric-index bookkeeping for the 16 stored fields                      */
/* ------------------------------------------------------------------------ */

/* Stored symmetric pair p = 0..5 <-> (i, j): xx xy xz yy yz zz. */
static const int PAIR_I[6] = {0, 0, 0, 1, 1, 2};
static const int PAIR_J[6] = {0, 1, 2, 1, 2, 2};
static int pair_of(int i, int j) {
  static const int P[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return P[i][j];
}

enum { F_ALPHA = 0, F_G = 1, F_K = 7, F_V = 13 };

/* ------------------------------------------------------------------------ */
/* Pointwise Bona-Masso right-hand sides (Sec. "Bona-Masso evolution eqs")   */
/* ------------------------------------------------------------------------ */

typedef struct {
  double alpha;
  double beta[3];     /* shift beta^i at the point */
  double B[3][3];     /* B_k^i = d_k beta^i / 2, index [k][i] */
  double g[3][3];     /* gamma_ij */
  double K[3][3];     /* K_ij */
  double V[3];        /* V_k */
  double A[3];        /* A_k = d_k ln alpha */
  double D[3][3][3];  /* D_kij = d_k gamma_ij / 2, index [k][i][j] */
} bm_state;

typedef struct {
  double S_alpha;      /* d_t alpha (Eq. alfan) */
  double S_g[3][3];    /* d_t gamma_ij */
  double S_K[3][3];    /* alpha S_ij: source of K_ij */
  double S_V[3];       /* Omega_k (Eq. Vsor) */
  double lam[3][3][3]; /* lambda^k_ij, index [k][i][j] */
  double S_ij[3][3];   /* S_ij itself (without the factor alpha) */
  double VB[3][3];     /* B part of the flux of V_k along r: B^r_k - B_k^r, [k][r] */
  double Qg;           /* the slicing's gauge function Q */
} bm_rhs;

static double inverse3(const double g[3][3], double gi[3][3]) {
  double det = g[0][0] * (g[1][1] * g[2][2] - g[1][2] * g[2][1]) -
               g[0][1] * (g[1][0] * g[2][2] - g[1][2] * g[2][0]) +
               g[0][2] * (g[1][0] * g[2][1] - g[1][1] * g[2][0]);
  gi[0][0] = (g[1][1] * g[2][2] - g[1][2] * g[2][1]) / det;
  gi[0][1] = (g[0][2] * g[2][1] - g[0][1] * g[2][2]) / det;
  gi[0][2] = (g[0][1] * g[1][2] - g[0][2] * g[1][1]) / det;
  gi[1][0] = (g[1][2] * g[2][0] - g[1][0] * g[2][2]) / det;
  gi[1][1] = (g[0][0] * g[2][2] - g[0][2] * g[2][0]) / det;
  gi[1][2] = (g[0][2] * g[1][0] - g[0][0] * g[1][2]) / det;
  gi[2][0] = (g[1][0] * g[2][1] - g[1][1] * g[2][0]) / det;
  gi[2][1] = (g[0][1] * g[2][0] - g[0][0] * g[2][1]) / det;
  gi[2][2] = (g[0][0] * g[1][1] - g[0][1] * g[1][0]) / det;
  return det;
}

static double kdelta(int a, int b) { return a == b ? 1.0 : 0.0; }

/* Evaluates lambda^k_ij, S_ij, Omega_k and the lapse and metric sources at
 * one point, following the paper's equations term by term, with zero shift
 * (reading R7). Matter: a perfect fluid at rest in the slice frame with
 * energy density rho and pressure P (both 0 in vacuum). */
static void bm_point(const bm_state* s, int slicing, double rho, double P, bm_rhs* r) {
  double gi[3][3];
  inverse3(s->g, gi);
  const double a = s->alpha;

  /* Raised quantities (reading R8). */
  double Kmix[3][3]; /* K^i_j = g^{im} K_mj */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t = 0;
      for (int m = 0; m < 3; ++m) t += gi[i][m] * s->K[m][j];
      Kmix[i][j] = t;
    }
  double trK = 0;
  for (int i = 0; i < 3; ++i) trK += Kmix[i][i];
  double trK2 = 0; /* tr(K^2) = K^i_j K^j_i */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trK2 += Kmix[i][j] * Kmix[j][i];

  double Vup[3], Aup[3];
  for (int k = 0; k < 3; ++k) {
    Vup[k] = 0;
    Aup[k] = 0;
    for (int m = 0; m < 3; ++m) {
      Vup[k] += gi[k][m] * s->V[m];
      Aup[k] += gi[k][m] * s->A[m];
    }
  }

  /* D_ki^r = g^{rm} D_kim (last index raised). */
  double Dl2u[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int rr = 0; rr < 3; ++rr) {
        double t = 0;
        for (int m = 0; m < 3; ++m) t += gi[rr][m] * s->D[k][i][m];
        Dl2u[k][i][rr] = t;
      }
  /* D^k_ij = g^{km} D_mij (first index raised). */
  double Du1[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double t = 0;
        for (int m = 0; m < 3; ++m) t += gi[k][m] * s->D[m][i][j];
        Du1[k][i][j] = t;
      }
  /* D_k^{rs} = g^{ra} g^{sb} D_kab (both last indices raised). */
  double Du23[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int rr = 0; rr < 3; ++rr)
      for (int ss = 0; ss < 3; ++ss) {
        double t = 0;
        for (int p = 0; p < 3; ++p)
          for (int q = 0; q < 3; ++q) t += gi[rr][p] * gi[ss][q] * s->D[k][p][q];
        Du23[k][rr][ss] = t;
      }
  /* D_kr^r and D^r_rk (the two traces in V_k). */
  double Dtr1[3], Dtr2[3];
  for (int k = 0; k < 3; ++k) {
    Dtr1[k] = 0;
    Dtr2[k] = 0;
    for (int rr = 0; rr < 3; ++rr)
      for (int m = 0; m < 3; ++m) {
        Dtr1[k] += gi[rr][m] * s->D[k][rr][m];
        Dtr2[k] += gi[rr][m] * s->D[m][rr][k];
      }
  }
  /* D_k^{kr}: first index contracted with the first raised index. */
  double Dkkr[3];
  for (int rr = 0; rr < 3; ++rr) {
    Dkkr[rr] = 0;
    for (int k = 0; k < 3; ++k) Dkkr[rr] += Du23[k][k][rr];
  }
  /* D^{ks}_s = g^{ka} D_ar^r (reading R10). */
  double Dtr1up[3];
  for (int k = 0; k < 3; ++k) {
    Dtr1up[k] = 0;
    for (int m = 0; m < 3; ++m) Dtr1up[k] += gi[k][m] * Dtr1[m];
  }

  /* Christoffel symbols of the three-metric:
   * Gamma^k_ij = g^{km} (d_i g_jm + d_j g_im - d_m g_ij)/2
   *            = g^{km} (D_ijm + D_jim - D_mij). */
  double Gam[3][3][3];
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double t = 0;
        for (int m = 0; m < 3; ++m)
          t += gi[k][m] * (s->D[i][j][m] + s->D[j][i][m] - s->D[m][i][j]);
        Gam[k][i][j] = t;
      }

  /* lambda^k_ij. */
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        r->lam[k][i][j] =
            Du1[k][i][j] +
            0.5 * kdelta(k, i) * (s->A[j] + 2 * s->V[j] - Dtr1[j]) +
            0.5 * kdelta(k, j) * (s->A[i] + 2 * s->V[i] - Dtr1[i]) -
            0.5 * Vup[k] * s->g[i][j];

  /* Scalar bracket of the gamma_ij/4 term. */
  double DG = 0; /* D_k^{rs} Gamma^k_rs */
  for (int k = 0; k < 3; ++k)
    for (int rr = 0; rr < 3; ++rr)
      for (int ss = 0; ss < 3; ++ss) DG += Du23[k][rr][ss] * Gam[k][rr][ss];
  double DD = 0; /* D_kr^r D^{ks}_s (reading R10) */
  for (int k = 0; k < 3; ++k) DD += Dtr1[k] * Dtr1up[k];
  double VA = 0; /* V^k A_k */
  for (int k = 0; k < 3; ++k) VA += Vup[k] * s->A[k];
  /* Matter (Sec. "Expansion of flat universe"): G_ij = P gamma_ij,
   * G_00 = rho alpha^2 (so alpha^2 G^00 = rho), G^0_k = 0 for a fluid at
   * rest; R^(4)_ij = G_ij - gamma_ij/2 (-alpha^2 G^00 + tr G). */
  double Gdn[3][3], trG = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) Gdn[i][j] = P * s->g[i][j];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) trG += gi[i][j] * Gdn[i][j];
  const double G00up = rho / (a * a);
  double R4[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R4[i][j] = Gdn[i][j] - 0.5 * s->g[i][j] * (-a * a * G00up + trG);
  const double bracket = -DG + DD - 2 * VA + trK2 - trK * trK + 2 * a * a * G00up;

  /* S_ij. */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t = -R4[i][j];
      /* -2 K_i^k K_kj + tr K K_ij (K_i^k = K_im g^{mk} = Kmix[k][i]) */
      for (int k = 0; k < 3; ++k) t += -2 * Kmix[k][i] * s->K[k][j];
      t += trK * s->K[i][j];
      /* + 2 D_ik^r D_rj^k + 2 D_jk^r D_ri^k */
      for (int k = 0; k < 3; ++k)
        for (int rr = 0; rr < 3; ++rr)
          t += 2 * Dl2u[i][k][rr] * Dl2u[rr][j][k] +
               2 * Dl2u[j][k][rr] * Dl2u[rr][i][k];
      /* + Gamma^k_kr Gamma^r_ij - Gamma^k_ri Gamma^r_kj */
      for (int k = 0; k < 3; ++k)
        for (int rr = 0; rr < 3; ++rr)
          t += Gam[k][k][rr] * Gam[rr][i][j] - Gam[k][rr][i] * Gam[rr][k][j];
      /* - (2 D_k^{kr} - A^r)(D_ijr + D_jir) */
      for (int rr = 0; rr < 3; ++rr)
        t -= (2 * Dkkr[rr] - Aup[rr]) * (s->D[i][j][rr] + s->D[j][i][rr]);
      /* + A_i (V_j - D_jk^k / 2) + A_j (V_i - D_ik^k / 2) */
      t += s->A[i] * (s->V[j] - 0.5 * Dtr1[j]) + s->A[j] * (s->V[i] - 0.5 * Dtr1[i]);
      /* - V^k D_kij */
      for (int k = 0; k < 3; ++k) t -= Vup[k] * s->D[k][i][j];
      /* + gamma_ij / 4 (...) */
      t += 0.25 * s->g[i][j] * bracket;
      r->S_ij[i][j] = t;
      r->S_K[i][j] = a * t;
    }

  /* Omega_k (Eq. Vsor), zero shift, fluid at rest (alpha^2 G^0_k = 0):
   * alpha [ A_r (K^r_k - trK delta^r_k) + (D_kr^s - 2 D_rk^s) K^r_s
   *         - K^r_k (D_rs^s - 2 D^j_jr) ]. */
  for (int k = 0; k < 3; ++k) {
    double t = 0;
    for (int rr = 0; rr < 3; ++rr) t += s->A[rr] * (Kmix[rr][k] - trK * kdelta(rr, k));
    for (int rr = 0; rr < 3; ++rr)
      for (int ss = 0; ss < 3; ++ss)
        t += (Dl2u[k][rr][ss] - 2 * Dl2u[rr][k][ss]) * Kmix[rr][ss];
    for (int rr = 0; rr < 3; ++rr) t -= Kmix[rr][k] * (Dtr1[rr] - 2 * Dtr2[rr]);
    r->S_V[k] = a * t;
  }

  /* Shift-derivative terms (Sec. "Bona-Masso evolution equations"), all
   * zero for a constant shift: B_ij = B_i^m gamma_mj (second index
   * lowered), B^r_s = g^{rl} B_ls (first raised), tr B = B_r^r. */
  double Bl[3][3], Bul[3][3], trB = 0;
  for (int i = 0; i < 3; ++i) {
    trB += s->B[i][i];
    for (int j = 0; j < 3; ++j) {
      double t = 0;
      for (int m = 0; m < 3; ++m) t += s->B[i][m] * s->g[m][j];
      Bl[i][j] = t;
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t = 0;
      for (int m = 0; m < 3; ++m) t += gi[i][m] * Bl[m][j];
      Bul[i][j] = t;
    }
  /* S_ij += (2 / alpha)(K_ir B_j^r + K_jr B_i^r - K_ij tr B) */
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double t = -s->K[i][j] * trB;
      for (int rr = 0; rr < 3; ++rr) t += s->K[i][rr] * s->B[j][rr] + s->K[j][rr] * s->B[i][rr];
      r->S_ij[i][j] += (2 / a) * t;
      r->S_K[i][j] = a * r->S_ij[i][j];
    }
  /* Omega_k += 2 (B_k^r - delta_k^r tr B) V_r + 2 (D_rk^s - delta^s_k D^j_jr) B^r_s */
  for (int k = 0; k < 3; ++k) {
    double t = 0;
    for (int rr = 0; rr < 3; ++rr) t += (s->B[k][rr] - trB * kdelta(k, rr)) * s->V[rr];
    for (int rr = 0; rr < 3; ++rr)
      for (int ss = 0; ss < 3; ++ss)
        t += (Dl2u[rr][k][ss] - kdelta(ss, k) * Dtr2[rr]) * Bul[rr][ss];
    r->S_V[k] += 2 * t;
  }
  /* V flux (reading R15): B^r_k - B_k^r along r */
  for (int k = 0; k < 3; ++k)
    for (int rr = 0; rr < 3; ++rr) r->VB[k][rr] = Bul[rr][k] - s->B[k][rr];

  /* Lapse (Eq. alfan): alpha (beta^r A_r - alpha Q); metric:
   * 2 beta^r D_rij - 2 alpha (K_ij - s_ij) with s_ij = 0 (B = 0). */
  double Qg = 0;
  if (slicing == 1) Qg = trK;
  else if (slicing == 2) Qg = trK / a;
  double bA = 0;
  for (int rr = 0; rr < 3; ++rr) bA += s->beta[rr] * s->A[rr];
  r->Qg = Qg;
  r->S_alpha = a * bA - a * a * Qg;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double bD = 0;
      for (int rr = 0; rr < 3; ++rr) bD += s->beta[rr] * s->D[rr][i][j];
      r->S_g[i][j] = 2 * bD - 2 * a * s->K[i][j] + 2 * (Bl[i][j] + Bl[j][i]);
    }
}

/* Exported pointwise evaluation for the tests: inputs alpha, gamma[6],
 * K[6], V[3], A[3], D[3][6] (stored pairs); outputs lam[3][6] (lambda^k_ij),
 * Sij[6] (S_ij without alpha), Omega[3], and the lapse source. */
void orc_bm_point(double alpha, const double* g6, const double* K6, const double* V3,
                  const double* A3, const double* D18, int slicing, double rho, double P,
                  double* lam18, double* S6, double* Om3, double* S_alpha) {
  bm_state s;
  bm_rhs r;
  s.alpha = alpha;
  memset(s.beta, 0, sizeof(s.beta));
  memset(s.B, 0, sizeof(s.B));
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      s.g[i][j] = g6[pair_of(i, j)];
      s.K[i][j] = K6[pair_of(i, j)];
      for (int k = 0; k < 3; ++k) s.D[k][i][j] = D18[6 * k + pair_of(i, j)];
    }
  for (int k = 0; k < 3; ++k) {
    s.V[k] = V3[k];
    s.A[k] = A3[k];
  }
  bm_point(&s, slicing, rho, P, &r);
  for (int k = 0; k < 3; ++k)
    for (int p = 0; p < 6; ++p) lam18[6 * k + p] = r.lam[k][PAIR_I[p]][PAIR_J[p]];
  for (int p = 0; p < 6; ++p) S6[p] = r.S_ij[PAIR_I[p]][PAIR_J[p]];
  for (int k = 0; k < 3; ++k) Om3[k] = r.S_V[k];
  *S_alpha = r.S_alpha;
}

/* ------------------------------------------------------------------------ */
/* Lattice helpers                                                           */
/* ------------------------------------------------------------------------ */

static int64_t wrap(int64_t i, int64_t n) {
  i %= n;
  return i < 0 ? i + n : i;
}

static int64_t cell_index(const orc_params* p, int64_t x, int64_t y, int64_t z) {
  return wrap(x, p->nx) + p->nx * (wrap(y, p->ny) + p->ny * wrap(z, p->nz));
}

static void cell_coords(const orc_params* p, int64_t c, int64_t* x, int64_t* y, int64_t* z) {
  *x = c % p->nx;
  *y = (c / p->nx) % p->ny;
  *z = c / (p->nx * p->ny);
}

static int check_params(const orc_params* p, vset_t* vs) {
  if (get_vset(p->vset, vs)) return -1;
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return -1;
  if (p->vset == 1 && (p->ny != 1 || p->nz != 1)) return -1;
  if (p->vset == 2 && p->nz != 1) return -1;
  if (!(p->tau > 0.5) || !(p->dx > 0) || !(p->dt > 0)) return -1;
  if (p->fluid_on && (!(p->t > 0) || !(p->fluid_t0 > 0))) return -1;
  if (p->deriv_mode < 0 || p->deriv_mode > 2) return -1;
  return 0;
}

/* Zeroth moment sum_l f_{F,l} at one cell (Sec. LBM, "macroscopic fields"),
 * summed in ascending velocity index. */
static double moment0(const vset_t* vs, int64_t cells, const double* f, int F, int64_t c) {
  double t = 0;
  for (int l = 0; l < vs->Q; ++l) t += f[((int64_t)F * vs->Q + l) * cells + c];
  return t;
}

/* Reading R4: A_k and D_kij at cell (x,y,z) from a field source `rho`
 * laid out [16][cells] (only alpha and gamma are used). */
static void derivatives(const orc_params* p, const double* rho, int64_t cells,
                        int64_t x, int64_t y, int64_t z, double A[3], double D[3][3][3]) {
  for (int k = 0; k < 3; ++k) {
    int64_t dxp = (k == 0), dyp = (k == 1), dzp = (k == 2);
    int64_t cp = cell_index(p, x + dxp, y + dyp, z + dzp);
    int64_t cm = cell_index(p, x - dxp, y - dyp, z - dzp);
    A[k] = (log(rho[F_ALPHA * cells + cp]) - log(rho[F_ALPHA * cells + cm])) / (2 * p->dx);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        int q = pair_of(i, j);
        D[k][i][j] = (rho[(F_G + q) * cells + cp] - rho[(F_G + q) * cells + cm]) / (4 * p->dx);
      }
  }
}

/* Fluid density and pressure at the time of the state a call reads. */
static void matter_now(const orc_params* p, double* rho, double* P) {
  *rho = 0;
  *P = 0;
  if (!p->fluid_on) return;
  const double q = p->fluid_t0 / p->t;
  *rho = p->fluid_rho0 * q * q;
  *P = p->fluid_w * *rho;
}

/* Shift at a cell: beta^i = the constant part plus the field's value, and
 * B_k^i = d_k beta^i / 2 by central differences of the field (reading R15;
 * zero without a field). */
static void shift_state(const orc_params* p, int64_t x, int64_t y, int64_t z, bm_state* s) {
  const int64_t cells = p->nx * p->ny * p->nz;
  for (int i = 0; i < 3; ++i) {
    s->beta[i] = p->beta[i];
    for (int k = 0; k < 3; ++k) s->B[k][i] = 0;
  }
  if (!p->beta_field) return;
  const int64_t c = cell_index(p, x, y, z);
  for (int i = 0; i < 3; ++i) s->beta[i] += p->beta_field[i * cells + c];
  for (int k = 0; k < 3; ++k) {
    const int64_t cp = cell_index(p, x + (k == 0), y + (k == 1), z + (k == 2));
    const int64_t cm = cell_index(p, x - (k == 0), y - (k == 1), z - (k == 2));
    for (int i = 0; i < 3; ++i)
      s->B[k][i] = (p->beta_field[i * cells + cp] - p->beta_field[i * cells + cm]) / (4 * p->dx);
  }
}

/* Unpacks the 16 stored values into a bm_state (derivatives and shift added
 * apart). */
static void unpack_fields(const double v[ORC_NF], bm_state* s) {
  s->alpha = v[F_ALPHA];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      s->g[i][j] = v[F_G + pair_of(i, j)];
      s->K[i][j] = v[F_K + pair_of(i, j)];
    }
  for (int k = 0; k < 3; ++k) s->V[k] = v[F_V + k];
}

/* The 16 macroscopic sources S_F in storage order. */
static void pack_sources(const bm_rhs* r, double S[ORC_NF]) {
  S[F_ALPHA] = r->S_alpha;
  for (int q = 0; q < 6; ++q) {
    S[F_G + q] = r->S_g[PAIR_I[q]][PAIR_J[q]];
    S[F_K + q] = r->S_K[PAIR_I[q]][PAIR_J[q]];
  }
  for (int k = 0; k < 3; ++k) S[F_V + k] = r->S_V[k];
}

/* Macroscopic flux of every field along each axis, read off the
 * equilibria's first moments: -beta^k K_ij + alpha lambda^k_ij for K_ij,
 * -beta^k V_i + B^k_i - B_i^k for V_i, zero for alpha and gamma_ij (their
 * shift terms are sources). s holds the fields the flux is taken at. */
static void pack_fluxes(const bm_rhs* r, const bm_state* s, double Fl[ORC_NF][3]) {
  for (int F = 0; F < ORC_NF; ++F)
    for (int k = 0; k < 3; ++k) Fl[F][k] = 0;
  for (int q = 0; q < 6; ++q)
    for (int k = 0; k < 3; ++k)
      Fl[F_K + q][k] = s->alpha * r->lam[k][PAIR_I[q]][PAIR_J[q]] -
                       s->beta[k] * s->K[PAIR_I[q]][PAIR_J[q]];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) Fl[F_V + i][k] = -s->beta[k] * s->V[i] + r->VB[i][k];
}

/* Steps 1-5 at one cell: given the uncorrected moments rho~ of all cells
 * (`mom`, [16][cells]) and the fields the derivatives are taken from
 * (`dsrc`: rho~ itself under R5, the previous step's corrected fields under
 * R17; only alpha and gamma, planes 0..6, are read), returns rho~ at this
 * cell, the sources S~, the corrected rho and the fluxes at rho. */
static void cell_macro(const orc_params* p, const double* mom, const double* dsrc, int64_t cells,
                       int64_t c, double rt[ORC_NF], double S[ORC_NF], double rho[ORC_NF],
                       double Fl[ORC_NF][3]) {
  double mrho, mP;
  matter_now(p, &mrho, &mP);
  int64_t x, y, z;
  cell_coords(p, c, &x, &y, &z);
  for (int F = 0; F < ORC_NF; ++F) rt[F] = mom[F * cells + c];
  bm_state s;
  bm_rhs r;
  derivatives(p, dsrc, cells, x, y, z, s.A, s.D);
  shift_state(p, x, y, z, &s);
  unpack_fields(rt, &s);
  bm_point(&s, p->slicing, mrho, mP, &r);
  pack_sources(&r, S);
  if (!p->sources_on)
    for (int F = 0; F < ORC_NF; ++F) S[F] = 0;
  /* rho = sum_l f + dt S / 2 (Sec. LBM, macroscopic variables). */
  for (int F = 0; F < ORC_NF; ++F) rho[F] = rt[F] + 0.5 * p->dt * S[F];
  /* Flux at the corrected moments with the same derivatives (R5). */
  unpack_fields(rho, &s);
  bm_point(&s, p->slicing, mrho, mP, &r);
  pack_fluxes(&r, &s, Fl);
}

/* Reading R18 at one cell: `rhos` ([16][cells]) holds the fixed point
 * rho = rho~ + dt S(rho)/2 of every cell. The sources are evaluated at it,
 * with A and D from its alpha and gamma; the corrected moments follow from
 * the moment rule with those sources, and the fluxes are taken at them. */
static void cell_macro_fixed(const orc_params* p, const double* mom, const double* rhos,
                             int64_t cells, int64_t c, double rt[ORC_NF], double S[ORC_NF],
                             double rho[ORC_NF], double Fl[ORC_NF][3]) {
  double mrho, mP;
  matter_now(p, &mrho, &mP);
  int64_t x, y, z;
  cell_coords(p, c, &x, &y, &z);
  double v[ORC_NF];
  for (int F = 0; F < ORC_NF; ++F) {
    rt[F] = mom[F * cells + c];
    v[F] = rhos[F * cells + c];
  }
  bm_state s;
  bm_rhs r;
  derivatives(p, rhos, cells, x, y, z, s.A, s.D);
  shift_state(p, x, y, z, &s);
  unpack_fields(v, &s);
  bm_point(&s, p->slicing, mrho, mP, &r);
  pack_sources(&r, S);
  if (!p->sources_on)
    for (int F = 0; F < ORC_NF; ++F) S[F] = 0;
  for (int F = 0; F < ORC_NF; ++F) rho[F] = rt[F] + 0.5 * p->dt * S[F];
  unpack_fields(rho, &s);
  bm_point(&s, p->slicing, mrho, mP, &r);
  pack_fluxes(&r, &s, Fl);
}

/* Reading R18 over the lattice: iterates rho <- rho~ + dt S(rho)/2 from
 * rho = rho~, A and D from the iterate, until no value changes by more than
 * 1e-15 of max(1, |rho|). out: [16][cells]. Returns -3 if 200 iterations do
 * not get there, -2 on allocation failure. */
static int fixed_point(const orc_params* p, const double* mom, int64_t cells, double* out) {
  double* nxt = (double*)malloc(sizeof(double) * ORC_NF * cells);
  if (!nxt) return -2;
  memcpy(out, mom, sizeof(double) * ORC_NF * cells);
  int rc = -3;
  for (int it = 0; it < 200; ++it) {
    double change = 0;
#pragma omp parallel for schedule(static) reduction(max : change)
    for (int64_t c = 0; c < cells; ++c) {
      double rt[ORC_NF], S[ORC_NF], rho[ORC_NF], Fl[ORC_NF][3];
      cell_macro_fixed(p, mom, out, cells, c, rt, S, rho, Fl);
      for (int F = 0; F < ORC_NF; ++F) {
        const double d = fabs(rho[F] - out[F * cells + c]) / fmax(1.0, fabs(rho[F]));
        if (d > change) change = d;
        nxt[F * cells + c] = rho[F];
      }
    }
    memcpy(out, nxt, sizeof(double) * ORC_NF * cells);
    if (!(change == change)) break; /* NaN */
    if (change <= 1e-15) {
      rc = 0;
      break;
    }
  }
  free(nxt);
  return rc;
}

/* Equilibrium (Eqs. alfa .. ekst): w_l [rho + c_l . Flux / c_s^2]. */
static double feq(const vset_t* vs, int l, double rho, const double Fl[3]) {
  double cf = 0;
  for (int k = 0; k < 3; ++k) cf += vs->c[l][k] * Fl[k];
  return vs->w[l] * (rho + cf / CS2);
}

/* ------------------------------------------------------------------------ */
/* Exported: initialisation, one step, moments, sampled step, constraints    */
/* ------------------------------------------------------------------------ */

static void all_moments(const vset_t* vs, int64_t cells, const double* f, double* mom) {
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < cells; ++c)
    for (int F = 0; F < ORC_NF; ++F) mom[F * cells + c] = moment0(vs, cells, f, F, c);
}

/* Reading R6. fields: [16][cells] initial macroscopic values. */
int orc_init(const orc_params* p, const double* fields, double* f_out) {
  vset_t vs;
  if (check_params(p, &vs)) return -1;
  double mrho, mP;
  matter_now(p, &mrho, &mP);
  const int64_t cells = p->nx * p->ny * p->nz;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t c = 0; c < cells; ++c) {
    int64_t x, y, z;
    cell_coords(p, c, &x, &y, &z);
    double v[ORC_NF], S[ORC_NF], Fl[ORC_NF][3];
    for (int F = 0; F < ORC_NF; ++F) v[F] = fields[F * cells + c];
    bm_state s;
    bm_rhs r;
    derivatives(p, fields, cells, x, y, z, s.A, s.D);
    shift_state(p, x, y, z, &s);
    unpack_fields(v, &s);
    bm_point(&s, p->slicing, mrho, mP, &r);
    pack_sources(&r, S);
    if (!p->sources_on)
      for (int F = 0; F < ORC_NF; ++F) S[F] = 0;
    pack_fluxes(&r, &s, Fl);
    for (int F = 0; F < ORC_NF; ++F)
      for (int l = 0; l < vs.Q; ++l) {
        double val = feq(&vs, l, v[F], Fl[F]) - 0.5 * p->dt * vs.w[l] * S[F];
        f_out[((int64_t)F * vs.Q + l) * cells + c] = val;
        if (!isfinite(val)) bad = 1;
      }
  }
  return bad ? -4 : 0;
}

/* Steps 1-5 at one cell in the context's derivative mode: `dsrc` is the
 * previous step's corrected fields under R17, the fixed point under R18,
 * and unused under R5. */
static void macro_mode(const orc_params* p, const double* mom, const double* dsrc, int64_t cells,
                       int64_t c, double rt[ORC_NF], double S[ORC_NF], double rho[ORC_NF],
                       double Fl[ORC_NF][3]) {
  if (p->deriv_mode == 2)
    cell_macro_fixed(p, mom, dsrc, cells, c, rt, S, rho, Fl);
  else
    cell_macro(p, mom, p->deriv_mode == 1 ? dsrc : mom, cells, c, rt, S, rho, Fl);
}

/* Post-collision values f*_{F,l} at one cell (Eq. numlb right-hand side with
 * the source distributions, Eqs. alfa .. ekstsor). Also returns the
 * corrected moments (rho_out, which R17 hands to the next step). */
static void collide_cell(const orc_params* p, const vset_t* vs, const double* f,
                         const double* mom, const double* dsrc, int64_t cells, int64_t c,
                         double fstar[ORC_NF][ORC_QMAX], double rho_out[ORC_NF]) {
  double rt[ORC_NF], S[ORC_NF], rho[ORC_NF], Fl[ORC_NF][3];
  macro_mode(p, mom, dsrc, cells, c, rt, S, rho, Fl);
  for (int F = 0; F < ORC_NF; ++F) rho_out[F] = rho[F];
  const double src_fac = 1.0 - 1.0 / (2.0 * p->tau);
  for (int F = 0; F < ORC_NF; ++F)
    for (int l = 0; l < vs->Q; ++l) {
      double fl = f[((int64_t)F * vs->Q + l) * cells + c];
      double fe = feq(vs, l, rho[F], Fl[F]);
      double Sl = vs->w[l] * src_fac * S[F];
      fstar[F][l] = fl - (fl - fe) / p->tau + p->dt * Sl;
    }
}

/* The derivative source of one step: NULL under R5, prev under R17 (which
 * must then be given), the lattice's fixed point under R18 (allocated here;
 * *owned tells the caller to free it). */
static int mode_source(const orc_params* p, const double* mom, const double* prev,
                       int64_t cells, const double** dsrc, double** owned) {
  *dsrc = NULL;
  *owned = NULL;
  if (p->deriv_mode == 1) {
    if (!prev) return -1;
    *dsrc = prev;
  } else if (p->deriv_mode == 2) {
    double* fx = (double*)malloc(sizeof(double) * ORC_NF * cells);
    if (!fx) return -2;
    int rc = fixed_point(p, mom, cells, fx);
    if (rc) {
      free(fx);
      return rc;
    }
    *dsrc = fx;
    *owned = fx;
  }
  return 0;
}

/* One full step f(n) -> f(n+1): collide, then stream to x + c_l (periodic).
 * prev_in / prev_out ([7][cells]: corrected alpha and gamma_ij) carry R17's
 * lagged fields; both are ignored (and may be NULL) in the other modes.
 * Returns -4 if any output is not finite. */
int orc_step_lag(const orc_params* p, const double* f_in, const double* prev_in, double* f_out,
                 double* prev_out) {
  vset_t vs;
  if (check_params(p, &vs)) return -1;
  if (p->deriv_mode == 1 && (!prev_in || !prev_out)) return -1;
  const int64_t cells = p->nx * p->ny * p->nz;
  double* mom = (double*)malloc(sizeof(double) * ORC_NF * cells);
  if (!mom) return -2;
  all_moments(&vs, cells, f_in, mom);
  const double* dsrc;
  double* owned;
  int rc = mode_source(p, mom, prev_in, cells, &dsrc, &owned);
  if (rc) {
    free(mom);
    return rc;
  }
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t c = 0; c < cells; ++c) {
    double fstar[ORC_NF][ORC_QMAX], rho[ORC_NF];
    collide_cell(p, &vs, f_in, mom, dsrc, cells, c, fstar, rho);
    if (p->deriv_mode == 1)
      for (int F = 0; F < 7; ++F) prev_out[F * cells + c] = rho[F];
    int64_t x, y, z;
    cell_coords(p, c, &x, &y, &z);
    for (int l = 0; l < vs.Q; ++l) {
      int64_t d = cell_index(p, x + vs.c[l][0], y + vs.c[l][1], z + vs.c[l][2]);
      for (int F = 0; F < ORC_NF; ++F) {
        f_out[((int64_t)F * vs.Q + l) * cells + d] = fstar[F][l];
        if (!isfinite(fstar[F][l])) bad = 1;
      }
    }
  }
  free(owned);
  free(mom);
  return bad ? -4 : 0;
}

/* One step under R5 or R18 (no lagged state). */
int orc_step(const orc_params* p, const double* f_in, double* f_out) {
  if (p->deriv_mode == 1) return -1;
  return orc_step_lag(p, f_in, NULL, f_out, NULL);
}

/* n steps, alternating two caller-owned buffers; the result ends in f_io.
 * The state's time advances by dt per step from p->t. */
int orc_run(const orc_params* p, double* f_io, double* scratch, int64_t n) {
  orc_params q = *p;
  for (int64_t i = 0; i < n; ++i) {
    int rc = orc_step(&q, f_io, scratch);
    q.t += q.dt;
    if (rc) return rc;
    vset_t vs;
    get_vset(p->vset, &vs);
    memcpy(f_io, scratch, sizeof(double) * ORC_NF * vs.Q * p->nx * p->ny * p->nz);
  }
  return 0;
}

/* Corrected macroscopic fields rho = sum f + dt S~/2 for every cell,
 * out: [16][cells], in the context's derivative mode (R17 reads the lagged
 * fields prev [7][cells]; the other modes ignore it). */
int orc_moments_lag(const orc_params* p, const double* f, const double* prev, double* out) {
  vset_t vs;
  if (check_params(p, &vs)) return -1;
  const int64_t cells = p->nx * p->ny * p->nz;
  double* mom = (double*)malloc(sizeof(double) * ORC_NF * cells);
  if (!mom) return -2;
  all_moments(&vs, cells, f, mom);
  const double* dsrc;
  double* owned;
  int rc = mode_source(p, mom, prev, cells, &dsrc, &owned);
  if (rc) {
    free(mom);
    return rc;
  }
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < cells; ++c) {
    double rt[ORC_NF], S[ORC_NF], rho[ORC_NF], Fl[ORC_NF][3];
    macro_mode(p, mom, dsrc, cells, c, rt, S, rho, Fl);
    for (int F = 0; F < ORC_NF; ++F) out[F * cells + c] = rho[F];
  }
  free(owned);
  free(mom);
  return 0;
}

int orc_moments(const orc_params* p, const double* f, double* out) {
  if (p->deriv_mode == 1) return -1;
  return orc_moments_lag(p, f, NULL, out);
}

/* One step evaluated only at the listed destination cells: out[n][16][Q] is
 * f_{F,l}(y, n+1) = f*_{F,l}(y - c_l, n). Moments are formed on the fly, so
 * this works at any lattice size for a handful of cells. */
int orc_step_cells(const orc_params* p, const double* f_in, int64_t n, const int64_t* cells_idx,
                   double* out) {
  vset_t vs;
  if (check_params(p, &vs)) return -1;
  if (p->deriv_mode != 0) return -1; /* reading R5 only */
  double mrho, mP;
  matter_now(p, &mrho, &mP);
  const int64_t cells = p->nx * p->ny * p->nz;
  int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(| : bad)
  for (int64_t i = 0; i < n; ++i) {
    int64_t y0, y1, y2;
    cell_coords(p, cells_idx[i], &y0, &y1, &y2);
    for (int l = 0; l < vs.Q; ++l) {
      int64_t sx = y0 - vs.c[l][0], sy = y1 - vs.c[l][1], sz = y2 - vs.c[l][2];
      /* Local moment table for the source cell and its six face neighbours;
       * other entries are never read by derivatives(). */
      int64_t nb[7];
      nb[0] = cell_index(p, sx, sy, sz);
      nb[1] = cell_index(p, sx + 1, sy, sz);
      nb[2] = cell_index(p, sx - 1, sy, sz);
      nb[3] = cell_index(p, sx, sy + 1, sz);
      nb[4] = cell_index(p, sx, sy - 1, sz);
      nb[5] = cell_index(p, sx, sy, sz + 1);
      nb[6] = cell_index(p, sx, sy, sz - 1);
      double rt[ORC_NF], S[ORC_NF], rho[ORC_NF], Fl[ORC_NF][3];
      /* Same arithmetic as cell_macro, reading moments computed here. */
      for (int F = 0; F < ORC_NF; ++F) rt[F] = moment0(&vs, cells, f_in, F, nb[0]);
      bm_state s;
      bm_rhs r;
      for (int k = 0; k < 3; ++k) {
        int64_t cp = nb[1 + 2 * k], cm = nb[2 + 2 * k];
        s.A[k] = (log(moment0(&vs, cells, f_in, F_ALPHA, cp)) -
                  log(moment0(&vs, cells, f_in, F_ALPHA, cm))) / (2 * p->dx);
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            int q = pair_of(a, b);
            s.D[k][a][b] = (moment0(&vs, cells, f_in, F_G + q, cp) -
                            moment0(&vs, cells, f_in, F_G + q, cm)) / (4 * p->dx);
          }
      }
      shift_state(p, sx, sy, sz, &s);
      unpack_fields(rt, &s);
      bm_point(&s, p->slicing, mrho, mP, &r);
      pack_sources(&r, S);
      if (!p->sources_on)
        for (int F = 0; F < ORC_NF; ++F) S[F] = 0;
      for (int F = 0; F < ORC_NF; ++F) rho[F] = rt[F] + 0.5 * p->dt * S[F];
      unpack_fields(rho, &s);
      bm_point(&s, p->slicing, mrho, mP, &r);
      pack_fluxes(&r, &s, Fl);
      const double src_fac = 1.0 - 1.0 / (2.0 * p->tau);
      for (int F = 0; F < ORC_NF; ++F) {
        double fl = f_in[((int64_t)F * vs.Q + l) * cells + nb[0]];
        double fe = feq(&vs, l, rho[F], Fl[F]);
        double Sl = vs.w[l] * src_fac * S[F];
        double v = fl - (fl - fe) / p->tau + p->dt * Sl;
        out[(i * ORC_NF + F) * vs.Q + l] = v;
        if (!isfinite(v)) bad = 1;
      }
    }
  }
  return bad ? -4 : 0;
}

/* ------------------------------------------------------------------------ */
/* Constraint monitoring (Sec. "3+1 ADM formalism": Hamiltonian and          */
/* momentum constraints; Sec. "Bona-Masso formulation": V_k definition)     */
/* ------------------------------------------------------------------------ */

/* Christoffel symbols Gamma^k_ij at a cell from central differences of the
 * corrected metric `rho` ([16][cells]). */
static void christoffel_at(const orc_params* p, const double* rho, int64_t cells, int64_t x,
                           int64_t y, int64_t z, double Gam[3][3][3], double gi[3][3],
                           double D[3][3][3]) {
  double A[3], g[3][3];
  derivatives(p, rho, cells, x, y, z, A, D);
  int64_t c = cell_index(p, x, y, z);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) g[i][j] = rho[(F_G + pair_of(i, j)) * cells + c];
  inverse3(g, gi);
  for (int k = 0; k < 3; ++k)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double t = 0;
        for (int m = 0; m < 3; ++m) t += gi[k][m] * (D[i][j][m] + D[j][i][m] - D[m][i][j]);
        Gam[k][i][j] = t;
      }
}

static double trK_at(const double* rho, int64_t cells, int64_t c) {
  double g[3][3], gi[3][3], t = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) g[i][j] = rho[(F_G + pair_of(i, j)) * cells + c];
  inverse3(g, gi);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) t += gi[i][j] * rho[(F_K + pair_of(i, j)) * cells + c];
  return t;
}

/* Per-cell constraint values at the corrected fields rho ([16][cells]):
 *   H   = R - K_ij K^ij + (tr K)^2 (vacuum Hamiltonian constraint), with
 *         R_ij = d_k Gamma^k_ij - d_j Gamma^k_ik + Gamma^k_km Gamma^m_ij
 *                - Gamma^k_jm Gamma^m_ik (the Ricci definition of the paper
 *         applied to the three-metric) and central differences of Gamma;
 *   M_i = D_j K^j_i - d_i tr K (vacuum momentum constraint);
 *   C_k = V_k - (D_kr^r - D^r_rk) (the definition of V_k).
 * out_cell: [cells][7] = H, M_x, M_y, M_z, C_x, C_y, C_z. */
int orc_constraint_fields(const orc_params* p, const double* rho, double* out_cell) {
  vset_t vs;
  if (check_params(p, &vs)) return -1;
  const int64_t cells = p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < cells; ++c) {
    int64_t x, y, z;
    cell_coords(p, c, &x, &y, &z);
    double Gam[3][3][3], gi[3][3], D[3][3][3];
    christoffel_at(p, rho, cells, x, y, z, Gam, gi, D);
    /* d_m Gamma^k_ij by central differences of neighbour Christoffels. */
    double dGam[3][3][3][3]; /* [m][k][i][j] */
    for (int m = 0; m < 3; ++m) {
      double Gp[3][3][3], Gm[3][3][3], tmp_gi[3][3], tmp_D[3][3][3];
      int dxp = (m == 0), dyp = (m == 1), dzp = (m == 2);
      christoffel_at(p, rho, cells, x + dxp, y + dyp, z + dzp, Gp, tmp_gi, tmp_D);
      christoffel_at(p, rho, cells, x - dxp, y - dyp, z - dzp, Gm, tmp_gi, tmp_D);
      for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j) dGam[m][k][i][j] = (Gp[k][i][j] - Gm[k][i][j]) / (2 * p->dx);
    }
    double Ric[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double t = 0;
        for (int k = 0; k < 3; ++k) {
          t += dGam[k][k][i][j] - dGam[j][k][i][k];
          for (int m = 0; m < 3; ++m) t += Gam[k][k][m] * Gam[m][i][j] - Gam[k][j][m] * Gam[m][i][k];
        }
        Ric[i][j] = t;
      }
    double R = 0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) R += gi[i][j] * Ric[i][j];
    double K[3][3], Kmix[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) K[i][j] = rho[(F_K + pair_of(i, j)) * cells + c];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double t = 0;
        for (int m = 0; m < 3; ++m) t += gi[i][m] * K[m][j];
        Kmix[i][j] = t;
      }
    double trK = 0, trK2 = 0;
    for (int i = 0; i < 3; ++i) trK += Kmix[i][i];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) trK2 += Kmix[i][j] * Kmix[j][i];
    out_cell[c * 7 + 0] = R - trK2 + trK * trK;

    /* Momentum constraint: g^{jk} (d_j K_ki - Gamma^m_jk K_mi - Gamma^m_ji K_km) - d_i trK. */
    double dK[3][3][3]; /* [m][i][j] = d_m K_ij */
    double dtrK[3];
    for (int m = 0; m < 3; ++m) {
      int dxp = (m == 0), dyp = (m == 1), dzp = (m == 2);
      int64_t cp = cell_index(p, x + dxp, y + dyp, z + dzp);
      int64_t cm = cell_index(p, x - dxp, y - dyp, z - dzp);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          dK[m][i][j] = (rho[(F_K + pair_of(i, j)) * cells + cp] -
                         rho[(F_K + pair_of(i, j)) * cells + cm]) / (2 * p->dx);
      dtrK[m] = (trK_at(rho, cells, cp) - trK_at(rho, cells, cm)) / (2 * p->dx);
    }
    for (int i = 0; i < 3; ++i) {
      double t = 0;
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k) {
          double cov = dK[j][k][i];
          for (int m = 0; m < 3; ++m) cov -= Gam[m][j][k] * K[m][i] + Gam[m][j][i] * K[k][m];
          t += gi[j][k] * cov;
        }
      out_cell[c * 7 + 1 + i] = t - dtrK[i];
    }
    /* V constraint. */
    for (int k = 0; k < 3; ++k) {
      double t1 = 0, t2 = 0;
      for (int rr = 0; rr < 3; ++rr)
        for (int m = 0; m < 3; ++m) {
          t1 += gi[rr][m] * D[k][rr][m];
          t2 += gi[rr][m] * D[m][rr][k];
        }
      out_cell[c * 7 + 4 + k] = rho[(F_V + k) * cells + c] - (t1 - t2);
    }
  }
  return 0;
}

/* Monitoring summary from the distributions f:
 * out[22] = H_L2, H_inf, M_L2, M_inf, C_L2, C_inf, sum_x rho~_F (F = 0..15),
 * where X_L2 = sqrt(mean over cells of the squared (vector) norm) and
 * X_inf = max over cells and components of |X|. */
int orc_constraints_lag(const orc_params* p, const double* f, const double* prev, double* out) {
  vset_t vs;
  if (check_params(p, &vs)) return -1;
  const int64_t cells = p->nx * p->ny * p->nz;
  double* rho = (double*)malloc(sizeof(double) * ORC_NF * cells);
  double* cf = (double*)malloc(sizeof(double) * 7 * cells);
  if (!rho || !cf) {
    free(rho);
    free(cf);
    return -2;
  }
  const int rc = orc_moments_lag(p, f, prev, rho);
  if (rc) {
    free(rho);
    free(cf);
    return rc;
  }
  orc_constraint_fields(p, rho, cf);
  double h2 = 0, hi = 0, m2 = 0, mi = 0, c2 = 0, ci = 0;
  for (int64_t c = 0; c < cells; ++c) {
    double h = cf[c * 7];
    h2 += h * h;
    if (fabs(h) > hi) hi = fabs(h);
    for (int k = 0; k < 3; ++k) {
      double m = cf[c * 7 + 1 + k], v = cf[c * 7 + 4 + k];
      m2 += m * m;
      c2 += v * v;
      if (fabs(m) > mi) mi = fabs(m);
      if (fabs(v) > ci) ci = fabs(v);
    }
  }
  out[0] = sqrt(h2 / cells);
  out[1] = hi;
  out[2] = sqrt(m2 / cells);
  out[3] = mi;
  out[4] = sqrt(c2 / cells);
  out[5] = ci;
  for (int F = 0; F < ORC_NF; ++F) {
    double t = 0;
    for (int64_t c = 0; c < cells; ++c) t += moment0(&vs, cells, f, F, c);
    out[6 + F] = t;
  }
  free(rho);
  free(cf);
  return 0;
}

int orc_constraints(const orc_params* p, const double* f, double* out) {
  if (p->deriv_mode == 1) return -1;
  return orc_constraints_lag(p, f, NULL, out);
}

/* ------------------------------------------------------------------------ */
/* Independently evolved A_k and D_kij (reading R16; Sec. "Bona-Masso        */
/* evolution equations", the remark after the first-order derivatives)       */
/* ------------------------------------------------------------------------ */
/* Fields 0..15 as above, then A_x A_y A_z (16..18) and D_kij at
 * 19 + 6 k + pair(i, j) (k = x, y, z; pairs in the order xx xy xz yy yz zz). */
#define ORC_NF_AD 37
enum { F_A = 16, F_D = 19 };

static int check_params_ad(const orc_params* p, vset_t* vs) {
  if (check_params(p, vs)) return -1;
  if (p->beta[0] != 0 || p->beta[1] != 0 || p->beta[2] != 0 || p->beta_field) return -1;
  return 0;
}

/* The 37 moments as a bm_state: A and D are the cell's own values. */
static void ad_unpack(const double v[ORC_NF_AD], bm_state* s) {
  unpack_fields(v, s);
  memset(s->beta, 0, sizeof(s->beta));
  memset(s->B, 0, sizeof(s->B));
  for (int k = 0; k < 3; ++k) {
    s->A[k] = v[F_A + k];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) s->D[k][i][j] = v[F_D + 6 * k + pair_of(i, j)];
  }
}

/* Sources of the 37 fields at state v (zero for A and D) and, at the same
 * state, the fluxes: those of the 16 fields, alpha Q along k for A_k and
 * alpha K_ij along k for D_kij. */
static void ad_rhs(const orc_params* p, const double v[ORC_NF_AD], double S[ORC_NF_AD],
                   double Fl[ORC_NF_AD][3]) {
  double mrho, mP;
  matter_now(p, &mrho, &mP);
  bm_state s;
  bm_rhs r;
  ad_unpack(v, &s);
  bm_point(&s, p->slicing, mrho, mP, &r);
  if (S) {
    pack_sources(&r, S);
    for (int F = ORC_NF; F < ORC_NF_AD; ++F) S[F] = 0;
    if (!p->sources_on)
      for (int F = 0; F < ORC_NF_AD; ++F) S[F] = 0;
  }
  if (Fl) {
    double F16[ORC_NF][3];
    pack_fluxes(&r, &s, F16);
    for (int F = 0; F < ORC_NF; ++F)
      for (int m = 0; m < 3; ++m) Fl[F][m] = F16[F][m];
    for (int k = 0; k < 3; ++k)
      for (int m = 0; m < 3; ++m) {
        Fl[F_A + k][m] = (m == k) ? s.alpha * r.Qg : 0;
        for (int q = 0; q < 6; ++q)
          Fl[F_D + 6 * k + q][m] = (m == k) ? s.alpha * s.K[PAIR_I[q]][PAIR_J[q]] : 0;
      }
  }
}

static void ad_moments_all(const vset_t* vs, int64_t cells, const double* f, double* mom) {
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < cells; ++c)
    for (int F = 0; F < ORC_NF_AD; ++F) mom[F * cells + c] = moment0(vs, cells, f, F, c);
}

/* Initial distributions from 37 given fields ([37][cells]), reading R6. */
int orc_ad_init37(const orc_params* p, const double* fields, double* f_out) {
  vset_t vs;
  if (check_params_ad(p, &vs)) return -1;
  const int64_t cells = p->nx * p->ny * p->nz;
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t c = 0; c < cells; ++c) {
    double v[ORC_NF_AD], S[ORC_NF_AD], Fl[ORC_NF_AD][3];
    for (int F = 0; F < ORC_NF_AD; ++F) v[F] = fields[F * cells + c];
    ad_rhs(p, v, S, Fl);
    for (int F = 0; F < ORC_NF_AD; ++F)
      for (int l = 0; l < vs.Q; ++l) {
        double val = feq(&vs, l, v[F], Fl[F]) - 0.5 * p->dt * vs.w[l] * S[F];
        f_out[((int64_t)F * vs.Q + l) * cells + c] = val;
        if (!isfinite(val)) bad = 1;
      }
  }
  return bad ? -4 : 0;
}

/* Initial distributions from the 16 fields ([16][cells]): A and D start as
 * the central differences of reading R4. */
int orc_ad_init(const orc_params* p, const double* fields, double* f_out) {
  vset_t vs;
  if (check_params_ad(p, &vs)) return -1;
  const int64_t cells = p->nx * p->ny * p->nz;
  double* all = (double*)malloc(sizeof(double) * ORC_NF_AD * cells);
  if (!all) return -2;
  memcpy(all, fields, sizeof(double) * ORC_NF * cells);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < cells; ++c) {
    int64_t x, y, z;
    cell_coords(p, c, &x, &y, &z);
    double A[3], D[3][3][3];
    derivatives(p, fields, cells, x, y, z, A, D);
    for (int k = 0; k < 3; ++k) {
      all[(F_A + k) * cells + c] = A[k];
      for (int q = 0; q < 6; ++q) all[(F_D + 6 * k + q) * cells + c] = D[k][PAIR_I[q]][PAIR_J[q]];
    }
  }
  int rc = orc_ad_init37(p, all, f_out);
  free(all);
  return rc;
}

/* One step of the 37-field scheme: every quantity is local to the cell. */
int orc_ad_step(const orc_params* p, const double* f_in, double* f_out) {
  vset_t vs;
  if (check_params_ad(p, &vs)) return -1;
  const int64_t cells = p->nx * p->ny * p->nz;
  double* mom = (double*)malloc(sizeof(double) * ORC_NF_AD * cells);
  if (!mom) return -2;
  ad_moments_all(&vs, cells, f_in, mom);
  const double src_fac = 1.0 - 1.0 / (2.0 * p->tau);
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t c = 0; c < cells; ++c) {
    double rt[ORC_NF_AD], S[ORC_NF_AD], rho[ORC_NF_AD], Fl[ORC_NF_AD][3];
    for (int F = 0; F < ORC_NF_AD; ++F) rt[F] = mom[F * cells + c];
    ad_rhs(p, rt, S, NULL);
    for (int F = 0; F < ORC_NF_AD; ++F) rho[F] = rt[F] + 0.5 * p->dt * S[F];
    ad_rhs(p, rho, NULL, Fl);
    int64_t x, y, z;
    cell_coords(p, c, &x, &y, &z);
    for (int l = 0; l < vs.Q; ++l) {
      int64_t d = cell_index(p, x + vs.c[l][0], y + vs.c[l][1], z + vs.c[l][2]);
      for (int F = 0; F < ORC_NF_AD; ++F) {
        double fl = f_in[((int64_t)F * vs.Q + l) * cells + c];
        double fe = feq(&vs, l, rho[F], Fl[F]);
        double v = fl - (fl - fe) / p->tau + p->dt * vs.w[l] * src_fac * S[F];
        f_out[((int64_t)F * vs.Q + l) * cells + d] = v;
        if (!isfinite(v)) bad = 1;
      }
    }
  }
  free(mom);
  return bad ? -4 : 0;
}

int orc_ad_run(const orc_params* p, double* f_io, double* scratch, int64_t n) {
  orc_params q = *p;
  vset_t vs;
  if (check_params_ad(p, &vs)) return -1;
  for (int64_t i = 0; i < n; ++i) {
    int rc = orc_ad_step(&q, f_io, scratch);
    q.t += q.dt;
    if (rc) return rc;
    memcpy(f_io, scratch, sizeof(double) * ORC_NF_AD * vs.Q * p->nx * p->ny * p->nz);
  }
  return 0;
}

/* Corrected moments of the 37 fields ([37][cells]); A and D have no source,
 * so theirs are the plain sums. */
int orc_ad_moments(const orc_params* p, const double* f, double* out) {
  vset_t vs;
  if (check_params_ad(p, &vs)) return -1;
  const int64_t cells = p->nx * p->ny * p->nz;
  double* mom = (double*)malloc(sizeof(double) * ORC_NF_AD * cells);
  if (!mom) return -2;
  ad_moments_all(&vs, cells, f, mom);
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < cells; ++c) {
    double rt[ORC_NF_AD], S[ORC_NF_AD];
    for (int F = 0; F < ORC_NF_AD; ++F) rt[F] = mom[F * cells + c];
    ad_rhs(p, rt, S, NULL);
    for (int F = 0; F < ORC_NF_AD; ++F) out[F * cells + c] = rt[F] + 0.5 * p->dt * S[F];
  }
  free(mom);
  return 0;
}
