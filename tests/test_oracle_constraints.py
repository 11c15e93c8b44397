"""Pins of the oracle's constraint monitor (Sec. "3+1 ADM formalism":
Hamiltonian and momentum constraints in vacuum; Sec. "Bona-Masso
formulation": the definition of V_k) against closed forms.
"""
import math

import numpy as np
import pytest

from paper_1505_02037_gb300 import workloads as W


def _conformal(N, eps=0.05, eps2=0.03):
    """gamma = psi^4 delta with psi = 1 + eps sin(a) sin(b) + eps2 cos(c); the
    scalar curvature is R = -8 psi^-5 lap(psi) (textbook conformal identity)."""
    X, Y, Z = W.coords((N, N, N), 1 / N)
    a, b, c = 2 * math.pi * X + 0.3, 2 * math.pi * Y + 0.7, 2 * math.pi * Z
    psi = 1 + eps * np.sin(a) * np.sin(b) + eps2 * np.cos(c)
    lap = -8 * math.pi ** 2 * eps * np.sin(a) * np.sin(b) - 4 * math.pi ** 2 * eps2 * np.cos(c)
    dpsi = [2 * math.pi * eps * np.cos(a) * np.sin(b), 2 * math.pi * eps * np.sin(a) * np.cos(b),
            -2 * math.pi * eps2 * np.sin(c)]
    rho = W.flat((N, N, N))
    for q in (1, 4, 6):
        rho[q] = psi ** 4
    return rho, -8 * psi ** -5 * lap, np.array([-4 * d / psi for d in dpsi])


def test_ricci_scalar_of_conformally_flat_metric(oracle_mod):
    errs = []
    for N in (12, 24):
        rho, R, _ = _conformal(N)
        o = oracle_mod.Oracle(3, (N, N, N), 1.0, 1 / N)
        cf = o.constraint_fields(rho)
        errs.append(np.abs(cf[:, 0] - R.reshape(-1)).max() / np.abs(R).max())
    assert 3.5 < errs[0] / errs[1] < 4.5, errs
    assert errs[1] < 3e-2


def test_v_constraint_of_conformally_flat_metric(oracle_mod):
    """With V = 0 stored, C_k = -(D_kr^r - D^r_rk) = -4 d_k psi / psi."""
    errs = []
    for N in (12, 24):
        rho, _, C = _conformal(N)
        o = oracle_mod.Oracle(3, (N, N, N), 1.0, 1 / N)
        cf = o.constraint_fields(rho)
        errs.append(np.abs(cf[:, 4:7] - C.reshape(3, -1).T).max() / np.abs(C).max())
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def test_momentum_and_hamiltonian_with_flat_metric(oracle_mod):
    """gamma = delta (Christoffels vanish exactly): M_i = d_j K_ji - d_i trK and
    H = (trK)^2 - K_ij K_ij, for trigonometric K_ij."""
    errs = []
    for N in (12, 24):
        X, Y, Z = W.coords((N, N, N), 1 / N)
        t = 2 * math.pi
        K = np.zeros((3, 3) + X.shape)
        dK = np.zeros((3, 3, 3) + X.shape)  # [m, i, j] = d_m K_ij
        comps = {(0, 0): (0.3, (0, 1, 0)), (0, 1): (0.2, (1, 0, 1)), (0, 2): (0.1, (0, 1, 1)),
                 (1, 1): (-0.2, (1, 0, 0)), (1, 2): (0.15, (1, 1, 0)), (2, 2): (0.25, (0, 0, 1))}
        for (i, j), (amp, k) in comps.items():
            ph = t * (k[0] * X + k[1] * Y + k[2] * Z) + 0.1 * (i + 2 * j)
            K[i, j] = K[j, i] = amp * np.sin(ph)
            for m in range(3):
                dK[m, i, j] = dK[m, j, i] = amp * t * k[m] * np.cos(ph)
        rho = W.flat((N, N, N))
        for q, (i, j) in enumerate(W.PAIRS):
            rho[7 + q] = K[i, j]
        o = oracle_mod.Oracle(3, (N, N, N), 1.0, 1 / N)
        cf = o.constraint_fields(rho)
        trK = K[0, 0] + K[1, 1] + K[2, 2]
        H = trK ** 2 - np.einsum("ij...,ij...->...", K, K)
        np.testing.assert_allclose(cf[:, 0], H.reshape(-1), rtol=0, atol=1e-13)
        dtr = dK[:, 0, 0] + dK[:, 1, 1] + dK[:, 2, 2]
        M = np.einsum("jji...->i...", dK) - dtr
        errs.append(np.abs(cf[:, 1:4] - M.reshape(3, -1).T).max() / np.abs(M).max())
    assert 3.5 < errs[0] / errs[1] < 4.5, errs


def test_constraints_on_the_diagonal_gauge_wave(oracle_mod):
    """The gauge wave is flat space in other coordinates: H and C vanish to
    round-off even on the lattice, and M falls as dr^2."""
    norms = []
    for N in (16, 32):
        shape = (N, N, N)
        o = oracle_mod.Oracle(3, shape, 1.0, 1 / N)
        cf = o.constraint_fields(W.gauge_wave(shape, 1 / N, 0.1, direction="xyz"))
        norms.append(np.abs(cf).max(axis=0))
    assert norms[1][0] < 1e-11 and norms[1][4:].max() < 1e-13, norms
    assert np.all(norms[0][1:4] / norms[1][1:4] > 3.4), norms


def test_constraints_on_the_diagonal_linear_wave(oracle_mod):
    """The linear wave satisfies H and M to O(A^2) only; C falls as dr^2."""
    A = 1e-3
    norms = []
    for N in (16, 32):
        shape = (N, N, N)
        o = oracle_mod.Oracle(3, shape, 1.0, 1 / N)
        cf = o.constraint_fields(W.linear_wave(shape, 1 / N, A, direction="xyz"))
        norms.append(np.abs(cf).max(axis=0))
    k = 2 * math.pi * math.sqrt(3)
    assert norms[1][:4].max() < 10 * (k * A) ** 2, norms
    assert np.all(norms[0][4:] / norms[1][4:] > 3.5), norms


def test_summary_norms_and_sums(oracle_mod):
    """The 22-value summary is the L2 (root mean square of the vector norm) and
    L-infinity norms of H, M, C at the corrected moments, and the lattice sums
    of sum_l f for all 16 fields."""
    O = oracle_mod
    shape = (6, 5, 4)
    c, w = O.velocity_set(3)
    f = W.random_distributions(19, w, shape, seed=2)
    o = O.Oracle(3, shape, 1.2, 1 / 6)
    out = o.constraints(f)
    cf = o.constraint_fields(o.moments(f))
    assert out[0] == pytest.approx(math.sqrt(np.mean(cf[:, 0] ** 2)), rel=1e-12)
    assert out[1] == pytest.approx(np.abs(cf[:, 0]).max(), rel=1e-14)
    assert out[2] == pytest.approx(math.sqrt(np.mean(np.sum(cf[:, 1:4] ** 2, axis=1))), rel=1e-12)
    assert out[3] == pytest.approx(np.abs(cf[:, 1:4]).max(), rel=1e-14)
    assert out[4] == pytest.approx(math.sqrt(np.mean(np.sum(cf[:, 4:7] ** 2, axis=1))), rel=1e-12)
    assert out[5] == pytest.approx(np.abs(cf[:, 4:7]).max(), rel=1e-14)
    np.testing.assert_allclose(out[6:], f.sum(axis=(1, 2)), rtol=0,
                               atol=1e-15 * np.abs(f).sum(axis=(1, 2)).max())
