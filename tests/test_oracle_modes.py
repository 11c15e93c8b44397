"""Pins of the oracle's two other readings of the time level of A_k and D_kij
(the paper is silent on it; Sec. "Lattice Boltzmann Model", moment rule, and
Sec. "Bona-Masso evolution equations", first-order derivatives):

* LAG (reading R17): A and D from central differences of the previous
  step's corrected alpha and gamma, the initial fields at the first step.
* FIXED (reading R18): the moment rule rho = rho~ + dt S(rho)/2 solved as an
  equation, A and D from rho itself.

Each pin checks the oracle against something other than its own step: an
independent evaluation of the moment rule in numpy (central differences
taken here, sources from the pinned pointwise right-hand sides), the
discrete budget of Eq. numlb, dimensional reduction, convergence to the
closed-form gauge wave, and flat space.
"""
import math

import numpy as np
import pytest

from paper_1505_02037_gb300 import workloads as W

PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def sources_numpy(O, rho_state, dsrc, dx, dims, slicing=1):
    """The 16 macroscopic sources at every cell of fields rho_state
    [16][nz][ny][nx], with A_k, D_kij by periodic central differences of
    dsrc's alpha and gamma (planes 0..6), evaluated here in numpy; the
    pointwise right-hand sides come from the pinned bm_point."""
    nz, ny, nx = rho_state.shape[1:]
    la = np.log(dsrc[0])
    A = np.zeros((3,) + la.shape)
    D = np.zeros((3, 6) + la.shape)
    for k in range(dims):
        ax = 2 - k
        A[k] = (np.roll(la, -1, ax) - np.roll(la, 1, ax)) / (2 * dx)
        for q in range(6):
            g = dsrc[1 + q]
            D[k, q] = (np.roll(g, -1, ax) - np.roll(g, 1, ax)) / (4 * dx)
    S = np.zeros_like(rho_state)
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                v = rho_state[:, z, y, x]
                lam, Sij, Om, Sa = O.bm_point(v[0], v[1:7], v[7:13], v[13:16], A[:, z, y, x],
                                              D[:, :, z, y, x], slicing)
                S[0, z, y, x] = Sa
                S[1:7, z, y, x] = -2 * v[0] * v[7:13]
                S[7:13, z, y, x] = v[0] * Sij
                S[13:16, z, y, x] = Om
    return S


def wave_state(shape, dx, seed=3):
    """Flat space plus smooth seeded Fourier modes in every field and
    direction, and noise: [16][nz][ny][nx]."""
    return W.add_noise(W.smooth_modes(shape, dx, 0.05, seed=seed), 1e-4, seed=seed + 1)


# ---------------------------------------------------------------------------
# LAG
# ---------------------------------------------------------------------------
def test_lag_moments_use_the_lagged_fields(oracle_mod):
    """First step: rho = rho~ + dt S(rho~; A, D of the initial fields)/2,
    evaluated independently; it differs from the SYNC reading. Second step:
    the lagged fields are exactly the first step's corrected alpha and gamma,
    and the moment rule uses them."""
    O = oracle_mod
    shape, dx, tau = (12, 10, 1), 1 / 12, 1.2
    fields = wave_state(shape, dx)
    o = O.Oracle(2, shape, tau, dx, deriv_mode=1)
    f, prev = o.lag_init(fields)
    for n in range(2):
        rt = f.sum(axis=1).reshape(16, 1, 10, 12)
        S = sources_numpy(O, rt, prev.reshape(7, 1, 10, 12), dx, 2)
        expect = (rt + 0.5 * dx * S).reshape(16, -1)
        got = o.moments_lag(f, prev)
        np.testing.assert_allclose(got, expect, rtol=0, atol=2e-14)
        sync = O.Oracle(2, shape, tau, dx).moments(f)
        assert np.abs(sync - got).max() > 1e-9  # the readings differ
        f1, prev1 = o.step_lag(f, prev)
        assert np.array_equal(prev1, got[:7])
        f, prev = f1, prev1


@pytest.mark.parametrize("vset", [2, 3])
def test_lag_discrete_budget(oracle_mod, vset):
    """Eq. numlb summed over velocities and cells: sum rho~(n+1) =
    sum rho~(n) + dt sum S~(n) with S~ read off the moment rule, so the
    collision uses the same lagged sources as the corrected moments."""
    O = oracle_mod
    shape = (8, 6, 1) if vset == 2 else (6, 5, 4)
    dx = 1 / shape[0]
    o = O.Oracle(vset, shape, 1.3, dx, deriv_mode=1)
    f, prev = o.lag_init(wave_state(shape, dx))
    f, prev = o.run_lag(f, prev, 2)
    rt = f.sum(axis=1).sum(axis=1)
    rho = o.moments_lag(f, prev).sum(axis=1)
    rt1 = o.step_lag(f, prev)[0].sum(axis=1).sum(axis=1)
    np.testing.assert_allclose(rt1 - rt, 2 * (rho - rt), rtol=1e-9, atol=1e-13)


def test_lag_x_aligned_3d_equals_1d(oracle_mod):
    """An x-aligned wave on D3Q19 (any ny, nz) runs exactly as on D1Q3, its
    x-marginal, under LAG too."""
    O = oracle_mod
    N, dx = 24, 1 / 24
    o1 = O.Oracle(1, (N, 1, 1), 1.5, dx, deriv_mode=1)
    o3 = O.Oracle(3, (N, 3, 2), 1.5, dx, deriv_mode=1)
    f1, p1 = o1.lag_init(W.gauge_wave((N, 1, 1), dx, 0.1))
    f3, p3 = o3.lag_init(W.gauge_wave((N, 3, 2), dx, 0.1))
    f1, p1 = o1.run_lag(f1, p1, 30)
    f3, p3 = o3.run_lag(f3, p3, 30)
    m1 = o1.moments_lag(f1, p1)
    m3 = o3.moments_lag(f3, p3).reshape(16, 6, N)
    assert np.abs(m3 - m1[:, None, :]).max() < 1e-13


def test_lag_gauge_wave_first_order_convergence(oracle_mod):
    """At fixed tau/dt the LAG error against the closed form at a fixed
    physical time falls linearly with the lattice spacing."""
    O = oracle_mod
    errs = []
    for N in (200, 400, 800):
        o = O.Oracle(1, (N, 1, 1), 4.5, 1 / N, deriv_mode=1)
        f, p = o.lag_init(W.gauge_wave((N, 1, 1), 1 / N, 1e-3))
        f, p = o.run_lag(f, p, N // 4)
        ex = W.gauge_wave((N, 1, 1), 1 / N, 1e-3, t=0.25).reshape(16, -1)
        errs.append(np.abs(o.moments_lag(f, p)[1] - ex[1]).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.85 < q < 1.15 for q in orders), (errs, orders)


# ---------------------------------------------------------------------------
# FIXED
# ---------------------------------------------------------------------------
def test_fixed_point_solves_the_moment_rule(oracle_mod):
    """The FIXED moments satisfy rho = rho~ + dt S(rho)/2 with A and D taken
    from rho itself, evaluated independently, to round-off."""
    O = oracle_mod
    shape, dx = (10, 8, 1), 1 / 10
    fields = wave_state(shape, dx, seed=5)
    o = O.Oracle(2, shape, 1.1, dx, deriv_mode=2)
    f = O.Oracle(2, shape, 1.1, dx).run(O.Oracle(2, shape, 1.1, dx).init(fields), 2)
    rho = o.moments(f).reshape(16, 1, 8, 10)
    rt = f.sum(axis=1).reshape(16, 1, 8, 10)
    S = sources_numpy(O, rho, rho, dx, 2)
    assert np.abs(rho - rt - 0.5 * dx * S).max() < 5e-15
    assert np.abs(rho - rt).max() > 1e-6  # the sources are not negligible


def test_fixed_gauge_wave_first_order_convergence(oracle_mod):
    O = oracle_mod
    errs = []
    for N in (200, 400, 800):
        o = O.Oracle(1, (N, 1, 1), 4.5, 1 / N, deriv_mode=2)
        f = o.run(o.init(W.gauge_wave((N, 1, 1), 1 / N, 1e-3)), N // 4)
        ex = W.gauge_wave((N, 1, 1), 1 / N, 1e-3, t=0.25).reshape(16, -1)
        errs.append(np.abs(o.moments(f)[1] - ex[1]).max())
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(0.85 < q < 1.15 for q in orders), (errs, orders)


def test_fixed_and_sync_moments_differ_at_second_order(oracle_mod):
    """The explicit moment rule (R5) and its fixed point differ by
    dt^2/4 S' S per step: halving dx quarters the difference."""
    O = oracle_mod
    diffs = []
    for N in (64, 128, 256):
        fields = W.gauge_wave((N, 1, 1), 1 / N, 0.05)
        s = O.Oracle(1, (N, 1, 1), 1.5, 1 / N)
        x = O.Oracle(1, (N, 1, 1), 1.5, 1 / N, deriv_mode=2)
        f = s.init(fields)
        diffs.append(np.abs(x.moments(f) - s.moments(f)).max())
    orders = [math.log2(diffs[i] / diffs[i + 1]) for i in range(2)]
    assert all(1.8 < q < 2.2 for q in orders), (diffs, orders)


# ---------------------------------------------------------------------------
# Both, and the stability finding
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("vset", [1, 2, 3])
@pytest.mark.parametrize("mode", [1, 2])
def test_flat_space_is_a_bitwise_fixed_point(oracle_mod, vset, mode):
    """As under SYNC: the first step moves values by at most an ulp of 1 (the
    weights do not sum to exactly 1 in binary); from then on the state is a
    bitwise fixed point (the lagged fields, one step behind, from the second
    step on)."""
    O = oracle_mod
    shape = {1: (16, 1, 1), 2: (8, 6, 1), 3: (6, 5, 4)}[vset]
    o = O.Oracle(vset, shape, 0.9, 1 / shape[0], deriv_mode=mode)
    flat = W.flat(shape)
    if mode == 1:
        f0, p0 = o.lag_init(flat)
        f, p = o.step_lag(f0, p0)
        assert np.abs(f - f0).max() <= 2.3e-16 and np.abs(p - p0).max() <= 4.5e-16
        f, p = o.step_lag(f, p)
        g, q = o.run_lag(f, p, 5)
        assert np.array_equal(f, g) and np.array_equal(p, q)
    else:
        f0 = o.init(flat)
        f = o.step(f0)
        assert np.abs(f - f0).max() <= 2.3e-16
        assert np.array_equal(o.run(f, 5), f)


def amplification(O, tau, mode, N):
    """Largest |eigenvalue| of one step linearised about flat space (D1Q3,
    N cells); for LAG the state is the distributions and the lagged fields."""
    o = O.Oracle(1, (N, 1, 1), tau, 1 / N, deriv_mode=mode)
    flat = W.flat((N, 1, 1))
    if mode == 1:
        f0, p0 = o.lag_init(flat)
        x0 = np.concatenate([f0.reshape(-1), p0.reshape(-1)])

        def F(x):
            a, b = o.step_lag(x[:f0.size].reshape(f0.shape), x[f0.size:].reshape(p0.shape))
            return np.concatenate([a.reshape(-1), b.reshape(-1)])
    else:
        f0 = o.init(flat)
        x0 = f0.reshape(-1)

        def F(x):
            return o.step(x.reshape(f0.shape)).reshape(-1)
    base = F(x0)
    J = np.zeros((x0.size, x0.size))
    for i in range(x0.size):
        g = x0.copy()
        g[i] += 1e-7
        J[:, i] = (F(g) - base) / 1e-7
    return float(np.abs(np.linalg.eigvals(J)).max())


def test_every_reading_is_unstable_at_the_configurations_tau(oracle_mod):
    """tau = 0.55 (of the range 0.51..0.6 the configurations use) is linearly
    unstable under SYNC, LAG and FIXED alike: the instability belongs to the
    method, not to the reading of the moment rule. At the paper's tau/dt =
    4.5 the fixed point is neutrally stable, SYNC grows slowly."""
    O = oracle_mod
    for mode in (0, 1, 2):
        assert amplification(O, 0.55, mode, 16) > 1.3, mode
    assert amplification(O, 4.5, 2, 32) < 1 + 1e-6
    assert 1.001 < amplification(O, 4.5, 0, 32) < 1.01
