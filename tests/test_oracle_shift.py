"""Pins of the oracle's constant-shift terms (Sec. "Bona-Masso evolution
equations" with a constant, uniform shift beta^i, so B_k^i = 0):

* lapse source alpha beta^r A_r, metric source 2 beta^r D_rij;
* flux -beta^k K_ij added to alpha lambda^k_ij in the K equilibria, flux
  -beta^k V_i in the V equilibria (the factor 1 - c.beta / c_s^2).

What fixes them is geometry, not the formulas: a zero-shift spacetime seen
from coordinates x' = x - beta t has shift beta^i and the same lapse, metric
and extrinsic curvature, so the fields at x' are the zero-shift fields at
x' + beta t. Hence (1) the shifted gauge wave is the gauge wave at u + beta t
(a closed form), and (2) for any initial data, the shifted run at time t is
the zero-shift run at time t translated by beta t; the scheme reaches both at
first order in the lattice spacing. A dropped term, a wrong sign or a
transposed index moves some field at the wrong speed and leaves an error of
the size of the data that does not fall with the spacing.
"""
import math

import numpy as np
import pytest

from paper_1505_02037_gb300 import workloads as W

AMP = 1e-3


def _shape(vset, N):
    return {1: (N, 1, 1), 2: (N, N, 1), 3: (N, N, N)}[vset]


def test_zero_shift_leaves_the_step_unchanged(oracle_mod):
    """A zero shift is the zero-shift system, bit for bit."""
    O = oracle_mod
    shape = (12, 10, 1)
    f0 = W.add_noise(W.smooth_modes(shape, 1 / 12, 0.01, 3), 1e-3, 4)
    a = O.Oracle(2, shape, 0.9, 1 / 12)
    b = O.Oracle(2, shape, 0.9, 1 / 12, shift=(0.0, 0.0, 0.0))
    fa, fb = a.init(f0), b.init(f0)
    assert np.array_equal(fa, fb)
    assert np.array_equal(a.run(fa, 3), b.run(fb, 3))


@pytest.mark.parametrize("v", [0.25, -0.3])
def test_shifted_gauge_wave_converges_to_its_closed_form(oracle_mod, v):
    """Gauge wave in coordinates moving at -v along x: beta^x = v,
    alpha = sqrt(H), gamma_xx = H, K_xx as without shift, all at x + v t (phase
    speed 1 - v). The error in alpha, gamma_xx and K_xx at t = 1/4 falls
    linearly with the spacing."""
    O = oracle_mod
    errs = []
    for N in (200, 400, 800):
        o = O.Oracle(1, (N, 1, 1), 4.5, 1 / N, shift=(v, 0, 0))
        f = o.run(o.init(W.gauge_wave((N, 1, 1), 1 / N, AMP, beta=(v, 0, 0))), N // 4)
        ex = W.gauge_wave((N, 1, 1), 1 / N, AMP, t=0.25, beta=(v, 0, 0)).reshape(16, -1)
        m = o.moments(f)
        errs.append([np.abs(m[F] - ex[F]).max() for F in (0, 1, 7)])
    errs = np.array(errs)
    orders = np.log2(errs[:-1] / errs[1:])
    assert np.all((orders > 0.85) & (orders < 1.15)), (errs, orders)
    assert errs[-1].max() < 0.2 * AMP


def _translation_errors(O, vset, N, beta, t, tau=4.5, seed=7):
    """max |shifted run - zero-shift run translated by beta t| per field."""
    shape = _shape(vset, N)
    f0 = W.smooth_modes(shape, 1 / N, AMP, seed, modes=1)
    n = int(round(t * N))
    a = O.Oracle(vset, shape, tau, 1 / N)
    b = O.Oracle(vset, shape, tau, 1 / N, shift=beta)
    ma = a.moments(a.run(a.init(f0), n)).reshape(16, shape[2], shape[1], shape[0])
    mb = b.moments(b.run(b.init(f0), n)).reshape(16, shape[2], shape[1], shape[0])
    cells = [beta[k] * t * N for k in range(3)]
    assert all(abs(c - round(c)) < 1e-9 for c in cells)  # whole cells
    ma = np.roll(ma, tuple(-int(round(c)) for c in cells[::-1]), axis=(1, 2, 3))
    return np.abs(mb - ma).max(axis=(1, 2, 3))


def test_shift_is_a_translation_d1q3(oracle_mod):
    """Generic smooth data (every field perturbed, constraints not imposed),
    beta^x = 1/2: the shifted run at t = 1/4 is the zero-shift run moved by
    1/8 of the box, each of the 16 fields to first order in the spacing."""
    E = np.array([_translation_errors(oracle_mod, 1, N, (0.5, 0.0, 0.0), 0.25)
                  for N in (256, 512, 1024)])
    orders = np.log2(E[:-1] / E[1:])
    assert np.all((orders > 0.85) & (orders < 1.25)), (E, orders)
    assert E[-1].max() < 0.15 * AMP


def test_oblique_shift_is_a_translation_d2q9(oracle_mod):
    """D2Q9, shift (1/4, -1/2) against a wave pattern along x, y and the
    diagonals: every field's distance to the translated zero-shift run
    at least halves from N = 64 to N = 256 (still short of the asymptotic
    order 1 at these sizes) and ends below 0.3 of the perturbation."""
    E = np.array([_translation_errors(oracle_mod, 2, N, (0.25, -0.5, 0.0), 0.25)
                  for N in (64, 256)])
    assert np.all(E[1] <= E[0] / 2), E
    assert E[1].max() < 0.3 * AMP


@pytest.mark.parametrize("vset", [2, 3])
def test_transverse_shift_components_drop_out_of_an_x_wave(oracle_mod, vset):
    """Data that depends on x alone: the shift's y and z components move
    nothing, so the D2Q9/D3Q19 run with shift (1/2, 0.3, -0.2) equals the D1Q3
    run with shift (1/2, 0, 0) to round-off (the sets' x marginals are D1Q3)."""
    O = oracle_mod
    N = 64
    shape = (N, 2, 1) if vset == 2 else (N, 2, 3)
    f1 = W.smooth_modes((N, 1, 1), 1 / N, 0.01, 11, modes=2)
    fields = np.broadcast_to(f1.reshape(16, 1, 1, N), (16, shape[2], shape[1], N)).copy()
    beta = (0.5, 0.3, -0.2) if vset == 3 else (0.5, 0.3, 0.0)
    a = O.Oracle(1, (N, 1, 1), 1.5, 1 / N, shift=(0.5, 0.0, 0.0))
    b = O.Oracle(vset, shape, 1.5, 1 / N, shift=beta)
    m1 = a.moments(a.run(a.init(f1), 20)).reshape(16, 1, 1, N)
    m3 = b.moments(b.run(b.init(fields), 20)).reshape(16, shape[2], shape[1], N)
    # round-off in a different summation order, grown by the step's
    # amplification (lambda(1.5)^20 is about 3)
    scale = np.abs(m1).max()
    assert np.abs(m3 - m1).max() <= 1e-11 * scale
    # and the shift did move the data (the test is not vacuous)
    c = O.Oracle(1, (N, 1, 1), 1.5, 1 / N)
    m0 = c.moments(c.run(c.init(f1), 20)).reshape(16, 1, 1, N)
    assert np.abs(m0 - m1).max() > 1e-3


# ---------------------------------------------------------------------------
# Static shift field: B_k^i = d_k beta^i / 2 terms
# ---------------------------------------------------------------------------
def _sheared_errors(O, N, A, v0=0.1, t=0.25, tau=1.0):
    shape = (N, N, 1)
    o = O.Oracle(2, shape, tau, 1 / N, shift_field=W.shear_shift(shape, 1 / N, v0))
    f = o.run(o.init(W.sheared_gauge_wave(shape, 1 / N, A, v0)), int(round(t * N)))
    ex = W.sheared_gauge_wave(shape, 1 / N, A, v0, t=t).reshape(16, -1)
    return np.abs(o.moments(f) - ex).max(axis=1)


@pytest.mark.parametrize("A", [0.0, 0.01])
def test_sheared_coordinates_converge_to_their_closed_form(oracle_mod, A):
    """Flat space (A = 0) and the gauge wave (A = 0.01) carried by the flow
    of the static shear shift beta = (0.1 sin(2 pi y), 0, 0): gamma_xy,
    gamma_yy, K_xy, K_yy and both V_x and V_y are nonzero, so every B term
    (metric source, K source, V flux and V source) acts. D2Q9, tau/dt = 1,
    t = 1/4: each nonzero field's error falls linearly with the spacing."""
    E = np.array([_sheared_errors(oracle_mod, N, A) for N in (64, 128, 256)])
    live = E[-1] > 0
    orders = np.log2(E[:-1, live] / E[1:, live])
    assert live[[2, 4, 8, 10, 13, 14]].all()
    assert np.all((orders > 0.85) & (orders < 1.25)), (E, orders)
    assert E[-1].max() < 0.01


def test_uniform_shift_field_is_the_constant_shift(oracle_mod):
    """A uniform field has B = 0: it runs exactly as the same constant shift."""
    O = oracle_mod
    shape = (16, 12, 1)
    f0 = W.add_noise(W.smooth_modes(shape, 1 / 16, 0.01, 5), 1e-4, 6)
    beta = (0.2, -0.1, 0.05)
    field = np.broadcast_to(np.array(beta).reshape(3, 1, 1, 1), (3, 1, 12, 16)).copy()
    a = O.Oracle(2, shape, 0.9, 1 / 16, shift=beta)
    b = O.Oracle(2, shape, 0.9, 1 / 16, shift_field=field)
    fa, fb = a.init(f0), b.init(f0)
    assert np.array_equal(fa, fb)
    assert np.array_equal(a.run(fa, 3), b.run(fb, 3))
