"""Pins of the oracle's matter terms (Sec. "Expansion of flat universe"): a
perfect fluid at rest enters S_ij through -R^(4)_ij + (gamma_ij/4) 2 alpha^2
G^00. The flat FLRW universe is an exact solution for every equation of
state P = w rho, so the oracle's sources must equal the closed-form time
derivatives there; and the paper reports its lattice run within 0.01 % of the
closed form."""
import numpy as np
import pytest

from paper_1505_02037_gb300 import workloads as W


@pytest.mark.parametrize("w", [0.0, 1.0 / 3.0, 1.0])
@pytest.mark.parametrize("t", [0.7, 1.0, 2.5])
def test_sources_equal_flrw_time_derivatives(oracle_mod, w, t):
    """d_t K_ij = alpha S_ij and d_t gamma_ij = -2 alpha K_ij on the closed
    form, for dust, radiation and the paper's stiff fluid."""
    q = W.flrw_exponent(w)
    g = t ** (2 * q)
    k = -q * t ** (2 * q - 1)
    dk = -q * (2 * q - 1) * t ** (2 * q - 2)  # d_t K_xx
    g6 = [g, 0, 0, g, 0, g]
    K6 = [k, 0, 0, k, 0, k]
    rho = W.flrw_density(t, w)
    lam, S, Om, Sa = oracle_mod.bm_point(1.0, g6, K6, [0, 0, 0], [0, 0, 0], np.zeros((3, 6)),
                                         slicing=0, rho=rho, P=w * rho)
    assert np.allclose(S, [dk, 0, 0, dk, 0, dk], rtol=1e-13, atol=1e-15), (S, dk)
    assert np.allclose(Om, 0) and Sa == 0.0 and np.allclose(lam, 0)
    # With pressure the same state is not a vacuum solution, so the matter
    # term is what makes it one. (For dust the term, (P/2) gamma_ij, is 0:
    # the density parts cancel.)
    if w > 0:
        _, S0, _, _ = oracle_mod.bm_point(1.0, g6, K6, [0, 0, 0], [0, 0, 0], np.zeros((3, 6)),
                                          slicing=0)
        assert abs(S0[0] - dk) > 1e-3 * abs(dk), (S0[0], dk)


def test_lattice_run_follows_friedmann(oracle_mod):
    """The paper's run: D3Q19, 4^3 cells, dt = dr = 0.001, tau/dt = 3, stiff
    fluid (P = rho = 1/(3 t^2)) from t = 1, geodesic slicing; gamma_xx stays
    within 0.01 % of t^(2/3) (and K_xx of -t^(-1/3)/3 within 0.1 %) over
    1000 steps."""
    shape = (4, 4, 4)
    o = oracle_mod.Oracle(3, shape, 3.0, 1e-3, slicing=0, fluid=(1.0 / 3.0, 1.0, 1.0))
    f = o.init(W.flrw(shape, t=1.0))
    done = 0
    for n in (250, 500, 1000):
        f = o.run(f, n - done, t=1.0 + done * 1e-3)
        done = n
        t = 1.0 + n * 1e-3
        m = o.moments(f, t=t)
        ex = W.flrw(shape, t=t)
        assert np.abs(m[1] / ex[1] - 1).max() < 1e-4, (n, np.abs(m[1] / ex[1] - 1).max())
        assert np.abs(m[7] / ex[7] - 1).max() < 1e-3, (n, np.abs(m[7] / ex[7] - 1).max())
        assert np.abs(m[2]).max() < 1e-12 and np.abs(m[0] - 1).max() < 1e-12
