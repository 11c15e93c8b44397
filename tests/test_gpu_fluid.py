"""The matter terms on the GPU (Sec. "Expansion of flat universe"): a perfect
fluid at rest, against the FP64 oracle and the flat FLRW closed form."""
import math

import numpy as np
import pytest

from paper_1505_02037_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02037_gb300 import lbnr
    lbnr.library()
    return lbnr


def rel(g, o, floor):
    g, o = g.reshape(16, -1), o.reshape(16, -1)
    return (np.abs(g - o).max(axis=1) / np.maximum(np.abs(o).max(axis=1), floor)).max()


def test_friedmann_run_fp64_matches_oracle_and_closed_form(L, oracle_mod):
    """The paper's run: D3Q19 4^3, dt = dr = 0.001, tau/dt = 3, stiff fluid
    P = rho = 1/(3 t^2) from t = 1, geodesic slicing. Each checkpoint equals
    the oracle to 1e-12, and gamma_xx is within 0.01 % of t^(2/3)."""
    shape, dt = (4, 4, 4), 1e-3
    lat = L.Lattice(3, shape, 3.0, dt, slicing=0)
    lat.set_fluid(1.0 / 3.0, 1.0, 1.0)
    lat.init(W.flrw(shape, t=1.0))
    o = oracle_mod.Oracle(3, shape, 3.0, dt, slicing=0, fluid=(1.0 / 3.0, 1.0, 1.0))
    f = o.init(W.flrw(shape, t=1.0))
    done = 0
    for n in (1, 10, 250, 1000):
        lat.step(n - done)
        f = o.run(f, n - done, t=1.0 + done * dt)
        done = n
        t = 1.0 + n * dt
        mo = o.moments(f, t=t)
        mg = lat.moments()
        assert rel(mg, mo, 0.1) < TOL64, n
        assert rel(lat.distributions(), f, 0.03) < TOL64, n
        assert np.abs(mg[1] / W.flrw(shape, t=t)[1] - 1).max() < 1e-4, n


def test_inhomogeneous_wave_with_fluid_fp64_matches_oracle(L, oracle_mod):
    """Every term at once: a diagonal gauge wave (A = 0.05) on 12^3 with a
    radiation fluid (w = 1/3, rho0 = 0.2 at t0 = 1.5), 20 steps, harmonic
    slicing, against the oracle."""
    N, shape = 12, (12, 12, 12)
    fields = W.gauge_wave(shape, 1 / N, 0.05, direction="xyz")
    lat = L.Lattice(3, shape, 1.5, 1 / N, slicing=1)
    lat.set_fluid(0.2, 1.0 / 3.0, 1.5)
    lat.init(fields)
    lat.step(20)
    o = oracle_mod.Oracle(3, shape, 1.5, 1 / N, slicing=1, fluid=(0.2, 1.0 / 3.0, 1.5))
    f = o.run(o.init(fields, t=1.5), 20, t=1.5)
    assert rel(lat.distributions(), f, 0.05 * math.pi / 3) < TOL64
    assert rel(lat.moments(), o.moments(f, t=1.5 + 20 / N), 0.05 * math.pi) < TOL64


@pytest.mark.parametrize("storage", ["dev_f32", "f32"])
def test_friedmann_run_reduced_precision(L, storage):
    """The same run stored in FP32 (deviations from flat space, or f itself).
    The homogeneous run is a time integration with nothing to amplify
    rounding, so its distance from the FP64 run grows at most linearly: the
    bar after n steps is 4 n units of 2^-24 on gamma_xx and K_xx. The distance
    to the closed form is bounded by that plus the FP64 run's own error."""
    shape, dt, n = (4, 4, 4), 1e-3, 1000
    runs = {}
    for st in ("f64", storage):
        lat = L.Lattice(3, shape, 3.0, dt, slicing=0, storage=st)
        lat.set_fluid(1.0 / 3.0, 1.0, 1.0)
        lat.init(W.flrw(shape, t=1.0))
        lat.step(n)
        runs[st] = lat.moments()
        lat.close()
    bar = 4 * n * 2.0 ** -24
    m, m64, ex = runs[storage], runs["f64"], W.flrw(shape, t=1.0 + n * dt)
    for F in (1, 7):
        assert np.abs(m[F] / m64[F] - 1).max() <= bar, (F, np.abs(m[F] / m64[F] - 1).max())
    e64 = np.abs(m64[1] / ex[1] - 1).max()
    assert e64 < 1e-4
    assert np.abs(m[1] / ex[1] - 1).max() <= e64 + bar


def test_fluid_off_is_vacuum(L):
    """rho0 = 0 switches the matter off: the run equals one that never set it,
    bit for bit."""
    shape = (10, 8, 6)
    fields = W.gauge_wave(shape, 0.1, 0.05, direction="x")
    a = L.Lattice(3, shape, 1.2, 0.1)
    b = L.Lattice(3, shape, 1.2, 0.1)
    b.set_fluid(0.3, 1.0, 1.0)
    b.set_fluid(0.0, 1.0, 1.0)
    a.init(fields)
    b.init(fields)
    a.step(7)
    b.step(7)
    assert np.array_equal(a.distributions(), b.distributions())


@pytest.mark.parametrize("with_field", [False, True])
def test_fluid_with_shift_fp64_matches_oracle(L, oracle_mod, with_field):
    """The fluid's term and the shift's terms together (constant shift, and
    with a smooth static shift field), diagonal gauge wave on 12^3, 10 steps,
    every 1+log slicing term, against the oracle at 1e-12."""
    N, shape = 12, (12, 12, 12)
    beta = (0.05, -0.03, 0.02)
    field = W.smooth_shift(shape, 1 / N, 0.04, seed=44) if with_field else None
    fields = W.gauge_wave(shape, 1 / N, 0.05, direction="xyz", beta=beta)
    lat = L.Lattice(3, shape, 1.5, 1 / N, slicing=2)
    lat.set_fluid(0.2, 1.0 / 3.0, 1.5)
    lat.set_shift(beta)
    if with_field:
        lat.set_shift_field(field)
    lat.init(fields)
    lat.step(10)
    o = oracle_mod.Oracle(3, shape, 1.5, 1 / N, slicing=2, fluid=(0.2, 1.0 / 3.0, 1.5),
                          shift=beta, shift_field=field)
    f = o.run(o.init(fields, t=1.5), 10, t=1.5)
    assert rel(lat.distributions(), f, 0.05 * math.pi / 3) < TOL64
    assert rel(lat.moments(), o.moments(f, t=1.5 + 10 / N), 0.05 * math.pi) < TOL64
