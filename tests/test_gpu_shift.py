"""GPU parity of the constant-shift terms (Sec. "Bona-Masso evolution
equations" with a constant, uniform beta^i): the CUDA path through the C-ABI
against the FP64 oracle, which the shifted gauge wave's closed form and the
shift-as-translation identity pin.

Metric as in the zero-shift parity tests: per field, max over cells of
|gpu - oracle| / max(max |oracle|, s_F), s_F = 1 for alpha and gamma and a
per-test scale for K and V. FP64 bar 1e-12; reduced precision within the
stated bound of the storage (same constants K_s as at zero shift, with the
amplification factor of the shifted step).
"""
import math

import numpy as np
import pytest

from paper_1505_02037_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
BETA = (0.3, -0.2, 0.1)
# K_s per storage (1D, 3D): the stated per-step rounding constants
KS = {"dev_bf16": (1.0e-2, 1.0e-2), "dev_f16": (1.0e-3, 1.0e-3),
      "dev_f32": (2.5e-7, 1.0e-6), "f32": (5.0e-5, 2.0e-4)}


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02037_gb300 import lbnr
    lbnr.library()
    return lbnr


def field_err(g, o, kscale):
    g = g.reshape(16, -1)
    o = o.reshape(16, -1)
    floor = np.array([1.0] * 7 + [kscale] * 9)
    return np.abs(g - o).max(axis=1) / np.maximum(np.abs(o).max(axis=1), floor)


# The scheme amplifies any perturbation by up to lambda(tau) per step and the
# stencil adds 1/(k dx), so two correct FP64 programs that round differently
# drift apart by more than 1e-12 over tens of steps. The bar is then 4 x the
# distance between the oracle and the oracle started from distributions
# perturbed by one ulp (seeded signs), at the same step.
def perturbed(f, seed=0):
    rng = np.random.default_rng(seed)
    return f * (1 + rng.choice([-1.0, 1.0], size=f.shape) * 2.2e-16)


def bar(spread):
    return max(TOL64, 4 * spread)


def dist_err(g, o, kscale):
    g = g.reshape(16, -1)
    o = o.reshape(16, -1)
    floor = np.array([1.0] * 7 + [kscale] * 9) / 3
    return np.abs(g - o).max(axis=1) / np.maximum(np.abs(o).max(axis=1), floor)


_lam = {}


def amplification(O, tau, beta, N=32):
    """Largest eigenvalue modulus of the oracle's shifted D1Q3 step
    linearised about flat space."""
    key = (tau, beta)
    if key not in _lam:
        o = O.Oracle(1, (N, 1, 1), tau, 1 / N, shift=beta)
        f0 = o.init(W.flat((N, 1, 1)))
        base = o.step(f0).reshape(-1)
        flat = f0.reshape(-1)
        J = np.zeros((flat.size, flat.size))
        for i in range(flat.size):
            g = flat.copy()
            g[i] += 1e-7
            J[:, i] = (o.step(g.reshape(f0.shape)).reshape(-1) - base) / 1e-7
        _lam[key] = float(np.abs(np.linalg.eigvals(J)).max())
    return _lam[key]


def bound(storage, three_d, N, tau, n, lam):
    k = KS[storage][1 if three_d else 0]
    growth = n if abs(lam - 1) < 1e-12 else (lam ** n - 1) / (lam - 1)
    return 3 * k * (N / (2 * math.pi)) / tau * growth


@pytest.mark.parametrize("vset,shape", [
    (1, (333, 1, 1)), (2, (37, 23, 1)), (3, (21, 13, 11)), (3, (2, 5, 3)), (1, (1, 1, 1)),
])
@pytest.mark.parametrize("streaming", [1, 2])
def test_random_state_steps_with_shift_fp64(L, oracle_mod, vset, shape, streaming):
    """Seeded random near-flat distributions, shift (0.3, -0.2, 0.1): every
    shift term active, ragged lattices, 1, 2 and 3 steps (both AA parities)."""
    Q = {1: 3, 2: 9, 3: 19}[vset]
    _, w = oracle_mod.velocity_set(vset)
    f0 = W.random_distributions(Q, w, shape, seed=2000 + vset)
    o = oracle_mod.Oracle(vset, shape, 0.8, 1 / shape[0], shift=BETA)
    lat = L.Lattice(vset, shape, 0.8, 1 / shape[0], streaming=streaming)
    lat.set_shift(BETA)
    lat.set_distributions(f0)
    f, fp = f0, perturbed(f0)
    for n in range(3):
        lat.step(1)
        f, fp = o.step(f), o.step(fp)
        # K and V floor: the random state's noise amplitude; bar: 1e-12 or
        # 4 x the oracle's own one-ulp spread at this step
        spread_d = dist_err(fp, f, 1e-3).max()
        spread_m = field_err(o.moments(fp), o.moments(f), 1e-3).max()
        assert dist_err(lat.distributions(), f, 1e-3).max() <= bar(spread_d), n
        assert field_err(lat.moments(), o.moments(f), 1e-3).max() <= bar(spread_m), n


@pytest.mark.parametrize("vset,shape,direction", [
    (1, (200, 1, 1), "x"), (2, (48, 48, 1), "xy"), (3, (20, 20, 20), "xyz"),
])
def test_shifted_gauge_wave_init_and_run_fp64(L, oracle_mod, vset, shape, direction):
    """The shifted gauge wave from its closed form (the device's own shifted
    equilibria at init), 40 steps, every field and distribution against the
    oracle (1e-12 at init; after 40 steps, 1e-12 or the one-ulp spread)."""
    N, A = shape[0], 0.05
    beta = (0.25, -0.15, 0.1)
    fields = W.gauge_wave(shape, 1 / N, A, direction=direction, beta=beta)
    lat = L.Lattice(vset, shape, 1.5, 1 / N)
    lat.set_shift(beta)
    lat.init(fields)
    o = oracle_mod.Oracle(vset, shape, 1.5, 1 / N, shift=beta)
    f = o.init(fields)
    assert dist_err(lat.distributions(), f, math.pi * A).max() < TOL64
    fp = perturbed(f)
    lat.step(40)
    f, fp = o.run(f, 40), o.run(fp, 40)
    spread = field_err(o.moments(fp), o.moments(f), math.pi * A).max()
    assert field_err(lat.moments(), o.moments(f), math.pi * A).max() <= bar(spread)
    spread_d = dist_err(fp, f, math.pi * A).max()
    assert dist_err(lat.distributions(), f, math.pi * A).max() <= bar(spread_d)


def test_zero_shift_runs_the_zero_shift_forms(L):
    """set_shift((0, 0, 0)), before or after a nonzero shift, gives the
    zero-shift launch forms back, bit for bit."""
    shape = (32, 16, 8)
    fields = W.add_noise(W.gauge_wave(shape, 1 / 32, 0.05), 1e-4, seed=6)
    ref = L.Lattice(3, shape, 1.5, 1 / 32, storage="f32", streaming=1)
    ref.init(fields)
    ref.step(5)
    a = L.Lattice(3, shape, 1.5, 1 / 32, storage="f32", streaming=1)
    a.set_shift((0.2, 0.0, 0.0))
    a.set_shift((0.0, 0.0, 0.0))
    a.init(fields)
    a.step(5)
    assert np.array_equal(ref.distributions(), a.distributions())


def test_shift_is_not_a_no_op(L):
    """The same data with and without a shift differ after a few steps (the
    shifted form is the one that ran)."""
    shape = (64, 1, 1)
    fields = W.gauge_wave(shape, 1 / 64, 0.05)
    a = L.Lattice(1, shape, 1.5, 1 / 64)
    b = L.Lattice(1, shape, 1.5, 1 / 64)
    b.set_shift((0.25, 0.0, 0.0))
    a.init(fields)
    b.init(fields)
    a.step(8)
    b.step(8)
    assert np.abs(a.moments() - b.moments()).max() > 1e-4


def test_constraints_with_shift_fp64(L, oracle_mod):
    """The monitor reads the corrected moments, whose sources carry the
    shift: the 22 values against the oracle at t = 0 and after 10 steps."""
    N = 16
    shape = (N, N, N)
    beta = (0.2, 0.1, -0.3)
    fields = W.add_noise(W.gauge_wave(shape, 1 / N, 0.1, direction="xyz", beta=beta), 1e-4,
                         seed=8)
    lat = L.Lattice(3, shape, 1.5, 1 / N)
    lat.set_shift(beta)
    lat.init(fields)
    o = oracle_mod.Oracle(3, shape, 1.5, 1 / N, shift=beta)
    f = o.init(fields)
    for n in (0, 10):
        if n:
            lat.step(n)
            f = o.run(f, n)
        g, r = lat.constraints(), o.constraints(f)
        np.testing.assert_allclose(g[:6], r[:6], rtol=1e-10, atol=0)
        np.testing.assert_allclose(g[6:], r[6:], rtol=1e-12, atol=1e-12)


def test_full_size_sampled_step_with_shift_fp64(L, oracle_mod):
    """128^3 D3Q19 FP64, one shifted step from a seeded noisy diagonal wave,
    sampled cells (corners and random interior cells) against the oracle's
    per-cell step."""
    N = 128
    shape = (N, N, N)
    fields = W.add_noise(W.gauge_wave(shape, 1 / N, 0.05, direction="xyz", beta=BETA), 1e-6,
                         seed=5)
    o = oracle_mod.Oracle(3, shape, 0.9, 1 / N, shift=BETA)
    f0 = o.init(fields)
    lat = L.Lattice(3, shape, 0.9, 1 / N)
    lat.set_shift(BETA)
    lat.set_distributions(f0)
    lat.step(1)
    rng = np.random.default_rng(17)
    corners = [x + N * (y + N * z) for x in (0, N - 1) for y in (0, N - 1) for z in (0, N - 1)]
    idx = np.array(corners + list(rng.integers(0, N ** 3, size=120)), dtype=np.int64)
    got = lat.cells_distributions(idx)
    ref = o.step_cells(f0, idx)
    scale = np.abs(ref).max(axis=(0, 2))
    assert (np.abs(got - ref).max(axis=(0, 2)) / scale).max() < TOL64


@pytest.mark.parametrize("storage", ["dev_f32", "dev_f16", "dev_bf16", "f32"])
@pytest.mark.parametrize("streaming", [1, 2])
def test_reduced_precision_shift_1d_within_stated_bound(L, oracle_mod, storage, streaming):
    """Shifted gauge wave (v = 0.25), D1Q3, N = 256, tau = 1.5, A = 0.01: each
    storage against the FP64 oracle within the stated bound after 1, 10 and
    32 steps."""
    N, tau, A, beta = 256, 1.5, 0.01, (0.25, 0.0, 0.0)
    lam = amplification(oracle_mod, tau, beta)
    o = oracle_mod.Oracle(1, (N, 1, 1), tau, 1 / N, shift=beta)
    f = o.init(W.gauge_wave((N, 1, 1), 1 / N, A, beta=beta))
    lat = L.Lattice(1, (N, 1, 1), tau, 1 / N, storage=storage, streaming=streaming)
    lat.set_shift(beta)
    lat.init(W.gauge_wave((N, 1, 1), 1 / N, A, beta=beta))
    done = 0
    for n in (1, 10, 32):
        lat.step(n - done)
        f = o.run(f, n - done)
        done = n
        lat.status()
        err = float(np.abs(lat.moments().reshape(16, N) - o.moments(f)).max() / A)
        assert err <= bound(storage, False, N, tau, n, lam), (n, err)


@pytest.mark.parametrize("storage,streaming", [("f32", 1), ("dev_f32", 1), ("f32", 2)])
def test_full_size_256_cubed_with_shift(L, oracle_mod, storage, streaming):
    """The benchmark's shifted workload, 256^3 D3Q19 with shift
    (0.1, 0.05, -0.05) on an x-aligned gauge wave: the y and z components move
    nothing (pinned on the oracle), so the 1D oracle with shift (0.1, 0, 0)
    gives every cell's expected value; 1 and 2 steps (both AA parities),
    within the bound."""
    N, tau, A = 256, 4.5, 0.01
    beta3, beta1 = (0.1, 0.05, -0.05), (0.1, 0.0, 0.0)
    lam = amplification(oracle_mod, tau, beta1)
    o = oracle_mod.Oracle(1, (N, 1, 1), tau, 1 / N, shift=beta1)
    f = o.init(W.gauge_wave((N, 1, 1), 1 / N, A, beta=beta1))
    lat = L.Lattice(3, (N, N, N), tau, 1 / N, storage=storage, streaming=streaming)
    lat.set_shift(beta3)
    lat.init(W.gauge_wave((N, N, N), 1 / N, A, beta=beta3))
    done = 0
    for n in (1, 2):
        lat.step(n - done)
        f = o.run(f, n - done)
        done = n
        lat.status()
        m = lat.moments().reshape(16, -1, N)
        err = float(np.abs(m - o.moments(f)[:, None, :]).max() / A)
        assert err <= bound(storage, True, N, tau, n, lam), (n, err)
    lat.close()


# ---------------------------------------------------------------------------
# Static shift field (B terms)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("vset,shape", [
    (2, (37, 23, 1)), (3, (21, 13, 11)), (3, (2, 5, 3)), (1, (333, 1, 1)),
])
@pytest.mark.parametrize("streaming", [1, 2])
def test_random_state_steps_with_shift_field_fp64(L, oracle_mod, vset, shape, streaming):
    """Seeded random near-flat distributions under a constant shift plus a
    smooth seeded field (every B term active), ragged lattices, 1, 2 and 3
    steps (both AA parities)."""
    Q = {1: 3, 2: 9, 3: 19}[vset]
    _, w = oracle_mod.velocity_set(vset)
    f0 = W.random_distributions(Q, w, shape, seed=3000 + vset)
    field = W.smooth_shift(shape, 1 / shape[0], 0.1, seed=40 + vset)
    beta = (0.05, -0.03, 0.02)
    o = oracle_mod.Oracle(vset, shape, 0.8, 1 / shape[0], shift=beta, shift_field=field)
    lat = L.Lattice(vset, shape, 0.8, 1 / shape[0], streaming=streaming)
    lat.set_shift(beta)
    lat.set_shift_field(field)
    lat.set_distributions(f0)
    f, fp = f0, perturbed(f0)
    for n in range(3):
        lat.step(1)
        f, fp = o.step(f), o.step(fp)
        # K and V floor: the random state's noise amplitude; bar: 1e-12 or
        # 4 x the oracle's own one-ulp spread at this step
        spread_d = dist_err(fp, f, 1e-3).max()
        spread_m = field_err(o.moments(fp), o.moments(f), 1e-3).max()
        assert dist_err(lat.distributions(), f, 1e-3).max() <= bar(spread_d), n
        assert field_err(lat.moments(), o.moments(f), 1e-3).max() <= bar(spread_m), n


@pytest.mark.parametrize("A", [0.0, 0.05])
def test_sheared_gauge_wave_init_and_run_fp64(L, oracle_mod, A):
    """Flat space and the gauge wave carried by the shear shift's flow, from
    their closed form, D2Q9 64^2, tau 1: init at 1e-12, then 32 steps against
    the oracle (1e-12 or the one-ulp spread)."""
    N, v0 = 64, 0.1
    shape = (N, N, 1)
    field = W.shear_shift(shape, 1 / N, v0)
    fields = W.sheared_gauge_wave(shape, 1 / N, A, v0)
    lat = L.Lattice(2, shape, 1.0, 1 / N)
    lat.set_shift_field(field)
    lat.init(fields)
    o = oracle_mod.Oracle(2, shape, 1.0, 1 / N, shift_field=field)
    f = o.init(fields)
    assert dist_err(lat.distributions(), f, 0.1).max() < TOL64
    fp = perturbed(f)
    lat.step(32)
    f, fp = o.run(f, 32), o.run(fp, 32)
    spread = field_err(o.moments(fp), o.moments(f), 0.1).max()
    assert field_err(lat.moments(), o.moments(f), 0.1).max() <= bar(spread)
    # and the GPU run is as close to the closed form as the oracle
    ex = W.sheared_gauge_wave(shape, 1 / N, A, v0, t=0.5).reshape(16, -1)
    e_gpu = np.abs(lat.moments() - ex).max()
    e_orc = np.abs(o.moments(f) - ex).max()
    assert abs(e_gpu - e_orc) <= 1e-9 + 1e-6 * e_orc


def test_uniform_shift_field_matches_the_constant_shift(L):
    """A uniform field has B = 0: the field form and the constant-shift form
    agree to round-off (they take V's flux by different routes)."""
    shape = (24, 20, 1)
    fields = W.add_noise(W.gauge_wave(shape, 1 / 24, 0.05), 1e-4, seed=2)
    beta = (0.2, -0.1, 0.0)
    uni = np.broadcast_to(np.array(beta).reshape(3, 1, 1, 1), (3, 1, 20, 24)).copy()
    a = L.Lattice(2, shape, 1.5, 1 / 24)
    a.set_shift(beta)
    b = L.Lattice(2, shape, 1.5, 1 / 24)
    b.set_shift_field(uni)
    a.init(fields)
    b.init(fields)
    a.step(6)
    b.step(6)
    assert dist_err(b.distributions(), a.distributions(), 0.1).max() < 1e-13


def test_removing_the_field_restores_the_previous_form(L):
    """set_shift_field(None) gives back the zero-shift forms, bit for bit."""
    shape = (32, 16, 8)
    fields = W.add_noise(W.gauge_wave(shape, 1 / 32, 0.05), 1e-4, seed=6)
    ref = L.Lattice(3, shape, 1.5, 1 / 32, storage="f32", streaming=1)
    ref.init(fields)
    ref.step(5)
    a = L.Lattice(3, shape, 1.5, 1 / 32, storage="f32", streaming=1)
    a.set_shift_field(W.smooth_shift(shape, 1 / 32, 0.1, seed=1))
    a.set_shift_field(None)
    a.init(fields)
    a.step(5)
    assert np.array_equal(ref.distributions(), a.distributions())


def test_constraints_with_shift_field_fp64(L, oracle_mod):
    """The monitor's corrected moments carry the field's B terms: the 22
    values against the oracle at t = 0 and after 10 steps."""
    N = 16
    shape = (N, N, N)
    field = W.smooth_shift(shape, 1 / N, 0.1, seed=12)
    fields = W.add_noise(W.gauge_wave(shape, 1 / N, 0.1, direction="xyz"), 1e-4, seed=8)
    lat = L.Lattice(3, shape, 1.5, 1 / N)
    lat.set_shift_field(field)
    lat.init(fields)
    o = oracle_mod.Oracle(3, shape, 1.5, 1 / N, shift_field=field)
    f = o.init(fields)
    for n in (0, 10):
        if n:
            lat.step(n)
            f = o.run(f, n)
        g, r = lat.constraints(), o.constraints(f)
        np.testing.assert_allclose(g[:6], r[:6], rtol=1e-10, atol=0)
        np.testing.assert_allclose(g[6:], r[6:], rtol=1e-12, atol=1e-12)


def test_full_size_sampled_step_with_shift_field_fp64(L, oracle_mod):
    """128^3 D3Q19 FP64 with a constant shift plus a smooth field, one step
    from a noisy diagonal wave, sampled cells against the oracle's per-cell
    step."""
    N = 128
    shape = (N, N, N)
    field = W.smooth_shift(shape, 1 / N, 0.1, seed=21)
    fields = W.add_noise(W.gauge_wave(shape, 1 / N, 0.05, direction="xyz"), 1e-6, seed=5)
    beta = (0.05, 0.02, -0.04)
    o = oracle_mod.Oracle(3, shape, 0.9, 1 / N, shift=beta, shift_field=field)
    f0 = o.init(fields)
    lat = L.Lattice(3, shape, 0.9, 1 / N)
    lat.set_shift(beta)
    lat.set_shift_field(field)
    lat.set_distributions(f0)
    lat.step(1)
    rng = np.random.default_rng(27)
    corners = [x + N * (y + N * z) for x in (0, N - 1) for y in (0, N - 1) for z in (0, N - 1)]
    idx = np.array(corners + list(rng.integers(0, N ** 3, size=120)), dtype=np.int64)
    got = lat.cells_distributions(idx)
    ref = o.step_cells(f0, idx)
    scale = np.abs(ref).max(axis=(0, 2))
    assert (np.abs(got - ref).max(axis=(0, 2)) / scale).max() < TOL64


@pytest.mark.parametrize("storage", ["dev_f32", "f32", "dev_bf16"])
def test_reduced_precision_shift_field_within_stated_bound(L, oracle_mod, storage):
    """Sheared gauge wave (A = 0.01), D2Q9 128^2, tau 1.5: each storage
    against the FP64 oracle after 1 and 10 steps, within the stated bound
    (3D constants, amplification of the D1Q3 step at shift 0.1)."""
    N, tau, A, v0 = 128, 1.5, 0.01, 0.1
    shape = (N, N, 1)
    field = W.shear_shift(shape, 1 / N, v0)
    fields = W.sheared_gauge_wave(shape, 1 / N, A, v0)
    lam = amplification(oracle_mod, tau, (v0, 0.0, 0.0))
    o = oracle_mod.Oracle(2, shape, tau, 1 / N, shift_field=field)
    f = o.init(fields)
    lat = L.Lattice(2, shape, tau, 1 / N, storage=storage)
    lat.set_shift_field(field)
    lat.init(fields)
    done = 0
    for n in (1, 10):
        lat.step(n - done)
        f = o.run(f, n - done)
        done = n
        lat.status()
        err = float(np.abs(lat.moments() - o.moments(f)).max() / A)
        assert err <= bound(storage, True, N, tau, n, lam), (n, err)


def test_full_size_256_cubed_shift_field_fp32_against_fp64(L, oracle_mod):
    """The benchmark's shift-field workload at full size: 256^3 D3Q19, shift
    (0.05, 0.02, -0.02) plus the divergence-free shear field of amplitude
    0.02, gauge wave A = 0.01, tau 4.5. The FP64 run (the same kernels held to
    1e-12 of the oracle above) is the reference: after 1 and 2 steps the FP32
    run is within the FP32 bound of it, on every cell."""
    N, tau, A = 256, 4.5, 0.01
    beta = (0.05, 0.02, -0.02)
    shape = (N, N, N)
    field = W.shear_shift3(shape, 1 / N, 0.02)
    fields = W.gauge_wave(shape, 1 / N, A, beta=beta)
    lam = amplification(oracle_mod, tau, (0.09, 0.0, 0.0))  # |beta| + field amplitude
    runs = {}
    for storage in ("f64", "f32"):
        lat = L.Lattice(3, shape, tau, 1 / N, storage=storage, streaming=1)
        lat.set_shift(beta)
        lat.set_shift_field(field)
        lat.init(fields)
        out = []
        for _ in range(2):
            lat.step(1)
            lat.status()
            out.append(lat.moments())
        runs[storage] = out
        lat.close()
    for n in (1, 2):
        err = float(np.abs(runs["f32"][n - 1] - runs["f64"][n - 1]).max() / A)
        assert err <= bound("f32", True, N, tau, n, lam), (n, err)


@pytest.mark.parametrize("storage", ["f32", "dev_f32", "dev_bf16"])
def test_shift_field_aa_equals_pingpong(L, storage):
    """The shift-field form in place (AA, both parities) against ping-pong, in
    each reduced storage: the same arithmetic, to a few rounding units."""
    shape = (20, 12, 8)
    beta = (0.05, -0.02, 0.03)
    field = W.smooth_shift(shape, 1 / 20, 0.05, seed=31)
    fields = W.add_noise(W.gauge_wave(shape, 1 / 20, 0.05, beta=beta), 1e-4, seed=32)
    tol = {"f32": 1e-5, "dev_f32": 1e-5, "dev_bf16": 3e-2}[storage]
    lats = []
    for streaming in (1, 2):
        lat = L.Lattice(3, shape, 1.2, 1 / 20, storage=storage, streaming=streaming)
        lat.set_shift(beta)
        lat.set_shift_field(field)
        lat.init(fields)
        lats.append(lat)
    for n in (1, 2, 3):
        for lat in lats:
            lat.step(n)
        a, b = lats[0].distributions(), lats[1].distributions()
        assert dist_err(b, a, 0.05 * math.pi).max() < tol, (storage, n)
