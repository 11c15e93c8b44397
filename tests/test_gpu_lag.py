"""The LAG derivative mode (reading R17: A_k and D_kij from the previous
step's corrected alpha and gamma, the initial fields at the first step) on
the GPU against the oracle's LAG step. In this mode the collide kernel
writes the next step's stencil planes itself and no moment pass runs.

FP64: 1e-12 relative per field (distributions, corrected moments and the
lagged fields), or 4 x the oracle's own one-ulp spread where the method's
conditioning is worse. Reduced precision: one step from the GPU's stored
state (distributions and lagged fields), within the derived bound of
onestep_bound.py, in every launch form.
"""
import math

import numpy as np
import pytest

from onestep_bound import field_max_err, first_order_max, one_step_bound
from paper_1505_02037_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
KV_FLOOR = 1e-3


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02037_gb300 import lbnr
    lbnr.library()
    return lbnr


def rel_err(g, o, kscale, nf=16):
    g = g.reshape(nf, -1)
    o = o.reshape(nf, -1)
    floor = np.array(([1.0] * 7 + [kscale] * 9)[:nf])
    return np.abs(g - o).max(axis=1) / np.maximum(np.abs(o).max(axis=1), floor)


def dist_err(g, o, kscale):
    g = g.reshape(16, -1)
    o = o.reshape(16, -1)
    floor = np.array([1.0] * 7 + [kscale] * 9) / 3
    return np.abs(g - o).max(axis=1) / np.maximum(np.abs(o).max(axis=1), floor)


def perturbed(f, seed=0):
    rng = np.random.default_rng(seed)
    return f * (1 + rng.choice([-1.0, 1.0], size=f.shape) * 2.2e-16)


def bar(spread):
    return max(TOL64, 4 * spread)


def smooth_state(shape, dx, seed):
    return W.add_noise(W.smooth_modes(shape, dx, 0.03, seed=seed), 1e-4, seed=seed + 1)


@pytest.mark.parametrize("vset,shape", [(1, (333, 1, 1)), (2, (37, 23, 1)), (3, (21, 13, 11)),
                                        (3, (64, 5, 3)), (3, (2, 5, 3))])
@pytest.mark.parametrize("streaming", [1, 2])
def test_lag_every_form_fp64(L, oracle_mod, vset, shape, streaming):
    """A smooth seeded state with noise, lagged fields one step behind it
    (the oracle's own LAG step from the initial fields), 3 more steps in
    every launch form: distributions, corrected moments and lagged fields."""
    dx = 1 / shape[0]
    o = oracle_mod.Oracle(vset, shape, 0.9, dx, deriv_mode=1)
    f0, p0 = o.step_lag(*o.lag_init(smooth_state(shape, dx, 40 + vset)))
    lat = L.Lattice(vset, shape, 0.9, dx, streaming=streaming, deriv_mode="lag")
    assert lat.deriv_mode == 1
    for v, name in enumerate(lat.variants):
        lat.set_variant(v)
        lat.set_distributions(f0)
        lat.set_lagged(p0)
        assert rel_err(lat.lagged(), p0, KV_FLOOR, 7).max() < 1e-15
        f, p, fp, pp = f0, p0, perturbed(f0), p0
        for n in range(3):
            lat.step(1)
            f, p = o.step_lag(f, p)
            fp, pp = o.step_lag(fp, pp)
            sd = dist_err(fp, f, KV_FLOOR).max()
            sm = rel_err(o.moments_lag(fp, pp), o.moments_lag(f, p), KV_FLOOR).max()
            sp = rel_err(pp, p, KV_FLOOR, 7).max()
            ed = dist_err(lat.distributions(), f, KV_FLOOR).max()
            em = rel_err(lat.moments(), o.moments_lag(f, p), KV_FLOOR).max()
            ep = rel_err(lat.lagged(), p, KV_FLOOR, 7).max()
            assert ed <= bar(sd), (name, n, ed, sd)
            assert em <= bar(sm), (name, n, em, sm)
            assert ep <= bar(sp), (name, n, ep, sp)
    lat.close()


@pytest.mark.parametrize("streaming", [1, 2])
def test_lag_diagonal_gauge_wave_from_init_fp64(L, oracle_mod, streaming):
    """The gauge wave along the (1,1,1) diagonal on 32^3 with seeded noise
    (so that the constraints are not zero), the first step's derivatives from
    the initial fields, 20 steps, every launch form, and the constraint
    monitor at the end."""
    N, A, tau = 32, 0.1, 1.5
    shape = (N, N, N)
    fields = W.add_noise(W.gauge_wave(shape, 1 / N, A, direction="xyz"), 1e-4, seed=21)
    o = oracle_mod.Oracle(3, shape, tau, 1 / N, deriv_mode=1)
    f0, p0 = o.lag_init(fields)
    f, p = o.run_lag(f0, p0, 20)
    fp, pp = o.run_lag(perturbed(f0), p0, 20)
    kscale = math.pi * A
    spread = rel_err(o.moments_lag(fp, pp), o.moments_lag(f, p), kscale).max()
    ref_c = o.constraints_lag(f, p)
    lat = L.Lattice(3, shape, tau, 1 / N, streaming=streaming, deriv_mode="lag")
    for v, name in enumerate(lat.variants):
        lat.set_variant(v)
        lat.init(fields)
        lat.step(20)
        em = rel_err(lat.moments(), o.moments_lag(f, p), kscale).max()
        assert em <= bar(spread), (name, em, spread)
    # constraint norms: 1e-10 relative; lattice sums: 1e-12 of the sum of the
    # magnitudes summed (a sum of values near zero, as for V, is no better
    # conditioned than that); either, or 4 x the oracle's one-ulp spread
    c = lat.constraints()
    spread_c = np.abs(o.constraints_lag(fp, pp) - ref_c)
    scale = np.concatenate([1e-10 * np.abs(ref_c[:6]),
                            1e-12 * np.abs(f.sum(axis=1)).sum(axis=1)])
    tol = np.maximum(scale, 4 * spread_c) + 1e-14
    bad = np.flatnonzero(np.abs(c - ref_c) > tol)
    assert bad.size == 0, [(int(i), c[i] - ref_c[i], tol[i]) for i in bad]
    lat.close()


def test_lag_checkpoint_resume_is_bitwise(L):
    """Distributions plus lagged fields are a LAG run's whole state."""
    shape = (64, 6, 5)
    fields = W.add_noise(W.gauge_wave(shape, 1 / 64, 0.05), 1e-5, seed=9)
    a = L.Lattice(3, shape, 2.0, 1 / 64, deriv_mode="lag")
    a.init(fields)
    a.step(7)
    f, p = a.distributions(), a.lagged()
    a.step(9)
    b = L.Lattice(3, shape, 2.0, 1 / 64, deriv_mode="lag")
    b.init(fields)
    b.step(7)  # same step parity as a
    b.set_distributions(f)
    b.set_lagged(p)
    b.step(9)
    assert np.array_equal(a.distributions(), b.distributions())
    assert np.array_equal(a.lagged(), b.lagged())


def test_lag_calls_are_refused_under_sync(L):
    lat = L.Lattice(1, (16, 1, 1), 1.0, 1 / 16)
    lat.init(W.flat((16, 1, 1)))
    with pytest.raises(L.LbnrError) as e:
        lat.lagged()
    assert e.value.code == -6


REDUCED = ["f32", "dev_f32", "dev_f16", "dev_bf16"]


@pytest.mark.parametrize("storage", REDUCED)
@pytest.mark.parametrize("vset,shape", [(2, (45, 29, 1)), (3, (37, 9, 5)), (3, (64, 9, 5))])
@pytest.mark.parametrize("streaming", [1, 2])
def test_lag_every_form_reduced_precision_one_step(L, oracle_mod, storage, vset, shape,
                                                   streaming):
    """Two single LAG steps in every form, each from the GPU's stored
    distributions and lagged fields, against the oracle's LAG step from the
    same values, within the derived one-step bound."""
    Q = {1: 3, 2: 9, 3: 19}[vset]
    c, w = oracle_mod.velocity_set(vset)
    tau, dx = 0.8, 1 / shape[0]
    o = oracle_mod.Oracle(vset, shape, tau, dx, deriv_mode=1)
    f0, p0 = o.step_lag(*o.lag_init(smooth_state(shape, dx, 60 + vset)))
    lat = L.Lattice(vset, shape, tau, dx, storage=storage, streaming=streaming, deriv_mode="lag")
    for v, name in enumerate(lat.variants):
        lat.set_variant(v)
        lat.set_distributions(f0)
        lat.set_lagged(p0)
        f_in, p_in = lat.distributions(), lat.lagged()
        for n in range(2):
            lat.step(1)
            ref, _ = o.step_lag(f_in, p_in)
            got = lat.distributions()
            rho = o.moments_lag(f_in, p_in)
            m1 = first_order_max(rho.reshape(16, *shape[::-1]), dx, vset)
            b = one_step_bound(storage, c, w, tau, dx, f_in, ref, rho[0].max(), m1)
            err = field_max_err(got, ref)
            bad = np.flatnonzero(err > b)
            assert bad.size == 0, (name, n, [(int(F), err[F], b[F]) for F in bad])
            f_in, p_in = got, lat.lagged()
    lat.close()
