"""Every launch form of the 16-field collide step against the oracle, on
general data (every metric component, every stencil direction), for every
velocity set and storage. The autotuner may pick any of these forms for a
run, so each one is held to the oracle, not only the default one.

FP64: 1e-12 relative per field, or 4 x the oracle's own one-ulp spread
where the method's conditioning is worse (as in test_gpu_parity.py).
Reduced precision: one step from the GPU's own stored state, against the
oracle's FP64 step from the same values, within the bound derived in
onestep_bound.py from the rounding units, Q and the stencil and relaxation
factors (Eq. numlb with the equilibria of Eqs. alfa-ekstsor and the
central-difference derivatives of Sec. "First order derivatives"). Both
streaming patterns are covered, and in place (AA) both step parities: the
even step runs the form itself, the odd step the form it hands over to.
"""
import math

import numpy as np
import pytest

from onestep_bound import field_max_err, first_order_max, one_step_bound
from paper_1505_02037_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
KV_FLOOR = 1e-3  # the random state's noise amplitude: K and V below it count as zero
REDUCED = ["f32", "dev_f32", "dev_f16", "dev_bf16"]


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


# ---------------------------------------------------------------------------
# FP64: every form at the 1e-12 bar
# ---------------------------------------------------------------------------
# Ragged lattices (a partial last tile of 32 cells) and lattices whose x
# extent is a multiple of 32 (one tile per row, and several).
SHAPES = [(1, (333, 1, 1)), (2, (37, 23, 1)), (3, (37, 9, 5)), (3, (2, 5, 3)),
          (1, (96, 1, 1)), (2, (64, 9, 1)), (3, (64, 5, 3)), (3, (32, 3, 2))]


@pytest.mark.parametrize("vset,shape", SHAPES)
@pytest.mark.parametrize("streaming", [1, 2])
def test_every_form_fp64_random_state(L, oracle_mod, vset, shape, streaming):
    """Seeded random near-flat state (every term of the step active), 3 steps
    in every launch form."""
    Q = {1: 3, 2: 9, 3: 19}[vset]
    _, w = oracle_mod.velocity_set(vset)
    f0 = W.random_distributions(Q, w, shape, seed=4000 + vset)
    o = oracle_mod.Oracle(vset, shape, 0.8, 1 / shape[0])
    lat = L.Lattice(vset, shape, 0.8, 1 / shape[0], streaming=streaming)
    assert len(lat.variants) >= 2
    for v, name in enumerate(lat.variants):
        lat.set_variant(v)
        lat.set_distributions(f0)
        f, fp = f0, perturbed(f0)
        for n in range(3):
            lat.step(1)
            f, fp = o.step(f), o.step(fp)
            sd = dist_err(fp, f, KV_FLOOR).max()
            sm = field_err(o.moments(fp), o.moments(f), KV_FLOOR).max()
            ed = dist_err(lat.distributions(), f, KV_FLOOR).max()
            em = field_err(lat.moments(), o.moments(f), KV_FLOOR).max()
            assert ed <= bar(sd), (name, n, ed, sd)
            assert em <= bar(sm), (name, n, em, sm)
    lat.close()


@pytest.mark.parametrize("vset,N,direction", [(3, 24, "xyz"), (2, 48, "xy")])
def test_every_form_fp64_diagonal_gauge_wave(L, oracle_mod, vset, N, direction):
    """The gauge wave along the lattice diagonal (every metric component and
    stencil direction active) from its closed form, 12 steps, every form."""
    A, tau = 0.1, 1.5
    shape = (N, N, N) if vset == 3 else (N, N, 1)
    fields = W.gauge_wave(shape, 1 / N, A, direction=direction)
    o = oracle_mod.Oracle(vset, shape, tau, 1 / N)
    f0 = o.init(fields)
    f, fp = o.run(f0, 12), o.run(perturbed(f0), 12)
    kscale = math.pi * A
    spread_m = field_err(o.moments(fp), o.moments(f), kscale).max()
    spread_d = dist_err(fp, f, kscale).max()
    for streaming in (1, 2):
        lat = L.Lattice(vset, shape, tau, 1 / N, streaming=streaming)
        for v, name in enumerate(lat.variants):
            lat.set_variant(v)
            lat.init(fields)
            lat.step(12)
            em = field_err(lat.moments(), o.moments(f), kscale).max()
            ed = dist_err(lat.distributions(), f, kscale).max()
            assert em <= bar(spread_m), (streaming, name, em, spread_m)
            assert ed <= bar(spread_d), (streaming, name, ed, spread_d)
        lat.close()


# ---------------------------------------------------------------------------
# Reduced precision: every form, one step at a time from the stored state
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("storage", REDUCED)
@pytest.mark.parametrize("vset,shape", [(1, (1000, 1, 1)), (2, (45, 29, 1)), (3, (37, 9, 5)),
                                        (1, (1024, 1, 1)), (2, (64, 29, 1)), (3, (64, 9, 5))])
@pytest.mark.parametrize("streaming", [1, 2])
def test_every_form_reduced_precision_one_step(L, oracle_mod, storage, vset, shape, streaming):
    """Seeded random near-flat state on ragged and row-aligned lattices; two single steps in
    every form (in place: the even and the odd layout), each against the
    oracle's step from the GPU's stored values, within the derived bound."""
    Q = {1: 3, 2: 9, 3: 19}[vset]
    c, w = oracle_mod.velocity_set(vset)
    tau, dx = 0.8, 1 / shape[0]
    f0 = W.random_distributions(Q, w, shape, seed=5000 + vset)
    o = oracle_mod.Oracle(vset, shape, tau, dx)
    lat = L.Lattice(vset, shape, tau, dx, storage=storage, streaming=streaming)
    for v, name in enumerate(lat.variants):
        lat.set_variant(v)
        lat.set_distributions(f0)
        f_in = lat.distributions()
        for n in range(2):
            lat.step(1)
            ref = o.step(f_in)
            got = lat.distributions()
            rho = o.moments(f_in)
            m1 = first_order_max(rho.reshape(16, *shape[::-1]), dx, vset)
            b = one_step_bound(storage, c, w, tau, dx, f_in, ref, rho[0].max(), m1)
            err = field_max_err(got, ref)
            bad = np.flatnonzero(err > b)
            assert bad.size == 0, (name, n, [(int(F), err[F], b[F]) for F in bad])
            f_in = got
    lat.close()


# ---------------------------------------------------------------------------
# Full size: 256^3, every reduced form, diagonal gauge wave, sampled cells
# ---------------------------------------------------------------------------
N_FULL = 256


@pytest.fixture(scope="module")
def diagonal_fields():
    return W.gauge_wave((N_FULL,) * 3, 1 / N_FULL, 0.01, direction="xyz")


def patch_indices(c, n=N_FULL, r=2):
    x, y, z = c % n, (c // n) % n, c // (n * n)
    w = 2 * r + 1
    out = np.empty(w ** 3, dtype=np.int64)
    for k in range(w):
        for j in range(w):
            for i in range(w):
                out[i + w * (j + w * k)] = ((x + i - r) % n) + n * (((y + j - r) % n) +
                                                                   n * ((z + k - r) % n))
    return out


def samples(seed, count=12):
    n = N_FULL
    rng = np.random.default_rng(seed)
    corners = [x + n * (y + n * z) for x in (0, n - 1) for y in (0, n - 1) for z in (0, n - 1)]
    edges = [31 + n * 5, 32 + n * (n - 1), 224 + n * (7 + n * 100)]  # tile edges along x
    return np.array(corners + edges + list(rng.integers(0, n ** 3, size=count)), dtype=np.int64)


@pytest.mark.parametrize("storage", REDUCED)
@pytest.mark.parametrize("streaming", [1, 2])
def test_every_form_full_size_diagonal_wave(L, oracle_mod, diagonal_fields, storage, streaming):
    """The precision configuration's lattice (256^3 D3Q19) with the gauge
    wave along the (1,1,1) diagonal, A = 0.01, tau = 1.5, in every launch
    form: two steps (in place: both layouts), each checked at corner, tile-
    edge and random cells against the oracle's step of the 5x5x5 periodic
    patch around the cell, filled from the GPU's stored state (the new value
    of a cell depends only on cells within distance 2)."""
    N, tau = N_FULL, 1.5
    c, w = oracle_mod.velocity_set(3)
    lat = L.Lattice(3, (N, N, N), tau, 1 / N, storage=storage, streaming=streaming)
    idx = samples(seed=31 + streaming)
    patches = np.concatenate([patch_indices(i) for i in idx])
    centre = 2 + 5 * (2 + 5 * 2)
    o = oracle_mod.Oracle(3, (5, 5, 5), tau, 1 / N)
    for v, name in enumerate(lat.variants):
        lat.set_variant(v)
        lat.init(diagonal_fields)
        for n in range(2):
            before = lat.cells_distributions(patches).reshape(len(idx), 125, 16, 19)
            lat.step(1)
            after = lat.cells_distributions(idx)                    # [n][16][19]
            f_in = np.ascontiguousarray(before.transpose(2, 3, 0, 1))  # [16][19][n][125]
            refs = np.empty((len(idx), 16, 19))
            for s in range(len(idx)):
                fp = np.ascontiguousarray(before[s].transpose(1, 2, 0)).reshape(16, 19, 125)
                refs[s] = o.step_cells(fp, np.array([centre], dtype=np.int64))[0]
            mom = f_in.sum(axis=1)                                   # [16][n][125]
            amax = float(mom[0].max())                               # largest lapse
            m1 = max(first_order_max(mom[:, s].reshape(16, 5, 5, 5), 1 / N, 3, periodic=False)
                     for s in range(len(idx)))
            b = one_step_bound(storage, c, w, tau, 1 / N, f_in.reshape(16, 19, -1),
                               np.ascontiguousarray(refs.transpose(1, 2, 0)), amax, m1)
            err = field_max_err(after.transpose(1, 2, 0), refs.transpose(1, 2, 0))
            bad = np.flatnonzero(err > b)
            assert bad.size == 0, (name, n, [(int(F), err[F], b[F]) for F in bad])
    lat.close()


@pytest.mark.parametrize("storage", ["f32", "dev_f32", "dev_bf16", "dev_f16"])
@pytest.mark.parametrize("streaming", [1, 2])
@pytest.mark.parametrize("deriv", ["sync", "lag"])
def test_block_shapes_of_the_word_form_are_bitwise_equal(L, storage, streaming, deriv):
    """The word form's block shapes (P1-reread, -64x4, -128x2) run the same
    code in different launch configurations: three steps from the same state
    give the same bits, in both streaming patterns and derivative modes."""
    shape = (67, 19, 7)  # a ragged last tile
    dx = 1 / shape[0]
    fields = W.add_noise(W.smooth_modes(shape, dx, 0.03, seed=5), 1e-4, seed=6)
    lat = L.Lattice(3, shape, 0.8, dx, storage=storage, streaming=streaming, deriv_mode=deriv)
    shapes = [v for v, name in enumerate(lat.variants)
              if name == "P1-reread" or name.startswith("P1-reread-")]
    assert len(shapes) >= 2, lat.variants
    ref = None
    for v in shapes:
        lat.set_variant(v)
        lat.init(fields)
        lat.step(3)
        got = (lat.distributions(), lat.lagged() if deriv == "lag" else None)
        if ref is None:
            ref = got
            continue
        assert np.array_equal(got[0], ref[0]), lat.variants[v]
        if deriv == "lag":
            assert np.array_equal(got[1], ref[1]), lat.variants[v]
    lat.close()
