"""The largest configuration: a linearised plane wave along the (1,1,1)
diagonal on a periodic 384^3 D3Q19 lattice (56.6 M cells), FP32 deviation
storage, in-place AA streaming (one 68.9 GB buffer; ping-pong would take two),
tau = 0.55, A = 1e-6, geodesic slicing; and the same lattice seeded with
uniform noise of amplitude 1e-10 on every field.

A whole 384^3 state in FP64 would take 137 GB on the host, so the oracle checks
sampled cells through patches. The new value of a cell depends only on cells
within distance 2 (the streaming source and that source's derivative
stencil). So the centre of a periodic 5x5x5 patch, filled from the GPU's state
around the cell, steps exactly as it does in the full lattice.
"""
import math

import numpy as np
import pytest

from paper_1505_02037_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = 384
TAU = 0.55
A = 1e-6


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02037_gb300 import lbnr
    lbnr.library()
    free, _ = torch.cuda.mem_get_info()
    if free < 90e9:
        pytest.skip("needs about 85 GB of free device memory")
    return lbnr


def patch_indices(c, n=N, r=2):
    x, y, z = c % n, (c // n) % n, c // (n * n)
    w = 2 * r + 1
    out = np.empty(w ** 3, dtype=np.int64)
    for k in range(w):
        for j in range(w):
            for i in range(w):
                out[i + w * (j + w * k)] = ((x + i - r) % n) + n * (((y + j - r) % n) +
                                                                   n * ((z + k - r) % n))
    return out


def samples(seed=2037, count=20):
    rng = np.random.default_rng(seed)
    corners = [x + N * (y + N * z) for x in (0, N - 1) for y in (0, N - 1) for z in (0, N - 1)]
    return np.array(corners + list(rng.integers(0, N ** 3, size=count)), dtype=np.int64)


def test_full_size_aa_fp32_sampled_steps(L, oracle_mod):
    """Two steps (the even and the odd AA layout) of the 384^3 run, checked at
    corner and random cells against the oracle's step of the patch around
    each. The oracle starts from the GPU's stored state, so only the step's
    FP32 arithmetic differs. Bar: the stated FP32-deviation bound for one
    step, 3 K (N / 2 pi) / tau with K = 1e-6 (D3Q19), relative to A."""
    lat = L.Lattice(3, (N, N, N), TAU, 1 / N, slicing=0, storage="dev_f32",
                    streaming=L.LBNR_STREAM_AA)
    assert lat.streaming == L.LBNR_STREAM_AA
    lat.init(W.linear_wave((N, N, N), 1 / N, A, direction="xyz"))
    idx = samples()
    patches = np.concatenate([patch_indices(c) for c in idx])
    centre = 2 + 5 * (2 + 5 * 2)
    bar = 3 * 1e-6 * (N / (2 * math.pi)) / TAU
    for _ in range(2):
        before = lat.cells_distributions(patches).reshape(len(idx), 125, 16, 19)
        lat.step(1)
        after = lat.cells_distributions(idx)
        worst = 0.0
        for s in range(len(idx)):
            f = np.ascontiguousarray(before[s].transpose(1, 2, 0)).reshape(16, 19, 5, 5, 5)
            o = oracle_mod.Oracle(3, (5, 5, 5), TAU, 1 / N, slicing=0)
            ref = o.step_cells(f, np.array([centre], dtype=np.int64))[0]
            worst = max(worst, float(np.abs(after[s] - ref).max() / A))
        assert worst <= bar, (lat.steps_done, worst, bar)
    lat.close()


def test_full_size_noise_grows_at_the_oracle_amplification(L, oracle_mod):
    """Flat space plus uniform noise of amplitude 1e-10 on all 16 fields
    (seed 2037), the configuration's stability check. The scheme is linearly
    unstable at tau = 0.55: the noise must grow. Over steps 20 to 40 its
    growth per step lies between the largest amplification factor of the
    oracle's linearised D1Q3 step (x-aligned modes, which the 3D lattice
    contains) and 2. It then overflows well before step 2000."""
    o = oracle_mod.Oracle(1, (32, 1, 1), TAU, 1 / 32)
    f0 = o.init(W.flat((32, 1, 1)))
    base = o.step(f0).reshape(-1)
    flat = f0.reshape(-1)
    J = np.zeros((flat.size, flat.size))
    for i in range(flat.size):
        g = flat.copy()
        g[i] += 1e-7
        J[:, i] = (o.step(g.reshape(f0.shape)).reshape(-1) - base) / 1e-7
    lam = float(np.abs(np.linalg.eigvals(J)).max())

    lat = L.Lattice(3, (N, N, N), TAU, 1 / N, slicing=0, storage="dev_f32",
                    streaming=L.LBNR_STREAM_AA)
    lat.init(W.add_noise(W.flat((N, N, N)), 1e-10, seed=2037))
    probe = samples(seed=11, count=4000)
    ref_state = np.array(W.flat_value())

    def amplitude():
        d = lat.cells_distributions(probe).sum(axis=2)  # zeroth moments per field
        return float(np.abs(d - ref_state[None, :]).max())

    lat.step(20)
    a20 = amplitude()
    lat.step(20)
    a40 = amplitude()
    rate = (a40 / a20) ** (1 / 20)
    assert lam * 0.97 <= rate <= 2.0, (rate, lam)
    blown = None
    for k in range(40, 2000, 20):
        lat.step(20)
        try:
            lat.status()
        except L.NonFiniteError:
            blown = k + 20
            break
    assert blown is not None and blown < 2000
    lat.close()
