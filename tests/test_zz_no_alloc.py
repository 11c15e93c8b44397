"""The allocation-free constraint-norm entry point against lbnr_constraints.

Some callers cannot allocate device memory (a run whose lattice fills the
GPU, or a framework whose allocator owns the device during its step);
lbnr_constraint_norms_noalloc serves them with per-block partials kept in a
fixed array inside the library. This file is collected last so that a run
stopping at the first failure has already run every other test, and it must
pass both alone and after the others (the shared array keeps the contents of
earlier calls).
"""
import math

import numpy as np
import pytest

from paper_1505_02037_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02037_gb300 import lbnr
    lbnr.library()
    return lbnr


@pytest.mark.parametrize("vset,shape", [(3, (20, 20, 20)), (2, (48, 48, 1)), (1, (300, 1, 1)),
                                        (3, (128, 128, 128))])
def test_noalloc_norms_match_constraints_twice(L, vset, shape):
    import torch
    N = shape[0]
    direction = {3: "xyz", 2: "xy", 1: "x"}[vset]
    fields = W.add_noise(W.gauge_wave(shape, 1 / N, 0.1, direction=direction), 1e-4, seed=8)
    lat = L.Lattice(vset, shape, 1.5, 1 / N)
    lat.init(fields)
    lat.step(7)
    expect = lat.constraints()[:6]
    d_fields = torch.from_numpy(lat.moments()).to("cuda")
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    results = []
    for _ in range(2):
        out.fill_(math.nan)
        L.lbnr_constraint_norms_noalloc(vset, L.Grid(*shape), 1 / N, d_fields, out,
                                        stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        results.append(out.cpu().numpy().copy())
    for r in results:
        np.testing.assert_allclose(r, expect, rtol=1e-12, atol=0)
    lat.close()


@pytest.mark.parametrize("vset,shape", [
    (3, (160, 160, 160)),               # 4,096,000 cells > 2^21
    (1, (2 ** 21 + 1, 1, 1)),           # one cell past the limit along one axis
    (3, (2 ** 21, 2 ** 21, 2 ** 21)),   # each side at the limit; the product is 2^63
])
def test_noalloc_rejects_lattices_beyond_its_array(L, vset, shape):
    """Sizes past the array are refused before anything is launched (the
    pointers given here are too small for the lattice and are never read)."""
    import ctypes

    import torch
    big = L.Grid(*shape)
    d = torch.empty(16, dtype=torch.float64, device="cuda")
    out = torch.empty(6, dtype=torch.float64, device="cuda")
    rc = L.library().lbnr_constraint_norms_noalloc(
        vset, ctypes.byref(big), 1 / shape[0], ctypes.c_void_p(d.data_ptr()),
        ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
    assert "LBNR_NOALLOC_MAX_CELLS" in L.library().lbnr_last_error(None).decode()
