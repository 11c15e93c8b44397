"""Host-side checks of the C-ABI library that need no GPU: it builds, loads,
exports every entry point include/lbnr.h declares, and rejects bad
arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "lbnr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(lbnr_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1505_02037_gb300 import lbnr
    return lbnr.library()


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert "lbnr_step" in names and "lbnr_create" in names
    for n in names:
        assert hasattr(lib, n), n


def test_default_opts(lib):
    from paper_1505_02037_gb300 import lbnr
    o = lbnr.lbnr_default_opts()
    assert (o.slicing, o.storage, o.streaming, o.sources_on) == (1, 0, 0, 1)
    assert o.dev_buffer is None and o.cuda_stream is None


@pytest.mark.parametrize("vset,shape,storage,streaming,expect", [
    (3, (128, 128, 128), 1, 1, 2 * 16 * 19 * 4 * 128 ** 3),
    (3, (128, 128, 128), 1, 2, 16 * 19 * 4 * 128 ** 3),
    (1, (200, 1, 1), 0, 1, 2 * 16 * 3 * 8 * 224),   # planes padded to 32 cells
    (2, (64, 48, 1), 3, 2, 16 * 9 * 2 * 64 * 48),
])
def test_workspace_bytes(vset, shape, storage, streaming, expect):
    """The workspace holds the distribution buffer(s) (planes padded to a
    multiple of 32 cells for the tensor copies) plus the stencil planes, the
    FP64 field planes and the reduction scratch."""
    from paper_1505_02037_gb300 import lbnr
    o = lbnr.lbnr_default_opts()
    o.storage, o.streaming = storage, streaming
    n = lbnr.lbnr_workspace_bytes(lbnr.Grid(*shape), vset, o)
    cells = shape[0] * shape[1] * shape[2]
    aux = 7 * cells * (8 if storage == 0 else 4)
    extra = aux + 16 * cells * 8 + 7 * cells * 8 + ((cells + 127) // 128) * 22 * 8 + (1 << 20)
    assert expect + extra <= n <= expect + extra + 10 * 256 + 1024


@pytest.mark.parametrize("vset,shape,tau,dx,dt,storage", [
    (1, (200, 2, 1), 0.6, 0.005, 0.005, 0),   # D1Q3 with ny > 1
    (2, (16, 16, 2), 0.6, 0.1, 0.1, 0),       # D2Q9 with nz > 1
    (3, (0, 4, 4), 0.6, 0.1, 0.1, 0),         # empty lattice
    (3, (4, 4, 4), 0.5, 0.1, 0.1, 0),         # tau = 1/2
    (3, (4, 4, 4), 0.7, 0.1, 0.2, 0),         # dt != dx
    (3, (4, 4, 4), 0.7, -0.1, -0.1, 0),       # negative spacing
    (3, (4, 4, 4), 0.7, 0.1, 0.1, 9),         # unknown storage
    (4, (4, 4, 4), 0.7, 0.1, 0.1, 0),         # unknown set
])
def test_create_rejects_bad_arguments_before_the_device(vset, shape, tau, dx, dt, storage):
    from paper_1505_02037_gb300 import lbnr
    o = lbnr.lbnr_default_opts()
    o.storage = storage
    with pytest.raises(lbnr.LbnrError) as e:
        lbnr.lbnr_create(lbnr.Grid(*shape), vset, tau, dx, dt, o)
    assert e.value.code == -1


def test_null_context_calls_fail_cleanly(lib):
    from paper_1505_02037_gb300 import lbnr
    assert lib.lbnr_step(None, 1) == -1
    assert lib.lbnr_status(None) == -1
    assert lib.lbnr_steps_done(None) == -1
    lib.lbnr_destroy(None)
    assert lib.lbnr_last_error(None)


def test_default_batch_opts(lib):
    from paper_1505_02037_gb300 import lbnr
    o = lbnr.lbnr_default_batch_opts()
    assert (o.storage, o.block, o.ctas_per_sm, o.sources_on) == (2, 256, 0, 1)
    assert o.wait_limit_ns == 2_000_000_000 and o.test_drop_arrival_run == -1


def _run(vset=1, shape=(64, 1, 1), tau=1.0, dx=1 / 64, steps=10, slicing=1):
    from paper_1505_02037_gb300 import lbnr
    return lbnr.RunDesc(vset, slicing, lbnr.Grid(*shape), tau, dx, steps)


@pytest.mark.parametrize("bad,storage", [
    (dict(vset=3, shape=(8, 8, 8)), 2),       # batched runs are 1D or 2D
    (dict(vset=1, shape=(64, 2, 1)), 2),      # D1Q3 with ny > 1
    (dict(vset=2, shape=(16, 16, 2)), 2),     # nz > 1
    (dict(shape=(0, 1, 1)), 2),               # empty
    (dict(tau=0.5), 2),                       # tau = 1/2
    (dict(dx=0.0), 2),                        # dx = 0
    (dict(steps=-1), 2),                      # negative step count
    (dict(slicing=3), 2),                     # unknown slicing
    (dict(vset=2, shape=(20000, 20000, 1)), 2),  # more than 2^28 cells
    (dict(), 7),                              # unknown storage
])
def test_batch_create_rejects_bad_runs_before_the_device(bad, storage):
    from paper_1505_02037_gb300 import lbnr
    o = lbnr.lbnr_default_batch_opts()
    o.storage = storage
    runs = [_run(), _run(**bad)]
    with pytest.raises(lbnr.LbnrError) as e:
        lbnr.lbnr_batch_create(runs, o)
    assert e.value.code == -1


def test_null_batch_calls_fail_cleanly(lib):
    assert lib.lbnr_batch_run(None, 1) == -1
    assert lib.lbnr_batch_status(None, None) == -1
    assert lib.lbnr_batch_steps_done(None, 0) == -1
    assert lib.lbnr_batch_plan(None, None, None, None, None) == -1
    lib.lbnr_batch_destroy(None)


def test_set_fluid_rejects_bad_arguments(lib):
    assert lib.lbnr_set_fluid(None, 0.1, 1.0, 1.0) == -1


def test_set_shift_rejects_a_null_context(lib):
    assert lib.lbnr_set_shift(None, 0.1, 0.0, 0.0) == -1
    assert lib.lbnr_set_shift(None, float("nan"), 0.0, 0.0) == -1
    assert lib.lbnr_set_shift_field(None, None) == -1


@pytest.mark.parametrize("vset,shape", [
    (3, (1291, 1291, 1291)),   # 2.15e9 cells: past the 2^31 cell limit
    (3, (610, 610, 610)),      # 19 planes x 227M cells: plane offsets past 2^32
    (2, (65536, 32768, 1)),    # 2^31 cells on the 2D lattice
    (1, (2 ** 31, 1, 1)),      # and on the 1D lattice
])
def test_create_rejects_lattices_beyond_the_index_limits(vset, shape):
    """All in-block offsets are 32-bit: lattices with 2^31 cells or more, or
    with Q x (cells padded to 32) of 2^32 or more, are refused before any
    device memory is touched."""
    from paper_1505_02037_gb300 import lbnr
    o = lbnr.lbnr_default_opts()
    o.streaming = lbnr.LBNR_STREAM_PINGPONG
    with pytest.raises(lbnr.LbnrError) as e:
        lbnr.lbnr_workspace_bytes(lbnr.Grid(*shape), vset, o)
    assert e.value.code == -1
    with pytest.raises(lbnr.LbnrError) as e:
        lbnr.lbnr_create(lbnr.Grid(*shape), vset, 1.0, 0.1, 0.1, o)
    assert e.value.code == -1


def test_largest_accepted_lattice_has_a_workspace_size():
    """Just inside the limits the workspace size is computed (no device
    needed): 600^3 D3Q19 in one AA buffer."""
    from paper_1505_02037_gb300 import lbnr
    o = lbnr.lbnr_default_opts()
    o.storage, o.streaming = 1, lbnr.LBNR_STREAM_AA
    n = lbnr.lbnr_workspace_bytes(lbnr.Grid(600, 600, 600), 3, o)
    assert n >= 16 * 19 * 4 * 600 ** 3


@pytest.mark.parametrize("vset,shape,tau,dx,dt,slicing,storage", [
    (3, (8, 8, 8), 1.0, 0.1, 0.1, 1, 2),      # deviation storage: not offered
    (3, (8, 8, 8), 1.0, 0.1, 0.2, 1, 0),      # dt != dx
    (3, (8, 8, 8), 0.5, 0.1, 0.1, 1, 0),      # tau <= 1/2
    (1, (8, 2, 1), 1.0, 0.1, 0.1, 1, 0),      # D1Q3 with ny > 1
    (4, (8, 8, 8), 1.0, 0.1, 0.1, 1, 0),      # unknown velocity set
    (3, (8, 8, 8), 1.0, 0.1, 0.1, 3, 1),      # unknown slicing
    (3, (1291, 1291, 1291), 1.0, 0.1, 0.1, 1, 1),  # past the 32-bit index limits
])
def test_ad_create_rejects_bad_arguments_before_the_device(lib, vset, shape, tau, dx, dt,
                                                           slicing, storage):
    """The 37-field context refuses bad arguments with LBNR_EINVAL before any
    CUDA call (no GPU here)."""
    from paper_1505_02037_gb300 import lbnr
    out = ctypes.c_void_p()
    g = lbnr.Grid(*shape)
    rc = lib.lbnr_ad_create(ctypes.byref(g), vset, tau, dx, dt, slicing, storage, None,
                            ctypes.byref(out))
    assert rc == -1 and not out.value


def test_ad_null_calls_fail_cleanly(lib):
    assert lib.lbnr_ad_step(None, 1) == -1
    assert lib.lbnr_ad_status(None) == -1
    assert lib.lbnr_ad_moments(None, None) == -1
    assert lib.lbnr_ad_steps_done(None) == -1
    lib.lbnr_ad_destroy(None)
