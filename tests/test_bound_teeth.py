"""The derived one-step reduced-precision bound (onestep_bound.py) must not
be vacuous: planted mistakes of the kind a launch form could make (a value
streamed to the wrong neighbour, two K_ij components or two V_k components
exchanged) must exceed it by a wide margin on the states the GPU tests use.
Runs on the oracle only."""
import numpy as np
import pytest

from onestep_bound import field_max_err, first_order_max, one_step_bound
from paper_1505_02037_gb300 import workloads as W

MARGIN = 20


@pytest.mark.parametrize("vset,shape", [(1, (1000, 1, 1)), (2, (45, 29, 1)), (3, (37, 9, 5))])
@pytest.mark.parametrize("storage", ["f32", "dev_f32", "dev_f16", "dev_bf16"])
def test_planted_mistakes_exceed_the_bound(oracle_mod, vset, shape, storage):
    Q = {1: 3, 2: 9, 3: 19}[vset]
    c, w = oracle_mod.velocity_set(vset)
    nx, ny, nz = shape
    f0 = W.random_distributions(Q, w, shape, seed=5000 + vset)
    o = oracle_mod.Oracle(vset, shape, 0.8, 1 / nx)
    ref = o.step(f0)
    rho = o.moments(f0)
    b = one_step_bound(storage, c, w, 0.8, 1 / nx, f0, ref, rho[0].max(),
                       first_order_max(rho.reshape(16, nz, ny, nx), 1 / nx, vset))
    wrong = ref.copy().reshape(16, Q, nz, ny, nx)
    l = 3 if ny > 1 else 1  # a velocity along y (along x in 1D)
    wrong[:, l] = np.roll(wrong[:, l], 1, axis=2 if ny > 1 else 3)
    for planted in (wrong.reshape(16, Q, -1), ref[[0, 1, 2, 3, 4, 5, 6, 7, 9, 8] + list(range(10, 16))],
                    ref[list(range(13)) + [14, 13, 15]]):
        e = field_max_err(planted, ref)
        assert (e / b).max() > MARGIN, (e / b).max()
