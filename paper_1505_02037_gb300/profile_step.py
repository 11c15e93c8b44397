"""Runs a few lattice Boltzmann steps of one launch form, for profilers.

  python -m paper_1505_02037_gb300.profile_step --storage f32 --n 128 \
      --variant 3 --steps 4 [--vset 3] [--tau 4.5] [--streaming 1]

Prints the per-kernel milliseconds of the timed steps (CUDA events). Used to
capture ncu reports of a single kernel on a small case.
"""
from __future__ import annotations

import argparse
import sys

from . import lbnr
from . import workloads as W


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--storage", default="f32")
    p.add_argument("--n", type=int, default=128)
    p.add_argument("--variant", type=int, default=0)
    p.add_argument("--steps", type=int, default=4)
    p.add_argument("--vset", type=int, default=3)
    p.add_argument("--tau", type=float, default=4.5)
    p.add_argument("--streaming", type=int, default=1)
    a = p.parse_args(argv)
    n = a.n
    shape = (n, n, n) if a.vset == 3 else ((n, n, 1) if a.vset == 2 else (n, 1, 1))
    lat = lbnr.Lattice(a.vset, shape, a.tau, 1 / n, storage=a.storage, streaming=a.streaming)
    if a.variant >= len(lat.variants):
        print(f"no launch form {a.variant}; have {lat.variants}")
        return 2
    lat.set_variant(a.variant)
    lat.init(W.gauge_wave(shape, 1 / n, 0.1))
    lat.step(a.steps)
    lat.status()
    ms = lat.step_timed(4)
    print(f"{a.storage} n={n} vset={a.vset} {lat.variants[a.variant]}: "
          f"ms per step aux {ms[0] / 4:.4f} collide {ms[1] / 4:.4f}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
