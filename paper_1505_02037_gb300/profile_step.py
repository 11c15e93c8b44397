"""Runs a few lattice Boltzmann steps of one launch form, for profilers.

  python -m paper_1505_02037_gb300.profile_step --storage f32 --n 128 \
      --variant 3 --steps 4 [--vset 3] [--tau 4.5] [--streaming 1] [--shift 0.25,0.1,-0.2]
  python -m paper_1505_02037_gb300.profile_step --ad --storage f32 --n 128 --steps 4 \
      [--variant FORM]
  python -m paper_1505_02037_gb300.profile_step --batch 16 --vset 2 --n 256 \
      --storage dev_f32 --steps 16 [--block 256 --per-sm 1]

Prints the per-kernel milliseconds of the timed steps (CUDA events). Used to
capture ncu reports of a single kernel on a small case. With --batch R the
batched ensemble kernel advances R copies of the wave (tau 2.0) by --steps
steps in each of four launches. With --shift the lattice carries that
constant shift and runs the shift-carrying launch form (--variant is ignored);
--shift-field AMP adds the static shear shift field of that amplitude (its
own form).
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
    p.add_argument("--variant", default="0", help="launch form: index or name")
    p.add_argument("--steps", type=int, default=4)
    p.add_argument("--vset", type=int, default=3)
    p.add_argument("--tau", type=float, default=4.5)
    p.add_argument("--streaming", type=int, default=1)
    p.add_argument("--batch", type=int, default=0)
    p.add_argument("--block", type=int, default=256)
    p.add_argument("--per-sm", type=int, default=1)
    p.add_argument("--shift", default=None, help="bx,by,bz")
    p.add_argument("--ad", action="store_true",
                   help="the 37-field scheme (A_k and D_kij evolved); f64 or f32 storage")
    p.add_argument("--shift-field", type=float, default=0.0,
                   help="amplitude of a static shear shift field")
    p.add_argument("--deriv", default="sync", choices=["sync", "lag"],
                   help="time level of A and D (lag: one kernel per step)")
    p.add_argument("--amplitude", type=float, default=0.1,
                   help="gauge-wave amplitude A (0: flat space)")
    a = p.parse_args(argv)
    if a.batch:
        return batch_main(a)
    if a.ad:
        return ad_main(a)
    n = a.n
    shape = (n, n, n) if a.vset == 3 else ((n, n, 1) if a.vset == 2 else (n, 1, 1))
    lat = lbnr.Lattice(a.vset, shape, a.tau, 1 / n, storage=a.storage, streaming=a.streaming,
                       deriv_mode=a.deriv)
    v = lat.variants.index(a.variant) if a.variant in lat.variants else (
        int(a.variant) if a.variant.isdigit() else -1)
    if not 0 <= v < len(lat.variants):
        print(f"no launch form {a.variant}; have {lat.variants}")
        return 2
    lat.set_variant(v)
    beta = tuple(float(v) for v in a.shift.split(",")) if a.shift else None
    if beta:
        lat.set_shift(beta)
    if a.shift_field:
        lat.set_shift_field(W.shear_shift3(shape, 1 / n, a.shift_field))
    lat.init(W.gauge_wave(shape, 1 / n, a.amplitude, beta=beta))
    lat.step(a.steps)
    lat.status()
    ms = lat.step_timed(4)
    form = ("P1-reread-shiftfield" if a.shift_field else
            "P1-reread-shift" if beta else lat.variants[v])
    print(f"{a.storage} n={n} vset={a.vset} {form} ({a.deriv}): "
          f"ms per step aux {ms[0] / 4:.4f} collide {ms[1] / 4:.4f}")
    return 0


def ad_main(a):
    n = a.n
    shape = (n, n, n) if a.vset == 3 else ((n, n, 1) if a.vset == 2 else (n, 1, 1))
    lat = lbnr.ADLattice(a.vset, shape, a.tau, 1 / n, storage=a.storage)
    if int(a.variant) >= 0:
        lat.set_form(int(a.variant))
    lat.init(W.gauge_wave(shape, 1 / n, 0.1))
    lat.step(a.steps)
    lat.status()
    ms = lat.step_timed(4)
    print(f"{a.storage} n={n} vset={a.vset} 37-field scheme, {lat.forms[lat.form]}: "
          f"ms per step {ms / 4:.4f}")
    lat.close()
    return 0


def batch_main(a):
    import torch
    n = a.n
    shape = (n, n, 1) if a.vset == 2 else (n, 1, 1)
    runs = [dict(vset=a.vset, shape=shape, tau=2.0, dx=1 / n, steps=a.steps)
            for _ in range(a.batch)]
    b = lbnr.Batch(runs, storage=a.storage, block=a.block, ctas_per_sm=a.per_sm,
                   deriv_mode=a.deriv)
    f = W.gauge_wave(shape, 1 / n, 0.01)
    for i in range(a.batch):
        b.init(i, f)
    times = []
    with torch.cuda.stream(b.stream):
        for _ in range(4):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(b.stream)
            b.run()
            e1.record(b.stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    b.check()
    p = b.plan()
    print(f"batch {a.batch} x {shape} {a.storage} ({a.deriv}): grid {p['grid']} x {p['block']}, "
          f"ms per launch of {a.steps} steps: " + " ".join(f"{t:.3f}" for t in times))
    return 0


if __name__ == "__main__":
    sys.exit(main())
