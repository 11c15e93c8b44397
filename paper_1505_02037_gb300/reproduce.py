"""The paper's validation sweeps on the GPU path (Sec. "Relaxation Time tau and
Numerical Diffusivity eta", Figs. gijl and simana), as numbers.

Gauge wave (Sec. "Gauge Wave") on the D2Q9 lattice, propagating along x on
the unit periodic box (d = 1), harmonic slicing, dt = dr = 1/N.

* tau sweep at N = 800 (dr = 0.00125): for each tau/dt, the mean over the
  first 500 steps of the relative error of gamma_xx, and the lifetime.
* Refinement at constant numerical diffusivity eta = c_s^2 (tau - 1/2) dr
  (tau in units of dt): tau = 1/2 + 3 eta N. For each N, the relative error at
  step 400 and the lifetime.

Readings (the paper leaves them open): the relative error at a step is
max_x |gamma_xx - gamma_xx(exact)| / A, and the mean error averages it over
the steps. Two lifetimes: the first step at which the error exceeds 10 % (the
figure quoted for the gauge wave in Sec. "Errors in the Validation Tests"),
and the crash step, the first at which the error exceeds 10 A or the moments
turn non-finite (numerical diffusion alone cannot take the error past 1: a
fully damped wave is off by at most A). The crash step is the "life-time" of
Fig. gijl's inset, the run going numerically unstable.

  python -m paper_1505_02037_gb300.reproduce [--amp 1e-3] [--json]
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from . import lbnr
from . import workloads as W

NY = 4  # the wave is uniform in y; a few rows keep every stencil direction live


def _run(N, tau, A, checkpoints, stop_at=None, storage="f64", check_every=10, crash_at=None,
         max_steps=200000):
    """Steps the D2Q9 gauge wave and returns {step: relative error}, the first
    checked step whose error exceeds stop_at, and (with crash_at) the first
    whose error exceeds crash_at (None where not reached). After the last
    checkpoint and stop_at are passed, checks come every 10 check_every steps."""
    shape = (N, NY, 1)
    dx = 1.0 / N
    lat = lbnr.Lattice(2, shape, tau, dx, storage=storage)
    lat.init(W.gauge_wave(shape, dx, A))
    errs, life, crash, done = {}, None, None, 0
    targets = sorted(set(checkpoints))
    last = max(targets) if targets else 0
    n = 0
    while True:
        every = check_every if (n < last or (stop_at is not None and life is None)) \
            else 10 * check_every
        nxt = n + every
        want = [t for t in targets if n < t <= nxt]
        step_to = want[0] if want else nxt
        lat.step(step_to - done)
        done = step_to
        n = step_to
        try:
            m = lat.moments().reshape(16, NY, N)
            exact = W.gauge_wave((N, 1, 1), dx, A, t=n * dx).reshape(16, 1, N)
            e = float(np.abs(m[1] - exact[1]).max() / A)
        except lbnr.NonFiniteError:
            e = float("inf")
        if not np.isfinite(e):
            e = float("inf")
        if n in targets:
            errs[n] = e
        if stop_at is not None and life is None and e > stop_at:
            life = n
        if crash_at is not None and crash is None and e > crash_at:
            crash = n
        done_life = stop_at is None or life is not None
        done_crash = crash_at is None or crash is not None
        if done_life and done_crash and n >= last:
            break
        if e == float("inf") and n >= last:
            break
        if n >= max_steps:
            break
    lat.close()
    return errs, life, crash


def tau_sweep(taus=(2.5, 3.0, 3.5, 4.0, 4.5, 5.0, 5.25), N=800, A=1e-3, crash=True):
    """Mean relative error of gamma_xx over steps 1..500, the step at which
    the error passes 10 %, and (crash) the crash step, for each tau/dt."""
    out = []
    for tau in taus:
        errs, life, cr = _run(N, tau, A, checkpoints=range(10, 501, 10), stop_at=0.1,
                              crash_at=10.0 if crash else None)
        out.append({"tau": tau, "eta": (tau - 0.5) / (3.0 * N),
                    "mean_rel_error_500": float(np.mean(list(errs.values()))),
                    "lifetime_steps": life, "crash_steps": cr})
    return out


def eta_refinement(Ns=(400, 800, 1200, 1600, 2400), eta=1.0 / 600.0, A=1e-3):
    """At constant eta = c_s^2 (tau - 1/2) dr: relative error at step 400 and
    the lifetime, for each N."""
    out = []
    for N in Ns:
        tau = 0.5 + 3.0 * eta * N
        errs, life, _ = _run(N, tau, A, checkpoints=[400], stop_at=0.1)
        out.append({"N": N, "tau": tau, "rel_error_400": errs[400], "lifetime_steps": life})
    return out


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--amp", type=float, default=1e-3)
    p.add_argument("--json", action="store_true")
    a = p.parse_args(argv)
    res = {"tau_sweep": tau_sweep(A=a.amp), "eta_refinement": eta_refinement(A=a.amp)}
    if a.json:
        print(json.dumps(res))
        return 0
    print("tau sweep, D2Q9 gauge wave, N = 800, A = %g" % a.amp)
    for r in res["tau_sweep"]:
        print(f"  tau/dt {r['tau']:5.2f}  eta {r['eta']:.6f}  mean error (500 steps) "
              f"{r['mean_rel_error_500']:.4f}  10 % at step {r['lifetime_steps']}  "
              f"crash at step {r['crash_steps']}")
    print("constant eta = 1/600 refinement")
    for r in res["eta_refinement"]:
        print(f"  N {r['N']:5d}  tau/dt {r['tau']:6.2f}  error at step 400 "
              f"{r['rel_error_400']:.4f}  10 % at step {r['lifetime_steps']}")
    return 0


if __name__ == "__main__":
    sys.exit(main())
