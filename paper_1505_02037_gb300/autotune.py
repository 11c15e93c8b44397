"""Autotuner for the collide kernel's launch form.

Each context offers a few launch forms (threads per cell, register-held or
shared-memory-staged distributions, consumer warps and pipeline depth of the
TMA-fed kernel). All give the same results; the tuner runs a few real steps
with each (best of a few timed runs, CUDA events per kernel) and keeps the
fastest. Results
are cached per (set, storage, streaming, lattice shape) for the process.
"""
from __future__ import annotations

_cache: dict = {}


def tune(lat, steps_per_trial: int = 4, trials: int = 2, verbose: bool = False) -> dict:
    """Chooses the fastest launch form for `lat` (a lbnr.Lattice that has
    been initialised). The trial steps advance the simulation like any other
    steps. Returns {name: ms per collide launch}."""
    key = (lat.vset, lat.storage, lat.streaming, lat.shape)
    names = lat.variants
    if key in _cache:
        lat.set_variant(_cache[key])
        return {}
    times = {}
    for v, name in enumerate(names):
        lat.set_variant(v)
        lat.step_timed(2)  # first launch pays for set-up
        best = float("inf")
        for _ in range(trials):
            _, ms = lat.step_timed(steps_per_trial)
            best = min(best, ms / steps_per_trial)
        times[name] = best
        if verbose:
            print(f"  {name}: {times[name]:.3f} ms per collide launch")
    best = min(range(len(names)), key=lambda v: times[names[v]])
    lat.set_variant(best)
    _cache[key] = best
    return times
