"""Autotuner for the collide kernel's launch form.

Each context offers a few launch forms (block shape of the one-thread-per-cell
kernel, register-held or re-read distributions, consumer warps and pipeline
depth of the bulk-copy-fed kernel). All give the same results within
rounding; the tuner runs a few real steps with each (best of a few timed
runs, CUDA events per kernel) and keeps the fastest. Results are cached per
(set, storage, streaming, derivative mode, lattice shape) for the process.
"""
from __future__ import annotations

_cache: dict = {}


def tune(lat, steps_per_trial: int = 4, trials: int = 2, verbose: bool = False) -> dict:
    """Chooses the fastest launch form for `lat` (a lbnr.Lattice that has
    been initialised). The trial steps advance the simulation like any other
    steps. Returns {name: ms per collide launch}."""
    key = (lat.vset, lat.storage, lat.streaming, lat.shape, lat.deriv_mode)
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


def batch_shapes(sm_resident_max: int = 4):
    """(threads per block, blocks per SM) pairs the batched kernel accepts:
    blocks of 256 threads at up to 255 registers (one per SM), blocks of 128
    at up to 168 registers (one to three per SM) or at up to 128 (four)."""
    shapes = [(256, 1), (128, 1), (128, 2), (128, 3), (128, 4)]
    return [s for s in shapes if s[1] <= sm_resident_max]


def tune_batch(batch, trial_steps: int = 64, trials: int = 2, shapes=None, reset=None,
               verbose: bool = False) -> dict:
    """Chooses the block shape of a lbnr.Batch: for each (threads per block,
    blocks per SM) the planner re-assigns the runs and launches of
    `trial_steps` steps per run are timed with CUDA events (best of
    `trials`, each after `reset()` when given, so that every shape steps the
    same states: runs that stop early would otherwise make later shapes look
    faster). Shapes the kernel cannot hold resident are skipped. The trial
    steps advance the runs; re-initialise them afterwards for a clean start.
    Returns {(block, per_sm): ms}."""
    import torch
    from .lbnr import LbnrError
    shapes = shapes or batch_shapes()
    times = {}
    for block, per_sm in shapes:
        try:
            batch.configure(block, per_sm)
        except LbnrError:
            continue
        plan = batch.plan()
        if plan["grid"] < per_sm * torch.cuda.get_device_properties(0).multi_processor_count:
            continue  # fewer blocks resident than asked for: same as a smaller shape
        with torch.cuda.stream(batch.stream):
            batch.run(trial_steps)  # first launch captures the graph
            best = float("inf")
            for _ in range(trials):
                if reset is not None:
                    reset()
                    batch.replan()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(batch.stream)
                batch.run(trial_steps)
                e1.record(batch.stream)
                e1.synchronize()
                best = min(best, e0.elapsed_time(e1))
        times[(block, per_sm)] = best
        if verbose:
            print(f"  block {block} x {per_sm}/SM (grid {plan['grid']}): {best:.3f} ms")
    if not times:
        raise RuntimeError("no block shape of the batched kernel could be planned")
    best = min(times, key=times.get)
    batch.configure(*best)
    return times
