"""GPU checks of the batched ensemble (one persistent cooperative launch that
advances many independent 1D/2D runs): every run against the FP64 oracle,
against the same run on its own context, team barriers, the bounded wait,
non-finite runs stopping, and the planner's output."""
import math

import numpy as np
import pytest

from paper_1505_02037_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_02037_gb300 import lbnr
    lbnr.library()
    return lbnr


def dist_err(g, o, kscale):
    g = g.reshape(16, -1)
    o = o.reshape(16, -1)
    floor = np.array([1.0] * 7 + [kscale] * 9) / 3
    return np.abs(g - o).max(axis=1) / np.maximum(np.abs(o).max(axis=1), floor)


def perturbed(f, seed=0):
    rng = np.random.default_rng(seed)
    return f * (1 + rng.choice([-1.0, 1.0], size=f.shape) * 2.2e-16)


def small_ensemble(n=10, seed=7, crossings=1, tau=(1.2, 2.0), n1=(33, 300), n2=(5, 40)):
    runs = W.ensemble(nruns=n, seed=seed, n1=n1, n2=n2, tau=tau, crossings=crossings)
    for r in runs:
        r["slicing"] = r["run"] % 3
    return runs


def make_batch(L, runs, **kw):
    b = L.Batch(runs, **kw)
    for i, r in enumerate(runs):
        b.init(i, W.ensemble_fields(r))
    return b


def test_batch_fp64_matches_oracle(L, oracle_mod):
    """Each run of a mixed 1D/2D ensemble (uneven N, tau, A, slicing, step
    count) equals the oracle's run to the FP64 bar (1e-12, or 4x the
    one-ulp spread of the oracle where the method's conditioning is worse)."""
    runs = small_ensemble()
    b = make_batch(L, runs, storage="f64")
    b.run()
    rc, per = b.status()
    assert rc == 0 and per == [0] * len(runs)
    for i, r in enumerate(runs):
        assert b.steps_done(i) == r["steps"]
        o = oracle_mod.Oracle(r["vset"], r["shape"], r["tau"], r["dx"], slicing=r["slicing"])
        f0 = o.init(W.ensemble_fields(r))
        f = o.run(f0, r["steps"])
        kscale = math.pi * r["A"]
        spread = dist_err(o.run(perturbed(f0), r["steps"]), f, kscale).max()
        err = dist_err(b.distributions(i), f, kscale).max()
        assert err <= max(TOL64, 4 * spread), (i, r, err, spread)
    b.close()


def team_ensemble():
    runs = [dict(vset=2, shape=(320, 320, 1), N=320, dx=1 / 320, tau=1.6, A=0.05,
                 direction="x", steps=24),
            dict(vset=2, shape=(256, 256, 1), N=256, dx=1 / 256, tau=1.9, A=0.02,
                 direction="xy", steps=24),
            dict(vset=1, shape=(4000, 1, 1), N=4000, dx=1 / 4000, tau=1.3, A=0.1,
                 direction="x", steps=24)]
    runs += small_ensemble(n=6, seed=11, crossings=1, n1=(20, 80), n2=(4, 24))
    for r in runs:
        r["steps"] = min(r["steps"], 24)
    return runs


def single_context(L, r, storage, variant=None):
    lat = L.Lattice(r["vset"], r["shape"], r["tau"], r["dx"], slicing=r.get("slicing", 1),
                    storage=storage, streaming=L.LBNR_STREAM_PINGPONG)
    if variant is not None:
        names = lat.variants
        pick = [v for v in variant if v in names]
        if not pick:
            lat.close()
            return None
        lat.set_variant(names.index(pick[0]))
    lat.init(W.ensemble_fields(r))
    return lat


def test_batch_team_runs_match_single_context(L):
    """Large runs get a team of blocks that meet at device barriers; with one
    block per SM the two big runs below need teams. Each run matches the same
    run stepped on its own context (same FP32 storage, the autotuner's default
    launch form, whose sums may round in another order). Bar: 4x the distance
    between that context's run and the same run started from distributions
    perturbed by one FP32 ulp (seeded signs)."""
    runs = team_ensemble()
    b = make_batch(L, runs, storage="dev_f32", block=256, ctas_per_sm=1)
    teams = b.plan()["teams"]
    assert teams[0] > 1 and teams[1] > 1
    b.run()
    assert b.check() == [0] * len(runs)
    for i, r in enumerate(runs):
        lat = single_context(L, r, "dev_f32")
        f0 = lat.distributions()
        lat2 = single_context(L, r, "dev_f32")
        rng = np.random.default_rng(i)
        lat2.set_distributions(f0 * (1 + rng.choice([-1.0, 1.0], size=f0.shape) * 2.0 ** -24))
        lat.step(r["steps"])
        lat2.step(r["steps"])
        ref = lat.distributions()
        kscale = math.pi * r["A"]
        spread = dist_err(lat2.distributions(), ref, kscale).max()
        err = dist_err(b.distributions(i), ref, kscale).max()
        assert err <= max(4 * spread, 1e-7), (i, teams[i], err, spread)
        lat.close()
        lat2.close()
    b.close()


@pytest.mark.parametrize("storage", ["f64", "dev_f32"])
def test_batch_bitwise_equals_single_context_same_form(L, storage):
    """With the single context on a one-thread-per-cell form (the per-cell
    arithmetic the batched kernel runs, in the same order; re-read, or
    register-held where the set has no re-read form), every run of the
    batch, team runs included, gives the same bits."""
    runs = team_ensemble()
    b = make_batch(L, runs, storage=storage, block=256, ctas_per_sm=1)
    b.run()
    assert b.check() == [0] * len(runs)
    for i, r in enumerate(runs):
        lat = single_context(L, r, storage, variant=("P1-reread", "P1-hold"))
        assert lat is not None
        lat.step(r["steps"])
        assert np.array_equal(b.distributions(i), lat.distributions()), i
        lat.close()
    b.close()


def test_batch_chunked_launches_equal_one_launch(L):
    """Two launches of k steps per run give the same bits as one of 2k."""
    runs = small_ensemble(n=8, seed=5, crossings=1)
    for r in runs:
        r["steps"] = 20
    b1 = make_batch(L, runs, storage="dev_f32")
    b1.run(10)
    b1.run(10)
    b2 = make_batch(L, runs, storage="dev_f32")
    b2.run()
    assert b1.check() == b2.check() == [0] * len(runs)
    for i in range(len(runs)):
        assert b1.steps_done(i) == b2.steps_done(i) == 20
        assert np.array_equal(b1.distributions(i), b2.distributions(i))
    b1.close()
    b2.close()


def test_batch_block_shapes_agree(L):
    """Every block shape the autotuner may choose gives the same bits (the
    per-cell arithmetic does not depend on the assignment)."""
    from paper_1505_02037_gb300 import autotune
    runs = small_ensemble(n=6, seed=3, crossings=1, n2=(40, 96))
    for r in runs:
        r["steps"] = 12
    ref = None
    for block, per_sm in autotune.batch_shapes():
        b = make_batch(L, runs, storage="dev_f32", block=block, ctas_per_sm=per_sm)
        b.run()
        assert b.check() == [0] * len(runs)
        out = [b.distributions(i) for i in range(len(runs))]
        if ref is None:
            ref = out
        else:
            for x, y in zip(out, ref):
                assert np.array_equal(x, y), (block, per_sm)
        b.close()


def test_batch_is_graph_captured(L):
    runs = small_ensemble(n=4, seed=9)
    b = make_batch(L, runs, storage="dev_f32")
    b.run(2)
    b.check()
    p = b.plan()
    assert p["graphed"]
    import torch
    assert p["grid"] % torch.cuda.get_device_properties(0).multi_processor_count == 0
    b.close()


def test_batch_wait_timeout_is_reported(L):
    """A team member that never arrives (test hook: the first arrival of one
    run's block 0 is dropped) makes the team's bounded waits run out: that run
    reports LBNR_ETIMEOUT and stops, every other run completes normally."""
    runs = [dict(vset=2, shape=(256, 256, 1), N=256, dx=1 / 256, tau=1.5, A=0.05,
                 direction="x", steps=6)]
    runs += small_ensemble(n=5, seed=13, crossings=1, n2=(4, 16))
    for r in runs:
        r["steps"] = min(r["steps"], 6)
    b = make_batch(L, runs, storage="dev_f32", ctas_per_sm=1, wait_limit_ns=50_000_000,
                   drop_arrival_run=0)
    assert b.plan()["teams"][0] > 1
    b.run()
    rc, per = b.status()
    assert rc == -5 and per[0] == -5 and per[1:] == [0] * (len(runs) - 1)
    assert b.steps_done(0) == 0
    for i in range(1, len(runs)):
        assert b.steps_done(i) == runs[i]["steps"]
    b.close()


def test_batch_nonfinite_run_stops(L):
    """At tau = 0.51 the scheme is linearly unstable and the run overflows
    within a few hundred steps: it reports LBNR_ENONFINITE and stops at the
    step that read the non-finite moments; the other runs are untouched."""
    runs = [dict(vset=1, shape=(200, 1, 1), N=200, dx=1 / 200, tau=0.51, A=0.1,
                 direction="x", steps=3000),
            dict(vset=1, shape=(200, 1, 1), N=200, dx=1 / 200, tau=1.9, A=0.1,
                 direction="x", steps=300)]
    b = make_batch(L, runs, storage="dev_f32")
    b.run()
    rc, per = b.status()
    assert per == [-4, 0] and rc == -4
    assert 0 < b.steps_done(0) < 3000
    assert b.steps_done(1) == 300
    d = b.distributions(1)
    assert np.isfinite(d).all()
    b.close()


def test_batch_replan_drops_stopped_runs_and_keeps_bits(L):
    """With re-planning before every launch, a run that went non-finite is
    left out of the next plan (team 0) and its blocks go to the others; the
    live runs give the same bits as without re-planning. Re-initialising the
    stopped run puts it back into the plan."""
    bad = dict(vset=1, shape=(200, 1, 1), N=200, dx=1 / 200, tau=0.51, A=0.1,
               direction="x", steps=200)
    runs = [bad] + team_ensemble()[:3]
    for r in runs[1:]:
        r["steps"] = 12
    b1 = make_batch(L, runs, storage="dev_f32", replan=True)
    b2 = make_batch(L, runs, storage="dev_f32")
    for _ in range(2):
        b1.run()
        b2.run()
    rc1, per1 = b1.status()
    rc2, per2 = b2.status()
    assert per1 == per2 == [-4, 0, 0, 0]
    b1.replan()
    assert b1.plan()["teams"][0] == 0 and min(b1.plan()["teams"][1:]) >= 1
    for i in range(1, len(runs)):
        assert b1.steps_done(i) == b2.steps_done(i) == 24
        assert np.array_equal(b1.distributions(i), b2.distributions(i)), i
    b1.init(0, W.ensemble_fields(bad))
    assert b1.plan()["teams"][0] == 1
    b1.close()
    b2.close()


def test_ensemble_configuration_first_16_runs(L, oracle_mod):
    """The ensemble configuration itself (seed 150502037): its first 16 runs,
    24 steps each. In FP64 every run equals the oracle's run to the FP64 bar;
    in FP32 deviation storage (the configuration's storage) every run equals,
    bit for bit, the same run stepped on its own context in the
    one-thread-per-cell form."""
    runs = W.ensemble(seed=150502037)[:16]
    for r in runs:
        r["steps"] = 24
    b64 = make_batch(L, runs, storage="f64")
    b64.run()
    b32 = make_batch(L, runs, storage="dev_f32")
    b32.run()
    assert b64.check() == [0] * 16 and b32.check() == [0] * 16
    for i, r in enumerate(runs):
        o = oracle_mod.Oracle(r["vset"], r["shape"], r["tau"], r["dx"])
        f0 = o.init(W.ensemble_fields(r))
        f = o.run(f0, 24)
        kscale = math.pi * r["A"]
        spread = dist_err(o.run(perturbed(f0), 24), f, kscale).max()
        err = dist_err(b64.distributions(i), f, kscale).max()
        assert err <= max(TOL64, 4 * spread), (i, r["shape"], r["tau"], err, spread)
        lat = single_context(L, r, "dev_f32", variant=("P1-reread", "P1-hold"))
        lat.step(24)
        assert np.array_equal(b32.distributions(i), lat.distributions()), i
        lat.close()
    b64.close()
    b32.close()


@pytest.mark.parametrize("teams", [False, True])
def test_batch_lag_fp64_matches_oracle(L, oracle_mod, teams):
    """Lagged derivatives (reading R17) in the batch: a step is the collide
    pass alone (it writes the next step's stencil planes) and one team
    barrier. Each run of a mixed ensemble, and of one whose large runs are
    split over teams of blocks, equals the oracle's LAG run to the FP64 bar."""
    runs = team_ensemble() if teams else small_ensemble(n=8, seed=13)
    kw = dict(block=256, ctas_per_sm=1) if teams else {}
    b = make_batch(L, runs, storage="f64", deriv_mode="lag", **kw)
    if teams:
        t = b.plan()["teams"]
        assert t[0] > 1 and t[1] > 1
    b.run()
    rc, per = b.status()
    assert rc == 0 and per == [0] * len(runs)
    for i, r in enumerate(runs):
        assert b.steps_done(i) == r["steps"]
        o = oracle_mod.Oracle(r["vset"], r["shape"], r["tau"], r["dx"],
                              slicing=r.get("slicing", 1), deriv_mode=1)
        f0, p0 = o.lag_init(W.ensemble_fields(r))
        f, _ = o.run_lag(f0, p0, r["steps"])
        fp, _ = o.run_lag(perturbed(f0), p0, r["steps"])
        kscale = math.pi * r["A"]
        spread = dist_err(fp, f, kscale).max()
        err = dist_err(b.distributions(i), f, kscale).max()
        assert err <= max(TOL64, 4 * spread), (i, r, err, spread)
    b.close()
