"""Pins of the oracle's velocity sets (Sec. "Lattice Boltzmann Model").

The tables are checked against the paper's printed matrices (golden file) and
against the exact isotropy identities the paper states ("accurate up to
second order"), in rational arithmetic.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "velocity_sets.txt")


def _golden():
    sets = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, l, cx, cy, cz, wn, wd = line.split()
        sets.setdefault(name, []).append(((int(cx), int(cy), int(cz)), Fraction(int(wn), int(wd))))
    return sets


@pytest.mark.parametrize("name,vset", [("D2Q9", 2), ("D3Q19", 3)])
def test_velocity_sets_match_paper(oracle_mod, name, vset):
    c, w = oracle_mod.velocity_set(vset)
    gold = _golden()[name]
    assert len(gold) == len(w)
    for l, (cg, wg) in enumerate(gold):
        assert tuple(c[l]) == cg
        assert w[l] == float(wg)


def _rational(w):
    return [Fraction(x).limit_denominator(1000) for x in w]


@pytest.mark.parametrize("vset", [1, 2, 3])
def test_isotropy_identities_exact(oracle_mod, vset):
    """sum w = 1, sum w c = 0, sum w c_a c_b = c_s^2 delta_ab (c_s^2 = 1/3),
    sum w c_a c_b c_c = 0, all exact; and every velocity appears with its
    opposite."""
    c, w = oracle_mod.velocity_set(vset)
    W = _rational(w)
    for x, xr in zip(w, W):
        assert float(xr) == x
    dim = {1: 1, 2: 2, 3: 3}[vset]
    assert sum(W) == 1
    for a in range(3):
        assert sum(Wl * int(cl[a]) for Wl, cl in zip(W, c)) == 0
        for b in range(3):
            m2 = sum(Wl * int(cl[a]) * int(cl[b]) for Wl, cl in zip(W, c))
            expect = Fraction(1, 3) if (a == b and a < dim) else 0
            assert m2 == expect
            for d in range(3):
                assert sum(Wl * int(cl[a]) * int(cl[b]) * int(cl[d]) for Wl, cl in zip(W, c)) == 0
    vecs = {tuple(v) for v in c}
    assert len(vecs) == len(c)
    for v in vecs:
        assert tuple(-x for x in v) in vecs


def test_d1q3_is_x_marginal(oracle_mod):
    """D1Q3's weights are the sums of the D2Q9 and D3Q19 weights over each
    class of equal c_x (the reading that lets x-aligned 2D/3D runs reduce to
    1D exactly)."""
    c1, w1 = oracle_mod.velocity_set(1)
    for v in (2, 3):
        c, w = oracle_mod.velocity_set(v)
        for cx, wx in zip(c1[:, 0], w1):
            assert np.isclose(w[c[:, 0] == cx].sum(), wx, rtol=0, atol=1e-15)
