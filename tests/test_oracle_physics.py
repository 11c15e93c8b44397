"""Pins of the oracle's pointwise Bona-Masso right-hand sides against the
mathematics they must reproduce, with no reuse of the formulas under test.

* K equation (Sec. "Bona-Masso evolution equations"): on arbitrary smooth
  data, -d_k(alpha lambda^k_ij) + alpha S_ij minus the textbook ADM right-hand
  side -D_i D_j alpha + alpha (R_ij - 2 K_ik K^k_j + trK K_ij) is exactly
  -(alpha/4) gamma_ij H, with H = R - K_ij K^ij + trK^2 the Hamiltonian
  constraint (the Einstein evolution system "solves the energy constraint").
  R_ij and the covariant derivatives come from exact symbolic derivatives of
  the metric; the divergence of alpha lambda from high-order central
  differences of the oracle's lambda.
* V equation (Eq. Vsor): Omega_k equals the time derivative of V's
  definition, obtained from d_t gamma = -2 alpha K, minus alpha times the
  momentum constraint.
* Gauge wave (Sec. "Gauge Wave") and linear wave (Sec. "Linear Wave"):
  closed-form residuals; rotation covariance of all outputs.
"""
import math

import numpy as np
import pytest

PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
CFD8 = [(1, 4 / 5), (2, -1 / 5), (3, 4 / 105), (4, -1 / 280)]


def full(v6):
    m = np.zeros((3, 3))
    for q, (i, j) in enumerate(PAIRS):
        m[i, j] = m[j, i] = v6[q]
    return m


def six(m):
    return np.array([m[i, j] for i, j in PAIRS])


class AnalyticData:
    """alpha(x), gamma_ij(x), K_ij(x): smooth trigonometric fields, with every
    first and second derivative taken symbolically."""

    def __init__(self, seed):
        # sympy is required: the ADM-identity pin must never skip silently
        import sympy as sp
        rng = np.random.default_rng(seed)
        x, y, z = X = sp.symbols("x y z")

        def wave(amp):
            k = rng.integers(-2, 3, size=3)
            ph = rng.uniform(0, 2 * math.pi)
            return sp.Float(amp) * sp.sin(k[0] * x + k[1] * y + k[2] * z + sp.Float(ph))

        al = 1 + wave(0.1) + wave(0.05)
        g = [[None] * 3 for _ in range(3)]
        K = [[None] * 3 for _ in range(3)]
        for i, j in PAIRS:
            g[i][j] = g[j][i] = (1 if i == j else 0) + wave(0.12)
            K[i][j] = K[j][i] = wave(0.25)
        L = lambda e: sp.lambdify(X, e, "math")
        self.al = L(al)
        self.dal = [L(sp.diff(al, a)) for a in X]
        self.ddal = [[L(sp.diff(al, a, b)) for b in X] for a in X]
        self.g = [[L(g[i][j]) for j in range(3)] for i in range(3)]
        self.dg = [[[L(sp.diff(g[i][j], X[k])) for j in range(3)] for i in range(3)]
                   for k in range(3)]
        self.ddg = [[[[L(sp.diff(g[i][j], X[k], X[l])) for j in range(3)] for i in range(3)]
                     for l in range(3)] for k in range(3)]
        self.K = [[L(K[i][j]) for j in range(3)] for i in range(3)]
        self.dK = [[[L(sp.diff(K[i][j], X[k])) for j in range(3)] for i in range(3)]
                   for k in range(3)]

    def state(self, p):
        a = self.al(*p)
        G = np.array([[self.g[i][j](*p) for j in range(3)] for i in range(3)])
        Km = np.array([[self.K[i][j](*p) for j in range(3)] for i in range(3)])
        A = np.array([self.dal[k](*p) for k in range(3)]) / a
        D = 0.5 * np.array([[[self.dg[k][i][j](*p) for j in range(3)] for i in range(3)]
                            for k in range(3)])
        gi = np.linalg.inv(G)
        # V_k from its definition (Sec. "Bona-Masso formulation") so that the
        # data satisfy it exactly.
        V = np.einsum("rm,krm->k", gi, D) - np.einsum("rm,mrk->k", gi, D)
        return a, G, Km, A, D, V, gi


def oracle_point(O, a, G, Km, A, D, V, slicing=1):
    D18 = np.array([six(D[k]) for k in range(3)])
    return O.bm_point(a, six(G), six(Km), V, A, D18, slicing)


def textbook_adm(data, p):
    """Exact ADM quantities at p: d_t K_ij (zero shift, vacuum), H, M_i, and
    d_t V_k implied by d_t gamma = -2 alpha K and d_t D_kij = -d_k(alpha K_ij)."""
    a, G, Km, A, D, V, gi = data.state(p)
    dG = np.array([[[data.dg[k][i][j](*p) for j in range(3)] for i in range(3)]
                   for k in range(3)])  # dG[k,i,j] = d_k g_ij
    ddG = np.array([[[[data.ddg[k][l][i][j](*p) for j in range(3)] for i in range(3)]
                     for l in range(3)] for k in range(3)])  # d_k d_l g_ij
    Gl = np.zeros((3, 3, 3))  # Gamma_kij = (d_i g_jk + d_j g_ik - d_k g_ij)/2
    dGl = np.zeros((3, 3, 3, 3))  # d_l Gamma_kij
    for k in range(3):
        for i in range(3):
            for j in range(3):
                Gl[k, i, j] = 0.5 * (dG[i, j, k] + dG[j, i, k] - dG[k, i, j])
                for l in range(3):
                    dGl[l, k, i, j] = 0.5 * (ddG[l, i, j, k] + ddG[l, j, i, k] - ddG[l, k, i, j])
    Gu = np.einsum("km,mij->kij", gi, Gl)
    dgi = -np.einsum("ka,lab,bm->lkm", gi, dG, gi)
    dGu = np.einsum("lkm,mij->lkij", dgi, Gl) + np.einsum("km,lmij->lkij", gi, dGl)
    Ric = (np.einsum("kkij->ij", dGu) - np.einsum("jkik->ij", dGu)
           + np.einsum("kkm,mij->ij", Gu, Gu) - np.einsum("kjm,mik->ij", Gu, Gu))
    da = np.array([data.dal[k](*p) for k in range(3)])
    dda = np.array([[data.ddal[i][j](*p) for j in range(3)] for i in range(3)])
    DDa = dda - np.einsum("kij,k->ij", Gu, da)
    Kud = gi @ Km
    trK, trK2 = np.trace(Kud), np.trace(Kud @ Kud)
    dtK = -DDa + a * (Ric - 2 * Km @ gi @ Km + trK * Km)
    H = np.einsum("ij,ij", gi, Ric) - trK2 + trK ** 2
    dKm = np.array([[[data.dK[k][i][j](*p) for j in range(3)] for i in range(3)]
                    for k in range(3)])
    dtrK = np.einsum("ijk,jk->i", dgi, Km) + np.einsum("jk,ijk->i", gi, dKm)
    covK = dKm - np.einsum("mjk,mi->jki", Gu, Km) - np.einsum("mji,km->jki", Gu, Km)
    M = np.einsum("jk,jki->i", gi, covK) - dtrK
    dtgi = 2 * a * gi @ Km @ gi
    dtD = -(np.einsum("k,ij->kij", da, Km) + a * dKm)
    dtV = (np.einsum("rm,krm->k", dtgi, D) - np.einsum("rm,mrk->k", dtgi, D)
           + np.einsum("rm,krm->k", gi, dtD) - np.einsum("rm,mrk->k", gi, dtD))
    return dtK, H, M, dtV


def flux_divergence(O, data, p, h=1e-2):
    div = np.zeros((3, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1
        for m, c in CFD8:
            for sgn in (1, -1):
                st = data.state(p + sgn * m * h * e)
                lam = oracle_point(O, *st[:6])[0]
                div += sgn * c * st[0] * full(lam[k]) / h
    return div


@pytest.mark.parametrize("seed", [11, 12])
def test_k_equation_is_adm_minus_quarter_hamiltonian(oracle_mod, seed):
    data = AnalyticData(seed)
    rng = np.random.default_rng(seed + 100)
    worst = 0.0
    for _ in range(4):
        p = rng.uniform(-3, 3, size=3)
        a, G, Km, A, D, V, gi = data.state(p)
        lam, S, Om, Sa = oracle_point(oracle_mod, a, G, Km, A, D, V)
        dtK, H, M, dtV = textbook_adm(data, p)
        bm = -flux_divergence(oracle_mod, data, p) + a * full(S)
        resid = bm - dtK + 0.25 * a * H * G
        scale = np.abs(dtK).max() + np.abs(a * H)
        worst = max(worst, np.abs(resid).max() / scale)
        assert abs(H) > 1e-3  # the data really violate the constraint
    assert worst < 1e-9, worst


@pytest.mark.parametrize("seed", [21, 22])
def test_v_equation_is_definition_rate_minus_momentum_constraint(oracle_mod, seed):
    data = AnalyticData(seed)
    rng = np.random.default_rng(seed + 100)
    for _ in range(4):
        p = rng.uniform(-3, 3, size=3)
        a, G, Km, A, D, V, gi = data.state(p)
        lam, S, Om, Sa = oracle_point(oracle_mod, a, G, Km, A, D, V)
        dtK, H, M, dtV = textbook_adm(data, p)
        assert np.abs(M).max() > 1e-3
        np.testing.assert_allclose(Om, dtV - a * M, rtol=0, atol=1e-13 * (1 + np.abs(dtV).max()))


@pytest.mark.parametrize("slicing,expect", [(0, "zero"), (1, "harmonic"), (2, "onelog")])
def test_lapse_source(oracle_mod, slicing, expect):
    data = AnalyticData(5)
    a, G, Km, A, D, V, gi = data.state(np.array([0.3, -0.2, 0.9]))
    _, _, _, Sa = oracle_point(oracle_mod, a, G, Km, A, D, V, slicing=slicing)
    trK = np.trace(np.linalg.inv(G) @ Km)
    ref = {"zero": 0.0, "harmonic": -a * a * trK, "onelog": -a * trK}[expect]
    assert Sa == pytest.approx(ref, rel=1e-14, abs=1e-15)


def _gauge_wave_point(u, A, d, n):
    ph = 2 * math.pi * u / d
    H = 1 - A * math.sin(ph)
    Hp = -A * 2 * math.pi / d * math.cos(ph)
    nn = np.outer(n, n)
    G = np.eye(3) + (H - 1) * nn
    Km = -(math.pi * A / d) * math.cos(ph) / math.sqrt(H) * nn
    Aa = 0.5 * Hp / H * n
    D = 0.5 * Hp * np.einsum("k,ij->kij", n, nn)
    return math.sqrt(H), G, Km, Aa, D, np.zeros(3), H, Hp


@pytest.mark.parametrize("direction", ["x", "diag", "random"])
def test_gauge_wave_closed_form(oracle_mod, direction):
    """With exact derivatives, the gauge wave makes S_ij = 0, Omega = 0,
    alpha lambda^k_ij = K_ij n^k and d_t alpha = -alpha^2 trK."""
    if direction == "x":
        n = np.array([1.0, 0, 0])
    elif direction == "diag":
        n = np.ones(3) / math.sqrt(3)
    else:
        n = np.random.default_rng(3).normal(size=3)
        n /= np.linalg.norm(n)
    for u in np.linspace(0.05, 0.95, 7):
        a, G, Km, Aa, D, V, H, Hp = _gauge_wave_point(u, 0.1, 1.0, n)
        lam, S, Om, Sa = oracle_point(oracle_mod, a, G, Km, Aa, D, V)
        assert np.abs(S).max() < 1e-14
        assert np.abs(Om).max() < 1e-14
        for k in range(3):
            np.testing.assert_allclose(a * full(lam[k]), Km * n[k], rtol=0, atol=1e-14)
        # harmonic slicing: d_t alpha = d_t sqrt(H) = -H'/(2 sqrt H)
        assert Sa == pytest.approx(-Hp / (2 * math.sqrt(H)), rel=1e-12)


def test_linear_wave_residual_is_quadratic(oracle_mod):
    """Linear wave (Sec. "Linear Wave"): the K equation's residual with exact
    derivatives shrinks as A^2 (the closed form is a linearised solution)."""
    res = []
    for A in (1e-2, 1e-3):
        d = 1.0
        worst = 0
        for u in np.linspace(0.05, 0.95, 5):
            vals = {}
            for m, _ in [(0, 0)] + CFD8:
                for sgn in ((1, -1) if m else (1,)):
                    uu = u + sgn * m * 1e-3
                    ph = 2 * math.pi * uu / d
                    b = A * math.sin(ph)
                    bp = 2 * math.pi * A / d * math.cos(ph)
                    G = np.diag([1.0, 1 + b, 1 - b])
                    Km = math.pi * A / d * math.cos(ph) * np.diag([0.0, 1.0, -1.0])
                    D = np.zeros((3, 3, 3))
                    D[0] = 0.5 * bp * np.diag([0.0, 1.0, -1.0])
                    V = np.array([-b * bp / (1 - b * b), 0, 0])
                    lam, S, Om, Sa = oracle_point(oracle_mod, 1.0, G, Km, np.zeros(3), D, V, 0)
                    vals[sgn * m] = (lam, S, Km)
            div = sum(c * (full(vals[m][0][0]) - full(vals[-m][0][0])) / 1e-3 for m, c in CFD8)
            ph = 2 * math.pi * u / d
            dtK = (2 * math.pi / d) * (math.pi * A / d) * math.sin(ph) * np.diag([0.0, 1.0, -1.0])
            worst = max(worst, np.abs(dtK + div - full(vals[0][1])).max())
        res.append(worst)
    ratio = res[0] / res[1]
    assert 50 < ratio < 200, res  # A^2 scaling: a factor 100 per decade


def test_rotation_covariance(oracle_mod):
    """lambda, S_ij, Omega and the lapse source transform as tensors of their
    index structure under a random rotation of all inputs."""
    rng = np.random.default_rng(7)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    R = q * np.sign(np.linalg.det(q))
    B = rng.normal(size=(3, 3))
    G = np.eye(3) + 0.2 * (B + B.T)
    Km = rng.normal(size=(3, 3)) * 0.3
    Km = Km + Km.T
    A = rng.normal(size=3) * 0.4
    V = rng.normal(size=3) * 0.4
    D = rng.normal(size=(3, 3, 3)) * 0.3
    D = D + D.transpose(0, 2, 1)
    a = 1.3
    lam, S, Om, Sa = oracle_point(oracle_mod, a, G, Km, A, D, V)
    G2 = R @ G @ R.T
    K2 = R @ Km @ R.T
    D2 = np.einsum("ka,ib,jc,abc->kij", R, R, R, D)
    lam2, S2, Om2, Sa2 = oracle_point(oracle_mod, a, G2, K2, R @ A, D2, R @ V)
    L1 = np.array([full(lam[k]) for k in range(3)])
    L2 = np.array([full(lam2[k]) for k in range(3)])
    np.testing.assert_allclose(L2, np.einsum("ka,ib,jc,abc->kij", R, R, R, L1), atol=1e-12)
    np.testing.assert_allclose(full(S2), R @ full(S) @ R.T, atol=1e-12)
    np.testing.assert_allclose(Om2, R @ Om, atol=1e-12)
    assert Sa2 == pytest.approx(Sa, rel=1e-12)
