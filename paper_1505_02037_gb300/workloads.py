"""Seeded synthetic inputs: the closed-form test spacetimes of Ilseven &
Mendoza (arXiv:1505.02037, Sec. "Tests and Results") sampled on a periodic
cell-centred lattice, plus seeded random distribution states.

This module holds no lattice Boltzmann arithmetic. Both the CUDA library's
tests and the CPU oracle take their inputs from here.

Field order (16 values per cell): alpha; gamma_xx, gamma_xy, gamma_xz,
gamma_yy, gamma_yz, gamma_zz; K_xx .. K_zz (same order); V_x, V_y, V_z.
Arrays are [16][nz][ny][nx] (x fastest), float64.

Grid: cell-centred, x_i = x0 + (i + 1/2) dx with x0 = -L/2, matching the
paper's x_r = -400 dr + (x - 1/2) dr for an 800-cell lattice (Sec. "Gauge
Wave").
"""
from __future__ import annotations

import math

import numpy as np

NF = 16
PAIRS = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


def coords(shape, dx, origin=None):
    """Cell-centre coordinates X, Y, Z of a (nx, ny, nz) lattice, each [nz, ny, nx]."""
    nx, ny, nz = shape
    o = [-0.5 * n * dx for n in shape] if origin is None else origin
    xs = o[0] + (np.arange(nx) + 0.5) * dx
    ys = o[1] + (np.arange(ny) + 0.5) * dx
    zs = o[2] + (np.arange(nz) + 0.5) * dx
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X, Y, Z


def _direction(direction, shape, dx):
    """Unit propagation vector n and the wavelength d for which a wave of
    phase 2 pi (n.x - t)/d is periodic on the box (side L = N dx)."""
    nx, ny, nz = shape
    L = nx * dx
    if direction == "x":
        return np.array([1.0, 0.0, 0.0]), L
    if direction == "xy":
        if ny != nx:
            raise ValueError("xy wave needs a square lattice")
        return np.array([1.0, 1.0, 0.0]) / math.sqrt(2), L / math.sqrt(2)
    if direction == "xyz":
        if not (ny == nx and nz == nx):
            raise ValueError("xyz wave needs a cubic lattice")
        return np.array([1.0, 1.0, 1.0]) / math.sqrt(3), L / math.sqrt(3)
    raise ValueError(direction)


def _pack(alpha, g, K, V, shape):
    nx, ny, nz = shape
    out = np.zeros((NF, nz, ny, nx))
    out[0] = alpha
    for p, (i, j) in enumerate(PAIRS):
        out[1 + p] = g[i][j]
        out[7 + p] = K[i][j]
    for k in range(3):
        out[13 + k] = V[k]
    return out


def _shifted_u(n, shape, dx, t, beta):
    """u = n.(x + beta t): a zero-shift solution seen from coordinates that
    move with the constant velocity -beta. In them the shift is beta^i, the
    lapse, metric and extrinsic curvature keep their values, and the fields
    at x are the zero-shift fields at x + beta t."""
    X, Y, Z = coords(shape, dx)
    b = (0.0, 0.0, 0.0) if beta is None else tuple(float(v) for v in beta)
    return n[0] * (X + b[0] * t) + n[1] * (Y + b[1] * t) + n[2] * (Z + b[2] * t)


def gauge_wave(shape, dx, A, t=0.0, direction="x", beta=None):
    """Gauge wave (Sec. "Gauge Wave"): ds^2 = -H dt^2 + H du^2 + (transverse),
    H = 1 - A sin(2 pi (u - t)/d), u = n.x; alpha = sqrt(H),
    gamma = delta + (H - 1) n n, K = -(pi A/d) cos(phase)/sqrt(H) n n, V = 0.
    Harmonic slicing. beta: a constant shift (u = n.(x + beta t))."""
    n, d = _direction(direction, shape, dx)
    u = _shifted_u(n, shape, dx, t, beta)
    ph = 2 * math.pi * (u - t) / d
    H = 1 - A * np.sin(ph)
    Knn = -(math.pi * A / d) * np.cos(ph) / np.sqrt(H)
    g = [[(1.0 if i == j else 0.0) + (H - 1) * n[i] * n[j] for j in range(3)] for i in range(3)]
    K = [[Knn * n[i] * n[j] for j in range(3)] for i in range(3)]
    zero = np.zeros_like(H)
    return _pack(np.sqrt(H), g, K, [zero, zero, zero], shape)


def shear_shift(shape, dx, v0):
    """Static shift field beta = (v(y), 0, 0), v(y) = v0 sin(2 pi y / L_y):
    [3][nz][ny][nx]."""
    nx, ny, nz = shape
    X, Y, Z = coords(shape, dx)
    out = np.zeros((3, nz, ny, nx))
    out[0] = v0 * np.sin(2 * math.pi * Y / (ny * dx))
    return out


def shear_shift3(shape, dx, v0):
    """Divergence-free static shift field on a 3D lattice: beta^x =
    v0 sin(2 pi y/L_y), beta^y = v0 sin(2 pi z/L_z), beta^z = v0 sin(2 pi x/L_x).
    Each component varies across its own direction only, so the coordinates
    it carries shear (the Jacobian grows linearly in time) rather than
    converge on the field's sinks (where a compressive field makes the metric
    grow exponentially). [3][nz][ny][nx]."""
    nx, ny, nz = shape
    X, Y, Z = coords(shape, dx)
    out = np.zeros((3, nz, ny, nx))
    out[0] = v0 * np.sin(2 * math.pi * Y / (ny * dx))
    out[1] = v0 * np.sin(2 * math.pi * Z / (nz * dx))
    out[2] = v0 * np.sin(2 * math.pi * X / (nx * dx))
    return out


def smooth_shift(shape, dx, amp, seed, modes=1):
    """A seeded smooth periodic shift field [3][nz][ny][nx]: per component a
    few Fourier modes of amplitude amp along the lattice's axes of extent
    > 1 (no constant part)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    X, Y, Z = coords(shape, dx)
    L = (nx * dx, ny * dx, nz * dx)
    live = [a for a, n in enumerate(shape) if n > 1]
    out = np.zeros((3, nz, ny, nx))
    for i in range(3):
        for _ in range(2):
            k = np.zeros(3)
            for a in live:
                k[a] = rng.integers(-modes, modes + 1) / L[a]
            if not k.any() and live:
                k[live[0]] = 1.0 / L[live[0]]
            ph = 2 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + rng.uniform(0, 2 * math.pi)
            out[i] += amp * rng.uniform(0.5, 1.0) * np.sin(ph)
    return out


def sheared_gauge_wave(shape, dx, A, v0, t=0.0):
    """The gauge wave along x (A = 0: flat space) in coordinates carried by
    the flow of the static shift field of shear_shift(v0): x = x' + v(y') t,
    y = y'. In them the shift is beta = (v(y'), 0, 0), alpha keeps its
    value, and gamma, K transform with the Jacobian J (dx/dy' = s = v'(y') t):
    gamma'_xx = H, gamma'_xy = H s, gamma'_yy = 1 + H s^2, K' = K_xx (1, s,
    s^2) on (xx, xy, yy). V_k is its defining combination of the exact
    derivatives of gamma'. Harmonic slicing. Needs ny > 1."""
    nx, ny, nz = shape
    X, Y, Z = coords(shape, dx)
    d = nx * dx
    ky = 2 * math.pi / (ny * dx)
    v = v0 * np.sin(ky * Y)
    s = v0 * ky * np.cos(ky * Y) * t          # v'(y) t
    s1 = -v0 * ky * ky * np.sin(ky * Y) * t   # v''(y) t
    ph = 2 * math.pi * ((X + v * t) - t) / d
    H = 1 - A * np.sin(ph)
    Hx = -A * np.cos(ph) * 2 * math.pi / d
    Kxx = -(math.pi * A / d) * np.cos(ph) / np.sqrt(H)
    zero, one = np.zeros_like(H), np.ones_like(H)
    g = [[H, H * s, zero], [H * s, 1 + H * s * s, zero], [zero, zero, one]]
    K = [[Kxx, Kxx * s, zero], [Kxx * s, Kxx * s * s, zero], [zero, zero, zero]]
    # D_kij = d_k gamma_ij / 2 (exact), then V_k = g^{rs} (D_krs - D_rsk)
    Dx = [[Hx, Hx * s, zero], [Hx * s, Hx * s * s, zero], [zero, zero, zero]]
    Dy = [[Hx * s, Hx * s * s + H * s1, zero],
          [Hx * s * s + H * s1, Hx * s ** 3 + 2 * H * s * s1, zero], [zero, zero, zero]]
    D = np.zeros((3, 3, 3) + H.shape)
    for i in range(3):
        for j in range(3):
            D[0, i, j] = 0.5 * Dx[i][j]
            D[1, i, j] = 0.5 * Dy[i][j]
    G = np.array([[g[i][j] for j in range(3)] for i in range(3)])
    Gi = np.linalg.inv(np.moveaxis(G, (0, 1), (-2, -1)))
    Gi = np.moveaxis(Gi, (-2, -1), (0, 1))
    V = np.einsum("rs...,krs...->k...", Gi, D) - np.einsum("rs...,rsk...->k...", Gi, D)
    return _pack(np.sqrt(H), g, K, [V[0], V[1], V[2]], shape)


def gauge_wave_derivatives(shape, dx, A, t=0.0, direction="x"):
    """Exact A_k = d_k ln alpha and D_kij = d_k gamma_ij / 2 of the gauge wave,
    [21][nz][ny][nx]: A_x A_y A_z, then D_kij at 3 + 6 k + pair (pairs xx xy
    xz yy yz zz). With H' = dH/du = -(2 pi A/d) cos(phase): A_k = H' n_k / (2H),
    D_kij = H' n_k n_i n_j / 2."""
    n, d = _direction(direction, shape, dx)
    u = _shifted_u(n, shape, dx, t, None)
    ph = 2 * math.pi * (u - t) / d
    H = 1 - A * np.sin(ph)
    Hu = -(2 * math.pi * A / d) * np.cos(ph)
    out = np.zeros((21,) + H.shape)
    for k in range(3):
        out[k] = 0.5 * Hu * n[k] / H
        for p, (i, j) in enumerate(PAIRS):
            out[3 + 6 * k + p] = 0.5 * Hu * n[k] * n[i] * n[j]
    return out


def _polarisation(direction):
    if direction == "x":
        return np.array([0.0, 1.0, 0.0]), np.array([0.0, 0.0, 1.0])
    if direction == "xy":
        return np.array([1.0, -1.0, 0.0]) / math.sqrt(2), np.array([0.0, 0.0, 1.0])
    if direction == "xyz":
        return (np.array([1.0, -1.0, 0.0]) / math.sqrt(2),
                np.array([1.0, 1.0, -2.0]) / math.sqrt(6))
    raise ValueError(direction)


def linear_wave(shape, dx, A, t=0.0, direction="x", beta=None):
    """Linear (gravitational) wave (Sec. "Linear Wave"): alpha = 1,
    gamma = delta + b (e1 e1 - e2 e2), b = A sin(2 pi (u - t)/d),
    K = (pi A/d) cos(phase) (e1 e1 - e2 e2). Geodesic slicing.
    V_k = -b b' n_k / (1 - b^2) is V's defining combination of the closed-form
    metric derivatives, with b' = db/du. beta: a constant shift
    (u = n.(x + beta t))."""
    n, d = _direction(direction, shape, dx)
    e1, e2 = _polarisation(direction)
    u = _shifted_u(n, shape, dx, t, beta)
    ph = 2 * math.pi * (u - t) / d
    b = A * np.sin(ph)
    bp = (2 * math.pi * A / d) * np.cos(ph)
    P = np.outer(e1, e1) - np.outer(e2, e2)
    g = [[(1.0 if i == j else 0.0) + b * P[i, j] for j in range(3)] for i in range(3)]
    K = [[(math.pi * A / d) * np.cos(ph) * P[i, j] for j in range(3)] for i in range(3)]
    Vn = -b * bp / (1 - b * b)
    V = [Vn * n[k] for k in range(3)]
    return _pack(np.ones_like(b), g, K, V, shape)


def kasner(shape, p=(-1 / 3, 2 / 3, 2 / 3), t=1.0):
    """Kasner vacuum solution in synchronous gauge (alpha = 1, geodesic slicing):
    gamma_ii = t^(2 p_i), K_ii = -p_i t^(2 p_i - 1), with sum p = sum p^2 = 1.
    Spatially homogeneous, so every lattice reduces it to one cell."""
    nx, ny, nz = shape
    one = np.ones((nz, ny, nx))
    g = [[(t ** (2 * p[i]) * one if i == j else 0 * one) for j in range(3)] for i in range(3)]
    K = [[(-p[i] * t ** (2 * p[i] - 1) * one if i == j else 0 * one) for j in range(3)]
         for i in range(3)]
    return _pack(one, g, K, [0 * one] * 3, shape)


def smooth_modes(shape, dx, amp, seed, modes=2):
    """Flat space plus, in every one of the 16 fields, a few smooth periodic
    Fourier modes of amplitude amp (seeded): generic initial data for the
    evolution system, constraints not imposed. Modes run along the lattice's
    axes of extent > 1, wave numbers 1..modes per box length."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    X, Y, Z = coords(shape, dx)
    L = (nx * dx, ny * dx, nz * dx)
    out = flat(shape).copy()
    live = [a for a, n in enumerate(shape) if n > 1]
    for F in range(NF):
        for _ in range(modes):
            k = np.zeros(3)
            for a in live:
                k[a] = rng.integers(-modes, modes + 1) / L[a]
            if not k.any():
                k[live[0]] = 1.0 / L[live[0]]
            ph = 2 * math.pi * (k[0] * X + k[1] * Y + k[2] * Z) + rng.uniform(0, 2 * math.pi)
            out[F] += amp * rng.uniform(0.5, 1.0) * np.sin(ph)
    return out


def flat(shape):
    """Minkowski space: alpha = 1, gamma = delta, K = V = 0."""
    nx, ny, nz = shape
    one = np.ones((nz, ny, nx))
    zero = np.zeros((nz, ny, nx))
    g = [[(one if i == j else zero) for j in range(3)] for i in range(3)]
    return _pack(one, g, [[zero] * 3] * 3, [zero] * 3, shape)


def add_noise(fields, amp, seed):
    """Adds uniform noise U[-amp, amp] to all 16 fields (seeded)."""
    rng = np.random.default_rng(seed)
    return fields + rng.uniform(-amp, amp, size=fields.shape)


def flat_value():
    """Flat-space value of each of the 16 fields."""
    v = np.zeros(NF)
    v[0] = 1.0
    v[1] = v[4] = v[6] = 1.0
    return v


def random_distributions(Q, weights, shape, seed, amp=1e-3, smooth_amp=2e-2):
    """A seeded distribution state f[16][Q][cells] near flat space:
    f = w_l (flat + smooth(x) + amp * u) with u ~ U[-1, 1] per value and a
    smooth periodic perturbation per field. Used to exercise every term of
    one step; it is not a solution of anything."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    X, Y, Z = coords(shape, 1.0 / nx)
    w = np.asarray(weights, dtype=np.float64)
    base = flat_value()
    f = np.empty((NF, Q, nz * ny * nx))
    for F in range(NF):
        kx, ky, kz = rng.integers(1, 3, size=3)
        ph = rng.uniform(0, 2 * math.pi, size=3)
        sm = smooth_amp * (np.sin(2 * math.pi * kx * X + ph[0])
                           * np.cos(2 * math.pi * ky * Y * (ny > 1) + ph[1])
                           * np.cos(2 * math.pi * kz * Z * (nz > 1) + ph[2]))
        sm = sm.reshape(-1)
        for lam in range(Q):
            f[F, lam] = w[lam] * (base[F] + sm + amp * rng.uniform(-1, 1, size=sm.shape))
    return f


def ensemble(nruns=512, seed=150502037, n1=(64, 4096), n2=(64, 512), tau=(0.51, 2.0),
             amp=(1e-3, 1e-1), crossings=10):
    """Seeded parameters of an ensemble of independent gauge-wave runs on the
    unit periodic box: each run is 1D (D1Q3, N cells) or 2D (D2Q9, N x N)
    with equal probability, N uniform in n1 (1D) or n2 (2D), dx = dt = 1/N,
    tau uniform in `tau`, A log-uniform in `amp`, and crossings * N steps.
    2D runs of even id propagate along x, odd ones along the (1,1) diagonal
    (wavelength 1/sqrt(2), so the wave is periodic on the box)."""
    rng = np.random.default_rng(seed)
    runs = []
    for r in range(nruns):
        dim = 1 + int(rng.integers(0, 2))
        lo, hi = n1 if dim == 1 else n2
        N = int(rng.integers(lo, hi + 1))
        t = float(rng.uniform(tau[0], tau[1]))
        A = float(math.exp(rng.uniform(math.log(amp[0]), math.log(amp[1]))))
        direction = "x" if (dim == 1 or r % 2 == 0) else "xy"
        shape = (N, 1, 1) if dim == 1 else (N, N, 1)
        runs.append(dict(run=r, vset=dim, shape=shape, N=N, dx=1.0 / N, tau=t, A=A,
                         direction=direction, steps=crossings * N))
    return runs


def ensemble_fields(spec):
    """Initial fields [16][cells] of one ensemble run (gauge wave, t = 0)."""
    return gauge_wave(spec["shape"], spec["dx"], spec["A"], direction=spec["direction"])


def flrw_exponent(w):
    """a(t) ~ t^q for a flat universe filled with a perfect fluid P = w rho
    (c^2 = 8 pi G = 1): q = 2 / (3 (1 + w))."""
    return 2.0 / (3.0 * (1.0 + w))


def flrw_density(t, w=1.0):
    """Energy density of that universe at time t: rho = 3 (q / t)^2 (for
    w = 1, 1 / (3 t^2) as in Sec. "Expansion of flat universe")."""
    q = flrw_exponent(w)
    return 3.0 * q * q / (t * t)


def flrw(shape, t=1.0, w=1.0):
    """Flat expanding universe in comoving coordinates, geodesic slicing:
    alpha = 1, gamma_ij = t^(2q) delta_ij (= t^(2/3) delta for w = 1, equal
    to delta at t = 1), K_ij = -(1/2) d_t gamma_ij = -q t^(2q-1) delta_ij,
    V = 0."""
    q = flrw_exponent(w)
    cells = int(np.prod(shape))
    out = np.zeros((NF, cells))
    out[0] = 1.0
    g = t ** (2 * q)
    k = -q * t ** (2 * q - 1)
    for qq in (0, 3, 5):  # xx, yy, zz
        out[1 + qq] = g
        out[7 + qq] = k
    return out
