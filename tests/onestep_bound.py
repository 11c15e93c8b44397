"""Bound on the difference between one reduced-precision step of the CUDA
path and the FP64 oracle's step taken from the same stored state.

Both sides start from the same stored values (the oracle reads them decoded
to FP64, exactly), so the difference comes only from the step's own FP32
arithmetic and from rounding its output to the storage type. With u the
unit roundoff of FP32 (2^-24), u_s that of the storage (2^-24 FP32, 2^-11
FP16, 2^-8 BF16), Q velocities, dx = dt, omega = 1/tau, and t_l the term a
moment sum adds (f_l for absolute storage, f_l - w_l rho_flat for
deviation storage), the contributions per output value are:

  output rounding    u_s |t_out|
  moment sums        sum_l t_l in FP32 is off by at most (Q - 1) u sum_l |t_l|
                     (E_mom; the lapse adds u for its logarithm)
  derivatives        central differences divide two such errors by 2 dx
                     (A_k) or 4 dx (D_kij):  dA = E_mom / dx, dD = E_mom / (2 dx)
  flux of K_ij       alpha lambda^k_ij; near flat space the coefficients of the
                     D and A components in one lambda^k_ij add to at most 4 and 1
                     (Sec. "Bona-Masso evolution equations"), so
                     dF = alpha_max (4 dD + dA)
  equilibrium        3 omega w_l c_l . F: at most 3 omega dF max_l(w_l sum_k |c_lk|)
                     (K fields only: alpha, gamma and V carry no flux at zero shift)
  corrected moment   omega w_l rho: omega w_max E_mom of the field itself
  update arithmetic  a few roundings of values of size |t|: 8 u (|t_in| + |t_out|)
  sources            S_ij (in the source of K_ij) and Omega_k (of V_k) are sums of
                     products of two first-order quantities (D, A, V, K) with metric
                     factors near 1; counting generously, at most C_S = 256
                     products. With M1 the largest first-order value and dM1 the
                     largest error of one (dD, dA, or a moment error),
                     dS <= C_S (2 M1 dM1 + 4 u M1^2). The source enters the
                     update through sigma w S and omega w dt S/2, together
                     w dt S, so it adds w_max dt dS (dt = dx cancels no 1/dx
                     here: dM1 already carries it).

The derivative terms carry 1/dx and dominate for absolute storage; for
deviation storage the sums are small (the fields' deviations from flat
space) and the output rounding dominates. The bound is twice the sum, so
that the orders of magnitude the derivation leaves out (products of two
errors, the V and source terms, which are multiplied by dt = dx and so
lose the 1/dx) stay inside it.
"""
import numpy as np

U_C = 2.0 ** -24
U_STORE = {"f32": 2.0 ** -24, "dev_f32": 2.0 ** -24, "dev_f16": 2.0 ** -11,
           "dev_bf16": 2.0 ** -8}
FLAT = np.array([1.0, 1, 0, 0, 1, 0, 1] + [0.0] * 9)
K_FIELDS = slice(7, 13)


def terms(storage, w, f):
    """Per value, what the moment sums add: f, or f - w_l rho_flat."""
    Q = len(w)
    f = f.reshape(16, Q, -1)
    if storage.startswith("dev"):
        return f - np.asarray(w).reshape(1, Q, 1) * FLAT.reshape(16, 1, 1)
    return f


C_S = 256


def one_step_bound(storage, c, w, tau, dx, f_in, f_out, alpha_max, first_order_max):
    """Per-field bound [16] on max |f_gpu - f_oracle| (distribution units)
    after one step. f_in: the input state around the compared cells
    [16][Q][cells] (decoded); f_out: the oracle's output at the compared
    cells [16][Q][cells]; alpha_max: the largest lapse of the state;
    first_order_max: the largest |D_kij|, |A_k|, |K_ij| or |V_k| of the
    state (M1)."""
    c = np.asarray(c)
    w = np.asarray(w, dtype=np.float64)
    Q = len(w)
    om = 1.0 / tau
    t_in = terms(storage, w, f_in)
    t_out = terms(storage, w, f_out)
    s_field = np.abs(t_in).sum(axis=1).max(axis=1)          # [16]: max_x sum_l |t_l|
    e_mom = (Q - 1) * U_C * s_field                          # [16]
    e_ag = e_mom[:7].max() + U_C                             # alpha (with its log) and gamma
    dA = e_ag / dx
    dD = e_ag / (2 * dx)
    dF = alpha_max * (4 * dD + dA)
    flux_w = (w * np.abs(c).sum(axis=1)).max()
    e_flux = np.zeros(16)
    e_flux[K_FIELDS] = 3 * om * dF * flux_w
    e_out = U_STORE[storage] * np.abs(t_out).max(axis=(1, 2))
    e_rho = om * w.max() * e_mom
    e_arith = 8 * U_C * (np.abs(t_in).max(axis=(1, 2)) + np.abs(t_out).max(axis=(1, 2)))
    M1 = first_order_max
    dM1 = max(dA, dD, e_mom[7:].max())
    e_src = w.max() * dx * C_S * (2 * M1 * dM1 + 4 * U_C * M1 ** 2)
    return 2 * (e_out + e_flux + e_rho + e_arith + e_src)


def first_order_max(rho, dx, dims, periodic=True):
    """Largest |D_kij|, |A_k|, |K_ij|, |V_k| of fields rho [16][nz][ny][nx],
    D and A by central differences along the lattice's first `dims` axes
    (periodic, or at interior points only for a patch cut out of a larger
    lattice)."""
    rho = np.asarray(rho)
    m = float(np.abs(rho[7:]).max())
    planes = [np.log(rho[0])] + [rho[1 + q] for q in range(6)]
    scale = [1 / (2 * dx)] + [1 / (4 * dx)] * 6
    for ax in range(dims):
        a = 2 - ax  # x is the last array axis
        for p, sc in zip(planes, scale):
            if periodic:
                d = np.roll(p, -1, a) - np.roll(p, 1, a)
            else:
                n = p.shape[a]
                d = np.take(p, range(2, n), a) - np.take(p, range(0, n - 2), a)
            m = max(m, float(np.abs(d).max()) * sc)
    return m


def field_max_err(g, o):
    """Per field: max |g - o| over velocities and cells; both [16][...]."""
    return np.abs(np.asarray(g).reshape(16, -1) - np.asarray(o).reshape(16, -1)).max(axis=1)
