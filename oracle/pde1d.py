"""Deterministic 1-D steady Parker-equation solver (test infrastructure only).

Independent check of the Monte Carlo method for the spherically symmetric
case (isotropic K = K0 beta P, uniform radial wind V, no drift).  It solves the
steady momentum-form transport equation (Eq. 5 with df/dt = 0),

    (1/r^2) d_r(r^2 K d_r f) - V d_r f + (2V/(3r)) d f / d lnP = 0,

on r in [r_in, R] with f(R, P) = f_LIS(P) (absorbing boundary = the LIS) and
d_r f(r_in) = 0 (reflecting inner boundary).  Because the lnP-derivative has a
positive coefficient, the problem is parabolic when marched toward *lower*
rigidity: with tau = lnP_top - lnP,

    d f / d tau = (3 r / (2 V)) [K f_rr + (2K/r - V) f_r],

started from f = f_LIS at lnP_top (modulation is negligible at 10^4 GV) and
integrated with Crank-Nicolson in tau and second-order central differences in
r.  The modulated intensity per kinetic energy follows from J = f P^2 (Sec. VI):
J(T0) = P0^2 f(r0, P0), with f_LIS = J_LIS / P^2 at the boundary.

The Monte Carlo estimator of Eq. 4 computes exactly this quantity, so the two
must agree to within the Euler-Maruyama step bias plus Monte Carlo error.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_banded

AU_KM = 1.495978707e8
DAY_S = 86400.0


def lis(T):
    T = np.asarray(T, np.float64)
    return T ** -2.7 / (1.0 + T ** -3.7)


def _beta_T(species, P):
    pn = P * abs(species["Z"]) / species["A"]
    E = np.sqrt(pn * pn + species["m0"] ** 2)
    return pn / E, pn * pn / (E + species["m0"])


def f_lis(species, P):
    """Phase-space density at the boundary, up to a constant: J_LIS(T) / P^2."""
    b, T = _beta_T(species, P)
    return lis(T) / P ** 2


def solve(species, K0, V_kms, r_in, R, r0, P0_list, n_r=1200, dlnP=2e-3, P_top=1e4):
    """Modulated J(T0) at r0 for each rigidity in P0_list (GV).

    K0 is a number, or a function of r (array in, array out) for a radially
    varying diffusion normalisation K = K0(r) beta P.  In the latter case the
    radial operator is discretised in conservative (flux) form,
    (1/r^2)[(r^2 K)_{i+1/2}(f_{i+1} - f_i) - (r^2 K)_{i-1/2}(f_i - f_{i-1})]/h^2,
    which needs K at the cell faces only and no derivative of K."""
    V = V_kms * DAY_S / AU_KM
    r = np.linspace(r_in, R, n_r + 1)
    h = r[1] - r[0]
    flux = callable(K0)
    if flux:
        K0_face = np.asarray(K0(np.concatenate([[r[0] - 0.5 * h], r + 0.5 * h])), np.float64)
        r_face = np.concatenate([[r[0] - 0.5 * h], r + 0.5 * h])
        w_lo = r_face[:-1] ** 2 * K0_face[:-1] / (r ** 2 * h ** 2)   # (r^2 K0)_{i-1/2} / (r_i^2 h^2)
        w_up = r_face[1:] ** 2 * K0_face[1:] / (r ** 2 * h ** 2)     # (r^2 K0)_{i+1/2} / (r_i^2 h^2)
    P0_list = np.asarray(P0_list, np.float64)
    y_top = math.log(P_top)
    y_bot = math.log(P0_list.min()) - 2 * dlnP
    n_y = int(math.ceil((y_top - y_bot) / dlnP))
    ys = y_top - dlnP * np.arange(n_y + 1)

    def coeffs(y):
        P = math.exp(y)
        b, _ = _beta_T(species, P)
        a = 3.0 * r / (2.0 * V)                # prefactor
        if flux:
            bP = b * P
            lo = a * (bP * w_lo + V / (2 * h))
            up = a * (bP * w_up - V / (2 * h))
            di = -a * bP * (w_lo + w_up)
            # reflecting inner boundary: ghost f_{-1} = f_1
            up0 = lo[0] + up[0]
            return lo, di, up, up0
        K = K0 * b * P
        c2 = a * K                             # of f_rr
        c1 = a * (2.0 * K / r - V)             # of f_r
        lo = c2 / h ** 2 - c1 / (2 * h)        # coefficient of f_{i-1}
        di = -2.0 * c2 / h ** 2                # of f_i
        up = c2 / h ** 2 + c1 / (2 * h)        # of f_{i+1}
        # reflecting inner boundary: ghost f_{-1} = f_1
        up0 = lo[0] + up[0]
        return lo, di, up, up0

    def apply(f, lo, di, up, up0):
        out = di * f
        out[1:-1] += lo[1:-1] * f[:-2] + up[1:-1] * f[2:]
        out[0] += up0 * f[1]
        out[-1] = 0.0
        return out

    f = np.full(n_r + 1, f_lis(species, math.exp(y_top)))
    i0 = np.searchsorted(r, r0)
    w0 = (r0 - r[i0 - 1]) / h
    f_at_r0 = [f[i0 - 1] * (1 - w0) + f[i0] * w0]
    for n in range(n_y):
        lo_n, di_n, up_n, up0_n = coeffs(ys[n])
        lo_m, di_m, up_m, up0_m = coeffs(ys[n + 1])
        rhs = f + 0.5 * dlnP * apply(f, lo_n, di_n, up_n, up0_n)
        # banded matrix of (I - dtau/2 L^{n+1})
        ab = np.zeros((3, n_r + 1))
        ab[1, :] = 1.0 - 0.5 * dlnP * di_m
        ab[0, 1:] = -0.5 * dlnP * up_m[:-1]
        ab[0, 1] = -0.5 * dlnP * up0_m
        ab[2, :-1] = -0.5 * dlnP * lo_m[1:]
        # Dirichlet row at R
        ab[1, -1] = 1.0
        ab[2, -2] = 0.0
        rhs[-1] = f_lis(species, math.exp(ys[n + 1]))
        f = solve_banded((1, 1), ab, rhs)
        f_at_r0.append(f[i0 - 1] * (1 - w0) + f[i0] * w0)
    f_at_r0 = np.asarray(f_at_r0)
    out = []
    for P0 in P0_list:
        y0 = math.log(P0)
        k = (y_top - y0) / dlnP
        k0 = int(math.floor(k))
        t = k - k0
        fr0 = f_at_r0[k0] * (1 - t) + f_at_r0[k0 + 1] * t
        out.append(P0 ** 2 * fr0)
    return np.asarray(out)


def force_field(species, K0, V_kms, R, r0, T0):
    """Force-field approximation: J(T)/P(T)^2 = J_LIS(T+Phi)/P(T+Phi)^2,
    phi = V (R - r0) / (3 K0) [GV], Phi = (|Z|/A) phi."""
    V = V_kms * DAY_S / AU_KM
    phi = V * (R - r0) / (3.0 * K0)
    Phi = abs(species["Z"]) / species["A"] * phi
    T0 = np.asarray(T0, np.float64)

    def P(T):
        return species["A"] / abs(species["Z"]) * np.sqrt(T * (T + 2 * species["m0"]))

    return lis(T0 + Phi) * P(T0) ** 2 / P(T0 + Phi) ** 2, phi
