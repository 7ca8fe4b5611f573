"""Deterministic 2-D steady transport solver for the axisymmetric heliosphere
without a current sheet (test infrastructure only: used by tests/, never by
the library).

Independent whole-path check of the SDE method for the anisotropic model: the
Parker-spiral diffusion tensor (K_par along the field, K_perp,r and K_perp,th
across it, Eq. 2), the two-speed wind, the termination-shock factor of K, and
the gradient-curvature drift of a unipolar field, v_d = sgn(q) sgn(A) curl(kappa_A e_B)
with kappa_A = beta P / (3 |B|) (the drift of Eq. 1).  Without a current sheet
none of these coefficients depends on the longitude, and neither does the
phase-space density seen from any (r, th), so the steady momentum-form
transport equation (Eq. 5 with df/dt = 0) reduces to (r, th):

    div(K grad f) - (V + v_d) . grad f + (1/3) div(V) df/dlnP = 0,
    div(K grad f) = r^-2 d_r(r^2 K_rr d_r f) + (r^2 sin th)^-1 d_th(sin th K_thth d_th f),

(a field with no th component makes K_rth = K_thph = 0, and K_rph does not act
on a longitude-independent f), div V = 2 V(th) / r.  Boundary conditions are
those of the SDE paths: f = f_LIS(P) on r = R_out (absorbing), d_r f = 0 on
r = r_in (reflecting), no flux through the poles.  As in the 1-D solver the
lnP term has a positive coefficient, so the problem is parabolic marched
toward lower rigidity in tau = lnP_top - lnP:

    df/dtau = (3 r / (2 V(th))) [div(K grad f) - (V + v_d) . grad f].

Discretisation: finite volumes, cell faces equally spaced in ln(r + 1 AU) and
in th; diffusive fluxes in conservative form (the Ito drift of the SDE never
appears here: the divergence form implies it); advection by central
differences with mirror ghosts at r_in and at the poles and the Dirichlet
ghost 2 f_LIS - f at R_out; BDF2 in tau after one backward-Euler step.  Every
coefficient scales with rigidity as beta P (K and kappa_A) or not at all
(the wind), so the spatial operator is assembled once as
S(P) = beta P S_1 + S_0 and only the linear solve is repeated per step.

The coefficients are computed here from the model's definitions (wind profile,
spiral angle, |B| normalised at 1 AU on the equator, kappa_A converted from SI
to AU^2/day); the drift is the curl of kappa_A e_B taken by central
differences of that analytic vector potential.  Nothing is shared with the SDE
oracle in cosmica_oracle.c.  The modulated intensity per kinetic energy is
J(T0) = P0^2 f(r0, th0, P0) with f_LIS = J_LIS / P^2, the quantity the Monte
Carlo estimator of Eq. 4 computes.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

AU_KM = 1.495978707e8
AU_M = 1.495978707e11
DAY_S = 86400.0
DEG = math.pi / 180.0


def lis(T):
    T = np.asarray(T, np.float64)
    return T ** -2.7 / (1.0 + T ** -3.7)


def _beta_T(species, P):
    pn = P * abs(species["Z"]) / species["A"]
    E = math.sqrt(pn * pn + species["m0"] ** 2)
    return pn / E, pn * pn / (E + species["m0"])


def f_lis(species, P):
    _, T = _beta_T(species, P)
    return float(lis(T)) / P ** 2


class _Model:
    """Coefficients per unit beta P [GV] of the axisymmetric model."""

    def __init__(self, p, species):
        self.p = p
        self.Vs = p["V_slow_kms"] * DAY_S / AU_KM
        self.Vf = p["V_fast_kms"] * DAY_S / AU_KM
        self.Om = 2.0 * math.pi / p["rot_period_day"]
        G_eq = self.Om / float(self.V(0.5 * math.pi))          # spiral at 1 AU on the equator
        self.B0 = p["B1AU_nT"] / math.sqrt(1.0 + G_eq * G_eq)   # |B| = B0 sqrt(1 + Gam^2) / r^2
        self.sign = math.copysign(1.0, species["Z"]) * p["polarity"]

    def V(self, th):
        lat = np.abs(0.5 * math.pi - np.asarray(th, np.float64))
        step = np.tanh((lat - self.p["lat_fast_deg"] * DEG) / (self.p["dlat_deg"] * DEG))
        return self.Vs + (self.Vf - self.Vs) * 0.5 * (1.0 + step)

    def gamma(self, r, th):
        return self.Om * r * np.sin(th) / self.V(th)

    def shock(self, r):
        p = self.p
        if p["R_ts"] <= 0.0:
            return np.ones_like(np.asarray(r, np.float64))
        return 1.0 - (1.0 - p["ts_K_factor"]) * 0.5 * (1.0 + np.tanh((r - p["R_ts"]) / p["dts_AU"]))

    def K1(self, r, th):
        """(K_rr, K_thth) / (beta P): the spiral angle psi has tan psi = Gamma."""
        Kpar = self.p["K0"] * self.shock(r)
        cos2 = 1.0 / (1.0 + self.gamma(r, th) ** 2)
        Krr = Kpar * cos2 + self.p["kperp_r_frac"] * Kpar * (1.0 - cos2)
        return Krr, self.p["kperp_th_frac"] * Kpar

    def A_ph1(self, r, th):
        """Azimuthal component of kappa_A e_B per unit beta P [AU^2/day]; e_B = (e_r - Gam e_ph)/|..|."""
        G = self.gamma(r, th)
        kappa = 1e9 * DAY_S / (3.0 * self.B0 * 1e-9 * AU_M * AU_M) * r * r / np.sqrt(1.0 + G * G)
        return -kappa * G / np.sqrt(1.0 + G * G)

    def drift1(self, r, th):
        """(v_r, v_th) / (beta P) of sgn(q) sgn(A) curl(kappa_A e_B) for a longitude-independent
        potential whose th component vanishes: v_r = d_th(sin th A_ph) / (r sin th),
        v_th = -d_r(r A_ph) / r (central differences of the analytic potential)."""
        if not self.p["drift_on"]:
            z = np.zeros(np.broadcast(r, th).shape)
            return z, z
        e = 1e-5
        vr = (np.sin(th + e) * self.A_ph1(r, th + e) - np.sin(th - e) * self.A_ph1(r, th - e)) / (2 * e)
        vr = vr / (r * np.sin(th))
        h = e * r
        vt = -((r + h) * self.A_ph1(r + h, th) - (r - h) * self.A_ph1(r - h, th)) / (2 * h) / r
        return self.sign * vr, self.sign * vt


def _grid(p, n_r, n_th):
    a = 1.0   # AU: faces equally spaced in ln(r + a)
    s = np.linspace(math.log(p["r_in"] + a), math.log(p["R_out"] + a), n_r + 1)
    rf = np.exp(s) - a
    rf[0], rf[-1] = p["r_in"], p["R_out"]
    tf = np.linspace(0.0, math.pi, n_th + 1)
    return rf, 0.5 * (rf[1:] + rf[:-1]), tf, 0.5 * (tf[1:] + tf[:-1])


def _operators(m, species, rf, rc, tf, tc):
    """S_1, b_1 (per unit beta P) and S_0, b_0 of the spatial operator S f + b f_LIS."""
    n_r, n_th = len(rc), len(tc)
    N = n_r * n_th
    R, r_in = rf[-1], rf[0]
    I, J = np.meshgrid(np.arange(n_r), np.arange(n_th), indexing="ij")
    ix = I * n_th + J
    dcos = np.cos(tf[:-1]) - np.cos(tf[1:])
    vol = ((rf[1:] ** 3 - rf[:-1] ** 3) / 3.0)[:, None] * dcos[None, :]
    parts = {1: ([], [], [], np.zeros(N)), 0: ([], [], [], np.zeros(N))}

    def add(which, i, j, v):
        rows, cols, vals, _ = parts[which]
        rows.append(np.ravel(i)); cols.append(np.ravel(j)); vals.append(np.ravel(v))

    def rhs(which, i, v):
        np.add.at(parts[which][3], np.ravel(i), np.ravel(v))

    # radial diffusive fluxes through interior faces, and through R_out to the boundary value
    Krr_f, _ = m.K1(rf[1:-1][:, None], tc[None, :])
    a = Krr_f * (rf[1:-1] ** 2)[:, None] * dcos[None, :] / (rc[1:] - rc[:-1])[:, None]
    lo, up = ix[:-1], ix[1:]
    add(1, lo, up, a / vol[:-1]); add(1, lo, lo, -a / vol[:-1])
    add(1, up, lo, a / vol[1:]); add(1, up, up, -a / vol[1:])
    Krr_R, _ = m.K1(np.full(n_th, R), tc)
    aR = Krr_R * R * R * dcos / (R - rc[-1])
    last = ix[-1]
    add(1, last, last, -aR / vol[-1]); rhs(1, last, aR / vol[-1])
    # latitudinal diffusive fluxes (the pole faces carry none: sin th = 0)
    _, Ktt_f = m.K1(rc[:, None], tf[1:-1][None, :])
    ring = ((rf[1:] ** 2 - rf[:-1] ** 2) / 2.0)[:, None]
    a = Ktt_f * np.sin(tf[1:-1])[None, :] * ring / (rc[:, None] * (tc[1:] - tc[:-1])[None, :])
    lo, up = ix[:, :-1], ix[:, 1:]
    add(1, lo, up, a / vol[:, :-1]); add(1, lo, lo, -a / vol[:, :-1])
    add(1, up, lo, a / vol[:, 1:]); add(1, up, up, -a / vol[:, 1:])
    # advection -u_r d_r f - (u_th / r) d_th f by central differences with ghosts
    RC, TC = np.meshgrid(rc, tc, indexing="ij")
    vr1, vt1 = m.drift1(RC, TC)
    r_lo = np.concatenate([[2.0 * r_in - rc[0]], rc[:-1]])
    r_hi = np.concatenate([rc[1:], [2.0 * R - rc[-1]]])
    t_lo = np.concatenate([[-tc[0]], tc[:-1]])
    t_hi = np.concatenate([tc[1:], [2.0 * math.pi - tc[-1]]])
    for which, ur, ut in ((0, m.V(TC), 0.0 * TC), (1, vr1, vt1 / RC)):
        c = -ur / (r_hi - r_lo)[:, None]            # times (f_{i+1} - f_{i-1})
        add(which, ix[:-1], ix[1:], c[:-1]); add(which, ix[1:], ix[:-1], -c[1:])
        add(which, ix[0], ix[0], -c[0])             # reflecting: ghost f_{-1} = f_0
        add(which, last, last, -c[-1]); rhs(which, last, 2.0 * c[-1])   # ghost 2 f_LIS - f
        ct = -ut / (t_hi - t_lo)[None, :]
        add(which, ix[:, :-1], ix[:, 1:], ct[:, :-1]); add(which, ix[:, 1:], ix[:, :-1], -ct[:, 1:])
        add(which, ix[:, 0], ix[:, 0], -ct[:, 0])    # across a pole the density is the same
        add(which, ix[:, -1], ix[:, -1], ct[:, -1])
    out = []
    for which in (1, 0):
        rows, cols, vals, b = parts[which]
        S = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))
        out += [S, b]
    return out


def solve(species, p, r0, th0, P0_list, n_r=80, n_th=90, dlnP=0.01, P_top=300.0):
    """Modulated J(T0) at (r0, th0) for each rigidity in P0_list (GV).

    p is a parameter dict with the keys of the model record (K0, kperp_r_frac,
    kperp_th_frac, B1AU_nT, V_slow_kms, V_fast_kms, lat_fast_deg, dlat_deg,
    polarity, drift_on, R_out, R_ts, ts_K_factor, dts_AU, r_in, rot_period_day);
    the model must be anisotropic, without a current sheet, shells or squashed
    boundaries."""
    if p.get("isotropic", 0.0) or p.get("hcs_on", 0.0) or p.get("n_shells", 0.0) or p.get("squashed", 0.0):
        raise ValueError("the 2-D solver covers the axisymmetric model without a current sheet")
    m = _Model(p, species)
    rf, rc, tf, tc = _grid(p, n_r, n_th)
    if not (rc[0] < r0 < rc[-1] and tc[0] < th0 < tc[-1]):
        raise ValueError("the observer must lie between cell centres")
    S1, b1, S0, b0 = _operators(m, species, rf, rc, tf, tc)
    N = n_r * n_th
    RC, TC = np.meshgrid(rc, tc, indexing="ij")
    M = sp.diags((3.0 * RC / (2.0 * m.V(TC))).ravel(), format="csc")
    MS1, MS0 = M @ S1, M @ S0
    Mb1, Mb0 = M @ b1, M @ b0
    Id = sp.identity(N, format="csc")
    # bilinear weights of the observer between cell centres
    i = int(np.searchsorted(rc, r0)) - 1
    j = int(np.searchsorted(tc, th0)) - 1
    wr = (r0 - rc[i]) / (rc[i + 1] - rc[i])
    wt = (th0 - tc[j]) / (tc[j + 1] - tc[j])

    def at_observer(f):
        F = f.reshape(n_r, n_th)
        return ((1 - wr) * ((1 - wt) * F[i, j] + wt * F[i, j + 1]) +
                wr * ((1 - wt) * F[i + 1, j] + wt * F[i + 1, j + 1]))

    P0_list = np.asarray(P0_list, np.float64)
    y_top = math.log(P_top)
    n_y = int(math.ceil((y_top - math.log(P0_list.min())) / dlnP)) + 2
    ys = y_top - dlnP * np.arange(n_y + 1)
    f = np.full(N, f_lis(species, P_top))
    f_prev = None
    seen = [at_observer(f)]
    for n in range(n_y):
        P = math.exp(ys[n + 1])
        bP = _beta_T(species, P)[0] * P
        L = bP * MS1 + MS0
        src = dlnP * f_lis(species, P) * (bP * Mb1 + Mb0)
        if f_prev is None:                       # backward Euler for the first step
            A, rhs = Id - dlnP * L, f + src
        else:                                    # BDF2
            A, rhs = 1.5 * Id - dlnP * L, 2.0 * f - 0.5 * f_prev + src
        f_prev, f = f, spla.splu(A.tocsc()).solve(rhs)
        seen.append(at_observer(f))
    seen = np.asarray(seen)
    out = []
    for P0 in P0_list:
        k = (y_top - math.log(P0)) / dlnP
        k0 = int(math.floor(k))
        t = k - k0
        out.append(P0 ** 2 * (seen[k0] * (1 - t) + seen[k0 + 1] * t))
    return np.asarray(out)
