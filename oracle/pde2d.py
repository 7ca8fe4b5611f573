"""Deterministic 2-D steady transport solver for the axisymmetric heliosphere
(test infrastructure only: used by tests/, never by the library).

Independent whole-path check of the SDE method for the anisotropic model: the
Parker-spiral diffusion tensor (K_par along the field, K_perp,r and K_perp,th
across it, Eq. 2), the two-speed wind, the termination-shock factor of K, and
the drift v_d = sgn(q) sgn(A) curl(kappa_A h e_B), kappa_A = beta P / (3 |B|)
(the drift of Eq. 1), of a unipolar field (h = 1) or of a field reversing
across a flat current sheet (zero tilt: h = tanh((pi/2 - th) / delta),
delta = max(2 r_L / r, delta_min), r_L = P / (c |B|)).  Then none of the
coefficients depends on the longitude, and neither does the phase-space
density seen from any (r, th), so the steady momentum-form transport equation
(Eq. 5 with df/dt = 0) reduces to (r, th):

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
in th (optionally narrowing toward the equator); diffusive fluxes in
conservative form (the Ito drift of the SDE never appears here: the divergence
form implies it); advection by central differences with mirror ghosts at r_in
and at the poles and the Dirichlet ghost 2 f_LIS - f at R_out; BDF2 in tau
after one backward-Euler step.  K and kappa_A scale with rigidity as beta P
and the wind not at all, so the diffusion and wind operators are assembled
once; the drift operator too, unless a current sheet makes its width depend
on the rigidity.

The coefficients are computed here from the model's definitions (wind profile,
spiral angle, |B| normalised at 1 AU on the equator, kappa_A converted from SI
to AU^2/day); the drift is the curl of kappa_A h e_B taken by central
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
C_MS = 299792458.0


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

    def polarity_h(self, r, th, P):
        """Flat current sheet: h = tanh((pi/2 - th) / delta), delta = max(2 r_L / r, delta_min),
        r_L = P / (c |B|); h = 1 without a sheet."""
        if not self.p["hcs_on"]:
            return 1.0
        G = self.gamma(r, th)
        rL = P * 1e9 / (C_MS * self.B0 * 1e-9 * AU_M) * r * r / np.sqrt(1.0 + G * G)
        delta = np.maximum(2.0 * rL / r, self.p["dcs_min_deg"] * DEG)
        return np.tanh((0.5 * math.pi - th) / delta)

    def A_ph1(self, r, th, P):
        """Azimuthal component of kappa_A h e_B per unit beta P [AU^2/day]; e_B = (e_r - Gam e_ph)/|..|."""
        G = self.gamma(r, th)
        kappa = 1e9 * DAY_S / (3.0 * self.B0 * 1e-9 * AU_M * AU_M) * r * r / np.sqrt(1.0 + G * G)
        return -kappa * self.polarity_h(r, th, P) * G / np.sqrt(1.0 + G * G)

    def drift1(self, r, th, P):
        """(v_r, v_th) / (beta P) of sgn(q) sgn(A) curl(kappa_A h e_B) for a longitude-independent
        potential whose th component vanishes: v_r = d_th(sin th A_ph) / (r sin th),
        v_th = -d_r(r A_ph) / r (central differences of the analytic potential)."""
        if not self.p["drift_on"]:
            z = np.zeros(np.broadcast(r, th).shape)
            return z, z
        e = 1e-5
        vr = (np.sin(th + e) * self.A_ph1(r, th + e, P) - np.sin(th - e) * self.A_ph1(r, th - e, P)) / (2 * e)
        vr = vr / (r * np.sin(th))
        h = e * r
        vt = -((r + h) * self.A_ph1(r + h, th, P) - (r - h) * self.A_ph1(r - h, th, P)) / (2 * h) / r
        return self.sign * vr, self.sign * vt


def _grid(p, n_r, n_th, th_stretch=0.0):
    """Cell faces equally spaced in ln(r + 1 AU); in th equally spaced, or, with
    th_stretch = a > 0, th = pi/2 + (pi/2) sinh(a x) / sinh(a) for x equally spaced
    in [-1, 1] (cells narrowest on the equator, where a current sheet lies)."""
    a = 1.0
    s = np.linspace(math.log(p["r_in"] + a), math.log(p["R_out"] + a), n_r + 1)
    rf = np.exp(s) - a
    rf[0], rf[-1] = p["r_in"], p["R_out"]
    if th_stretch > 0.0:
        x = np.linspace(-1.0, 1.0, n_th + 1)
        tf = 0.5 * math.pi + 0.5 * math.pi * np.sinh(th_stretch * x) / math.sinh(th_stretch)
    else:
        tf = np.linspace(0.0, math.pi, n_th + 1)
    tf[0], tf[-1] = 0.0, math.pi
    return rf, 0.5 * (rf[1:] + rf[:-1]), tf, 0.5 * (tf[1:] + tf[:-1])


class _Assembler:
    """Finite-volume pieces of the spatial operator S f + b f_LIS on one grid."""

    def __init__(self, rf, rc, tf, tc):
        self.rf, self.rc, self.tf, self.tc = rf, rc, tf, tc
        self.n_r, self.n_th = len(rc), len(tc)
        self.N = self.n_r * self.n_th
        I, J = np.meshgrid(np.arange(self.n_r), np.arange(self.n_th), indexing="ij")
        self.ix = I * self.n_th + J
        self.dcos = np.cos(tf[:-1]) - np.cos(tf[1:])
        self.vol = ((rf[1:] ** 3 - rf[:-1] ** 3) / 3.0)[:, None] * self.dcos[None, :]
        self.RC, self.TC = np.meshgrid(rc, tc, indexing="ij")
        R, r_in = rf[-1], rf[0]
        self.dr2 = (np.concatenate([rc[1:], [2.0 * R - rc[-1]]]) -
                    np.concatenate([[2.0 * r_in - rc[0]], rc[:-1]]))
        self.dt2 = (np.concatenate([tc[1:], [2.0 * math.pi - tc[-1]]]) - np.concatenate([[-tc[0]], tc[:-1]]))

    def _new(self):
        return [], [], [], np.zeros(self.N)

    @staticmethod
    def _add(part, i, j, v):
        part[0].append(np.ravel(i)); part[1].append(np.ravel(j)); part[2].append(np.ravel(v))

    def _done(self, part):
        rows, cols, vals, b = part
        S = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(self.N, self.N))
        return S, b

    def diffusion(self, K1):
        """div(K grad f) for K = (K_rr, K_thth)(r, th) = K1(r, th): fluxes through interior faces,
        through R_out to the boundary value, none through r_in or the poles."""
        rf, rc, tf, tc, ix, vol, dcos = self.rf, self.rc, self.tf, self.tc, self.ix, self.vol, self.dcos
        part = self._new()
        Krr_f, _ = K1(rf[1:-1][:, None], tc[None, :])
        a = Krr_f * (rf[1:-1] ** 2)[:, None] * dcos[None, :] / (rc[1:] - rc[:-1])[:, None]
        lo, up = ix[:-1], ix[1:]
        self._add(part, lo, up, a / vol[:-1]); self._add(part, lo, lo, -a / vol[:-1])
        self._add(part, up, lo, a / vol[1:]); self._add(part, up, up, -a / vol[1:])
        R = rf[-1]
        Krr_R, _ = K1(np.full(self.n_th, R), tc)
        aR = Krr_R * R * R * dcos / (R - rc[-1])
        self._add(part, ix[-1], ix[-1], -aR / vol[-1])
        np.add.at(part[3], ix[-1], aR / vol[-1])
        _, Ktt_f = K1(rc[:, None], tf[1:-1][None, :])
        ring = ((rf[1:] ** 2 - rf[:-1] ** 2) / 2.0)[:, None]
        a = Ktt_f * np.sin(tf[1:-1])[None, :] * ring / (rc[:, None] * (tc[1:] - tc[:-1])[None, :])
        lo, up = ix[:, :-1], ix[:, 1:]
        self._add(part, lo, up, a / vol[:, :-1]); self._add(part, lo, lo, -a / vol[:, :-1])
        self._add(part, up, lo, a / vol[:, 1:]); self._add(part, up, up, -a / vol[:, 1:])
        return self._done(part)

    def advection(self, ur, ut):
        """-u_r d_r f - (u_th / r) d_th f for cell-centred velocities, central differences with
        mirror ghosts at r_in and the poles and the Dirichlet ghost 2 f_LIS - f at R_out."""
        ix = self.ix
        part = self._new()
        c = -ur / self.dr2[:, None]
        self._add(part, ix[:-1], ix[1:], c[:-1]); self._add(part, ix[1:], ix[:-1], -c[1:])
        self._add(part, ix[0], ix[0], -c[0])
        self._add(part, ix[-1], ix[-1], -c[-1])
        np.add.at(part[3], ix[-1], 2.0 * c[-1])
        ct = -(ut / self.RC) / self.dt2[None, :]
        self._add(part, ix[:, :-1], ix[:, 1:], ct[:, :-1]); self._add(part, ix[:, 1:], ix[:, :-1], -ct[:, 1:])
        self._add(part, ix[:, 0], ix[:, 0], -ct[:, 0])
        self._add(part, ix[:, -1], ix[:, -1], ct[:, -1])
        return self._done(part)


def solve(species, p, r0, th0, P0_list, n_r=80, n_th=90, dlnP=0.01, P_top=300.0, th_stretch=0.0):
    """Modulated J(T0) at (r0, th0) for each rigidity in P0_list (GV).

    p is a parameter dict with the keys of the model record (K0, kperp_r_frac,
    kperp_th_frac, B1AU_nT, V_slow_kms, V_fast_kms, lat_fast_deg, dlat_deg,
    polarity, drift_on, hcs_on, tilt_deg, dcs_min_deg, R_out, R_ts, ts_K_factor,
    dts_AU, r_in, rot_period_day); the model must be anisotropic and
    axisymmetric: no current sheet, or a flat one (tilt 0), no shells or
    squashed boundaries."""
    if p.get("isotropic", 0.0) or p.get("n_shells", 0.0) or p.get("squashed", 0.0):
        raise ValueError("the 2-D solver covers the anisotropic axisymmetric model")
    if p.get("hcs_on", 0.0) and p.get("tilt_deg", 0.0) != 0.0:
        raise ValueError("a tilted current sheet is not axisymmetric")
    m = _Model(p, species)
    rf, rc, tf, tc = _grid(p, n_r, n_th, th_stretch)
    if not (rc[0] < r0 < rc[-1] and tc[0] < th0 < tc[-1]):
        raise ValueError("the observer must lie between cell centres")
    asm = _Assembler(rf, rc, tf, tc)
    RC, TC = asm.RC, asm.TC
    M = sp.diags((3.0 * RC / (2.0 * m.V(TC))).ravel(), format="csc")
    SK, bK = asm.diffusion(m.K1)
    SV, bV = asm.advection(m.V(TC), 0.0 * TC)
    MSK, MSV, MbK, MbV = M @ SK, M @ SV, M @ bK, M @ bV
    sheet = bool(p.get("hcs_on", 0.0)) and bool(p["drift_on"])

    def drift(P):
        vr1, vt1 = m.drift1(RC, TC, P)
        SD, bD = asm.advection(vr1, vt1)
        return M @ SD, M @ bD

    if not sheet:
        MSD, MbD = drift(1.0)          # without a sheet the drift per beta P is rigidity-free
    N = asm.N
    Id = sp.identity(N, format="csc")
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
        if sheet:
            MSD, MbD = drift(P)
        L = bP * (MSK + MSD) + MSV
        src = dlnP * f_lis(species, P) * (bP * (MbK + MbD) + MbV)
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
