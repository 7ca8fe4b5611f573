"""Pins of the oracle's heliospheric coefficients (Eq. 3's A and B).

Every check recomputes the quantity by a route the oracle does not take:
  * the diffusion tensor against its definition K = K_par b b^T + K_perp,r n n^T
    + K_perp,th e_th e_th^T (eigen-decomposition) and 2K = L L^T;
  * the Ito drift of the spherical coordinates, A^q = (div K) . grad q + K : Hess q,
    from Cartesian finite differences of the Cartesian tensor (Ito's lemma) --
    independent of the spherical divergence formula the oracle uses;
  * the drift velocity against a Cartesian finite-difference curl of
    kappa_A h e_B, against the closed-form gradient-curvature drift of the
    Parker field, and against its divergence (zero);
  * the magnetic field against div B = 0 and |B|(1 AU, equator) = B1AU;
  * the drift direction against the physics of the two polarity epochs.
"""
import math

import numpy as np
import pytest

from paper_2502_06319_gb300 import workloads as W

AU_M, DAY_S = 1.495978707e11, 86400.0


def _basis(th, ph):
    er = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    et = np.array([math.cos(th) * math.cos(ph), math.cos(th) * math.sin(ph), -math.sin(th)])
    ep = np.array([-math.sin(ph), math.cos(ph), 0.0])
    return np.stack([er, et, ep], axis=1)  # columns


def _sph(x):
    r = float(np.linalg.norm(x))
    th = math.acos(x[2] / r)
    ph = math.atan2(x[1], x[0]) % (2 * math.pi)
    return r, th, ph


def _cart(r, th, ph):
    return r * _basis(th, ph)[:, 0]


def _ev(orc, p, sp, x, lnP):
    r, th, ph = _sph(x)
    return orc.evaluate(p, sp, r, th, ph, lnP)


def _Kphys(e):
    return np.array([[e["Krr"], e["Krt"], e["Krp"]],
                     [e["Krt"], e["Ktt"], e["Ktp"]],
                     [e["Krp"], e["Ktp"], e["Kpp"]]])


def _Kcart(orc, p, sp, x, lnP):
    r, th, ph = _sph(x)
    Q = _basis(th, ph)
    return Q @ _Kphys(orc.evaluate(p, sp, r, th, ph, lnP)) @ Q.T


POINTS = [(1.0, 1.2, 0.3), (3.0, 0.7, 2.0), (12.0, 1.9, 4.0), (47.0, 0.35, 5.5),
          (90.0, 2.6, 1.1), (84.0, 1.45, 0.2)]
SPECIES = [W.PROTON, W.HELIUM4, W.ELECTRON]


def _models():
    return {
        "full": W.params(),
        "ts": W.params(R_ts=85.0, R_out=122.0, tilt_deg=60.0),
        "unipolar": W.params(hcs_on=0.0),
        "aniso_th": W.params(kperp_r_frac=0.05, kperp_th_frac=0.01, polarity=-1.0),
    }


@pytest.mark.parametrize("model", list(_models()))
def test_tensor_is_rotated_diagonal_and_cholesky(orc, model):
    p = _models()[model]
    for (r, th, ph) in POINTS:
        for sp in SPECIES:
            lnP = math.log(3.0)
            e = orc.evaluate(p, sp, r, th, ph, lnP)
            K = _Kphys(e)
            assert np.allclose(K, K.T)
            w = np.sort(np.linalg.eigvalsh(K))
            Kpar = e["Kpar"]
            expect = np.sort([Kpar, p["kperp_r_frac"] * Kpar, p["kperp_th_frac"] * Kpar])
            assert np.allclose(w, expect, rtol=1e-12), (w, expect)
            assert np.all(w > 0)
            # b is along the Parker spiral: eigenvector of K_par is (1, 0, -Gamma)/sqrt(1+Gamma^2)
            G = e["Gam"]
            b = np.array([1.0, 0.0, -G]) / math.sqrt(1 + G * G)
            assert np.allclose(K @ b, Kpar * b, rtol=1e-12, atol=1e-12 * Kpar)
            L = np.array([[e["L00"], 0, 0], [e["L10"], e["L11"], 0], [e["L20"], e["L21"], e["L22"]]])
            assert np.allclose(L @ L.T, 2 * K, rtol=1e-13, atol=1e-14 * Kpar)


@pytest.mark.parametrize("model", ["full", "ts", "aniso_th"])
def test_ito_drift_from_cartesian_divergence(orc, model):
    check_ito_drift(orc, _models()[model], W.PROTON, math.log(2.0), POINTS)


def check_ito_drift(orc, p, sp, lnP, points, hrel=3e-5):
    """Coordinate Ito drift and noise covariance against Cartesian finite differences
    (step hrel * r; truncation error falls as its square)."""
    for (r, th, ph) in points:
        x = _cart(r, th, ph)
        hstep = hrel * r
        # div K (Cartesian): d_i K_ij
        divK = np.zeros(3)
        for i in range(3):
            d = np.zeros(3); d[i] = hstep
            dK = (_Kcart(orc, p, sp, x + d, lnP) - _Kcart(orc, p, sp, x - d, lnP)) / (2 * hstep)
            divK += dK[i, :]
        Kc = _Kcart(orc, p, sp, x, lnP)

        def grads(y):
            rr, tt, pp = _sph(y)
            Q = _basis(tt, pp)
            return np.stack([Q[:, 0], Q[:, 1] / rr, Q[:, 2] / (rr * math.sin(tt))])  # rows: grad r, th, ph

        g0 = grads(x)
        hess = np.zeros((3, 3, 3))
        for i in range(3):
            d = np.zeros(3); d[i] = hstep
            hess[:, i, :] = (grads(x + d) - grads(x - d)) / (2 * hstep)
        A_expect = g0 @ divK + np.einsum("qij,ij->q", hess, Kc)
        e = orc.evaluate(p, sp, r, th, ph, lnP)
        A = np.array([e["Ar"], e["Ath"], e["Aph"]])
        # the two Ito terms cancel strongly in the azimuthal component: scale by their size
        scale = np.abs(g0) @ np.abs(divK) + np.einsum("qij,ij->q", np.abs(hess), np.abs(Kc))
        assert np.all(np.abs(A - A_expect) < 1e-5 * scale), (r, th, ph, A, A_expect)
        # noise covariance of the coordinates: (L L^T)_ab / (h_a h_b) = grad q_a . 2K . grad q_b
        L = np.array([[e["L00"], 0, 0], [e["L10"], e["L11"], 0], [e["L20"], e["L21"], e["L22"]]])
        hsc = np.array([1.0, r, r * math.sin(th)])
        cov = (L @ L.T) / np.outer(hsc, hsc)
        assert np.allclose(cov, g0 @ (2 * Kc) @ g0.T, rtol=1e-10, atol=1e-14)


def _W_cart(orc, p, sp, x, lnP):
    r, th, ph = _sph(x)
    e = orc.evaluate(p, sp, r, th, ph, lnP)
    return _basis(th, ph) @ np.array([e["Wr"], 0.0, e["Wph"]])


def _curl(f, x, hstep):
    J = np.zeros((3, 3))
    for i in range(3):
        d = np.zeros(3); d[i] = hstep
        J[:, i] = (f(x + d) - f(x - d)) / (2 * hstep)   # J[j, i] = d_i f_j
    return np.array([J[2, 1] - J[1, 2], J[0, 2] - J[2, 0], J[1, 0] - J[0, 1]])


def _div(f, x, hstep):
    s = 0.0
    for i in range(3):
        d = np.zeros(3); d[i] = hstep
        s += (f(x + d)[i] - f(x - d)[i]) / (2 * hstep)
    return s


@pytest.mark.parametrize("model", ["full", "ts", "unipolar", "aniso_th"])
@pytest.mark.parametrize("sp", SPECIES, ids=["p", "he4", "e"])
def test_drift_is_curl_and_divergence_free(orc, model, sp):
    check_drift_curl(orc, _models()[model], sp, POINTS, model)


def check_drift_curl(orc, p, sp, points, model="", hrel=2e-6):
    """Drift = sgn(qA) curl(kappa_A h e_B) by finite differences (step hrel * r), and
    divergence-free."""
    for lnP in (math.log(0.5), math.log(20.0)):
        for (r, th, ph) in points:
            x = _cart(r, th, ph)
            hstep = hrel * r
            e = orc.evaluate(p, sp, r, th, ph, lnP)
            Q = _basis(th, ph)
            vd = Q @ np.array([e["vdr"], e["vdth"], e["vdph"]])
            s = math.copysign(1, sp["Z"]) * p["polarity"]
            curl = s * _curl(lambda y: _W_cart(orc, p, sp, y, lnP), x, hstep)
            tol = 1e-5 * (np.linalg.norm(curl) + abs(e["Wr"]) / r + abs(e["Wph"]) / r)
            assert np.linalg.norm(vd - curl) < tol, (model, r, th, ph, vd, curl)

            def vd_cart(y):
                ee = _ev(orc, p, sp, y, lnP)
                rr, tt, pp = _sph(y)
                return _basis(tt, pp) @ np.array([ee["vdr"], ee["vdth"], ee["vdph"]])

            # the sheet is thin: a small step keeps the O(h^2) truncation negligible
            div = _div(vd_cart, x, min(1e-6, hrel) * r)
            assert abs(div) < 1e-4 * np.linalg.norm(vd) / r + 1e-12, (div, np.linalg.norm(vd))


def test_gradient_curvature_drift_closed_form(orc):
    # Uniform wind, unipolar field: v_d = (2 C_A r / (1+G^2)^2) (-G cot th, (2+G^2) G, G^2 cot th)
    # with C_A = beta P / (3 B0) [Jokipii, Levy & Hubbard 1977; Burger & Potgieter 1989].
    p = W.params(hcs_on=0.0, V_fast_kms=400.0)
    for sp in SPECIES:
        for (r, th, ph) in POINTS:
            lnP = math.log(4.0)
            e = orc.evaluate(p, sp, r, th, ph, lnP)
            Vs = 400.0 * DAY_S / 1.495978707e8
            Om = 2 * math.pi / 25.38
            B0 = 5.0 / math.sqrt(1 + (Om / Vs) ** 2)
            CA = e["beta"] * e["P"] * 1e9 / (3 * B0 * 1e-9) / (AU_M ** 2 / DAY_S)
            G = Om * r * math.sin(th) / Vs
            cot = 1 / math.tan(th)
            pre = 2 * CA * r / (1 + G * G) ** 2 * math.copysign(1, sp["Z"]) * p["polarity"]
            expect = pre * np.array([-G * cot, (2 + G * G) * G, G * G * cot])
            got = np.array([e["vdr"], e["vdth"], e["vdph"]])
            assert np.allclose(got, expect, rtol=1e-11, atol=1e-13 * np.abs(expect).max())


def test_field_divergence_free_and_normalised(orc):
    p = W.params()
    e = orc.evaluate(p, W.PROTON, 1.0, math.pi / 2, 0.0, 0.0)
    assert math.isclose(e["Bmag"], 5.0, rel_tol=1e-14)
    Vs = 400.0 * DAY_S / 1.495978707e8
    assert math.isclose(e["Gam"], 2 * math.pi / 25.38 / Vs, rel_tol=1e-12)  # tanh tail at the equator ~1e-13
    # unipolar field, and the sheet field at rigidities where its width is the fixed floor
    for model, lnP in ((W.params(hcs_on=0.0), 0.0), (W.params(), math.log(0.05))):
        def Bc(y):
            ee = _ev(orc, model, W.PROTON, y, lnP)
            rr, tt, pp = _sph(y)
            return _basis(tt, pp) @ np.array([ee["Br"], 0.0, ee["Bph"]])
        for (r, th, ph) in POINTS[:4]:
            x = _cart(r, th, ph)
            ee = orc.evaluate(model, W.PROTON, r, th, ph, lnP)
            if model["hcs_on"]:
                assert ee["delta_cs"] == pytest.approx(math.radians(1.0))
            div = _div(Bc, x, 1e-5 * r)
            assert abs(div) < 1e-6 * np.linalg.norm(Bc(x)) / r, (r, th, ph, div)


def test_wind_profile_and_momentum_term(orc):
    p = W.params()
    Vs = 400.0 * DAY_S / 1.495978707e8
    Vf = 760.0 * DAY_S / 1.495978707e8
    for th, expect in ((math.pi / 2, Vs), (0.05, Vf), (math.pi - 0.05, Vf),
                       (math.pi / 2 - math.radians(30), 0.5 * (Vs + Vf)),
                       (math.pi / 2 + math.radians(30), 0.5 * (Vs + Vf))):
        e = orc.evaluate(p, W.PROTON, 5.0, th, 0.0, 0.0)
        assert math.isclose(e["V"], expect, rel_tol=1e-9)
        assert math.isclose(e["dlnP"], 2 * e["V"] / (3 * 5.0), rel_tol=1e-15)


def test_termination_shock_factor(orc):
    p = W.params(R_ts=85.0, R_out=122.0)
    assert orc.evaluate(p, W.PROTON, 40.0, 1.0, 0.0, 0.0)["g"] == pytest.approx(1.0, abs=1e-15)
    assert orc.evaluate(p, W.PROTON, 85.0, 1.0, 0.0, 0.0)["g"] == pytest.approx(0.75, abs=1e-15)
    assert orc.evaluate(p, W.PROTON, 110.0, 1.0, 0.0, 0.0)["g"] == pytest.approx(0.5, abs=1e-15)


@pytest.mark.parametrize("polarity", [1.0, -1.0])
@pytest.mark.parametrize("sp", [W.PROTON, W.ELECTRON], ids=["p", "e"])
def test_drift_direction_physics(orc, polarity, sp):
    """qA > 0: drift inward and toward the equator at high latitudes, outward along
    the current sheet; qA < 0: the reverse."""
    p = W.params(polarity=polarity, tilt_deg=5.0)
    qa = polarity * math.copysign(1, sp["Z"])
    lnP = math.log(1.0)
    north = orc.evaluate(p, sp, 10.0, 0.4, 0.0, lnP)
    south = orc.evaluate(p, sp, 10.0, math.pi - 0.4, 0.0, lnP)
    assert qa * north["vdr"] < 0 and qa * north["vdth"] > 0
    assert qa * south["vdr"] < 0 and qa * south["vdth"] < 0
    # on the sheet (flat part: phase where sin(phi*) = 0)
    e0 = orc.evaluate(p, sp, 10.0, math.pi / 2, 0.0, lnP)
    Om = 2 * math.pi / 25.38
    ph = (-Om * 10.0 / e0["V"]) % (2 * math.pi)
    sheet = orc.evaluate(p, sp, 10.0, math.pi / 2, ph, lnP)
    assert abs(sheet["h"]) < 1e-6
    assert qa * sheet["vdr"] > 0


def test_full_model_reduces_to_isotropic_pathwise(orc):
    """With K_perp = K_par, one wind speed and no drift, the general (spiral-rotated)
    branch must integrate the same paths as the isotropic branch."""
    common = dict(drift_on=0.0, hcs_on=0.0, dt_fixed=0.02, R_out=20.0)
    iso = W.params(isotropic=1.0, V_const_kms=400.0, **common)
    full = W.params(kperp_r_frac=1.0, kperp_th_frac=1.0, V_fast_kms=400.0, V_slow_kms=400.0, **common)
    a = orc.run(iso, W.PROTON, [1.0, 5.0], [100, 100], seed=3)
    b = orc.run(full, W.PROTON, [1.0, 5.0], [100, 100], seed=3)
    same = a["steps"] == b["steps"]
    assert same.mean() >= 0.97
    for k in ("r", "th", "lnP", "s"):
        rel = np.abs(a[k][same] - b[k][same]) / np.maximum(np.abs(a[k][same]), 1e-300)
        assert np.median(rel) < 1e-9, k


def test_drift_sign_is_the_product_of_charge_and_polarity_signs(orc):
    """v_d carries sgn(q) sgn(A): a proton in the A < 0 epoch and a particle of the proton's
    mass and opposite charge in the A > 0 epoch follow the same paths, bit for bit; swapping
    only one of the two signs changes them."""
    anti = {"A": 1, "Z": -1, "m0": W.PROTON["m0"]}
    T, N = [0.3, 3.0], [20, 20]
    a = orc.run(W.params(polarity=-1.0), W.PROTON, T, N, seed=12)
    b = orc.run(W.params(polarity=1.0), anti, T, N, seed=12)
    for k in ("r", "th", "ph", "lnP", "s", "steps", "status"):
        assert np.array_equal(a[k], b[k]), k
    c = orc.run(W.params(polarity=1.0), W.PROTON, T, N, seed=12)
    assert not np.array_equal(a["steps"], c["steps"])


def test_units_against_hand_worked_values(orc):
    """Hand-worked numbers (to the digits quoted): a 1 GeV proton has P = 1.696038 GV and
    beta = 0.875026; 400 and 760 km/s are 0.231019 and 0.438937 AU/day; the spiral at 1 AU on
    the equator has Gamma = (2 pi / 25.38 d) / 0.231019 AU/d = 1.0716; kappa_A = beta P / (3 |B|)
    for beta P = 1 GV and |B| = 5 nT is 6.667e16 m^2/s = 0.25738 AU^2/day."""
    P = float(orc.rigidity(W.PROTON, 1.0))
    assert abs(P - 1.696038) < 5e-7 and abs(float(orc.beta(W.PROTON, P)) - 0.875026) < 5e-7
    p = W.params(hcs_on=0.0)
    e = orc.evaluate(p, W.PROTON, 1.0, math.pi / 2, 0.0, math.log(P))
    assert abs(e["V"] - 0.231019) < 5e-7
    assert abs(orc.evaluate(p, W.PROTON, 1.0, 0.01, 0.0, 0.0)["V"] - 0.438937) < 5e-7
    assert abs(e["Gam"] - 1.0716) < 5e-5
    assert abs(e["Bmag"] - 5.0) < 1e-12
    # |kappa_A h e_B| with h = 1 at 1 AU on the equator, per GV of beta P
    kA = math.hypot(e["Wr"], e["Wph"]) / (e["beta"] * e["P"])
    assert abs(kA - 0.25738) < 5e-5
