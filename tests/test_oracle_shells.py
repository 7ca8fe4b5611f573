"""Pins of the radial shells of the inner heliosphere (Sec. II.B): the region
inside the termination shock split into shells, each with its own K0 and
current-sheet tilt, blended across the edges (C^1 cubic smoothstep).

  * constant tables reproduce the single-region model bit for bit (paths);
  * inside a shell, away from the edges, every coefficient equals that of the
    single-region model with that shell's K0 and tilt, bit for bit;
  * at the edges: the shells' own values at R_e -+ w, their mean at R_e, and
    the analytic radial derivative against central differences;
  * inside the blend windows, the Ito drift against Cartesian finite
    differences and the drift against the finite-difference curl (with points
    placed inside the current sheet, where the tilt's radial change matters);
  * the spherically symmetric model with shells of different K0 against the
    independent 1-D PDE solver in conservative form (K at cell faces only).
"""
import math

import numpy as np
import pytest

from oracle import pde1d
from paper_2502_06319_gb300 import workloads as W
from tests.test_oracle_model import SPECIES, check_drift_curl, check_ito_drift

K0S = [22.0, 9.0, 14.0, 30.0, 6.0, 12.0, 18.0, 25.0, 7.5, 11.0, 16.0, 28.0, 10.0, 19.0, 13.0]
TILTS = [10.0, 35.0, 60.0, 20.0, 72.0, 45.0, 15.0, 55.0, 30.0, 65.0, 8.0, 40.0, 50.0, 25.0, 70.0]


def _shell_model(**kw):
    base = dict(R_ts=85.0, R_out=122.0, n_shells=15, shell_K0=K0S, shell_tilt_deg=TILTS, shell_blend_AU=0.5)
    base.update(kw)
    return W.params(**base)


DR = 85.0 / 15


def test_constant_tables_reproduce_single_region_paths(orc):
    p0 = W.params(R_ts=85.0, R_out=122.0, tilt_deg=30.0, K0=14.0)
    p1 = _shell_model(shell_K0=[14.0] * 15, shell_tilt_deg=[30.0] * 15)
    T, N = [0.3, 3.0, 30.0], [25, 25, 25]
    a = orc.run(p0, W.PROTON, T, N, seed=3)
    b = orc.run(p1, W.PROTON, T, N, seed=3)
    for k in ("r", "th", "ph", "lnP", "s", "steps", "status"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("k", [0, 1, 4, 9, 14])
def test_inside_a_shell_equals_single_region_model(orc, k):
    p = _shell_model()
    q = W.params(R_ts=85.0, R_out=122.0, K0=K0S[k], tilt_deg=TILTS[k])
    r = (k + 0.5) * DR if k < 14 else 100.0      # the outermost shell continues past the shock
    for sp in SPECIES:
        for th, ph in ((1.3, 0.4), (1.62, 2.5), (0.5, 5.0)):
            a = orc.evaluate(p, sp, r, th, ph, math.log(2.5))
            b = orc.evaluate(q, sp, r, th, ph, math.log(2.5))
            for name in a:
                assert a[name] == b[name] or (math.isnan(a[name]) and math.isnan(b[name])), (k, name)


def _iso_shells(**kw):
    return _shell_model(isotropic=1.0, drift_on=0.0, hcs_on=0.0, R_ts=0.0, R_out=85.0, **kw)


def test_blend_values_at_the_edges(orc):
    p = _iso_shells()
    lnP = math.log(3.0)
    e0 = orc.evaluate(p, W.PROTON, 1.0, 1.0, 0.0, lnP)
    bP = e0["beta"] * e0["P"]
    K0_at = lambda r: orc.evaluate(p, W.PROTON, r, 1.0, 0.0, lnP)["Kpar"] / bP
    w = 0.5
    for e in range(1, 15):
        Re = e * DR
        assert math.isclose(K0_at(Re - w), K0S[e - 1], rel_tol=1e-14)
        assert math.isclose(K0_at(Re + w), K0S[e], rel_tol=1e-14)
        assert math.isclose(K0_at(Re), 0.5 * (K0S[e - 1] + K0S[e]), rel_tol=1e-14)
        # monotone between the two shells' values across the window
        vals = [K0_at(Re + x) for x in np.linspace(-w, w, 21)]
        assert np.all(np.diff(vals) * np.sign(K0S[e] - K0S[e - 1]) >= -1e-12)


def test_radial_derivative_against_central_differences(orc):
    p = _iso_shells()
    lnP = math.log(3.0)
    Krr = lambda r: orc.evaluate(p, W.PROTON, r, 1.0, 0.0, lnP)["Krr"]
    for e in (1, 3, 7, 14):
        Re = e * DR
        for x in (-0.49, -0.3, -0.05, 0.0, 0.17, 0.42, 0.49, 0.8, -0.9):
            r = Re + x
            h = 1e-5
            fd = (Krr(r + h) - Krr(r - h)) / (2 * h)
            an = orc.evaluate(p, W.PROTON, r, 1.0, 0.0, lnP)["dKrr_dr"]
            scale = abs(K0S[e] - K0S[e - 1]) * 3.0 / (2 * 0.5) * Krr(r) / K0S[e]
            assert abs(an - fd) < 1e-6 * scale, (e, x, an, fd)
            if abs(x) > 0.5:
                assert an == 0.0          # outside the window the shell is uniform


def _sheet_points(orc, p, radii, phis, h_target=0.3):
    """Points inside the current sheet (h = h_target) in blend windows: there the sheet
    tilt's radial change enters the drift."""
    pts = []
    for r, ph in zip(radii, phis):
        f = lambda th: orc.evaluate(p, W.PROTON, r, th, ph, math.log(2.0))["h"] - h_target
        grid = np.linspace(0.15, math.pi - 0.15, 400)
        vals = [f(t) for t in grid]
        i = next(i for i in range(len(grid) - 1) if vals[i] * vals[i + 1] < 0)
        lo, hi = grid[i], grid[i + 1]
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if f(lo) * f(mid) <= 0:
                hi = mid
            else:
                lo = mid
        pts.append((r, 0.5 * (lo + hi), ph))
    return pts


WINDOW_RADII = [DR - 0.2, 2 * DR + 0.3, 8 * DR - 0.1, 14 * DR + 0.25]
WINDOW_PHIS = [0.9, 2.2, 4.1, 5.6]


def test_ito_drift_in_blend_windows(orc):
    p = _shell_model()
    pts = [(r, th, ph) for r in WINDOW_RADII for th, ph in ((1.1, 0.3), (2.0, 3.3))]
    for sp in SPECIES:
        # the blend windows are 1 AU wide: a step well below that keeps the truncation small
        check_ito_drift(orc, p, sp, math.log(2.0), pts, hrel=3e-6)


@pytest.mark.parametrize("sp", SPECIES, ids=["p", "he4", "e"])
def test_drift_curl_in_blend_windows_inside_the_sheet(orc, sp):
    p = _shell_model()
    # edges between moderate tilts (10-35, 35-60, 55-30, 8-40 deg): at steeper sheets the
    # radial turnover of h is too sharp for a finite-difference divergence
    pts = _sheet_points(orc, p, [DR - 0.2, 2 * DR + 0.3, 8 * DR - 0.1, 11 * DR + 0.2], WINDOW_PHIS)
    # the tilt term is a visible part of dh/dr at these points
    for (r, th, ph) in pts:
        e = orc.evaluate(p, sp, r, th, ph, math.log(2.0))
        assert abs(e["dh_dr"]) > 1e-3
    # inside the sheet h turns over within ~0.01 AU radially: a fine step for the curl
    check_drift_curl(orc, p, sp, pts, "shells", hrel=1e-7)


def _K0_profile(r, K0s, n, R_edge, w):
    """The blended shell profile, written out independently for the PDE's face values."""
    dR = R_edge / n
    out = np.empty_like(r)
    for i, x in enumerate(r):
        v = K0s[min(max(int(x // dR), 0), n - 1)]
        for e in range(1, n):
            Re = e * dR
            if Re - w <= x <= Re + w:
                t = (x - (Re - w)) / (2 * w)
                v = K0s[e - 1] + (K0s[e] - K0s[e - 1]) * t * t * (3 - 2 * t)
        out[i] = v
    return out


def test_spectrum_with_radial_shells_matches_pde(orc):
    # spherically symmetric: isotropic K = K0(r) beta P with five shells out to 100 AU
    K0s = [30.0, 8.0, 20.0, 6.0, 15.0]
    p = W.params(isotropic=1.0, drift_on=0.0, hcs_on=0.0, dt_fixed=0.01, n_shells=5, shell_K0=K0s,
                 shell_tilt_deg=[0.0] * 5, shell_blend_AU=2.0)
    T0 = np.array([0.3, 1.0])
    P0 = np.sqrt(T0 * (T0 + 2 * W.PROTON["m0"]))
    prof = lambda r: _K0_profile(r, K0s, 5, 100.0, 2.0)
    J_pde = pde1d.solve(W.PROTON, prof, 400.0, 0.1, 100.0, 1.0, P0, n_r=1000, dlnP=3e-3)
    J_one = pde1d.solve(W.PROTON, 30.0, 400.0, 0.1, 100.0, 1.0, P0, n_r=800, dlnP=3e-3)
    assert np.all(np.abs(J_pde / J_one - 1) > 0.05)   # the shells change the answer
    res = orc.run(p, W.PROTON, T0, [6000, 6000], seed=31)
    J, S = orc.spectrum_unbinned(res, W.PROTON, T0)
    assert np.all(np.abs(J - J_pde) < 3.0 * S + 0.015 * J_pde), (J, J_pde, S)


def test_solar_cycle_series_and_shell_tables():
    ser = W.solar_cycle_series(seed=20250212, n_rot=200)
    assert len(ser["K0"]) == 200 and len(ser["tilt_deg"]) == 200
    assert np.all((np.array(ser["K0"]) >= 5.0) & (np.array(ser["K0"]) <= 30.0))
    assert np.all((np.array(ser["tilt_deg"]) >= 5.0) & (np.array(ser["tilt_deg"]) <= 75.0))
    p = W.shell_params(ser, rotation=60, n_shells=15)
    # shell k carries the conditions of k rotations before the observation
    assert p["n_shells"] == 15.0
    assert list(p["shell_K0"]) == [ser["K0"][60 - k] for k in range(15)]
    assert list(p["shell_tilt_deg"]) == [ser["tilt_deg"][60 - k] for k in range(15)]


def test_pde_flux_form_grid_converged_with_shells():
    # the conservative discretisation with a radially varying K converges under refinement
    K0s = [30.0, 8.0, 20.0, 6.0, 15.0]
    prof = lambda r: _K0_profile(r, K0s, 5, 100.0, 2.0)
    T0 = np.array([0.3, 1.0])
    P0 = np.sqrt(T0 * (T0 + 2 * W.PROTON["m0"]))
    a = pde1d.solve(W.PROTON, prof, 400.0, 0.1, 100.0, 1.0, P0, n_r=800, dlnP=3e-3)
    b = pde1d.solve(W.PROTON, prof, 400.0, 0.1, 100.0, 1.0, P0, n_r=1600, dlnP=1.5e-3)
    assert np.all(np.abs(b / a - 1) < 2e-3), (a, b)
