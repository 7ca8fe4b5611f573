"""Pins of the oracle's SDE integration on the spherically symmetric model.

Isotropic K = K0 beta P with uniform radial wind is the spherically symmetric 1-D model of
Sec. IV.B.  Against it the oracle is pinned by results it does not compute
itself:
  * V = 0: the process is reflected Brownian motion (generator K Laplacian).
    Its mean exit time from the shell r_in < r < R solves K (u'' + 2u'/r) = -1,
    u(R) = 0, u'(r_in) = 0, and its exit points obey the harmonic measure of
    the shell: E[(rho^l + c_l rho^-(l+1)) P_l(cos gamma)] = r0^l + c_l r0^-(l+1)
    with c_l = l r_in^(2l+1) / (l+1) (Neumann at r_in).
  * V = 0 leaves the rigidity unchanged (Eq. 6: d lnP = 2V/(3r) ds).
  * With wind, the modulated spectrum of Eq. 4 equals the solution of the
    steady transport equation (Eq. 5) from an independent Crank-Nicolson
    solver, up to the Euler-Maruyama step bias, which shrinks with dt.
  * The force-field approximation holds loosely above ~1 GeV.
  * The Monte Carlo error falls as N^-1/2.
"""
import math

import numpy as np
import pytest
from scipy.special import eval_legendre

from oracle import pde1d
from paper_2502_06319_gb300 import workloads as W

SIEGMUND = 0.5826  # -zeta(1/2)/sqrt(2 pi): mean overshoot of a Gaussian walk, in step sd


def _bm_params(**kw):
    base = dict(isotropic=1.0, drift_on=0.0, hcs_on=0.0, V_const_kms=0.0, R_out=10.0,
                r_in=0.5, r0=2.0, dt_fixed=1e-4)
    base.update(kw)
    return W.params(**base)


@pytest.fixture(scope="module")
def bm_runs(orc):
    out = {}
    for name, th0, ph0 in (("equator", math.pi / 2, 0.0), ("near_pole", 0.15, 1.0)):
        p = _bm_params(th0=th0, ph0=ph0)
        res = orc.run(p, W.PROTON, [1.0], [6000], seed=11 if name == "equator" else 12)
        out[name] = (p, res)
    return out


def _K(orc, p):
    return orc.evaluate(p, W.PROTON, p["r0"], p["th0"], p["ph0"], math.log(float(orc.rigidity(W.PROTON, 1.0))))["Kpar"]


@pytest.mark.parametrize("name", ["equator", "near_pole"])
def test_mean_exit_time_closed_form(orc, bm_runs, name):
    p, res = bm_runs[name]
    assert np.all(res["status"] == orc.EXIT)
    K = _K(orc, p)
    R = p["R_out"] + SIEGMUND * math.sqrt(2.0 * K * p["dt_fixed"])
    r0, ri = p["r0"], p["r_in"]
    expect = (R * R - r0 * r0) / (6.0 * K) - ri ** 3 / (3.0 * K) * (1.0 / r0 - 1.0 / R)
    s = res["s"]
    sem = s.std(ddof=1) / math.sqrt(len(s))
    assert abs(s.mean() - expect) < 3.5 * sem, (s.mean(), expect, sem)


@pytest.mark.parametrize("name", ["equator", "near_pole"])
def test_exit_points_harmonic_measure(orc, bm_runs, name):
    p, res = bm_runs[name]
    th0, ph0, r0, ri = p["th0"], p["ph0"], p["r0"], p["r_in"]
    x0 = np.array([math.sin(th0) * math.cos(ph0), math.sin(th0) * math.sin(ph0), math.cos(th0)])
    x = np.stack([np.sin(res["th"]) * np.cos(res["ph"]), np.sin(res["th"]) * np.sin(res["ph"]),
                  np.cos(res["th"])], axis=1)
    cg = x @ x0
    rho = res["r"]
    for l in (1, 2, 3):
        c = l * ri ** (2 * l + 1) / (l + 1)
        val = (rho ** l + c * rho ** (-l - 1)) * eval_legendre(l, cg)
        expect = r0 ** l + c * r0 ** (-l - 1)
        sem = val.std(ddof=1) / math.sqrt(len(val))
        assert abs(val.mean() - expect) < 4.0 * sem, (l, val.mean(), expect, sem)


def test_no_wind_keeps_rigidity(orc, bm_runs):
    p, res = bm_runs["equator"]
    lnP0 = math.log(float(orc.rigidity(W.PROTON, 1.0)))
    assert np.all(res["lnP"] == lnP0)


@pytest.fixture(scope="module")
def pde_ref():
    T0 = np.array([0.3, 1.0])
    P0 = np.array([float(x) for x in (W.PROTON["A"] / W.PROTON["Z"] * np.sqrt(T0 * (T0 + 2 * W.PROTON["m0"])))])
    return T0, pde1d.solve(W.PROTON, 11.5, 400.0, 0.1, 100.0, 1.0, P0, n_r=800, dlnP=3e-3)


def test_pde_solver_grid_converged(pde_ref):
    T0, J = pde_ref
    P0 = W.PROTON["A"] / W.PROTON["Z"] * np.sqrt(T0 * (T0 + 2 * W.PROTON["m0"]))
    J2 = pde1d.solve(W.PROTON, 11.5, 400.0, 0.1, 100.0, 1.0, P0, n_r=1600, dlnP=1.5e-3)
    assert np.all(np.abs(J2 / J - 1) < 1e-3)


def test_spectrum_matches_pde(orc, pde_ref):
    T0, J_pde = pde_ref
    errs = {}
    for dt in (0.1, 0.01):
        p = W.params(isotropic=1.0, drift_on=0.0, hcs_on=0.0, dt_fixed=dt)
        res = orc.run(p, W.PROTON, T0, [5000, 5000], seed=7)
        J, S = orc.spectrum_unbinned(res, W.PROTON, T0)
        errs[dt] = (J - J_pde) / J_pde
        if dt == 0.01:
            # Euler-Maruyama bias at dt = 0.01 day is ~1 %; allow it plus 3 sigma
            assert np.all(np.abs(J - J_pde) < 3.0 * S + 0.015 * J_pde), (J, J_pde, S)
    # the step bias shrinks with dt (paired streams)
    assert abs(errs[0.01][1]) < abs(errs[0.1][1])


def test_force_field_loose(orc):
    job = W.config0()
    res = orc.job_run(job)
    J, S = orc.spectrum_unbinned(res, job.species, job.T_in)
    ff, phi = pde1d.force_field(job.species, 11.5, 400.0, 100.0, 1.0, job.T_in)
    assert abs(phi - 0.663) < 1e-3
    assert abs(J[0] / ff[0] - 1.0) < 0.20


def test_monte_carlo_error_falls_as_inverse_sqrt_n(orc):
    p = W.params(isotropic=1.0, drift_on=0.0, hcs_on=0.0, dt_fixed=0.1)
    Ns = [200, 800, 3200]
    sds = []
    for N in Ns:
        Js = []
        for seed in range(24):
            res = orc.run(p, W.PROTON, [1.0], [N], seed=1000 + seed)
            Js.append(orc.spectrum_unbinned(res, W.PROTON, [1.0])[0][0])
        sds.append(np.std(Js, ddof=1))
    slope = np.polyfit(np.log(Ns), np.log(sds), 1)[0]
    assert abs(slope + 0.5) < 0.15, (slope, sds)


def test_spectrum_identity_without_modulation(orc):
    # V = 0: every path exits with P = P0, so Eq. 4 returns the LIS itself.
    p = _bm_params(R_out=3.0, r0=1.0, r_in=0.1, dt_fixed=1e-3)
    T0 = np.array([0.5, 2.0, 20.0])
    res = orc.run(p, W.PROTON, T0, [50, 50, 50], seed=2)
    J, S = orc.spectrum_unbinned(res, W.PROTON, T0)
    assert np.allclose(J, orc.lis(T0), rtol=1e-12, atol=0)
    assert np.all(S < 1e-12 * J)


def test_histogram_and_binned_estimator_by_brute_force(orc):
    rng = np.random.default_rng(0)
    n = 300
    run = {"lnP": rng.uniform(math.log(0.05), math.log(2000.0), n),
           "status": rng.choice([1, 1, 1, 1, 2, 3], n).astype(np.uint8),
           "energy": rng.integers(0, 3, n)}
    nb, Pmin, Pmax = 16, 0.1, 1000.0
    H = orc.histogram(run, 3, Pmin, Pmax, nb)
    # scalar loop
    H2 = np.zeros_like(H)
    edges = [10 ** (math.log10(Pmin) + i * (math.log10(Pmax) - math.log10(Pmin)) / nb) for i in range(nb + 1)]
    for lnP, st, e in zip(run["lnP"], run["status"], run["energy"]):
        if st != 1:
            H2[e, nb + 2] += 1
            continue
        P = math.exp(lnP)
        if P < edges[0]:
            H2[e, 0] += 1
        elif P >= edges[-1]:
            H2[e, nb + 1] += 1
        else:
            b = max(i for i in range(nb) if edges[i] <= P * (1 + 1e-15))
            H2[e, 1 + b] += 1
    assert np.array_equal(H, H2)
    assert H.sum() == n
    T0 = [0.5, 1.0, 3.0]
    J, S = orc.spectrum_from_hist(H, W.PROTON, T0, Pmin, Pmax, nb)
    for e in range(3):
        vals = []
        for b in range(nb):
            Pc = math.sqrt(edges[b] * edges[b + 1])
            pn = Pc
            Tc = math.sqrt(pn * pn + W.PROTON["m0"] ** 2) - W.PROTON["m0"]
            vals += [orc.lis(Tc) / Pc ** 2] * int(H[e, 1 + b])
        P0 = math.sqrt(T0[e] * (T0[e] + 2 * W.PROTON["m0"]))
        pref = P0 ** 2
        assert math.isclose(J[e], pref * np.mean(vals), rel_tol=1e-9)
        assert math.isclose(S[e], pref * np.std(vals, ddof=1) / math.sqrt(len(vals)), rel_tol=1e-9)
