"""Pins of the moving detection point (Sec. IV.A): the quasi-particle sample of
every energy is divided among the positions of the detector's orbit.

  * the split itself, on hand-worked cases;
  * the spherically symmetric model: the radial process and the rigidity do
    not depend on the start angles at all (bit for bit), and the
    orbit-averaged spectrum equals the weighted mean of the steady transport
    equation's solutions at the orbit's radii (independent Crank-Nicolson
    solver), up to the Euler-Maruyama step bias;
  * the synthetic polar orbit the orbit bench uses samples equal times
    (Kepler's equation recovered from the radii).
"""
import math

import numpy as np

from oracle import pde1d
from paper_2502_06319_gb300 import workloads as W


def test_split_hand_worked(orc):
    # n = 7, weights 1 : 2 : 4 -> cuts floor(0), floor(7 * 1/7), floor(7 * 3/7) -> counts 1, 2, 4
    pos = [(1.0, 1.0, 0.0, 1.0), (2.0, 1.0, 0.0, 2.0), (3.0, 1.0, 0.0, 4.0)]
    st = orc.orbit_starts([7], pos)
    assert st[:, 0].tolist() == [1.0, 2.0, 2.0, 3.0, 3.0, 3.0, 3.0]
    # n = 10, weights 1 : 1 : 1 -> cuts 0, floor(10/3) = 3, floor(20/3) = 6 -> counts 3, 3, 4
    pos = [(1.0, 1.0, 0.0, 1.0), (2.0, 1.0, 0.0, 1.0), (3.0, 1.0, 0.0, 1.0)]
    st = orc.orbit_starts([10, 2], pos)
    assert st[:10, 0].tolist() == [1.0] * 3 + [2.0] * 3 + [3.0] * 4
    # n = 2 over three positions: cuts 0, 0, 1 -> the first position gets none
    assert st[10:, 0].tolist() == [2.0, 3.0]
    # counts track the weights to within one particle and every particle is placed once
    rng = np.random.default_rng(3)
    for _ in range(20):
        w = rng.uniform(0.1, 5.0, rng.integers(1, 9))
        n = int(rng.integers(0, 5000))
        st = orc.orbit_starts([n], [(1.0 + k, 1.0, 0.0, wk) for k, wk in enumerate(w)])
        assert len(st) == n
        counts = np.array([(st[:, 0] == 1.0 + k).sum() for k in range(len(w))])
        assert np.all(np.abs(counts - n * w / w.sum()) <= 1.0)
        assert np.all(np.diff(st[:, 0]) >= 0)   # contiguous runs in position order


def test_single_default_position_is_the_fixed_point_run(orc):
    p = W.params()
    T, N = [0.5, 5.0], [40, 40]
    a = orc.run(p, W.PROTON, T, N, seed=9)
    b = orc.run(p, W.PROTON, T, N, seed=9, positions=[(p["r0"], p["th0"], p["ph0"], 2.5)])
    for k in ("r", "th", "ph", "lnP", "s", "steps", "status"):
        assert np.array_equal(a[k], b[k]), k


def test_isotropic_radial_process_ignores_start_angles(orc):
    # K isotropic and the wind radial: dr and d lnP depend on r alone (Eq. 3, Eq. 6), so
    # the same Philox stream gives the same r, lnP, s and exit step from any start angles
    p = W.params(isotropic=1.0, drift_on=0.0, hcs_on=0.0, dt_fixed=0.1)
    T, N = [1.0], [200]
    a = orc.run(p, W.PROTON, T, N, seed=4, positions=[(3.0, math.pi / 2, 0.0, 1.0)])
    b = orc.run(p, W.PROTON, T, N, seed=4, positions=[(3.0, 0.4, 2.0, 1.0)])
    for k in ("r", "lnP", "s", "steps", "status"):
        assert np.array_equal(a[k], b[k]), k
    assert not np.array_equal(a["th"], b["th"])


def test_orbit_spectrum_is_weighted_mean_of_pde_solutions(orc):
    # detector spending 3/4 of the time at 1 AU and 1/4 at 10 AU
    K0, V, r_in, R = 11.5, 400.0, 0.1, 100.0
    T0 = np.array([0.3, 1.0])
    P0 = W.PROTON["A"] / W.PROTON["Z"] * np.sqrt(T0 * (T0 + 2 * W.PROTON["m0"]))
    J1 = pde1d.solve(W.PROTON, K0, V, r_in, R, 1.0, P0, n_r=800, dlnP=3e-3)
    J10 = pde1d.solve(W.PROTON, K0, V, r_in, R, 10.0, P0, n_r=800, dlnP=3e-3)
    expect = 0.75 * J1 + 0.25 * J10
    assert np.all(J10 > 1.05 * J1)   # the two radii are distinguishable
    p = W.params(isotropic=1.0, drift_on=0.0, hcs_on=0.0, dt_fixed=0.01)
    pos = [(1.0, math.pi / 2, 0.0, 3.0), (10.0, 1.2, 0.5, 1.0)]
    res = orc.run(p, W.PROTON, T0, [6000, 6000], seed=21, positions=pos)
    J, S = orc.spectrum_unbinned(res, W.PROTON, T0)
    # Euler-Maruyama bias at dt = 0.01 day is ~1 % (as for the fixed point); plus 3 sigma
    assert np.all(np.abs(J - expect) < 3.0 * S + 0.015 * expect), (J, expect, S)
    # a swapped split (3/4 at 10 AU) is excluded
    swapped = 0.25 * J1 + 0.75 * J10
    assert np.all(np.abs(J - swapped) > 3.0 * S)


def test_synthetic_polar_orbit_samples_equal_times():
    # the orbit of `bench.py --workload orbit`: a Kepler ellipse sampled at equal steps of mean
    # anomaly.  From each radius alone, cos E = (1 - r/a)/e gives the eccentric anomaly (up to
    # the half of the orbit) and M = E - e sin E must fall on (k + 1/2) 2 pi / n
    a, e, inc, n = 3.35, 0.6, 80.0, 12
    orbit = W.polar_orbit(n, a, e, inc)
    assert len(orbit) == n and all(q[3] == 1.0 for q in orbit)
    p = W.params()
    for k, (r, th, ph, _) in enumerate(orbit):
        assert a * (1 - e) < r < a * (1 + e) and p["r_in"] < r < p["R_out"]
        assert math.radians(90.0 - inc) - 1e-12 <= th <= math.radians(90.0 + inc) + 1e-12
        assert 0.0 <= ph < 2.0 * math.pi
        E = math.acos((1.0 - r / a) / e)
        M = E - e * math.sin(E)
        Mk = 2.0 * math.pi * (k + 0.5) / n
        assert min(abs(M - Mk), abs(2.0 * math.pi - M - Mk)) < 1e-9, (k, M, Mk)
    # the perihelion passage sweeps the latitude fastest: both ends of the sampled orbit
    # (next to perihelion) are at high latitude, the middle (aphelion) near the ecliptic
    lat = [90.0 - math.degrees(q[1]) for q in orbit]
    assert lat[0] > 45.0 and lat[-1] < -45.0 and abs(lat[n // 2]) < 10.0
