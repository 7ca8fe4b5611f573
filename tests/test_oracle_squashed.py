"""Pins of the nose-squashed heliosphere (Sec. II.B: inner heliosphere and
heliosheath squashed toward the nose): the termination shock and the outer
boundary are spheroids about the nose axis with the Sun on the axis.

  * the shock factor g is at its midpoint exactly on the shock surface, at the
    nose, the tail and the flank distances given by the spheroid's definition;
    its angular derivatives against central differences;
  * the Ito drift (which gains d/dphi terms) against Cartesian finite
    differences at points straddling the squashed shock;
  * every exit lies outside the outer spheroid and within a step of it;
  * Brownian motion (no wind, isotropic constant K) in an offset spheroid:
    the closed-form mean exit time of an ellipsoid, and the harmonic moments
    E[h(X_exit)] = h(x0) for h = the axial coordinate and for a quadratic
    harmonic polynomial (the exit distribution over the surface);
  * squashed = 0 leaves every path unchanged (the spherical model).
"""
import math

import numpy as np

from paper_2502_06319_gb300 import workloads as W
from tests.test_oracle_model import check_ito_drift

NOSE = (1.25, 0.7)   # nose direction (colatitude, longitude)


def _axis():
    th, ph = NOSE
    return np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])


def _dir(th, ph):
    return np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])


def _ray_distance(R, t, f, mu):
    """Distance along direction mu to the spheroid with nose distance R, tail R t, flank semi-axis R f
    (textbook quadratic root)."""
    a, b, c = R * (1 + t) / 2, R * f, R * (t - 1) / 2
    A = mu * mu / a ** 2 + (1 - mu * mu) / b ** 2
    B = mu * c / a ** 2
    C = c * c / a ** 2 - 1
    return (-B + math.sqrt(B * B - A * C)) / A


def _squashed(**kw):
    base = dict(R_ts=85.0, R_out=122.0, squashed=1.0, nose_th=NOSE[0], nose_ph=NOSE[1],
                ts_tail=1.35, ts_flank=1.15, hp_tail=1.6, hp_flank=1.25)
    base.update(kw)
    return W.params(**base)


def _dir_at_mu(mu, az=0.3):
    """A direction (th, ph) at angle acos(mu) from the nose."""
    n = _axis()
    e1 = np.cross(n, [0.0, 0.0, 1.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    s = math.sqrt(max(0.0, 1 - mu * mu))
    d = mu * n + s * (math.cos(az) * e1 + math.sin(az) * e2)
    return math.acos(d[2]), math.atan2(d[1], d[0]) % (2 * math.pi)


def test_shock_surface_at_nose_tail_and_flank(orc):
    p = _squashed()
    f = p["ts_K_factor"]
    mid = 1.0 - (1.0 - f) * 0.5
    a, b, c = 85.0 * (1 + 1.35) / 2, 85.0 * 1.15, 85.0 * (1.35 - 1) / 2
    for mu, R in ((1.0, 85.0), (-1.0, 85.0 * 1.35), (0.0, b * math.sqrt(1 - c * c / (a * a)))):
        th, ph = _dir_at_mu(mu) if abs(mu) < 1 else ((NOSE[0], NOSE[1]) if mu > 0 else
                                                     (math.pi - NOSE[0], NOSE[1] + math.pi))
        e = orc.evaluate(p, W.PROTON, R, th, ph, math.log(2.0))
        assert math.isclose(e["g"], mid, rel_tol=1e-12, abs_tol=1e-12), (mu, e["g"], mid)
    for mu in (-0.8, -0.3, 0.2, 0.65, 0.95):
        th, ph = _dir_at_mu(mu, az=1.1)
        R = _ray_distance(85.0, 1.35, 1.15, mu)
        e = orc.evaluate(p, W.PROTON, R, th, ph, math.log(2.0))
        assert math.isclose(e["g"], mid, rel_tol=1e-11), (mu, e["g"])


def test_shock_factor_angular_derivatives(orc):
    p = _squashed()
    for mu in (-0.7, -0.1, 0.4, 0.9):
        th, ph = _dir_at_mu(mu, az=2.0)
        R = _ray_distance(85.0, 1.35, 1.15, mu) + 0.4
        g = lambda t, q: orc.evaluate(p, W.PROTON, R, t, q, math.log(2.0))["g"]
        e = orc.evaluate(p, W.PROTON, R, th, ph, math.log(2.0))
        h = 1e-6
        fd_th = (g(th + h, ph) - g(th - h, ph)) / (2 * h)
        fd_ph = (g(th, ph + h) - g(th, ph - h)) / (2 * h)
        assert abs(e["dg_dth"] - fd_th) < 1e-6 * (abs(fd_th) + 1e-3), (mu, e["dg_dth"], fd_th)
        assert abs(e["dg_dph"] - fd_ph) < 1e-6 * (abs(fd_ph) + 1e-3), (mu, e["dg_dph"], fd_ph)
        assert abs(fd_th) + abs(fd_ph) > 1e-3          # the shock's tilt is felt here


def test_ito_drift_across_the_squashed_shock(orc):
    p = _squashed()
    pts = []
    for mu, az, dr in ((-0.6, 0.4, -0.5), (0.3, 1.9, 0.3), (0.8, 4.0, 0.0), (-0.2, 5.2, 1.0)):
        th, ph = _dir_at_mu(mu, az)
        pts.append((_ray_distance(85.0, 1.35, 1.15, mu) + dr, th, ph))
    for sp in (W.PROTON, W.ELECTRON):
        check_ito_drift(orc, p, sp, math.log(2.0), pts, hrel=3e-6)


def test_exits_lie_on_the_outer_spheroid(orc):
    p = _squashed(R_ts=0.0, R_out=12.0, hp_tail=1.8, hp_flank=1.3, max_steps=5e6)
    res = orc.run(p, W.PROTON, [0.5, 5.0], [150, 150], seed=8)
    assert np.all(res["status"] == orc.EXIT)
    a, b, c = 12.0 * 2.8 / 2, 12.0 * 1.3, 12.0 * 0.8 / 2
    n = _axis()
    for r, th, ph in zip(res["r"], res["th"], res["ph"]):
        x = r * _dir(th, ph)
        xa = x @ n
        Q = (xa + c) ** 2 / a ** 2 + (r * r - xa * xa) / b ** 2
        assert Q >= 1.0
        # within a few steps of the surface (the largest step is sqrt(2 K dt_max) ~ 1.9 AU here)
        assert r - _ray_distance(12.0, 1.8, 1.3, xa / r) < 6.0


def _bm(**kw):
    base = dict(isotropic=1.0, drift_on=0.0, hcs_on=0.0, V_const_kms=0.0, R_ts=0.0, r_in=0.05,
                dt_fixed=1e-4, squashed=1.0, nose_th=NOSE[0], nose_ph=NOSE[1], R_out=6.0,
                hp_tail=2.0, hp_flank=1.3, r0=2.0, th0=1.0, ph0=2.2)
    base.update(kw)
    return W.params(**base)


def test_brownian_exit_from_offset_spheroid(orc):
    p = _bm()
    res = orc.run(p, W.PROTON, [1.0], [6000], seed=19)
    assert np.all(res["status"] == orc.EXIT)
    K = orc.evaluate(p, W.PROTON, 2.0, 1.0, 2.2, math.log(float(orc.rigidity(W.PROTON, 1.0))))["Kpar"]
    a, b, c = 6.0 * 3.0 / 2, 6.0 * 1.3, 6.0 * 1.0 / 2
    # discrete-time overshoot: the effective surface lies 0.5826 sqrt(2 K dt) further out
    d = 0.5826 * math.sqrt(2 * K * p["dt_fixed"])
    a, b = a + d, b + d
    n = _axis()
    x0 = 2.0 * _dir(1.0, 2.2)
    xa0 = x0 @ n
    xp0 = x0 - xa0 * n
    Q0 = (xa0 + c) ** 2 / a ** 2 + (xp0 @ xp0) / b ** 2
    expect = (1 - Q0) / (2 * K * (1 / a ** 2 + 2 / b ** 2))
    s = res["s"]
    sem_s = s.std(ddof=1) / math.sqrt(len(s))
    assert abs(s.mean() - expect) < 3.5 * sem_s, (s.mean(), expect, sem_s)
    # harmonic moments of the exit distribution: x_a (linear) and x_a^2 - x_u^2 (quadratic)
    u = np.cross(n, [0.0, 0.0, 1.0])
    u /= np.linalg.norm(u)
    X = res["r"][:, None] * np.stack([_dir(t, q) for t, q in zip(res["th"], res["ph"])])
    for h, h0 in ((X @ n, xa0), ((X @ n) ** 2 - (X @ u) ** 2, xa0 ** 2 - (x0 @ u) ** 2)):
        sem = h.std(ddof=1) / math.sqrt(len(h))
        assert abs(h.mean() - h0) < 4.0 * sem, (h.mean(), h0, sem)
    # the sphere of the same nose distance is clearly different (exit time ~ R^2 / (6K))
    assert abs(s.mean() - (36.0 - 4.0) / (6 * K)) > 10 * sem_s


def test_unsquashed_paths_unchanged(orc):
    p0 = W.params(R_ts=85.0, R_out=122.0)
    p1 = dict(p0, squashed=0.0, nose_th=0.3, nose_ph=1.0, ts_tail=1.5, hp_tail=1.7)
    a = orc.run(p0, W.PROTON, [0.5, 5.0], [30, 30], seed=4)
    b = orc.run(p1, W.PROTON, [0.5, 5.0], [30, 30], seed=4)
    for k in ("r", "th", "ph", "lnP", "s", "steps", "status"):
        assert np.array_equal(a[k], b[k]), k
