"""Pin of the adaptive step rule (Sec. IV.A: the step is adapted so that the
advective displacement stays small against the diffusive one; the reading
implemented on both sides is dt = min(dt_max, eps_adv 2 K_rr / A_r^2,
eps_diff r^2 / K_rr, eps_diff (r delta)^2 / K_thth), floored at dt_min).

The Euler-Maruyama spectrum of Eq. 4 carries a bias that must vanish as the
steps shrink.  Its leading term comes from testing for the exit only after each
step (discrete monitoring of an absorbing boundary: the path overshoots by
O(sqrt(dt)), Siegmund's correction), so with every limit of the rule multiplied
by c -- eps_adv, eps_diff, dt_max and dt_min alike, which multiplies every step
by c -- the spectrum must behave as J(c) = J_0 (1 + b sqrt(c) + O(c)), J_0 the
exact solution.  Against the independent 2-D PDE solution (oracle/pde2d.py) of
a drift-free, strongly anisotropic heliosphere, where this bias is largest,
the oracle's spectra at c = 16, 4 and 1 must
  (i)   deviate from the PDE less and less as c shrinks, each step of c by
        more than the Monte Carlo error,
  (ii)  with deviations in the ratio sqrt(4) = 2 between successive c, and
  (iii) extrapolate (Richardson in sqrt(c): J_0 = 2 J(1) - J(4)) to the PDE.
A step rule that does not follow its limits (a step fixed elsewhere, a floor
or cap that binds), or an Euler-Maruyama step whose limit is not the transport
equation, fails (i)-(iii); at the default limits (c = 1) the bias of this model
is a few per cent, so a rule that took steps several times larger than its
limits allow would show as a deviation far outside (i)'s sequence.
"""
import math

import numpy as np
import pytest

from oracle import pde2d
from paper_2502_06319_gb300 import workloads as W

T0 = [0.3, 1.0, 3.0]
N = 20000


def _model(c=1.0):
    p = W.params(R_out=20.0, R_ts=10.0, drift_on=0.0, hcs_on=0.0, kperp_r_frac=0.2, kperp_th_frac=0.2)
    return dict(p, eps_adv=0.01 * c, eps_diff=0.01 * c, dt_max=0.1 * c, dt_min=1e-4 * c)


@pytest.fixture(scope="module")
def pde():
    P0 = [W.PROTON["A"] / abs(W.PROTON["Z"]) * math.sqrt(T * (T + 2 * W.PROTON["m0"])) for T in T0]
    return np.asarray(pde2d.solve(W.PROTON, _model(), 1.0, math.pi / 2, P0, n_r=60, n_th=60, dlnP=0.01))


def _pooled(d, s):
    """Inverse-variance mean over the energies of the relative deviations d with errors s."""
    w = 1.0 / s ** 2
    return float((w * d).sum() / w.sum()), float(1.0 / math.sqrt(w.sum()))


def test_bias_vanishes_as_sqrt_of_the_step(orc, pde):
    dev, err, J, S = {}, {}, {}, {}
    for c in (16.0, 4.0, 1.0):
        res = orc.run(_model(c), W.PROTON, T0, [N] * len(T0), seed=31)
        assert np.all(res["status"] == orc.EXIT)
        J[c], S[c] = orc.spectrum_unbinned(res, W.PROTON, T0)
        dev[c], err[c] = _pooled(J[c] / pde - 1.0, S[c] / pde)
        print(f"c = {c:4.0f}: steps/path {res['steps'].mean():8.1f}, J/J_pde - 1 = {dev[c]:+.4f} +- {err[c]:.4f}")
    # (i) monotone approach from below, each step resolved
    assert dev[16.0] < dev[4.0] < dev[1.0] < 0.0
    for a, b in ((16.0, 4.0), (4.0, 1.0)):
        assert dev[b] - dev[a] > 3.0 * math.hypot(err[a], err[b]), (a, b, dev, err)
    # (ii) the leading bias scales as sqrt(dt): successive ratios near 2
    for a, b in ((16.0, 4.0), (4.0, 1.0)):
        ratio = dev[a] / dev[b]
        assert 1.4 < ratio < 2.9, (a, b, ratio)
    # (iii) Richardson extrapolation in sqrt(c) reaches the PDE solution
    J0 = 2.0 * J[1.0] - J[4.0]
    S0 = np.hypot(2.0 * S[1.0], S[4.0])
    assert np.all(np.abs(J0 - pde) < 3.0 * S0 + 0.005 * pde), (J0 / pde - 1, S0 / pde)
