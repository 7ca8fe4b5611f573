"""The energy formulation (Eq. 1, integrated as a T-SDE with the loss weight of
Eq. 4) against the momentum formulation (Eq. 5-6, L = 0).

Eq. 1 for the density per unit kinetic energy U = 4 pi J / v gives, in the
backward form of Eq. 2, the drift A_T = (2/3)(V/r) alpha T (Eq. 6, left) and
the loss L = div V - (1/3) div V d(alpha T)/dT = (2V/(3r)) (1 + beta^2).  Along
a path d ln(P^2/beta) = (1 + beta^2) d lnP = L ds, so the weight exp(-sum L ds)
must equal (P0^2/beta0) / (P_ex^2/beta_ex), and both formulations must give
the same spectrum.  This pins the estimator J(T0) = P0^2 <J_LIS(T_ex)/P_ex^2>
(J = f P^2 as intensity per unit kinetic energy) by a route independent of it.
"""
import math

import numpy as np
import pytest

from oracle import pde1d
from paper_2502_06319_gb300 import workloads as W


def _both(orc, p, sp, T, n, seed):
    mom = orc.run(p, sp, T, n, seed=seed)
    en = orc.run(dict(p, formulation=1.0), sp, T, n, seed=seed)
    return mom, en


def test_loss_weight_equals_rigidity_ratio_pathwise(orc):
    p = W.params(isotropic=1.0, drift_on=0.0, hcs_on=0.0, dt_fixed=0.005)
    T = [0.2, 1.0, 10.0]
    mom, en = _both(orc, p, W.PROTON, T, [200, 200, 200], 31)
    P0 = orc.rigidity(W.PROTON, np.asarray(T))[en["energy"]]
    Pex = np.exp(en["lnP"])
    expect = np.log(P0 ** 2 / orc.beta(W.PROTON, P0)) - np.log(Pex ** 2 / orc.beta(W.PROTON, Pex))
    assert np.all(en["lw"] < 0)
    # Euler-Maruyama in T and in the loss integral: agreement to O(dt), relative
    assert np.all(np.abs(en["lw"] - expect) <= 0.01 * np.abs(expect) + 1e-12)
    assert np.all(mom["lw"] == 0.0)


def test_energy_and_momentum_forms_give_the_same_spectrum(orc):
    p = W.params(isotropic=1.0, drift_on=0.0, hcs_on=0.0, dt_fixed=0.01)
    T = np.array([0.3, 1.0])
    mom, en = _both(orc, p, W.PROTON, T, [4000, 4000], 41)
    Jm, Sm = orc.spectrum_unbinned(mom, W.PROTON, T)
    Je, Se = orc.spectrum_energy_form(en, W.PROTON, T)
    P0 = W.PROTON["A"] / W.PROTON["Z"] * np.sqrt(T * (T + 2 * W.PROTON["m0"]))
    Jp = pde1d.solve(W.PROTON, 11.5, 400.0, 0.1, 100.0, 1.0, P0, n_r=800, dlnP=3e-3)
    # paired paths: the two estimates agree far inside their Monte Carlo errors
    assert np.all(np.abs(Je / Jm - 1) < 0.01), (Je, Jm)
    # both agree with the PDE solution to the EM bias plus 3 sigma
    for J, S in ((Jm, Sm), (Je, Se)):
        assert np.all(np.abs(J - Jp) < 3 * S + 0.015 * Jp), (J, Jp, S)


def test_full_model_forms_agree(orc):
    p = W.params(R_out=40.0)
    T = [0.5, 5.0]
    mom, en = _both(orc, p, W.PROTON, T, [300, 300], 43)
    Jm, Sm = orc.spectrum_unbinned(mom, W.PROTON, T)
    Je, Se = orc.spectrum_energy_form(en, W.PROTON, T)
    assert np.all(np.abs(Je - Jm) < 3 * np.hypot(Sm, Se) + 0.01 * Jm), (Je, Jm, Sm, Se)
