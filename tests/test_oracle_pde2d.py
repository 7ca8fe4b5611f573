"""Whole-path pin of the anisotropic model with drifts: the SDE oracle against an
independent deterministic solution of the steady transport equation.

With a unipolar field, or a field reversing across a flat (untilted) current
sheet, the model is axisymmetric and the steady momentum-form equation (Eq. 5)
is a 2-D problem in (r, th), solved by oracle/pde2d.py in conservative
finite-volume form.  It shares no code with the SDE oracle: the Ito drift, the
Cholesky factor, the step rule and the path loop of the SDE never appear in
it, so a dropped or mis-signed term anywhere in the step (Eq. 3) changes the
Monte Carlo spectrum but not the PDE's.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import pde1d, pde2d
from paper_2502_06319_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "pde2d_axisymmetric.json")

# coarse grids the tests solve on, and their agreement with the stored fine-grid solutions
COARSE = {"unipolar": (dict(n_r=60, n_th=60, dlnP=0.01), 1e-3),
          "flat_sheet": (dict(n_r=60, n_th=90, dlnP=0.02, th_stretch=1.5), 1.5e-3)}
# paths per energy of the Monte Carlo comparison (the sheet holds paths longer: smaller steps)
PATHS = {"unipolar": 8000, "flat_sheet": 6000}


@pytest.fixture(scope="module")
def golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _P0(sp, T0):
    return np.array([sp["A"] / abs(sp["Z"]) * math.sqrt(T * (T + 2 * sp["m0"])) for T in T0])


def _cases(golden, name, species="proton"):
    cases = [c for c in golden["cases"] if c["name"] == name and c["species_name"] == species]
    assert [c["params"]["polarity"] for c in cases] == [1.0, -1.0]
    return cases


def test_reduces_to_the_1d_solver():
    # K_perp = K_par and one wind speed, no drift: the spherically symmetric problem
    T0 = [0.3, 1.0, 3.0]
    P0 = _P0(W.PROTON, T0)
    p = W.params(R_out=20.0, kperp_r_frac=1.0, kperp_th_frac=1.0, V_fast_kms=400.0, drift_on=0.0, hcs_on=0.0)
    J2 = pde2d.solve(W.PROTON, p, 1.0, math.pi / 2, P0, n_r=100, n_th=8, dlnP=0.01)
    J1 = pde1d.solve(W.PROTON, 11.5, 400.0, 0.1, 20.0, 1.0, P0, n_r=1600, dlnP=1.5e-3, P_top=300.0)
    assert np.all(np.abs(J2 / J1 - 1) < 1e-3), (J2, J1)


def test_rejects_models_outside_its_scope():
    for extra in (dict(hcs_on=1.0, tilt_deg=10.0), dict(isotropic=1.0), dict(n_shells=2.0)):
        with pytest.raises(ValueError):
            pde2d.solve(W.PROTON, W.params(R_out=20.0, **extra), 1.0, 1.0, [1.0], n_r=8, n_th=8)


@pytest.mark.parametrize("name", list(COARSE))
def test_grid_converged(golden, name):
    r0, th0 = golden["observer"]
    grid, tol = COARSE[name]
    for case in _cases(golden, name):
        J = pde2d.solve(case["species"], case["params"], r0, th0, _P0(case["species"], golden["T0"]), **grid)
        assert np.all(np.abs(J / np.array(case["J"]) - 1) < tol), (J, case["J"])


@pytest.mark.parametrize("name", list(COARSE))
def test_sde_spectrum_matches_pde_with_drifts(orc, golden, name):
    """Both polarity epochs: within 3 sigma plus 0.5 %.  The allowance covers the bias of
    the Euler-Maruyama step and of testing for the exit only after each step, measured
    with 2-4e4 paths per energy at the default step control as 0.16-0.37 % (unipolar)
    and at most 0.25 % (flat sheet), shrinking as all step limits are divided by 4,
    plus the PDE's grid error (below 3e-4)."""
    T0 = golden["T0"]
    out = []
    for case in _cases(golden, name):
        sp = case["species"]
        res = orc.run(case["params"], sp, T0, [PATHS[name]] * len(T0), seed=21)
        assert np.all(res["status"] == orc.EXIT)
        J, S = orc.spectrum_unbinned(res, sp, T0)
        Jp = np.array(case["J"])
        assert np.all(np.abs(J - Jp) < 3.0 * S + 0.005 * Jp), (case["params"]["polarity"], J, Jp, S)
        out.append((J, S))
    # the drift decides: the two epochs differ by far more than their errors
    (Ja, Sa), (Jb, Sb) = out
    assert np.all(np.abs(Ja - Jb) > 10.0 * (Sa + Sb)), (Ja, Jb)


def test_energy_form_matches_pde_with_drifts(orc, golden):
    """The energy formulation (Eq. 1 with the loss weight of Eq. 4) meets the same bar
    against the same PDE solutions (unipolar field, both epochs)."""
    T0 = golden["T0"]
    for case in _cases(golden, "unipolar"):
        sp = case["species"]
        p = dict(case["params"], formulation=1.0)
        res = orc.run(p, sp, T0, [PATHS["unipolar"]] * len(T0), seed=21)
        J, S = orc.spectrum_energy_form(res, sp, T0)
        Jp = np.array(case["J"])
        assert np.all(np.abs(J - Jp) < 3.0 * S + 0.005 * Jp), (case["params"]["polarity"], J, Jp, S)


def test_other_species_match_pde(orc, golden):
    """He-4 (A/Z = 2) and electrons (negative charge, beta ~ 1) with the unipolar field, both
    epochs, within 3 sigma plus 0.5 %; the drift's sign follows sgn(q) sgn(A), so the epoch
    that favours protons disfavours electrons."""
    T0 = golden["T0"]
    for species in ("he4", "electron"):
        J_by_pol = {}
        for case in _cases(golden, "unipolar", species):
            res = orc.run(case["params"], case["species"], T0, [PATHS["unipolar"]] * len(T0), seed=21)
            J, S = orc.spectrum_unbinned(res, case["species"], T0)
            Jp = np.array(case["J"])
            assert np.all(np.abs(J - Jp) < 3.0 * S + 0.005 * Jp), (species, case["params"]["polarity"], J, Jp, S)
            J_by_pol[case["params"]["polarity"]] = Jp
        favoured = J_by_pol[1.0] > J_by_pol[-1.0]
        assert np.all(favoured) if species == "he4" else not np.any(favoured), (species, J_by_pol)
