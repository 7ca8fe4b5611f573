"""Pins of the oracle's deterministic FP64 elementary functions against libm.

The oracle and the FP64 GPU path share one classical algorithm per function
(Cody-Waite reduction + truncated series) so that paths through the chaotic
current-sheet region agree bit for bit.  Here each function is checked against
the platform libm over the argument ranges the step uses (and beyond).
"""
import numpy as np
import pytest


def _ulp_err(got, ref):
    return np.abs(got - ref) / np.spacing(np.abs(ref))


RANGES = {
    "exp": [(-30.0, 30.0), (-700.0, 700.0), (-1e-8, 1e-8)],
    "log": [(1e-12, 1.0), (0.5, 2.0), (1.0, 1e300), (2.3e-10, 1.0)],
    "sin": [(-7.0, 7.0), (0.0, 1000.0), (-1e-6, 1e-6)],
    "cos": [(-7.0, 7.0), (0.0, 1000.0)],
    "atan": [(-5.0, 5.0), (-1e6, 1e6), (-0.3, 0.3)],
}
TOL_ULP = {"exp": 3, "log": 3, "sin": 3, "cos": 3, "atan": 3}


@pytest.mark.parametrize("name", list(RANGES))
def test_relative_accuracy(orc, name):
    rng = np.random.default_rng(1)
    ref_fn = {"exp": np.exp, "log": np.log, "sin": np.sin, "cos": np.cos, "atan": np.arctan}[name]
    for lo, hi in RANGES[name]:
        if name == "log" and hi / lo > 1e3:
            x = np.exp(rng.uniform(np.log(lo), np.log(hi), 200_000))
        else:
            x = rng.uniform(lo, hi, 200_000)
        got = orc.fn(name, x)
        ref = ref_fn(x)
        if name in ("sin", "cos"):
            # near a zero of sin/cos the reduced argument carries the absolute error
            err = np.abs(got - ref) / np.maximum(np.spacing(np.abs(ref)), np.spacing(np.abs(x)) * 2e-3 + 1e-300)
            err = np.minimum(err, np.abs(got - ref) / 1.2e-16)
        else:
            err = _ulp_err(got, ref)
        assert err.max() <= TOL_ULP[name], (name, lo, hi, err.max(), x[np.argmax(err)])


def test_tanh_absolute_accuracy(orc):
    rng = np.random.default_rng(2)
    for lo, hi in [(-25.0, 25.0), (-1.0, 1.0), (-1e-3, 1e-3)]:
        x = rng.uniform(lo, hi, 200_000)
        got = orc.fn("tanh", x)
        assert np.abs(got - np.tanh(x)).max() < 4e-16
    assert orc.fn("tanh", np.array([0.0, 30.0, -30.0])).tolist() == [0.0, 1.0, -1.0]


def test_special_values(orc):
    assert orc.fn("exp", np.array([0.0]))[0] == 1.0
    assert orc.fn("log", np.array([1.0]))[0] == 0.0
    assert orc.fn("sin", np.array([0.0]))[0] == 0.0
    assert orc.fn("cos", np.array([0.0]))[0] == 1.0
    assert orc.fn("atan", np.array([0.0]))[0] == 0.0
    assert np.isnan(orc.fn("exp", np.array([np.nan]))[0])
    assert orc.fn("exp", np.array([800.0]))[0] == np.inf
    assert orc.fn("exp", np.array([-800.0]))[0] == 0.0
    # odd symmetry
    x = np.linspace(0.01, 10, 1000)
    assert np.array_equal(orc.fn("atan", -x), -orc.fn("atan", x))
    assert np.array_equal(orc.fn("tanh", -x), -orc.fn("tanh", x))
