"""Degenerate starts of a path, through the C ABI, against the FP64 oracle.

* A detection point on the inner reflecting sphere (r0 = r_in): the first
  inward step is reflected at once (Sec. IV.A's boundary handling as read here:
  r <- 2 r_in - r).
* A detection point 1e-10 AU inside the outer boundary: about half of the
  paths leave on their first step (the absorbing boundary of Eq. 3's loop,
  tested after each step).  In the mixed path the start is the float-float
  pair (100, -1e-10), whose high word equals R_out; only an exact test of the
  pair keeps these particles inside until they have stepped.
* The same start with a limit of one step: every path ends on step 1, either
  outside (EXIT) or at the limit (STEP_LIMIT).

FP64 paths must equal the oracle's (same status and exit step, state within
1e-10).  The mixed paths draw the same Philox words, so where the first step
decides, both accumulations must end each path as the FP64 path does.
"""
import numpy as np
import pytest

from paper_2502_06319_gb300 import cosmica as cz
from paper_2502_06319_gb300 import workloads as W
from tests.gpu_util import compare_paths, gpu_run

pytestmark = pytest.mark.gpu

T = [0.3, 3.0, 30.0]
N = [24, 24, 24]
R_OUT = 100.0


def test_start_on_the_inner_sphere(orc):
    p = W.params(r0=0.1, r_in=0.1)
    job = W.Job(p, W.PROTON, T, N, seed=17)
    g, out, m = gpu_run(job)
    m.close()
    o = orc.job_run(job)
    frac, worst = compare_paths(g, o)
    assert frac >= 0.999 and worst <= 1e-10, (frac, worst)
    for prec in (cz.PREC_MIXED, cz.PREC_MIXED_F64ACC):
        gm, outm, mm = gpu_run(job, precision=prec)
        mm.close()
        assert np.all(gm["status"] == cz.PATH_EXIT)
        assert np.all(gm["r"] >= R_OUT)


@pytest.mark.parametrize("max_steps", [1, 100_000_000])
def test_start_a_hair_inside_the_outer_boundary(orc, max_steps):
    p = W.params(r0=R_OUT - 1e-10, R_out=R_OUT, max_steps=max_steps)
    job = W.Job(p, W.PROTON, T, N, seed=17)
    g, out, m = gpu_run(job)
    m.close()
    o = orc.job_run(job)
    frac, worst = compare_paths(g, o)
    assert frac == 1.0 and worst <= 1e-10, (frac, worst)
    first = g["steps"] == 1
    out_first = first & (g["status"] == cz.PATH_EXIT)
    assert 0.2 < out_first.mean() < 0.8, out_first.mean()   # many leave on step 1, not all
    if max_steps == 1:
        assert np.all(first)
        assert set(np.unique(g["status"])) == {cz.PATH_EXIT, cz.PATH_STEP_LIMIT}
    for prec in (cz.PREC_MIXED, cz.PREC_MIXED_F64ACC):
        gm, outm, mm = gpu_run(job, precision=prec)
        mm.close()
        # paired paths: the same particles leave on step 1, the others step on
        mf = (gm["steps"] == 1) & (gm["status"] == cz.PATH_EXIT)
        assert np.array_equal(mf, out_first), (prec, np.flatnonzero(mf != out_first))
        if max_steps == 1:
            assert np.array_equal(gm["status"], g["status"])
            assert np.allclose(gm["r"], g["r"], rtol=1e-5, atol=0.0)
        else:
            assert np.all(gm["status"] == cz.PATH_EXIT)
