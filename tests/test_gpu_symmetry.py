"""Symmetries of the step on the GPU (both precisions): a centred sessile drop in a
vertical field stays mirror-symmetric in x, and y-uniform data on a periodic y axis
stays y-uniform.  The kernels evaluate mirrored faces in different threads and
orders, so the bounds are round-off over the run, not bitwise."""
import numpy as np
import pytest

from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

pytestmark = pytest.mark.gpu
TOL = {lbfs.FP64: 1e-10, lbfs.MIXED: 1e-4}


@pytest.mark.parametrize("precision", [lbfs.FP64, lbfs.MIXED])
def test_mirror_symmetry_vertical_field(precision):
    c = I.case(64, 32, radius=12.0, bo_m=2.0, field_angle_deg=90.0, stefan=0.2)
    s = lbfs.Solver(precision=precision, max_cases=1)
    s.set_case(0, c)
    s.step(200)
    out = s.fields(0, [I.C, I.HE, I.P, I.U, I.V, I.PHI])
    s.close()
    for f, sgn in ((I.C, 1), (I.HE, 1), (I.P, 1), (I.U, -1), (I.V, 1), (I.PHI, 1)):
        a = out[f]
        scale = max(float(np.max(np.abs(a))), 1e-30)
        assert np.max(np.abs(a - sgn * a[:, ::-1])) <= TOL[precision] * scale, I.FIELD_NAMES[f]


@pytest.mark.parametrize("precision", [lbfs.FP64, lbfs.MIXED])
def test_one_dimensional_reduction(precision):
    nx, ny = 48, 8
    c = I.case(nx, ny, periodic_y=1, init=2, T_init=0.5, stefan=0.0, latent=2.0, chi_l=0, chi_s=0,
               thermal_dirichlet=(1, 0, 0, 0), wall_T=(-1.0, 0.0, 0.0, 0.0))
    s = lbfs.Solver(precision=precision, max_cases=1)
    s.set_case(0, c)
    xs = np.arange(nx) + 0.5
    C = (0.5 + 0.5 * np.tanh((24 - xs) / 2.0))[None, :] * np.ones((ny, 1))
    cp = C * c["cp_l"] + (1 - C) * c["cp_g"]
    s.set_fields(0, {I.C: C, I.HE: cp * 0.5 + c["latent"],
                     I.MX: (1e-3 * np.sin(xs / 3.0))[None, :] * np.ones((ny, 1))})
    s.step(100)
    out = s.fields(0, [I.C, I.HE, I.P, I.U, I.V])
    s.close()
    tol = 1e-12 if precision == lbfs.FP64 else 1e-6
    for f in (I.C, I.HE, I.P, I.U):
        a = out[f]
        assert np.max(np.abs(a - a[:1, :])) <= tol * max(float(np.max(np.abs(a))), 1e-30), I.FIELD_NAMES[f]
    assert np.max(np.abs(out[I.V])) <= tol * max(float(np.max(np.abs(out[I.U]))), 1e-30)
