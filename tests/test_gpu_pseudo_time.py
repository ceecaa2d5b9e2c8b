"""The paper's own magnetic solver on the GPU (explicit pseudo-time relaxation of the
magnetic LBFS, Sec. 3.2, Eqs. 12-18) against the oracle's per-direction
implementation, step for step; and its fixed point against the direct solve."""
import numpy as np
import pytest

import oracle
from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

pytestmark = pytest.mark.gpu


def _case(**kw):
    args = dict(init=1, radius=2.5, drop_x=4.0, drop_y=4.0, T_init=1.0, H0=0.05, field_angle_deg=20.0,
                chi_l=2.0, chi_s=2.0)
    args.update(kw)
    return I.case(8, 8, **args)


@pytest.mark.parametrize("kw", [dict(), dict(dts=0.3), dict(mag_bc=1),
                                dict(periodic_x=1, field_angle_deg=90.0),
                                dict(dts=0.7, field_angle_deg=65.0)])
def test_pseudo_time_steps_match_oracle(kw):
    c = _case(**kw)
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1)
    s.set_case(0, c)
    o = oracle.Oracle(c)
    for n in (1, 7, 60):
        s.potential_pseudo_time(0, n, 0.05)
        o.pseudo_time_potential(n, 0.05)
        got, ref = s.field(0, I.PHI), o.get(I.PHI)
        assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    s.close()


@pytest.mark.parametrize("prec", [lbfs.FP64, lbfs.MIXED])
def test_pseudo_time_fixed_point_is_the_direct_solution(prec):
    c = _case()
    o = oracle.Oracle(c)
    assert o.solve_potential() == 0
    direct = o.get(I.PHI)
    s = lbfs.Solver(precision=prec, max_cases=1)
    s.set_case(0, c)
    s.potential_pseudo_time(0, 3000, 0.05)
    got = s.field(0, I.PHI)
    s.close()
    tol = 1e-11 if prec == lbfs.FP64 else 1e-6
    assert np.max(np.abs(got - direct)) <= tol * np.max(np.abs(direct))


def test_pseudo_time_rejects_bad_arguments():
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1)
    s.set_case(0, _case())
    for it, dt in ((-1, 0.05), (5, 0.0), (5, -1.0)):
        with pytest.raises(lbfs.LbfsError):
            s.potential_pseudo_time(0, it, dt)
    s.close()
