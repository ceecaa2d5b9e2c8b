"""Wetting walls (contact angle theta_w) on the GPU: FP64 parity with the oracle on a
ragged multi-tile sessile drop with freezing and a field on, the cap angle a drop
relaxes to in mixed precision, and the argument check."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

from parity import assert_parity

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("theta", [64.0, 98.0, 135.0])
def test_wetting_parity_fp64(theta):
    c = I.case(70, 27, radius=10.0, bo_m=1.0, field_angle_deg=90.0, stefan=0.2, contact_angle_deg=theta,
               rho_s=0.9, gravity=-1e-4)
    ref = oracle.Oracle(c, threads=4)
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1)
    s.set_case(0, c)
    for n in (1, 40, 160):
        ref.step(n)
        s.step(n)
        assert_parity(s, 0, ref, 1e-9)
    s.close()


def _cap_angle(C, H_m):
    row = C[0]
    idx = np.where(row >= 0.5)[0]
    i0, i1 = idx.min(), idx.max()
    xl = i0 + 0.5 - (row[i0] - 0.5) / (row[i0] - row[i0 - 1])
    xr = i1 + 0.5 + (row[i1] - 0.5) / (row[i1] - row[i1 + 1])
    return 2.0 * math.degrees(math.atan((H_m - 0.5) / (0.5 * (xr - xl))))


@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_drop_relaxes_to_the_contact_angle_mixed(theta):
    c = I.case(128, 64, radius=24.0, contact_angle_deg=theta, thermal_dirichlet=(0, 0, 0, 0), T_init=1.0,
               chi_l=0, chi_s=0, stefan=0.0, latent=10.0)
    s = lbfs.Solver(precision=lbfs.MIXED, max_cases=1, use_graph=True)
    s.set_case(0, c)
    s.step(12000)
    ang = _cap_angle(s.field(0, I.C), s.diagnostics(0)[0]["H_m"])
    s.close()
    assert abs(ang - theta) < 5.0, ang


def test_contact_angle_range_is_checked():
    s = lbfs.Solver(precision=lbfs.MIXED, max_cases=1)
    for bad in (0.0, 180.0, -5.0, float("nan")):
        with pytest.raises(lbfs.LbfsError):
            s.set_case(0, I.case(32, 16, contact_angle_deg=bad))
    s.close()
