"""The paper's main physical finding as a sanity check (a trend, not parity): a
vertical uniform field elongates the ferrofluid drop and lengthens its freezing
time; a horizontal field flattens it and shortens freezing (Sec. 5.1, 5.3); the
effect grows with Bo_m.  Also the one-dimensional Stefan estimate of the freezing
time, t ~ (H_m / 2 lambda)^2 / alpha with lambda = sqrt(C_p dT / 2L), is within a
factor of two (the droplet is not a slab)."""
import math

import pytest

from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_field_orientation_changes_freezing_time():
    base = dict(radius=18.0, stefan=0.1, chi_l=2.0, chi_s=2.0)
    cases = [I.case(96, 64, bo_m=0.0, **base),
             I.case(96, 64, bo_m=1.0, field_angle_deg=90.0, **base),
             I.case(96, 64, bo_m=2.0, field_angle_deg=90.0, **base),
             I.case(96, 64, bo_m=1.0, field_angle_deg=0.0, **base),
             I.case(96, 64, bo_m=2.0, field_angle_deg=0.0, **base)]
    s = lbfs.Solver(precision=lbfs.MIXED, max_cases=len(cases), use_graph=True)
    for k, c in enumerate(cases):
        s.set_case(k, c)
    s.step(600)   # the shape settles early (the field acts mostly before freezing)
    # droplet height H_m: the highest C = 1/2 crossing, interpolated between cell centres
    H = [s.diagnostics(k)[0]["H_m"] for k in range(len(cases))]
    tf = [-1.0] * len(cases)
    for _ in range(200):
        st = s.step(500)
        tf = [x["t_freeze"] for x in st]
        if min(tf) > 0:
            break
    s.close()
    t0, tv1, tv2, th1, th2 = tf
    print("heights", H, "t_freeze", tf)
    assert min(tf) > 0
    assert H[2] > H[0] > H[4]                      # vertical elongates, horizontal flattens
    assert tv2 > tv1 > t0 > th1 > th2              # and the freezing times follow
    # one-dimensional Stefan estimate with the liquid properties of the defaults
    c = cases[0]
    lam = math.sqrt(c["cp_l"] * 1.0 / (2.0 * 1.0 / c["stefan"]))
    alpha = c["lam_s"] / (c["rho_s"] * c["cp_s"])
    est = (H[0] / (2.0 * lam)) ** 2 / alpha
    assert 0.5 * est < t0 < 2.0 * est, (t0, est)
