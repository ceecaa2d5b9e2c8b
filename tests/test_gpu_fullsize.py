"""Parity at the full workload sizes, in the launch configuration bench.py times
(the autotuned 32 x 8 tile), on sampled outputs the oracle computes window by
window: one step of a cell depends only on cells within nine of it (three per
Runge-Kutta stage) once the step's potential is fixed.  The GPU's state before a
step, and the potential it solved for that step, are cut into windows; the oracle
advances each window one step with that potential, and the window interiors (a
12-cell margin dropped on every side that is not a real wall) are compared: FP64
within 1e-9 of each field's scale, mixed precision within 1e-4 (one step of FP32
fluxes on the same state; the momentum is a small residual of larger balances).
On the 4096x2048 case the check is made at step 13 and again at step 500, so the
first 500 steps of that workload are covered."""
import math

import numpy as np
import pytest

import oracle
from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
STATE = [I.HE, I.P, I.C, I.MX, I.MY, I.FSPREV]
CMP = [I.HE, I.P, I.C, I.MX, I.MY, I.T, I.FL]
MARGIN = 12
BENCH_TILE = 10  # the shape the autotuner keeps for these grids (32 x 8, four blocks of 256 threads per SM)


def _windows(nx, ny, R, angle):
    """(x0, y0, w, h) windows: on the drop's interface, on the bottom wall under the
    contact line, and in the gas"""
    cx = nx // 2
    w = 64
    out = [(cx - w // 2, min(int(0.6 * R), ny - w - 1), w, w),
           (cx + int(R) - w // 2, 0, w, w),
           (max(cx - int(1.6 * R), 1), min(int(1.2 * R), ny - w - 1), w, w)]
    return [(max(x, 0), max(y, 0), min(w, nx - max(x, 0)), min(h, ny - max(y, 0))) for x, y, w, h in out]


def _window_case(case, x0, y0, w, h):
    c = dict(case, nx=w, ny=h, flags=oracle.FLAG_KEEP_POTENTIAL)
    bottom = y0 == 0
    c["thermal_dirichlet"] = (0, 0, case["thermal_dirichlet"][2] if bottom else 0, 0)
    return c, bottom


@pytest.mark.parametrize("precision,tol", [(lbfs.FP64, 1e-9), (lbfs.MIXED, 1e-4)])
@pytest.mark.parametrize("cfg,warm", [("huge", 12), ("huge", 499), ("large", 12), ("medium", 12)])
def test_fullsize_windows(cfg, warm, precision, tol):
    case = {"huge": I.config_huge, "large": I.config_large, "medium": I.config_medium}[cfg]()
    s = lbfs.Solver(precision=precision, max_cases=1, tile=BENCH_TILE, use_graph=True)
    s.set_case(0, case)
    s.step(warm)
    before = s.fields(0, STATE)
    s.step(1)
    after = s.fields(0, CMP + [I.PHI])
    s.close()
    worst = 0.0
    for (x0, y0, w, h) in _windows(case["nx"], case["ny"], case["radius"], case["field_angle_deg"]):
        wc, bottom = _window_case(case, x0, y0, w, h)
        o = oracle.Oracle(wc)
        sl = (slice(y0, y0 + h), slice(x0, x0 + w))
        o.set_state({f: before[f][sl] for f in STATE})
        # the window's walls hold the far field in window coordinates: shift the
        # potential by the far field at the window origin (gradients unchanged)
        H0 = math.sqrt(case["bo_m"] * case["sigma"] / (2.0 * case["radius"]))
        a = math.radians(case["field_angle_deg"])
        o.set(I.PHI, after[I.PHI][sl] + H0 * (x0 * math.cos(a) + y0 * math.sin(a)))
        o.step(1)
        ys = slice(0 if bottom else MARGIN, h - MARGIN)
        xs = slice(MARGIN, w - MARGIN)
        for f in CMP:
            ref = o.get(f)[ys, xs]
            got = after[f][sl][ys, xs]
            scale = max(float(np.max(np.abs(after[f]))), 1e-30) if f not in (I.FL,) else 1.0
            err = float(np.max(np.abs(got - ref))) / scale
            worst = max(worst, err)
            assert err <= tol, (cfg, (x0, y0), I.FIELD_NAMES[f], err)
    print(f"{cfg} after {warm + 1} steps, precision {precision}: worst window error {worst:.2e}")
