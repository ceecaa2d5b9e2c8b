"""Sec. 5 diagnostics (droplet height H_m, largest droplet speed and Peclet number,
Fourier number, local heat flux on the cold substrate) of the CUDA path against the
oracle: on seeded random states, after stepping a ragged sessile drop, and on the
full 1024x512 and 4096x2048 grids (the oracle evaluating the GPU's state)."""
import numpy as np
import pytest

import oracle
from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

from parity import set_both

pytestmark = pytest.mark.gpu
TOL = 1e-9
STATE = [I.PHI, I.HE, I.P, I.C, I.MX, I.MY, I.FSPREV]
KEYS = ("H_m", "U_max", "Pe", "Fo", "Q_wall")


def _check(got, ref, tol, keys=KEYS):
    (dg, qg), (dr, qr) = got, ref
    for k in keys:
        assert abs(dg[k] - dr[k]) <= tol * max(abs(dr[k]), 1e-300), (k, dg[k], dr[k])
    scale = max(float(np.max(np.abs(qr))), 1e-300)
    assert float(np.max(np.abs(qg - qr))) <= tol * scale


@pytest.fixture(scope="module")
def solver_fp64():
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1)
    yield s
    s.close()


@pytest.mark.parametrize("seed", range(3))
def test_random_state(solver_fp64, seed):
    """every branch of Eq. 8 in the wall rows, droplet and gas cells, nonzero momentum"""
    c = I.case(24, 16, radius=6.0, stefan=0.0, latent=10.0, rho_s=0.9)
    st = I.random_state(24, 16, seed=seed, latent=10.0)
    ref = oracle.Oracle(c)
    solver_fp64.set_case(0, c)
    set_both(solver_fp64, 0, ref, st)
    _check(solver_fp64.diagnostics(0), ref.diagnostics(), 1e-12)


@pytest.mark.parametrize("nx,ny,angle", [(70, 27, 90.0), (40, 20, 0.0)])
def test_ragged_sessile_drop_over_steps(solver_fp64, nx, ny, angle):
    c = I.case(nx, ny, radius=0.4 * ny, bo_m=1.5, field_angle_deg=angle, stefan=0.2)
    ref = oracle.Oracle(c, threads=4)
    solver_fp64.set_case(0, c)
    _check(solver_fp64.diagnostics(0), ref.diagnostics(), 1e-12)
    for n in (1, 40, 160):
        ref.step(n)
        solver_fp64.step(n)
        _check(solver_fp64.diagnostics(0), ref.diagnostics(), TOL)


def test_adiabatic_and_periodic_bottom_give_no_wall_flux(solver_fp64):
    for kw in (dict(thermal_dirichlet=(1, 0, 0, 0), wall_T=(-1.0, 0, 0, 0)),
               dict(periodic_y=1, thermal_dirichlet=(0, 0, 0, 0))):
        c = I.case(16, 8, init=2, T_init=1.0, stefan=0.0, latent=10.0, chi_l=0, chi_s=0, **kw)
        solver_fp64.set_case(0, c)
        d, q = solver_fp64.diagnostics(0)
        assert d["Q_wall"] == 0.0 and not q.any()


def test_mixed_precision_diagnostics_track_fp64():
    c = I.config_small()
    out = {}
    for prec in (lbfs.FP64, lbfs.MIXED):
        s = lbfs.Solver(precision=prec, max_cases=1)
        s.set_case(0, c)
        s.step(400)
        out[prec] = s.diagnostics(0)
        s.close()
    _check(out[lbfs.MIXED], out[lbfs.FP64], 1e-4)


@pytest.mark.parametrize("cfg", ["large", "huge"])
@pytest.mark.parametrize("prec", [lbfs.FP64, lbfs.MIXED])
def test_full_size(cfg, prec):
    """the GPU's state after a few steps, evaluated by the oracle in FP64 (the mixed
    state is exported exactly: FP32 values are FP64 numbers)"""
    case = getattr(I, f"config_{cfg}")()
    s = lbfs.Solver(precision=prec, max_cases=1, use_graph=True)
    s.set_case(0, case)
    st = s.step(3)[0]
    got = s.diagnostics(0)
    state = s.fields(0, STATE)
    s.close()
    ref = oracle.Oracle(case)
    ref.set_state(state)
    dr, qr = ref.diagnostics()
    # the oracle's clock was not advanced: take Fo from its definition at the GPU's t
    dr["Fo"] = case["lam_l"] * st["t"] / (case["rho_l"] * case["cp_l"] * case["radius"] ** 2)
    _check(got, (dr, qr), 1e-12)
