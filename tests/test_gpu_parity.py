"""CUDA path (FP64) against the FP64 CPU oracle, element by element: within 1e-9 of
each field's largest magnitude after N steps (random seeded states, every branch of
the enthalpy inversion, ragged tiles, walls and periodic axes, the 128 x 64 case)."""
import numpy as np
import pytest

import oracle
from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

from parity import assert_parity, set_both, compare

pytestmark = pytest.mark.gpu
TOL = 1e-9


@pytest.fixture(scope="module")
def solver_fp64():
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1)
    yield s
    s.close()


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("angle,chi", [(0.0, 0.0), (45.0, 1.0), (90.0, 1.0)])
def test_random_state_8x8(solver_fp64, seed, angle, chi):
    c = I.case(8, 8, radius=3.0, H0=0.02, field_angle_deg=angle, chi_l=chi, chi_s=chi,
               stefan=0.0, latent=10.0, rho_s=0.9, gravity=-1e-4)
    st = I.random_state(8, 8, seed=seed, latent=10.0)
    ref = oracle.Oracle(c)
    solver_fp64.set_case(0, c)
    set_both(solver_fp64, 0, ref, st)
    for n in (1, 5):
        ref.step(n)
        solver_fp64.step(n)
        assert_parity(solver_fp64, 0, ref, TOL)


@pytest.mark.parametrize("nx,ny", [(40, 20), (70, 27)])
def test_ragged_sessile_drop(solver_fp64, nx, ny):
    """several tiles and a ragged tail in both directions"""
    c = I.case(nx, ny, radius=0.4 * ny, bo_m=1.5, field_angle_deg=30.0, stefan=0.2)
    ref = oracle.Oracle(c, threads=4)
    solver_fp64.set_case(0, c)
    for n in (1, 50, 150):
        ref.step(n)
        solver_fp64.step(n)
        assert_parity(solver_fp64, 0, ref, TOL)


def test_periodic_axes_and_insulating_walls(solver_fp64):
    c = I.case(48, 32, periodic_x=1, init=1, radius=8.0, drop_x=20.0, drop_y=14.0, mag_bc=0,
               bo_m=1.0, field_angle_deg=90.0, stefan=0.3, thermal_dirichlet=(0, 0, 1, 1),
               wall_T=(0, 0, -1.0, 0.5))
    ref = oracle.Oracle(c, threads=4)
    solver_fp64.set_case(0, c)
    ref.step(60)
    solver_fp64.step(60)
    assert_parity(solver_fp64, 0, ref, TOL)
    c2 = I.case(48, 32, mag_bc=1, init=1, radius=8.0, drop_x=24.0, drop_y=16.0, bo_m=1.0,
                field_angle_deg=90.0, periodic_y=1, thermal_dirichlet=(1, 0, 0, 0),
                wall_T=(-1.0, 0, 0, 0), stefan=0.0, latent=4.0)
    ref = oracle.Oracle(c2, threads=4)
    solver_fp64.set_case(0, c2)
    ref.step(60)
    solver_fp64.step(60)
    assert_parity(solver_fp64, 0, ref, TOL)


def test_noisy_state_all_walls(solver_fp64):
    """cell-to-cell noise exercises the reconstruction slopes at every face"""
    c = I.case(36, 20, radius=7.0, H0=0.03, field_angle_deg=70.0, chi_l=2.0, chi_s=2.0,
               stefan=0.0, latent=5.0, thermal_dirichlet=(1, 1, 1, 1), wall_T=(-0.5, 0.2, -1.0, 0.3))
    st = I.random_state(36, 20, seed=11, latent=5.0, noise=0.05)
    ref = oracle.Oracle(c)
    solver_fp64.set_case(0, c)
    set_both(solver_fp64, 0, ref, st)
    ref.step(3)
    solver_fp64.step(3)
    assert_parity(solver_fp64, 0, ref, TOL)


def test_potential_solve_matches(solver_fp64):
    c = I.case(64, 32, radius=12.0, bo_m=2.0, field_angle_deg=45.0, chi_l=2.0, chi_s=2.0)
    ref = oracle.Oracle(c)
    solver_fp64.set_case(0, c)
    ref.step(1)
    stats = solver_fp64.step(1)[0]
    assert stats["pot_resid"] <= 1e-13 and stats["pot_cycles"] >= 1
    assert_parity(solver_fp64, 0, ref, 1e-11, fields=[I.PHI])


def test_potential_solve_large_coarsest_level(solver_fp64):
    """a periodic axis that halves to an odd size at once leaves a coarsest level of
    2060 cells, above the one-warp conjugate-gradient limit: the block-wide solve"""
    c = I.case(1030, 8, periodic_x=1, radius=3.0, bo_m=2.0, field_angle_deg=30.0,
               chi_l=2.0, chi_s=2.0)
    ref = oracle.Oracle(c)
    solver_fp64.set_case(0, c)
    ref.step(1)
    stats = solver_fp64.step(1)[0]
    assert stats["pot_resid"] <= 1e-13 and stats["pot_cycles"] >= 1
    assert_parity(solver_fp64, 0, ref, 1e-11, fields=[I.PHI])


@pytest.mark.slow
def test_config_small_2000_steps(solver_fp64):
    """the 128 x 64 sessile-drop case (vertical field, Bo_m = 0.5, chi = 1, Ste = 0.1)"""
    c = I.config_small()
    ref = oracle.Oracle(c, threads=8)
    solver_fp64.set_case(0, c)
    for n in (500, 1500):
        ref.step(n)
        solver_fp64.step(n)
        assert_parity(solver_fp64, 0, ref, TOL)
    st = solver_fp64.step(0)[0]
    ost = ref.stats()
    assert abs(st["Q_L"] - ost["Q_L"]) <= 1e-9
    assert abs(st["sum_C"] - ost["sum_C"]) <= 1e-9 * ost["sum_C"]


def test_stats_match_oracle(solver_fp64):
    c = I.case(48, 24, radius=9.0, bo_m=0.5, stefan=0.5)
    ref = oracle.Oracle(c)
    solver_fp64.set_case(0, c)
    ref.step(40)
    st = solver_fp64.step(40)[0]
    o = ref.stats()
    for k in ("sum_C", "sum_He", "sum_Fl_drop", "n_drop", "Q_L", "t"):
        assert st[k] == pytest.approx(o[k], rel=1e-10, abs=1e-12), k
    assert solver_fp64.last_launch_count() > 40 * 4
