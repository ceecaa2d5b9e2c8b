"""Physical-unit front end: Eq. 49 (Maxwell model) special cases and dilute limit,
the ferrofluid latent heat, Eq. 50's groups, and that the SI -> lattice mapping keeps
every dimensionless group of the problem."""
import math

import pytest

from paper_2511_10257_gb300 import units as U
from golden import load as golden


def test_maxwell_special_cases():
    assert U.maxwell(0.6, 7.0, 0.0) == pytest.approx(0.6, rel=1e-15)    # no particles
    assert U.maxwell(0.6, 0.6, 0.3) == pytest.approx(0.6, rel=1e-15)    # n = 1
    assert U.maxwell(0.6, 7.0, 1.0) == pytest.approx(7.0, rel=1e-15)    # all particles
    # dilute limit: slope 3 (n - 1)/(n + 2) at phi = 0
    h, n = 1e-7, 7.0 / 0.6
    slope = (U.maxwell(0.6, 7.0, h) / 0.6 - 1.0) / h
    assert slope == pytest.approx(3 * (n - 1) / (n + 2), rel=1e-5)
    # monotone in phi for n > 1, bounded by the two phases
    vals = [U.maxwell(0.6, 7.0, p / 10) for p in range(11)]
    assert all(b > a for a, b in zip(vals, vals[1:])) and 0.6 <= min(vals) and max(vals) <= 7.0


def test_latent_heat_and_groups():
    assert U.ferrofluid_latent(333000.0, 0.1) == pytest.approx(299700.0)
    assert U.stefan(3000.0, 0.0, -20.0, 300009.0) == pytest.approx(3000 * 20 / 300009.0)
    H = U.field_from_bond(1.5, 2e-3, 0.00307)
    assert U.magnetic_bond(H, 2e-3, 0.00307) == pytest.approx(1.5, rel=1e-14)
    assert U.fourier(0.72, 1580.0, 3000.0, 1e-3, 10.0) == pytest.approx(0.72 * 10 / (1580 * 3000 * 1e-6))


def _si():
    t3 = {r[0]: (float(r[1]), float(r[2])) for r in golden.rows("table3_ferrofluid.txt")}
    return dict(rho_l=t3["rho"][0], rho_s=t3["rho"][1], rho_g=1.2, mu_l=t3["mu"][0], mu_g=1.8e-5,
                cp_l=t3["cp"][0], cp_s=t3["cp"][1], cp_g=1005.0, lam_l=t3["lambda"][0],
                lam_s=t3["lambda"][1], lam_g=0.026, sigma=t3["sigma"][0], L=t3["L"][0],
                T_m=t3["T_m"][0], T_w=-20.0, T_0=0.0, R0=1e-3, chi=1.2, bo_m=1.0, field_angle_deg=0.0)


def test_lattice_mapping_keeps_the_groups():
    si = _si()
    case, sc = U.lattice_case(si, 256, 128, R_cells=48.0, nu_lattice=0.05)
    D, Dl = 2 * si["R0"], 2 * case["radius"]
    # Stefan number (Eq. 50) with the cold wall
    ste = U.stefan(si["cp_l"], si["T_m"], si["T_w"], si["L"])
    assert case["cp_l"] * (case["T_m"] - case["wall_T"][2]) / case["latent"] == pytest.approx(ste, rel=1e-14)
    # Prandtl and Laplace numbers of the liquid, and the viscosity and diffusivity ratios
    pr = lambda mu, cp, lam: mu * cp / lam
    assert pr(case["mu_l"], case["cp_l"], case["lam_l"]) == pytest.approx(pr(si["mu_l"], si["cp_l"], si["lam_l"]),
                                                                          rel=1e-13)
    la = lambda s, r, d, m: s * r * d / (m * m)
    assert la(case["sigma"], case["rho_l"], Dl, case["mu_l"]) == pytest.approx(
        la(si["sigma"], si["rho_l"], D, si["mu_l"]), rel=1e-13)
    for a, b in (("rho_s", "rho_l"), ("rho_g", "rho_l"), ("mu_g", "mu_l"), ("cp_s", "cp_l"),
                 ("cp_g", "cp_l"), ("lam_s", "lam_l"), ("lam_g", "lam_l")):
        assert case[a] / case[b] == pytest.approx(si[a] / si[b], rel=1e-13), a
    # Fourier number at the same physical time
    t = 3.7
    assert U.fourier(case["lam_l"], case["rho_l"], case["cp_l"], case["radius"], t / sc["t0"]) == pytest.approx(
        U.fourier(si["lam_l"], si["rho_l"], si["cp_l"], si["R0"], t), rel=1e-13)
    assert case["bo_m"] == 1.0 and case["chi_l"] == 1.2 and case["mu_l"] == pytest.approx(0.05)
    assert case["T_m"] == 0.0 and case["wall_T"][2] == -1.0 and case["T_init"] == 0.0


def test_field_strength_input_gives_the_same_bond_number():
    si = _si()
    del si["bo_m"]
    si["H"] = U.field_from_bond(0.8, 2 * si["R0"], si["sigma"])
    case, _ = U.lattice_case(si, 64, 32, R_cells=12.0)
    assert case["bo_m"] == pytest.approx(0.8, rel=1e-13)


def test_rejects_a_warm_wall():
    si = _si()
    si["T_w"] = 5.0
    with pytest.raises(ValueError):
        U.lattice_case(si, 64, 32, R_cells=12.0)
