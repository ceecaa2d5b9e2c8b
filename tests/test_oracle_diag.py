"""Pins of the oracle's Sec. 5 diagnostics: the local wall heat flux
Q = -lambda dT/dy at y = 0 (Sec. 5.2, second-order one-sided difference), the
droplet height H_m (Sec. 5.1), the Peclet and Fourier numbers (Eq. 50)."""
import math

import numpy as np
import pytest
from scipy.special import erf

import oracle
from paper_2511_10257_gb300 import inputs as I
from test_oracle_physics import neumann_k

CS2 = 1.0 / 3.0


def _column_case(nx=6, ny=8, **kw):
    args = dict(init=2, T_init=1.0, stefan=0.0, latent=10.0, chi_l=0, chi_s=0)
    args.update(kw)
    return I.case(nx, ny, **args)


def _He_of_T(c, T):
    """H_e of a C = 1 cell at temperature T: solid below T_m, liquid above (Eq. 8)."""
    return np.where(T < c["T_m"], c["cp_s"] * T, c["cp_l"] * T + c["latent"])


@pytest.mark.parametrize("a,b,phase", [(4.0, -0.1, "liquid"), (0.5, 0.05, "solid")])
def test_wall_heat_flux_exact_for_quadratic_profiles(a, b, phase):
    """The one-sided difference through T_w, T(1/2), T(3/2) is exact for a quadratic
    in y, so Q = -lambda a, with the first cell's conductivity."""
    c = _column_case()
    o = oracle.Oracle(c)
    Tw = c["wall_T"][I.BOTTOM]
    y = (np.arange(c["ny"]) + 0.5)[:, None] * np.ones((1, c["nx"]))
    T = Tw + a * y + b * y * y
    o.set(I.HE, _He_of_T(c, T))
    assert np.all(o.get(I.FL)[0] == (1.0 if phase == "liquid" else 0.0))
    d, q = o.diagnostics()
    lam = c["lam_l"] if phase == "liquid" else c["lam_s"]
    np.testing.assert_allclose(q, -lam * a, rtol=1e-13)
    assert d["Q_wall"] == pytest.approx(-lam * a * c["nx"], rel=1e-13)


def test_wall_heat_flux_needs_a_cold_wall():
    c = _column_case(thermal_dirichlet=(1, 0, 0, 0), wall_T=(-1.0, 0, 0, 0))
    d, q = oracle.Oracle(c).diagnostics()
    assert d["Q_wall"] == 0.0 and not q.any()
    c = _column_case(periodic_y=1, thermal_dirichlet=(0, 0, 0, 0))
    d, q = oracle.Oracle(c).diagnostics()
    assert d["Q_wall"] == 0.0 and not q.any()


def test_wall_heat_flux_matches_neumann_solution():
    """Sec. 4.1's conductive freezing turned to run in y (cold bottom wall, warm top,
    periodic x) with a moving front (Ste_s = Ste_l = 0.1, alpha = 0.3).  The solid
    branch of Eq. 47 gives the wall flux Q = -lambda_s (T_m - T_b)/(erf(k) sqrt(pi alpha_s t)).
    The enthalpy method holds the cell that contains the front at T_m, so the
    instantaneous wall slope steps as the front crosses cells (up to half a cell over
    the front distance, ~10 % here); integrated over t = 500..3000, while the front
    crosses seven cells, the oracle's Q is within 1 % of the exact integral."""
    alpha, L, ny = 0.3, 10.0, 200
    Tb, T0, Tm = -1.0, 1.0, 0.0
    c = I.case(1, ny, periodic_x=1, init=2, T_init=T0, stefan=0.0, latent=L, rho_s=1.0,
               cp_s=1.0, cp_l=1.0, lam_s=alpha, lam_l=alpha, chi_l=0, chi_s=0,
               thermal_dirichlet=(0, 0, 1, 1), wall_T=(0.0, 0.0, Tb, T0))
    o = oracle.Oracle(c)
    k = neumann_k((Tm - Tb) / L, (T0 - Tm) / L, alpha, alpha)
    A = alpha * (Tm - Tb) / (erf(k) * math.sqrt(math.pi * alpha))   # |Q| sqrt(t)
    o.step(1000)
    ts, qs = [], []
    for n in range(501):
        if n:
            o.step(10)
        ts.append(o.stats()["t"])
        qs.append(o.diagnostics()[1][0])
    ts, qs = np.array(ts), np.array(qs)
    assert ts[0] == 500.0 and ts[-1] == 3000.0
    assert np.all(qs < 0) and np.all(np.abs(-qs * np.sqrt(ts) / A - 1) < 0.12)
    exact = -A * 2.0 * (math.sqrt(ts[-1]) - math.sqrt(ts[0]))
    assert np.trapezoid(qs, ts) == pytest.approx(exact, rel=0.01)


def test_height_exact_for_linear_columns():
    """C linear in y in each column crosses 1/2 at a known height, and linear
    interpolation between cell centres is exact for it; H_m is the largest."""
    c = _column_case(nx=5, ny=40)
    o = oracle.Oracle(c)
    h = np.array([7.3, 12.55, 30.0, 3.9, 21.25])
    y = (np.arange(c["ny"]) + 0.5)[:, None]
    o.set(I.C, 0.5 - (y - h[None, :]) / 60.0)
    d, _ = o.diagnostics()
    assert d["H_m"] == pytest.approx(30.0, abs=1e-12)
    o.set(I.C, np.ones((c["ny"], c["nx"])))
    assert o.diagnostics()[0]["H_m"] == c["ny"]
    o.set(I.C, np.zeros((c["ny"], c["nx"])))
    assert o.diagnostics()[0]["H_m"] == 0.0


def test_height_of_the_initial_hemisphere_is_its_radius():
    """The initial sessile drop C = 1/2 + 1/2 tanh(2 (R - r)/xi) crosses 1/2 at r = R;
    the column next to the centre has its crossing at sqrt(R^2 - 1/4)."""
    for R in (12.0, 24.0):
        c = I.case(128, 64, radius=R, bo_m=0.0)
        d, _ = oracle.Oracle(c).diagnostics()
        assert d["H_m"] == pytest.approx(math.sqrt(R * R - 0.25), abs=0.02)


def test_speed_and_peclet_over_droplet_cells():
    """U_max is the largest |u| over cells with C >= 1/2 (faster gas cells are ignored);
    Pe = U_max 2 R_0 / alpha_l and Fo = lambda_l t/(rho_l C_p,l R_0^2) (Eq. 50)."""
    c = _column_case(nx=6, ny=6, radius=10.0)
    o = oracle.Oracle(c)
    C = np.ones((6, 6))
    C[5, :] = 0.2                      # a gas row on top
    u = np.zeros((6, 6))
    v = np.zeros((6, 6))
    u[2, 3], v[2, 3] = 3e-3, -4e-3     # speed 5e-3 in the drop
    u[5, 1] = 0.1                      # faster, but gas
    o.set(I.C, C)
    o.set(I.HE, c["cp_l"] * 1.0 + c["latent"])   # liquid, T = 1
    rho = np.where(C >= 0.5, c["rho_l"], C * c["rho_l"] + (1 - C) * c["rho_g"])
    o.set(I.MX, u * rho * CS2)
    o.set(I.MY, v * rho * CS2)
    d, _ = o.diagnostics()
    assert d["U_max"] == pytest.approx(5e-3, rel=1e-13)
    alpha_l = c["lam_l"] / (c["rho_l"] * c["cp_l"])
    assert d["Pe"] == pytest.approx(5e-3 * 20.0 / alpha_l, rel=1e-13)
    assert d["Fo"] == 0.0
    o.step(3)
    d, _ = o.diagnostics()
    assert d["Fo"] == pytest.approx(c["lam_l"] * 3 * c["dt"] / (c["rho_l"] * c["cp_l"] * 100.0),
                                    rel=1e-15)
