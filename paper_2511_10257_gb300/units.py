"""Physical-unit front end: the paper's SI properties (Tables 2 and 3) to a lattice-unit
case description for the solver, the Maxwell model of the ferrofluid's effective
properties (Eq. 49), its latent heat, and the dimensionless groups of Eq. 50.

The mapping keeps every dimensionless group of the SI problem: the unit of length is
the cell (dx = R_0 / R_cells), the unit of density the liquid density, the unit of
heat capacity the liquid's, temperatures are measured from T_m in units of T_m - T_w
(so T_m = 0 and the cold wall at -1), and the unit of time follows from the lattice
kinematic viscosity nu_lattice chosen for the liquid.  Numerical parameters the paper
does not fix (interface width xi, mobility, Q_g, time steps) keep the lattice
defaults of inputs.DEFAULTS.  Host arithmetic only; no device code.
"""
from __future__ import annotations

import math

from . import inputs

MU0 = 4e-7 * math.pi   # vacuum permeability, H/m


def maxwell(omega_l: float, omega_f: float, phi: float) -> float:
    """Eq. 49: effective property of a suspension of particles (property omega_f,
    volume fraction phi) in a continuous phase (omega_l):
    omega_e / omega_l = 1 + 3 (n - 1) phi / ((n + 2) - (n - 1) phi), n = omega_f / omega_l."""
    n = omega_f / omega_l
    return omega_l * (1.0 + 3.0 * (n - 1.0) * phi / ((n + 2.0) - (n - 1.0) * phi))


def ferrofluid_latent(L_w: float, phi: float) -> float:
    """Latent heat of the ferrofluid, L_f = (1 - phi) L_w (Sec. 5)."""
    return (1.0 - phi) * L_w


def stefan(cp_l: float, T_m: float, T_w: float, L: float) -> float:
    """Eq. 50: Ste = C_p,l (T_m - T_w) / L."""
    return cp_l * (T_m - T_w) / L


def fourier(lam_l: float, rho_l: float, cp_l: float, R0: float, t: float) -> float:
    """Eq. 50: Fo = lambda_l t / (rho_l C_p,l R_0^2)."""
    return lam_l * t / (rho_l * cp_l * R0 * R0)


def magnetic_bond(H: float, D: float, sigma: float, mu0: float = MU0) -> float:
    """Eq. 50: Bo_m = mu_0 H^2 D / sigma, D the droplet diameter."""
    return mu0 * H * H * D / sigma


def field_from_bond(bo_m: float, D: float, sigma: float, mu0: float = MU0) -> float:
    """The field strength H of a magnetic Bond number (Eq. 50 solved for H)."""
    return math.sqrt(bo_m * sigma / (mu0 * D))


# Table 3 (Sec. 5): the water-based ferrofluid droplet, SI units
TABLE3 = dict(mu_l=0.016, sigma=0.00307, rho_l=1580.0, rho_s=1450.0, cp_l=3000.0, cp_s=1670.0,
              lam_l=0.72, lam_s=2.32, L=300009.0, T_m=0.0)


def lattice_case(si: dict, nx: int, ny: int, R_cells: float, nu_lattice: float = 0.05, **overrides):
    """A solver case (inputs.case) and the unit scales for an SI problem.

    si holds: rho_l, rho_s, rho_g, mu_l, mu_g (mu_s defaults to mu_l), cp_l, cp_s, cp_g,
    lam_l, lam_s, lam_g, sigma, L, T_m, T_w, T_0 (initial temperature), R0 (m), chi (the
    droplet's susceptibility, e.g. mu_m - 1 from Table 2), and either bo_m or H (A/m),
    plus field_angle_deg.  Returns (case, scales) with scales = dict(dx, t0, rho0, cp0,
    dT): SI length = dx * lattice length, SI time = t0 * lattice time.
    """
    R0 = float(si["R0"])
    dx = R0 / float(R_cells)
    rho0, cp0 = float(si["rho_l"]), float(si["cp_l"])
    nu_l = si["mu_l"] / si["rho_l"]
    t0 = nu_lattice * dx * dx / nu_l
    dT = float(si["T_m"] - si["T_w"])
    if dT <= 0.0:
        raise ValueError("the cold wall must be below the melting temperature")
    mu_unit = rho0 * dx * dx / t0
    lam_unit = rho0 * cp0 * dx * dx / t0
    sigma_unit = rho0 * dx ** 3 / t0 ** 2
    if "bo_m" in si:
        bo_m = float(si["bo_m"])
    else:
        bo_m = magnetic_bond(float(si["H"]), 2.0 * R0, float(si["sigma"]))
    mu_s = si.get("mu_s", si["mu_l"])
    chi = float(si.get("chi", 0.0))
    kw = dict(
        radius=float(R_cells),
        rho_l=1.0, rho_s=si["rho_s"] / rho0, rho_g=si["rho_g"] / rho0,
        mu_l=si["mu_l"] / mu_unit, mu_s=mu_s / mu_unit, mu_g=si["mu_g"] / mu_unit,
        cp_l=1.0, cp_s=si["cp_s"] / cp0, cp_g=si["cp_g"] / cp0,
        lam_l=si["lam_l"] / lam_unit, lam_s=si["lam_s"] / lam_unit, lam_g=si["lam_g"] / lam_unit,
        sigma=si["sigma"] / sigma_unit,
        stefan=0.0, latent=si["L"] / (cp0 * dT),
        T_m=0.0, T_init=(si["T_0"] - si["T_m"]) / dT,
        wall_T=(0.0, 0.0, -1.0, 0.0),
        bo_m=bo_m, chi_l=chi, chi_s=chi, chi_g=0.0,
        field_angle_deg=float(si.get("field_angle_deg", 90.0)),
    )
    kw.update(overrides)
    case = inputs.case(nx, ny, **kw)
    return case, dict(dx=dx, t0=t0, rho0=rho0, cp0=cp0, dT=dT)
