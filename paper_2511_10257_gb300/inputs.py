"""Seeded synthetic inputs shared by the CUDA path's tests and the oracle's tests.

This module holds case descriptions (plain numbers), the project's default
lattice-unit parameters, the seeded 64-case sweep, and seeded random state fields.
It contains none of the solver's arithmetic: no equilibria, no enthalpy
inversion, no mixture rule, no initial-condition profile.  Each side (library and
oracle) turns a case description into fields with its own code.

Units are lattice units (dx = 1).  The physical parameters the paper leaves open
(gas properties, interface width, mobility, time steps) take the defaults below;
ratios follow the paper's Table 3 where it gives one (rho_s/rho_l = 1450/1580,
C_p,s/C_p,l = 1670/3000, lambda_s/lambda_l = 2.32/0.72).
"""
from __future__ import annotations

import math

import numpy as np

# field identifiers shared by both sides (bit positions of the library's field mask)
PHI, HE, T, FL, P, U, V, C, MUC, RHO, MX, MY, FSPREV = range(13)
FIELD_NAMES = ["phi", "He", "T", "Fl", "p", "u", "v", "C", "muc", "rho", "mx", "my", "Fs_prev"]

# walls
LEFT, RIGHT, BOTTOM, TOP = range(4)

DEFAULTS = dict(
    periodic_x=0, periodic_y=0,
    thermal_dirichlet=(0, 0, 1, 0),          # cold bottom wall, adiabatic elsewhere
    wall_T=(0.0, 0.0, -1.0, 0.0),
    mag_bc=0,
    init=0,                                  # sessile drop on the bottom wall
    radius=24.0, drop_x=0.0, drop_y=0.0,
    T_init=0.0,
    H0=0.0, field_angle_deg=90.0, bo_m=0.0, stefan=0.1, latent=10.0,
    T_m=0.0,
    rho_l=1.0, rho_g=0.1, rho_s=1450.0 / 1580.0,
    mu_l=0.05, mu_g=0.005, mu_s=0.05,
    cp_l=1.0, cp_g=1.0, cp_s=1670.0 / 3000.0,
    lam_l=0.05, lam_g=0.01, lam_s=0.05 * 2.32 / 0.72,
    chi_l=1.0, chi_g=0.0, chi_s=1.0,
    sigma=0.01, xi=4.0, mobility=0.05, Q_g=1.0, gravity=0.0,
    dt=0.5, dts=0.5,
    contact_angle_deg=90.0,                  # neutral wetting (no-flux phase field)
)


def case(nx: int, ny: int, **kw) -> dict:
    """A full case description: DEFAULTS overridden by keyword arguments."""
    d = dict(DEFAULTS)
    d.update(nx=int(nx), ny=int(ny))
    for k, v in kw.items():
        if k not in d and k not in ("flags",):
            raise KeyError(f"unknown case field {k!r}")
        d[k] = v
    return d


# ---- the five workload configurations ------------------------------------------
def config_small() -> dict:
    """128x64, sessile drop R = 24, vertical field Bo_m = 0.5, chi = 1, Ste = 0.1."""
    return case(128, 64, radius=24.0, field_angle_deg=90.0, bo_m=0.5, chi_l=1.0, chi_s=1.0,
                stefan=0.1)


def config_medium() -> dict:
    """512x256, R = 96, vertical field Bo_m = 1.0, chi = 1, Ste = 0.1."""
    return case(512, 256, radius=96.0, field_angle_deg=90.0, bo_m=1.0, stefan=0.1)


def config_large() -> dict:
    """1024x512, R = 192, horizontal field Bo_m = 1.5, chi = 2, Ste = 0.05."""
    return case(1024, 512, radius=192.0, field_angle_deg=0.0, bo_m=1.5, chi_l=2.0, chi_s=2.0,
                stefan=0.05)


def config_huge() -> dict:
    """4096x2048, R = 768, field at 45 degrees, Bo_m = 1.0, chi = 1."""
    return case(4096, 2048, radius=768.0, field_angle_deg=45.0, bo_m=1.0, stefan=0.1)


class SplitMix64:
    """SplitMix64 (Steele, Lea and Flood 2014): state += 0x9E3779B97F4A7C15, then
    two xor-shift-multiply rounds.  Used for the seeded case sweep."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """uniform in [0, 1) from the top 53 bits"""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def sweep_cases(n: int = 64, seed: int = 0, nx_min: int = 128, nx_max: int = 512,
                nx_step: int = 8) -> list:
    """The seeded batched sweep: grids drawn uniformly from nx_min x nx_min/2 to
    nx_max x nx_max/2 (nx a multiple of nx_step, ny = nx/2), droplet radius 0.375 ny,
    field angle uniform in [0, 90] degrees, Bo_m uniform in [0, 2], Stefan number
    uniform in [0.05, 0.2], chi = 1."""
    rng = SplitMix64(seed)
    choices = list(range(nx_min, nx_max + 1, nx_step))
    out = []
    for _ in range(n):
        nx = choices[min(int(rng.uniform() * len(choices)), len(choices) - 1)]
        ny = nx // 2
        angle = 90.0 * rng.uniform()
        bo = 2.0 * rng.uniform()
        ste = 0.05 + 0.15 * rng.uniform()
        out.append(case(nx, ny, radius=0.375 * ny, field_angle_deg=angle, bo_m=bo, stefan=ste))
    return out


# ---- seeded random states for parity tests --------------------------------------
def _smooth_field(rng: np.random.Generator, nx: int, ny: int, modes: int = 3) -> np.ndarray:
    """sum of a few random low-wavenumber sinusoids, values roughly in [-1, 1]"""
    x = (np.arange(nx) + 0.5)[None, :]
    y = (np.arange(ny) + 0.5)[:, None]
    f = np.zeros((ny, nx))
    for _ in range(modes):
        kx = rng.integers(0, 3) * 2 * math.pi / nx
        ky = rng.integers(0, 3) * 2 * math.pi / ny
        ph = rng.uniform(0, 2 * math.pi)
        f += rng.uniform(0.3, 1.0) * np.cos(kx * x + ky * y + ph)
    return f / modes


def random_state(nx: int, ny: int, seed: int, latent: float = 10.0, amp_u: float = 0.02,
                 noise: float = 0.0) -> dict:
    """A seeded state spanning every branch of the enthalpy inversion: H_e drawn
    around [-0.6, latent + 0.6] (solid, mushy and liquid cells), C a smooth field in
    roughly [-0.05, 1.05] (both sides of 1/2), small p and momentum, a previous
    solid fraction in [0, 1], and a potential near a uniform field.  noise adds
    cell-to-cell white noise of that relative size."""
    rng = np.random.default_rng(seed)
    sm = lambda: _smooth_field(rng, nx, ny)
    wn = lambda: rng.uniform(-1, 1, size=(ny, nx)) if noise > 0 else 0.0
    c_f = 0.5 + 0.55 * sm() + noise * wn()
    he_f = 0.5 * latent + (0.5 * latent + 0.6) * sm() * 1.6 + noise * latent * wn()
    p_f = 0.01 * sm() + 0.01 * noise * wn()
    mx_f = amp_u * sm() + amp_u * noise * wn()
    my_f = amp_u * sm() + amp_u * noise * wn()
    fs_f = np.clip(0.5 + 0.6 * sm(), 0.0, 1.0)
    xs = (np.arange(nx) + 0.5)[None, :]
    ys = (np.arange(ny) + 0.5)[:, None]
    phi_f = -0.01 * (0.3 * xs + 0.7 * ys) + 0.001 * sm()
    return {HE: he_f, P: p_f, MX: mx_f, MY: my_f, C: c_f, FSPREV: fs_f, PHI: phi_f}
