"""Pins of the FP64 oracle's building blocks against what the paper and the
mathematics fix: D2Q9 moment identities (Sec. 3, Eqs. 13-14, 20, 28, 29, A-4),
the enthalpy inversion table (Eq. 8), the mixture rule (Eq. 11) special cases and
the exact reduction of the per-direction LBFS face flux to compact two-point
fluxes at a streaming step of half a cell (Eqs. 16-18, 22-24, 33-35, 44)."""
import math

import numpy as np
import pytest

import oracle
from golden import load as golden
from paper_2511_10257_gb300 import inputs as I

EX = [0, 1, 0, -1, 0, 1, -1, -1, 1]
EY = [0, 0, 1, 0, -1, 1, 1, -1, -1]
CS2 = 1.0 / 3.0


def _moments(vals):
    v = np.asarray(vals)
    ex, ey = np.array(EX, float), np.array(EY, float)
    return (v.sum(), np.array([(ex * v).sum(), (ey * v).sum()]),
            np.array([[(ex * ex * v).sum(), (ex * ey * v).sum()],
                      [(ey * ex * v).sum(), (ey * ey * v).sum()]]))


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_moments(seed):
    """Sec. 3: sum f_eq = p, sum e f_eq = rho c_s^2 u, sum ee f_eq = c_s^2 (p I + rho uu);
    sum g_eq = C, sum e g_eq = C u, sum ee g_eq = mu_c Q_g I; sum h_eq = H_e,
    sum e h_eq = C_p T u, sum ee h_eq = C_p T uu + C_p,ref T c_s^2 I (A-4, whose
    printed form drops the factor T)."""
    rng = np.random.default_rng(seed)
    c = I.case(8, 8, Q_g=rng.uniform(0.5, 2.0))
    p, muc, T = rng.uniform(-1, 1, 3)
    u, v = rng.uniform(-0.1, 0.1, 2)
    C = rng.uniform(0, 1)
    He = rng.uniform(-2, 12)
    rho, cp = rng.uniform(0.1, 1.0, 2)
    fs, gs, hs = zip(*[oracle.equilibria(c, a, p, u, v, C, muc, T, He, rho, cp) for a in range(9)])
    uvec = np.array([u, v])
    m0, m1, m2 = _moments(fs)
    assert m0 == pytest.approx(p, abs=1e-14)
    np.testing.assert_allclose(m1, rho * CS2 * uvec, atol=1e-15)
    np.testing.assert_allclose(m2, CS2 * (p * np.eye(2) + rho * np.outer(uvec, uvec)), atol=1e-15)
    m0, m1, m2 = _moments(gs)
    assert m0 == pytest.approx(C, abs=1e-14)
    np.testing.assert_allclose(m1, C * uvec, atol=1e-15)
    np.testing.assert_allclose(m2, muc * c["Q_g"] * np.eye(2), atol=1e-14)
    cp_ref = 0.5 * (c["cp_s"] + c["cp_l"])
    m0, m1, m2 = _moments(hs)
    assert m0 == pytest.approx(He, abs=1e-13)
    np.testing.assert_allclose(m1, cp * T * uvec, atol=1e-15)
    np.testing.assert_allclose(m2, cp * T * np.outer(uvec, uvec) + cp_ref * T * CS2 * np.eye(2),
                               atol=1e-14)


def test_d2q9_weights_from_equilibrium():
    """With p = 1 and u = 0, f_eq_a equals the weight: 4/9, 1/9 (axis), 1/36 (diagonal)."""
    c = I.case(8, 8)
    w = [oracle.equilibria(c, a, 1.0, 0, 0, 0, 0, 0, 0, 1.0, 1.0)[0] for a in range(9)]
    np.testing.assert_allclose(w, [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4, rtol=0, atol=1e-16)


def test_mixture_special_cases():
    """Eq. 11: fully solid gives the solid value, fully liquid (C = 1) the liquid
    value, gas (C = 0) the gas value, and it is affine in F_s and in C."""
    assert oracle.mix(1.0, 0.3, 7.0, 2.0, 5.0) == 7.0
    assert oracle.mix(0.0, 1.0, 7.0, 2.0, 5.0) == 2.0
    assert oracle.mix(0.0, 0.0, 7.0, 2.0, 5.0) == 5.0
    assert oracle.mix(0.5, 0.5, 7.0, 2.0, 5.0) == pytest.approx(0.5 * 7 + 0.25 * 2 + 0.25 * 5)


# Eq. 8 with T_s = T_l = T_m; values worked out by hand (tests/golden/eq8_inversion.txt)
EQ8_TABLE = [(args, expect) for args, expect, _ in golden.eq8_table()]


def test_eq8_fixture_is_complete():
    assert len(EQ8_TABLE) == 10


@pytest.mark.parametrize("args,expect", EQ8_TABLE)
def test_enthalpy_inversion_table(args, expect):
    T_m, L, cps, cpl, cpg, C, He = args
    c = I.case(8, 8, T_m=T_m, latent=L, stefan=0.0, cp_s=cps, cp_l=cpl, cp_g=cpg)
    T, Fl = oracle.eq8(c, He, C)
    assert T == pytest.approx(expect[0], abs=1e-15)
    assert Fl == pytest.approx(expect[1], abs=1e-15)


def test_enthalpy_inversion_is_continuous_and_monotone():
    """Eq. 8 is continuous in H_e for a droplet cell and T, F_l are non-decreasing."""
    c = I.case(8, 8, latent=10.0, stefan=0.0)
    He = np.linspace(-3, 14, 3401)
    out = np.array([oracle.eq8(c, h, 0.9) for h in He])
    assert np.all(np.diff(out[:, 0]) >= -1e-15) and np.all(np.diff(out[:, 1]) >= -1e-15)
    assert np.max(np.abs(np.diff(out[:, 0]))) < 0.02 and np.max(np.abs(np.diff(out[:, 1]))) < 0.01
    # Stefan number route: L = C_p,l (T_m - T_wall,bottom) / Ste
    c2 = I.case(8, 8, stefan=0.2, wall_T=(0, 0, -1.0, 0))
    T, Fl = oracle.eq8(c2, 2.5, 1.0)   # L = 5 -> half melted
    assert Fl == pytest.approx(0.5, abs=1e-15) and T == 0.0


def _flat_state(nx, ny, T=None, C=None, p=0.0, mx=0.0, my=0.0, **kw):
    c = I.case(nx, ny, init=2, T_init=1.0, stefan=0.0, latent=10.0, chi_l=0, chi_s=0, **kw)
    o = oracle.Oracle(c)
    L = c["latent"]
    if C is None:
        C = np.ones((ny, nx))
    if T is not None:
        cpL = C * c["cp_l"] + (1 - C) * c["cp_g"]
        o.set(I.HE, cpL * T + L)
    o.set(I.C, C)
    o.set(I.P, p)
    o.set(I.MX, mx)
    o.set(I.MY, my)
    return c, o


def test_magnetic_lbfs_flux_is_compact_two_point_at_half_step():
    """Eqs. 13, 16-18, 44, 45: at dts = 1/2 the per-direction magnetic flux equals
    -mu_f (phi_B - phi_A) exactly, so the steady magnetic LBFS is the five-point
    variable-coefficient Laplacian."""
    rng = np.random.default_rng(1)
    nx, ny = 9, 7
    c, o = _flat_state(nx, ny)
    phi = rng.normal(size=(ny, nx))
    o.set(I.PHI, phi)
    for axis in (0, 1):
        for _ in range(10):
            i = int(rng.integers(1, nx)) if axis == 0 else int(rng.integers(0, nx))
            j = int(rng.integers(0, ny)) if axis == 0 else int(rng.integers(1, ny))
            mu = rng.uniform(1, 3)
            a, b = ((j, i - 1), (j, i)) if axis == 0 else ((j - 1, i), (j, i))
            F = o.mag_lbfs_flux(axis, i, j, mu)
            assert F == pytest.approx(-mu * (phi[b] - phi[a]), rel=1e-12, abs=1e-13)


def test_thermal_flux_is_compact_conduction_at_half_step():
    """Eqs. 20-24, 44, 45 with u = 0: the per-direction enthalpy flux is exactly
    -(lambda_f/rho_f)(T_B - T_A) at dts = 1/2 (the C_p,ref T part of h_eq)."""
    rng = np.random.default_rng(2)
    nx, ny = 8, 6
    T = rng.uniform(0.1, 2.0, size=(ny, nx))
    c, o = _flat_state(nx, ny, T=T)
    lam_rho = c["lam_l"] / c["rho_l"]
    for axis in (0, 1):
        for i, j in [(3, 2), (5, 4), (1, 1), (6, 3)]:
            F = o.face_flux(axis, i, j)
            a, b = ((j, i - 1), (j, i)) if axis == 0 else ((j - 1, i), (j, i))
            assert F[0] == pytest.approx(-lam_rho * (T[b] - T[a]), rel=1e-12, abs=1e-14)
            assert abs(F[1]) < 1e-15 and abs(F[4]) < 1e-15   # no mass or phase flux


def test_phase_field_flux_is_compact_diffusion_at_half_step():
    """Eqs. 29, 31-35 with u = 0: the per-direction C flux is -M_c (mu_B - mu_A)."""
    rng = np.random.default_rng(3)
    nx, ny = 10, 8
    C = 0.5 + 0.3 * np.sin(np.arange(nx) / 2.0)[None, :] * np.cos(np.arange(ny) / 3.0)[:, None]
    c, o = _flat_state(nx, ny, T=np.ones((ny, nx)), C=C)
    mu = o.get(I.MUC)
    # mu_c = 2 beta C (C-1)(2C-1) - kappa lap C at an interior cell, by hand
    beta, kappa = 12 * c["sigma"] / c["xi"], 1.5 * c["xi"] * c["sigma"]
    j, i = 4, 5
    lap = C[j, i + 1] + C[j, i - 1] + C[j + 1, i] + C[j - 1, i] - 4 * C[j, i]
    assert mu[j, i] == pytest.approx(2 * beta * C[j, i] * (C[j, i] - 1) * (2 * C[j, i] - 1) - kappa * lap,
                                     rel=1e-13)
    for axis in (0, 1):
        for i, j in [(3, 2), (5, 4), (2, 6), (7, 3)]:
            F = o.face_flux(axis, i, j)
            a, b = ((j, i - 1), (j, i)) if axis == 0 else ((j - 1, i), (j, i))
            assert F[4] == pytest.approx(-c["mobility"] * (mu[b] - mu[a]), rel=1e-11, abs=1e-15)


def test_viscous_flux_linear_regime():
    """Eqs. 28, 30, 32 (with '+'), 34: for a small shear v(x) at uniform p and rho the
    tangential momentum flux is -c_s^2 mu (v_B - v_A), i.e. the viscous stress with
    positive viscosity; the literal '-' sign of Eq. 32 reverses it."""
    nx, ny = 8, 4
    amp = 1e-7
    v = amp * np.sin(2 * np.pi * np.arange(nx) / nx)[None, :] * np.ones((ny, 1))
    c, o = _flat_state(nx, ny, T=np.ones((ny, nx)), my=v * CS2)   # rho = 1
    mu = c["mu_l"]
    for i in (2, 3, 5):
        F = o.face_flux(0, i, 1)
        expect = -CS2 * mu * (v[1, i] - v[1, i - 1])
        assert F[3] == pytest.approx(expect, rel=1e-5)
    c2 = dict(c, flags=oracle.FLAG_LITERAL_FSTAR_SIGN)
    o2 = oracle.Oracle(c2)
    o2.set(I.HE, np.ones((ny, nx)) + c["latent"])
    o2.set(I.MY, v * CS2)
    F = o2.face_flux(0, 3, 1)
    assert np.sign(F[3]) == -np.sign(-CS2 * mu * (v[1, 3] - v[1, 2]))


def test_pressure_flux_is_compatibility_momentum():
    """Eq. 45 + Eq. 43: the p flux through a face is the interface (rho u c_s^2).n,
    which for uniform p and u = 0 vanishes and for a pressure jump at rest is the
    artificial-compressibility term (p_A - p_B)/6 at dts = 1/2."""
    nx, ny = 6, 4
    p = np.zeros((ny, nx))
    p[:, 3:] = 1e-3
    c, o = _flat_state(nx, ny, T=np.ones((ny, nx)), p=p)
    F = o.face_flux(0, 3, 1)
    assert F[1] == pytest.approx((0.0 - 1e-3) / 6.0, rel=1e-12)
    F = o.face_flux(0, 1, 1)
    assert abs(F[1]) < 1e-18


def test_random_states_cover_every_inversion_branch():
    """The seeded parity inputs reach solid, mushy and liquid droplet cells and gas
    cells, and the oracle steps them without producing non-finite values."""
    st = I.random_state(16, 12, seed=3, latent=10.0, noise=0.05)
    c = I.case(16, 12, stefan=0.0, latent=10.0, H0=0.02, radius=4.0)
    o = oracle.Oracle(c)
    o.set_state(st)
    Fl, C = o.get(I.FL), o.get(I.C)
    drop = C >= 0.5
    assert np.any(Fl[drop] == 0.0) and np.any((Fl[drop] > 0) & (Fl[drop] < 1)) and np.any(Fl[drop] == 1.0)
    assert np.any(~drop)
    o.step(3)
    assert o.stats()["nonfinite"] == 0
