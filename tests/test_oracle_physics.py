"""Physics pins of the FP64 oracle: what the paper's benchmarks and the mathematics
fix for the full time step (Table 1), independent of any implementation.

- energy and phase-field mass conservation (flux form of Eq. 42)
- solid held at rest (F_IBM and the rest reading of Eq. 9)
- conductive freezing against the two-phase Neumann solution (Sec. 4.1, Eqs. 47-48)
- shear-wave decay (viscous term of Eq. 34 with the corrected sign of Eq. 32)
- Laplace law for a free 2-D drop (surface tension F_surf = -C grad mu_c)
- circular inclusion in a uniform field (Eq. 4 with a susceptibility jump)
- the paper's pseudo-time magnetic LBFS (Eqs. 12-18) converging to the direct solve
- mirror symmetry and 1-D reduction of the whole step
"""
import math

import numpy as np
import pytest
from scipy.special import erf, erfc
from scipy.optimize import brentq

import oracle
from golden import load as golden
from paper_2511_10257_gb300 import inputs as I

CS2 = 1.0 / 3.0


def test_energy_conservation_adiabatic():
    """u = 0 (single phase, chi = 0, rho_s = rho_l), adiabatic walls, an internal hot and
    a cold region so that cells freeze and melt: sum H_e is constant to round-off."""
    nx, ny = 24, 16
    c = I.case(nx, ny, init=2, stefan=0.0, latent=2.0, chi_l=0, chi_s=0, rho_s=1.0,
               thermal_dirichlet=(0, 0, 0, 0), T_init=0.0)
    o = oracle.Oracle(c)
    x = (np.arange(nx) + 0.5)[None, :]
    y = (np.arange(ny) + 0.5)[:, None]
    He = 1.0 + 1.8 * np.sin(2 * np.pi * x / nx) * np.cos(np.pi * y / ny)
    o.set(I.HE, He)
    s0 = o.stats()["sum_He"]
    o.step(300)
    st = o.stats()
    assert abs(st["sum_He"] - s0) <= 1e-12 * abs(s0)
    assert np.all(o.get(I.U) == 0.0) and np.all(o.get(I.V) == 0.0)
    Fl = o.get(I.FL)
    assert Fl.min() < 0.5 and Fl.max() == 1.0   # both phases present


def test_phase_field_mass_conservation_with_flow_and_field():
    """rho_s = rho_l (no volume-change source), no-flux walls, cooling, magnetic field
    and surface tension on: sum C is constant to round-off."""
    c = I.case(48, 24, radius=9.0, bo_m=1.0, field_angle_deg=60.0, rho_s=1.0, stefan=0.1)
    o = oracle.Oracle(c)
    s0 = o.stats()["sum_C"]
    o.step(60)
    st = o.stats()
    assert st["nonfinite"] == 0
    assert abs(st["sum_C"] - s0) <= 1e-12 * s0
    assert np.max(np.abs(o.get(I.U))) > 1e-6      # the field does drive a flow
    assert st["Q_L"] > 0.0                       # and freezing has started


def test_solid_is_at_rest():
    """Wherever F_s = 1 the velocity is exactly zero (rest reading of Eq. 9)."""
    c = I.case(32, 16, radius=10.0, bo_m=2.0, field_angle_deg=90.0, stefan=1.0)
    o = oracle.Oracle(c)
    o.step(120)
    Fl = o.get(I.FL)
    solid = Fl == 0.0
    assert solid.sum() > 10
    assert np.all(o.get(I.U)[solid] == 0.0) and np.all(o.get(I.V)[solid] == 0.0)
    assert np.max(np.abs(o.get(I.U)[Fl == 1.0])) > 0.0


def neumann_k(St_s, St_l, a_s, a_l):
    """root of St_s e^{-k^2}/erf k - St_l sqrt(a_l/a_s) e^{-k^2 a_s/a_l}/erfc(k sqrt(a_s/a_l)) = k sqrt(pi),
    the Stefan condition of the two-phase Neumann problem (Carslaw and Jaeger)"""
    r = math.sqrt(a_s / a_l)
    f = lambda k: (St_s * math.exp(-k * k) / erf(k)
                   - St_l / r * math.exp(-k * k * r * r) / erfc(k * r) - k * math.sqrt(math.pi))
    return brentq(f, 1e-6, 3.0, xtol=1e-15)


def neumann_T(x, t, k, Tb, T0, Tm, a_s, a_l):
    X = 2 * k * math.sqrt(a_s * t)
    sol = Tb + (Tm - Tb) * erf(x / (2 * np.sqrt(a_s * t))) / erf(k)
    liq = T0 - (T0 - Tm) * erfc(x / (2 * np.sqrt(a_l * t))) / erfc(k * math.sqrt(a_s / a_l))
    return np.where(x < X, sol, liq), X


def _conduction_case(nx, alpha, L):
    return I.case(nx, 1, periodic_y=1, init=2, T_init=1.0, stefan=0.0, latent=L,
                  rho_s=1.0, cp_s=1.0, cp_l=1.0, lam_s=alpha, lam_l=alpha, chi_l=0, chi_s=0,
                  thermal_dirichlet=(1, 1, 0, 0), wall_T=(-1.0, 1.0, 0.0, 0.0))


def test_neumann_moving_front():
    """Sec. 4.1 with a moving front: Ste_s = Ste_l = 0.1 (L = 10), alpha = 0.3.  The
    front position X = sum F_s stays within a quarter cell of 2 k sqrt(alpha t); the
    mean temperature error is below 2e-3.  Pointwise, the enthalpy method holds the
    cell that contains the front at T_m, so the largest error is of the order of the
    solid gradient times half a cell (below 4e-2 here)."""
    alpha, L, nx = 0.3, 10.0, 200
    c = _conduction_case(nx, alpha, L)
    o = oracle.Oracle(c)
    k = neumann_k(1.0 / L, 1.0 / L, alpha, alpha)
    assert 0.18 < k < 0.2
    x = np.arange(nx) + 0.5
    for t_end in (1000.0, 2000.0, 3000.0):
        o.step(int(round((t_end - o.stats()["t"]) / c["dt"])))
        T_exact, X = neumann_T(x, t_end, k, -1.0, 1.0, 0.0, alpha, alpha)
        T = o.get(I.T)[0]
        Xs = np.sum(1.0 - o.get(I.FL)[0])
        assert abs(Xs - X) < 0.25, (t_end, Xs, X)
        err = np.abs(T - T_exact)
        assert err.mean() < 2e-3 and err.max() < 4e-2


def test_neumann_paper_parameters():
    """Sec. 4.1's set (tests/golden/neumann_sec41.txt): alpha = 0.4, L = 250, T_b = -1,
    T_0 = 1, T_m = 0, on a lattice with 20 cells per unit length, compared at the
    paper's t = 5, 10, 15: front position within 0.15 cell, liquid profile within 5e-3,
    mean error below 1e-3."""
    g = golden.keyed("neumann_sec41.txt")
    assert g["rho_l"] == g["rho_s"] == 1.0 and g["cp_l"] == g["cp_s"] == 1.0
    assert g["alpha_s"] == g["alpha_l"]
    alpha, L, Tb, T0, Tm = g["alpha_s"], g["L"], g["T_b"], g["T_0"], g["T_m"]
    nx, s = 240, 20.0
    c = _conduction_case(nx, alpha, L)
    assert c["wall_T"][0] == Tb and c["T_init"] == T0 and c["T_m"] == Tm
    o = oracle.Oracle(c)
    k = neumann_k((Tm - Tb) / L, (T0 - Tm) / L, alpha, alpha)
    assert k == pytest.approx(g["k"], abs=1e-5)
    x = np.arange(nx) + 0.5
    for t_paper in g["times"]:
        t_lat = t_paper * s * s
        o.step(int(round((t_lat - o.stats()["t"]) / c["dt"])))
        T_exact, X = neumann_T(x, t_lat, k, Tb, T0, Tm, alpha, alpha)
        T = o.get(I.T)[0]
        Xs = np.sum(1.0 - o.get(I.FL)[0])
        err = np.abs(T - T_exact)
        assert abs(Xs - X) < 0.15
        assert err[x > X + 1].max() < 5e-3 and err.mean() < 1e-3


def test_default_ratios_follow_table3():
    """The lattice defaults take the solid/liquid ratios of Table 3
    (tests/golden/table3_ferrofluid.txt) for density, heat capacity and conductivity."""
    t = {r[0]: (float(r[1]), float(r[2])) for r in golden.rows("table3_ferrofluid.txt")}
    d = I.DEFAULTS
    assert d["rho_s"] / d["rho_l"] == pytest.approx(t["rho"][1] / t["rho"][0], rel=1e-15)
    assert d["cp_s"] / d["cp_l"] == pytest.approx(t["cp"][1] / t["cp"][0], rel=1e-15)
    assert d["lam_s"] / d["lam_l"] == pytest.approx(t["lambda"][1] / t["lambda"][0], rel=1e-15)


def _shear_wave(flags=0, steps=2000):
    N = 64
    c = I.case(4, N, periodic_x=1, periodic_y=1, init=2, T_init=1.0, chi_l=0, chi_s=0,
               thermal_dirichlet=(0, 0, 0, 0), stefan=0.0, latent=10.0, flags=flags)
    o = oracle.Oracle(c)
    U = 1e-3
    y = (np.arange(N) + 0.5)[:, None] * np.ones((1, 4))
    o.set(I.MX, U * np.sin(2 * np.pi * y / N) * CS2)   # rho = 1
    o.step(steps)
    u = o.get(I.U)[:, 0]
    amp = 2.0 / N * np.sum(u * np.sin(2 * np.pi * (np.arange(N) + 0.5) / N))
    nu = c["mu_l"] / c["rho_l"]
    expect = U * math.exp(-nu * (2 * np.pi / N) ** 2 * steps * c["dt"])
    return amp, expect


def test_shear_wave_decay():
    """Viscous decay of u_x = U sin(2 pi y / N): amplitude exp(-nu k^2 t) within 1 %."""
    amp, expect = _shear_wave()
    assert amp == pytest.approx(expect, rel=1e-2)


def test_shear_wave_catches_literal_fstar_sign():
    """With the printed '-' of Eq. 32 the viscosity is negative and the wave grows."""
    amp, expect = _shear_wave(flags=oracle.FLAG_LITERAL_FSTAR_SIGN, steps=400)
    assert not (abs(amp - expect) <= 1e-2 * expect)
    assert amp > 1e-3


def _laplace_run(R, n=64, steps=1500, flags=0):
    c = I.case(n, n, periodic_x=1, periodic_y=1, init=1, radius=R, drop_x=n / 2, drop_y=n / 2,
               T_init=1.0, chi_l=0, chi_s=0, thermal_dirichlet=(0, 0, 0, 0), flags=flags)
    o = oracle.Oracle(c, threads=4)
    o.step(steps)
    P = o.get(I.P) + o.get(I.C) * o.get(I.MUC)
    Rm = math.sqrt(o.stats()["sum_C"] / math.pi)
    return P[n // 2, n // 2] - P[2, 2], Rm, o


@pytest.mark.slow
def test_laplace_law():
    """Free 2-D drops: the jump of p + C mu_c across the interface is sigma / R, so a
    linear fit against 1/R has slope sigma within 5 %."""
    rows = [_laplace_run(R) for R in (8.0, 11.0, 14.0)]
    dP = np.array([r[0] for r in rows])
    invR = np.array([1.0 / r[1] for r in rows])
    slope, icpt = np.polyfit(invR, dP, 1)
    sigma = I.DEFAULTS["sigma"]
    assert slope == pytest.approx(sigma, rel=0.05)
    assert abs(icpt) < 0.1 * sigma / 8.0


def test_literal_muc_sign_breaks_the_interface():
    """With the printed '+kappa lap C' the Cahn-Hilliard equation is anti-diffusive: the
    drop does not keep a bounded smooth interface."""
    c = I.case(32, 32, periodic_x=1, periodic_y=1, init=1, radius=8.0, drop_x=16, drop_y=16,
               T_init=1.0, chi_l=0, chi_s=0, thermal_dirichlet=(0, 0, 0, 0),
               flags=oracle.FLAG_LITERAL_MUC_SIGN)
    o = oracle.Oracle(c)
    o.step(200)
    C = o.get(I.C)
    good = oracle.Oracle(dict(c, flags=0))
    good.step(200)
    Cg = good.get(I.C)
    assert Cg.max() < 1.05 and Cg.min() > -0.05
    assert not (np.all(np.isfinite(C)) and C.max() < 1.05 and C.min() > -0.05)


def test_circular_inclusion_field():
    """A diffuse disk of susceptibility chi in a uniform far field: the interior field
    is uniform with |H_in| = 2 H0 / (2 + chi) (cylinder, demagnetising factor 1/2).
    The interface width (xi = 4 at R = 20) and the walls at 6.4 R shift the sharp-
    interface value by about 1.8 % per unit chi, so the bound is 2 % x chi."""
    n, R = 256, 20.0
    for chi in (1.0, 2.0):
        c = I.case(n, n, init=1, radius=R, drop_x=n / 2, drop_y=n / 2, T_init=1.0,
                   H0=0.01, bo_m=0.0, field_angle_deg=30.0, chi_l=chi, chi_s=chi, chi_g=0.0)
        o = oracle.Oracle(c)
        assert o.solve_potential() == 0
        phi = o.get(I.PHI)
        m = n // 2
        Hx = -(phi[m - 8:m + 8, m - 7:m + 9] - phi[m - 8:m + 8, m - 9:m + 7]) / 2
        Hy = -(phi[m - 7:m + 9, m - 8:m + 8] - phi[m - 9:m + 7, m - 8:m + 8]) / 2
        H = np.hypot(Hx, Hy)
        assert H.mean() == pytest.approx(2 * 0.01 / (2 + chi), rel=0.02 * chi)
        assert H.std() < 0.01 * H.mean()
        ang = math.degrees(math.atan2(Hy.mean(), Hx.mean()))
        assert ang == pytest.approx(30.0, abs=0.5)


def test_uniform_permeability_gives_exact_uniform_field():
    """Uniform chi: the potential is the exact linear far field to round-off."""
    c = I.case(20, 12, init=2, T_init=1.0, H0=0.02, field_angle_deg=35.0, chi_l=1.5, chi_s=1.5)
    o = oracle.Oracle(c)
    o.set(I.PHI, np.zeros((12, 20)))
    assert o.solve_potential() == 0
    x = (np.arange(20) + 0.5)[None, :]
    y = (np.arange(12) + 0.5)[:, None]
    t = math.radians(35.0)
    exact = -0.02 * (x * math.cos(t) + y * math.sin(t))
    np.testing.assert_allclose(o.get(I.PHI), exact, atol=1e-14, rtol=0)


def test_pseudo_time_magnetic_lbfs_reaches_direct_solution():
    """Integrating Eq. 17 with the per-direction LBFS flux (Eqs. 13, 16, 44, 45) in
    pseudo time converges to the potential of the direct steady solve."""
    c = I.case(8, 8, init=1, radius=2.5, drop_x=4.0, drop_y=4.0, T_init=1.0, H0=0.05,
               field_angle_deg=20.0, chi_l=2.0, chi_s=2.0)
    a = oracle.Oracle(c)
    assert a.solve_potential() == 0
    direct = a.get(I.PHI)
    b = oracle.Oracle(c)
    b.pseudo_time_potential(3000, 0.05)
    np.testing.assert_allclose(b.get(I.PHI), direct, atol=1e-11, rtol=0)


def test_mirror_symmetry_vertical_field():
    """Centred sessile drop, vertical field: the step is mirror-symmetric in x."""
    c = I.case(32, 16, radius=9.0, bo_m=2.0, field_angle_deg=90.0, stefan=0.2)
    o = oracle.Oracle(c)
    o.step(40)
    for f, sgn in ((I.C, 1), (I.HE, 1), (I.P, 1), (I.U, -1), (I.V, 1), (I.PHI, 1)):
        a = o.get(f)
        scale = max(np.max(np.abs(a)), 1e-30)
        assert np.max(np.abs(a - sgn * a[:, ::-1])) <= 1e-12 * scale, I.FIELD_NAMES[f]


def test_one_dimensional_reduction():
    """y-uniform initial data with periodic y stays y-uniform to round-off."""
    nx, ny = 24, 6
    c = I.case(nx, ny, periodic_y=1, init=2, T_init=0.5, stefan=0.5, chi_l=0, chi_s=0,
               thermal_dirichlet=(1, 0, 0, 0), wall_T=(-1.0, 0.0, 0.0, 0.0))
    o = oracle.Oracle(c)
    xs = np.arange(nx) + 0.5
    C = (0.5 + 0.5 * np.tanh((12 - xs) / 2.0))[None, :] * np.ones((ny, 1))
    o.set(I.C, C)
    o.set(I.MX, (1e-3 * np.sin(xs / 3.0))[None, :] * np.ones((ny, 1)))
    o.step(50)
    for f in (I.C, I.HE, I.P, I.U, I.V):
        a = o.get(f)
        assert np.max(np.abs(a - a[:1, :])) <= 1e-13 * max(np.max(np.abs(a)), 1e-30)
    assert np.max(np.abs(o.get(I.V))) <= 1e-18


def _aspect(o, n):
    """a/b of the drop from second moments of C (an ellipse has I_aa / I_bb = (a/b)^2)"""
    Cf = np.clip(o.get(I.C), 0.0, 1.0)
    x = np.arange(n) + 0.5
    X, Y = np.meshgrid(x, x)
    cx, cy = (Cf * X).sum() / Cf.sum(), (Cf * Y).sum() / Cf.sum()
    return math.sqrt((Cf * (X - cx) ** 2).sum() / (Cf * (Y - cy) ** 2).sum())


@pytest.mark.slow
def test_ferrofluid_drop_small_deformation():
    """Sec. 4.3: a free ferrofluid drop (chi = 2) in a uniform field along x elongates
    along the field.  Minimising surface plus magnetic co-energy for an ellipse with
    demagnetising factor b/(a+b) gives, to first order in Bo_m (diameter-based),
    a/b - 1 = chi^2 Bo_m / (3 (2 + chi)^2).  The overdamped approach to the steady
    shape is extrapolated (Aitken) from the last three samples; within 5 %."""
    n, R, chi, bo = 64, 10.0, 2.0, 1.0
    c = I.case(n, n, init=1, radius=R, drop_x=n / 2, drop_y=n / 2, T_init=1.0, bo_m=bo,
               field_angle_deg=0.0, chi_l=chi, chi_s=chi, thermal_dirichlet=(0, 0, 0, 0),
               mu_l=0.3, mu_s=0.3, mu_g=0.03)
    o = oracle.Oracle(c, threads=4)
    vals = []
    for _ in range(10):
        o.step(200)
        vals.append(_aspect(o, n) - 1.0)
    a, b, cc = vals[-3:]
    d1, d2 = b - a, cc - b
    assert d1 > 0 and 0 < d2 < d1
    steady = cc + d2 * d2 / (d1 - d2)
    expect = chi * chi * bo / (3.0 * (2.0 + chi) ** 2)
    assert steady == pytest.approx(expect, rel=0.05)


def _dense_potential(c, C):
    """Eq. 4 on the five-point stencil assembled as a dense matrix and solved directly:
    face coefficient the mean of the two cells' mu_m = 1 + chi(C) (all liquid or gas,
    F_s = 0), a Dirichlet wall holding the far field phi_w = -H0 (x cos a + y sin a) at
    the wall face half a cell from the centre, an insulating wall carrying no flux."""
    ny, nx = C.shape
    mu = 1.0 + (c["chi_g"] + C * (c["chi_l"] - c["chi_g"]))
    a = math.radians(c["field_angle_deg"])
    far = lambda x, y: -c["H0"] * (x * math.cos(a) + y * math.sin(a))
    n = nx * ny
    A = np.zeros((n, n))
    b = np.zeros(n)
    for j in range(ny):
        for i in range(nx):
            k = j * nx + i
            for di, dj, wall in ((-1, 0, 0), (1, 0, 1), (0, -1, 2), (0, 1, 3)):
                ii, jj = i + di, j + dj
                periodic = c["periodic_x"] if di else c["periodic_y"]
                if 0 <= ii < nx and 0 <= jj < ny or periodic:
                    ii, jj = ii % nx, jj % ny
                    mf = 0.5 * (mu[j, i] + mu[jj, ii])
                    A[k, k] += mf
                    A[k, jj * nx + ii] -= mf
                elif not (c["mag_bc"] == 1 and wall < 2):
                    x = 0.0 if wall == 0 else (nx if wall == 1 else i + 0.5)
                    y = 0.0 if wall == 2 else (ny if wall == 3 else j + 0.5)
                    A[k, k] += 2.0 * mu[j, i]
                    b[k] += 2.0 * mu[j, i] * far(x, y)
    return np.linalg.solve(A, b).reshape(ny, nx)


@pytest.mark.parametrize("kw", [dict(), dict(mag_bc=1, field_angle_deg=90.0), dict(periodic_x=1),
                                dict(field_angle_deg=0.0)])
def test_potential_matches_dense_solve(kw):
    """the oracle's iterative potential solve against a dense direct solve of Eq. 4 on a
    12x10 grid with a smooth random C (chi_l = 2), to 1e-11 of the field's scale"""
    args = dict(init=2, T_init=1.0, stefan=0.0, latent=10.0, chi_l=2.0, chi_s=2.0, chi_g=0.0,
                H0=0.05, bo_m=0.0, field_angle_deg=30.0)
    args.update(kw)
    c = I.case(12, 10, **args)
    o = oracle.Oracle(c)
    rng = np.random.default_rng(3)
    X, Y = np.meshgrid(np.arange(12) + 0.5, np.arange(10) + 0.5)
    C = np.clip(0.5 + 0.6 * np.sin(0.5 * X + rng.uniform(0, 6)) * np.cos(0.4 * Y + rng.uniform(0, 6)), 0, 1)
    o.set(I.C, C)
    cp = C * c["cp_l"] + (1 - C) * c["cp_g"]
    o.set(I.HE, cp * 1.0 + c["latent"])       # T = 1 everywhere: no solid, F_s = 0
    assert np.all(o.get(I.FL) == 1.0)
    assert o.solve_potential() == 0
    phi = o.get(I.PHI)
    ref = _dense_potential(c, C)
    assert np.max(np.abs(phi - ref)) <= 1e-11 * np.max(np.abs(ref))


@pytest.mark.parametrize("angle,N", [(0.0, 1.0 / 3.0), (90.0, 2.0 / 3.0)])
def test_elliptic_inclusion_field(angle, N):
    """A diffuse elliptic cylinder (semi-axes a = 30 along x, b = 15 along y) of
    susceptibility chi = 1 in a uniform far field along a principal axis: the interior
    field is uniform, |H_in| = H0 / (1 + chi N) with the demagnetising factor
    N = b/(a + b) along x and a/(a + b) along y.  Diffuse-interface bound as for the disk."""
    n, a, b, chi, H0 = 256, 30.0, 15.0, 1.0, 0.01
    c = I.case(n, n, init=2, T_init=1.0, stefan=0.0, latent=10.0, H0=H0, bo_m=0.0, field_angle_deg=angle,
               chi_l=chi, chi_s=chi, chi_g=0.0)
    o = oracle.Oracle(c)
    X, Y = np.meshgrid(np.arange(n) + 0.5 - n / 2, np.arange(n) + 0.5 - n / 2)
    g = np.sqrt((X / a) ** 2 + (Y / b) ** 2)
    grad = np.sqrt((X / a ** 2) ** 2 + (Y / b ** 2) ** 2) / np.maximum(g, 1e-12)
    d = (1.0 - g) / np.maximum(grad, 1e-12)          # signed distance to the ellipse, first order
    o.set(I.C, 0.5 + 0.5 * np.tanh(2.0 * d / c["xi"]))
    assert o.solve_potential() == 0
    phi = o.get(I.PHI)
    m = n // 2
    Hx = -(phi[m - 4:m + 4, m - 7:m + 9] - phi[m - 4:m + 4, m - 9:m + 7]) / 2
    Hy = -(phi[m - 3:m + 5, m - 8:m + 8] - phi[m - 5:m + 3, m - 8:m + 8]) / 2
    H = np.hypot(Hx, Hy)
    assert H.mean() == pytest.approx(H0 / (1.0 + chi * N), rel=0.03)
    assert H.std() < 0.01 * H.mean()
