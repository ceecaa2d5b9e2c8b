"""Pins of the oracle's source terms and wall shear against closed forms.

The volume-change sources of the phase field and the pressure (Eqs. 9, 10 and 41),
the immersed-boundary force F_IBM, gravity F_g = rho g, and the wall shear
-c_s^2 mu du_t/dn of the no-slip walls.  Each pin is a result that the mathematics
fixes independently of the oracle's code:

- a uniform state in a periodic box has no flux divergence, so every cell follows
  the ordinary differential equations of the sources alone; a third-order
  Runge-Kutta step of a linear autonomous system reproduces its Taylor polynomial
  of degree three exactly;
- a uniform fluid under gravity in a periodic box falls freely, v = g t;
- gravity along two no-slip walls drives plane Poiseuille flow, whose steady
  profile for the second-order finite-volume scheme with the wall half a cell
  from the first centre is the parabola rho g x (W - x) / (2 mu) plus the constant
  rho g / (8 mu).

Every pin is shown to fail when the oracle carries a planted mistake in the term
it pins (the ORACLE_FLAG_PLANT_* switches).
"""
import numpy as np
import pytest

import oracle
from paper_2511_10257_gb300 import inputs as I

CS2 = 1.0 / 3.0


def P3(z):
    """degree-three Taylor polynomial of exp(z)"""
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0


def _uniform_freezing(flags=0, C0=0.9):
    """One step of a uniform mushy state in a periodic box: returns the fields after
    the step and the closed forms.  T_m = 0, so F_l = H_e / L for C >= 1/2 and H_e,
    hence F_s, stay constant over the step (no flux divergence, C_p T div u = 0).

    The lagged rate dF_s/dt = S is held over the step.  With a = (1 - rho_s/rho_l) S:
      C' = a C                         ->  C^1 = C0 P3(a dt)
      p' = c_s^2 a rho(C),  rho(C) = a0 + a1 C (Eq. 11 at fixed F_s)
                                       ->  p^1 = p0 + c_s^2 a a0 dt + c_s^2 a1 C0 (P3(a dt) - 1)
      m' = c_s^2 F_IBM = -S m          ->  m^1 = F_l m0 P3(-S dt)   (the step-end rest rule)
    """
    L = 2.0
    c = I.case(4, 4, periodic_x=1, periodic_y=1, init=2, stefan=0.0, latent=L, chi_l=0, chi_s=0,
               thermal_dirichlet=(0, 0, 0, 0), flags=flags)
    He, Fs_prev, p0, mx0, my0 = 0.8, 0.5, 0.01, 0.003, -0.002
    o = oracle.Oracle(c)
    o.set_state({I.C: C0, I.HE: He, I.FSPREV: Fs_prev, I.P: p0, I.MX: mx0, I.MY: my0})
    o.step(1)
    Fl = He / L
    Fs = 1.0 - Fl
    dt = c["dt"]
    S = (Fs - Fs_prev) / dt
    a = (1.0 - c["rho_s"] / c["rho_l"]) * S
    a0 = Fs * c["rho_s"] + (1.0 - Fs) * c["rho_g"]
    a1 = (1.0 - Fs) * (c["rho_l"] - c["rho_g"])
    exact = {
        I.C: C0 * P3(a * dt),
        I.P: p0 + CS2 * a * a0 * dt + CS2 * a1 * C0 * (P3(a * dt) - 1.0),
        I.MX: Fl * mx0 * P3(-S * dt),
        I.MY: Fl * my0 * P3(-S * dt),
        I.HE: He,
    }
    return o, exact


@pytest.mark.parametrize("C0", [0.9, 1.0])
def test_uniform_freezing_sources_closed_form(C0):
    o, exact = _uniform_freezing(C0=C0)
    for f, e in exact.items():
        got = o.get(f)
        assert np.ptp(got) == 0.0                      # the state stays uniform
        assert abs(got[0, 0] - e) <= 1e-14 * abs(e), (I.FIELD_NAMES[f], got[0, 0], e)
    # the volume grows as liquid turns into the lighter solid
    assert exact[I.C] > C0


@pytest.mark.parametrize("flag,fields", [
    (oracle.FLAG_PLANT_VOLUME_SIGN, (I.C, I.P)),
    (oracle.FLAG_PLANT_IBM_SIGN, (I.MX, I.MY)),
])
def test_uniform_freezing_pin_catches_planted_mistakes(flag, fields):
    o, exact = _uniform_freezing(flags=flag)
    for f in fields:
        err = abs(o.get(f)[0, 0] - exact[f]) / abs(exact[f])
        assert err > 1e-3, (I.FIELD_NAMES[f], err)


def _free_fall(flags=0, steps=40):
    g, rho = -3e-4, 1.6
    c = I.case(4, 4, periodic_x=1, periodic_y=1, init=2, stefan=0.0, latent=2.0, chi_l=0, chi_s=0,
               rho_l=rho, rho_s=rho, thermal_dirichlet=(0, 0, 0, 0), gravity=g, flags=flags)
    o = oracle.Oracle(c)
    o.step(steps)
    return o.get(I.V), g * steps * c["dt"]


def test_free_fall_in_a_periodic_box():
    """A uniform fluid under gravity in a periodic box falls freely: v = g t, with
    nothing else changing (the source c_s^2 rho g of the momentum c_s^2 rho u)."""
    v, exact = _free_fall()
    assert np.ptp(v) == 0.0
    assert abs(v[0, 0] - exact) <= 1e-12 * abs(exact)


def test_free_fall_catches_planted_gravity_sign():
    v, exact = _free_fall(flags=oracle.FLAG_PLANT_GRAVITY_SIGN)
    assert abs(v[0, 0] - exact) > 0.5 * abs(exact)


def _poiseuille(flags=0, W=16, steps=8000):
    """Gravity along y between no-slip walls at x = 0 and x = W, periodic in y."""
    g, rho, mu = 2e-5, 1.6, 0.08
    c = I.case(W, 1, periodic_y=1, init=2, stefan=0.0, latent=2.0, chi_l=0, chi_s=0, rho_l=rho,
               rho_s=rho, mu_l=mu, mu_s=mu, thermal_dirichlet=(0, 0, 0, 0), gravity=g, flags=flags)
    o = oracle.Oracle(c)
    o.step(steps)
    x = np.arange(W) + 0.5
    A = rho * g / (2.0 * mu)
    return o, A * x * (W - x), A


def test_plane_poiseuille_profile():
    """Steady plane Poiseuille flow (viscous time W^2/(pi^2 nu) ~ 170, run to t = 4000):
    - within 1 % of the exact parabola rho g x (W - x) / (2 mu);
    - within 2e-3 of the exact solution of the second-order finite-volume scheme whose
      wall lies half a cell from the first centre, the parabola plus rho g/(8 mu): in
      the first cell mu (v_1 - v_0) - 2 mu v_0 = -rho g holds for that profile;
    - no cross flow and no pressure gradient."""
    o, vex, A = _poiseuille()
    v = o.get(I.V)[0]
    assert np.max(np.abs(v - vex)) <= 1e-2 * vex.max()
    assert np.max(np.abs(v - (vex + A / 4.0))) <= 2e-3 * vex.max()
    assert np.max(np.abs(o.get(I.U))) < 1e-15
    assert np.ptp(o.get(I.P)) < 1e-15


@pytest.mark.parametrize("flag", [oracle.FLAG_PLANT_GRAVITY_SIGN, oracle.FLAG_PLANT_WALL_SIDE,
                                  oracle.FLAG_PLANT_WALL_FULL])
def test_poiseuille_catches_planted_mistakes(flag):
    with np.errstate(all="ignore"):
        o, vex, A = _poiseuille(flags=flag)
        v = o.get(I.V)[0]
        err = np.max(np.abs(v - vex)) / vex.max()
    assert not (err <= 1e-2), (flag, err)


def test_closed_box_phase_field_mass_change_is_the_volume_source():
    """In a box with no-flux walls the phase-field fluxes telescope (Eq. 42), so the
    sum over the cells of R_C is the sum of the volume-change source alone,
    (1 - rho_s/rho_l) sum C dF_s/dt, on any state.  A random state with every branch
    of the enthalpy inversion and a flow."""
    nx, ny = 12, 10
    c = I.case(nx, ny, radius=4.0, bo_m=0.5, field_angle_deg=30.0)
    o = oracle.Oracle(c)
    st = I.random_state(nx, ny, seed=5, latent=10.0)   # L = 1/Ste = 10
    o.set_state(st)
    R = o.rhs()
    C, Fsp = st[I.C], st[I.FSPREV]
    Fl = o.get(I.FL)
    S = ((1.0 - Fl) - Fsp) / c["dt"]
    src = (1.0 - c["rho_s"] / c["rho_l"]) * np.sum(C * S)
    assert abs(src) > 1e-3
    assert abs(R[4].sum() - src) <= 1e-12 * np.sum(np.abs(C * S))
    o2 = oracle.Oracle(dict(c, flags=oracle.FLAG_PLANT_VOLUME_SIGN))
    o2.set_state(st)
    assert abs(o2.rhs()[4].sum() - src) > 0.5 * abs(src)
