"""The paper's closed-form benchmarks run directly on the CUDA path, in FP64 and in
mixed precision: the two-phase Neumann solution of conductive freezing (Sec. 4.1)
and the Laplace law of a free drop.  These pin the GPU path to the mathematics, not
only to the oracle."""
import math

import numpy as np
import pytest

from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

from test_oracle_physics import neumann_k, neumann_T

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [lbfs.FP64, lbfs.MIXED])
def test_neumann_moving_front_gpu(precision):
    alpha, L, nx = 0.3, 10.0, 200
    c = I.case(nx, 4, periodic_y=1, init=2, T_init=1.0, stefan=0.0, latent=L, rho_s=1.0, cp_s=1.0,
               cp_l=1.0, lam_s=alpha, lam_l=alpha, chi_l=0, chi_s=0, thermal_dirichlet=(1, 1, 0, 0),
               wall_T=(-1.0, 1.0, 0.0, 0.0))
    s = lbfs.Solver(precision=precision, max_cases=1, use_graph=True)
    s.set_case(0, c)
    k = neumann_k(1.0 / L, 1.0 / L, alpha, alpha)
    x = np.arange(nx) + 0.5
    t = 0.0
    for t_end in (1000.0, 2000.0, 3000.0):
        s.step(int(round((t_end - t) / c["dt"])))
        t = t_end
        T_exact, X = neumann_T(x, t_end, k, -1.0, 1.0, 0.0, alpha, alpha)
        f = s.fields(0, [I.T, I.FL])
        assert np.max(np.abs(f[I.T] - f[I.T][:1])) < 1e-12   # y-uniform
        Xs = float(np.sum(1.0 - f[I.FL][0]))
        err = np.abs(f[I.T][0] - T_exact)
        assert abs(Xs - X) < 0.25 and err.mean() < 2e-3 and err.max() < 4e-2
    s.close()


@pytest.mark.parametrize("precision", [lbfs.FP64, lbfs.MIXED])
def test_laplace_law_gpu(precision):
    n = 64
    radii = (8.0, 11.0, 14.0)
    cases = [I.case(n, n, periodic_x=1, periodic_y=1, init=1, radius=R, drop_x=n / 2, drop_y=n / 2,
                    T_init=1.0, chi_l=0, chi_s=0, thermal_dirichlet=(0, 0, 0, 0)) for R in radii]
    s = lbfs.Solver(precision=precision, max_cases=len(cases), use_graph=True)
    for k, c in enumerate(cases):
        s.set_case(k, c)
    st = s.step(1500)
    dP, invR = [], []
    for k in range(len(cases)):
        f = s.fields(k, [I.P, I.C, I.MUC])
        P = f[I.P] + f[I.C] * f[I.MUC]
        dP.append(P[n // 2, n // 2] - P[2, 2])
        invR.append(1.0 / math.sqrt(st[k]["sum_C"] / math.pi))
    s.close()
    slope, icpt = np.polyfit(np.array(invR), np.array(dP), 1)
    assert slope == pytest.approx(I.DEFAULTS["sigma"], rel=0.05)
