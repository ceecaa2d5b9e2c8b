"""Execution modes of the CUDA path: graph replay and batching change nothing in the
results (bitwise), and the mixed-precision path stays within the stated error of the
FP64 path (liquid fraction L-infinity 1e-4, freezing time 0.5 %)."""
import numpy as np
import pytest

from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

pytestmark = pytest.mark.gpu
IDS = [I.HE, I.P, I.C, I.MX, I.MY, I.PHI, I.FSPREV]


def _run(cases, precision, steps, use_graph=False):
    s = lbfs.Solver(precision=precision, max_cases=len(cases), use_graph=use_graph)
    for k, c in enumerate(cases):
        s.set_case(k, c)
    st = s.step(steps)
    out = [s.fields(k, IDS) for k in range(len(cases))]
    s.close()
    return out, st


@pytest.mark.parametrize("precision", [lbfs.MIXED, lbfs.FP64])
def test_graph_replay_is_bitwise_equal_to_eager(precision):
    c = I.case(96, 48, radius=18.0, bo_m=1.0, field_angle_deg=70.0, stefan=0.3)
    a, sa = _run([c], precision, 30, use_graph=False)
    b, sb = _run([c], precision, 30, use_graph=True)
    for f in IDS:
        assert np.array_equal(a[0][f], b[0][f]), I.FIELD_NAMES[f]
    assert sa[0]["Q_L"] == sb[0]["Q_L"]


@pytest.mark.parametrize("precision", [lbfs.FP64, lbfs.MIXED])
def test_batched_cases_equal_each_case_alone(precision):
    cases = [I.case(64, 32, radius=12.0, bo_m=0.5, field_angle_deg=0.0, stefan=0.2),
             I.case(96, 48, radius=18.0, bo_m=1.5, field_angle_deg=90.0, stefan=0.1),
             I.case(40, 24, radius=9.0, bo_m=1.0, field_angle_deg=33.0, stefan=0.15, chi_l=2.0, chi_s=2.0)]
    batch, sb = _run(cases, precision, 25)
    for k, c in enumerate(cases):
        alone, sa = _run([c], precision, 25)
        for f in IDS:
            assert np.array_equal(batch[k][f], alone[0][f]), (k, I.FIELD_NAMES[f])
        assert sb[k]["sum_C"] == sa[0]["sum_C"]


def _freeze(case, precision, max_steps, chunk=500):
    s = lbfs.Solver(precision=precision, max_cases=1, use_graph=True)
    s.set_case(0, case)
    snaps, ql = [], []
    n = 0
    while n < max_steps:
        st = s.step(chunk)[0]
        n += chunk
        snaps.append(s.fields(0, [I.FL, I.C]))
        ql.append(st["Q_L"])
        if st["t_freeze"] > 0:
            break
    s.close()
    return st["t_freeze"], snaps, np.array(ql)


@pytest.mark.slow
def test_mixed_precision_error_small_case():
    """128 x 64 case (vertical field, Bo_m 0.5) to full freeze, mixed against FP64 on
    the same GPU, sampled every 500 steps:
      - freezing time within 0.5 %;
      - droplet liquid fraction Q_L(t) (Eq. 51) within 1e-4 at every sample;
      - no cell on different sides of the C = 1/2 phase-change switch;
      - pointwise F_l within 2e-2: only cells at the moving front differ, by the
        front's time offset times its speed."""
    c = I.config_small()
    t64, s64, q64 = _freeze(c, lbfs.FP64, 40000)
    t32, s32, q32 = _freeze(c, lbfs.MIXED, 40000)
    assert t64 > 0 and t32 > 0
    n = min(len(s64), len(s32))
    flerr, dis = 0.0, 0
    for k in range(n):
        a, b = s64[k], s32[k]
        agree = (a[I.C] >= 0.5) == (b[I.C] >= 0.5)
        dis = max(dis, int((~agree).sum()))
        flerr = max(flerr, float(np.max(np.abs(a[I.FL] - b[I.FL])[agree])))
    qerr = float(np.max(np.abs(q64[:n] - q32[:n])))
    print(f"t_freeze FP64 {t64:.4f} mixed {t32:.4f} rel {(t32 - t64) / t64:.2e}; "
          f"Q_L Linf {qerr:.2e}; F_l Linf {flerr:.2e}; switch disagreements {dis}")
    assert abs(t32 - t64) <= 0.005 * t64
    assert qerr <= 1e-4
    assert dis == 0
    assert flerr <= 2e-2


def test_mixed_precision_conserves_phase_field_mass():
    """rho_s = rho_l: sum C is conserved by the flux form; in mixed precision the drift
    over 2000 steps stays at FP32 rounding level (no systematic growth)."""
    c = I.case(128, 64, radius=24.0, bo_m=0.5, rho_s=1.0, stefan=0.1)
    s = lbfs.Solver(precision=lbfs.MIXED, max_cases=1, use_graph=True)
    s.set_case(0, c)
    c0 = s.step(0)[0]["sum_C"]
    c1 = s.step(2000)[0]["sum_C"]
    s.close()
    assert abs(c1 - c0) <= 2e-6 * c0


@pytest.mark.parametrize("precision", [lbfs.MIXED, lbfs.FP64])
def test_tile_shapes_give_identical_fields(precision):
    """Every face is computed with the same arithmetic whichever tile holds it, so all
    tile shapes give bitwise-identical fields; the autotuner keeps one of them."""
    c = I.case(100, 52, radius=19.0, bo_m=1.2, field_angle_deg=20.0, stefan=0.25)
    ref = None
    for tile in range(len(lbfs.TILE_SHAPES)):
        s = lbfs.Solver(precision=precision, max_cases=1, tile=tile)
        s.set_case(0, c)
        s.step(15)
        got = s.fields(0, IDS)
        if tile == 0:
            chosen, ms = s.autotune(reps=2)
            assert 0 <= chosen < len(lbfs.TILE_SHAPES) and all(m > 0 for m in ms)
            s.step(5)
            after = s.fields(0, IDS)
        s.close()
        if ref is None:
            ref = got
        for f in IDS:
            assert np.array_equal(got[f], ref[f]), (tile, I.FIELD_NAMES[f])
    s = lbfs.Solver(precision=precision, max_cases=1)
    s.set_case(0, c)
    s.step(20)
    plain = s.fields(0, IDS)
    s.close()
    for f in IDS:
        assert np.array_equal(after[f], plain[f]), I.FIELD_NAMES[f]


@pytest.mark.parametrize("precision", [lbfs.MIXED, lbfs.FP64])
def test_every_warm_step_ends_converged(precision):
    """Each step's potential solve ends with the residual of the corrected potential
    at or below the tolerance, in eager steps and in graph replay."""
    c = I.case(96, 48, radius=18.0, bo_m=1.5, field_angle_deg=60.0, stefan=0.3)
    tol = 1e-6 if precision == lbfs.MIXED else 1e-13
    for graph in (False, True):
        s = lbfs.Solver(precision=precision, max_cases=1, use_graph=graph)
        s.set_case(0, c)
        s.step(1)
        st = s.step(200)[0]
        s.close()
        assert 0.0 < st["pot_resid_max"] <= tol, st
        assert st["pot_resid"] <= tol
        assert st["pot_cycles_mean"] >= (1.0 if precision == lbfs.FP64 else 0.0)


def test_warm_solve_reports_a_missed_tolerance():
    """One warm cycle cannot take the mixed potential to 1e-13: lbfs_step says so."""
    c = I.case(96, 48, radius=18.0, bo_m=1.5, field_angle_deg=60.0, stefan=0.3)
    s = lbfs.Solver(precision=lbfs.MIXED, max_cases=1, mg_tol=1e-13, mg_warm_cycles=1)
    s.set_case(0, c)
    s.step(1)
    status, st = s.step(5, raise_on_error=False)
    s.close()
    assert status == lbfs.ENOTCONVERGED
    assert st[0]["pot_resid_max"] > 1e-13


@pytest.mark.parametrize("precision", [lbfs.MIXED, lbfs.FP64])
def test_plain_cycle_launches_give_identical_fields(precision):
    """The warm cycles as a conditional graph loop or as plain launches are the same
    computation: bitwise-identical fields, eager and replayed."""
    c = I.case(96, 48, radius=18.0, bo_m=1.5, field_angle_deg=60.0, stefan=0.3)
    out = []
    for plain in (False, True):
        for graph in (False, True):
            s = lbfs.Solver(precision=precision, max_cases=1, use_graph=graph, mg_plain_cycles=plain)
            s.set_case(0, c)
            st = s.step(40)[0]
            out.append((s.fields(0, IDS), st))
            s.close()
    for got, st in out[1:]:
        for f in IDS:
            assert np.array_equal(got[f], out[0][0][f]), I.FIELD_NAMES[f]
        assert st["pot_resid_max"] == out[0][1]["pot_resid_max"]


def test_fp64_extrapolated_start_saves_cycles():
    """From the third step after a state is set, the FP64 solve starts from the potential
    extrapolated linearly in time and needs fewer refinement cycles than the second
    step, which starts from the previous potential; every step still meets 1e-13."""
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1, use_graph=True)
    s.set_case(0, I.config_small())
    s.step(300)
    s.set_fields(0, s.fields(0, IDS))   # a fresh start: the extrapolation begins again
    cyc = []
    for _ in range(12):
        st = s.step(1)[0]
        assert st["pot_resid"] <= 1e-13, st
        cyc.append(st["pot_cycles"])
    s.close()
    assert np.mean(cyc[2:]) < cyc[1], cyc
