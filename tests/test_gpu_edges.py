"""Edge cases of the C ABI on the GPU: a context with no case, zero steps, the
smallest grid (4 x 4, one ragged tile) against the oracle, and the argument checks
(each rejected with LBFS_EINVAL before anything is allocated or launched)."""
import ctypes as ct

import numpy as np
import pytest

import oracle
from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

from parity import assert_parity

pytestmark = pytest.mark.gpu
EINVAL = 1


def test_context_without_cases_steps_to_zero_stats():
    s = lbfs.Solver(precision=lbfs.MIXED, max_cases=3)
    st = s.step(5)
    assert all(x["t"] == 0.0 and x["sum_C"] == 0.0 for x in st)
    s.set_case(1, I.case(32, 16, radius=6.0))
    st = s.step(2)
    assert st[0]["t"] == 0.0 and st[2]["t"] == 0.0
    assert st[1]["t"] == pytest.approx(2 * 0.5) and st[1]["sum_C"] > 0
    s.close()


@pytest.mark.parametrize("precision", [lbfs.FP64, lbfs.MIXED])
def test_zero_steps_change_nothing(precision):
    s = lbfs.Solver(precision=precision, max_cases=1)
    s.set_case(0, I.case(40, 20, radius=8.0, bo_m=1.0))
    ids = [I.PHI, I.HE, I.P, I.C, I.MX, I.MY]
    before = s.fields(0, ids)
    st = s.step(0)[0]
    after = s.fields(0, ids)
    s.close()
    assert st["t"] == 0.0
    for f in ids:
        assert np.array_equal(before[f], after[f]), I.FIELD_NAMES[f]


def test_smallest_grid_matches_oracle():
    c = I.case(4, 4, radius=1.5, bo_m=0.5, stefan=0.2)
    ref = oracle.Oracle(c)
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1)
    s.set_case(0, c)
    for n in (1, 20):
        ref.step(n)
        s.step(n)
        assert_parity(s, 0, ref, 1e-9)
    s.close()


def test_arguments_are_checked():
    s = lbfs.Solver(precision=lbfs.MIXED, max_cases=2)
    bad_cases = [I.case(3, 16), I.case(16, 3), dict(I.case(16, 8), flags=1), I.case(16, 8, dt=2.0),
                 I.case(65536, 65536, radius=10.0),
                 I.case(33, 1 << 25, radius=10.0),   # 33 x 2^25 cells, but rows padded to 64: 2^31
                 I.case(16, 8, radius=0.0), I.case(16, 8, xi=0.0),
                 I.case(16, 8, rho_l=0.0), I.case(16, 8, mu_l=-1.0)]
    for c in bad_cases:
        with pytest.raises(lbfs.LbfsError) as e:
            s.set_case(0, c)
        assert e.value.status == EINVAL
    L, h = s._L, s._h
    desc = lbfs.make_desc(I.case(16, 8))
    assert L.lbfs_set_case(h, 2, ct.byref(desc)) == EINVAL           # case id out of range
    assert L.lbfs_set_case(h, -1, ct.byref(desc)) == EINVAL
    buf = np.zeros(16 * 8)
    ptr = buf.ctypes.data_as(ct.POINTER(ct.c_double))
    assert L.lbfs_fields(h, 0, 1 << I.C, ptr) == EINVAL             # case 0 is not defined
    s.set_case(0, I.case(16, 8))
    assert L.lbfs_fields(h, 0, 0, ptr) == EINVAL                    # empty mask
    assert L.lbfs_fields(h, 0, 1 << 13, ptr) == EINVAL              # unknown field
    assert L.lbfs_fields(h, 0, 1 << I.C, None) == EINVAL            # no buffer
    assert L.lbfs_set_fields(h, 0, 1 << I.T, ptr) == EINVAL         # T is derived, not settable
    with pytest.raises(lbfs.LbfsError):
        s.step(-1)
    assert L.lbfs_fields(h, 0, 1 << I.C, ptr) == 0                  # the context is still usable
    s.step(1)
    s.close()


def test_calls_select_the_context_device():
    """set_case, set_fields and fields run on the context's device even when another
    device is current in the calling thread."""
    torch = pytest.importorskip("torch")
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two devices")
    c = I.case(32, 16, radius=6.0, bo_m=1.0)
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1, device=0)
    torch.cuda.set_device(1)
    try:
        s.set_case(0, c)
        st = I.random_state(32, 16, seed=3)
        s.set_fields(0, st)
        s.step(3)
        got = s.fields(0, [I.C, I.HE])
    finally:
        torch.cuda.set_device(0)
        s.close()
    ref = oracle.Oracle(c)
    ref.set_state(st)
    ref.step(3)
    for f in (I.C, I.HE):
        assert np.max(np.abs(got[f] - ref.get(f))) <= 1e-9 * np.max(np.abs(ref.get(f)))
