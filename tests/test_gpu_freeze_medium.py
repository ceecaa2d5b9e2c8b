"""The 512x256 case (R = 96, vertical field, Bo_m = 1, chi = 1, Ste = 0.1) run to full
freeze in mixed precision and in FP64, the freezing times (Eq. 51) compared: the mixed
form within 0.5 %, and its liquid fraction Q_L(t) beside the FP64 one every CHUNK steps.
About 430,000 steps each; the FP64 run takes about 20 minutes on a GB300, so the test
runs only when LBFS_LONG_TESTS=1.  The FP64 potential is converged to 1e-10 instead of
1e-13 to bound that time (the mixed one to its usual 1e-6)."""
import os

import numpy as np
import pytest

from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(os.environ.get("LBFS_LONG_TESTS") != "1",
                                 reason="about 20 minutes of GPU time; set LBFS_LONG_TESTS=1")]
CHUNK = 2000


def _to_freeze(precision, mg_tol, max_steps=1_000_000):
    s = lbfs.Solver(precision=precision, max_cases=1, use_graph=True, mg_tol=mg_tol)
    s.set_case(0, I.config_medium())
    ql, n, st = [], 0, None
    while n < max_steps:
        st = s.step(CHUNK)[0]
        n += CHUNK
        ql.append(st["Q_L"])
        if st["t_freeze"] > 0:
            break
    s.close()
    return st["t_freeze"], np.array(ql), n


def test_medium_case_freezing_time_mixed_against_fp64():
    t32, q32, n32 = _to_freeze(lbfs.MIXED, 0.0)
    t64, q64, n64 = _to_freeze(lbfs.FP64, 1e-10)
    assert t32 > 0 and t64 > 0
    m = min(len(q32), len(q64))
    rel = (t32 - t64) / t64
    print(f"\n512x256 to freeze: t_freeze mixed {t32:.1f}, FP64 {t64:.1f}, relative error {rel:.2e}; "
          f"Q_L L-inf {np.max(np.abs(q32[:m] - q64[:m])):.2e} over {m} samples every {CHUNK} steps "
          f"({n32} and {n64} steps run)")
    assert abs(rel) <= 0.005
