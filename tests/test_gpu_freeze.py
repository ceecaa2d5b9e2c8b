"""The 128x64 sessile ferrofluid drop (R = 24, vertical field, Bo_m = 0.5, chi = 1,
Ste = 0.1) run on the GPU until it has frozen, against the oracle's own run to
freeze stored in tests/golden/c1_freeze_oracle.json (written by
tests/golden/make_c1_freeze.py, which calls only the oracle).

FP64: the freezing time (Eq. 51, first t with Q_L >= 0.99) and the Q_L history agree
to 1e-6.  Mixed precision: the freezing time is within 1e-4 of the oracle's."""
import json
import os

import pytest

from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "c1_freeze_oracle.json")


def _run(prec):
    with open(GOLDEN) as f:
        g = json.load(f)
    s = lbfs.Solver(precision=prec, max_cases=1, use_graph=True)
    s.set_case(0, I.config_small())
    hist = []
    n = 0
    for n_ref, _ in g["Q_L_every_500_steps"]:
        st = s.step(n_ref - n)[0]
        n = n_ref
        hist.append(st["Q_L"])
    s.close()
    return g, st, hist


def test_fp64_freeze_matches_oracle():
    g, st, hist = _run(lbfs.FP64)
    assert st["t_freeze"] > 0 and g["t_freeze"] > 0
    assert st["t_freeze"] == pytest.approx(g["t_freeze"], rel=1e-6)
    for (n, q_ref), q in zip(g["Q_L_every_500_steps"], hist):
        assert abs(q - q_ref) <= 1e-6, (n, q, q_ref)


def test_mixed_freeze_time_matches_oracle():
    g, st, _ = _run(lbfs.MIXED)
    assert st["t_freeze"] == pytest.approx(g["t_freeze"], rel=1e-4)
