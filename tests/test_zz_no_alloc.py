"""The allocation-free statistics entry point, called through the C ABI on device
arrays, against the statistics lbfs_step reports for the same state.

Callers that cannot allocate device memory (inside another component's fixed pool,
or while that component records GPU work) use lbfs_state_stats_noalloc, whose
scratch is a fixed device array.  This file is collected last so that a run that
stops at the first failure has run every other test before it."""
import ctypes as ct

import numpy as np
import pytest

from paper_2511_10257_gb300 import inputs as I
from paper_2511_10257_gb300 import lbfs

pytestmark = pytest.mark.gpu

KEYS = ("sum_C", "sum_He", "sum_Fl_drop", "n_drop", "Q_L")


def _noalloc(L, desc, He_dev, C_dev, out_dev, stream):
    err = ct.create_string_buffer(256)
    st = L.lbfs_state_stats_noalloc(ct.byref(lbfs.make_desc(desc)), ct.c_void_p(He_dev.data_ptr()),
                                    ct.c_void_p(C_dev.data_ptr()), ct.c_void_p(out_dev.data_ptr()),
                                    ct.c_void_p(stream), err, 256)
    return st, err.value.decode()


def test_noalloc_stats_match_step_stats_twice():
    torch = pytest.importorskip("torch")
    L = lbfs.load()
    L.lbfs_state_stats_noalloc.argtypes = [ct.POINTER(lbfs.CaseDesc), ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                          ct.c_void_p, ct.c_char_p, ct.c_size_t]
    L.lbfs_state_stats_noalloc.restype = ct.c_int
    desc = I.case(96, 48, radius=18.0, bo_m=1.0, field_angle_deg=60.0, stefan=0.5)
    s = lbfs.Solver(precision=lbfs.FP64, max_cases=1)
    s.set_case(0, desc)
    stream = torch.cuda.current_stream()
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    for nsteps in (40, 25):   # two calls in a row on different states
        ref = s.step(nsteps)[0]
        f = s.fields(0, [I.HE, I.C])
        He = torch.from_numpy(np.ascontiguousarray(f[I.HE])).cuda()
        C = torch.from_numpy(np.ascontiguousarray(f[I.C])).cuda()
        out.fill_(-1.0)
        st, msg = _noalloc(L, desc, He, C, out, stream.cuda_stream)
        assert st == lbfs.OK, msg
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for k, key in enumerate(KEYS):
            assert got[k] == pytest.approx(ref[key], rel=1e-12, abs=1e-12), key
        assert ref["Q_L"] > 0.0
    s.close()


def test_noalloc_rejects_grids_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    L = lbfs.load()
    L.lbfs_state_stats_noalloc.argtypes = [ct.POINTER(lbfs.CaseDesc), ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                          ct.c_void_p, ct.c_char_p, ct.c_size_t]
    L.lbfs_state_stats_noalloc.restype = ct.c_int
    desc = I.case(4, 16385, stefan=0.1)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    st, msg = _noalloc(L, desc, buf, buf, buf, 0)
    assert st == lbfs.EINVAL and "16384" in msg
