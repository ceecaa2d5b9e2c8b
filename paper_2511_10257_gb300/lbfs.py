"""Thin ctypes binding of the C ABI in include/lbfs.h (argument marshalling only).

Every step of the solver runs in the CUDA library liblbfs.so; this module only
builds the C structs, passes pointers and turns status codes into exceptions.
There is no fallback: if the library is missing or no CUDA device is present,
the calls raise.
"""
from __future__ import annotations

import ctypes as ct
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbfs.so")

FP64, MIXED = 0, 1
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EDIVERGED, ENOTCONVERGED = range(7)
STATUS_NAMES = {0: "LBFS_OK", 1: "LBFS_EINVAL", 2: "LBFS_ENOMEM", 3: "LBFS_ECUDA",
                4: "LBFS_ETIMEOUT", 5: "LBFS_EDIVERGED", 6: "LBFS_ENOTCONVERGED"}
SETTABLE = (0, 1, 4, 7, 10, 11, 12)

ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_size_t, ct.c_void_p)
FREE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_void_p)


class LbfsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Config(ct.Structure):
    _fields_ = [("device", ct.c_int32), ("precision", ct.c_int32), ("max_cases", ct.c_int32),
                ("use_graph", ct.c_int32), ("cuda_stream", ct.c_void_p),
                ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN), ("alloc_user", ct.c_void_p),
                ("mg_max_cycles", ct.c_int32), ("mg_tol", ct.c_double), ("tile", ct.c_int32),
                ("mg_warm_cycles", ct.c_int32), ("mg_plain_cycles", ct.c_int32), ("reserved", ct.c_int32 * 5)]


class CaseDesc(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int32), ("ny", ct.c_int32),
        ("periodic_x", ct.c_int32), ("periodic_y", ct.c_int32),
        ("thermal_dirichlet", ct.c_int32 * 4), ("wall_T", ct.c_double * 4),
        ("mag_bc", ct.c_int32), ("init", ct.c_int32),
        ("radius", ct.c_double), ("drop_x", ct.c_double), ("drop_y", ct.c_double),
        ("T_init", ct.c_double), ("H0", ct.c_double), ("field_angle_deg", ct.c_double),
        ("bo_m", ct.c_double), ("stefan", ct.c_double), ("latent", ct.c_double), ("T_m", ct.c_double),
        ("rho_l", ct.c_double), ("rho_g", ct.c_double), ("rho_s", ct.c_double),
        ("mu_l", ct.c_double), ("mu_g", ct.c_double), ("mu_s", ct.c_double),
        ("cp_l", ct.c_double), ("cp_g", ct.c_double), ("cp_s", ct.c_double),
        ("lam_l", ct.c_double), ("lam_g", ct.c_double), ("lam_s", ct.c_double),
        ("chi_l", ct.c_double), ("chi_g", ct.c_double), ("chi_s", ct.c_double),
        ("sigma", ct.c_double), ("xi", ct.c_double), ("mobility", ct.c_double), ("Q_g", ct.c_double),
        ("gravity", ct.c_double), ("dt", ct.c_double), ("dts", ct.c_double),
        ("contact_angle_deg", ct.c_double),
        ("flags", ct.c_int32), ("pad_", ct.c_int32),
    ]


class CaseStats(ct.Structure):
    _fields_ = [("sum_C", ct.c_double), ("sum_He", ct.c_double), ("sum_Fl_drop", ct.c_double),
                ("n_drop", ct.c_double), ("Q_L", ct.c_double), ("t", ct.c_double),
                ("t_freeze", ct.c_double), ("pot_resid", ct.c_double),
                ("pot_cycles", ct.c_int32), ("nonfinite", ct.c_int32),
                ("pot_resid_max", ct.c_double), ("pot_cycles_mean", ct.c_double)]


class CaseDiag(ct.Structure):
    _fields_ = [("H_m", ct.c_double), ("U_max", ct.c_double), ("Pe", ct.c_double),
                ("Fo", ct.c_double), ("Q_wall", ct.c_double)]


EXPORTS = ("lbfs_create", "lbfs_set_case", "lbfs_set_fields", "lbfs_step", "lbfs_fields",
           "lbfs_diagnostics", "lbfs_potential_pseudo_time", "lbfs_last_launch_count", "lbfs_timing", "lbfs_timing_read", "lbfs_autotune",
           "lbfs_destroy", "lbfs_last_error")
TILE_SHAPES = [(32, 8), (32, 16), (64, 8), (16, 16), (64, 4), (16, 16), (32, 8), (16, 16), (32, 8), (16, 16),
               (32, 8), (16, 15), (32, 7)]
TILE_NAMES = ["32x8", "32x16", "64x8", "16x16", "64x4", "16x16/3", "32x8/3", "16x16/4", "32x8/4", "16x16/4t",
              "32x8/4t", "16x15/4t", "32x7/4t"]
TIMING_STAGE, TIMING_POTENTIAL, TIMING_FINALIZE = range(3)

_lib = None


def load(path: str = LIB_PATH):
    """Load liblbfs.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} is missing: build it with paper_2511_10257_gb300.build.build()")
    L = ct.CDLL(path)
    vp = ct.c_void_p
    L.lbfs_create.argtypes = [ct.POINTER(Config), ct.POINTER(vp)]
    L.lbfs_set_case.argtypes = [vp, ct.c_int32, ct.POINTER(CaseDesc)]
    L.lbfs_set_fields.argtypes = [vp, ct.c_int32, ct.c_uint32, ct.POINTER(ct.c_double)]
    L.lbfs_step.argtypes = [vp, ct.c_int32, ct.POINTER(CaseStats)]
    L.lbfs_fields.argtypes = [vp, ct.c_int32, ct.c_uint32, ct.POINTER(ct.c_double)]
    L.lbfs_diagnostics.argtypes = [vp, ct.c_int32, ct.POINTER(CaseDiag), ct.POINTER(ct.c_double)]
    L.lbfs_potential_pseudo_time.argtypes = [vp, ct.c_int32, ct.c_int32, ct.c_double]
    L.lbfs_last_launch_count.argtypes = [vp]
    L.lbfs_last_launch_count.restype = ct.c_int64
    L.lbfs_destroy.argtypes = [vp]
    L.lbfs_destroy.restype = None
    L.lbfs_last_error.argtypes = [vp]
    L.lbfs_last_error.restype = ct.c_char_p
    L.lbfs_timing.argtypes = [vp, ct.c_int32]
    L.lbfs_autotune.argtypes = [vp, ct.c_int32, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_double), ct.c_int32]
    L.lbfs_timing_read.argtypes = [vp, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64), ct.c_int32]
    for name in ("lbfs_create", "lbfs_set_case", "lbfs_set_fields", "lbfs_step", "lbfs_fields",
                 "lbfs_diagnostics", "lbfs_potential_pseudo_time", "lbfs_timing", "lbfs_timing_read", "lbfs_autotune"):
        getattr(L, name).restype = ct.c_int
    _lib = L
    return L


def make_desc(d: dict) -> CaseDesc:
    c = CaseDesc()
    for name, typ in CaseDesc._fields_:
        if name == "pad_":
            continue
        if name == "flags":
            c.flags = int(d.get("flags", 0))
        elif name == "thermal_dirichlet":
            for i in range(4):
                c.thermal_dirichlet[i] = int(d[name][i])
        elif name == "wall_T":
            for i in range(4):
                c.wall_T[i] = float(d[name][i])
        elif typ is ct.c_int32:
            setattr(c, name, int(d[name]))
        else:
            setattr(c, name, float(d[name]))
    return c


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


class Solver:
    """A context of one or more cases advanced together on one GPU.

    stream: an int cudaStream_t handle to borrow (e.g. torch's current stream), or
    None for a stream owned by the context.  torch_alloc: route device memory
    through torch's caching allocator.
    """

    def __init__(self, precision: int = FP64, max_cases: int = 1, device: int = 0,
                 use_graph: bool = False, stream=None, torch_alloc: bool = False,
                 mg_max_cycles: int = 0, mg_tol: float = 0.0, tile: int = 0, mg_warm_cycles: int = 0,
                 mg_plain_cycles: bool = False):
        self._L = load()
        self._h = ct.c_void_p()
        cfg = Config()
        cfg.device = device
        cfg.precision = precision
        cfg.max_cases = max_cases
        cfg.use_graph = 1 if use_graph else 0
        cfg.cuda_stream = stream
        cfg.mg_max_cycles = mg_max_cycles
        cfg.mg_tol = mg_tol
        cfg.tile = tile
        cfg.mg_warm_cycles = mg_warm_cycles
        cfg.mg_plain_cycles = 1 if mg_plain_cycles else 0
        self._keep = []
        if torch_alloc:
            import torch

            def _alloc(nbytes, user):
                return torch.cuda.caching_allocator_alloc(int(nbytes), device)

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep += [fa, ff]
            cfg.dev_alloc, cfg.dev_free = fa, ff
        st = self._L.lbfs_create(ct.byref(cfg), ct.byref(self._h))
        if st != OK:
            raise LbfsError(st, "lbfs_create failed")
        self.max_cases = max_cases
        self.precision = precision
        self.shapes = {}
        self._mg_tol = mg_tol

    def mg_tol_used(self) -> float:
        """the potential's convergence tolerance in effect (the library's default when 0)"""
        return self._mg_tol if self._mg_tol > 0 else (1e-13 if self.precision == FP64 else 1e-6)

    def _check(self, st: int):
        if st != OK:
            msg = self._L.lbfs_last_error(self._h)
            raise LbfsError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._L.lbfs_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_case(self, case_id: int, desc: dict):
        self._check(self._L.lbfs_set_case(self._h, int(case_id), ct.byref(make_desc(desc))))
        self.shapes[case_id] = (int(desc["ny"]), int(desc["nx"]))

    def set_fields(self, case_id: int, fields: dict):
        ids = sorted(fields)
        ny, nx = self.shapes[case_id]
        buf = np.empty((len(ids), ny, nx), dtype=np.float64)
        for k, f in enumerate(ids):
            buf[k] = np.broadcast_to(np.asarray(fields[f], dtype=np.float64), (ny, nx))
        mask = sum(1 << int(f) for f in ids)
        self._check(self._L.lbfs_set_fields(self._h, int(case_id), mask, _dptr(buf)))

    def set_fields_packed(self, case_id: int, ids, packed: np.ndarray):
        """import fields from one C-contiguous FP64 array of shape (len(ids), ny, nx),
        ids in increasing order, passed to the library without a copy (e.g. pinned
        host memory)"""
        ids = [int(i) for i in ids]
        ny, nx = self.shapes[case_id]
        if (ids != sorted(ids) or packed.dtype != np.float64 or not packed.flags.c_contiguous
                or packed.shape != (len(ids), ny, nx)):
            raise ValueError("packed must be C-contiguous float64 of shape (len(ids), ny, nx), ids sorted")
        mask = sum(1 << f for f in ids)
        self._check(self._L.lbfs_set_fields(self._h, int(case_id), mask, _dptr(packed)))

    def fields_into(self, case_id: int, ids, out: np.ndarray):
        """export fields into a caller-owned C-contiguous FP64 array of shape
        (len(ids), ny, nx), ids in increasing order (no intermediate copy)"""
        ids = [int(i) for i in ids]
        ny, nx = self.shapes[case_id]
        if (ids != sorted(ids) or out.dtype != np.float64 or not out.flags.c_contiguous
                or out.shape != (len(ids), ny, nx)):
            raise ValueError("out must be C-contiguous float64 of shape (len(ids), ny, nx), ids sorted")
        mask = sum(1 << f for f in ids)
        self._check(self._L.lbfs_fields(self._h, int(case_id), mask, _dptr(out)))
        return out

    def step(self, nsteps: int = 1, raise_on_error: bool = True):
        out = (CaseStats * self.max_cases)()
        st = self._L.lbfs_step(self._h, int(nsteps), out)
        stats = [{n: getattr(o, n) for n, _ in CaseStats._fields_} for o in out]
        if raise_on_error:
            self._check(st)
        return stats if raise_on_error else (st, stats)

    def fields(self, case_id: int, ids) -> dict:
        ids = sorted(int(i) for i in ids)
        ny, nx = self.shapes[case_id]
        out = np.empty((len(ids), ny, nx), dtype=np.float64)
        mask = sum(1 << f for f in ids)
        self._check(self._L.lbfs_fields(self._h, int(case_id), mask, _dptr(out)))
        return {f: out[k] for k, f in enumerate(ids)}

    def diagnostics(self, case_id: int = 0):
        """Sec. 5 diagnostics: (dict of H_m, U_max, Pe, Fo, Q_wall; wall heat flux Q per column)."""
        d = CaseDiag()
        q = np.zeros(self.shapes[case_id][1])
        self._check(self._L.lbfs_diagnostics(self._h, int(case_id), ct.byref(d), _dptr(q)))
        return {n: getattr(d, n) for n, _ in CaseDiag._fields_}, q

    def potential_pseudo_time(self, case_id: int, iters: int, dtau: float):
        """the paper's pseudo-time magnetic LBFS: `iters` explicit steps on the stored potential"""
        self._check(self._L.lbfs_potential_pseudo_time(self._h, int(case_id), int(iters), float(dtau)))

    def field(self, case_id: int, fid: int) -> np.ndarray:
        return self.fields(case_id, [fid])[fid]

    def last_launch_count(self) -> int:
        return int(self._L.lbfs_last_launch_count(self._h))

    def autotune(self, reps: int = 5):
        """time every stage tile shape on the current cases and keep the fastest;
        returns (chosen id, [ms per launch for each shape])"""
        n = len(TILE_SHAPES)
        chosen = ct.c_int32()
        ms = (ct.c_double * n)()
        self._check(self._L.lbfs_autotune(self._h, int(reps), ct.byref(chosen), ms, n))
        return chosen.value, list(ms)

    def timing(self, enable: bool):
        self._check(self._L.lbfs_timing(self._h, 1 if enable else 0))

    def timing_read(self):
        """accumulated (ms, event pairs) per kernel class: stage, potential, finalize"""
        ms = (ct.c_double * 3)()
        cnt = (ct.c_int64 * 3)()
        self._check(self._L.lbfs_timing_read(self._h, ms, cnt, 3))
        return [(ms[k], cnt[k]) for k in range(3)]
