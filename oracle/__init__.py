"""ctypes wrapper of the FP64 CPU oracle (lbfs_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
CPU-baseline leg of bench.py.  The library (paper_2511_10257_gb300) never imports
this package and shares no code with it.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbfs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C11, OpenMP if present)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbfs_oracle.h"))):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class OracleCase(ct.Structure):
    _fields_ = [
        ("nx", ct.c_int32), ("ny", ct.c_int32),
        ("periodic_x", ct.c_int32), ("periodic_y", ct.c_int32),
        ("thermal_dirichlet", ct.c_int32 * 4),
        ("wall_T", ct.c_double * 4),
        ("mag_bc", ct.c_int32), ("init", ct.c_int32),
        ("radius", ct.c_double), ("drop_x", ct.c_double), ("drop_y", ct.c_double),
        ("T_init", ct.c_double),
        ("H0", ct.c_double), ("field_angle_deg", ct.c_double),
        ("bo_m", ct.c_double), ("stefan", ct.c_double), ("latent", ct.c_double),
        ("T_m", ct.c_double),
        ("rho_l", ct.c_double), ("rho_g", ct.c_double), ("rho_s", ct.c_double),
        ("mu_l", ct.c_double), ("mu_g", ct.c_double), ("mu_s", ct.c_double),
        ("cp_l", ct.c_double), ("cp_g", ct.c_double), ("cp_s", ct.c_double),
        ("lam_l", ct.c_double), ("lam_g", ct.c_double), ("lam_s", ct.c_double),
        ("chi_l", ct.c_double), ("chi_g", ct.c_double), ("chi_s", ct.c_double),
        ("sigma", ct.c_double), ("xi", ct.c_double), ("mobility", ct.c_double),
        ("Q_g", ct.c_double), ("gravity", ct.c_double),
        ("dt", ct.c_double), ("dts", ct.c_double), ("contact_angle_deg", ct.c_double),
        ("flags", ct.c_int32), ("pad_", ct.c_int32),
    ]


class OracleStats(ct.Structure):
    _fields_ = [("sum_C", ct.c_double), ("sum_He", ct.c_double), ("sum_Fl_drop", ct.c_double),
                ("n_drop", ct.c_double), ("Q_L", ct.c_double), ("t", ct.c_double),
                ("t_freeze", ct.c_double), ("pot_resid", ct.c_double),
                ("pot_iters", ct.c_int32), ("nonfinite", ct.c_int32)]


class OracleDiag(ct.Structure):
    _fields_ = [("H_m", ct.c_double), ("U_max", ct.c_double), ("Pe", ct.c_double),
                ("Fo", ct.c_double), ("Q_wall", ct.c_double)]


FLAG_LITERAL_FSTAR_SIGN = 1
FLAG_LITERAL_MUC_SIGN = 2
FLAG_KEEP_POTENTIAL = 4
# planted mistakes, for showing that a pin catches them (tests only)
FLAG_PLANT_VOLUME_SIGN = 8
FLAG_PLANT_GRAVITY_SIGN = 16
FLAG_PLANT_WALL_SIDE = 32
FLAG_PLANT_WALL_FULL = 64
FLAG_PLANT_IBM_SIGN = 128

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ct.CDLL(build())
        L = _lib
        pd = ct.POINTER(ct.c_double)
        L.oracle_create.argtypes = [ct.POINTER(OracleCase), ct.POINTER(ct.c_void_p)]
        L.oracle_destroy.argtypes = [ct.c_void_p]
        L.oracle_step.argtypes = [ct.c_void_p, ct.c_int32]
        L.oracle_get_field.argtypes = [ct.c_void_p, ct.c_int32, pd]
        L.oracle_set_field.argtypes = [ct.c_void_p, ct.c_int32, pd]
        L.oracle_get_stats.argtypes = [ct.c_void_p, ct.POINTER(OracleStats)]
        L.oracle_set_threads.argtypes = [ct.c_int32]
        L.oracle_eq8.argtypes = [ct.POINTER(OracleCase), ct.c_double, ct.c_double, pd, pd]
        L.oracle_mix.argtypes = [ct.c_double] * 5
        L.oracle_mix.restype = ct.c_double
        L.oracle_equilibria.argtypes = [ct.POINTER(OracleCase), ct.c_int32] + [ct.c_double] * 9 + [pd] * 3
        L.oracle_face_flux.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32, pd]
        L.oracle_mag_lbfs_flux.argtypes = [ct.c_void_p, ct.c_int32, ct.c_int32, ct.c_int32, ct.c_double]
        L.oracle_mag_lbfs_flux.restype = ct.c_double
        L.oracle_solve_potential.argtypes = [ct.c_void_p]
        L.oracle_pseudo_time_potential.argtypes = [ct.c_void_p, ct.c_int32, ct.c_double]
        L.oracle_rhs.argtypes = [ct.c_void_p, pd]
        L.oracle_diagnostics.argtypes = [ct.c_void_p, ct.POINTER(OracleDiag), pd]
    return _lib


def make_case(d: dict) -> OracleCase:
    c = OracleCase()
    for name, typ in OracleCase._fields_:
        if name == "pad_":
            continue
        if name == "flags":
            c.flags = int(d.get("flags", 0))
            continue
        v = d[name]
        if name in ("thermal_dirichlet",):
            for i in range(4):
                c.thermal_dirichlet[i] = int(v[i])
        elif name == "wall_T":
            for i in range(4):
                c.wall_T[i] = float(v[i])
        elif typ is ct.c_int32:
            setattr(c, name, int(v))
        else:
            setattr(c, name, float(v))
    return c


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


class Oracle:
    """One case advanced by the FP64 CPU oracle."""

    def __init__(self, case: dict, threads: int = 1):
        self.case = dict(case)
        self.nx, self.ny = int(case["nx"]), int(case["ny"])
        self._c = make_case(case)
        h = ct.c_void_p()
        rc = lib().oracle_create(ct.byref(self._c), ct.byref(h))
        if rc != 0:
            raise ValueError(f"oracle_create failed ({rc})")
        self._h = h
        lib().oracle_set_threads(int(threads))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().oracle_destroy(h)
            self._h = None

    def step(self, n: int = 1) -> int:
        return lib().oracle_step(self._h, int(n))

    def get(self, field: int) -> np.ndarray:
        out = np.empty((self.ny, self.nx), dtype=np.float64)
        if lib().oracle_get_field(self._h, int(field), _ptr(out)) != 0:
            raise ValueError(f"bad field {field}")
        return out

    def set(self, field: int, arr) -> None:
        a = np.ascontiguousarray(np.broadcast_to(np.asarray(arr, dtype=np.float64),
                                                 (self.ny, self.nx)))
        if lib().oracle_set_field(self._h, int(field), _ptr(a)) != 0:
            raise ValueError(f"field {field} cannot be set")

    def set_state(self, fields: dict) -> None:
        for f, a in fields.items():
            self.set(f, a)

    def stats(self) -> dict:
        s = OracleStats()
        lib().oracle_get_stats(self._h, ct.byref(s))
        return {n: getattr(s, n) for n, _ in OracleStats._fields_}

    def diagnostics(self):
        """(dict of H_m, U_max, Pe, Fo, Q_wall; local wall heat flux Q per column)"""
        d = OracleDiag()
        q = np.zeros(self.nx)
        lib().oracle_diagnostics(self._h, ct.byref(d), _ptr(q))
        return {n: getattr(d, n) for n, _ in OracleDiag._fields_}, q

    def face_flux(self, axis: int, i: int, j: int) -> np.ndarray:
        out = np.zeros(5)
        lib().oracle_face_flux(self._h, int(axis), int(i), int(j), _ptr(out))
        return out

    def mag_lbfs_flux(self, axis: int, i: int, j: int, mu_face: float) -> float:
        return lib().oracle_mag_lbfs_flux(self._h, int(axis), int(i), int(j), float(mu_face))

    def solve_potential(self) -> int:
        return lib().oracle_solve_potential(self._h)

    def pseudo_time_potential(self, iters: int, dtau: float) -> None:
        lib().oracle_pseudo_time_potential(self._h, int(iters), float(dtau))

    def rhs(self) -> np.ndarray:
        out = np.zeros((5, self.ny, self.nx))
        lib().oracle_rhs(self._h, _ptr(out))
        return out


def eq8(case: dict, He: float, C: float):
    c = make_case(case)
    T, Fl = ct.c_double(), ct.c_double()
    lib().oracle_eq8(ct.byref(c), float(He), float(C), ct.byref(T), ct.byref(Fl))
    return T.value, Fl.value


def equilibria(case: dict, a: int, p, u, v, C, muc, T, He, rho, cp):
    c = make_case(case)
    f, g, h = ct.c_double(), ct.c_double(), ct.c_double()
    lib().oracle_equilibria(ct.byref(c), int(a), float(p), float(u), float(v), float(C), float(muc),
                            float(T), float(He), float(rho), float(cp), ct.byref(f), ct.byref(g),
                            ct.byref(h))
    return f.value, g.value, h.value


def mix(Fs, C, gs, gl, gg):
    return lib().oracle_mix(float(Fs), float(C), float(gs), float(gl), float(gg))
