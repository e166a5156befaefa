"""ctypes front end of the FP64 C projectors in ``projectors.c`` (test infrastructure).

The shared object is compiled with gcc on first use (or by ``build()``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "projectors.c")
_SO = os.path.join(_HERE, "liboracle_projectors.so")
_lib = None


class _Geom(ctypes.Structure):
    _fields_ = [("beam", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("pix", ctypes.c_double), ("na", ctypes.c_int),
                ("ang", ctypes.POINTER(ctypes.c_double)), ("nd", ctypes.c_int),
                ("du", ctypes.c_double), ("sod", ctypes.c_double), ("sdd", ctypes.c_double),
                ("cosv", ctypes.POINTER(ctypes.c_double)),
                ("sinv", ctypes.POINTER(ctypes.c_double))]


def build(force: bool = False) -> str:
    """Compile the C oracle (plain -O2, no fast-math, OpenMP over independent
    outputs) and return the .so path."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        gp = ctypes.POINTER(_Geom)
        for name in ("og_forward", "og_forward_T", "og_back", "og_back_T"):
            f = getattr(lib, name)
            f.argtypes = [gp, dp, dp]
            f.restype = None
        for name in ("og_forward_ray", "og_back_T_ray", "og_back_pixel", "og_forward_T_pixel"):
            f = getattr(lib, name)
            f.argtypes = [gp, dp, ctypes.c_int, ctypes.c_int]
            f.restype = ctypes.c_double
        lib.og_threads.argtypes = []
        lib.og_threads.restype = ctypes.c_int
        lib.og_set_threads.argtypes = [ctypes.c_int]
        lib.og_set_threads.restype = None
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Projectors:
    """The four FP64 operators of one scan geometry (a ``gkb_inputs.Geometry``)."""

    def __init__(self, geom):
        self.geom = geom
        self._ang = np.ascontiguousarray(geom.angles, dtype=np.float64)
        self._cos = np.cos(self._ang)
        self._sin = np.sin(self._ang)
        self._g = _Geom({"parallel": 0, "fan": 1, "fan_arc": 2}[geom.beam], geom.nx, geom.ny, float(geom.pixel),
                        geom.n_angles, _dptr(self._ang), geom.n_det, float(geom.det_width),
                        float(geom.sod), float(geom.sdd), _dptr(self._cos), _dptr(self._sin))
        self.n = geom.nx * geom.ny
        self.m = geom.n_angles * geom.n_det
        self.lib = _load()
        self.calls = {"A": 0, "B": 0, "AT": 0, "BT": 0}

    def _apply(self, name, v, n_in, n_out, key):
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
        if v.size != n_in:
            raise ValueError(f"{key}: expected {n_in} entries, got {v.size}")
        out = np.empty(n_out)
        getattr(self.lib, name)(ctypes.byref(self._g), _dptr(v), _dptr(out))
        self.calls[key] += 1
        return out

    def A(self, x):
        """Sinogram (n_angles*n_det, angle-major) = A x."""
        return self._apply("og_forward", x, self.n, self.m, "A")

    def AT(self, y):
        return self._apply("og_forward_T", y, self.m, self.n, "AT")

    def B(self, y):
        """Image (ny*nx, row-major) = B y."""
        return self._apply("og_back", y, self.m, self.n, "B")

    def BT(self, x):
        return self._apply("og_back_T", x, self.n, self.m, "BT")

    # single entries
    def A_ray(self, x, a, d):
        x = np.ascontiguousarray(x, dtype=np.float64)
        return self.lib.og_forward_ray(ctypes.byref(self._g), _dptr(x), int(a), int(d))

    def B_pixel(self, y, i, j):
        y = np.ascontiguousarray(y, dtype=np.float64)
        return self.lib.og_back_pixel(ctypes.byref(self._g), _dptr(y), int(i), int(j))

    def AT_pixel(self, y, i, j):
        y = np.ascontiguousarray(y, dtype=np.float64)
        return self.lib.og_forward_T_pixel(ctypes.byref(self._g), _dptr(y), int(i), int(j))

    def BT_ray(self, x, a, d):
        x = np.ascontiguousarray(x, dtype=np.float64)
        return self.lib.og_back_T_ray(ctypes.byref(self._g), _dptr(x), int(a), int(d))


def threads() -> int:
    """Threads the oracle's parallel loops use (OMP_NUM_THREADS, default all cores)."""
    return int(_load().og_threads())


def set_threads(n: int) -> None:
    """Set the oracle's thread count for later calls (results do not depend on it)."""
    _load().og_set_threads(int(n))
