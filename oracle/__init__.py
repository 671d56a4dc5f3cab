"""ctypes loader for the FP64 CPU oracle (``kx_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by tests, by the smoke check and by the
benchmark's CPU-baseline leg, never by the library itself.  The oracle shares
no code with the GPU path.  ``build()`` compiles it with ``-O2
-ffp-contract=off`` so that no multiply-add is fused behind the formulas'
backs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kx_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib: Optional[ctypes.CDLL] = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC",
                               "-pthread", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def configure(L: ctypes.CDLL) -> ctypes.CDLL:
    """Declare the argument types of the oracle's C entry points on a loaded library."""
    L.ora_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]
    L.ora_free.argtypes = [ctypes.c_void_p]
    L.ora_free.restype = None
    L.ora_sizes.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.ora_species_thermo.argtypes = [ctypes.c_void_p, ctypes.c_double] + [_D] * 5
    L.ora_production_rates.argtypes = [ctypes.c_void_p, _D, _D, _D, ctypes.c_long, _D, ctypes.c_long, ctypes.c_int]
    L.ora_reaction_detail.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _D, _D]
    L.ora_rates_of_progress.argtypes = [ctypes.c_void_p, _D, _D, _D, ctypes.c_long, _D, ctypes.c_long,
                                        ctypes.c_int]
    L.ora_reaction_gross.argtypes = [ctypes.c_void_p, _D, _D, _D, ctypes.c_long, _D, ctypes.c_long, ctypes.c_int]
    L.ora_gross_scale.argtypes = [ctypes.c_void_p, _D, _D, _D, ctypes.c_long, _D, ctypes.c_long, ctypes.c_int]
    L.ora_thermo.argtypes = [ctypes.c_void_p, _D, _D, _D, ctypes.c_long, _D, _D, ctypes.c_long, ctypes.c_int]
    L.ora_species_transport.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _D, _D, _D]
    L.ora_transport.argtypes = [ctypes.c_void_p, _D, _D, _D, ctypes.c_long, _D, _D, _D, ctypes.c_long,
                                ctypes.c_int]
    L.ora_wilke_phi.argtypes = [ctypes.c_void_p, ctypes.c_double, _D]
    L.ora_jacobian.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _D, _D]
    return L


def build_variant(source: str, out_so: str) -> ctypes.CDLL:
    """Compile another oracle source text (the tests' planted mistakes, on the
    CPU) with the oracle's own flags and load it."""
    src = out_so + ".cpp"
    with open(src, "w") as f:
        f.write(source)
    subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-shared", "-fPIC", "-pthread",
                           "-o", out_so, src])
    return configure(ctypes.CDLL(out_so))


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = configure(ctypes.CDLL(build()))
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


DETAIL_FIELDS = ("kf", "kr", "Kc", "Rf", "Rr", "c", "X", "Pr", "F", "q")


class Oracle:
    """One mechanism loaded into the oracle.  Arrays are SoA float64:
    T[n], p[n], Y[ns, n] (species-major)."""

    def __init__(self, path: str, nthreads: int = 1, library: Optional[ctypes.CDLL] = None):
        self.L = library if library is not None else lib()
        h = ctypes.c_void_p()
        if self.L.ora_load(path.encode(), ctypes.byref(h)) != 0:
            raise RuntimeError(f"oracle cannot load {path}")
        self.h = h
        ns, nr = ctypes.c_int(), ctypes.c_int()
        self.L.ora_sizes(h, ctypes.byref(ns), ctypes.byref(nr))
        self.ns, self.nr = ns.value, nr.value
        self.nthreads = nthreads

    def __del__(self):
        if getattr(self, "h", None) is not None:
            self.L.ora_free(self.h)
            self.h = None

    @staticmethod
    def _state(T, p, Y):
        T = np.ascontiguousarray(T, np.float64); p = np.ascontiguousarray(p, np.float64)
        Y = np.ascontiguousarray(Y, np.float64)
        return T, p, Y

    def species_thermo(self, T: float):
        out = [np.zeros(self.ns) for _ in range(5)]
        self.L.ora_species_thermo(self.h, float(T), *[_p(o) for o in out])
        return dict(zip(("cp_R", "h_RT", "s_R", "g_RT", "g_closed"), out))

    def production_rates(self, T, p, Y, nthreads: Optional[int] = None):
        T, p, Y = self._state(T, p, Y)
        n = T.shape[0]
        w = np.zeros((self.ns, n))
        self.L.ora_production_rates(self.h, _p(T), _p(p), _p(Y), n, _p(w), n, nthreads or self.nthreads)
        return w

    def rates_of_progress(self, T, p, Y, nthreads: Optional[int] = None):
        T, p, Y = self._state(T, p, Y)
        n = T.shape[0]
        q = np.zeros((self.nr, n))
        self.L.ora_rates_of_progress(self.h, _p(T), _p(p), _p(Y), n, _p(q), n, nthreads or self.nthreads)
        return q

    def reaction_gross(self, T, p, Y, nthreads: Optional[int] = None):
        T, p, Y = self._state(T, p, Y)
        n = T.shape[0]
        g = np.zeros((self.nr, n))
        self.L.ora_reaction_gross(self.h, _p(T), _p(p), _p(Y), n, _p(g), n, nthreads or self.nthreads)
        return g

    def reaction_detail(self, T: float, p: float, Y):
        Y = np.ascontiguousarray(Y, np.float64)
        out = np.zeros((self.nr, len(DETAIL_FIELDS)))
        self.L.ora_reaction_detail(self.h, float(T), float(p), _p(Y), _p(out))
        return {f: out[:, i].copy() for i, f in enumerate(DETAIL_FIELDS)}

    def gross_scale(self, T, p, Y, nthreads: Optional[int] = None):
        T, p, Y = self._state(T, p, Y)
        n = T.shape[0]
        s = np.zeros(n)
        self.L.ora_gross_scale(self.h, _p(T), _p(p), _p(Y), n, _p(s), n, nthreads or self.nthreads)
        return s

    def thermo(self, T, p, Y, nthreads: Optional[int] = None):
        T, p, Y = self._state(T, p, Y)
        n = T.shape[0]
        cp, h = np.zeros(n), np.zeros(n)
        self.L.ora_thermo(self.h, _p(T), _p(p), _p(Y), n, _p(cp), _p(h), n, nthreads or self.nthreads)
        return cp, h

    def species_transport(self, T: float, p: float):
        eta, lam, D = np.zeros(self.ns), np.zeros(self.ns), np.zeros((self.ns, self.ns))
        self.L.ora_species_transport(self.h, float(T), float(p), _p(eta), _p(lam), _p(D))
        return eta, lam, D

    def wilke_phi(self, T: float):
        phi = np.zeros((self.ns, self.ns))
        self.L.ora_wilke_phi(self.h, float(T), _p(phi))
        return phi

    def transport(self, T, p, Y, nthreads: Optional[int] = None):
        T, p, Y = self._state(T, p, Y)
        n = T.shape[0]
        mu, lam, D = np.zeros(n), np.zeros(n), np.zeros((self.ns, n))
        self.L.ora_transport(self.h, _p(T), _p(p), _p(Y), n, _p(mu), _p(lam), _p(D), n, nthreads or self.nthreads)
        return mu, lam, D

    def jacobian(self, T: float, p: float, Y):
        Y = np.ascontiguousarray(Y, np.float64)
        J = np.zeros((self.ns, self.ns + 1))
        self.L.ora_jacobian(self.h, float(T), float(p), _p(Y), _p(J))
        return J
