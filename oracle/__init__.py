"""The oracle: a plain, slow FP64 CPU reference for the batched chemistry solve.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / --impl reference legs of bench.py may import it.  It shares no
code with the CUDA path (its own JSON reading in mech.py, its own numerics in
camp_oracle.c, its own integer-structure enumeration in structure.py).

Every function follows the CAMP paper (arXiv 2111.07436): the forcing and
Jacobian sums of Sect. 2.4.2, the rate constants of Table 2, and a
variable-order BDF with Newton iteration as named in Sect. 2.4.1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import mech as _mech
from . import structure as _structure

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libcamp_oracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force=False):
    """Compile camp_oracle.c with gcc (no FMA contraction, so x86 and Arm agree)."""
    src = os.path.join(_HERE, "camp_oracle.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
                           "-pthread", src, "-o", tmp, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        mp = ctypes.POINTER(_mech.OmMech)
        L.om_rate_constants.argtypes = [mp, _dp, _dp, _dp]
        L.om_forcing.argtypes = [mp, _dp, _dp, _dp, _dp]
        L.om_jacobian.argtypes = [mp, _dp, _dp, _dp, _dp]
        L.om_forcing_env.argtypes = [mp, _dp, _dp, _dp, _dp, _dp]
        L.om_jacobian_env.argtypes = [mp, _dp, _dp, _dp, _dp, _dp]
        L.om_water.argtypes = [mp, _dp, _dp, _dp]
        L.om_lu_factor.argtypes = [ctypes.c_int, _dp, _ip]
        L.om_lu_factor.restype = ctypes.c_int
        L.om_lu_solve.argtypes = [ctypes.c_int, _dp, _ip, _dp]
        L.om_bdf_coefficients.argtypes = [ctypes.c_int, _dp, _dp]
        L.om_integrate.argtypes = [mp, _dp, _dp, ctypes.c_double, ctypes.c_double, _dp,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_double, _ip, _dp]
        L.om_integrate.restype = ctypes.c_int
        L.om_solve.argtypes = [mp, ctypes.c_int64, _dp, _dp, ctypes.c_double, ctypes.c_double,
                               _dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _ip, _ip, _dp,
                               ctypes.c_int]
        L.om_bdf_step.argtypes = [mp, _dp, _dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                  _dp, ctypes.c_int, _dp, _dp]
        L.om_bdf_step.restype = ctypes.c_double
    return _lib


def _opt(step, size):
    """An optional in/out float64 array as a pointer (None -> NULL)."""
    if step is None:
        return None
    if not (isinstance(step, np.ndarray) and step.dtype == np.float64 and step.flags.c_contiguous
            and step.size == size):
        raise ValueError("step must be a contiguous float64 array of one value per cell")
    return _p(step)


def _p(a, t=_dp):
    return a.ctypes.data_as(t)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def bdf_coefficients(q):
    """(l[0..q], local-error constant) of the order-q BDF in Nordsieck form."""
    l = np.zeros(7)
    c = np.zeros(1)
    lib().om_bdf_coefficients(q, _p(l), _p(c))
    return l[: q + 1].copy(), float(c[0])


def dense_lu_solve(A, b):
    """Solve A x = b with the oracle's partial-pivot LU."""
    A = _f64(A).copy()
    x = _f64(b).copy()
    n = A.shape[0]
    piv = np.zeros(n, dtype=np.int32)
    if lib().om_lu_factor(n, _p(A), _p(piv, _ip)):
        raise np.linalg.LinAlgError("singular")
    lib().om_lu_solve(n, _p(A), _p(piv, _ip), _p(x))
    return x


class Mechanism:
    """A parsed mechanism plus the oracle's numerics on it."""

    def __init__(self, text):
        self.m = _mech.parse(text)
        self._c, self._keep = _mech.to_ctypes(self.m)
        self.n = self.m.n
        self.n_env = self.m.n_env
        self.n_rxn = len(self.m.processes)

    @property
    def _ptr(self):
        return ctypes.byref(self._c)

    def structure(self):
        return _structure.structure(self.m)

    def rate_constants(self, env):
        env = _f64(env)
        kf = np.zeros(self.n_rxn)
        kr = np.zeros(self.n_rxn)
        lib().om_rate_constants(self._ptr, _p(env), _p(kf), _p(kr))
        return kf, kr

    @property
    def has_water(self):
        """True when a ZSR water parameter makes the sections' liquid volume a
        function of the state (then forcing and jacobian need the cell's env)."""
        return bool(self.m.electrolytes)

    def _env_for(self, env):
        if env is None:
            if self.has_water:
                raise ValueError("a mechanism with a water parameter needs the cell's env")
            return np.zeros(max(1, self.n_env))
        return _f64(env)

    def forcing(self, kf, kr, y, env=None):
        """f(y) from the rate constants (and, with a water parameter, the
        cell's env for the liquid volume at y)."""
        f = np.zeros(self.n)
        lib().om_forcing_env(self._ptr, _p(self._env_for(env)), _p(_f64(kf)), _p(_f64(kr)),
                             _p(_f64(y)), _p(f))
        return f

    def jacobian(self, kf, kr, y, env=None):
        """df/dy, dense [n, n]; with a water parameter the chain-rule term of
        Sect. 2.2.2 is included."""
        J = np.zeros((self.n, self.n))
        lib().om_jacobian_env(self._ptr, _p(self._env_for(env)), _p(_f64(kf)), _p(_f64(kr)),
                              _p(_f64(y)), _p(J))
        return J

    def water(self, env, y):
        """Liquid volume of every section at y [m^3 per m^3 air]."""
        L = np.zeros(max(1, self.m.n_sections))
        lib().om_water(self._ptr, _p(_f64(env)), _p(_f64(y)), _p(L))
        return L[: self.m.n_sections]

    def _atol(self, atol):
        a = np.atleast_1d(_f64(atol))
        if a.size not in (1, self.n):
            raise ValueError("atol must be a scalar or one value per species")
        return a

    def integrate(self, y0, env, dt, rtol, atol, max_steps=10000, hmin_frac=1e-10, step=None):
        """One cell: returns (y, status, stats[steps, newton, jac, errfail]).
        step: None (cold start) or a 1-element float64 array, in/out: the
        warm-start step size (see camp_oracle.c, integrate_cell)."""
        y = _f64(y0).copy()
        a = self._atol(atol)
        st = np.zeros(4, dtype=np.int32)
        s = lib().om_integrate(self._ptr, _p(_f64(env)), _p(y), dt, rtol, _p(a), a.size,
                               max_steps, hmin_frac, _p(st, _ip), _opt(step, 1))
        return y, s, st

    def solve(self, y0, env, dt, rtol, atol, threads=None, max_steps=10000, hmin_frac=1e-10,
              step=None):
        """Many cells, y0 [C, n] and env [C, n_env]: returns (y, status, stats [C, 4]).
        step: None (cold starts) or a float64 array [C], in/out warm-start
        step sizes."""
        y = _f64(y0).copy()
        env = _f64(env)
        C = y.shape[0]
        if y.shape != (C, self.n) or env.shape != (C, self.n_env):
            raise ValueError("shape mismatch")
        a = self._atol(atol)
        status = np.zeros(C, dtype=np.int32)
        stats = np.zeros((C, 4), dtype=np.int32)
        threads = threads or os.cpu_count() or 1
        lib().om_solve(self._ptr, C, _p(y), _p(env), dt, rtol, _p(a), a.size, max_steps,
                       hmin_frac, _p(status, _ip), _p(stats, _ip), _opt(step, C), threads)
        return y, status, stats

    def bdf_step(self, env, z, q, h, rtol, atol):
        """One fixed (h, q) step from Nordsieck array z [(q+1), n]."""
        z = _f64(z)
        a = self._atol(atol)
        zo = np.zeros_like(z)
        e = np.zeros(self.n)
        err = lib().om_bdf_step(self._ptr, _p(_f64(env)), _p(z), q, h, rtol, _p(a), a.size,
                                _p(zo), _p(e))
        return zo, e, err
