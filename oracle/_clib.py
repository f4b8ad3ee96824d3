"""ctypes binding of oracle.c (test infrastructure; see oracle/__init__.py)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from .build import build_oracle

_lib = None

_D = C.POINTER(C.c_double)
_U32 = C.POINTER(C.c_uint32)


class _OrcChain(C.Structure):
    _fields_ = [("n", C.c_int), ("sigma", _D), ("eps", _D), ("q", _D), ("mass", _D),
                ("kb", C.c_double), ("r0", C.c_double), ("ktheta", C.c_double),
                ("theta0", C.c_double), ("dih_k", _D), ("dih_phase", _D),
                ("ke", C.c_double), ("nonbonded", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build_oracle())
        L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
        L.orc_philox_bulk.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_long, _U32, _D]
        L.orc_chain_energy.argtypes = [C.POINTER(_OrcChain), _D, C.c_double, C.c_double, _D]
        L.orc_chain_energy.restype = C.c_double
        L.orc_chain_rc.argtypes = [C.POINTER(_OrcChain), _D]
        L.orc_chain_rc.restype = C.c_double
        L.orc_chain_forces.argtypes = [C.POINTER(_OrcChain), _D, C.c_double, C.c_double, _D]
        L.orc_chain_kinetic.argtypes = [C.POINTER(_OrcChain), _D]
        L.orc_chain_kinetic.restype = C.c_double
        L.orc_chain_init_velocities.argtypes = [C.POINTER(_OrcChain), C.c_double, C.c_uint64,
                                                C.c_uint32, _D]
        L.orc_chain_run.argtypes = [C.POINTER(_OrcChain), C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_long, C.c_long, C.c_long,
                                    C.c_uint64, C.c_uint32, _D, _D, C.c_int, _D]
        L.orc_chain_run.restype = C.c_long
        L.orc_chain_run_from.argtypes = [C.POINTER(_OrcChain), C.c_double, C.c_double, C.c_double,
                                         C.c_double, C.c_double, C.c_long, C.c_long, C.c_long, C.c_long,
                                         C.c_uint64, C.c_uint32, _D, _D, C.c_int, _D]
        L.orc_chain_run_from.restype = C.c_long
        L.orc_od1d_force.argtypes = [C.c_double] * 4
        L.orc_od1d_force.restype = C.c_double
        L.orc_od1d_run.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_long, C.c_long, C.c_long, C.c_uint64,
                                   C.c_uint32, C.c_double, _D, _D]
        L.orc_od1d_run.restype = C.c_long
        L.orc_od1d_run_from.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                        C.c_double, C.c_long, C.c_long, C.c_long, C.c_long, C.c_uint64,
                                        C.c_uint32, C.c_double, _D, _D]
        L.orc_od1d_run_from.restype = C.c_long
        L.orc_chain_smd.argtypes = [C.POINTER(_OrcChain), C.c_double, C.c_double, C.c_double, C.c_double,
                                    C.c_double, C.c_double, C.c_long, C.c_long, C.c_long, C.c_uint64, C.c_uint32,
                                    _D, _D, _D, _D]
        L.orc_chain_smd.restype = C.c_long
        L.orc_od1d_smd.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                   C.c_double, C.c_long, C.c_long, C.c_long, C.c_uint64, C.c_uint32, C.c_double,
                                   _D, _D]
        L.orc_od1d_smd.restype = C.c_long
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), o.ctypes.data_as(_U32))
    return o


def philox_bulk(seed, c0, c1, c2, c3, n):
    """n consecutive blocks (c0 + i, c1, c2, c3): raw uint32 [n, 4], normals [n, 4]."""
    raw = np.zeros((n, 4), dtype=np.uint32)
    nor = np.zeros((n, 4), dtype=np.float64)
    lib().orc_philox_bulk(seed, c0, c1, c2, c3, n, raw.ctypes.data_as(_U32), _dp(nor))
    return raw, nor


class Chain:
    """Oracle view of a ChainParams (keeps the FP64 arrays alive)."""

    def __init__(self, p):
        self.p = p
        self._arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in
                      (p.sigma, p.epsilon, p.charge, p.mass, p.dih_k, p.dih_phase)]
        s, e, q, m, dk, dph = self._arrs
        self.s = _OrcChain(p.n, _dp(s), _dp(e), _dp(q), _dp(m), p.kb, p.r0, p.ktheta, p.theta0,
                           _dp(dk), _dp(dph), p.ke, int(p.nonbonded))
        self.n = p.n

    def energy(self, r, lam, k):
        r = np.ascontiguousarray(r, dtype=np.float64)
        parts = np.zeros(6)
        e = lib().orc_chain_energy(C.byref(self.s), _dp(r), lam, k, _dp(parts))
        return e, parts

    def forces(self, r, lam, k):
        r = np.ascontiguousarray(r, dtype=np.float64)
        f = np.zeros_like(r)
        lib().orc_chain_forces(C.byref(self.s), _dp(r), lam, k, _dp(f))
        return f

    def rc(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        return lib().orc_chain_rc(C.byref(self.s), _dp(r))

    def kinetic(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64)
        return lib().orc_chain_kinetic(C.byref(self.s), _dp(v))

    def init_velocities(self, kT, seed, uid):
        v = np.zeros((self.n, 3))
        lib().orc_chain_init_velocities(C.byref(self.s), kT, seed, uid, _dp(v))
        return v

    def run(self, r0, lam, k, kT, dt, gamma, n_steps, n_equil, stride, seed, uid,
            v0=None, step0=0):
        """One replica in one window (time steps numbered from step0);
        returns (samples, r_final, v_final).  Velocities are drawn when v0 is
        None."""
        r = np.array(r0, dtype=np.float64, order="C", copy=True)
        v = np.zeros_like(r) if v0 is None else np.array(v0, dtype=np.float64, order="C", copy=True)
        n_samp = max(0, (n_steps - n_equil) // stride)
        out = np.zeros(max(n_samp, 1))
        ns = lib().orc_chain_run_from(C.byref(self.s), lam, k, kT, dt, gamma, step0, n_steps, n_equil, stride,
                                      seed, uid, _dp(r), _dp(v), int(v0 is None), _dp(out))
        if ns < 0:
            raise FloatingPointError("oracle chain run became non-finite")
        return out[:ns], r, v

    def smd(self, r0, lam1, vdt, k, kT, dt, gamma, n_steps, n_equil, stride, seed, uid):
        """Constant-velocity pull of one replica: (x records, work records,
        r_final, v_final)."""
        r = np.array(r0, dtype=np.float64, order="C", copy=True)
        v = np.zeros_like(r)
        n = max(0, (n_steps - n_equil) // stride)
        xo, wo = np.zeros(max(n, 1)), np.zeros(max(n, 1))
        ns = lib().orc_chain_smd(C.byref(self.s), lam1, vdt, k, kT, dt, gamma, n_steps, n_equil, stride, seed, uid,
                                 _dp(r), _dp(v), _dp(xo), _dp(wo))
        if ns < 0:
            raise FloatingPointError("oracle chain run became non-finite")
        return xo[:ns], wo[:ns], r, v


def od1d_force(a, lam, k, x):
    return lib().orc_od1d_force(a, lam, k, x)


def od1d_smd(a, lam1, vdt, k, kT, gamma, dt, n_steps, n_equil, stride, seed, uid, x0):
    """Constant-velocity pull of the 1D model: (x records, work records)."""
    n = max(0, (n_steps - n_equil) // stride)
    xo, wo = np.zeros(max(n, 1)), np.zeros(max(n, 1))
    ns = lib().orc_od1d_smd(a, lam1, vdt, k, kT, gamma, dt, n_steps, n_equil, stride, seed, uid, x0, _dp(xo), _dp(wo))
    return xo[:ns], wo[:ns]


def od1d_run(a, lam, k, kT, gamma, dt, n_steps, n_equil, stride, seed, uid, x0, step0=0):
    n_samp = max(0, (n_steps - n_equil) // stride)
    out = np.zeros(max(n_samp, 1))
    xf = C.c_double(0.0)
    ns = lib().orc_od1d_run_from(a, lam, k, kT, gamma, dt, step0, n_steps, n_equil, stride, seed, uid, x0,
                                 _dp(out), C.byref(xf))
    return out[:ns], xf.value
