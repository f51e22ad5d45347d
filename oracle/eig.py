"""Eigenvalues of the state matrix and the stability statistics (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Section II-B-2: a scenario is small-signal unstable when some eigenvalue has a
non-negative real part.  The arithmetic is in ``eig.c`` (balancing, Householder
Hessenberg, Francis double-shift QR); this module loads it (compiling it with
gcc on first use) and computes the decision statistics.

The state matrix handed in is the one with rotor angles referred to one machine
(see ``oracle/dynamics``), which has no structural zero mode, so the statistics
run over every eigenvalue.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eig.c")
_LIB = os.path.join(_HERE, "_eig.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile eig.c into a shared object beside it (plain gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_eigvals.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int)]
        lib.oracle_eigvals.restype = ctypes.c_int
        lib.oracle_hessenberg.argtypes = [ctypes.c_int, dp, ctypes.c_int]
        lib.oracle_hessenberg.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def eigvals(A, balance: bool = True):
    """Eigenvalues of a real square matrix; returns (complex array, ok, sweeps)."""
    a = np.array(A, dtype=np.float64, order="C", copy=True)
    n = a.shape[0]
    wr = np.zeros(n)
    wi = np.zeros(n)
    sweeps = ctypes.c_int(0)
    rc = _load().oracle_eigvals(n, _dp(a), _dp(wr), _dp(wi), int(balance), ctypes.byref(sweeps))
    return wr + 1j * wi, rc == 0, sweeps.value


def hessenberg(A, balance: bool = True):
    a = np.array(A, dtype=np.float64, order="C", copy=True)
    _load().oracle_hessenberg(a.shape[0], _dp(a), int(balance))
    return a


def stability_stats(lam):
    """(max real part, minimum damping ratio) over all eigenvalues; the damping
    ratio of s is -Re(s)/|s| (1 for s = 0)."""
    lam = np.asarray(lam)
    if lam.size == 0:
        return -np.inf, np.inf
    mag = np.abs(lam)
    zeta = np.where(mag > 0, -lam.real / np.where(mag > 0, mag, 1.0), 1.0)
    return float(np.max(lam.real)), float(np.min(zeta))
