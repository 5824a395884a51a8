"""Python entry to the FP64 direct-sum oracle (``direct.c``), Eq. (1), and
the gradient of its potential with respect to the target position.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Pinned by tests/test_oracle_direct.py against closed forms (unit charges on
the vertices of a cube), Newton's shell theorem, the kernel's symmetry and
homogeneity, and brute-force enumeration in pure Python; the gradient by
tests/test_oracle_gradient.py against the closed form of one charge, central
differences of the potential, symmetry and a vanishing Laplacian.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "direct.c")
_LIB = os.path.join(_HERE, "liboracle_direct.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile direct.c into liboracle_direct.so with gcc (OpenMP)."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_direct_sum.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int,
                                          dp, ctypes.c_int64, dp]
        lib.oracle_direct_sum.restype = None
        lib.oracle_direct_gradient.argtypes = [dp, dp, ctypes.c_int64, ctypes.c_int,
                                               dp, ctypes.c_int64, dp]
        lib.oracle_direct_gradient.restype = None
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the direct sum uses."""
    return _load().oracle_num_threads()


def direct_sum(sources, charges, targets=None):
    """phi_j = sum_{i: x_i != y_j} q_i / (4 pi |x_i - y_j|) in FP64.

    sources (ns,3), charges (ns,) or (ns,nrhs), targets (nt,3) (default: the
    sources).  Returns (nt,) or (nt,nrhs) matching the charges' rank.
    """
    src = np.ascontiguousarray(sources, dtype=np.float64)
    q = np.asarray(charges, dtype=np.float64)
    vec = q.ndim == 1
    q = np.ascontiguousarray(q.reshape(len(src), -1))
    tgt = src if targets is None else np.ascontiguousarray(targets, dtype=np.float64)
    nrhs = q.shape[1]
    phi = np.empty((len(tgt), nrhs), dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    if len(tgt) and nrhs:
        _load().oracle_direct_sum(src.ctypes.data_as(dp), q.ctypes.data_as(dp),
                                  len(src), nrhs, tgt.ctypes.data_as(dp),
                                  len(tgt), phi.ctypes.data_as(dp))
    return phi[:, 0] if vec else phi


def direct_gradient(sources, charges, targets=None):
    """grad_j = sum_{i: x_i != y_j} q_i (x_i - y_j) / (4 pi |x_i - y_j|^3) in
    FP64: the gradient of direct_sum's potential with respect to the target
    position (the field is minus this).

    sources (ns,3), charges (ns,) or (ns,nrhs), targets (nt,3) (default: the
    sources).  Returns (nt,3) or (nt,nrhs,3) matching the charges' rank.
    """
    src = np.ascontiguousarray(sources, dtype=np.float64)
    q = np.asarray(charges, dtype=np.float64)
    vec = q.ndim == 1
    q = np.ascontiguousarray(q.reshape(len(src), -1))
    tgt = src if targets is None else np.ascontiguousarray(targets, dtype=np.float64)
    nrhs = q.shape[1]
    grad = np.empty((len(tgt), nrhs, 3), dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    if len(tgt) and nrhs:
        _load().oracle_direct_gradient(src.ctypes.data_as(dp), q.ctypes.data_as(dp),
                                       len(src), nrhs, tgt.ctypes.data_as(dp),
                                       len(tgt), grad.ctypes.data_as(dp))
    return grad[:, 0, :] if vec else grad
