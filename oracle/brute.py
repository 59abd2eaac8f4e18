"""ctypes loader for oracle/brute.c (brute-force Eq. 5 with Neumaier sums).

The C file is compiled with gcc into oracle/_build/ on first use (or by
__graft_entry__.build()).  -ffp-contract=off keeps the arithmetic identical on
x86-64 and aarch64 hosts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brute.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_OUT_DIR, "libttq_oracle.so")
_lib = None

FAMILY = {"C": 0, "D": 1, "E": 2, "TEST": 3}
FORM = {"rn": 0, "cube": 1}


def build(force: bool = False) -> str:
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.ttq_oracle_brute.restype = ctypes.c_double
        lib.ttq_oracle_brute.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, dp, dp]
        lib.ttq_oracle_brute_sym.restype = ctypes.c_double
        lib.ttq_oracle_brute_sym.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        lib.ttq_oracle_g.restype = None
        lib.ttq_oracle_g.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int64, dp, dp]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def brute_sum(problem) -> float:
    """sum over all multi-indices of prod w * g (no family constant)."""
    lib = _load()
    N = np.array(problem.N, dtype=np.int32)
    nodes = np.ascontiguousarray(np.concatenate(problem.nodes), dtype=np.float64)
    weights = np.ascontiguousarray(np.concatenate(problem.weights), dtype=np.float64)
    return lib.ttq_oracle_brute(FAMILY[problem.family], FORM[problem.form], problem.n, problem.d,
                                N.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(nodes), _dp(weights))


def brute_sum_symmetric(problem) -> float:
    """Same sum over sorted tuples with multinomial counts (C/D, R^n form, one rule)."""
    if problem.form != "rn" or problem.family not in ("C", "D"):
        raise ValueError("symmetric reduction needs C/D in the R^n form")
    for k in range(1, problem.d):
        if not (np.array_equal(problem.nodes[k], problem.nodes[0])
                and np.array_equal(problem.weights[k], problem.weights[0])):
            raise ValueError("symmetric reduction needs the same rule in every mode")
    lib = _load()
    nodes = np.ascontiguousarray(problem.nodes[0], dtype=np.float64)
    weights = np.ascontiguousarray(problem.weights[0], dtype=np.float64)
    return lib.ttq_oracle_brute_sym(FAMILY[problem.family], problem.n, problem.d, len(nodes),
                                    _dp(nodes), _dp(weights))


def g_c(family: str, form: str, n: int, X: np.ndarray) -> np.ndarray:
    lib = _load()
    X = np.ascontiguousarray(X, dtype=np.float64)
    out = np.empty(X.shape[0])
    lib.ttq_oracle_g(FAMILY[family], FORM[form], n, X.shape[1], X.shape[0], _dp(X), _dp(out))
    return out
