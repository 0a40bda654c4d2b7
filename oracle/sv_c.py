"""ctypes front of the plain C state-vector oracle (sv.c); test infrastructure only.

`final_state(circuit)` returns U_L ... U_1 |0^n> as a flat complex128 array of 2^n
entries (qubit 0 the most significant index bit), the same quantity and conventions as
`statevector.final_state` without cuts, for registers too large for the numpy version
(n = 30 takes 16 GiB).  The library is compiled with gcc on first use.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "sv.c")
LIB = os.path.join(HERE, "_build", "libsv.so")

_lib = None


def compile_library() -> str:
    """gcc -O2 -fopenmp; rebuilt when sv.c is newer than the library."""
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", LIB, SRC], check=True)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(compile_library())
        lib.sv_final_state.restype = ctypes.c_int
        lib.sv_final_state.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p]
        _lib = lib
    return _lib


def final_state(circuit) -> np.ndarray:
    arity, qubits, mats = circuit.gate_array()
    arity = np.ascontiguousarray(arity, dtype=np.int32)
    qubits = np.ascontiguousarray(qubits, dtype=np.int32)
    mats = np.ascontiguousarray(mats, dtype=np.float64)
    psi = np.empty(1 << circuit.n_qubits, dtype=np.complex128)
    rc = _load().sv_final_state(circuit.n_qubits, len(arity), arity.ctypes.data, qubits.ctypes.data,
                                mats.ctypes.data, psi.ctypes.data)
    if rc != 0:
        raise ValueError("sv_final_state: bad circuit")
    return psi


def amplitudes(circuit, bitstrings) -> np.ndarray:
    """<x|psi> for each row x of `bitstrings` (entry q = bit of qubit q)."""
    bits = np.atleast_2d(np.asarray(bitstrings, dtype=np.int64))
    w = 1 << np.arange(circuit.n_qubits - 1, -1, -1, dtype=np.int64)
    return final_state(circuit)[bits @ w]
