"""ctypes binding of the C boundary (include/tnc.h).  Argument marshalling only: every
step of the contraction path runs in the library's CUDA kernels.

The functions keep the C names (`tnc_amplitudes`, `tnc_contract`, ...).  The classes
`Plan` and `Context` wrap the handles for convenience.  The library is loaded from this
package directory; when it is missing every call raises (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import json
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtnc.so")

TNC_OK = 0
TNC_E_INVALID_ARG = 1
TNC_E_OOM = 2
TNC_E_CUDA = 3
TNC_E_TIMEOUT = 4
TNC_E_PLAN = 5
TNC_E_UNSUPPORTED = 6
TNC_E_IO = 7

TNC_C64 = 0
TNC_CHALF = 1
TNC_CBF16 = 2
PRECISIONS = {"c64": TNC_C64, "chalf": TNC_CHALF, "cbf16": TNC_CBF16}


class TncError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"tnc status {status}: {msg}")
        self.status = status


class tnc_plan_opts(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64),
        ("trials", C.c_int32),
        ("log2_cap", C.c_int32),
        ("slices_min", C.c_int32),
        ("slices_max", C.c_int32),
        ("temperature", C.c_double),
        ("mode", C.c_int32),
        ("objective", C.c_int32),
        ("slicing", C.c_int32),
        ("branch_exchange", C.c_int32),
        ("cluster_chains", C.c_int32),
    ]


class tnc_plan_info(C.Structure):
    _fields_ = [
        ("log2_flops_per_slice", C.c_double),
        ("log2_total_flops", C.c_double),
        ("slicing_overhead", C.c_double),
        ("max_log2_size", C.c_int32),
        ("n_sliced", C.c_int32),
        ("n_steps", C.c_int32),
        ("n_leaves", C.c_int32),
        ("n_open", C.c_int32),
        ("n_kernels", C.c_int32),
        ("n_gemm", C.c_int32),
        ("n_gepdot", C.c_int32),
        ("n_absorb", C.c_int32),
        ("n_fused", C.c_int32),
        ("narrow_max", C.c_double),
        ("model_seconds_per_slice", C.c_double),
        ("log2_executed_flops", C.c_double),
        ("log2_executed_flops_merged", C.c_double),
    ]


class tnc_tune_info(C.Structure):
    _fields_ = [
        ("steps_tuned", C.c_int32),
        ("steps_changed", C.c_int32),
        ("candidates", C.c_int32),
        ("reserved0", C.c_int32),
        ("seconds_default", C.c_double),
        ("seconds_tuned", C.c_double),
        ("reserved", C.c_double * 4),
    ]


class tnc_exec_opts(C.Structure):
    _fields_ = [
        ("precision", C.c_int32),
        ("wave", C.c_int32),
        ("use_graph", C.c_int32),
        ("fuse", C.c_int32),
        ("profile", C.c_int32),
        ("reserved", C.c_int32 * 3),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libtnc.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(the contraction path has no CPU fallback)"
        )
    lib = C.CDLL(path)
    vp, i32, i64, u8p = C.c_void_p, C.c_int32, C.c_int64, C.POINTER(C.c_uint8)
    sig = {
        "tnc_circuit_from_gates": [i32, i64, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_double), C.POINTER(vp)],
        "tnc_network_build": [vp, u8p, C.POINTER(vp)],
        "tnc_plan_greedy": [vp, C.POINTER(tnc_plan_opts), C.POINTER(vp)],
        "tnc_plan_get_info": [vp, C.POINTER(tnc_plan_info)],
        "tnc_plan_sliced_cuts": [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), i32],
        "tnc_circuit_random_grid": [i32, i32, i32, C.c_uint64, i32, C.POINTER(vp)],
        "tnc_circuit_export": [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32), C.POINTER(C.c_double), i64],
        "tnc_plan_slice_stats": [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int32),
                                 C.POINTER(C.c_double), i32],
        "tnc_plan_open_qubits": [vp, C.POINTER(C.c_int32), i32],
        "tnc_plan_describe": [vp, C.c_char_p, i64, C.POINTER(C.c_int64)],
        "tnc_plan_save": [vp, C.c_char_p],
        "tnc_plan_update_gates": [vp, i64, C.POINTER(C.c_double)],
        "tnc_plan_load": [C.c_char_p, C.POINTER(vp)],
        "tnc_context_create": [i32, C.POINTER(vp)],
        "tnc_amplitudes": [vp, vp, C.POINTER(tnc_exec_opts), u8p, i64, i64, i64, vp, vp],
        "tnc_amplitudes_ids": [vp, vp, C.POINTER(tnc_exec_opts), u8p, i64, C.POINTER(C.c_int64), i64, vp, vp],
        "tnc_adjoint": [vp, vp, C.POINTER(tnc_exec_opts), u8p, i64, vp, vp, vp, vp],
        "tnc_contract": [vp, i32, vp, i32, C.POINTER(C.c_int32), vp, i32, C.POINTER(C.c_int32), vp, i32,
                         C.POINTER(C.c_int32), C.POINTER(C.c_int32), vp],
        "tnc_sync": [vp],
        "tnc_contract_noalloc": [i32, vp, i32, C.POINTER(C.c_int32), vp, i32, C.POINTER(C.c_int32), vp, i32,
                                 C.POINTER(C.c_int32), C.POINTER(C.c_int32), vp],
        "tnc_profile_read": [vp, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_double),
                             C.POINTER(C.c_double), C.POINTER(C.c_int32), i32, C.POINTER(C.c_int32)],
        "tnc_autotune": [vp, vp, C.POINTER(tnc_exec_opts), u8p, i64, i64, i64, C.POINTER(tnc_tune_info)],
        "tnc_tune_save": [C.c_char_p],
        "tnc_tune_load": [C.c_char_p],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int32
    for name in ("tnc_circuit_destroy", "tnc_network_destroy", "tnc_plan_destroy", "tnc_context_destroy"):
        f = getattr(lib, name)
        f.argtypes = [vp]
        f.restype = None
    lib.tnc_tune_clear.argtypes = []
    lib.tnc_tune_clear.restype = None
    lib.tnc_tune_size.argtypes = []
    lib.tnc_tune_size.restype = C.c_int64
    lib.tnc_last_error.restype = C.c_char_p
    lib.tnc_last_error.argtypes = []
    lib.tnc_version.restype = C.c_char_p
    lib.tnc_version.argtypes = []
    _lib = lib
    return lib


def _check(status: int):
    if status != TNC_OK:
        raise TncError(status, _lib.tnc_last_error().decode())


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


# ------------------------------------------------------------------------- raw calls
def tnc_circuit_from_gates(n_qubits: int, arity: np.ndarray, qubits: np.ndarray, matrices: np.ndarray):
    lib = load_library()
    arity = np.ascontiguousarray(arity, dtype=np.int32)
    qubits = np.ascontiguousarray(qubits, dtype=np.int32).reshape(-1)
    matrices = np.ascontiguousarray(matrices, dtype=np.float64).reshape(-1)
    h = C.c_void_p()
    _check(lib.tnc_circuit_from_gates(n_qubits, len(arity), _i32p(arity), _i32p(qubits),
                                      matrices.ctypes.data_as(C.POINTER(C.c_double)), C.byref(h)))
    return h


def tnc_network_build(circuit, open_mask: Optional[np.ndarray]):
    lib = load_library()
    h = C.c_void_p()
    if open_mask is None:
        _check(lib.tnc_network_build(circuit, None, C.byref(h)))
    else:
        m = np.ascontiguousarray(open_mask, dtype=np.uint8)
        _check(lib.tnc_network_build(circuit, m.ctypes.data_as(C.POINTER(C.c_uint8)), C.byref(h)))
    return h


def tnc_plan_greedy(network, seed=1, trials=16, log2_cap=26, slices_min=0, slices_max=64, temperature=0.5, mode=0,
                    objective=0, slicing=0, branch_exchange=0, cluster_chains=0):
    lib = load_library()
    o = tnc_plan_opts(seed, trials, log2_cap, slices_min, slices_max, temperature, mode, objective, slicing,
                      branch_exchange, cluster_chains)
    h = C.c_void_p()
    _check(lib.tnc_plan_greedy(network, C.byref(o), C.byref(h)))
    return h


# ------------------------------------------------------------------------- wrappers
class GateList:
    """A circuit as the packed arrays of the C boundary (the layout of
    tnc_circuit_from_gates): arity (G,), qubits (G, 2), matrices (G, 32).  Plan.greedy
    takes it like any object with `n_qubits` and `gate_array()`."""

    def __init__(self, n_qubits: int, arity: np.ndarray, qubits: np.ndarray, matrices: np.ndarray):
        self.n_qubits = int(n_qubits)
        self.arity, self.qubits, self.matrices = arity, qubits, matrices

    def __len__(self) -> int:
        return len(self.arity)

    def gate_array(self):
        return self.arity, self.qubits, self.matrices


def circuit_export(handle) -> GateList:
    """The gates of a C circuit handle (tnc_circuit_export)."""
    lib = load_library()
    n, g = C.c_int32(), C.c_int64()
    _check(lib.tnc_circuit_export(handle, C.byref(n), C.byref(g), None, None, None, 0))
    arity = np.zeros(g.value, dtype=np.int32)
    qubits = np.zeros((g.value, 2), dtype=np.int32)
    mats = np.zeros((g.value, 32), dtype=np.float64)
    _check(lib.tnc_circuit_export(handle, None, None, _i32p(arity), _i32p(qubits),
                                  mats.ctypes.data_as(C.POINTER(C.c_double)), g.value))
    return GateList(n.value, arity, qubits, mats)


def random_grid(rows: int, cols: int, cycles: int, seed: int = 1, fsim_mode: str = "fixed") -> GateList:
    """The library's seeded random grid circuit (tnc_circuit_random_grid)."""
    lib = load_library()
    h = C.c_void_p()
    _check(lib.tnc_circuit_random_grid(rows, cols, cycles, seed, {"fixed": 0, "uniform": 1}[fsim_mode], C.byref(h)))
    try:
        return circuit_export(h)
    finally:
        lib.tnc_circuit_destroy(h)


class Plan:
    """A contraction plan (tree + slices + compiled steps) of a circuit's network."""

    def __init__(self, handle, n_qubits: int):
        self.h = handle
        self.n_qubits = n_qubits

    @classmethod
    def greedy(cls, circuit, open_qubits: Sequence[int] = (), seed: int = 1, trials: int = 16, log2_cap: int = 26,
               slices_min: int = 0, slices_max: int = 64, temperature: float = 0.5, mode: str = "greedy",
               objective: str = "flops", slicing: str = "eq1", branch_exchange: bool = False,
               cluster_chains: bool = False) -> "Plan":
        """Plan for an `inputs.Circuit` (gate list) with the given open output qubits.
        mode: "greedy" (balanced pairwise order), "stem" (one tensor absorbs leaves) or
        "split" (a seeded balanced bisection of the qubits; the indices between the two
        sides are sliced and each side is one stem absorbing fused blocks of gates).
        objective: which trial is kept -- "flops" (fewest multiply-adds) or "time" (least
        modeled GB300 time).
        slicing: "eq1" (index overhead of Eq. 1) or "reuse" (lifetime-aware: executed cost
        under tree-like reuse).  branch_exchange: reorder consecutive contractions of the
        kept trial while that lowers the slicing's cost.  cluster_chains: fused chains may
        hold tiles of up to 2^15 entries on a thread-block cluster (default 2^12, one CTA)."""
        lib = load_library()
        arity, qubits, mats = circuit.gate_array()
        ch = tnc_circuit_from_gates(circuit.n_qubits, arity, qubits, mats)
        try:
            mask = np.zeros(circuit.n_qubits, dtype=np.uint8)
            mask[list(open_qubits)] = 1
            nh = tnc_network_build(ch, mask)
            try:
                ph = tnc_plan_greedy(nh, seed, trials, log2_cap, slices_min, slices_max, temperature,
                                     {"greedy": 0, "stem": 1, "split": 2}[mode], {"flops": 0, "time": 1}[objective],
                                     {"eq1": 0, "reuse": 1}[slicing], int(bool(branch_exchange)),
                                     int(bool(cluster_chains)))
            finally:
                lib.tnc_network_destroy(nh)
        finally:
            lib.tnc_circuit_destroy(ch)
        return cls(ph, circuit.n_qubits)

    @classmethod
    def load(cls, path: str) -> "Plan":
        lib = load_library()
        h = C.c_void_p()
        _check(lib.tnc_plan_load(path.encode(), C.byref(h)))
        p = cls(h, 0)
        p.n_qubits = p.describe()["n_qubits"]
        return p

    def update_gates(self, matrices):
        """New gate values for the same gates: a list of d x d complex arrays U[out, in]
        (d = 2 or 4), or the packed (n_gates, 32) float64 layout of the C boundary."""
        if isinstance(matrices, np.ndarray) and matrices.dtype == np.float64 and matrices.ndim == 2:
            packed = np.ascontiguousarray(matrices)
        else:
            packed = np.zeros((len(matrices), 32))
            for g, u in enumerate(matrices):
                flat = np.asarray(u, dtype=np.complex128).reshape(-1)
                packed[g, 0 : 2 * flat.size : 2] = flat.real
                packed[g, 1 : 2 * flat.size : 2] = flat.imag
        _check(load_library().tnc_plan_update_gates(self.h, len(packed), packed.ctypes.data_as(C.POINTER(C.c_double))))

    def save(self, path: str):
        _check(load_library().tnc_plan_save(self.h, path.encode()))

    def info(self) -> dict:
        i = tnc_plan_info()
        _check(load_library().tnc_plan_get_info(self.h, C.byref(i)))
        return {name: getattr(i, name) for name, _ in tnc_plan_info._fields_}

    def slice_stats(self) -> dict:
        """Per sliced index (slice bit t): lifetime (first / last step holding it), steps that
        depend on it, and its Eq. 1 and tree-reuse overheads (tnc_plan_slice_stats)."""
        n = self.info()["n_sliced"]
        m = max(n, 1)
        first, last, dep, post = (np.zeros(m, dtype=np.int32) for _ in range(4))
        ov, rov, ms = np.zeros(m), np.zeros(m), np.zeros(m)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        _check(load_library().tnc_plan_slice_stats(self.h, _i32p(first), _i32p(last), _i32p(dep), dp(ov), dp(rov),
                                                   _i32p(post), dp(ms), m))
        return {"first_step": first[:n], "last_step": last[:n], "dep_steps": dep[:n], "overhead": ov[:n],
                "reuse_overhead": rov[:n], "post_steps": post[:n], "merge_saving": ms[:n]}

    def sliced_cuts(self):
        n = self.info()["n_sliced"]
        q = np.zeros(max(n, 1), dtype=np.int32)
        c = np.zeros(max(n, 1), dtype=np.int32)
        _check(load_library().tnc_plan_sliced_cuts(self.h, _i32p(q), _i32p(c), max(n, 1)))
        return [(int(q[t]), int(c[t])) for t in range(n)]

    def open_qubits(self):
        n = self.info()["n_open"]
        q = np.zeros(max(n, 1), dtype=np.int32)
        _check(load_library().tnc_plan_open_qubits(self.h, _i32p(q), max(n, 1)))
        return [int(x) for x in q[:n]]

    def describe(self) -> dict:
        lib = load_library()
        n = C.c_int64()
        _check(lib.tnc_plan_describe(self.h, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(lib.tnc_plan_describe(self.h, buf, n.value, C.byref(n)))
        return json.loads(buf.value.decode())

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.tnc_plan_destroy(self.h)
            self.h = None


class Context:
    """A device context (one GPU, one stream, scratch)."""

    def __init__(self, device: int = 0):
        lib = load_library()
        self.h = C.c_void_p()
        _check(lib.tnc_context_create(device, C.byref(self.h)))
        self.device = device

    def sync(self):
        _check(_lib.tnc_sync(self.h))

    def amplitudes(self, plan: Plan, bitstrings: Optional[np.ndarray], precision: str = "c64",
                   slice_begin: int = 0, slice_count: Optional[int] = None, wave: int = 0, out=None,
                   stream: int = 0, profile: bool = False, fuse: bool = True, use_graph: bool = False,
                   merge: bool = False, persistent: bool = False) -> np.ndarray:
        """Amplitudes of every row x every open-qubit assignment, summed over the slices.

        `out` may be a host numpy complex128 array or a torch complex128 CUDA tensor of
        shape (batch, 2^n_open); a new host array is returned when it is None.
        merge: post-lifetime merging (Sec. III-B) on calls that cover every slice with
        tree-like reuse: each sliced index is summed right after the step that contracts it
        (tnc_exec_opts.reserved[1] = 1).
        persistent: each wave's steps as one persistent launch when every step is a SIMT
        contraction (tnc_exec_opts.reserved[2] = 1); bit-identical to per-step launches."""
        lib = load_library()
        info = plan.info()
        if slice_count is None:
            slice_count = (1 << info["n_sliced"]) - slice_begin
        if bitstrings is None:
            batch = 1
            bp = None
        else:
            bs = np.ascontiguousarray(bitstrings, dtype=np.uint8)
            if bs.ndim == 1:
                bs = bs[None, :]
            batch = bs.shape[0]
            bp = bs.ctypes.data_as(C.POINTER(C.c_uint8))
        n_out = 1 << info["n_open"]
        if out is None:
            out = np.zeros((batch, n_out), dtype=np.complex128)
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        opts = tnc_exec_opts(PRECISIONS[precision] if isinstance(precision, str) else int(precision), wave,
                             int(use_graph), int(fuse), int(profile))
        opts.reserved[1] = int(merge)
        opts.reserved[2] = int(persistent)
        _check(lib.tnc_amplitudes(self.h, plan.h, C.byref(opts), bp, batch, slice_begin, slice_count,
                                  C.c_void_p(ptr), C.c_void_p(stream)))
        return out

    def amplitudes_ids(self, plan: Plan, bitstrings: Optional[np.ndarray], slice_ids, precision: str = "c64",
                       wave: int = 0, out=None, stream: int = 0, fuse: bool = True, profile: bool = False,
                       persistent: bool = False) -> np.ndarray:
        """Amplitudes summed over the listed slice ids (tnc_amplitudes_ids); `persistent` as in
        amplitudes()."""
        lib = load_library()
        info = plan.info()
        ids = np.ascontiguousarray(slice_ids, dtype=np.int64)
        if bitstrings is None:
            batch, bp = 1, None
        else:
            bs = np.ascontiguousarray(bitstrings, dtype=np.uint8)
            if bs.ndim == 1:
                bs = bs[None, :]
            batch, bp = bs.shape[0], bs.ctypes.data_as(C.POINTER(C.c_uint8))
        if out is None:
            out = np.zeros((batch, 1 << info["n_open"]), dtype=np.complex128)
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        opts = tnc_exec_opts(PRECISIONS[precision] if isinstance(precision, str) else int(precision), wave, 0,
                             int(fuse), int(profile))
        opts.reserved[2] = int(persistent)
        _check(lib.tnc_amplitudes_ids(self.h, plan.h, C.byref(opts), bp, batch,
                                      ids.ctypes.data_as(C.POINTER(C.c_int64)), len(ids), C.c_void_p(ptr),
                                      C.c_void_p(stream)))
        return out

    def autotune(self, plan: Plan, bitstrings: Optional[np.ndarray], precision: str = "chalf",
                 slice_begin: int = 0, slice_count: Optional[int] = None, wave: int = 0, fuse: bool = True) -> dict:
        """Time the admissible configurations of every tensor-core step of the program this
        call shape uses and keep the fastest (tnc_autotune).  Returns the tuning counts."""
        lib = load_library()
        info = plan.info()
        if slice_count is None:
            slice_count = (1 << info["n_sliced"]) - slice_begin
        if bitstrings is None:
            batch, bp = 1, None
        else:
            bs = np.ascontiguousarray(bitstrings, dtype=np.uint8)
            if bs.ndim == 1:
                bs = bs[None, :]
            batch, bp = bs.shape[0], bs.ctypes.data_as(C.POINTER(C.c_uint8))
        opts = tnc_exec_opts(PRECISIONS[precision] if isinstance(precision, str) else int(precision), wave, 0,
                             int(fuse), 0)
        ti = tnc_tune_info()
        _check(lib.tnc_autotune(self.h, plan.h, C.byref(opts), bp, batch, slice_begin, slice_count, C.byref(ti)))
        return {k: getattr(ti, k) for k in ("steps_tuned", "steps_changed", "candidates", "seconds_default",
                                             "seconds_tuned")}

    def adjoint(self, plan: Plan, bitstrings: Optional[np.ndarray], weights: np.ndarray, arities, stream: int = 0,
                memory_mib: int = 0):
        """Gate environments dL/dU_g of L = sum_{b,i} weights[b, i] * amp[b, i] (holomorphic
        derivative), over all slices.  `arities` lists each gate's arity (1 or 2).  Returns
        (list of d x d complex128 arrays, amplitudes (batch, 2^n_open)).  `memory_mib` > 0 caps
        the forward intermediates kept per instance; the largest are recomputed instead."""
        lib = load_library()
        info = plan.info()
        n_out = 1 << info["n_open"]
        if bitstrings is None:
            batch, bp = 1, None
        else:
            bs = np.ascontiguousarray(bitstrings, dtype=np.uint8)
            if bs.ndim == 1:
                bs = bs[None, :]
            batch, bp = bs.shape[0], bs.ctypes.data_as(C.POINTER(C.c_uint8))
        w = np.ascontiguousarray(np.asarray(weights, dtype=np.complex128).reshape(batch, n_out))
        n_gates = len(arities)
        env = np.zeros((n_gates, 32))
        amps = np.zeros((batch, n_out), dtype=np.complex128)
        opts = tnc_exec_opts(TNC_C64, 0, 0, 1, 0)
        opts.reserved[0] = int(memory_mib)
        _check(lib.tnc_adjoint(self.h, plan.h, C.byref(opts), bp, batch, C.c_void_p(w.ctypes.data),
                               C.c_void_p(env.ctypes.data), C.c_void_p(amps.ctypes.data), C.c_void_p(stream)))
        out = []
        for g, a in enumerate(arities):
            d = 1 << int(a)
            out.append((env[g, 0 : 2 * d * d : 2] + 1j * env[g, 1 : 2 * d * d : 2]).reshape(d, d))
        return out, amps

    def profile_read(self, cap: int = 4096) -> dict:
        """Per-step device times of the last profiled amplitudes call (see tnc_profile_read)."""
        ms = np.zeros(cap + 1)
        launches = np.zeros(cap, dtype=np.int32)
        flops = np.zeros(cap)
        byts = np.zeros(cap)
        kind = np.zeros(cap, dtype=np.int32)
        n = C.c_int32()
        dp = C.POINTER(C.c_double)
        _check(_lib.tnc_profile_read(self.h, ms.ctypes.data_as(dp), _i32p(launches), flops.ctypes.data_as(dp),
                                     byts.ctypes.data_as(dp), _i32p(kind), cap, C.byref(n)))
        k = n.value
        return {"ms": ms[:k], "total_ms": float(ms[k]), "launches": launches[:k], "flops": flops[:k],
                "bytes": byts[:k], "kind": kind[:k]}

    def contract(self, precision: str, a, labels_a, b, labels_b, c, labels_c, stream: int = 0) -> int:
        """C = A * B on planar device tensors (torch tensors of the storage dtype, 2*2^rank
        entries).  Returns C's exponent: the result is c * 2^exponent."""
        lib = load_library()
        la = np.ascontiguousarray(labels_a, dtype=np.int32)
        lb = np.ascontiguousarray(labels_b, dtype=np.int32)
        lc = np.ascontiguousarray(labels_c, dtype=np.int32)
        e = C.c_int32()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(lib.tnc_contract(self.h, prec, C.c_void_p(a.data_ptr()), len(la), _i32p(la), C.c_void_p(b.data_ptr()),
                                len(lb), _i32p(lb), C.c_void_p(c.data_ptr()), len(lc), _i32p(lc), C.byref(e),
                                C.c_void_p(stream)))
        return int(e.value)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.tnc_context_destroy(self.h)
            self.h = None


def tnc_contract_noalloc(precision, a, labels_a, b, labels_b, c, labels_c, stream: int = 0) -> int:
    """C = A * B without any device allocation (see include/tnc.h).  a, b, c are planar
    device tensors (torch) on the current device.  Returns C's exponent."""
    lib = load_library()
    la = np.ascontiguousarray(labels_a, dtype=np.int32)
    lb = np.ascontiguousarray(labels_b, dtype=np.int32)
    lc = np.ascontiguousarray(labels_c, dtype=np.int32)
    e = C.c_int32()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _check(lib.tnc_contract_noalloc(prec, C.c_void_p(a.data_ptr()), len(la), _i32p(la), C.c_void_p(b.data_ptr()),
                                    len(lb), _i32p(lb), C.c_void_p(c.data_ptr()), len(lc), _i32p(lc), C.byref(e),
                                    C.c_void_p(stream)))
    return int(e.value)


def version() -> str:
    return load_library().tnc_version().decode()


def tune_save(path: str) -> None:
    """Write the process-wide tuning cache to `path` (tnc_tune_save)."""
    _check(load_library().tnc_tune_save(path.encode()))


def tune_load(path: str) -> None:
    """Merge the tuning cache file at `path` into the process-wide cache (tnc_tune_load)."""
    _check(load_library().tnc_tune_load(path.encode()))


def tune_clear() -> None:
    load_library().tnc_tune_clear()


def tune_size() -> int:
    return int(load_library().tnc_tune_size())
