"""Error norms and random-circuit statistics used to judge amplitudes against the oracle."""
from __future__ import annotations

import numpy as np


def rel_err_norm(a: np.ndarray, ref: np.ndarray) -> float:
    """||a - ref||_2 / ||ref||_2 over the batch (norm-wise relative error)."""
    a = np.asarray(a, dtype=np.complex128).reshape(-1)
    ref = np.asarray(ref, dtype=np.complex128).reshape(-1)
    return float(np.linalg.norm(a - ref) / np.linalg.norm(ref))


def rel_err_max(a: np.ndarray, ref: np.ndarray, n_qubits: int) -> float:
    """max_b |a_b - ref_b| / max(|ref_b|, 2^(-n/2) * 1e-3)."""
    a = np.asarray(a, dtype=np.complex128).reshape(-1)
    ref = np.asarray(ref, dtype=np.complex128).reshape(-1)
    floor = 2.0 ** (-n_qubits / 2.0) * 1e-3
    return float(np.max(np.abs(a - ref) / np.maximum(np.abs(ref), floor)))


def xeb_sampled(p_of_samples: np.ndarray, n_qubits: int) -> float:
    """Linear XEB F = 2^n * mean_x p(x) - 1 over bitstrings x sampled from the circuit."""
    return float((2.0 ** n_qubits) * np.mean(p_of_samples) - 1.0)


def xeb_weighted(p_ref: np.ndarray, p: np.ndarray, n_qubits: int) -> float:
    """XEB over a fixed batch, each bitstring weighted by its reference probability:
    F = 2^n * sum p_ref * p / sum p_ref - 1 (the sampled form's expectation)."""
    p_ref = np.asarray(p_ref, dtype=np.float64).reshape(-1)
    p = np.asarray(p, dtype=np.float64).reshape(-1)
    return float((2.0 ** n_qubits) * np.sum(p_ref * p) / np.sum(p_ref) - 1.0)


def porter_thomas(probs: np.ndarray):
    """Statistics of N*p over all N = 2^n outcomes: mean, second moment, KS distance to Exp(1)."""
    p = np.asarray(probs, dtype=np.float64).reshape(-1)
    n_out = p.size
    x = np.sort(n_out * p)
    emp = np.arange(1, n_out + 1) / n_out
    cdf = 1.0 - np.exp(-x)
    ks = float(np.max(np.maximum(np.abs(emp - cdf), np.abs(emp - 1.0 / n_out - cdf))))
    return float(np.mean(n_out * p)), float(np.mean((n_out * p) ** 2)), ks
