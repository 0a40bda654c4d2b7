"""Seeded bitstring batches and random tensors.

Bit order convention used everywhere: qubit q of an n-qubit register is bit
(n - 1 - q) of the state-vector index (qubit 0 is the most significant bit).
A bitstring is a uint8 row of n entries, entry q = bit of qubit q.
"""
from __future__ import annotations

from typing import List, Tuple

import numpy as np


def random_bitstrings(n: int, batch: int, seed: int) -> np.ndarray:
    """`batch` uniformly random n-bit strings, shape (batch, n), uint8."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, 2, size=(batch, n), dtype=np.uint8)


def subcube_spec(n: int, n_open: int, seed: int) -> Tuple[np.ndarray, List[int]]:
    """A sub-cube batch: the last `n_open` qubits are open, the rest fixed at random bits.

    Returns (fixed_bits[n] uint8 with 0 at open positions, open_qubits ascending).
    The batch enumerates all 2^n_open assignments of the open qubits; entry i sets open
    qubit open_qubits[j] to bit (n_open - 1 - j) of i (first open qubit most significant).
    """
    rng = np.random.default_rng(seed)
    bits = rng.integers(0, 2, size=n, dtype=np.uint8)
    open_q = list(range(n - n_open, n))
    bits[open_q] = 0
    return bits, open_q


def subcube_bitstrings(fixed_bits: np.ndarray, open_qubits: List[int]) -> np.ndarray:
    """Expand a sub-cube spec into explicit bitstrings, shape (2^len(open), n)."""
    k = len(open_qubits)
    n = len(fixed_bits)
    out = np.tile(np.asarray(fixed_bits, dtype=np.uint8), (1 << k, 1))
    idx = np.arange(1 << k)
    for j, q in enumerate(open_qubits):
        out[:, q] = (idx >> (k - 1 - j)) & 1
    assert out.shape == (1 << k, n)
    return out


def random_complex(shape, sigma: float, seed: int) -> np.ndarray:
    """Complex normal entries with E|z|^2 = sigma^2 (Re, Im ~ N(0, sigma^2/2)), complex128."""
    rng = np.random.default_rng(seed)
    s = sigma / np.sqrt(2.0)
    re = rng.normal(0.0, s, size=shape)
    im = rng.normal(0.0, s, size=shape)
    return (re + 1j * im).astype(np.complex128)


def random_labels_perm(labels: List[int], seed: int) -> List[int]:
    """A seeded random permutation of an index-label list (tensor axis order)."""
    rng = np.random.default_rng(seed)
    perm = rng.permutation(len(labels))
    return [labels[i] for i in perm]
