"""Dense FP64 state-vector oracle.

amp(x) = <x| U_L ... U_1 |0^n>  -- the quantity the tensor-network contraction of a
circuit computes exactly (Sec. I: a circuit is represented as a tensor network and
contracted to a single node; Sec. II-A).

Conventions: qubit q is axis q of the state reshaped to (2,)*n, i.e. bit (n-1-q) of the
flat index (qubit 0 most significant).  A 2-qubit gate on (a, b) has matrix index
2*bit(a) + bit(b), U[out, in].

Slicing (Sec. II-A; Sec. III-A: slicing index a gives two subtasks, one per component
of a) is written here as inserting the projector P_b = |b><b| on one wire segment.  A
wire segment is named by a *cut* (q, j): qubit q's wire after the first j gates that
act on q.  Because P_0 + P_1 = I, the sum over all slice assignments is the amplitude.
"""
from __future__ import annotations

from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

Cut = Tuple[int, int]  # (qubit, number of gates on that qubit before the cut)


def zero_state(n: int) -> np.ndarray:
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    return psi


def apply_matrix(psi: np.ndarray, qubits: Sequence[int], u: np.ndarray) -> np.ndarray:
    """psi' = (U on `qubits`) psi, for a state tensor of shape (2,)*n."""
    k = len(qubits)
    ut = np.asarray(u, dtype=np.complex128).reshape((2,) * (2 * k))
    # contract U's input axes (k..2k-1) with the state's qubit axes
    out = np.tensordot(ut, psi, axes=(list(range(k, 2 * k)), list(qubits)))
    # tensordot puts U's output axes first; move them back to the qubit positions
    return np.moveaxis(out, list(range(k)), list(qubits))


def project(psi: np.ndarray, q: int, bit: int) -> np.ndarray:
    """psi' = P_bit on qubit q."""
    out = psi.copy()
    idx = [slice(None)] * psi.ndim
    idx[q] = 1 - bit
    out[tuple(idx)] = 0.0
    return out


def final_state(circuit, cuts: Optional[Dict[Cut, int]] = None) -> np.ndarray:
    """U_L...U_1|0>, with P_bit inserted at every cut in `cuts` ({(q, j): bit})."""
    n = circuit.n_qubits
    psi = zero_state(n)
    count = [0] * n
    cuts = dict(cuts or {})

    def cut_here(q):
        nonlocal psi
        key = (q, count[q])
        if key in cuts:
            psi = project(psi, q, cuts[key])

    for g in circuit.gates:
        for q in g.qubits:
            cut_here(q)
        psi = apply_matrix(psi, g.qubits, g.matrix)
        for q in g.qubits:
            count[q] += 1
    for q in range(n):
        cut_here(q)
    return psi


def flat_index(bits: np.ndarray) -> np.ndarray:
    """Flat state index of each bitstring row (qubit 0 most significant)."""
    bits = np.atleast_2d(np.asarray(bits, dtype=np.int64))
    n = bits.shape[1]
    w = 1 << np.arange(n - 1, -1, -1, dtype=np.int64)
    return bits @ w


def amplitudes(psi: np.ndarray, bitstrings: np.ndarray) -> np.ndarray:
    return psi.reshape(-1)[flat_index(bitstrings)]


def circuit_amplitudes(circuit, bitstrings, cuts=None) -> np.ndarray:
    return amplitudes(final_state(circuit, cuts), bitstrings)


# ----------------------------------------------------------------------------------
# Explicit unitary, for brute-force pins on tiny registers.
# ----------------------------------------------------------------------------------
def full_operator(n: int, qubits: Sequence[int], u: np.ndarray) -> np.ndarray:
    """The 2^n x 2^n matrix of U acting on `qubits`, built entry by entry.

    <y|Op|x> = U[y_Q, x_Q] * delta(y_rest, x_rest), with y_Q, x_Q read from the bits of
    the acted-on qubits in `qubits` order (first qubit most significant).
    """
    dim = 1 << n
    op = np.zeros((dim, dim), dtype=np.complex128)
    qs = list(qubits)
    others = [q for q in range(n) if q not in qs]
    for x in range(dim):
        xb = [(x >> (n - 1 - q)) & 1 for q in range(n)]
        xq = 0
        for q in qs:
            xq = 2 * xq + xb[q]
        for yq in range(1 << len(qs)):
            yb = list(xb)
            for t, q in enumerate(qs):
                yb[q] = (yq >> (len(qs) - 1 - t)) & 1
            y = 0
            for q in range(n):
                y = 2 * y + yb[q]
            op[y, x] += u[yq, xq]
    del others
    return op


def explicit_unitary(circuit) -> np.ndarray:
    n = circuit.n_qubits
    total = np.eye(1 << n, dtype=np.complex128)
    for g in circuit.gates:
        total = full_operator(n, g.qubits, g.matrix) @ total
    return total


# ----------------------------------------------------------------------------------
# Gradient environments.
# ----------------------------------------------------------------------------------
def bra_state(n: int, bitstrings: np.ndarray, weights: np.ndarray) -> np.ndarray:
    """|chi> = sum_b conj(w_b) |x_b>, so that <chi|psi> = sum_b w_b <x_b|psi>."""
    chi = np.zeros(1 << n, dtype=np.complex128)
    np.add.at(chi, flat_index(bitstrings), np.conj(np.asarray(weights, dtype=np.complex128)))
    return chi.reshape((2,) * n)


def environment(psi_before: np.ndarray, phi_after: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    """E[o, i] = sum_rest conj(phi[o, rest]) * psi[i, rest] over the gate's qubits."""
    k = len(qubits)
    n = psi_before.ndim
    rest = [a for a in range(n) if a not in qubits]
    p = np.transpose(psi_before, list(qubits) + rest).reshape(1 << k, -1)
    f = np.transpose(phi_after, list(qubits) + rest).reshape(1 << k, -1)
    return np.conj(f) @ p.T


def gate_environments(circuit, bitstrings: np.ndarray, weights: np.ndarray) -> List[np.ndarray]:
    """dL/dG_t[o, i] for L = sum_b w_b amp(x_b), for every gate t (holomorphic derivative).

    With psi_{t-1} = G_{t-1}...G_1|0> and <phi_t| = <chi| G_L ... G_{t+1}:
        L = sum_{o,i,rest} conj(phi_t[o,rest]) G_t[o,i] psi_{t-1}[i,rest].
    Walks backwards from the final state using G^dagger = G^{-1} (unitary gates).
    """
    n = circuit.n_qubits
    psi = final_state(circuit)
    phi = bra_state(n, bitstrings, weights)
    envs: List[Optional[np.ndarray]] = [None] * len(circuit.gates)
    for t in range(len(circuit.gates) - 1, -1, -1):
        g = circuit.gates[t]
        udag = np.conj(np.asarray(g.matrix)).T
        psi = apply_matrix(psi, g.qubits, udag)  # now psi_{t-1}
        envs[t] = environment(psi, phi, g.qubits)
        phi = apply_matrix(phi, g.qubits, udag)  # <phi_{t-1}| = <phi_t| G_t
    return envs  # type: ignore[return-value]
