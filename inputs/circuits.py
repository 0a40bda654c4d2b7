"""Grid random quantum circuits (RQCs) of the kind the paper simulates (Sec. I, Sec. VII).

The paper evaluates Zuchongzhi-56/60 circuits (Sec. VII); those circuit files are not
available here, so seeded synthetic grid circuits with the same structure stand in:
every cycle applies one random single-qubit gate per qubit, drawn from
{sqrt(X), sqrt(Y), sqrt(W)} with no immediate repeat on a qubit, then fSim gates on
one class of nearest-neighbour couplers, cycling through the classes A, B, C, D.

Readings (the paper never prints its gates):
  * sqrt(X) = (I - iX)/sqrt2, sqrt(Y) = (I - iY)/sqrt2, sqrt(W) = (I - iW)/sqrt2 with
    W = (X + Y)/sqrt2.  Each squares to -i times its Pauli, i.e. the Pauli up to phase.
  * fSim(theta, phi) = [[1,0,0,0],[0,c,-is,0],[0,-is,c,0],[0,0,0,e^{-i phi}]] in the
    basis |q_a q_b>, q_a = gates' first qubit (the lower index), the more significant bit.
  * Coupler classes on a rows x cols grid, qubit q = r*cols + c:
      A: (r,c)-(r,c+1), c even;  B: (r,c)-(r,c+1), c odd;
      C: (r,c)-(r+1,c), r even;  D: (r,c)-(r+1,c), r odd.
    Cycle k uses class pattern[k % len(pattern)], default "ABCD".
  * Cycle 0 draws each qubit's gate uniformly from the three; later cycles draw
    uniformly from the two gates that differ from that qubit's previous one.
    Draws are consumed qubit-major within each cycle from numpy's PCG64 seeded by `seed`.
  * Exactly `cycles` cycles (1q layer then 2q layer); no trailing 1q layer.

Matrices are complex128, indexed U[out, in].
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

_S2 = 1.0 / np.sqrt(2.0)

SQRT_X = _S2 * np.array([[1.0, -1.0j], [-1.0j, 1.0]], dtype=np.complex128)
SQRT_Y = _S2 * np.array([[1.0, -1.0], [1.0, 1.0]], dtype=np.complex128)
SQRT_W = _S2 * np.array(
    [[1.0, -np.exp(0.25j * np.pi)], [np.exp(-0.25j * np.pi), 1.0]], dtype=np.complex128
)
SINGLE_QUBIT_SET = (SQRT_X, SQRT_Y, SQRT_W)
SINGLE_QUBIT_NAMES = ("sqrt_x", "sqrt_y", "sqrt_w")


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) as a 4x4 matrix in the basis |q_a q_b> (q_a most significant)."""
    c, s = np.cos(theta), np.sin(theta)
    u = np.zeros((4, 4), dtype=np.complex128)
    u[0, 0] = 1.0
    u[1, 1] = c
    u[1, 2] = -1.0j * s
    u[2, 1] = -1.0j * s
    u[2, 2] = c
    u[3, 3] = np.exp(-1.0j * phi)
    return u


@dataclass
class Gate:
    """One gate: qubits it acts on, its matrix U[out, in], and where it came from.

    For a 2-qubit gate the 4-dim index is 2*bit(qubits[0]) + bit(qubits[1]).
    `params` holds (theta, phi) for fSim gates so callers can differentiate by angle.
    """

    qubits: Tuple[int, ...]
    matrix: np.ndarray
    kind: str = "custom"
    params: Optional[Tuple[float, float]] = None


@dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate] = field(default_factory=list)
    rows: int = 0
    cols: int = 0
    cycles: int = 0
    seed: int = 0

    def __len__(self) -> int:
        return len(self.gates)

    def gate_array(self):
        """Packed gate list: (arity[int32], qubits[int32,2], matrices[float64, 32]).

        Matrices are row-major U[out, in], interleaved (re, im), zero-padded to 4x4.
        This is the layout the C boundary's `tnc_circuit_from_gates` reads.
        """
        g = len(self.gates)
        arity = np.zeros(g, dtype=np.int32)
        qubits = np.full((g, 2), -1, dtype=np.int32)
        mats = np.zeros((g, 32), dtype=np.float64)
        for i, gate in enumerate(self.gates):
            a = len(gate.qubits)
            arity[i] = a
            qubits[i, :a] = gate.qubits
            d = 1 << a
            flat = np.asarray(gate.matrix, dtype=np.complex128).reshape(d * d)
            mats[i, 0 : 2 * d * d : 2] = flat.real
            mats[i, 1 : 2 * d * d : 2] = flat.imag
        return arity, qubits, mats


def couplers(rows: int, cols: int, cls: str) -> List[Tuple[int, int]]:
    """Nearest-neighbour pairs of one coupler class, lower qubit index first."""
    out = []
    if cls in "AB":
        parity = 0 if cls == "A" else 1
        for r in range(rows):
            for c in range(parity, cols - 1, 2):
                out.append((r * cols + c, r * cols + c + 1))
    elif cls in "CD":
        parity = 0 if cls == "C" else 1
        for r in range(parity, rows - 1, 2):
            for c in range(cols):
                out.append((r * cols + c, (r + 1) * cols + c))
    else:
        raise ValueError(f"unknown coupler class {cls!r}")
    return out


def grid_circuit(
    rows: int,
    cols: int,
    cycles: int,
    seed: int = 1,
    fsim_mode: str = "fixed",
    param_seed: Optional[int] = None,
    pattern: str = "ABCD",
    fixed_angles: Tuple[float, float] = (np.pi / 2, np.pi / 6),
) -> Circuit:
    """Seeded grid RQC.

    fsim_mode: "fixed" uses fSim(pi/2, pi/6) everywhere; "uniform" draws theta and phi
    uniformly in [0, pi] per gate from PCG64(param_seed) (default seed + 1000).
    """
    n = rows * cols
    rng = np.random.default_rng(seed)
    prng = np.random.default_rng(seed + 1000 if param_seed is None else param_seed)
    circ = Circuit(n_qubits=n, rows=rows, cols=cols, cycles=cycles, seed=seed)
    prev = [-1] * n
    for cyc in range(cycles):
        for q in range(n):
            if prev[q] < 0:
                choice = int(rng.integers(3))
            else:
                others = [g for g in range(3) if g != prev[q]]
                choice = others[int(rng.integers(2))]
            prev[q] = choice
            circ.gates.append(
                Gate((q,), SINGLE_QUBIT_SET[choice].copy(), SINGLE_QUBIT_NAMES[choice])
            )
        cls = pattern[cyc % len(pattern)]
        for a, b in couplers(rows, cols, cls):
            if fsim_mode == "fixed":
                theta, phi = fixed_angles
            elif fsim_mode == "uniform":
                theta, phi = (float(x) for x in prng.uniform(0.0, np.pi, size=2))
            else:
                raise ValueError(f"unknown fsim_mode {fsim_mode!r}")
            circ.gates.append(Gate((a, b), fsim(theta, phi), "fsim", (theta, phi)))
    return circ


def custom_circuit(n_qubits: int, gates: Sequence[Tuple[Sequence[int], np.ndarray]]) -> Circuit:
    """Circuit from explicit (qubits, matrix) pairs."""
    c = Circuit(n_qubits=n_qubits)
    for qs, m in gates:
        c.gates.append(Gate(tuple(int(q) for q in qs), np.asarray(m, dtype=np.complex128)))
    return c
