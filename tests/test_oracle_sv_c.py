"""Pins for the plain C state-vector oracle (oracle/sv.c): brute force, qubit order,
the stored two-qubit values, unit norm, and agreement with the numpy oracle."""
import os

import numpy as np
import pytest

from inputs import SQRT_X, SQRT_Y, fsim, grid_circuit
from inputs.circuits import custom_circuit
from oracle import statevector as sv
from oracle import sv_c

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("rows,cols,cycles", [(2, 2, 4), (2, 3, 5), (1, 4, 6)])
def test_c_statevector_matches_explicit_unitary(rows, cols, cycles):
    c = grid_circuit(rows, cols, cycles, seed=7, fsim_mode="uniform")
    assert np.allclose(sv_c.final_state(c), sv.explicit_unitary(c)[:, 0], atol=1e-13)


def test_c_statevector_qubit_order():
    x = np.array([[0, 1], [1, 0]], dtype=complex)
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    # X on qubit 2, then CNOT with control 2 (listed first) and target 0 -> |101> = index 5
    psi = sv_c.final_state(custom_circuit(3, [((2,), x), ((2, 0), cnot)]))
    assert np.isclose(psi[5], 1.0) and np.isclose(np.sum(np.abs(psi) ** 2), 1.0)


def test_c_statevector_golden_two_qubit_values():
    c = custom_circuit(2, [((0,), SQRT_X), ((1,), SQRT_Y), ((0, 1), fsim(np.pi / 2, np.pi / 6))])
    with open(os.path.join(GOLDEN, "two_qubit_fsim.txt")) as f:
        rows = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    psi = sv_c.final_state(c)
    for bits, re, im in rows:
        assert abs(psi[int(bits, 2)] - complex(float(re), float(im))) < 1e-14


def test_c_statevector_norm_and_numpy_agreement():
    c = grid_circuit(4, 4, 10, seed=3, fsim_mode="uniform", param_seed=4)
    psi = sv_c.final_state(c)
    assert abs(1.0 - np.sum(np.abs(psi) ** 2)) < 1e-12
    assert np.allclose(psi, sv.final_state(c).reshape(-1), atol=1e-14)


def test_c_statevector_rejects_bad_gates():
    c = custom_circuit(2, [((0, 1), fsim(0.1, 0.2))])
    c.gates[0].qubits = (0, 0)
    with pytest.raises(ValueError):
        sv_c.final_state(c)
