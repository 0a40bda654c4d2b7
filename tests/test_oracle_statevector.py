"""Pins for the state-vector oracle: closed forms, brute force, invariants, statistics."""
import itertools
import os

import numpy as np
import pytest

from inputs import SQRT_W, SQRT_X, SQRT_Y, fsim, grid_circuit, random_bitstrings
from inputs.circuits import couplers, custom_circuit
from oracle import metrics, statevector as sv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
I2 = np.eye(2, dtype=complex)


# ---------------------------------------------------------------- gates (input readings)
def test_single_qubit_gates_square_to_paulis():
    # each gate is the square root of its Pauli up to the phase -i
    assert np.allclose(SQRT_X @ SQRT_X, -1j * X)
    assert np.allclose(SQRT_Y @ SQRT_Y, -1j * Y)
    w = (X + Y) / np.sqrt(2)
    assert np.allclose(SQRT_W @ SQRT_W, -1j * w)
    for g in (SQRT_X, SQRT_Y, SQRT_W):
        assert np.allclose(g.conj().T @ g, I2)


def test_fsim_closed_forms():
    assert np.allclose(fsim(0.0, 0.0), np.eye(4))
    iswap_like = np.array([[1, 0, 0, 0], [0, 0, -1j, 0], [0, -1j, 0, 0], [0, 0, 0, 1]])
    assert np.allclose(fsim(np.pi / 2, 0.0), iswap_like)
    cz_like = np.diag([1, 1, 1, -1]).astype(complex)
    assert np.allclose(fsim(0.0, np.pi), cz_like)
    rng = np.random.default_rng(0)
    for _ in range(5):
        u = fsim(*rng.uniform(0, np.pi, 2))
        assert np.allclose(u.conj().T @ u, np.eye(4))


def test_couplers_partition_grid_edges():
    rows, cols = 5, 6
    edges = set()
    for cls in "ABCD":
        cl = couplers(rows, cols, cls)
        used = [q for e in cl for q in e]
        assert len(used) == len(set(used)), "a class uses a qubit twice"
        for a, b in cl:
            ra, ca, rb, cb = a // cols, a % cols, b // cols, b % cols
            assert abs(ra - rb) + abs(ca - cb) == 1 and a < b
            edges.add((a, b))
    expect = rows * (cols - 1) + (rows - 1) * cols
    assert len(edges) == expect


def test_grid_circuit_no_repeat_and_seeded():
    c1 = grid_circuit(3, 4, 8, seed=1)
    c2 = grid_circuit(3, 4, 8, seed=1)
    assert all(np.array_equal(a.matrix, b.matrix) and a.qubits == b.qubits for a, b in zip(c1.gates, c2.gates))
    last = {}
    for g in c1.gates:
        if len(g.qubits) == 1:
            q = g.qubits[0]
            assert last.get(q) != g.kind
            last[q] = g.kind


# ---------------------------------------------------------------- brute force
def test_full_operator_matches_kron_for_adjacent_qubits():
    rng = np.random.default_rng(1)
    u = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    n = 4
    for a in range(n - 1):
        ref = np.kron(np.kron(np.eye(1 << a), u), np.eye(1 << (n - a - 2)))
        assert np.allclose(sv.full_operator(n, (a, a + 1), u), ref)
    v = rng.normal(size=(2, 2)) + 1j * rng.normal(size=(2, 2))
    for a in range(n):
        ref = np.kron(np.kron(np.eye(1 << a), v), np.eye(1 << (n - a - 1)))
        assert np.allclose(sv.full_operator(n, (a,), v), ref)


def test_full_operator_reversed_pair_is_swap_conjugate():
    rng = np.random.default_rng(2)
    u = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
    swap = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)
    assert np.allclose(sv.full_operator(2, (1, 0), u), swap @ u @ swap)


@pytest.mark.parametrize("rows,cols,cycles", [(2, 2, 4), (2, 3, 5), (1, 4, 6)])
def test_statevector_matches_explicit_unitary(rows, cols, cycles):
    c = grid_circuit(rows, cols, cycles, seed=7, fsim_mode="uniform")
    psi = sv.final_state(c).reshape(-1)
    ref = sv.explicit_unitary(c)[:, 0]
    assert np.allclose(psi, ref, atol=1e-13)


def test_golden_two_qubit_amplitudes():
    c = custom_circuit(2, [((0,), SQRT_X), ((1,), SQRT_Y), ((0, 1), fsim(np.pi / 2, np.pi / 6))])
    rows = []
    with open(os.path.join(GOLDEN, "two_qubit_fsim.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                bits, re, im = line.split()
                rows.append(([int(ch) for ch in bits], complex(float(re), float(im))))
    bs = np.array([r[0] for r in rows], dtype=np.uint8)
    amps = sv.circuit_amplitudes(c, bs)
    assert np.allclose(amps, [r[1] for r in rows], atol=1e-14)


def test_qubit_order_with_cnot():
    cnot = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    # X on qubit 0 then CNOT(control 0, target 2) on 3 qubits -> |101>
    c = custom_circuit(3, [((0,), X), ((0, 2), cnot)])
    psi = sv.final_state(c)
    assert np.isclose(psi[1, 0, 1], 1.0) and np.isclose(np.sum(np.abs(psi) ** 2), 1.0)
    # control listed first even when it is the higher qubit: X on 2, CNOT(2 -> 0) -> |101>
    c = custom_circuit(3, [((2,), X), ((2, 0), cnot)])
    assert np.isclose(sv.final_state(c)[1, 0, 1], 1.0)
    # flat index: qubit 0 most significant
    assert sv.flat_index(np.array([[1, 0, 1]]))[0] == 5


def test_product_state_closed_form():
    rng = np.random.default_rng(3)
    n = 5
    gates, per_q = [], [np.eye(2, dtype=complex) for _ in range(n)]
    for _ in range(3):
        for q in range(n):
            g = (SQRT_X, SQRT_Y, SQRT_W)[rng.integers(3)]
            gates.append(((q,), g))
            per_q[q] = g @ per_q[q]
    c = custom_circuit(n, gates)
    bs = np.array(list(itertools.product((0, 1), repeat=n)), dtype=np.uint8)
    amps = sv.circuit_amplitudes(c, bs)
    ref = np.array([np.prod([per_q[q][b[q], 0] for q in range(n)]) for b in bs])
    assert np.allclose(amps, ref, atol=1e-14)


# ---------------------------------------------------------------- invariants
def test_unit_norm():
    psi = sv.final_state(grid_circuit(3, 4, 8, seed=1))
    assert abs(1.0 - np.sum(np.abs(psi) ** 2)) < 1e-12


def test_projector_slices_sum_to_amplitude():
    c = grid_circuit(3, 3, 6, seed=11)
    rng = np.random.default_rng(5)
    count = [0] * c.n_qubits
    for g in c.gates:
        for q in g.qubits:
            count[q] += 1
    cuts = []
    while len(cuts) < 4:
        q = int(rng.integers(c.n_qubits))
        j = int(rng.integers(1, count[q]))
        if (q, j) not in cuts:
            cuts.append((q, j))
    bs = random_bitstrings(c.n_qubits, 16, seed=9)
    full = sv.circuit_amplitudes(c, bs)
    total = np.zeros_like(full)
    for bits in itertools.product((0, 1), repeat=len(cuts)):
        total += sv.circuit_amplitudes(c, bs, dict(zip(cuts, bits)))
    assert np.allclose(total, full, atol=1e-14)
    # a cut on the input segment with bit 1 annihilates |0>
    assert np.allclose(sv.circuit_amplitudes(c, bs, {(0, 0): 1}), 0.0)
    assert np.allclose(sv.circuit_amplitudes(c, bs, {(0, 0): 0}), full)


@pytest.mark.slow
def test_porter_thomas_statistics():
    c = grid_circuit(4, 4, 12, seed=1)
    p = np.abs(sv.final_state(c).reshape(-1)) ** 2
    mean, m2, ks = metrics.porter_thomas(p)
    assert abs(mean - 1.0) < 1e-10  # exact: follows from unit norm
    n_out = p.size
    assert abs(m2 - 2.0 * n_out / (n_out + 1)) < 0.2  # Haar expectation, +-10%
    assert ks < 0.05


# ---------------------------------------------------------------- gradients
def _loss(c, bs, w):
    return np.sum(w * sv.circuit_amplitudes(c, bs))


def test_gate_environments_against_finite_differences_and_brute_force():
    c = grid_circuit(2, 3, 4, seed=5, fsim_mode="uniform")
    bs = random_bitstrings(c.n_qubits, 4, seed=6)
    rng = np.random.default_rng(8)
    w = rng.normal(size=4) + 1j * rng.normal(size=4)
    envs = sv.gate_environments(c, bs, w)
    loss = _loss(c, bs, w)
    h = 1e-3
    for t in (0, 7, len(c.gates) - 1, len(c.gates) // 2):
        g = c.gates[t]
        d = g.matrix.shape[0]
        # linear in G_t: <E_t, G_t> reproduces the loss exactly
        assert np.isclose(np.sum(envs[t] * g.matrix), loss, atol=1e-12)
        for o, i in [(0, 0), (d - 1, 0), (0, d - 1)]:
            orig = g.matrix.copy()
            g.matrix = orig.copy()
            g.matrix[o, i] += h
            lp = _loss(c, bs, w)
            g.matrix = orig.copy()
            g.matrix[o, i] -= h
            lm = _loss(c, bs, w)
            g.matrix = orig
            assert np.isclose((lp - lm) / (2 * h), envs[t][o, i], atol=1e-9)
    # brute force through the explicit unitary: dL/dG_t[o,i] = <chi| U_after (E_oi on Q) U_before |0>
    n = c.n_qubits
    chi = sv.bra_state(n, bs, w).reshape(-1)
    t = 5
    g = c.gates[t]
    before = np.eye(1 << n, dtype=complex)
    for gg in c.gates[:t]:
        before = sv.full_operator(n, gg.qubits, gg.matrix) @ before
    after = np.eye(1 << n, dtype=complex)
    for gg in c.gates[t + 1 :]:
        after = sv.full_operator(n, gg.qubits, gg.matrix) @ after
    d = g.matrix.shape[0]
    for o in range(d):
        for i in range(d):
            e = np.zeros((d, d), dtype=complex)
            e[o, i] = 1.0
            val = np.conj(chi) @ (after @ (sv.full_operator(n, g.qubits, e) @ before[:, 0]))
            assert np.isclose(val, envs[t][o, i], atol=1e-12)
