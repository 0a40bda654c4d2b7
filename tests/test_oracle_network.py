"""Pins for the oracle's own tensor-network contraction: it must reproduce the state
vector for any order, per slice and summed over slices (Sec. II-A, Sec. III-A)."""
import itertools

import numpy as np
import pytest

from inputs import grid_circuit, random_bitstrings, subcube_bitstrings, subcube_spec
from oracle import network as tn
from oracle import statevector as sv


def _wire_counts(c):
    count = [0] * c.n_qubits
    for g in c.gates:
        for q in g.qubits:
            count[q] += 1
    return count


def test_all_amplitudes_match_statevector():
    c = grid_circuit(2, 3, 5, seed=3, fsim_mode="uniform")
    n = c.n_qubits
    out = tn.network_amplitudes(c, None, list(range(n)))
    psi = sv.final_state(c)
    assert np.allclose(out, psi, atol=1e-13)


def test_closed_bitstrings_tiny_config():
    # 12-qubit 3x4 grid, 8 cycles, 64 seeded bitstrings
    c = grid_circuit(3, 4, 8, seed=1)
    bs = random_bitstrings(c.n_qubits, 64, seed=2)
    got = tn.batch_amplitudes(c, bs)
    ref = sv.circuit_amplitudes(c, bs)
    assert np.allclose(got, ref, atol=1e-13)


def test_subcube_matches_statevector():
    c = grid_circuit(3, 3, 6, seed=4)
    fixed, open_q = subcube_spec(c.n_qubits, 4, seed=5)
    got = tn.network_amplitudes(c, fixed, open_q).reshape(-1)
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    assert np.allclose(got, ref, atol=1e-13)


def test_slices_match_projector_statevector_and_sum():
    c = grid_circuit(3, 3, 6, seed=12)
    count = _wire_counts(c)
    rng = np.random.default_rng(0)
    cuts = []
    while len(cuts) < 3:
        q = int(rng.integers(c.n_qubits))
        j = int(rng.integers(1, count[q]))
        if (q, j) not in cuts:
            cuts.append((q, j))
    fixed, open_q = subcube_spec(c.n_qubits, 3, seed=1)
    bs = subcube_bitstrings(fixed, open_q)
    total = 0
    for bits in itertools.product((0, 1), repeat=len(cuts)):
        assign = dict(zip(cuts, bits))
        got = tn.network_amplitudes(c, fixed, open_q, assign).reshape(-1)
        ref = sv.circuit_amplitudes(c, bs, assign)
        assert np.allclose(got, ref, atol=1e-13)
        total = total + got
    assert np.allclose(total, sv.circuit_amplitudes(c, bs), atol=1e-13)


def test_subslicing_under_small_cap_is_exact():
    c = grid_circuit(3, 3, 8, seed=2)
    fixed, open_q = subcube_spec(c.n_qubits, 3, seed=2)
    free = tn.network_amplitudes(c, fixed, open_q, cap_log2=30)
    tensors, open_labels = tn.circuit_tensors(c, fixed, open_q)
    extra, _ = tn.choose_subslices([t.labels for t in tensors], open_labels, 5)
    assert len(extra) > 0  # the cap really forces sub-slicing
    capped = tn.network_amplitudes(c, fixed, open_q, cap_log2=5)
    assert np.allclose(free, capped, atol=1e-13)


def test_order_independence():
    c = grid_circuit(2, 3, 4, seed=9)
    fixed, open_q = subcube_spec(c.n_qubits, 2, seed=3)
    tensors, open_labels = tn.circuit_tensors(c, fixed, open_q)
    ref = tn.contract_network(tensors, open_labels)
    rng = np.random.default_rng(4)
    for _ in range(3):
        # a random valid order: contract random pairs of live tensors
        live = list(range(len(tensors)))
        nxt = len(tensors)
        order = []
        while len(live) > 1:
            i, j = rng.choice(len(live), 2, replace=False)
            a, b = live[i], live[j]
            order.append((a, b))
            live = [x for x in live if x not in (a, b)] + [nxt]
            nxt += 1
        got = tn.contract_network(tensors, open_labels, order)
        assert np.allclose(got, ref, atol=1e-13)
