"""GPU parity of qubit-split plans (mode "split": a sliced separator between two halves of
the qubits, each half one stem absorbing fused blocks) against the FP64 state vector.

Tolerances: complex64 1e-5 and complex-half 1e-2 norm-wise, as for every other plan.  A
single slice is compared with the state vector of the circuit with projectors on the
sliced wire segments (oracle.statevector, the same route as the other per-slice tests).
"""
import numpy as np
import pytest

from inputs import grid_circuit, subcube_bitstrings, subcube_spec
from oracle import metrics
from oracle import statevector as sv
from paper_2504_09186_gb300 import tnc as T

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "chalf": 1e-2}


@pytest.fixture(scope="module")
def ctx():
    return T.Context(0)


@pytest.mark.parametrize("objective", ["flops", "time"])
@pytest.mark.parametrize("precision", ["c64", "chalf"])
def test_split_plan_all_slices_against_statevector(ctx, precision, objective):
    # 3 x 4 grid, 10 cycles, 2 open qubits, cap 2^8: 12 sliced separator indices
    c = grid_circuit(3, 4, 10, seed=1)
    fixed, open_q = subcube_spec(c.n_qubits, 2, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=4, log2_cap=8, mode="split", objective=objective)
    assert p.info()["n_sliced"] >= 8
    got = ctx.amplitudes(p, fixed[None, :], precision)[0]
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    assert metrics.rel_err_norm(got, ref) <= TOL[precision]
    # the explicit list of every slice id sums to the same amplitudes
    ids = np.arange(1 << p.info()["n_sliced"], dtype=np.int64)
    got_ids = ctx.amplitudes_ids(p, fixed[None, :], ids, precision)[0]
    assert metrics.rel_err_norm(got_ids, ref) <= TOL[precision]


@pytest.mark.parametrize("precision", ["c64", "chalf"])
def test_split_plan_sampled_slices_with_tensor_core_blocks(ctx, precision):
    # 4 x 5 grid, 12 cycles, 4 open qubits, cap 2^16, fused blocks chosen by modeled time:
    # the stems absorb blocks through tensor-core steps.  Seeded slices, one at a time,
    # against the projector state vector of each slice.
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(c.n_qubits, 4, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=4, log2_cap=16, mode="split", objective="time")
    if precision == "chalf":
        assert sum(st["tc"] for st in p.describe()["steps"]) >= 1
    cuts = p.sliced_cuts()
    s = len(cuts)
    bs = subcube_bitstrings(fixed, open_q)
    rng = np.random.default_rng(11)
    for sid in [0, (1 << s) - 1] + [int(x) for x in rng.integers(0, 1 << s, 4)]:
        assign = {cut: (sid >> t) & 1 for t, cut in enumerate(cuts)}
        ref = sv.circuit_amplitudes(c, bs, assign)
        got = ctx.amplitudes_ids(p, fixed[None, :], [sid], precision)[0]
        if np.linalg.norm(ref) < 1e-12:
            assert np.linalg.norm(got) < 1e-9
        else:
            assert metrics.rel_err_norm(got, ref) <= TOL[precision]


def test_sixty_qubit_slice_against_the_oracle(ctx):
    """The 60-qubit grid circuit itself (6 x 10, 24 cycles, one bitstring): a split plan at
    cap 2^26 slices over a hundred indices, so one slice (about 2^36 multiply-adds) is within
    the FP64 oracle's reach.  A seeded slice id (indices 63 and up at 0) on the GPU against the
    oracle's network contraction with the same cuts fixed.  complex64 within 1e-5; complex-half
    within the bound derived for one slice, 4 * 2^-11 * sqrt(stored tensors) (every stored
    tensor rounded once to fp16, the roundings adding in quadrature)."""
    from inputs import random_bitstrings
    from oracle import network as tn

    c = grid_circuit(6, 10, 24, seed=1)
    bits = random_bitstrings(60, 1, seed=4)[0]
    p = T.Plan.greedy(c, open_qubits=[], seed=3, trials=4, log2_cap=26, mode="split", objective="time")
    info = p.info()
    assert info["n_sliced"] > 100 and info["max_log2_size"] <= 26
    cuts = p.sliced_cuts()
    sid = int(np.random.default_rng(9).integers(0, 1 << 62))
    tensors, open_labels = tn.circuit_tensors(c, bits, [])
    tensors = tn.fix_labels(tensors, {("w", q, j): (sid >> t) & 1 for t, (q, j) in enumerate(cuts)})
    order, extra = tn.search_order([t.labels for t in tensors], open_labels, 23, trials=2)
    ref = 0.0
    for k in range(1 << len(extra)):
        sub = tn.fix_labels(tensors, {lab: (k >> t) & 1 for t, lab in enumerate(extra)})
        ref = ref + complex(tn.contract_network(sub, open_labels, order))
    assert abs(ref) > 0
    got64 = complex(ctx.amplitudes_ids(p, bits[None, :], [sid], "c64")[0, 0])
    got16 = complex(ctx.amplitudes_ids(p, bits[None, :], [sid], "chalf")[0, 0])
    assert abs(got64 - ref) <= 1e-5 * abs(ref)
    bound = 4 * 2.0 ** -11 * np.sqrt(info["n_leaves"] + info["n_steps"])
    assert abs(got16 - ref) <= bound * abs(ref)
