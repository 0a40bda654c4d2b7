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
