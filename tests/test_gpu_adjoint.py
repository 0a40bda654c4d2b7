"""GPU parity of the adjoint contraction (gate environments) against the FP64 oracle.

The oracle's environments come from forward/backward state vectors (an independent
route); the GPU ones from walking the contraction tree in reverse.  complex64 arithmetic
with FP64 accumulation: norm-wise relative error <= 1e-5 over all gate environments.
"""
import numpy as np
import pytest
import torch

from inputs import grid_circuit, random_bitstrings, subcube_bitstrings, subcube_spec
from oracle import metrics
from oracle import statevector as sv
from paper_2504_09186_gb300 import tnc as T
from paper_2504_09186_gb300.autograd import amplitudes as ad_amplitudes, fsim_torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    return T.Context(0)


def _arities(c):
    return [len(g.qubits) for g in c.gates]


def _flat(envs):
    return np.concatenate([np.asarray(e).reshape(-1) for e in envs])


def test_adjoint_unsliced_batch(ctx):
    c = grid_circuit(3, 3, 6, seed=3, fsim_mode="uniform")
    bs = random_bitstrings(9, 8, seed=4)
    w = np.random.default_rng(5).normal(size=8) + 1j * np.random.default_rng(6).normal(size=8)
    p = T.Plan.greedy(c, open_qubits=[], trials=4, log2_cap=26)
    env, amps = ctx.adjoint(p, bs, w[:, None], _arities(c))
    ref = sv.gate_environments(c, bs, w)
    assert metrics.rel_err_norm(_flat(env), _flat(ref)) <= 1e-5
    assert metrics.rel_err_norm(amps[:, 0], sv.circuit_amplitudes(c, bs)) <= 1e-5


def test_adjoint_sliced_subcube_and_identity(ctx):
    c = grid_circuit(4, 4, 10, seed=2, fsim_mode="uniform")
    fixed, open_q = subcube_spec(16, 3, seed=3)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=8, slices_min=2)
    assert p.info()["n_sliced"] >= 2
    rng = np.random.default_rng(8)
    w = rng.normal(size=8) + 1j * rng.normal(size=8)
    env, amps = ctx.adjoint(p, fixed[None, :], w[None, :], _arities(c))
    bs = subcube_bitstrings(fixed, open_q)
    ref = sv.gate_environments(c, bs, w)
    assert metrics.rel_err_norm(_flat(env), _flat(ref)) <= 1e-5
    # amplitude is linear in every gate: <E_g, U_g> = L for each g
    loss = np.sum(w * amps[0])
    for g, e in zip(c.gates, env):
        assert abs(np.sum(e * g.matrix) - loss) <= 1e-5 * abs(loss)


def test_gradient_config_20_qubits(ctx):
    # 20-qubit 4x5 grid, 12 cycles, fSim angles uniform in [0, pi], 256 bitstrings
    c = grid_circuit(4, 5, 12, seed=1, fsim_mode="uniform", param_seed=5)
    bs = random_bitstrings(20, 256, seed=6)
    rng = np.random.default_rng(7)
    w = rng.normal(size=256) + 1j * rng.normal(size=256)
    p = T.Plan.greedy(c, open_qubits=[], seed=3, trials=8, log2_cap=20)
    env, amps = ctx.adjoint(p, bs, w[:, None], _arities(c))
    ref = sv.gate_environments(c, bs, w)
    assert metrics.rel_err_norm(_flat(env), _flat(ref)) <= 1e-5
    assert metrics.rel_err_norm(amps[:, 0], sv.circuit_amplitudes(c, bs)) <= 1e-5


def test_autograd_fsim_angles_against_finite_differences(ctx):
    from inputs.circuits import fsim

    c = grid_circuit(3, 3, 6, seed=9, fsim_mode="uniform", param_seed=10)
    bs = random_bitstrings(9, 6, seed=11)
    coef = np.random.default_rng(12).normal(size=6) + 1j * np.random.default_rng(13).normal(size=6)
    p = T.Plan.greedy(c, open_qubits=[], trials=4, log2_cap=26)
    fs = [i for i, g in enumerate(c.gates) if g.kind == "fsim"]
    theta = torch.tensor([c.gates[i].params[0] for i in fs], dtype=torch.float64, requires_grad=True)
    phi = torch.tensor([c.gates[i].params[1] for i in fs], dtype=torch.float64, requires_grad=True)
    gates = []
    k = 0
    for g in c.gates:
        if g.kind == "fsim":
            gates.append(fsim_torch(theta[k], phi[k]))
            k += 1
        else:
            gates.append(torch.from_numpy(g.matrix))
    amps = ad_amplitudes(p, ctx, bs, _arities(c), gates)[:, 0]
    loss = torch.real(torch.sum(torch.from_numpy(coef) * amps))
    loss.backward()

    def loss_at(j, which, h):
        mats = [g.matrix.copy() for g in c.gates]
        th, ph = list(c.gates[fs[j]].params)
        if which == 0:
            th += h
        else:
            ph += h
        mats[fs[j]] = fsim(th, ph)
        cc = grid_circuit(3, 3, 6, seed=9, fsim_mode="uniform", param_seed=10)
        for g, m in zip(cc.gates, mats):
            g.matrix = m
        return float(np.real(np.sum(coef * sv.circuit_amplitudes(cc, bs))))

    h = 1e-3
    for j in (0, len(fs) // 2, len(fs) - 1):
        for which, grad in ((0, theta.grad), (1, phi.grad)):
            fd = (loss_at(j, which, h) - loss_at(j, which, -h)) / (2 * h)
            assert abs(float(grad[j]) - fd) <= 1e-4 * max(1.0, abs(fd)), (j, which, float(grad[j]), fd)


@pytest.mark.parametrize("sliced", [False, True])
def test_adjoint_recompute_matches_store_all(ctx, sliced):
    # a budget below the intermediates' size drops the largest and recomputes them from
    # their children in the backward pass: same kernels on the same inputs, bit-identical
    c = grid_circuit(4, 5, 12, seed=1, fsim_mode="uniform", param_seed=5)
    if sliced:
        fixed, open_q = subcube_spec(20, 4, seed=3)
        p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=12, slices_min=2)
        bs, n_out = fixed[None, :], 16
    else:
        p = T.Plan.greedy(c, open_qubits=[], seed=3, trials=8, log2_cap=20)
        bs, n_out = random_bitstrings(20, 16, seed=6), 1
    rng = np.random.default_rng(7)
    w = rng.normal(size=(len(bs), n_out)) + 1j * rng.normal(size=(len(bs), n_out))
    env0, amps0 = ctx.adjoint(p, bs, w, _arities(c))
    env1, amps1 = ctx.adjoint(p, bs, w, _arities(c), memory_mib=1)
    assert np.array_equal(amps0, amps1)
    assert all(np.array_equal(a, b) for a, b in zip(env0, env1))
