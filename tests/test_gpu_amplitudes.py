"""GPU parity of amplitudes through the C boundary against the FP64 oracle.

Tolerances (norm-wise relative error over the batch): complex64 path 1e-5 and
complex-half 1e-2, as required of the two paths.  complex-bf16 has no stated tolerance;
its bound here is derived: every stored tensor (each leaf and each intermediate) is
rounded once to bf16 with unit roundoff u = 2^-9, the amplitude is multilinear in the
stored tensors, so independent relative perturbations of size ~u add in quadrature:
err ~ u * sqrt(n_stored).  The bound is 4 u sqrt(n_stored).
"""
import itertools

import numpy as np
import pytest

from inputs import grid_circuit, random_bitstrings, subcube_bitstrings, subcube_spec
from inputs.circuits import custom_circuit, SQRT_X, fsim
from oracle import metrics
from oracle import statevector as sv
from paper_2504_09186_gb300 import tnc as T

pytestmark = pytest.mark.gpu

TOL = {"c64": 1e-5, "chalf": 1e-2, "cbf16": 4e-2}


def bf16_bound(plan):
    info = plan.info()
    return 4.0 * 2.0 ** -9 * np.sqrt(info["n_leaves"] + info["n_steps"])


@pytest.fixture(scope="module")
def ctx():
    return T.Context(0)


@pytest.mark.parametrize("precision", ["c64", "chalf", "cbf16"])
def test_tiny_config_batch_of_bitstrings(ctx, precision):
    # 12-qubit 3x4 grid, 8 cycles, unsliced, 64 seeded bitstrings
    c = grid_circuit(3, 4, 8, seed=1)
    bs = random_bitstrings(c.n_qubits, 64, seed=2)
    p = T.Plan.greedy(c, open_qubits=[], seed=3, trials=8, log2_cap=26)
    assert p.info()["n_sliced"] == 0
    got = ctx.amplitudes(p, bs, precision)[:, 0]
    ref = sv.circuit_amplitudes(c, bs)
    err = metrics.rel_err_norm(got, ref)
    tol = bf16_bound(p) if precision == "cbf16" else TOL[precision]
    assert err <= tol, err


@pytest.mark.parametrize("precision", ["c64", "chalf"])
def test_all_open_is_the_state(ctx, precision):
    c = grid_circuit(3, 3, 6, seed=4, fsim_mode="uniform")
    n = c.n_qubits
    p = T.Plan.greedy(c, open_qubits=list(range(n)), seed=1, trials=4, log2_cap=26)
    got = ctx.amplitudes(p, None, precision)[0]
    ref = sv.final_state(c).reshape(-1)
    assert metrics.rel_err_norm(got, ref) <= TOL[precision]


def test_sliced_plan_each_slice_and_sum(ctx):
    c = grid_circuit(4, 4, 10, seed=1)
    n = c.n_qubits
    fixed, open_q = subcube_spec(n, 4, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=9, slices_min=3)
    cuts = p.sliced_cuts()
    s = len(cuts)
    assert s >= 3
    bs = subcube_bitstrings(fixed, open_q)
    total = 0
    for sid in range(1 << s):
        assign = {cut: (sid >> t) & 1 for t, cut in enumerate(cuts)}
        ref = sv.circuit_amplitudes(c, bs, assign)
        got = ctx.amplitudes(p, fixed[None, :], "c64", slice_begin=sid, slice_count=1)[0]
        assert metrics.rel_err_norm(got, ref) <= 1e-5 or np.linalg.norm(ref) < 1e-12
        total = total + ref
    full = ctx.amplitudes(p, fixed[None, :], "c64")[0]
    assert metrics.rel_err_norm(full, sv.circuit_amplitudes(c, bs)) <= 1e-5
    assert np.allclose(total, sv.circuit_amplitudes(c, bs), atol=1e-12)


def test_wave_sizes_are_deterministic(ctx):
    c = grid_circuit(4, 4, 10, seed=1)
    fixed, open_q = subcube_spec(16, 3, seed=2)
    bs = np.stack([fixed, 1 - fixed, fixed])
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=9, slices_min=3)
    outs = [ctx.amplitudes(p, bs, "c64", wave=w) for w in (0, 1, 3, 5)]
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])  # same fixed summation order, bit-identical
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(1 - fixed, open_q))
    assert metrics.rel_err_norm(outs[0][1], ref) <= 1e-5


def test_cuda_graph_replay_is_identical(ctx):
    # several waves; graphs are captured on the second call and replayed afterwards
    c = grid_circuit(4, 4, 10, seed=1)
    fixed, open_q = subcube_spec(16, 3, seed=2)
    bs = np.stack([fixed, 1 - fixed])
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=9, slices_min=3)
    for prec in ("c64", "chalf"):
        ref = ctx.amplitudes(p, bs, prec, wave=3)
        for _ in range(3):
            got = ctx.amplitudes(p, bs, prec, wave=3, use_graph=True)
            assert np.array_equal(got, ref)


def test_half_precision_scaling_keeps_small_amplitudes(ctx):
    # 20 qubits: amplitudes ~2^-10, intermediates far below fp16's normal range without scaling
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(20, 6, seed=3)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=16, slices_min=2)
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    for prec in ("c64", "chalf", "cbf16"):
        got = ctx.amplitudes(p, fixed[None, :], prec)[0]
        tol = bf16_bound(p) if prec == "cbf16" else TOL[prec]
        assert metrics.rel_err_norm(got, ref) <= tol, prec


def test_edge_cases(ctx):
    # a qubit with no gates, a single 2-qubit gate, and an empty slice range is rejected
    c = custom_circuit(3, [((0,), SQRT_X), ((0, 1), fsim(0.3, 0.2))])
    bs = np.array(list(itertools.product((0, 1), repeat=3)), dtype=np.uint8)
    p = T.Plan.greedy(c, open_qubits=[], trials=2)
    got = ctx.amplitudes(p, bs, "c64")[:, 0]
    assert metrics.rel_err_norm(got, sv.circuit_amplitudes(c, bs)) <= 1e-6
    with pytest.raises(T.TncError):
        ctx.amplitudes(p, bs, "c64", slice_begin=0, slice_count=2)
    with pytest.raises(T.TncError):
        ctx.amplitudes(p, bs * 2, "c64")


@pytest.mark.parametrize("rows,cols,cycles,n_open,cap", [(4, 4, 10, 4, 12), (4, 5, 12, 6, 18)])
def test_stem_plan_fused_chains(ctx, rows, cols, cycles, n_open, cap):
    # stem order: one tensor absorbs the leaves; long absorb chains run as fused kernels
    c = grid_circuit(rows, cols, cycles, seed=1)
    n = c.n_qubits
    fixed, open_q = subcube_spec(n, n_open, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=cap, mode="stem")
    info = p.info()
    assert info["n_fused"] >= 4
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    for prec in ("c64", "chalf"):
        fused = ctx.amplitudes(p, fixed[None, :], prec, fuse=True)[0]
        plain = ctx.amplitudes(p, fixed[None, :], prec, fuse=False)[0]
        assert metrics.rel_err_norm(fused, ref) <= TOL[prec], prec
        assert metrics.rel_err_norm(plain, ref) <= TOL[prec], prec


@pytest.mark.parametrize("precision", ["c64", "chalf"])
def test_tree_reuse_across_slices_is_bit_identical(ctx, precision, monkeypatch):
    # steps whose subtree fixes no sliced index (or only some) run once per assignment of the
    # indices they depend on (Sec. III-B tree-like reuse); the values cannot change
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(20, 6, seed=3)
    bs = np.stack([fixed, 1 - fixed])
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=14, slices_min=4)
    assert p.info()["n_sliced"] >= 4
    got = ctx.amplitudes(p, bs, precision, profile=True)
    flops_reuse = ctx.profile_read()["flops"].sum()
    monkeypatch.setenv("TNC_NO_REUSE", "1")
    ctx1 = T.Context(0)
    ref = ctx1.amplitudes(p, bs, precision, profile=True)
    flops_all = ctx1.profile_read()["flops"].sum()
    assert np.array_equal(got, ref)
    assert flops_reuse < flops_all  # some steps ran fewer times
    exact = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    assert metrics.rel_err_norm(got[0], exact) <= TOL[precision]


def test_sharded_slices_with_gpu_chunks(ctx, tmp_path):
    # chunks of consecutive slice ids through the library, every chunk verified by rerun
    # (the GPU sums are deterministic, so the rerun must be bit-identical)
    from paper_2504_09186_gb300 import shard

    c = grid_circuit(4, 4, 10, seed=1)
    fixed, open_q = subcube_spec(16, 3, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=9, slices_min=4)
    n = 1 << p.info()["n_sliced"]
    run = shard.gpu_chunk(ctx, p, fixed[None, :], "c64")
    spec = shard.ShardSpec(n_slices=n, chunk=4)
    got = shard.run_rank(spec, run, shard.CheckpointStore(str(tmp_path), 0), verify_fraction=1.0)
    full = ctx.amplitudes(p, fixed[None, :], "c64")
    assert np.allclose(got, full, rtol=1e-12, atol=1e-15)
    assert metrics.rel_err_norm(got[0], sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))) <= 1e-5


@pytest.mark.parametrize("precision,tol", [("c64", 1e-5), ("chalf", 1e-2)])
def test_lifetime_aware_slicing_and_branch_exchange_plan(ctx, precision, tol):
    """A plan sliced by executed cost under tree-like reuse, with branch exchange, contracts
    to the state-vector amplitudes, and its reuse run equals the run of every slice."""
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(20, 6, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=14, slices_min=4, slicing="reuse",
                      branch_exchange=True)
    assert p.info()["n_sliced"] >= 4
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    got = ctx.amplitudes(p, fixed[None, :], precision)[0]
    assert metrics.rel_err_norm(got, ref) <= tol
    n = 1 << p.info()["n_sliced"]
    parts = sum(ctx.amplitudes(p, fixed[None, :], precision, slice_begin=s, slice_count=1)[0] for s in range(n))
    assert metrics.rel_err_norm(parts, got) <= 1e-12 if precision == "c64" else metrics.rel_err_norm(parts, got) <= tol


def test_concurrent_branches_with_splits_match_serial(monkeypatch):
    """A plan with split-K steps (GEPDOT-shaped) and many small branches: the concurrent
    schedule equals the serial one bit for bit, per slice and over all slices."""
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(20, 2, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=12, slices_min=3)
    ctx = T.Context(0)
    got = {prec: ctx.amplitudes(p, fixed[None, :], prec) for prec in ("c64", "chalf")}
    one = ctx.amplitudes(p, fixed[None, :], "chalf", slice_begin=1, slice_count=1)
    monkeypatch.setenv("TNC_SERIAL", "1")
    ctx1 = T.Context(0)
    for prec in ("c64", "chalf"):
        assert np.array_equal(got[prec], ctx1.amplitudes(p, fixed[None, :], prec))
    assert np.array_equal(one, ctx1.amplitudes(p, fixed[None, :], "chalf", slice_begin=1, slice_count=1))


def test_library_random_grid_circuit_against_statevector(ctx):
    """A circuit made by tnc_circuit_random_grid (uniform fSim angles) contracts to the
    state-vector amplitudes of its exported gates, in c64 and chalf."""
    gl = T.random_grid(4, 4, 10, seed=7, fsim_mode="uniform")
    gates = []
    for g in range(len(gl)):
        a = int(gl.arity[g])
        d = 1 << a
        m = gl.matrices[g, 0:2 * d * d:2] + 1j * gl.matrices[g, 1:2 * d * d:2]
        gates.append((gl.qubits[g, :a], m.reshape(d, d)))
    circ = custom_circuit(16, gates)
    fixed, open_q = subcube_spec(16, 4, seed=2)
    p = T.Plan.greedy(gl, open_qubits=open_q, seed=3, trials=8, log2_cap=12, slices_min=2)
    ref = sv.circuit_amplitudes(circ, subcube_bitstrings(fixed, open_q))
    for prec, tol in (("c64", 1e-5), ("chalf", 1e-2)):
        assert metrics.rel_err_norm(ctx.amplitudes(p, fixed[None, :], prec)[0], ref) <= tol


def test_amplitudes_over_listed_slice_ids(ctx):
    """tnc_amplitudes_ids: the sum over a listed subset (out of order, one id repeated) equals
    the sum of single-slice calls in list order, and a contiguous list equals the range call,
    bit for bit."""
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(20, 4, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=12, slices_min=4)
    n = 1 << p.info()["n_sliced"]
    ids = [5, 1, n - 1, 1, 7]
    for prec in ("c64", "chalf"):
        got = ctx.amplitudes_ids(p, fixed[None, :], ids, prec)
        acc = np.zeros_like(got)
        for sid in ids:
            acc = acc + ctx.amplitudes(p, fixed[None, :], prec, slice_begin=sid, slice_count=1)
        assert np.array_equal(got, acc)
        rng = ctx.amplitudes(p, fixed[None, :], prec, slice_begin=2, slice_count=6)
        assert np.array_equal(ctx.amplitudes_ids(p, fixed[None, :], list(range(2, 8)), prec), rng)
    with pytest.raises(T.TncError):
        ctx.amplitudes_ids(p, fixed[None, :], [n], "c64")


@pytest.mark.parametrize("precision", ["c64", "chalf"])
def test_post_lifetime_merging(ctx, precision):
    """Post-lifetime merging (Sec. III-B): on a 20-qubit plan whose 12 sliced indices die
    early, summing each index right after the step that contracts it gives the state-vector
    amplitudes within the precision's bar, agrees with the unmerged call, runs exactly the
    executed multiply-adds the planner predicts for it (2^27.7 against 2^29.1), and is
    deterministic."""
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(20, 4, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=12, slices_min=8, slices_max=64)
    info = p.info()
    assert info["log2_executed_flops_merged"] < info["log2_executed_flops"] - 1
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    plain = ctx.amplitudes(p, fixed[None, :], precision, profile=True, fuse=False)[0]
    f_plain = float(ctx.profile_read()["flops"].sum())
    merged = ctx.amplitudes(p, fixed[None, :], precision, profile=True, fuse=False, merge=True)[0]
    f_merged = float(ctx.profile_read()["flops"].sum())
    tol = TOL[precision]
    assert metrics.rel_err_norm(plain, ref) <= tol
    assert metrics.rel_err_norm(merged, ref) <= tol
    assert metrics.rel_err_norm(merged, plain) <= tol
    assert f_plain == pytest.approx(8 * 2.0 ** info["log2_executed_flops"], rel=1e-9)
    assert f_merged == pytest.approx(8 * 2.0 ** info["log2_executed_flops_merged"], rel=1e-9)
    assert np.array_equal(merged, ctx.amplitudes(p, fixed[None, :], precision, fuse=False, merge=True)[0])


@pytest.mark.parametrize("precision", ["c64", "chalf"])
def test_cluster_cooperative_chains(ctx, precision):
    """Fused chains whose on-chip tile exceeds one CTA's 2^12 entries run on a thread-block
    cluster (Sec. IV): 20-qubit stem plan whose chains hold tiles of 2^15 entries over eight
    CTAs, links reading their inputs from peer CTAs' shared memory.  Against the state vector,
    and against the same plan without fusion."""
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(20, 6, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=20, mode="stem", cluster_chains=True)
    chains = p.describe()["chains"]
    assert any(ch["tile_bits"] > 12 for ch in chains)
    assert all(ch["tile_bits"] <= 12 for ch in T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=20,
                                                               mode="stem").describe()["chains"])
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    fused = ctx.amplitudes(p, fixed[None, :], precision, fuse=True, profile=True)[0]
    assert 2 in set(int(k) for k in ctx.profile_read()["kind"])  # the chain kernels ran
    plain = ctx.amplitudes(p, fixed[None, :], precision, fuse=False)[0]
    assert metrics.rel_err_norm(fused, ref) <= TOL[precision]
    assert metrics.rel_err_norm(fused, plain) <= TOL[precision]
    # deterministic
    assert np.array_equal(fused, ctx.amplitudes(p, fixed[None, :], precision, fuse=True)[0])


@pytest.mark.parametrize("precision", ["c64", "chalf"])
def test_persistent_steps_launch(precision, monkeypatch):
    """Every step of a SIMT program in one persistent launch per wave (TNC_NO_TC=1 puts all
    steps of this 20-qubit plan on the SIMT kernels): bit-identical to the per-step launches,
    eagerly and graph-replayed, with tree-like reuse over all slices, over listed slice ids,
    and with one-instance waves whose final GEPDOT splits over K (the reduce runs inside the
    launch after a grid barrier); against the state vector at the path's tolerance."""
    monkeypatch.setenv("TNC_NO_TC", "1")
    ctx = T.Context(0)
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(c.n_qubits, 2, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=18)
    assert p.info()["n_sliced"] >= 1
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    row = fixed[None, :]
    for wave in (0, 1):
        base = ctx.amplitudes(p, row, precision, wave=wave, profile=True)[0]
        kinds = set(int(k) for k in ctx.profile_read()["kind"])
        assert kinds <= {0, 1, 7}
        if wave == 1:
            assert kinds & {1, 7}  # the final GEPDOT (split over K in one-instance waves)
        per = ctx.amplitudes(p, row, precision, wave=wave, persistent=True, profile=True)[0]
        prof = ctx.profile_read()
        assert set(int(k) for k in prof["kind"]) == {8} and int(prof["launches"][0]) >= 1
        assert np.array_equal(per, base)
        for _ in range(3):
            assert np.array_equal(ctx.amplitudes(p, row, precision, wave=wave, persistent=True, use_graph=True)[0], base)
        assert metrics.rel_err_norm(per, ref) <= TOL[precision]
    ids = np.array([0, 3, 1], dtype=np.int64) % (1 << p.info()["n_sliced"])
    a = ctx.amplitudes_ids(p, row, ids, precision)
    b = ctx.amplitudes_ids(p, row, ids, precision, persistent=True)
    assert np.array_equal(a, b)
