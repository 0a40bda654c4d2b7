"""The 30-qubit workload end to end against stored FP64 state-vector amplitudes.

5x6 grid circuit, 14 cycles (seed 1); a 1024-amplitude sub-cube (qubits 20..29 open, the
other bits from seed 2); greedy plan (seed 3, 64 trials) with exactly 6 sliced indices and
every intermediate at most 2^26 entries.  All 64 slices are contracted and summed; the
expected values were written by tests/golden/make_s30_golden.py with the C state-vector
oracle.  Bars: complex64 <= 1e-5 and complex-half <= 1e-2 norm-wise relative error, and the
sub-cube XEB of the half-precision result within 1% of the oracle's.
"""
import os

import numpy as np
import pytest

from inputs import grid_circuit, subcube_spec
from oracle import metrics
from paper_2504_09186_gb300 import tnc as T

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "s30_subcube_amplitudes.txt")


def _golden():
    v = np.loadtxt(GOLDEN)
    return v[:, 0] + 1j * v[:, 1]


@pytest.fixture(scope="module")
def s30():
    c = grid_circuit(5, 6, 14, seed=1)
    fixed, open_q = subcube_spec(30, 10, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=64, log2_cap=26, slices_min=6, slices_max=6)
    return c, fixed, p


def test_s30_plan_shape(s30):
    _, _, p = s30
    info = p.info()
    assert info["n_sliced"] == 6 and info["max_log2_size"] <= 26 and info["n_open"] == 10


def test_s30_all_slices_against_statevector(s30):
    _, fixed, p = s30
    ctx = T.Context(0)
    ref = _golden()
    half = ctx.amplitudes(p, fixed[None, :], "chalf", profile=True)[0]
    kinds = set(int(k) for k in ctx.profile_read()["kind"])
    assert {4, 5} <= kinds  # TMA tensor-core steps, one-CTA-per-tile and persistent
    full = ctx.amplitudes(p, fixed[None, :], "c64")[0]
    assert metrics.rel_err_norm(full, ref) <= 1e-5
    assert metrics.rel_err_norm(half, ref) <= 1e-2
    # per amplitude: the errors of the 1024 entries are many independent roundings summed,
    # about complex normal with rms sigma <= tol * rms(ref) when the norm-wise bar holds;
    # a complex normal exceeds 5 sigma with probability e^-25, so over 1024 entries every
    # |a_b - ref_b| <= 5 tol rms(ref), and rel_err_max (the relative error of each entry,
    # floored at 2^-15 * 1e-3) is at most that over the smallest floored |ref_b|
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    floor = np.maximum(np.abs(ref), 2.0 ** -15 * 1e-3)
    for got, tol in ((full, 1e-5), (half, 1e-2)):
        assert np.all(np.abs(got - ref) <= 5 * tol * rms)
        assert metrics.rel_err_max(got, ref, 30) <= 5 * tol * rms / floor.min()
    p_ref = np.abs(ref) ** 2
    f_ref = metrics.xeb_weighted(p_ref, p_ref, 30)
    f_half = metrics.xeb_weighted(p_ref, np.abs(half) ** 2, 30)
    assert abs(f_half - f_ref) <= 0.01 * abs(f_ref)


@pytest.fixture
def clean_tuning_cache():
    T.load_library()
    T.tune_clear()
    yield
    T.tune_clear()


def test_s30_autotuned_against_statevector(s30, tmp_path, clean_tuning_cache):
    """Tile configurations chosen by timing keep parity, runs stay deterministic, and a
    program built later from the saved cache runs the same configurations bit for bit."""
    _, fixed, p = s30
    ctx = T.Context(0)
    ref = _golden()
    info = ctx.autotune(p, fixed[None, :], "chalf")
    assert info["steps_tuned"] > 0 and info["candidates"] >= info["steps_tuned"]
    assert info["seconds_tuned"] <= info["seconds_default"] * (1 + 1e-9)
    tuned = ctx.amplitudes(p, fixed[None, :], "chalf")[0]
    assert np.array_equal(tuned, ctx.amplitudes(p, fixed[None, :], "chalf")[0])
    assert metrics.rel_err_norm(tuned, ref) <= 1e-2
    p_ref = np.abs(ref) ** 2
    f_ref = metrics.xeb_weighted(p_ref, p_ref, 30)
    assert abs(metrics.xeb_weighted(p_ref, np.abs(tuned) ** 2, 30) - f_ref) <= 0.01 * abs(f_ref)
    path = tmp_path / "tune.txt"
    T.tune_save(str(path))
    n = T.tune_size()
    assert n <= info["steps_changed"]
    T.tune_clear()
    T.tune_load(str(path))
    assert T.tune_size() == n
    ctx2 = T.Context(0)  # a new context builds its own program from the cache
    assert np.array_equal(ctx2.amplitudes(p, fixed[None, :], "chalf")[0], tuned)


@pytest.mark.parametrize("precision", ["chalf", "c64"])
def test_s30_concurrent_branches_match_serial(s30, precision, monkeypatch):
    """Independent subtrees run on concurrent streams (with the arena's memory hazards and the
    shared split-K buffer as dependencies); eager, graph-captured and graph-replayed calls are
    bit-identical to running every launch on one stream."""
    _, fixed, p = s30
    ctx = T.Context(0)
    conc = ctx.amplitudes(p, fixed[None, :], precision)[0]
    graph = [ctx.amplitudes(p, fixed[None, :], precision, use_graph=True)[0] for _ in range(3)]
    monkeypatch.setenv("TNC_SERIAL", "1")
    ser = T.Context(0).amplitudes(p, fixed[None, :], precision)[0]
    assert np.array_equal(conc, ser)
    for g in graph:
        assert np.array_equal(g, ser)
