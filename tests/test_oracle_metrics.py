"""Pins of oracle/metrics.py against closed forms and hand-worked values.

Each case is chosen so that a plausible slip in the metric (a dropped "- 1", a missing or
doubled 2^n factor, a floor taken in the wrong place, an off-by-one in the empirical CDF)
changes the value by far more than the tolerance.
"""
import numpy as np
import pytest

from oracle import metrics


def test_rel_err_norm_hand_worked():
    # ||(3, 4i) - (0, 0)|| over ||(0, 5)||: a - ref = (3, -1i), norm sqrt(10); ||ref|| = 5
    a = np.array([3.0, 4.0j])
    ref = np.array([0.0, 5.0j])
    assert metrics.rel_err_norm(a, ref) == pytest.approx(np.sqrt(10.0) / 5.0, rel=1e-15)


def test_rel_err_max_floor_hand_worked():
    # n = 4 qubits: floor = 2^-2 * 1e-3 = 2.5e-4.
    # entry 0: |1.001 - 1| / 1 = 1e-3
    # entry 1: |5e-5| / max(1e-6, 2.5e-4) = 0.2   (without the floor it would be 50)
    # entry 2: exact -> 0
    ref = np.array([1.0, 1e-6, 0.5j])
    a = np.array([1.001, 1e-6 + 5e-5, 0.5j])
    assert metrics.rel_err_max(a, ref, 4) == pytest.approx(0.2, rel=1e-9)
    # above the floor the relative error of the entry is what counts
    assert metrics.rel_err_max(a[:1], ref[:1], 4) == pytest.approx(1e-3, rel=1e-9)
    # the floor shrinks with n: at n = 30 it is 2^-15 * 1e-3 ~ 3.05e-8, below 1e-6
    assert metrics.rel_err_max(a[1:2], ref[1:2], 30) == pytest.approx(50.0, rel=1e-9)


def test_xeb_weighted_uniform_is_zero():
    # p = 2^-n on every bitstring: F = 2^n * 2^-n * sum(p_ref) / sum(p_ref) - 1 = 0 exactly,
    # whatever the reference weights
    n = 10
    rng = np.random.default_rng(1)
    p_ref = rng.exponential(size=1 << 6) * 2.0 ** -n
    assert metrics.xeb_weighted(p_ref, np.full(p_ref.size, 2.0 ** -n), n) == pytest.approx(0.0, abs=1e-12)


def test_xeb_weighted_porter_thomas_is_one():
    # Over all N = 2^n bitstrings with N*p ~ Exp(1) (normalised), F = N * sum p^2 - 1, whose
    # expectation is 2N/(N+1) - 1 ~ 1; the sampling spread of N*sum p^2 is about
    # sqrt(20/N) ~ 0.018 at N = 2^16 (fourth moment of Exp(1) is 24).
    n = 16
    rng = np.random.default_rng(2)
    p = rng.exponential(size=1 << n)
    p /= p.sum()
    f = metrics.xeb_weighted(p, p, n)
    assert f == pytest.approx(1.0, abs=0.08)
    # a distribution concentrated on one bitstring: F = 2^n - 1
    q = np.zeros(1 << n)
    q[3] = 1.0
    assert metrics.xeb_weighted(q, q, n) == pytest.approx(2.0 ** n - 1.0, rel=1e-12)


def test_xeb_sampled_two_qubit_hand_worked():
    # n = 2, p = (1/2, 1/4, 1/8, 1/8).  Four samples x = 00, 00, 01, 10 have probabilities
    # 1/2, 1/2, 1/4, 1/8: mean 11/32, F = 4 * 11/32 - 1 = 3/8.
    # The expectation over samples drawn from p is 4 * sum p^2 - 1 = 4 * 11/32 - 1 = 3/8 too.
    assert metrics.xeb_sampled(np.array([0.5, 0.5, 0.25, 0.125]), 2) == pytest.approx(0.375, rel=1e-15)
    # uniform samples of a uniform distribution: F = 0
    assert metrics.xeb_sampled(np.full(7, 0.25), 2) == pytest.approx(0.0, abs=1e-15)


@pytest.mark.parametrize("n_out", [64, 4096, 1 << 16])
def test_porter_thomas_ks_of_exact_quantile_grid(n_out):
    # x_i = F^-1((i - 1/2) / N) for Exp(1): the empirical CDF steps sit exactly 1/(2N) above
    # and below the CDF at every x_i, so the KS distance is 1/(2N).
    u = (np.arange(1, n_out + 1) - 0.5) / n_out
    x = -np.log1p(-u)
    rng = np.random.default_rng(n_out)
    probs = rng.permutation(x) / n_out  # order must not matter
    mean, m2, ks = metrics.porter_thomas(probs)
    assert ks == pytest.approx(0.5 / n_out, rel=1e-9)
    # midpoint quadrature of the first two moments of Exp(1) (1 and 2); the error of the
    # last cell, around the integrable log singularity, is O(log N / N)
    tol = 4.0 * np.log(n_out) / n_out
    assert mean == pytest.approx(1.0, abs=tol)
    assert m2 == pytest.approx(2.0, abs=4.0 * np.log(n_out) ** 2 / n_out)


def test_porter_thomas_ks_detects_a_non_exponential_law():
    # N*p uniform on (0, 2): same mean as Exp(1); KS = sup |u/2 - (1 - e^-u)| on (0, 2),
    # attained where e^-u = 1/2 (u = ln 2): ln2/2 - 1/2 + ... = 1/2 - ln(2)/2 ~ 0.1534
    n_out = 1 << 14
    x = (np.arange(n_out) + 0.5) / n_out * 2.0
    _, _, ks = metrics.porter_thomas(x / n_out)
    assert ks == pytest.approx(0.5 - np.log(2.0) / 2.0, abs=2e-4)
