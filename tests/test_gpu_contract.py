"""GPU parity of single pairwise contractions (tnc_contract) against the FP64 oracle.

Inputs are complex normal(0, 1/sqrt(K)) with seeded random index permutations of A, B
and C (the single-step sweep workload), rounded to the storage precision on the host;
the oracle contracts the rounded inputs exactly in FP64, so the remaining error is FP32
accumulation plus one rounding of the output: norm-wise <= 1e-5 (c64), 2e-3 (fp16,
unit roundoff 2^-11 times a margin), 1e-2 (bf16, 2^-8 times a margin).
"""
import numpy as np
import pytest
import torch

from inputs import random_complex, random_labels_perm
from oracle import metrics, pairwise
from paper_2504_09186_gb300 import tnc as T

pytestmark = pytest.mark.gpu

DT = {"c64": torch.float32, "chalf": torch.float16, "cbf16": torch.bfloat16}
TOL = {"c64": 1e-5, "chalf": 2e-3, "cbf16": 1e-2}


@pytest.fixture(scope="module")
def ctx():
    return T.Context(0)


def make_case(m, k, n, seed):
    la = random_labels_perm(list(range(m)) + list(range(100, 100 + k)), seed)
    lb = random_labels_perm(list(range(100, 100 + k)) + list(range(200, 200 + n)), seed + 1)
    lc = random_labels_perm(list(range(m)) + list(range(200, 200 + n)), seed + 2)
    sigma = 1.0 / np.sqrt(2.0 ** k) if k else 1.0
    a = random_complex(1 << len(la), sigma, seed + 3)
    b = random_complex(1 << len(lb), sigma, seed + 4)
    return a, la, b, lb, lc


def to_planar(x, dtype):
    t = torch.from_numpy(np.concatenate([x.real, x.imag])).to(dtype)
    back = t.to(torch.float64).numpy()
    n = x.size
    return t.cuda(), back[:n] + 1j * back[n:]


def run(ctx, precision, a, la, b, lb, lc):
    ta, aq = to_planar(a, DT[precision])
    tb, bq = to_planar(b, DT[precision])
    tc = torch.empty(2 << len(lc), dtype=DT[precision], device="cuda")
    e = ctx.contract(precision, ta, la, tb, lb, tc, lc)
    torch.cuda.synchronize()
    cc = tc.to(torch.float64).cpu().numpy()
    n = 1 << len(lc)
    return (cc[:n] + 1j * cc[n:]) * 2.0 ** e, aq, bq


SMALL = [(2, 3, 2), (0, 5, 0), (3, 0, 2), (6, 10, 6), (10, 4, 1), (9, 2, 2), (1, 14, 1), (4, 12, 3), (7, 9, 7), (12, 6, 0)]


@pytest.mark.parametrize("precision", ["c64", "chalf", "cbf16"])
@pytest.mark.parametrize("shape", SMALL)
def test_small_shapes_elementwise(ctx, precision, shape):
    a, la, b, lb, lc = make_case(*shape, seed=31 * sum(shape) + shape[0])
    got, aq, bq = run(ctx, precision, a, la, b, lb, lc)
    ref = pairwise.contract(aq, la, bq, lb, lc)
    assert metrics.rel_err_norm(got, ref) <= TOL[precision]


LARGE = [(2, 22, 2), (12, 8, 8), (16, 2, 2), (8, 14, 8)]


@pytest.mark.parametrize("precision", ["c64", "chalf"])
@pytest.mark.parametrize("shape", LARGE)
def test_large_shapes_sampled(ctx, precision, shape):
    a, la, b, lb, lc = make_case(*shape, seed=7 * sum(shape))
    got, aq, bq = run(ctx, precision, a, la, b, lb, lc)
    rng = np.random.default_rng(sum(shape))
    idx = np.unique(np.concatenate([[0, len(got) - 1], rng.integers(0, len(got), 62)]))
    ref = pairwise.contract_at(aq, la, bq, lb, lc, idx)
    assert metrics.rel_err_norm(got[idx], ref) <= TOL[precision]


# GEPDOT shapes (few outputs, long K; Sec. V-B) whose CTAs walk two or more K steps after
# the split over K: raw tiles streamed through the cp.async ring (profile kind 7);
# elementwise against the oracle and bit for bit against the kernel that loads each K step
# synchronously (same k order per thread).
GEPDOT = [(2, 22, 2), (1, 23, 3), (3, 21, 4), (0, 22, 2), (4, 20, 1)]


@pytest.mark.parametrize("precision", ["c64", "chalf", "cbf16"])
@pytest.mark.parametrize("shape", GEPDOT)
def test_gepdot_streamed(ctx, precision, shape, monkeypatch):
    a, la, b, lb, lc = make_case(*shape, seed=17 * sum(shape) + shape[2])
    got, aq, bq = run(ctx, precision, a, la, b, lb, lc)
    assert int(ctx.profile_read(cap=1)["kind"][0]) == 7
    ref = pairwise.contract(aq, la, bq, lb, lc)
    assert metrics.rel_err_norm(got, ref) <= TOL[precision]
    monkeypatch.setenv("TNC_NO_STREAM", "1")
    ctx1 = T.Context(0)
    sync, _, _ = run(ctx1, precision, a, la, b, lb, lc)
    assert int(ctx1.profile_read(cap=1)["kind"][0]) in (0, 1)
    assert np.array_equal(got, sync)


# Long K loops over a thin operand (at most 4 rows or columns; not GEPDOT-sized outputs): the
# same ring, the same checks.
THIN = [(12, 14, 2), (14, 12, 1), (2, 13, 10)]


@pytest.mark.parametrize("precision", ["c64", "chalf"])
@pytest.mark.parametrize("shape", THIN)
def test_thin_long_k_streamed(ctx, precision, shape, monkeypatch):
    a, la, b, lb, lc = make_case(*shape, seed=19 * sum(shape) + shape[0])
    got, aq, bq = run(ctx, precision, a, la, b, lb, lc)
    assert int(ctx.profile_read(cap=1)["kind"][0]) == 7
    assert metrics.rel_err_norm(got, pairwise.contract(aq, la, bq, lb, lc)) <= TOL[precision]
    monkeypatch.setenv("TNC_NO_STREAM", "1")
    ctx1 = T.Context(0)
    sync, _, _ = run(ctx1, precision, a, la, b, lb, lc)
    assert np.array_equal(got, sync)
