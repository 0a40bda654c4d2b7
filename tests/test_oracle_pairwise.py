"""Pins for the single pairwise contraction (Sec. II-A, the M x K x N GEMM view)."""
import numpy as np
import pytest

from inputs import random_complex, random_labels_perm
from oracle import pairwise as pw


def _case(ra_free, rk, rb_free, seed):
    labels_a = list(range(ra_free)) + list(range(100, 100 + rk))
    labels_b = list(range(100, 100 + rk)) + list(range(200, 200 + rb_free))
    la = random_labels_perm(labels_a, seed)
    lb = random_labels_perm(labels_b, seed + 1)
    lc = random_labels_perm(list(range(ra_free)) + list(range(200, 200 + rb_free)), seed + 2)
    a = random_complex(1 << len(la), 1.0, seed + 3)
    b = random_complex(1 << len(lb), 1.0, seed + 4)
    return a, la, b, lb, lc


@pytest.mark.parametrize("shape", [(2, 3, 2), (0, 3, 2), (3, 0, 2), (2, 4, 0), (0, 5, 0), (1, 1, 1), (3, 2, 3)])
def test_einsum_matches_loops(shape):
    a, la, b, lb, lc = _case(*shape, seed=sum(shape) * 10 + shape[0])
    ref = pw.contract_loops(a, la, b, lb, lc)
    got = pw.contract(a, la, b, lb, lc)
    assert np.allclose(got, ref, atol=1e-13)
    idx = list(range(0, 1 << len(lc), max(1, (1 << len(lc)) // 5)))
    assert np.allclose(pw.contract_at(a, la, b, lb, lc, idx), ref[idx], atol=1e-13)


def test_textbook_gemm_layout():
    # A has labels [k0..k2 (low bits), m0..m1], B [n0..n1, k0..k2], C [n0.., m0..]:
    # as matrices A[m, k] = a[k + 8 m], B[k, n] = b[n + 4 k], C[m, n] = c[n + 4 m].
    m_l, k_l, n_l = [0, 1], [10, 11, 12], [20, 21]
    a = np.arange(32) * (1 + 0.5j)
    b = np.arange(32)[::-1] * (0.25 - 1j)
    c = pw.contract(a, k_l + m_l, b, n_l + k_l, n_l + m_l)
    am = a.reshape(4, 8)
    bm = b.reshape(8, 4)
    cm = np.zeros((4, 4), dtype=complex)
    for i in range(4):
        for j in range(4):
            for k in range(8):
                cm[i, j] += am[i, k] * bm[k, j]
    assert np.allclose(c.reshape(4, 4), cm)
