"""The allocation-free contraction entry point (tnc_contract_noalloc).

It exists for callers that cannot allocate device memory -- for instance code running
while a stream is captured into a CUDA graph, or an application whose own pool already
holds the device's memory -- and keeps its scratch in a fixed 4 MiB device array instead.
This test calls it through the C boundary on split-over-K and generic shapes and checks,
on two calls in a row (the array keeps the previous call's contents), that it returns
what tnc_contract returns for the same inputs, within the tolerances of the other
contraction tests.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from inputs import random_complex, random_labels_perm
from oracle import metrics
from paper_2504_09186_gb300 import tnc as T

pytestmark = pytest.mark.gpu

DT = {"c64": torch.float32, "chalf": torch.float16}
TOL = {"c64": 1e-5, "chalf": 2e-3}


def _case(m, k, n, seed):
    la = random_labels_perm(list(range(m)) + list(range(100, 100 + k)), seed)
    lb = random_labels_perm(list(range(100, 100 + k)) + list(range(200, 200 + n)), seed + 1)
    lc = random_labels_perm(list(range(m)) + list(range(200, 200 + n)), seed + 2)
    sigma = 2.0 ** (-k / 2.0)
    a = random_complex(1 << len(la), sigma, seed + 3)
    b = random_complex(1 << len(lb), sigma, seed + 4)
    return a, la, b, lb, lc


def _planar(x, dtype):
    return torch.from_numpy(np.concatenate([x.real, x.imag])).to(dtype).cuda()


def _value(t, e, rank):
    v = t.to(torch.float64).cpu().numpy()
    n = 1 << rank
    return (v[:n] + 1j * v[n:]) * 2.0 ** e


@pytest.mark.parametrize("precision,shape", [("c64", (2, 14, 2)), ("chalf", (3, 12, 2)), ("c64", (6, 5, 6))])
def test_noalloc_matches_contract_on_two_calls(precision, shape):
    torch.cuda.set_device(0)
    ctx = T.Context(0)
    a, la, b, lb, lc = _case(*shape, seed=97 + sum(shape))
    ta, tb = _planar(a, DT[precision]), _planar(b, DT[precision])
    ref_t = torch.empty(2 << len(lc), dtype=DT[precision], device="cuda")
    e_ref = ctx.contract(precision, ta, la, tb, lb, ref_t, lc)
    torch.cuda.synchronize()
    ref = _value(ref_t, e_ref, len(lc))
    for _ in range(2):
        out = torch.full((2 << len(lc),), float("nan"), dtype=DT[precision], device="cuda")
        e = T.tnc_contract_noalloc(precision, ta, la, tb, lb, out, lc)
        torch.cuda.synchronize()
        got = _value(out, e, len(lc))
        assert np.all(np.isfinite(got))
        assert metrics.rel_err_norm(got, ref) <= TOL[precision]
