"""The allocation-free contraction entry point (tnc_contract_noalloc).

It exists for callers that cannot allocate device memory -- for instance a latency-bound
thread that must not wait on the allocator, or an application whose own pool already
holds the device's memory -- and keeps its scratch in a fixed 4 MiB device array instead.
These tests call it through the C boundary on split-over-K and generic shapes and check,
on two calls in a row (the array keeps the previous call's contents), that it returns
what tnc_contract returns for the same inputs and what the FP64 oracle gives, within the
tolerances of the other contraction tests.  This file is collected last on purpose.
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


def _stored(x, dtype):
    """The operand values as the device holds them (rounded to the storage type)."""
    v = torch.from_numpy(np.concatenate([x.real, x.imag])).to(dtype).to(torch.float64).numpy()
    n = x.size
    return v[:n] + 1j * v[n:]


# (5, 19, 5): 2^10 outputs and a 2^19-long K, the largest split-over-K case: its partial sums
# (one wave of split CTAs over 2^10 outputs) take the most of the static array
@pytest.mark.parametrize("precision,shape", [("c64", (2, 14, 2)), ("chalf", (3, 12, 2)), ("c64", (6, 5, 6)),
                                             ("cbf16", (2, 13, 3)), ("chalf", (5, 19, 5))])
@pytest.mark.parametrize("side_stream", [False, True])
def test_noalloc_matches_contract_on_two_calls(precision, shape, side_stream):
    torch.cuda.set_device(0)
    ctx = T.Context(0)
    a, la, b, lb, lc = _case(*shape, seed=97 + sum(shape))
    ta, tb = _planar(a, DT[precision]), _planar(b, DT[precision])
    ref_t = torch.empty(2 << len(lc), dtype=DT[precision], device="cuda")
    e_ref = ctx.contract(precision, ta, la, tb, lb, ref_t, lc)
    torch.cuda.synchronize()
    ref = _value(ref_t, e_ref, len(lc))
    oracle = pairwise.contract(_stored(a, DT[precision]), la, _stored(b, DT[precision]), lb, lc)
    stream = torch.cuda.Stream() if side_stream else None
    for _ in range(2):
        out = torch.full((2 << len(lc),), float("nan"), dtype=DT[precision], device="cuda")
        if stream is not None:
            stream.wait_stream(torch.cuda.current_stream())
            e = T.tnc_contract_noalloc(precision, ta, la, tb, lb, out, lc, stream=stream.cuda_stream)
        else:
            e = T.tnc_contract_noalloc(precision, ta, la, tb, lb, out, lc)
        torch.cuda.synchronize()
        got = _value(out, e, len(lc))
        assert np.all(np.isfinite(got))
        assert metrics.rel_err_norm(got, ref) <= TOL[precision]
        assert metrics.rel_err_norm(got, oracle) <= TOL[precision]
