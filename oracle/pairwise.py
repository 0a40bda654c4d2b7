"""A single pairwise contraction of binary-index tensors, in FP64.

Sec. II-A: the contraction of two tensors is an Einstein summation over their common
indices, organised as an M x K x N matrix product with the common indices along K.
Tensors here are flat complex arrays of 2^rank entries with a label list; label
position p is bit p of the flat index (position 0 least significant), which is the
storage convention of the GPU library's tensors as well.

Three evaluations, from the plain definition:
  * `contract`   -- numpy einsum over the (2,)*rank views (library primitive);
  * `contract_loops` -- explicit loops over every output and common assignment (tiny sizes);
  * `contract_at` -- chosen output entries one at a time (any size: the sums run over K).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def _view(flat: np.ndarray, rank: int) -> np.ndarray:
    """(2,)*rank view whose axis p is label position p (bit p of the flat index)."""
    # numpy's C order makes axis 0 the most significant bit; reverse the axes
    return np.asarray(flat).reshape((2,) * rank).transpose(list(range(rank - 1, -1, -1))) if rank else np.asarray(flat).reshape(())


def split_labels(la: Sequence[int], lb: Sequence[int]):
    sa, sb = set(la), set(lb)
    common = [x for x in la if x in sb]
    free_a = [x for x in la if x not in sb]
    free_b = [x for x in lb if x not in sa]
    return free_a, common, free_b


def contract(a: np.ndarray, la: Sequence[int], b: np.ndarray, lb: Sequence[int], lc: Sequence[int]) -> np.ndarray:
    """C[lc] = sum over common labels of A[la] * B[lb]; returns C flat (bit p = lc[p])."""
    free_a, common, free_b = split_labels(la, lb)
    assert sorted(lc) == sorted(free_a + free_b), "output labels must be the free labels"
    letters = {}
    for x in list(la) + list(lb):
        if x not in letters:
            letters[x] = chr(ord("a") + len(letters)) if len(letters) < 26 else chr(ord("A") + len(letters) - 26)
    sa = "".join(letters[x] for x in la)
    sb = "".join(letters[x] for x in lb)
    sc = "".join(letters[x] for x in lc)
    va = _view(np.asarray(a, dtype=np.complex128), len(la))
    vb = _view(np.asarray(b, dtype=np.complex128), len(lb))
    vc = np.einsum(f"{sa},{sb}->{sc}", va, vb)
    # back to flat with bit p = lc[p]: axis p must become the (rank-1-p)-th numpy axis
    r = len(lc)
    return np.ascontiguousarray(vc.transpose(list(range(r - 1, -1, -1)))).reshape(-1) if r else vc.reshape(1)


def _addr(assign: dict, labels: Sequence[int]) -> int:
    return sum(assign[x] << p for p, x in enumerate(labels))


def contract_loops(a, la, b, lb, lc) -> np.ndarray:
    """The same contraction by explicit Python loops (use only for a few thousand terms)."""
    free_a, common, free_b = split_labels(la, lb)
    out = np.zeros(1 << len(lc), dtype=np.complex128)
    for c_idx in range(1 << len(lc)):
        assign = {x: (c_idx >> p) & 1 for p, x in enumerate(lc)}
        acc = 0.0 + 0.0j
        for k_idx in range(1 << len(common)):
            for p, x in enumerate(common):
                assign[x] = (k_idx >> p) & 1
            acc += complex(a[_addr(assign, la)]) * complex(b[_addr(assign, lb)])
        out[c_idx] = acc
    return out


def contract_at(a, la, b, lb, lc, c_indices: Sequence[int]) -> np.ndarray:
    """Selected output entries C[c] (flat indices in the lc layout), each as one dot
    product over all common assignments (numpy fancy indexing + a sum)."""
    free_a, common, free_b = split_labels(la, lb)
    kk = np.arange(1 << len(common), dtype=np.int64)
    # address contributions of the common labels in A and B
    ka = np.zeros_like(kk)
    kb = np.zeros_like(kk)
    for p, x in enumerate(common):
        bit = (kk >> p) & 1
        ka += bit << la.index(x)
        kb += bit << lb.index(x)
    out = np.empty(len(c_indices), dtype=np.complex128)
    a = np.asarray(a)
    b = np.asarray(b)
    for t, c in enumerate(c_indices):
        base_a = 0
        base_b = 0
        for p, x in enumerate(lc):
            bit = (int(c) >> p) & 1
            if x in free_a:
                base_a += bit << la.index(x)
            else:
                base_b += bit << lb.index(x)
        out[t] = np.sum(a[base_a + ka].astype(np.complex128) * b[base_b + kb].astype(np.complex128))
    return out
