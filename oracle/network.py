"""The oracle's own tensor network of a circuit and a plain pairwise contraction of it.

Sec. II-A: nodes are tensors, edges are shared indices; contracting two tensors sums
over their common indices and leaves a tensor over the rest; a circuit is contracted
edge by edge until one tensor remains.  Every index has dimension 2 (Sec. III-A).

Network (one tensor per gate, no merging):
  * gate t on qubits Q: a rank-2|Q| tensor with axes [out_q for q in Q] + [in_q for q in Q];
    the wire segment of qubit q after j gates on q carries the label ("w", q, j);
  * |0> on every input segment (q, 0); <x_q| on every closed output segment;
    open output segments stay as free labels of the result.
Slicing (Sec. II-A, Sec. III-A) fixes a label to 0 or 1 in every tensor that carries it.

The contraction order here is the oracle's own: greedy on the increase in size (ties by
tensor id), best of a few trials perturbed by seeded Gumbel noise.  If some intermediate
would exceed 2^cap_log2 elements the oracle fixes extra labels and sums over their
values, which is exact because sum_b |b><b| = I (the same identity that makes slicing
exact).  The order only changes rounding and speed, never the value: the tests contract
the same network in random orders and compare.
"""
from __future__ import annotations

import heapq
import itertools
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

Label = Tuple[str, int, int]


class Tensor:
    __slots__ = ("labels", "data")

    def __init__(self, labels: Sequence[Label], data: np.ndarray):
        self.labels = tuple(labels)
        self.data = np.asarray(data, dtype=np.complex128)
        assert self.data.ndim == len(self.labels), (self.data.shape, self.labels)


def circuit_tensors(circuit, out_bits: Optional[Sequence[int]], open_qubits: Sequence[int] = ()):
    """Tensors of the circuit network and the list of open labels (in `open_qubits` order).

    out_bits[q] gives the closed output bit of qubit q (ignored for open qubits).
    """
    n = circuit.n_qubits
    count = [0] * n
    tensors: List[Tensor] = []
    for g in circuit.gates:
        k = len(g.qubits)
        outs = [("w", q, count[q] + 1) for q in g.qubits]
        ins = [("w", q, count[q]) for q in g.qubits]
        tensors.append(Tensor(outs + ins, np.asarray(g.matrix).reshape((2,) * (2 * k))))
        for q in g.qubits:
            count[q] += 1
    for q in range(n):
        tensors.append(Tensor([("w", q, 0)], np.array([1.0, 0.0])))
    open_set = set(open_qubits)
    for q in range(n):
        if q in open_set:
            continue
        v = np.zeros(2)
        v[int(out_bits[q])] = 1.0
        tensors.append(Tensor([("w", q, count[q])], v))
    open_labels = [("w", q, count[q]) for q in open_qubits]
    return tensors, open_labels


def fix_labels(tensors: List[Tensor], fixed: Dict[Label, int]) -> List[Tensor]:
    """Slice: every tensor carrying a fixed label keeps only that component."""
    out = []
    for t in tensors:
        idx = []
        labels = []
        for lab in t.labels:
            if lab in fixed:
                idx.append(int(fixed[lab]))
            else:
                idx.append(slice(None))
                labels.append(lab)
        out.append(Tensor(labels, t.data[tuple(idx)]))
    return out


def _pair_labels(a: Tuple[Label, ...], b: Tuple[Label, ...], keep: set) -> Tuple[Label, ...]:
    sb = set(b)
    sa = set(a)
    res = [x for x in a if (x not in sb) or (x in keep)]
    res += [x for x in b if (x not in sa)]
    return tuple(res)


def greedy_order(label_sets: List[Tuple[Label, ...]], open_labels: Sequence[Label], rng=None, temperature: float = 0.0):
    """Greedy pairwise order on label sets: repeatedly contract the pair sharing a label
    that minimises size(out) - size(a) - size(b); ties by (smaller id, larger id).  With
    `rng`, the score (sign(s) log2(1+|s|)) is perturbed by -temperature * Gumbel noise.

    Returns (pairs as (i, j) of live ids; new ids appended in order, max log2 size,
    list of (log2 size, labels) of every intermediate).
    """
    keep = set(open_labels)
    live: Dict[int, frozenset] = {i: frozenset(ls) for i, ls in enumerate(label_sets)}
    owners: Dict[Label, set] = {}
    for i, ls in live.items():
        for lab in ls:
            owners.setdefault(lab, set()).add(i)

    def out_of(i, j):
        a, b = live[i], live[j]
        return (a ^ b) | (a & b & keep)

    def score(i, j):
        a, b = live[i], live[j]
        s = 2.0 ** len(out_of(i, j)) - 2.0 ** len(a) - 2.0 ** len(b)
        t = np.sign(s) * np.log2(1.0 + abs(s))
        if rng is not None and temperature > 0:
            t -= temperature * rng.gumbel()
        return (t, min(i, j), max(i, j))

    heap = []
    # candidate pairs in a fixed order, so the seeded noise does not depend on the
    # process's string-hash seed (label sets are frozensets of tuples with strings)
    for i, j in sorted({tuple(sorted(ow)) for ow in owners.values() if len(ow) == 2}):
        heapq.heappush(heap, score(i, j))
    next_id = len(label_sets)
    pairs = []
    inter = []
    max_log = max((len(ls) for ls in label_sets), default=0)
    while len(live) > 1:
        pick = None
        while heap:
            _, i, j = heapq.heappop(heap)
            if i in live and j in live:
                pick = (i, j)
                break
        if pick is None:
            ids = sorted(live, key=lambda t: (len(live[t]), t))
            pick = (min(ids[0], ids[1]), max(ids[0], ids[1]))
        i, j = pick
        out = out_of(i, j)
        for lab in live[i]:
            owners[lab].discard(i)
        for lab in live[j]:
            owners[lab].discard(j)
        del live[i], live[j]
        live[next_id] = out
        nbrs = set()
        for lab in out:
            owners.setdefault(lab, set()).add(next_id)
            nbrs |= owners[lab]
        nbrs.discard(next_id)
        for k in sorted(nbrs):
            heapq.heappush(heap, score(k, next_id))
        pairs.append((i, j))
        inter.append((len(out), tuple(sorted(out))))
        max_log = max(max_log, len(out))
        next_id += 1
    return pairs, max_log, inter


def _tree_sets(label_sets, pairs, open_labels):
    """Union and output label sets of every step of a tree."""
    keep = set(open_labels)
    sets = [frozenset(s) for s in label_sets]
    unions = []
    for i, j in pairs:
        a, b = sets[i], sets[j]
        unions.append(a | b)
        sets.append((a ^ b) | (a & b & keep))
    return sets, unions


def slice_tree(label_sets, pairs, open_labels, cap_log2: int, max_extra: int = 30):
    """Labels to fix on a fixed tree so that no tensor exceeds 2^cap_log2 entries.

    Each round fixes, among the labels of the oversized tensors, the one that leaves the
    smallest cost sum_steps 2^|union - fixed| (ties by label order).  Returns
    (fixed labels, cost of one sub-contraction)."""
    sets, unions = _tree_sets(label_sets, pairs, open_labels)
    keep = set(open_labels)
    fixed: set = set()

    def cost(fx):
        return sum(2.0 ** len(u - fx) for u in unions)

    extra: List[Label] = []
    while len(extra) < max_extra:
        over = [s for s in sets if len(s - fixed) > cap_log2]
        if not over:
            break
        cand = sorted({lab for s in over for lab in s if lab not in fixed and lab not in keep})
        if not cand:
            break
        best = min(cand, key=lambda lab: (cost(fixed | {lab}), lab))
        fixed.add(best)
        extra.append(best)
    return extra, cost(fixed)


def search_order(label_sets, open_labels, cap_log2: int, trials: int = 8, seed: int = 0, temperature: float = 1.0):
    """Best of `trials` greedy orders (trial 0 unperturbed), each sliced to the cap on its
    tree; minimises 2^extra * cost.  Returns (pairs, extra labels)."""
    rng = np.random.default_rng(seed)
    best = None
    for t in range(trials):
        pairs, _, _ = greedy_order(label_sets, open_labels, rng if t else None, temperature)
        extra, c = slice_tree(label_sets, pairs, open_labels, cap_log2)
        total = (2.0 ** len(extra)) * c
        if best is None or total < best[0]:
            best = (total, pairs, extra)
    return best[1], best[2]


def contract_pair(a: Tensor, b: Tensor, keep: set) -> Tensor:
    """One pairwise contraction: sum over common labels not in `keep` (np.tensordot)."""
    common = [x for x in a.labels if x in set(b.labels) and x not in keep]
    if any(x in keep for x in a.labels if x in set(b.labels)):
        raise ValueError("an open label is shared by two tensors")
    ax_a = [a.labels.index(x) for x in common]
    ax_b = [b.labels.index(x) for x in common]
    data = np.tensordot(a.data, b.data, axes=(ax_a, ax_b))
    labels = [x for x in a.labels if x not in common] + [x for x in b.labels if x not in common]
    return Tensor(labels, data)


def contract_network(tensors: List[Tensor], open_labels: Sequence[Label], order=None) -> np.ndarray:
    """Contract all tensors (in `order` or the greedy order) to the open labels, in order."""
    if order is None:
        order, _, _ = greedy_order([t.labels for t in tensors], open_labels)
    keep = set(open_labels)
    live: Dict[int, Tensor] = dict(enumerate(tensors))
    next_id = len(tensors)
    for i, j in order:
        live[next_id] = contract_pair(live.pop(i), live.pop(j), keep)
        next_id += 1
    (res,) = live.values()
    perm = [res.labels.index(x) for x in open_labels]
    return np.transpose(res.data, perm) if perm else res.data.reshape(())


def choose_subslices(label_sets, open_labels, cap_log2: int, max_extra: int = 30):
    """Labels to fix (beyond the given slices) so that the plain greedy order stays under
    the cap; returns (labels, max log2 size without them)."""
    pairs, max_log, _ = greedy_order([tuple(ls) for ls in label_sets], open_labels)
    extra, _ = slice_tree(label_sets, pairs, open_labels, cap_log2, max_extra)
    return extra, max_log


def network_amplitudes(
    circuit,
    out_bits: Optional[Sequence[int]],
    open_qubits: Sequence[int] = (),
    cuts: Optional[Dict[Tuple[int, int], int]] = None,
    cap_log2: int = 24,
    trials: int = 8,
) -> np.ndarray:
    """Amplitudes over the open qubits (sub-cube order: first open qubit most significant).

    `cuts` {(q, j): bit} slices the wire of qubit q after j gates.  Returns an array of
    shape (2,)*len(open_qubits) (a 0-d array when every output is closed).
    """
    tensors, open_labels = circuit_tensors(circuit, out_bits, open_qubits)
    fixed = {("w", q, j): b for (q, j), b in (cuts or {}).items()}
    tensors = fix_labels(tensors, fixed)
    order, extra = search_order([t.labels for t in tensors], open_labels, cap_log2, trials=trials)
    total = None
    for bits in itertools.product((0, 1), repeat=len(extra)):
        # fixing labels keeps every tensor, so the tree stays valid
        sub = fix_labels(tensors, dict(zip(extra, bits)))
        val = contract_network(sub, open_labels, order)
        total = val if total is None else total + val
    return total


def batch_amplitudes(circuit, bitstrings: np.ndarray, cuts=None, cap_log2: int = 24) -> np.ndarray:
    """amp(x) for each closed bitstring row, one network contraction per bitstring."""
    return np.array(
        [complex(network_amplitudes(circuit, row, (), cuts, cap_log2)) for row in np.asarray(bitstrings)]
    )
