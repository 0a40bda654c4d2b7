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

The contraction order here is the oracle's own: greedy on the increase in size, with
ties broken by tensor id.  If some intermediate would exceed 2^cap_log2 elements the
oracle fixes extra labels and sums over their values, which is exact because
sum_b |b><b| = I (the same identity that makes slicing exact).
"""
from __future__ import annotations

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


def greedy_order(label_sets: List[Tuple[Label, ...]], open_labels: Sequence[Label]):
    """Greedy pairwise order on label sets: repeatedly contract the pair sharing a label
    that minimises size(out) - size(a) - size(b); ties by (smaller id, larger id).

    Returns (pairs as (i, j) of live ids; new ids appended in order, max log2 size,
    list of (log2 size, labels) of every intermediate).
    """
    keep = set(open_labels)
    live: Dict[int, Tuple[Label, ...]] = {i: ls for i, ls in enumerate(label_sets)}
    by_label: Dict[Label, set] = {}
    for i, ls in live.items():
        for lab in ls:
            by_label.setdefault(lab, set()).add(i)
    next_id = len(label_sets)
    pairs = []
    inter = []
    max_log = max((len(ls) for ls in label_sets), default=0)
    while len(live) > 1:
        best = None
        for lab, owners in by_label.items():
            if len(owners) < 2:
                continue
            for i, j in itertools.combinations(sorted(owners), 2):
                out = _pair_labels(live[i], live[j], keep)
                score = (2.0 ** len(out) - 2.0 ** len(live[i]) - 2.0 ** len(live[j]), i, j)
                if best is None or score < best[0]:
                    best = (score, i, j, out)
        if best is None:
            # no shared labels left: outer products, smallest first
            ids = sorted(live, key=lambda t: (len(live[t]), t))
            i, j = ids[0], ids[1]
            out = _pair_labels(live[i], live[j], keep)
        else:
            _, i, j, out = best
        pairs.append((i, j))
        for lab in live[i]:
            by_label[lab].discard(i)
        for lab in live[j]:
            by_label[lab].discard(j)
        del live[i], live[j]
        live[next_id] = out
        for lab in out:
            by_label.setdefault(lab, set()).add(next_id)
        inter.append((len(out), out))
        max_log = max(max_log, len(out))
        next_id += 1
    return pairs, max_log, inter


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


def choose_subslices(label_sets, open_labels, cap_log2: int, max_extra: int = 24):
    """Labels to fix (beyond the given slices) so that the greedy order stays under the cap.

    Picks, each round, the label occurring in the most intermediates above the cap.
    """
    extra: List[Label] = []
    sets = [tuple(ls) for ls in label_sets]
    while True:
        _, max_log, inter = greedy_order(sets, open_labels)
        if max_log <= cap_log2 or len(extra) >= max_extra:
            return extra, max_log
        votes: Dict[Label, Tuple[int, int]] = {}
        for lg, labs in inter:
            if lg > cap_log2:
                for lab in labs:
                    if lab in open_labels:
                        continue
                    c, m = votes.get(lab, (0, 0))
                    votes[lab] = (c + 1, max(m, lg))
        if not votes:
            return extra, max_log
        pick = max(votes.items(), key=lambda kv: (kv[1][0], kv[1][1], kv[0]))[0]
        extra.append(pick)
        sets = [tuple(x for x in ls if x != pick) for ls in sets]


def network_amplitudes(
    circuit,
    out_bits: Optional[Sequence[int]],
    open_qubits: Sequence[int] = (),
    cuts: Optional[Dict[Tuple[int, int], int]] = None,
    cap_log2: int = 24,
) -> np.ndarray:
    """Amplitudes over the open qubits (sub-cube order: first open qubit most significant).

    `cuts` {(q, j): bit} slices the wire of qubit q after j gates.  Returns an array of
    shape (2,)*len(open_qubits) (a 0-d array when every output is closed).
    """
    tensors, open_labels = circuit_tensors(circuit, out_bits, open_qubits)
    fixed = {("w", q, j): b for (q, j), b in (cuts or {}).items()}
    tensors = fix_labels(tensors, fixed)
    extra, _ = choose_subslices([t.labels for t in tensors], open_labels, cap_log2)
    order = None
    total = None
    for bits in itertools.product((0, 1), repeat=len(extra)):
        sub = fix_labels(tensors, dict(zip(extra, bits)))
        if order is None:
            order, _, _ = greedy_order([t.labels for t in sub], open_labels)
        val = contract_network(sub, open_labels, order)
        total = val if total is None else total + val
    return total


def batch_amplitudes(circuit, bitstrings: np.ndarray, cuts=None, cap_log2: int = 24) -> np.ndarray:
    """amp(x) for each closed bitstring row, one network contraction per bitstring."""
    return np.array(
        [complex(network_amplitudes(circuit, row, (), cuts, cap_log2)) for row in np.asarray(bitstrings)]
    )
