"""CPU tests of the C boundary: exported symbols, argument checks, planner invariants."""
import json
import math
import os
import re

import numpy as np
import pytest

from inputs import grid_circuit, subcube_spec
from paper_2504_09186_gb300 import tnc as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    return T.load_library()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tnc_\w+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert T.version().startswith("tnc-gb300")


def test_invalid_arguments_are_reported(lib):
    arity = np.array([3], dtype=np.int32)
    with pytest.raises(T.TncError) as e:
        T.tnc_circuit_from_gates(2, arity, np.zeros(2, np.int32), np.zeros(32))
    assert e.value.status == T.TNC_E_INVALID_ARG and "arity" in str(e.value)
    with pytest.raises(T.TncError) as e:
        T.tnc_circuit_from_gates(2, np.array([2], np.int32), np.array([1, 1], np.int32), np.zeros(32))
    assert "repeated qubit" in str(e.value)
    with pytest.raises(T.TncError):
        T.tnc_circuit_from_gates(0, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0))
    c = grid_circuit(2, 2, 2, seed=1)
    with pytest.raises(T.TncError) as e:
        T.Plan.greedy(c, trials=0)
    assert e.value.status == T.TNC_E_INVALID_ARG


def _recount(desc):
    """Independent recount of one slice's cost and largest tensor from the JSON plan."""
    tensors = desc["tensors"]
    cost = 0.0
    biggest = max(len(t["labels"]) for t in tensors)
    for a, b in desc["tree"]:
        u = set(tensors[a]["labels"]) | set(tensors[b]["labels"])
        cost += 2.0 ** len(u)
    return cost, biggest


@pytest.mark.parametrize("mode", ["greedy", "stem", "split"])
@pytest.mark.parametrize("rows,cols,cycles,n_open,cap,smin", [(3, 4, 8, 0, 26, 0), (4, 4, 10, 4, 12, 3), (3, 3, 6, 2, 8, 0)])
def test_plan_invariants(rows, cols, cycles, n_open, cap, smin, mode):
    c = grid_circuit(rows, cols, cycles, seed=1)
    n = c.n_qubits
    _, open_q = subcube_spec(n, n_open, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=cap, slices_min=smin, mode=mode)
    info = p.info()
    d = p.describe()
    L = len(d["leaves"])
    # a valid binary tree covering every leaf exactly once, SSA order
    used = set()
    for s, (a, b) in enumerate(d["tree"]):
        assert a < L + s and b < L + s and a != b
        assert a not in used and b not in used
        used |= {a, b}
    assert used == set(range(L + len(d["tree"]) - 1))
    # each leaf is a group of gates, every gate in exactly one leaf
    gates = sorted(g for lf in d["leaves"] for g in lf["gates"])
    assert gates == list(range(len(c.gates)))
    # recount of cost and size
    cost, biggest = _recount(d)
    assert math.isclose(math.log2(cost), info["log2_flops_per_slice"], rel_tol=1e-12)
    assert biggest == info["max_log2_size"] <= cap
    assert info["n_sliced"] >= smin
    # the root carries exactly the open output legs
    root = d["tensors"][d["root"]]["labels"]
    assert len(root) == n_open
    # sliced edges are inner wire segments
    for e in d["sliced"]:
        q, cut, kind, is_open = d["edges"][e]
        assert kind == 0 and not is_open
    assert p.open_qubits() == list(open_q)


def _subtree_leaves(d, node):
    L = len(d["leaves"])
    out, stack = set(), [node]
    while stack:
        x = stack.pop()
        if x < L:
            out.add(x)
        else:
            stack.extend(d["tree"][x - L])
    return out


@pytest.mark.parametrize("rows,cols,cycles,cap", [(4, 6, 12, 16), (4, 5, 10, 12), (3, 6, 8, 10)])
def test_split_plan_slices_a_separator(rows, cols, cycles, cap):
    """mode "split": the root joins two stems, one per side of a qubit bisection.  Every
    index joining the sides is sliced unless the cap left room for it (then the root
    contracts it); indices inside a side are sliced only when that side alone exceeds the
    cap.  Each side's leaves act on its own qubits (the straddling 2-qubit leaves excepted),
    and every intermediate stays within the cap."""
    c = grid_circuit(rows, cols, cycles, seed=1)
    p = T.Plan.greedy(c, seed=3, trials=4, log2_cap=cap, mode="split")
    d, info = p.describe(), p.info()
    L = len(d["leaves"])
    sets = _contraction_sets(d)
    root_a, root_b = d["tree"][-1]
    side = {}
    for s_, r in enumerate((root_a, root_b)):
        for leaf in _subtree_leaves(d, r):
            side[leaf] = s_
    assert len(side) == L
    owners = {}
    for i in range(L):
        for e in sets[i]:
            owners.setdefault(e, []).append(i)
    crossing = {e for e, ow in owners.items() if len(ow) == 2 and side[ow[0]] != side[ow[1]]}
    sliced = set(d["sliced"])
    released = crossing - sliced
    assert released == (sets[root_a] & sets[root_b]) - sliced
    # an index inside a side is sliced only if some intermediate exceeds the cap without it
    for e in sliced - crossing:
        assert max(len(x - (sliced - {e})) for x in sets) > cap
    # the qubits each side acts on apart from straddling leaves are disjoint
    qubits = [set(), set()]
    for i in range(L):
        qubits[side[i]] |= {d["edges"][e][0] for e in sets[i] if e not in crossing}
    assert not (qubits[0] & qubits[1])
    cost, biggest = _recount(d)
    assert math.isclose(math.log2(cost), info["log2_flops_per_slice"], rel_tol=1e-12)
    assert biggest == info["max_log2_size"] <= cap


def test_s60_split_plan_total_is_bounded():
    """The 60-qubit 6 x 10 grid, 24 cycles, one bitstring, cap 2^32: the qubit-split plan
    slices the legs of the fSim gates across the middle column boundary.  Its total cost
    2^s * C (complex multiply-adds of all slices) must stay below 2^105, against 2^136.6 for
    the greedy tree this circuit got before (width 86 unsliced, 93 sliced indices).  Any
    plan under this cap needs at least 28 sliced indices: every balanced separator of the
    network is at least the 60 wires of a time cut."""
    c = grid_circuit(6, 10, 24, seed=1)
    p = T.Plan.greedy(c, open_qubits=[], seed=3, trials=4, log2_cap=32, mode="split", objective="time")
    info = p.info()
    d = p.describe()
    cost, biggest = _recount(d)
    total = math.log2(cost) + info["n_sliced"]
    assert math.isclose(total, info["log2_total_flops"], rel_tol=1e-12)
    assert biggest <= 32
    assert 28 <= info["n_sliced"] <= 66
    assert total <= 105.0


def test_same_seed_same_plan_and_roundtrip(tmp_path):
    c = grid_circuit(4, 4, 10, seed=1)
    _, open_q = subcube_spec(16, 3, seed=2)
    p1 = T.Plan.greedy(c, open_qubits=open_q, seed=5, trials=6, log2_cap=11)
    p2 = T.Plan.greedy(c, open_qubits=open_q, seed=5, trials=6, log2_cap=11)
    assert p1.describe() == p2.describe()
    path = str(tmp_path / "plan.bin")
    p1.save(path)
    p3 = T.Plan.load(path)
    d1, d3 = p1.describe(), p3.describe()
    assert d1["tree"] == d3["tree"] and d1["sliced"] == d3["sliced"] and d1["steps"] == d3["steps"]
    with open(path, "r+b") as f:
        f.seek(20)
        f.write(b"\xff\xff\xff\xff")
    with pytest.raises(T.TncError):
        T.Plan.load(path)


def test_slicing_overhead_is_eq1_product():
    # overhead reported = 2^s * C_sliced / C_unsliced; each sliced index had O(a) >= 1
    c = grid_circuit(4, 4, 10, seed=1)
    p = T.Plan.greedy(c, seed=3, trials=4, log2_cap=10)
    info = p.info()
    assert info["n_sliced"] > 0
    assert info["slicing_overhead"] >= 1.0 - 1e-12
    assert math.isclose(info["log2_total_flops"], info["log2_flops_per_slice"] + info["n_sliced"], rel_tol=1e-12)


def test_stem_plan_is_a_stem_and_fuses():
    # every step of a stem plan absorbs a leaf into the previous result (Sec. II-A stem)
    c = grid_circuit(4, 4, 10, seed=1)
    p = T.Plan.greedy(c, seed=3, trials=4, log2_cap=12, mode="stem")
    d = p.describe()
    L = len(d["leaves"])
    for s, (a, b) in enumerate(d["tree"]):
        assert min(a, b) < L  # one operand is a leaf
        if s > 0:
            assert max(a, b) == L + s - 1  # the other is the previous result
    chains = {}
    for i, st in enumerate(d["steps"]):
        if st["chain"] >= 0:
            chains.setdefault(st["chain"], []).append(i)
    assert chains and all(len(v) >= 2 for v in chains.values())
    assert p.info()["n_fused"] == sum(len(v) for v in chains.values())


def test_plan_objectives_pick_their_own_minimum():
    # same seed and trials: the same candidate trees; each objective keeps its own minimum
    c = grid_circuit(4, 5, 12, seed=1)
    _, open_q = subcube_spec(20, 6, seed=2)
    kw = dict(open_qubits=open_q, seed=4, trials=24, log2_cap=14, slices_min=2)
    pf = T.Plan.greedy(c, objective="flops", **kw).info()
    pt = T.Plan.greedy(c, objective="time", **kw).info()
    assert pt["model_seconds_per_slice"] * 2 ** pt["n_sliced"] <= pf["model_seconds_per_slice"] * 2 ** pf["n_sliced"] * (1 + 1e-12)
    assert pf["log2_total_flops"] <= pt["log2_total_flops"] + 1e-12
    assert pf["model_seconds_per_slice"] > 0


def test_tuning_cache_file_roundtrip_and_rejection(tmp_path):
    """The autotuner's cache file: load merges entries, save writes them back in key order,
    and a malformed file is rejected without changing the cache."""
    T.load_library()
    T.tune_clear()
    assert T.tune_size() == 0
    src = tmp_path / "tune.txt"
    src.write_text("tnc-tune 1\n"
                   "p1.a30.b28.c26.bn256.bk32.om3.on2.ok10.d1.z4096 128 1 1 0\n"
                   "p2.a20.b18.c16.bn128.bk16.om1.on1.ok6.d0.z64 64 0 4 3\n")
    T.tune_load(str(src))
    assert T.tune_size() == 2
    out = tmp_path / "saved.txt"
    T.tune_save(str(out))
    assert out.read_text() == src.read_text()
    for bad in ("tnc-tune 2\n",                                   # unknown version
                "tnc-tune 1\nkey 96 0 1 0\n",                     # tile width not 64/128/256
                "tnc-tune 1\nkey 128 0 3 0\n",                    # split not a power of two
                "tnc-tune 1\nkey 128 2 1 0\n",                    # persistent not 0/1
                "tnc-tune 1\nkey 128 0 1 2\n",                    # unknown pipeline depth
                "tnc-tune 1\nkey 128 0\n"):                       # short line
        f = tmp_path / "bad.txt"
        f.write_text(bad)
        with pytest.raises(T.TncError):
            T.tune_load(str(f))
        assert T.tune_size() == 2
    with pytest.raises(T.TncError):
        T.tune_load(str(tmp_path / "missing.txt"))
    T.tune_clear()
    assert T.tune_size() == 0


def test_tensor_core_layouts_allow_direct_epilogues():
    """The compiler orders a tensor-core step's K tile so that its operands' producers store
    their results straight from registers: positions 0..2 of such a result are the producer's
    first three tile columns and position 3 its first tile row.  On the 30-qubit plan the two
    largest steps and most of the others qualify."""
    c = grid_circuit(5, 6, 14, seed=1)
    fixed, open_q = subcube_spec(30, 10, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=64, log2_cap=26, slices_min=6, slices_max=6)
    d = p.describe()
    ten = d["tensors"]
    tc = [s for s in d["steps"] if s["tc"]]
    assert tc
    direct = []
    for s in tc:
        t = s["tc_tile"]
        la, lb, lc = ten[s["a"]]["labels"], ten[s["b"]]["labels"], ten[s["c"]]["labels"]
        rows, cols = (lb, la) if t["swap"] else (la, lb)
        kt, nt = len(t["Kt"]), {64: 6, 128: 7, 256: 8}[t["bn"]]
        # operands lead with Kt then Mt / Nt (the TMA boxes)
        assert rows[:kt] == t["Kt"] and cols[:kt] == t["Kt"]
        assert rows[kt:kt + 7] == t["Mt"] and cols[kt:kt + nt] == t["Nt"]
        log2_flops = len(set(la) | set(lb))
        direct.append((log2_flops, lc[:3] == t["Nt"][:3] and lc[3] == t["Mt"][0]))
    direct.sort()
    assert direct[-1][1] and direct[-2][1]
    assert sum(dr for _, dr in direct) >= 0.75 * len(direct)


def _contraction_sets(d):
    """Label sets of every tree node with the sliced labels kept: leaves without their closed
    output legs (fixed per bitstring), intermediates as symmetric differences."""
    sets = []
    for lf in d["leaves"]:
        sets.append({e for e in lf["labels"] if not (d["edges"][e][2] == 2 and not d["edges"][e][3])})
    for a, b in d["tree"]:
        sets.append(sets[a] ^ sets[b])
    return sets


@pytest.mark.parametrize("slicing,exchange", [("eq1", False), ("eq1", True), ("reuse", False), ("reuse", True)])
def test_slice_stats_and_executed_cost_recount(slicing, exchange):
    """Lifetimes, dependent steps, Eq. 1 and tree-reuse overheads of every sliced index, and
    the executed cost under tree-like reuse (Sec. III-B), recounted from the plan's tree."""
    c = grid_circuit(4, 4, 10, seed=1)
    _, open_q = subcube_spec(16, 3, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=5, trials=6, log2_cap=10, slices_min=4, slicing=slicing,
                      branch_exchange=exchange)
    d, info, st = p.describe(), p.info(), p.slice_stats()
    sets = _contraction_sets(d)
    L, S = len(d["leaves"]), d["sliced"]
    assert info["max_log2_size"] <= 10 and len(S) >= 4

    def deps(e):
        dep = [e in sets[i] for i in range(L)]
        for a, b in d["tree"]:
            dep.append(dep[a] or dep[b])
        return dep

    def cost(sl):
        return sum(2.0 ** len((sets[a] | sets[b]) - set(sl)) for a, b in d["tree"])

    def reuse_cost(sl):
        dmask = [sum(1 << j for j, e in enumerate(sl) if e in sets[i]) for i in range(L)]
        tot = 0.0
        for a, b in d["tree"]:
            dmask.append(dmask[a] | dmask[b])
            tot += 2.0 ** (len((sets[a] | sets[b]) - set(sl)) + bin(dmask[-1]).count("1"))
        return tot

    assert math.isclose(info["log2_executed_flops"], math.log2(reuse_cost(S)), rel_tol=1e-12)
    for t, e in enumerate(S):
        steps = [k for k, (a, b) in enumerate(d["tree"]) if e in sets[a] or e in sets[b]]
        assert st["first_step"][t] == steps[0] and st["last_step"][t] == steps[-1]
        assert st["dep_steps"][t] == sum(deps(e)[L:])
        rest = [x for x in S if x != e]
        assert math.isclose(st["overhead"][t], 2 * cost(S) / cost(rest), rel_tol=1e-12)
        assert math.isclose(st["reuse_overhead"][t], reuse_cost(S) / reuse_cost(rest), rel_tol=1e-12)
        # post-lifetime steps and the share of the executed cost merging would save
        dep = deps(e)
        post = [k for k in range(len(d["tree"])) if k > steps[-1] and dep[L + k]]
        assert st["post_steps"][t] == len(post)
        dmask = [sum(1 << j for j, x in enumerate(S) if x in sets[i]) for i in range(L)]
        for a, b in d["tree"]:
            dmask.append(dmask[a] | dmask[b])
        saved = sum(0.5 * 2.0 ** (len((sets[a] | sets[b]) - set(S)) + bin(dmask[L + k]).count("1"))
                    for k, (a, b) in enumerate(d["tree"]) if k in post)
        assert math.isclose(st["merge_saving"][t], saved / reuse_cost(S), rel_tol=1e-12, abs_tol=1e-300)


def test_branch_exchange_never_raises_the_slicing_cost():
    """Branch exchange keeps the kept trial's slice set and only takes swaps that lower the
    cost its slicing uses: Eq. 1's per-slice cost, or the executed cost under reuse."""
    c = grid_circuit(5, 6, 14, seed=1)
    fixed, open_q = subcube_spec(30, 10, seed=2)
    kw = dict(open_qubits=open_q, seed=3, trials=16, log2_cap=26, slices_min=6, slices_max=6)
    for slicing, key in (("eq1", "log2_flops_per_slice"), ("reuse", "log2_executed_flops")):
        a = T.Plan.greedy(c, slicing=slicing, **kw)
        b = T.Plan.greedy(c, slicing=slicing, branch_exchange=True, **kw)
        assert a.describe()["sliced"] == b.describe()["sliced"]
        assert b.info()[key] <= a.info()[key] + 1e-12
        assert b.info()["max_log2_size"] <= 26


def test_plan_options_roundtrip_and_bad_values(tmp_path):
    """The slicing and branch-exchange options survive a plan file round trip with the same
    tree, slices, executed cost and statistics; out-of-range values are rejected."""
    c = grid_circuit(4, 4, 10, seed=1)
    _, open_q = subcube_spec(16, 3, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=5, trials=4, log2_cap=10, slices_min=3, slicing="reuse",
                      branch_exchange=True)
    path = str(tmp_path / "plan_v5.bin")
    p.save(path)
    q = T.Plan.load(path)
    dp, dq = p.describe(), q.describe()
    assert dp["tree"] == dq["tree"] and dp["sliced"] == dq["sliced"] and dp["steps"] == dq["steps"]
    assert p.info()["log2_executed_flops"] == q.info()["log2_executed_flops"]
    sp, sq = p.slice_stats(), q.slice_stats()
    assert all(np.array_equal(sp[k], sq[k]) for k in sp)
    for bad in (dict(objective=2), dict(slicing=2), dict(branch_exchange=-1), dict(cluster_chains=2)):
        arity, qubits, mats = c.gate_array()
        ch = T.tnc_circuit_from_gates(c.n_qubits, arity, qubits, mats)
        nh = T.tnc_network_build(ch, np.zeros(c.n_qubits, dtype=np.uint8))
        try:
            with pytest.raises(T.TncError) as e:
                T.tnc_plan_greedy(nh, 1, 2, 12, 0, 64, 0.5, 0, **bad)
            assert e.value.status == T.TNC_E_INVALID_ARG
        finally:
            T.load_library().tnc_network_destroy(nh)
            T.load_library().tnc_circuit_destroy(ch)


def _gates_of(gl):
    """(qubits, matrix) pairs of a GateList (the boundary's packed layout)."""
    out = []
    for g in range(len(gl)):
        a = int(gl.arity[g])
        d = 1 << a
        m = gl.matrices[g, 0:2 * d * d:2] + 1j * gl.matrices[g, 1:2 * d * d:2]
        out.append((tuple(int(q) for q in gl.qubits[g, :a]), m.reshape(d, d)))
    return out


@pytest.mark.parametrize("rows,cols,cycles,mode", [(3, 4, 8, "fixed"), (2, 5, 6, "uniform"), (4, 4, 5, "fixed")])
def test_random_grid_circuit_is_the_papers_family(rows, cols, cycles, mode):
    """tnc_circuit_random_grid: per cycle one of {sqrt X, sqrt Y, sqrt W} on every qubit (never
    the qubit's previous one), then fSim on the A, B, C, D coupler classes in turn -- the same
    gates and couplers as the seeded Python generator's family; fixed fSim(pi/2, pi/6) or
    angles in [0, pi); unitary; deterministic per seed."""
    from inputs.circuits import SINGLE_QUBIT_SET, couplers, fsim

    gl = T.random_grid(rows, cols, cycles, seed=11, fsim_mode=mode)
    n = rows * cols
    assert gl.n_qubits == n
    gates = _gates_of(gl)
    i, prev = 0, [-1] * n
    for k in range(cycles):
        for q in range(n):
            qs, m = gates[i]
            i += 1
            assert qs == (q,)
            idx = [t for t, u in enumerate(SINGLE_QUBIT_SET) if np.allclose(m, u, atol=1e-15)]
            assert len(idx) == 1 and idx[0] != prev[q]
            prev[q] = idx[0]
        for pair in couplers(rows, cols, "ABCD"[k % 4]):
            qs, m = gates[i]
            i += 1
            assert qs == pair
            if mode == "fixed":
                assert np.allclose(m, fsim(np.pi / 2, np.pi / 6), atol=1e-15)
            else:
                theta = np.arctan2(-m[1, 2].imag, m[1, 1].real)
                phi = -np.angle(m[3, 3]) % (2 * np.pi)
                assert 0 <= theta < np.pi and 0 <= phi < np.pi
                assert np.allclose(m, fsim(theta, phi), atol=1e-12)
    assert i == len(gates)
    for _, m in gates:
        assert np.allclose(m.conj().T @ m, np.eye(len(m)), atol=1e-14)
    again = T.random_grid(rows, cols, cycles, seed=11, fsim_mode=mode)
    assert np.array_equal(again.matrices, gl.matrices) and np.array_equal(again.qubits, gl.qubits)
    other = T.random_grid(rows, cols, cycles, seed=12, fsim_mode=mode)
    assert not np.array_equal(other.matrices, gl.matrices)
    # the exported gates rebuild the same circuit through tnc_circuit_from_gates
    arity, qubits, mats = gl.gate_array()
    h = T.tnc_circuit_from_gates(n, arity, qubits, mats)
    try:
        back = T.circuit_export(h)
    finally:
        T.load_library().tnc_circuit_destroy(h)
    assert np.array_equal(back.matrices, gl.matrices) and np.array_equal(back.arity, gl.arity)


def test_random_grid_rejects_bad_arguments():
    for args in ((0, 3, 2), (9, 8, 2), (2, 2, -1)):
        with pytest.raises(T.TncError) as e:
            T.random_grid(*args)
        assert e.value.status == T.TNC_E_INVALID_ARG
    with pytest.raises(KeyError):
        T.random_grid(2, 2, 2, fsim_mode="other")


def _merged_executed_recount(d):
    """Executed complex multiply-adds of all slices of one row under tree-like reuse, with
    and without post-lifetime merging, recounted from the plan description: a tensor depends
    on the sliced indices its leaves hold; with merging, the step whose two operands both
    depend on an index sums its result over it (not at the root step), so later tensors no
    longer depend on it."""
    L = len(d["leaves"])
    sliced = list(d["sliced"])
    bit = {e: t for t, e in enumerate(sliced)}
    dep = [frozenset(bit[e] for e in lf["labels"] if e in bit) for lf in d["leaves"]]
    mdep = list(dep)
    plain = merged = 0.0
    n = len(d["tree"])
    for s_, (a, b) in enumerate(d["tree"]):
        u = len(set(d["tensors"][a]["labels"]) | set(d["tensors"][b]["labels"]))
        full_plain = dep[a] | dep[b]
        plain += 2.0 ** (u + len(full_plain))
        dep.append(full_plain)
        full = mdep[a] | mdep[b]
        merged += 2.0 ** (u + len(full))
        both = (mdep[a] & mdep[b]) if s_ + 1 < n else frozenset()
        mdep.append(full - both)
    return plain, merged


def test_post_lifetime_merging_cost_recount():
    # a 20-qubit plan whose sliced indices die early: merging halves the later steps' runs
    c = grid_circuit(4, 5, 12, seed=1)
    _, open_q = subcube_spec(20, 4, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=12, slices_min=8, slices_max=64)
    info, d = p.info(), p.describe()
    plain, merged = _merged_executed_recount(d)
    assert math.isclose(math.log2(plain), info["log2_executed_flops"], rel_tol=1e-12)
    assert math.isclose(math.log2(merged), info["log2_executed_flops_merged"], rel_tol=1e-12)
    assert merged <= 0.75 * plain
    # the 60-qubit split plan: every separator index lives until the root, nothing to merge
    s60 = T.Plan.greedy(grid_circuit(6, 10, 24, seed=1), open_qubits=[], seed=3, trials=2, log2_cap=32, mode="split")
    i60 = s60.info()
    assert math.isclose(i60["log2_executed_flops_merged"], i60["log2_executed_flops"], rel_tol=1e-12)


@pytest.mark.parametrize("rows,cols,cycles,n_open,cap", [(4, 5, 12, 2, 18), (4, 5, 10, 2, 16), (4, 5, 14, 0, 20)])
def test_gepdot_split_counts(rows, cols, cycles, n_open, cap):
    """Split-K GEPDOT steps (M N <= 2^10 outputs, K >= 2^12): the CTAs of a step fill at most one
    wave of two per SM (152 SMs) over the tiles of all instances a plan's program holds
    (2^min(s, 12)), each CTA keeps at least four outer K steps, and a step is split-K exactly
    when its split count exceeds one."""
    c = grid_circuit(rows, cols, cycles, seed=1)
    _, open_q = subcube_spec(c.n_qubits, n_open, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=cap)
    inst = 2 ** min(p.info()["n_sliced"], 12)
    seen = 0
    for st in p.describe()["steps"]:
        m = len(st["Mt"]) + len(st["Mo"])
        k = len(st["Kt"]) + len(st["Ko"])
        n = len(st["Nt"]) + len(st["No"])
        if st["tc"] or not (m + n <= 10 and k >= 12):
            continue
        seen += 1
        tiles = 2 ** (len(st["Mo"]) + len(st["No"])) * inst
        split = st["splitk"]
        assert split >= 1
        assert split <= max(1, -(-2 * 152 // tiles))
        assert split == 1 or split * 4 <= 2 ** len(st["Ko"])
        assert (st["kind"] == 1) == (split > 1)
    assert seen >= 1
