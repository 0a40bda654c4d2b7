"""GPU parity of the tensor-core (tcgen05) complex GEMM step against the FP64 oracle.

Single contractions go through tnc_contract with operand layouts that qualify for the
tensor-core kernel (the same three common labels at positions 0..2 of A and B, M and N
>= 2^7, K >= 2^6); whole plans go through tnc_amplitudes.  Same tolerances as the SIMT
kernel: fp16 storage 2e-3, bf16 1e-2 (one rounding of the output; FP32 accumulation).
"""
import numpy as np
import pytest
import torch

from inputs import grid_circuit, random_complex, random_labels_perm, subcube_bitstrings, subcube_spec
from oracle import metrics, pairwise
from oracle import statevector as sv
from paper_2504_09186_gb300 import tnc as T

pytestmark = pytest.mark.gpu

DT = {"chalf": torch.float16, "cbf16": torch.bfloat16}
TOL = {"chalf": 2e-3, "cbf16": 1e-2}


@pytest.fixture(scope="module")
def ctx():
    return T.Context(0)


def kmajor_case(m, k, n, seed):
    ks = list(range(100, 100 + k))
    la = ks[:3] + random_labels_perm(list(range(m)) + ks[3:], seed)
    lb = ks[:3] + random_labels_perm(ks[3:] + list(range(200, 200 + n)), seed + 1)
    lc = random_labels_perm(list(range(m)) + list(range(200, 200 + n)), seed + 2)
    sigma = 1.0 / np.sqrt(2.0 ** k)
    a = random_complex(1 << len(la), sigma, seed + 3)
    b = random_complex(1 << len(lb), sigma, seed + 4)
    return a, la, b, lb, lc


def tma_case(m, k, n, seed, direct=False):
    """Layouts the TMA kernel loads directly: A = [Kt | 7 row labels | rest], B = [Kt | 5-8
    column labels | rest], C's three lowest labels among the tile labels (direct: the first
    three tile columns in order, so the epilogue stores from registers without staging)."""
    kt = 5 if k >= 5 else 4
    nt = 8 if (n >= 8 and k > kt + 3) else (7 if n >= 7 else (6 if n >= 6 else 5))
    ks = list(range(100, 100 + k))
    ms = list(range(m))
    ns = list(range(200, 200 + n))
    la = ks[:kt] + ms[:7] + random_labels_perm(ms[7:] + ks[kt:], seed)
    lb = ks[:kt] + ns[:nt] + random_labels_perm(ns[nt:] + ks[kt:], seed + 1)
    if direct:
        lc = ns[:3] + ms[:5] + random_labels_perm(ms[5:] + ns[3:], seed + 2)
    else:
        lc = [ns[0], ms[0], ns[1]] + random_labels_perm(ms[1:] + ns[2:], seed + 2)
    sigma = 1.0 / np.sqrt(2.0 ** k)
    a = random_complex(1 << len(la), sigma, seed + 3)
    b = random_complex(1 << len(lb), sigma, seed + 4)
    return a, la, b, lb, lc


def run(ctx, precision, a, la, b, lb, lc):
    def planar(x):
        t = torch.from_numpy(np.concatenate([x.real, x.imag])).to(DT[precision])
        back = t.to(torch.float64).numpy()
        return t.cuda(), back[: x.size] + 1j * back[x.size:]

    ta, aq = planar(a)
    tb, bq = planar(b)
    tc = torch.empty(2 << len(lc), dtype=DT[precision], device="cuda")
    e = ctx.contract(precision, ta, la, tb, lb, tc, lc)
    torch.cuda.synchronize()
    cc = tc.to(torch.float64).cpu().numpy()
    n = 1 << len(lc)
    return (cc[:n] + 1j * cc[n:]) * 2.0 ** e, aq, bq


# (m, k, n): 128/64-wide N tiles, 64/32/16-wide K tiles, role swap (m < n), split over K
SHAPES = [(7, 6, 7), (8, 8, 8), (9, 10, 7), (7, 12, 9), (10, 7, 8), (8, 15, 6), (9, 4, 8), (8, 5, 9),
          (6, 8, 9), (7, 4, 10), (7, 14, 6)]


@pytest.mark.parametrize("precision", ["chalf", "cbf16"])
@pytest.mark.parametrize("shape", SHAPES)
def test_tc_contract_elementwise(ctx, precision, shape):
    a, la, b, lb, lc = kmajor_case(*shape, seed=11 * sum(shape) + shape[0])
    got, aq, bq = run(ctx, precision, a, la, b, lb, lc)
    if len(got) <= 1 << 16:
        ref = pairwise.contract(aq, la, bq, lb, lc)
        err = metrics.rel_err_norm(got, ref)
    else:
        idx = np.random.default_rng(1).integers(0, len(got), 256)
        err = metrics.rel_err_norm(got[idx], pairwise.contract_at(aq, la, bq, lb, lc, idx))
    assert err <= TOL[precision], err


# the last four: N = 2^5, 32-wide tiles (16-column TMEM loads in the epilogue), split and not
TMA_SHAPES = [(7, 4, 6), (7, 5, 7), (8, 9, 8), (9, 12, 7), (10, 4, 9), (8, 15, 6), (7, 14, 7), (7, 6, 8), (9, 8, 10),
              (9, 8, 5), (8, 13, 5), (7, 4, 5), (12, 10, 5)]


@pytest.mark.parametrize("precision", ["chalf", "cbf16"])
@pytest.mark.parametrize("shape", TMA_SHAPES)
def test_tma_contract(ctx, precision, shape):
    a, la, b, lb, lc = tma_case(*shape, seed=13 * sum(shape) + shape[2], direct=shape[0] % 2 == 1)
    got, aq, bq = run(ctx, precision, a, la, b, lb, lc)
    assert int(ctx.profile_read(cap=1)["kind"][0]) in (4, 5)  # a TMA tensor-core kernel ran
    if len(got) <= 1 << 16:
        err = metrics.rel_err_norm(got, pairwise.contract(aq, la, bq, lb, lc))
    else:
        idx = np.random.default_rng(3).integers(0, len(got), 256)
        err = metrics.rel_err_norm(got[idx], pairwise.contract_at(aq, la, bq, lb, lc, idx))
    assert err <= TOL[precision], err


def test_tma_large_sampled(ctx):
    a, la, b, lb, lc = tma_case(14, 12, 10, seed=6)
    got, aq, bq = run(ctx, "chalf", a, la, b, lb, lc)
    idx = np.unique(np.concatenate([[0, len(got) - 1], np.random.default_rng(4).integers(0, len(got), 126)]))
    assert metrics.rel_err_norm(got[idx], pairwise.contract_at(aq, la, bq, lb, lc, idx)) <= TOL["chalf"]


def test_tc_contract_large_sampled(ctx):
    # the shape of the largest step of the 30-qubit plan, at one slice: M=2^14, K=2^12, N=2^10
    a, la, b, lb, lc = kmajor_case(14, 12, 10, seed=5)
    got, aq, bq = run(ctx, "chalf", a, la, b, lb, lc)
    idx = np.unique(np.concatenate([[0, len(got) - 1], np.random.default_rng(2).integers(0, len(got), 126)]))
    ref = pairwise.contract_at(aq, la, bq, lb, lc, idx)
    assert metrics.rel_err_norm(got[idx], ref) <= TOL["chalf"]


@pytest.mark.parametrize("precision", ["chalf", "cbf16"])
def test_tc_steps_inside_a_plan(ctx, precision):
    # 20-qubit 4x5 grid, 12 cycles: its plan has tensor-core steps
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(20, 6, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=16, log2_cap=20)
    assert sum(s["tc"] for s in p.describe()["steps"]) >= 1
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    got = ctx.amplitudes(p, fixed[None, :], precision)[0]
    info = p.info()
    tol = 1e-2 if precision == "chalf" else 4 * 2.0 ** -9 * np.sqrt(info["n_leaves"] + info["n_steps"])
    assert metrics.rel_err_norm(got, ref) <= tol


# Short K loops over >= 4 x 152 output tiles take the persistent TMA kernel (two TMEM
# accumulators, epilogue overlapped with the next tile): BN = 128 with 16- and 32-wide K
# tiles, BN = 64; one to eight K tiles per output tile.
PERSIST_SHAPES = [(12, 4, 12), (14, 5, 10), (12, 6, 12), (17, 7, 7), (16, 8, 8), (17, 4, 6)]


@pytest.mark.parametrize("direct", [False, True])
@pytest.mark.parametrize("precision", ["chalf", "cbf16"])
@pytest.mark.parametrize("shape", PERSIST_SHAPES)
def test_tma_persistent_kernel(ctx, precision, shape, direct, monkeypatch):
    # direct: C's lowest labels are the first tile columns, so both kernels store from
    # registers; otherwise through the staging buffer
    a, la, b, lb, lc = tma_case(*shape, seed=7 * sum(shape) + shape[0], direct=direct)
    got, aq, bq = run(ctx, precision, a, la, b, lb, lc)
    assert int(ctx.profile_read(cap=1)["kind"][0]) == 5  # the persistent kernel ran
    # sampled outputs against the oracle, first and last entries included
    idx = np.unique(np.concatenate([[0, len(got) - 1], np.random.default_rng(5).integers(0, len(got), 510)]))
    assert metrics.rel_err_norm(got[idx], pairwise.contract_at(aq, la, bq, lb, lc, idx)) <= TOL[precision]
    # every tile against the one-CTA-per-tile kernel: same MMAs in the same order, same epilogue
    monkeypatch.setenv("TNC_NO_PERSIST", "1")
    ctx1 = T.Context(0)
    ref, _, _ = run(ctx1, precision, a, la, b, lb, lc)
    assert int(ctx1.profile_read(cap=1)["kind"][0]) == 4
    assert np.array_equal(got, ref)


# 256-wide tiles with the direct epilogue over >= 2 x 152 output tiles take the persistent
# kernel with one TMEM buffer: it drains the accumulators (half stored at once, half held in
# registers), hands TMEM back and stores while the next tile's MMAs run.  2^4 .. 2^7 K tiles
# of 32 per output tile; one to sixteen tiles across N.
WIDE_SHAPES = [(14, 12, 10), (13, 9, 11), (15, 9, 9), (12, 10, 12), (16, 9, 8)]


@pytest.mark.parametrize("precision", ["chalf", "cbf16"])
@pytest.mark.parametrize("shape", WIDE_SHAPES)
def test_tma_persistent_wide_kernel(ctx, precision, shape, monkeypatch):
    a, la, b, lb, lc = tma_case(*shape, seed=5 * sum(shape) + shape[1], direct=True)
    got, aq, bq = run(ctx, precision, a, la, b, lb, lc)
    assert int(ctx.profile_read(cap=1)["kind"][0]) == 5  # the persistent kernel ran
    idx = np.unique(np.concatenate([[0, len(got) - 1], np.random.default_rng(8).integers(0, len(got), 510)]))
    assert metrics.rel_err_norm(got[idx], pairwise.contract_at(aq, la, bq, lb, lc, idx)) <= TOL[precision]
    # every tile bit for bit against the one-CTA-per-tile kernel
    monkeypatch.setenv("TNC_NO_PERSIST", "1")
    ctx1 = T.Context(0)
    ref, _, _ = run(ctx1, precision, a, la, b, lb, lc)
    assert int(ctx1.profile_read(cap=1)["kind"][0]) == 4
    assert np.array_equal(got, ref)


# Layouts the tensor-core kernels cannot load in place (a free label at the lowest position
# of each operand): TTGT -- permute into the tensor-core layouts, contract, permute back.
TTGT_SHAPES = [(8, 6, 7), (9, 8, 8), (10, 5, 6), (7, 10, 9), (12, 4, 12)]


def ttgt_case(m, k, n, seed):
    ms, ks, ns = list(range(m)), list(range(100, 100 + k)), list(range(200, 200 + n))
    la = [ms[0]] + random_labels_perm(ms[1:] + ks, seed)
    lb = [ns[0]] + random_labels_perm(ks + ns[1:], seed + 1)
    lc = random_labels_perm(ms + ns, seed + 2)
    sigma = 1.0 / np.sqrt(2.0 ** k)
    return random_complex(1 << len(la), sigma, seed + 3), la, random_complex(1 << len(lb), sigma, seed + 4), lb, lc


@pytest.mark.parametrize("precision", ["chalf", "cbf16"])
@pytest.mark.parametrize("shape", TTGT_SHAPES)
def test_ttgt_random_layouts(ctx, precision, shape):
    a, la, b, lb, lc = ttgt_case(*shape, seed=11 * sum(shape) + shape[1])
    got, aq, bq = run(ctx, precision, a, la, b, lb, lc)
    assert int(ctx.profile_read(cap=1)["kind"][0]) == 6  # permute, tensor-core GEMM, permute
    if len(got) <= 1 << 16:
        err = metrics.rel_err_norm(got, pairwise.contract(aq, la, bq, lb, lc))
    else:
        idx = np.unique(np.concatenate([[0, len(got) - 1], np.random.default_rng(9).integers(0, len(got), 510)]))
        err = metrics.rel_err_norm(got[idx], pairwise.contract_at(aq, la, bq, lb, lc, idx))
    assert err <= TOL[precision], err


# Every output entry of the persistent kernels at the dominant step shape of the 30-qubit
# plan (M = 2^14, K = 2^12, N = 2^10, one instance) against the FP64 oracle, element by
# element.  Bound per entry: the output is rounded once to the storage type (unit roundoff
# u = 2^-11 fp16, 2^-8 bf16 per real component, so at most 2u |c| for the complex entry),
# plus the FP32 accumulation over K = 2^12 products, whose typical size is
# 2^-24 sqrt(K) rms(C) = 2^-18 rms(C); 1e-4 rms(C) leaves a wide margin for it.
FULL_CASES = [((14, 12, 10), True), ((14, 5, 10), True), ((14, 5, 10), False)]
UNIT = {"chalf": 2.0 ** -11, "cbf16": 2.0 ** -8}


@pytest.mark.parametrize("precision", ["chalf", "cbf16"])
@pytest.mark.parametrize("shape,direct", FULL_CASES)
def test_persistent_kernels_every_output_against_oracle(ctx, precision, shape, direct):
    a, la, b, lb, lc = tma_case(*shape, seed=3 * sum(shape) + int(direct), direct=direct)
    got, aq, bq = run(ctx, precision, a, la, b, lb, lc)
    assert int(ctx.profile_read(cap=1)["kind"][0]) == 5  # a persistent kernel ran
    ref = pairwise.contract(aq, la, bq, lb, lc)
    assert len(ref) == 1 << (shape[0] + shape[2])
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    bound = 2 * UNIT[precision] * np.abs(ref) + 1e-4 * rms
    bad = np.flatnonzero(np.abs(got - ref) > bound)
    assert bad.size == 0, (bad[:8], got[bad[:8]], ref[bad[:8]])
    assert metrics.rel_err_norm(got, ref) <= TOL[precision]


# complex64 on the tensor cores (3xTF32): every FP32 operand entry is split into a TF32 high
# part and a TF32 low part, and each real product is summed from three TF32 products.  Per
# product the dropped low x low term and the rounding of the low parts are each about
# 2^-22 |a b|; with FP32 accumulation the output error stays near FP32's own.  Bars: the
# complex64 norm-wise 1e-5, and per entry 2^-16 |c| + 2^-16 rms(C) (the largest of the
# K = 2^4..2^15 coherent sums of 2^-21 |a||b| stays below 2^-21 sqrt(K) rms(C) <= 2^-13.5
# rms(C) only in the worst case; random signs keep it near 2^-21 rms(C)).
C64_SHAPES = [(7, 4, 6), (7, 5, 7), (8, 9, 8), (9, 12, 7), (10, 4, 9), (7, 14, 7), (9, 8, 5), (7, 4, 5),
              (12, 10, 5), (9, 8, 10), (8, 15, 6)]


@pytest.mark.parametrize("shape", C64_SHAPES)
def test_tma_contract_complex64_tf32(ctx, shape):
    a, la, b, lb, lc = tma_case(*shape, seed=17 * sum(shape) + shape[1], direct=shape[2] % 2 == 0)
    ta = torch.from_numpy(np.concatenate([a.real, a.imag])).to(torch.float32).cuda()
    tb = torch.from_numpy(np.concatenate([b.real, b.imag])).to(torch.float32).cuda()
    aq = ta.cpu().double().numpy()
    bq = tb.cpu().double().numpy()
    aq = aq[: a.size] + 1j * aq[a.size:]
    bq = bq[: b.size] + 1j * bq[b.size:]
    tc = torch.empty(2 << len(lc), dtype=torch.float32, device="cuda")
    e = ctx.contract("c64", ta, la, tb, lb, tc, lc)
    torch.cuda.synchronize()
    assert int(ctx.profile_read(cap=1)["kind"][0]) == 4  # the TMA tensor-core kernel ran
    cc = tc.double().cpu().numpy()
    n = 1 << len(lc)
    got = (cc[:n] + 1j * cc[n:]) * 2.0 ** e
    if n <= 1 << 18:
        idx = np.arange(n)
        ref = pairwise.contract(aq, la, bq, lb, lc)
    else:
        idx = np.unique(np.concatenate([[0, n - 1], np.random.default_rng(3).integers(0, n, 2046)]))
        ref = pairwise.contract_at(aq, la, bq, lb, lc, idx)
    got = got[idx]
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    assert metrics.rel_err_norm(got, ref) <= 1e-5
    assert np.all(np.abs(got - ref) <= 2.0 ** -16 * (np.abs(ref) + rms))


@pytest.mark.parametrize("no_tc64", [False, True])
def test_complex64_plan_on_tensor_cores(no_tc64, monkeypatch):
    # 20-qubit 4x5 grid, 12 cycles, 6 open qubits: the plan's large steps run on the 3xTF32
    # kernel (or, with TNC_NO_TC64=1, on the SIMT kernels); both meet the complex64 bar
    if no_tc64:
        monkeypatch.setenv("TNC_NO_TC64", "1")
    ctx64 = T.Context(0)
    c = grid_circuit(4, 5, 12, seed=1)
    fixed, open_q = subcube_spec(20, 6, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=16, log2_cap=20)
    ref = sv.circuit_amplitudes(c, subcube_bitstrings(fixed, open_q))
    got = ctx64.amplitudes(p, fixed[None, :], "c64", profile=True)[0]
    kinds = set(int(k) for k in ctx64.profile_read()["kind"])
    assert (4 in kinds) != no_tc64
    assert metrics.rel_err_norm(got, ref) <= 1e-5
