#!/usr/bin/env python
"""Benchmark of the sliced tensor-network contraction path on GB300.

Workload (default): the 30-qubit 5x6 grid random circuit, 14 cycles (seed 1); greedy plan
(seed 3, 64 trials) sliced to 2^6 slices with every intermediate at most 2^26 entries;
a sub-cube batch of 1024 amplitudes (10 open qubits, the other 20 bits seeded).  One
step = all 64 slices of that batch, summed in FP64.  Metric: slices/s of the
complex-half path (fp16 storage, FP32 arithmetic), with the complex64 path beside it,
both with their amplitude error.

Launch: `python bench.py [--steps K --warmup W]`; under torchrun each rank contracts its
own sub-cube batch (independent problems, no collective on the data path: weak scaling).
`--impl reference` times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "s30": dict(rows=5, cols=6, cycles=14, seed=1, n_open=10, subcube_seed=2, plan_seed=3, trials=64, cap=26,
                smin=6, smax=6),
    "t12": dict(rows=3, cols=4, cycles=8, seed=1, n_open=4, subcube_seed=2, plan_seed=3, trials=8, cap=26,
                smin=0, smax=64),
}

PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
FP32_LANES_PER_SM = 128
N_SM = 152


def measured_traffic(kind, flops_launch):
    """DRAM bytes (read + write) of one launch of the dominant kernel, from a committed ncu
    summary of a kernel of the same kind: per-instance bytes of a one-instance capture times the
    launch's instances.  None when no summary matches the kind and the launch's flops, or when
    the kernel's source changed since the capture (its SHA-1 is recorded beside the figures)."""
    import glob
    import hashlib
    import re

    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        txt = open(path).read()

        def get(key):
            m = re.search(rf"^{key}: (\S+)$", txt, re.M)
            return m.group(1) if m else None

        vals = [get(k) for k in ("traffic_kind", "traffic_flops_per_instance", "traffic_dram_bytes_per_instance",
                                 "traffic_kernel_source", "traffic_kernel_source_sha1")]
        if None in vals or int(vals[0]) != kind:
            continue
        src = os.path.join(ROOT, vals[3])
        if not os.path.exists(src) or hashlib.sha1(open(src, "rb").read()).hexdigest() != vals[4]:
            continue
        inst = flops_launch / float(vals[1])
        if abs(inst - round(inst)) > 1e-9 or round(inst) < 1:
            continue
        return float(vals[2]) * round(inst)
    return None


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        d["_source"] = "measured"
        return d
    d = dict(PEAKS_FALLBACK)
    d["_source"] = "fallback"
    return d


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="s30", choices=sorted(WORKLOADS) + ["s60", "d20", "sw"],
                    help="s30 (default) / t12: sliced sub-cube amplitudes; s60: per-slice throughput of the "
                         "60-qubit circuit; d20: adjoint gradients; sw: single-step contraction sweep")
    ap.add_argument("--plan-trials", type=int, default=0, help="planner trials (0: the workload's own)")
    ap.add_argument("--s60-slices", type=int, default=256, help="seeded slice sample of the s60 workload")
    ap.add_argument("--s60-trials", type=int, default=4, help="planner trials (qubit bisections) of the s60 workload")
    ap.add_argument("--s60-c64", type=int, default=2, help="slices of the sample also run alone in complex64")
    ap.add_argument("--s60-sum-c64", type=int, default=256,
                    help="the first slices of the sample summed in complex-half and complex64")
    ap.add_argument("--sw-shapes", default="", help="log2 M,K,N triples 'm,k,n;m,k,n' (default: a fixed set)")
    ap.add_argument("--precision", default="chalf", choices=["chalf", "cbf16", "c64"])
    ap.add_argument("--no-compare", action="store_true", help="skip the complex64 comparison run")
    ap.add_argument("--no-autotune", action="store_true",
                    help="run the heuristic tile configurations (no timing of the tensor-core steps first)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-cap", type=int, default=23, help="log2 size cap of the oracle sample")
    ap.add_argument("--ref-subslices", type=int, default=4, help="oracle sub-slices per reference step")
    ap.add_argument("--plan", default="greedy", choices=["greedy", "stem"],
                    help="greedy: balanced pairwise order; stem: one tensor absorbs leaves (fused chains)")
    ap.add_argument("--no-fuse", action="store_true", help="run stem absorptions as separate kernels")
    ap.add_argument("--cluster-chains", action="store_true",
                    help="stem plan: fused chains of up to 2^15 entries on thread-block clusters")
    return ap.parse_args()


def max_over_ranks(ms, dist):
    """The whole job is as slow as its slowest rank: max of a per-rank time over the ranks
    (NCCL on GPUs, gloo on the host)."""
    if dist is None:
        return ms
    import torch

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(name, rank):
    from inputs import grid_circuit, subcube_spec

    w = WORKLOADS[name]
    circ = grid_circuit(w["rows"], w["cols"], w["cycles"], seed=w["seed"])
    fixed, open_q = subcube_spec(circ.n_qubits, w["n_open"], seed=w["subcube_seed"] + rank)
    return w, circ, fixed, open_q


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def __enter__(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.tmp.name], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            time.sleep(0.5)  # first sample lands before the timed region starts
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.tmp is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.tmp.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(power) if power else None}


# --------------------------------------------------------------------------- oracle sample
def oracle_sample(circ, fixed, open_q, cuts, cap_log2):
    """Prepare a bounded oracle sample: slice 0 of the given slicing (cuts fixed to 0),
    split further by the oracle's own sub-slicing at 2^cap_log2; returns (run, n_sub):
    `run(i)` contracts sub-slice i, and a whole slice is the n_sub sub-slices."""
    from oracle import network as tn

    tensors, open_labels = tn.circuit_tensors(circ, fixed, open_q)
    tensors = tn.fix_labels(tensors, {("w", q, j): 0 for (q, j) in cuts})
    order, extra = tn.search_order([t.labels for t in tensors], open_labels, cap_log2, trials=8)

    def run(i=0):
        sub = tn.fix_labels(tensors, {lab: (i >> t) & 1 for t, lab in enumerate(extra)})
        return tn.contract_network(sub, open_labels, order)

    return run, 2 ** len(extra)


def oracle_slice_cuts(circ, fixed, open_q, n_sliced, cap_log2):
    """The oracle's own slicing of the workload (no product code): the wire segments its
    greedy order slices to keep every intermediate within 2^cap_log2 entries; the first
    n_sliced of them define the slices, as (qubit, segment) cuts."""
    from oracle import network as tn

    tensors, open_labels = tn.circuit_tensors(circ, fixed, open_q)
    _, extra = tn.search_order([t.labels for t in tensors], open_labels, cap_log2, trials=4)
    cuts = [(lab[1], lab[2]) for lab in extra if lab[0] == "w"][:n_sliced]
    if len(cuts) < n_sliced:
        raise RuntimeError(f"the oracle's slicing gave {len(cuts)} cuts, fewer than {n_sliced}")
    return cuts


def timed_oracle(run, n_sub, min_seconds):
    """Run sub-slices 0, 1, ... until at least `min_seconds` passed; returns (count, seconds)."""
    t0 = time.perf_counter()
    k = 0
    while k < n_sub:
        run(k)
        k += 1
        if time.perf_counter() - t0 >= min_seconds:
            break
    return k, time.perf_counter() - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w, circ, fixed, open_q = workload(args.workload, 0)
    cuts = oracle_slice_cuts(circ, fixed, open_q, w["smin"], w["cap"])
    run, n_sub = oracle_sample(circ, fixed, open_q, cuts, args.cpu_sample_cap)
    per_step = min(args.ref_subslices, n_sub)
    for _ in range(args.warmup):
        run(0)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for i in range(per_step):
            run(i)
    dt = (time.perf_counter() - t0) / args.steps
    value = per_step / (dt * n_sub)
    cores = cpu_cores()
    line = {
        "impl": "reference", "metric": "slices/s", "value": value, "unit": "slices/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload}: 5x6 grid RQC, 14 cycles, 2^6 slices, cap 2^26, 1024-amplitude sub-cube",
                   "plan": args.plan},
        "cpu_baseline": {"value": value, "unit": "slices/s", "cores": cores, "kind": "oracle",
                         "sample": f"each step = sub-slices 0..{per_step - 1} of the {n_sub} oracle sub-contractions of "
                                   f"slice 0 (FP64, cap 2^{args.cpu_sample_cap}); slices/s = {per_step} / (step time * {n_sub})"},
        "e2e": {"value": value, "unit": "slices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# --------------------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    from oracle import metrics
    from paper_2504_09186_gb300 import tnc as T

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w, circ, fixed, open_q = workload(args.workload, rank)
    if args.plan_trials > 0:
        w = dict(w, trials=args.plan_trials)
    plan = T.Plan.greedy(circ, open_qubits=open_q, seed=w["plan_seed"], trials=w["trials"], log2_cap=w["cap"],
                         slices_min=w["smin"], slices_max=w["smax"] if args.plan == "greedy" else 64, mode=args.plan,
                         cluster_chains=args.cluster_chains)
    info = plan.info()
    fuse = not args.no_fuse
    n_slices = 1 << info["n_sliced"]
    ctx = T.Context(local)
    # a dedicated stream: the library enqueues on it and the CUDA events below time it
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    n_out = 1 << info["n_open"]
    out = torch.zeros((1, n_out), dtype=torch.complex128, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > L2 (129 MB)
    bits = np.ascontiguousarray(fixed[None, :], dtype=np.uint8)

    # tile configurations of the tensor-core steps chosen by timing (setup, untimed)
    tune = None
    if not args.no_autotune and args.precision != "c64":
        t0 = time.perf_counter()
        tune = ctx.autotune(plan, bits, args.precision, fuse=fuse)
        tune["setup_s"] = time.perf_counter() - t0

    def timed(precision, steps, warmup, profile):
        for _ in range(warmup):
            ctx.amplitudes(plan, bits, precision, out=out, stream=stream.cuda_stream, fuse=fuse)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        total = 0.0
        prof = None
        for _ in range(steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.amplitudes(plan, bits, precision, out=out, stream=stream.cuda_stream, profile=profile, fuse=fuse)
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
            if profile:
                p = ctx.profile_read()
                if prof is None:
                    prof = p
                else:
                    prof["ms"] = prof["ms"] + p["ms"]
                    prof["launches"] = prof["launches"] + p["launches"]
                    prof["flops"] = prof["flops"] + p["flops"]
                    prof["bytes"] = prof["bytes"] + p["bytes"]
        torch.cuda.synchronize()
        ms = max_over_ranks(total / steps, dist)
        return ms, prof, out.cpu().numpy()[0].copy()

    with ClockSampler(local) as clk:
        ms, prof, amp = timed(args.precision, args.steps, args.warmup, True)
    clocks = clk.summary()
    value = n_slices * world / (ms / 1e3)

    peaks = load_peaks()
    # complex64 beside it, and the error of both against each other / the oracle golden
    c64 = None
    if not args.no_compare and args.precision != "c64":
        ms64, prof64, amp64 = timed("c64", max(1, min(args.steps, 3)), 1, True)
        c64 = {"slices_per_s": n_slices * world / (ms64 / 1e3), "ms_per_step": ms64,
               "rel_err_vs_c64": metrics.rel_err_norm(amp, amp64)}
        if prof64 is not None and len(prof64["ms"]):
            k64 = int(np.argmax(prof64["ms"]))
            tf32 = measure_tf32_peak()
            r64 = roofline_tf32(int(prof64["kind"][k64]), prof64["flops"][k64] / prof64["launches"][k64],
                                prof64["bytes"][k64] / prof64["launches"][k64],
                                prof64["ms"][k64] / prof64["launches"][k64], tf32, peaks)
            r64["traffic"] = None
            r64["kernel"] = {"step": k64, "kind": int(prof64["kind"][k64]),
                             "share_of_step_time": float(prof64["ms"][k64] / prof64["ms"].sum())}
            c64["roofline"] = r64
            c64["tf32_peak_tflops_measured"] = tf32
            c64["tensor_core_steps"] = int(sum(1 for x in prof64["kind"] if int(x) == 4))
    golden = os.path.join(ROOT, "tests", "golden", "s30_subcube_amplitudes.txt")
    err_golden = None
    if args.workload == "s30" and rank == 0 and os.path.exists(golden):
        ref = np.loadtxt(golden)
        ref = ref[:, 0] + 1j * ref[:, 1]
        err_golden = metrics.rel_err_norm(amp, ref)
        if c64 is not None:
            c64["rel_err_vs_oracle"] = metrics.rel_err_norm(amp64, ref)

    # end to end: host bitstrings in, host amplitudes out, through the public API
    host_out = np.zeros((1, n_out), dtype=np.complex128)
    for _ in range(2):  # first call eager, second captures the CUDA graph of the wave
        ctx.amplitudes(plan, bits, args.precision, out=host_out, use_graph=True, fuse=fuse)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.amplitudes(plan, bits, args.precision, out=host_out, use_graph=True, fuse=fuse)
    e2e_s = (time.perf_counter() - t0) / args.steps
    h2d = bits.nbytes + n_slices * (8 + 4) + 12
    d2h = host_out.nbytes

    # roofline of the dominant kernel (largest device time), from the live events
    k = int(np.argmax(prof["ms"]))
    per_launch_ms = prof["ms"][k] / prof["launches"][k]
    kind = int(prof["kind"][k])
    flops_launch = prof["flops"][k] / prof["launches"][k]
    bytes_launch = prof["bytes"][k] / prof["launches"][k]
    roof = roofline_of(kind, flops_launch, bytes_launch, per_launch_ms, peaks)
    if roof["bound"] == "tensor":
        # the timed region is well under a second at full clocks: the burst peak applies
        roof["frac_of_sustained"] = roof["achieved"] / peaks["bf16_tflops_sustained"]
    roof["traffic"] = measured_traffic(kind, flops_launch)
    roof["kernel"] = {"step": k, "kind": kind, "share_of_step_time": float(prof["ms"][k] / max(1e-9, prof["ms"].sum())),
                      "ms_per_launch": per_launch_ms, "flops_per_launch": flops_launch, "bytes_per_launch": bytes_launch}
    roof["peak_source"] = peaks["_source"]
    order = np.argsort(-prof["ms"])[:8]
    top_steps = [{"step": int(i), "kind": int(prof["kind"][i]), "ms_per_step": float(prof["ms"][i] / args.steps),
                  "launches_per_step": int(prof["launches"][i] // args.steps)} for i in order]
    total_flops = float(prof["flops"].sum()) / args.steps
    waves = int(prof["launches"].min() / args.steps)
    launches = int(prof["launches"].sum() / args.steps) + 3 * waves  # + leaf gather, leaf scales, root sum per wave

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cuts = oracle_slice_cuts(circ, fixed, open_q, w["smin"], w["cap"])
        run, n_sub = oracle_sample(circ, fixed, open_q, cuts, args.cpu_sample_cap)
        k, dt = timed_oracle(run, n_sub, 10.0)
        cpu = {"value": k / (dt * n_sub), "unit": "slices/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": f"sub-slices 0..{k - 1} of the {n_sub} oracle sub-contractions of slice 0 (FP64, cap "
                         f"2^{args.cpu_sample_cap}), {dt:.1f} s; slices/s = {k} / (t * {n_sub})"}

    if rank == 0:
        line = {
            "metric": "slices/s", "value": value, "unit": "slices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"chalf": "f16", "cbf16": "bf16", "c64": "f32"}[args.precision],
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {w['rows']}x{w['cols']} grid RQC, {w['cycles']} cycles, "
                                   f"{n_slices} slices (cap 2^{w['cap']}), {n_out}-amplitude sub-cube per GPU",
                       "precision": args.precision, "slices_per_step": n_slices * world,
                       "plan": args.plan, "plan_trials": w["trials"], "fused_chains": bool(fuse and info["n_fused"] > 0), "cluster_chains": bool(args.cluster_chains),
                       "plan_log2_cmacs_per_slice": info["log2_flops_per_slice"], "sliced_indices": info["n_sliced"],
                       "complex_tflops": total_flops / (ms / 1e3) / 1e12,
                       "l2": "256 MiB flush before every timed step; intermediates up to 2^26 entries > L2",
                       "parallelism": f"replicas x{world} (independent sub-cubes)",
                       "autotune": tune},
            "complex64": c64,
            "rel_err_vs_oracle": err_golden,
            "e2e": {"value": n_slices * world / e2e_s, "unit": "slices/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "top_steps": top_steps,
            "roofline": roof,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# --------------------------------------------------------------------------- other workloads
def measure_tf32_peak():
    """Dense TF32 tensor throughput of this GPU, measured: cuBLAS FP32 GEMM with TF32 math,
    8192^3 (2 N^3 flops), best of 10 launches timed with CUDA events."""
    import torch

    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        n = 8192
        a = torch.randn(n, n, device="cuda", dtype=torch.float32)
        b = torch.randn(n, n, device="cuda", dtype=torch.float32)
        for _ in range(3):
            torch.matmul(a, b)
        best = None
        for _ in range(10):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
        return 2.0 * n ** 3 / (best * 1e-3) / 1e12
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev


def roofline_tf32(kind, flops, nbytes, ms, tf32_peak, peaks):
    """Roofline of a complex64 launch.  On the 3xTF32 tensor-core kernel (kind 4) every real
    product is three TF32 products, so the tensor pipe executes 3x the algorithmic flops:
    achieved = 3 flops / time against the measured TF32 peak, tensor-bound above that
    balance.  Complex64 SIMT kernels: roofline_of."""
    if kind != 4:
        return roofline_of(kind, flops, nbytes, ms, peaks)
    if 3 * flops / max(nbytes, 1.0) >= tf32_peak * 1e3 / peaks["hbm_gbs"]:
        r = {"bound": "tensor", "achieved": 3 * flops / (ms * 1e-3) / 1e12, "peak": tf32_peak, "unit": "TFLOP/s",
             "peak_kind": "cuBLAS TF32 GEMM 8192^3, measured in this run",
             "complex_tflops": flops / (ms * 1e-3) / 1e12}
    else:
        r = {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
             "peak_kind": "STREAM-style copy, measured"}
    r["frac"] = r["achieved"] / r["peak"]
    return r


def roofline_of(kind, flops, nbytes, ms, peaks):
    """Roofline of one kernel launch from its algorithmic flops / bytes and device time.
    Tensor-core kernels (kinds 3-6) are tensor-bound above the machine balance
    (bf16 peak / HBM bandwidth), SIMT kernels above the FP32-ALU balance; HBM-bound below."""
    alu = N_SM * FP32_LANES_PER_SM * 2 * peaks.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    intensity = flops / max(nbytes, 1.0)
    tc = kind in (3, 4, 5, 6)
    if tc and intensity >= peaks["bf16_tflops"] * 1e3 / peaks["hbm_gbs"]:
        r = {"bound": "tensor", "achieved": flops / (ms * 1e-3) / 1e12, "peak": peaks["bf16_tflops"], "unit": "TFLOP/s",
             "peak_kind": "burst (cuBLAS bf16, measured)"}
    elif not tc and intensity >= alu * 1e3 / peaks["hbm_gbs"]:
        r = {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": alu, "unit": "TFLOP/s",
             "peak_kind": "152 SMs x 128 FP32 lanes x 2 flops x max SM clock"}
    else:
        r = {"bound": "hbm", "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
             "peak_kind": "STREAM-style copy, measured"}
    r["frac"] = r["achieved"] / r["peak"]
    return r


SW_POINTS = [(14, 12, 10), (12, 12, 12), (16, 8, 16), (16, 12, 12), (12, 16, 12), (12, 20, 12), (16, 4, 16),
             (4, 16, 16), (16, 16, 4), (8, 16, 8), (8, 24, 8), (4, 24, 4), (2, 24, 2), (1, 24, 1), (2, 20, 2)]


def sweep_labels(m, k, n, layout, seed):
    """Index labels of one sweep point.  'random': seeded random axis orders of A, B and C.
    'arranged': the order the step compiler gives tensor-core steps (K tile labels, then
    the M / N tile labels, lowest; C led by three tile columns, then the tile rows, then the
    other tile columns), the rest random; for GEPDOT shapes (M N <= 2^10, K >= 2^12) both
    operands lead with all common labels in one order."""
    rng = np.random.default_rng(seed)
    ms, ks, ns = list(range(m)), list(range(100, 100 + k)), list(range(200, 200 + n))
    perm = lambda v: [int(x) for x in rng.permutation(v)] if v else []
    if layout == "arranged" and m + n <= 10 and k >= 12:
        # GEPDOT: both operands lead with the common labels in one order (contiguous K runs)
        return ks + perm(ms), ks + perm(ns), perm(ms + ns)
    if layout == "arranged":
        kt = 5 if k >= 5 else 4
        nt = 8 if (n >= 8 and k > kt + 3) else (7 if n >= 7 else 6)
        return (ks[:kt] + ms[:7] + perm(ms[7:] + ks[kt:]), ks[:kt] + ns[:nt] + perm(ns[nt:] + ks[kt:]),
                ns[:3] + ms[:7] + ns[3:nt] + perm(ms[7:] + ns[nt:]))
    return perm(ms + ks), perm(ks + ns), perm(ms + ns)


def run_sweep(args):
    import torch

    from paper_2504_09186_gb300 import tnc as T

    torch.cuda.set_device(0)
    ctx = T.Context(0)
    peaks = load_peaks()
    dt = {"chalf": torch.float16, "cbf16": torch.bfloat16, "c64": torch.float32}
    pts = [tuple(int(x) for x in s.split(",")) for s in args.sw_shapes.split(";")] if args.sw_shapes else SW_POINTS
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    tf32 = measure_tf32_peak()
    out = []
    for (m, k, n) in pts:
        gepdot = m + n <= 10 and k >= 12
        layouts = ["arranged", "random"] if ((m >= 7 and n >= 6 and k >= 4) or gepdot) else ["random"]
        for layout in layouts:
            seed = 1000003 * m + 1009 * k + n + (7 if layout == "random" else 0)
            la, lb, lc = sweep_labels(m, k, n, layout, seed)
            for prec in ("chalf", "cbf16", "c64"):
                if prec == "c64" and (m + k + n > 40 or max(m + k, k + n, m + n) > 28):
                    continue  # keep each complex64 point (SIMT on random layouts) under a few seconds
                if prec == "cbf16" and layout == "random":
                    continue  # same kernels and rates as chalf
                g = torch.Generator(device="cuda")
                g.manual_seed(seed)
                sig = (2.0 ** -k) ** 0.5 / 2 ** 0.5
                a = torch.randn(2 << len(la), dtype=dt[prec], device="cuda", generator=g).mul_(sig)
                b = torch.randn(2 << len(lb), dtype=dt[prec], device="cuda", generator=g).mul_(sig)
                c = torch.empty(2 << len(lc), dtype=dt[prec], device="cuda")
                for _ in range(args.warmup):
                    ctx.contract(prec, a, la, b, lb, c, lc)
                times = []
                for _ in range(args.steps):
                    flush.zero_()
                    ctx.contract(prec, a, la, b, lb, c, lc)
                    pr = ctx.profile_read(cap=1)
                    times.append(float(pr["ms"][0]))
                ms = statistics.median(times)
                kind, fl, by = int(pr["kind"][0]), float(pr["flops"][0]), float(pr["bytes"][0])
                r = roofline_tf32(kind, fl, by, ms, tf32, peaks) if prec == "c64" else roofline_of(kind, fl, by, ms, peaks)
                out.append({"m": m, "k": k, "n": n, "layout": layout, "precision": prec, "kernel_kind": kind,
                            "launches": int(pr["launches"][0]), "ms": ms, "tflops": fl / ms / 1e9,
                            "gbs": by / ms / 1e6, "bound": r["bound"], "frac": r["frac"]})
                del a, b, c
                torch.cuda.empty_cache()
    head = next((p for p in out if (p["m"], p["k"], p["n"], p["layout"], p["precision"]) == (14, 12, 10, "arranged", "chalf")), out[0])
    line = {"metric": "complex TFLOP/s per contraction step", "value": head["tflops"], "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": "sw: single pairwise contractions, log2 (M,K,N) points, complex normal(0, 1/sqrt(K))",
                       "value_point": [head["m"], head["k"], head["n"], head["layout"], head["precision"]],
                       "l2": "256 MiB flush before every timed call", "timing": "contraction kernels only (CUDA events)",
                       "tf32_peak_tflops_measured": tf32,
                       "c64_frac": "3xTF32 tensor-core points: 3 x 8MNK / time over the measured TF32 peak"},
            "points": out}
    print(json.dumps(line))


def run_s60(args):
    """60-qubit workload: the qubit-split plan (cap 2^32), a seeded sample of distinct slice
    ids contracted by one tnc_amplitudes_ids call; per-slice throughput, the total cost of
    the plan, and complex-half against complex64 per slice and on a summed subset."""
    import torch

    from inputs import grid_circuit, random_bitstrings
    from paper_2504_09186_gb300 import tnc as T

    torch.cuda.set_device(0)
    circ = grid_circuit(6, 10, 24, seed=1)
    bits = random_bitstrings(60, 1, seed=4)
    t0 = time.perf_counter()
    plan = T.Plan.greedy(circ, open_qubits=[], seed=3, trials=args.s60_trials, log2_cap=32, mode="split",
                         objective="time")
    plan_s = time.perf_counter() - t0
    info = plan.info()
    s = info["n_sliced"]
    rng = np.random.default_rng(4)
    space = 1 << min(s, 62)
    ids, seen = [], set()
    while len(ids) < args.s60_slices:
        x = int(rng.integers(0, space))
        if x not in seen:
            seen.add(x)
            ids.append(x)
    ctx = T.Context(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = torch.zeros((1, 1), dtype=torch.complex128, device="cuda")
    peaks = load_peaks()

    def timed(prec, sids, profile=False):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.amplitudes_ids(plan, bits, sids, prec, out=out, stream=stream.cuda_stream, profile=profile)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), complex(out.cpu().numpy()[0, 0])

    tune = None
    if not args.no_autotune:
        t0 = time.perf_counter()
        tune = ctx.autotune(plan, bits, "chalf", slice_begin=ids[0], slice_count=1)
        tune["setup_s"] = time.perf_counter() - t0
    for _ in range(max(1, args.warmup)):
        timed("chalf", ids[:1])
    with ClockSampler(0) as clk:
        ms_all, amp_sum = timed("chalf", ids)
    clocks = clk.summary()
    per_slice_s = ms_all / len(ids) / 1e3
    value = 1.0 / per_slice_s
    # per-step device times on a few slices (a separate, profiled call)
    n_prof = min(4, len(ids))
    ms_prof, _ = timed("chalf", ids[:n_prof], profile=True)
    prof = ctx.profile_read()
    k = int(np.argmax(prof["ms"]))
    roof = roofline_of(int(prof["kind"][k]), prof["flops"][k] / prof["launches"][k], prof["bytes"][k] / prof["launches"][k],
                       prof["ms"][k] / prof["launches"][k], peaks)
    roof["traffic"] = None
    roof["kernel"] = {"step": k, "kind": int(prof["kind"][k]), "share_of_slice_time": float(prof["ms"][k] / prof["ms"].sum()),
                      "profiled_slices": n_prof}
    # complex-half against complex64: single slices, and the sum over the first few
    cmp64 = []
    per16 = []
    for sid in ids[: args.s60_c64]:
        _, a16 = timed("chalf", [sid])
        ms64, a64 = timed("c64", [sid])
        per16.append(a16)
        cmp64.append({"slice": sid, "ms_c64": ms64, "rel_err_chalf_vs_c64": abs(a16 - a64) / max(abs(a64), 1e-300)})
    summed = None
    if args.s60_sum_c64 > 0:
        sub = ids[: args.s60_sum_c64]
        _, s16 = timed("chalf", sub)
        ms64, s64 = timed("c64", sub)
        summed = {"slices": len(sub), "ms_c64": ms64, "rel_err_chalf_vs_c64": abs(s16 - s64) / max(abs(s64), 1e-300)}
    line = {"metric": "slices/s", "value": value, "unit": "slices/s", "n_gpus": 1, "steps": 1,
            "warmup": max(1, args.warmup), "ms_per_step": ms_all, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": "s60: 6x10 grid RQC, 24 cycles, cap 2^32 chalf entries, one bitstring; qubit-split "
                                   "plan; one tnc_amplitudes_ids call over a seeded sample of distinct slice ids",
                       "slices_per_step": len(ids), "slice_id_seed": 4, "sliced_indices": s,
                       "plan_mode": "split", "plan_trials": args.s60_trials, "plan_seconds": plan_s,
                       "plan_log2_cmacs_per_slice": info["log2_flops_per_slice"],
                       "log2_total_cmacs": info["log2_total_flops"],
                       "log2_executed_cmacs_all_slices_with_reuse": info["log2_executed_flops"],
                       "log2_executed_cmacs_all_slices_with_reuse_and_merging": info["log2_executed_flops_merged"],
                       "plan_max_log2_size": info["max_log2_size"],
                       "plan_model_seconds_per_slice": info["model_seconds_per_slice"],
                       "complex_tflops": 8 * 2 ** info["log2_flops_per_slice"] * value / 1e12,
                       "extrapolated_total_log2_seconds": s - float(np.log2(value)), "autotune": tune,
                       "l2": "intermediates of 2^27..2^32 entries (0.5..16 GiB): L2-cold by size"},
            "amplitude_sum_chalf": [amp_sum.real, amp_sum.imag],
            "complex64": {"per_slice": cmp64, "summed": summed}, "roofline": roof, "clocks": clocks,
            "profiled_ms": ms_prof}
    print(json.dumps(line))


def run_d20(args):
    import torch

    from inputs import grid_circuit, random_bitstrings
    from paper_2504_09186_gb300 import tnc as T

    torch.cuda.set_device(0)
    circ = grid_circuit(4, 5, 12, seed=1, fsim_mode="uniform", param_seed=5)
    bits = random_bitstrings(20, 256, seed=6)
    rng = np.random.default_rng(7)
    w = rng.normal(size=256) + 1j * rng.normal(size=256)
    plan = T.Plan.greedy(circ, open_qubits=[], seed=3, trials=8, log2_cap=20)
    ar = [len(g.qubits) for g in circ.gates]
    ctx = T.Context(0)
    for _ in range(args.warmup):
        ctx.adjoint(plan, bits, w[:, None], ar)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.adjoint(plan, bits, w[:, None], ar)
    adj_s = (time.perf_counter() - t0) / args.steps
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.amplitudes(plan, bits, "c64")
    fwd_s = (time.perf_counter() - t0) / args.steps
    line = {"metric": "gradient evaluations/s", "value": 1.0 / adj_s, "unit": "adjoint calls/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": adj_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "d20: 4x5 grid RQC, 12 cycles, fSim angles U[0,pi], 256 bitstrings, complex64; "
                                   "one call = amplitudes + gradients w.r.t. every gate (host buffers, wall clock)",
                       "n_gates": len(ar), "forward_only_ms": fwd_s * 1e3}}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        if args.workload in WORKLOADS:
            run_reference(args)
        elif int(os.environ.get("RANK", "0")) == 0:
            print(json.dumps({"impl": "reference", "unavailable": f"the oracle arm times the s30/t12 workloads only"}))
    elif args.workload == "sw":
        run_sweep(args)
    elif args.workload == "s60":
        run_s60(args)
    elif args.workload == "d20":
        run_d20(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
