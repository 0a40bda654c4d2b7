"""Slice sharding on the host: chunks dealt to ranks, checkpoints, resumption after a rank
stops, verification reruns, and the gloo combination of two ranks.  The chunk values come
from the oracle (per-slice amplitudes by projectors), so the sum is checked against the
unsliced state vector."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

from inputs import grid_circuit, subcube_bitstrings, subcube_spec
from oracle import statevector as sv
from paper_2504_09186_gb300 import shard
from paper_2504_09186_gb300 import tnc as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _problem():
    c = grid_circuit(3, 4, 8, seed=1)
    fixed, open_q = subcube_spec(12, 3, seed=2)
    p = T.Plan.greedy(c, open_qubits=open_q, seed=3, trials=8, log2_cap=7, slices_min=4)
    cuts = p.sliced_cuts()
    bs = subcube_bitstrings(fixed, open_q)

    def chunk(begin, count, calls=None):
        if calls is not None:
            calls.append(begin)
        tot = 0
        for sid in range(begin, begin + count):
            tot = tot + sv.circuit_amplitudes(c, bs, {cut: (sid >> t) & 1 for t, cut in enumerate(cuts)})
        return np.asarray(tot, dtype=np.complex128)[None, :]

    return c, bs, len(cuts), chunk


def test_chunks_sum_to_the_amplitudes(tmp_path):
    c, bs, s, chunk = _problem()
    spec = shard.ShardSpec(n_slices=1 << s, chunk=3)
    got = shard.run_rank(spec, chunk, shard.CheckpointStore(str(tmp_path), 0), verify_fraction=0.5)
    assert spec.n_chunks == ((1 << s) + 2) // 3
    assert np.allclose(got[0], sv.circuit_amplitudes(c, bs), atol=1e-12)


def test_resume_after_a_stop_computes_only_the_rest(tmp_path):
    c, bs, s, chunk = _problem()
    spec = shard.ShardSpec(n_slices=1 << s, chunk=2, world=2, rank=1)
    store = shard.CheckpointStore(str(tmp_path), 1)
    calls = []
    with pytest.raises(RuntimeError):
        shard.run_rank(spec, lambda b, n: chunk(b, n, calls), store, stop_after=2)
    assert len(calls) == 2
    calls2 = []
    resumed = shard.run_rank(spec, lambda b, n: chunk(b, n, calls2), shard.CheckpointStore(str(tmp_path), 1))
    assert len(calls2) == len(spec.chunks()) - 2 and not set(calls) & set(calls2)
    clean = shard.run_rank(spec, chunk, shard.CheckpointStore(str(tmp_path / "clean"), 1))
    assert np.array_equal(resumed, clean)


def test_verification_rerun_catches_a_wrong_checkpoint(tmp_path):
    _, _, s, chunk = _problem()
    spec = shard.ShardSpec(n_slices=1 << s, chunk=4)
    store = shard.CheckpointStore(str(tmp_path), 0)
    shard.run_rank(spec, chunk, store)
    # a silently wrong result that was checkpointed with a consistent digest
    bad = store.load(1)
    bad[0, 0] += 1e-9
    store.save(1, bad)
    with pytest.raises(shard.VerificationError):
        shard.run_rank(spec, chunk, shard.CheckpointStore(str(tmp_path), 0), verify_fraction=1.0)
    # a damaged file (digest mismatch) is recomputed instead of trusted
    with open(os.path.join(str(tmp_path), "chunk2.npy"), "r+b") as f:
        f.seek(-8, 2)
        f.write(b"\x00" * 8)
    assert not shard.CheckpointStore(str(tmp_path), 0).has(2)


def _free_port():
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _rank(rank, world, port, directory, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_2504_09186_gb300 import shard as sh

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, _, s, chunk = _problem()
        spec = sh.ShardSpec(n_slices=1 << s, chunk=2, world=world, rank=rank)
        part = sh.run_rank(spec, chunk, sh.CheckpointStore(directory, rank), verify_fraction=0.25, seed=5)
        out[rank] = sh.combine(part, dist)
    finally:
        dist.destroy_process_group()


def test_two_ranks_combine_to_the_amplitudes(tmp_path):
    c, bs, _, _ = _problem()
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, str(tmp_path), out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(180)
            assert p.exitcode == 0
        res = dict(out)
    assert np.array_equal(res[0], res[1])
    assert np.allclose(res[0][0], sv.circuit_amplitudes(c, bs), atol=1e-12)
