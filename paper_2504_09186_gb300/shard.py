"""Slice sharding across processes, with checkpoints, resumption and verification reruns.

The slices of a plan are independent subtasks whose amplitudes add (Sec. III-A).  A run over
the slice ids [0, n_slices) is cut into chunks of consecutive ids, and the chunks are dealt
to the ranks round-robin.
  * Every finished chunk's FP64 partial sum is checkpointed: one `.npy` file per chunk,
    written atomically, with its SHA-256 recorded in the rank's manifest.
  * A restarted rank reloads the chunks it has and computes only the rest.
  * Before summing, a seeded fraction of the finished chunks is recomputed and compared bit
    for bit with the checkpoint (the re-run-and-compare of Sec. VI).  The library's sums are
    deterministic, so any difference is an error.
  * Ranks combine their partial sums by gathering them and adding in rank order, so every
    rank holds the same result.

The chunk computation is a callable `chunk(begin, count) -> complex128 array`, so the host
logic runs and is tested without a GPU; `gpu_chunk` is the library's own.
"""
from __future__ import annotations

import hashlib
import io
import json
import os
from dataclasses import dataclass
from typing import Callable, Dict, List, Optional

import numpy as np

Chunk = Callable[[int, int], np.ndarray]


class VerificationError(RuntimeError):
    """A recomputed chunk differs from its checkpoint."""


@dataclass(frozen=True)
class ShardSpec:
    n_slices: int  # slice ids [0, n_slices)
    chunk: int     # slices per chunk
    world: int = 1
    rank: int = 0

    def __post_init__(self):
        if self.n_slices < 1 or self.chunk < 1 or self.world < 1 or not 0 <= self.rank < self.world:
            raise ValueError("bad shard spec")

    @property
    def n_chunks(self) -> int:
        return (self.n_slices + self.chunk - 1) // self.chunk

    def chunks(self) -> List[int]:
        """Chunk ids of this rank, in order."""
        return list(range(self.rank, self.n_chunks, self.world))

    def span(self, cid: int):
        begin = cid * self.chunk
        return begin, min(self.chunk, self.n_slices - begin)


def _sha(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


class CheckpointStore:
    """Per-chunk FP64 partial sums of one rank under `directory`, with a SHA-256 manifest."""

    def __init__(self, directory: str, rank: int):
        self.dir = directory
        os.makedirs(directory, exist_ok=True)
        self.manifest_path = os.path.join(directory, f"rank{rank}.json")
        self.manifest: Dict[str, str] = {}
        if os.path.exists(self.manifest_path):
            with open(self.manifest_path) as f:
                self.manifest = json.load(f)

    def _path(self, cid: int) -> str:
        return os.path.join(self.dir, f"chunk{cid}.npy")

    def has(self, cid: int) -> bool:
        """True when the chunk's file exists and matches the manifest's digest."""
        path = self._path(cid)
        if str(cid) not in self.manifest or not os.path.exists(path):
            return False
        return _sha(np.load(path)) == self.manifest[str(cid)]

    def load(self, cid: int) -> np.ndarray:
        return np.load(self._path(cid))

    def save(self, cid: int, part: np.ndarray) -> None:
        part = np.ascontiguousarray(part, dtype=np.complex128)
        buf = io.BytesIO()
        np.save(buf, part)
        tmp = self._path(cid) + ".tmp"
        with open(tmp, "wb") as f:
            f.write(buf.getvalue())
        os.replace(tmp, self._path(cid))
        self.manifest[str(cid)] = _sha(part)
        tmp = self.manifest_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(self.manifest, f)
        os.replace(tmp, self.manifest_path)


def run_rank(spec: ShardSpec, chunk: Chunk, store: CheckpointStore, verify_fraction: float = 0.0,
             seed: int = 0, stop_after: Optional[int] = None) -> np.ndarray:
    """Compute (or reload) this rank's chunks, verify a seeded fraction of them by
    recomputation, and return the rank's partial sum (added in chunk-id order).

    `stop_after`: stop with RuntimeError after computing that many chunks (a failure
    injected on the host, to exercise resumption)."""
    parts: Dict[int, np.ndarray] = {}
    computed = 0
    for cid in spec.chunks():
        if store.has(cid):
            parts[cid] = store.load(cid)
            continue
        if stop_after is not None and computed >= stop_after:
            raise RuntimeError(f"rank {spec.rank} stopped after {computed} chunks")
        begin, count = spec.span(cid)
        part = np.asarray(chunk(begin, count), dtype=np.complex128)
        store.save(cid, part)
        parts[cid] = part
        computed += 1
    if verify_fraction > 0 and parts:
        rng = np.random.default_rng([seed, spec.rank])
        ids = sorted(parts)
        n = max(1, int(np.ceil(verify_fraction * len(ids))))
        for cid in sorted(rng.choice(ids, size=min(n, len(ids)), replace=False).tolist()):
            begin, count = spec.span(cid)
            again = np.asarray(chunk(begin, count), dtype=np.complex128)
            if not np.array_equal(again, parts[cid]):
                raise VerificationError(f"chunk {cid} (slices {begin}..{begin + count - 1}) differs on recomputation")
    total = None
    for cid in sorted(parts):
        total = parts[cid].copy() if total is None else total + parts[cid]
    return total


def combine(partial: np.ndarray, dist=None) -> np.ndarray:
    """Sum of the ranks' partial sums, added in rank order (identical on every rank)."""
    if dist is None or dist.get_world_size() == 1:
        return partial
    import torch

    t = torch.from_numpy(np.ascontiguousarray(partial).view(np.float64).copy())
    if dist.get_backend() == "nccl":
        t = t.cuda()
    out = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(out, t)
    total = None
    for o in out:
        v = o.cpu().numpy().view(np.complex128).reshape(partial.shape)
        total = v.copy() if total is None else total + v
    return total


def gpu_chunk(ctx, plan, bitstrings, precision: str = "chalf") -> Chunk:
    """The library's chunk: amplitudes of `bitstrings` summed over slice ids [begin, begin + count)."""
    def run(begin: int, count: int) -> np.ndarray:
        return ctx.amplitudes(plan, bitstrings, precision, slice_begin=begin, slice_count=count)

    return run
