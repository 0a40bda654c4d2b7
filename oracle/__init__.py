"""FP64 CPU oracle for sliced tensor-network contraction of random-circuit amplitudes.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline
leg of `bench.py` may import this package.  The GPU library never imports, links or
calls it, and this package imports nothing from the GPU library: the two share only
the seeded input generators in `inputs/`.

What it computes (all complex128, plain and slow on purpose):

* `statevector` -- amp(x) = <x| U_L ... U_1 |0^n> by applying every gate to a dense
  2^n state (the plain definition the tensor-network method reaches, Sec. I, Sec. II-A).
  A *slice* (Sec. II-A, Sec. III-A: fixing a sliced index to 0 or 1) is evaluated by
  inserting the projector |b><b| on that wire segment, so sum over slices = amplitude.
  Gradient environments dA/dG for every gate come from forward/backward states.
* `network` -- the oracle's own tensor network (one tensor per gate, boundary vectors)
  and a pairwise contraction of it (Sec. II-A: contract tensors sharing an index until
  one remains), with its own greedy order, fixed sliced indices, and exact sub-slicing
  when an intermediate would exceed a size cap.
* `pairwise` -- a single binary-index contraction C = A * B over common labels
  (Sec. II-A, the M x K x N view), by einsum, by explicit loops, or one output at a time.
* `metrics` -- error norms, XEB and Porter-Thomas statistics.

Parity pins for each part live in `tests/test_oracle_*.py`.
"""
