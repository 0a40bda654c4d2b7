"""Writes s30_subcube_amplitudes.txt: the FP64 state-vector amplitudes of the 1024-bitstring
sub-cube of the 30-qubit 5x6 grid circuit (14 cycles, circuit seed 1; open qubits 20..29,
the other bits from sub-cube seed 2), in sub-cube order (first open qubit most significant).

Only the oracle and the seeded input generators are used: amp(x) = <x| U_L ... U_1 |0^n>
(Sec. I, Sec. II-A) by the plain C state vector (16 GiB of host memory, ~15 min on 8 cores).
Also writes the oracle's full-distribution statistics used by the XEB check.
Run from the repository root:  python tests/golden/make_s30_golden.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from inputs import grid_circuit, subcube_bitstrings, subcube_spec  # noqa: E402
from oracle import sv_c  # noqa: E402


def main():
    t0 = time.time()
    c = grid_circuit(5, 6, 14, seed=1)
    fixed, open_q = subcube_spec(30, 10, seed=2)
    bs = subcube_bitstrings(fixed, open_q)
    psi = sv_c.final_state(c)
    w = 1 << np.arange(29, -1, -1, dtype=np.int64)
    amps = psi[bs.astype(np.int64) @ w]
    norm = float(np.sum(np.abs(psi) ** 2))
    p = np.abs(psi) ** 2
    second = float((1 << 30) * np.sum(p * p))
    del psi, p
    out = os.path.join(HERE, "s30_subcube_amplitudes.txt")
    with open(out, "w") as f:
        f.write("# FP64 state-vector amplitudes, 5x6 grid RQC, 14 cycles, circuit seed 1 (Sec. I, Sec. II-A)\n")
        f.write(f"# sub-cube: open qubits {open_q[0]}..{open_q[-1]}, fixed bits {''.join(map(str, fixed))} (seed 2)\n")
        f.write(f"# full-state norm {norm:.15f}; 2^n sum p^2 = {second:.6f} (Porter-Thomas: ~2)\n")
        f.write("# one row per sub-cube entry i (first open qubit = most significant bit of i): re im\n")
        for a in amps:
            f.write(f"{a.real:.17e} {a.imag:.17e}\n")
    print(f"wrote {out} in {time.time() - t0:.0f} s; norm {norm:.15f}; 2^n sum p^2 {second:.4f}")


if __name__ == "__main__":
    main()
