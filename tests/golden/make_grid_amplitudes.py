"""Write FP64 reference amplitudes of a random grid circuit with the oracle's
in-place state-vector method (Section 1) -- the expected values of the
full-size contraction-tree tests, which the oracle cannot contract as a
tensor network in reasonable time.

Usage: python tests/golden/make_grid_amplitudes.py ROWS COLS DEPTH [N_BITSTRINGS]
Writes tests/golden/grid{ROWS}x{COLS}_d{DEPTH}_amplitudes.txt.  The circuit is
qcs_inputs.random_grid_circuit(ROWS, COLS, DEPTH, seed=0) (fSim(pi/2, pi/6));
the bitstrings are qcs_inputs.random_bitstrings(n, N, seed=1).  Needs 16 * 2^n
bytes of host memory (16 GiB at n = 30).
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import qcs_inputs as qi  # noqa: E402


def main():
    rows, cols, depth = (int(v) for v in sys.argv[1:4])
    count = int(sys.argv[4]) if len(sys.argv) > 4 else 8
    n = rows * cols
    circ = qi.random_grid_circuit(rows, cols, depth, seed=0)
    bits = qi.random_bitstrings(n, count, seed=1)
    t0 = time.time()
    psi = oracle.statevector_inplace(circ)
    norm = float(np.vdot(psi, psi).real)
    amps = [psi[oracle.bit_index(x)] for x in bits]
    path = os.path.join(HERE, f"grid{rows}x{cols}_d{depth}_amplitudes.txt")
    with open(path, "w") as f:
        f.write(f"# FP64 amplitudes <x|U|0> of qcs_inputs.random_grid_circuit({rows}, {cols}, {depth}, "
                f"seed=0), bitstrings qcs_inputs.random_bitstrings({n}, {count}, seed=1)\n")
        f.write(f"# written by tests/golden/make_grid_amplitudes.py (oracle.statevector_inplace, "
                f"{time.time() - t0:.0f} s); sum of |amplitude|^2 over all 2^{n} states = {norm:.15f}\n")
        f.write("# format: bitstring re im\n")
        for x, a in zip(bits, amps):
            f.write("".join(str(int(b)) for b in x) + f" {a.real:.17e} {a.imag:.17e}\n")
    print(path)


if __name__ == "__main__":
    main()
