"""Write FP64 partial amplitudes of sampled slices (Section 5.3) of a random
grid circuit with the oracle's tensor-network contraction -- the expected
values of the large sliced-contraction test.

Usage: python tests/golden/make_sliced_partials.py ROWS COLS DEPTH N_SLICED N_SAMPLES
Writes tests/golden/slices{ROWS}x{COLS}_d{DEPTH}.txt.  Circuit
qcs_inputs.random_grid_circuit(ROWS, COLS, DEPTH, seed=0), bitstring
qcs_inputs.random_bitstrings(n, 1, seed=1)[0].  The oracle picks the sliced
indices itself (oracle.slice_labels_by_weight on its own randomised greedy
order), draws N_SAMPLES value assignments with numpy seed 7, and contracts
each sliced network in FP64 (numpy tensordot steps).
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
    rows, cols, depth, n_sliced, n_samples = (int(v) for v in sys.argv[1:6])
    n = rows * cols
    circ = qi.random_grid_circuit(rows, cols, depth, seed=0)
    bits = qi.random_bitstrings(n, 1, seed=1)[0]
    tens, outl = oracle.circuit_tn(circ, bits)
    order0 = oracle.random_greedy_order(tens, outl, seeds=range(6))
    labels = oracle.slice_labels_by_weight(tens, outl, order0, n_sliced)
    sub0 = oracle.slice_network(tens, {l: 0 for l in labels})
    order = oracle.random_greedy_order(sub0, outl, seeds=range(6))
    flops, big = oracle.order_cost(sub0, order, outl)
    g = np.random.default_rng(7)
    samples = [tuple(int(v) for v in g.integers(0, 2, size=n_sliced)) for _ in range(n_samples)]
    path = os.path.join(HERE, f"slices{rows}x{cols}_d{depth}.txt")
    lines = []
    t0 = time.time()
    for vals in samples:
        sub = oracle.slice_network(tens, dict(zip(labels, vals)))
        a = complex(oracle.contract_network(sub, outl, order))
        lines.append("".join(str(v) for v in vals) + f" {a.real:.17e} {a.imag:.17e}")
        print(lines[-1], f"{time.time() - t0:.0f} s", flush=True)
    with open(path, "w") as f:
        f.write(f"# FP64 partial amplitudes: qcs_inputs.random_grid_circuit({rows}, {cols}, {depth}, seed=0), "
                f"bitstring qcs_inputs.random_bitstrings({n}, 1, seed=1)[0], each with the sliced indices "
                f"fixed to one sampled assignment\n")
        f.write(f"# written by tests/golden/make_sliced_partials.py (oracle contraction, {flops:.3e} flops "
                f"and 2^{big} largest intermediate per slice, {time.time() - t0:.0f} s)\n")
        f.write("sliced " + " ".join(str(l) for l in labels) + "\n")
        f.write("# format: values of the sliced indices (in the order above) re im\n")
        for ln in lines:
            f.write(ln + "\n")
    print(path)


if __name__ == "__main__":
    main()
