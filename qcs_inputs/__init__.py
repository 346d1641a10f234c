"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method (no splitting, statistics,
selection, contraction or GEMM).  It only draws the synthetic data that both
sides consume:

* CGEMM operands with a controlled exponent spread (the CGEMM sweep workload,
  and the uniform (-1, 1) inputs of the CGEMM unit test in Section 3);
* the random quantum circuits (grid, depth, gate choice, fSim parameters);
* random bitstrings;
* the Type-1/2/3 element initialisations of the exploratory experiment in
  Section 5.2.

Every generator takes an explicit integer seed and uses numpy's PCG64, so the
same call gives the same values on any machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

__all__ = [
    "cgemm_operand",
    "uniform_operand",
    "Gate",
    "Circuit",
    "random_grid_circuit",
    "random_bitstrings",
    "typed_matrix",
    "SQRT_GATES",
    "fsim",
]


def _flatten(seed):
    if isinstance(seed, (tuple, list)):
        out = []
        for s in seed:
            out.extend(_flatten(s))
        return out
    return [int(seed)]


def _rng(seed) -> np.random.Generator:
    """PCG64 generator from an integer seed or a (nested) tuple of integers."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(_flatten(seed))))


# ---------------------------------------------------------------------------
# CGEMM operands
# ---------------------------------------------------------------------------

def cgemm_operand(rows: int, cols: int, s: int, seed, ld: int | None = None) -> np.ndarray:
    """Column-major complex64 matrix with ``ld >= rows``.

    Real and imaginary parts are drawn independently as N(0, 1) * 2**e with
    e ~ Uniform int [-s, s] per real scalar.  The result is returned as a
    Fortran-ordered (ld, cols) complex64 array whose first ``rows`` rows hold
    the matrix; padding rows (if ``ld > rows``) hold NaN so that a kernel that
    reads them is caught.
    """
    ld = rows if ld is None else ld
    assert ld >= rows
    g = _rng(seed)
    re = g.standard_normal((rows, cols), dtype=np.float64)
    im = g.standard_normal((rows, cols), dtype=np.float64)
    if s > 0:
        re = re * np.exp2(g.integers(-s, s + 1, size=(rows, cols)))
        im = im * np.exp2(g.integers(-s, s + 1, size=(rows, cols)))
    out = np.full((ld, cols), np.nan + 1j * np.nan, dtype=np.complex64, order="F")
    out[:rows, :] = (re + 1j * im).astype(np.complex64)
    return out


def sgemm_operand(rows: int, cols: int, s: int, seed, ld: int | None = None) -> np.ndarray:
    """Column-major float32 matrix with ``ld >= rows``: entries N(0, 1) * 2**e
    with e ~ Uniform int [-s, s] per scalar; padding rows hold NaN."""
    ld = rows if ld is None else ld
    assert ld >= rows
    g = _rng(seed)
    x = g.standard_normal((rows, cols), dtype=np.float64)
    if s > 0:
        x = x * np.exp2(g.integers(-s, s + 1, size=(rows, cols)))
    out = np.full((ld, cols), np.nan, dtype=np.float32, order="F")
    out[:rows, :] = x.astype(np.float32)
    return out


def uniform_operand(rows: int, cols: int, seed) -> np.ndarray:
    """Column-major complex64 matrix with parts ~ U(-1, 1) (Section 3 unit test)."""
    g = _rng(seed)
    re = g.uniform(-1.0, 1.0, size=(rows, cols))
    im = g.uniform(-1.0, 1.0, size=(rows, cols))
    return np.asfortranarray((re + 1j * im).astype(np.complex64))


def line_scaled_operand(rows: int, cols: int, s: int, axis: int, seed,
                        ld: int | None = None) -> np.ndarray:
    """Column-major complex64 matrix whose rows (axis 0) or columns (axis 1)
    each carry one random binade: parts ~ N(0, 1) * 2**e_line with
    e_line ~ Uniform int [-s, s] per line, drawn once for the line's real and
    imaginary parts alike.  Padding rows (ld > rows) hold NaN."""
    ld = rows if ld is None else ld
    assert ld >= rows
    g = _rng(seed)
    re = g.standard_normal((rows, cols), dtype=np.float64)
    im = g.standard_normal((rows, cols), dtype=np.float64)
    e = g.integers(-s, s + 1, size=rows if axis == 0 else cols)
    f = np.exp2(e)[:, None] if axis == 0 else np.exp2(e)[None, :]
    out = np.full((ld, cols), np.nan + 1j * np.nan, dtype=np.complex64, order="F")
    out[:rows, :] = ((re + 1j * im) * f).astype(np.complex64)
    return out


def typed_matrix(rows: int, cols: int, kind: int, seed) -> np.ndarray:
    """Type-1/2/3 element initialisation of Section 5.2 (complex64, column-major).

    Type-1: parts ~ N(0, 1e-4) read as variance 1e-4 (standard deviation 1e-2).
    Type-2: Type-1 scaled by 1e-6.
    Type-3: Type-2 with 10 to 20 randomly chosen elements set to 1.
    """
    g = _rng(seed)
    re = g.normal(0.0, 1e-2, size=(rows, cols))
    im = g.normal(0.0, 1e-2, size=(rows, cols))
    x = re + 1j * im
    if kind >= 2:
        x = x * 1e-6
    if kind >= 3:
        cnt = int(g.integers(10, 21))
        flat = g.choice(rows * cols, size=cnt, replace=False)
        xf = x.reshape(-1, order="F")
        xf[flat] = 1.0
        x = xf.reshape(rows, cols, order="F")
    return np.asfortranarray(x.astype(np.complex64))


# ---------------------------------------------------------------------------
# Random quantum circuits
# ---------------------------------------------------------------------------

def _sqrt_pauli(p: np.ndarray) -> np.ndarray:
    # For an involutory Hermitian P, (1+i)/2 * (I - iP) squares to P.
    return (1 + 1j) / 2 * (np.eye(2) - 1j * p)


_X = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_Y = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_W = (_X + _Y) / np.sqrt(2.0)

#: The single-qubit gate set {sqrt(X), sqrt(Y), sqrt(W)}, W = (X + Y)/sqrt(2).
SQRT_GATES = {
    "sqrtX": _sqrt_pauli(_X),
    "sqrtY": _sqrt_pauli(_Y),
    "sqrtW": _sqrt_pauli(_W),
}
_SQRT_NAMES = ("sqrtX", "sqrtY", "sqrtW")


def _cos_sin(theta: float) -> Tuple[float, float]:
    """cos and sin of theta, evaluated on arguments reduced against pi/2 and
    pi so that a quarter or half turn gives an exact zero.  np.cos(np.pi / 2)
    is 6.1e-17, the rounding error of the double nearest pi/2, not a
    property of the gate: left in, it makes every "zero" of fSim(pi/2, .) a
    tiny nonzero that spreads through a network's intermediates."""
    theta = float(theta)
    c = np.sin(np.pi / 2 - abs(theta))
    s = np.sin(theta) if abs(theta) <= np.pi / 2 else np.sin(np.copysign(np.pi, theta) - theta)
    return float(c), float(s)


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) in the basis |00>, |01>, |10>, |11> (complex128)."""
    c, s = _cos_sin(theta)
    return np.array(
        [
            [1, 0, 0, 0],
            [0, c, -1j * s, 0],
            [0, -1j * s, c, 0],
            [0, 0, 0, np.exp(-1j * phi)],
        ],
        dtype=np.complex128,
    )


@dataclass
class Gate:
    """One gate: ``qubits`` it acts on, its unitary ``matrix`` (2^k x 2^k,
    complex128, row index = output basis state), and for fSim gates the
    ``params`` (theta, phi).  Basis ordering of a two-qubit gate is
    ``2*b(qubits[0]) + b(qubits[1])``."""

    name: str
    qubits: Tuple[int, ...]
    matrix: np.ndarray
    params: Tuple[float, ...] = ()


@dataclass
class Circuit:
    n_qubits: int
    gates: List[Gate] = field(default_factory=list)
    rows: int = 0
    cols: int = 0
    depth: int = 0

    def fsim_indices(self) -> List[int]:
        return [i for i, g in enumerate(self.gates) if g.name == "fsim"]


def grid_edges(rows: int, cols: int, pattern: int) -> List[Tuple[int, int]]:
    """Nearest-neighbour edges of one of four alternating patterns on a
    rows x cols grid (qubit index r*cols + c): 0 horizontal even, 1 horizontal
    odd, 2 vertical even, 3 vertical odd."""
    e = []
    if pattern in (0, 1):
        for r in range(rows):
            for c in range(pattern, cols - 1, 2):
                e.append((r * cols + c, r * cols + c + 1))
    else:
        for r in range(pattern - 2, rows - 1, 2):
            for c in range(cols):
                e.append((r * cols + c, (r + 1) * cols + c))
    return e


def random_grid_circuit(
    rows: int,
    cols: int,
    depth: int,
    seed,
    theta: float | None = np.pi / 2,
    phi: float | None = np.pi / 6,
    param_seed=None,
) -> Circuit:
    """Random grid circuit: ``depth`` cycles, each a layer of single-qubit
    gates drawn uniformly and independently from {sqrt(X), sqrt(Y), sqrt(W)}
    on every qubit, then fSim gates on the edges of pattern ``cycle % 4``.

    With ``theta``/``phi`` None, every fSim gets its own (theta, phi) drawn
    from Uniform[0, pi] with ``param_seed``.
    """
    n = rows * cols
    g = _rng(seed)
    pg = _rng(param_seed) if (theta is None or phi is None) else None
    circ = Circuit(n_qubits=n, rows=rows, cols=cols, depth=depth)
    for cyc in range(depth):
        choice = g.integers(0, 3, size=n)
        for q in range(n):
            name = _SQRT_NAMES[int(choice[q])]
            circ.gates.append(Gate(name, (q,), SQRT_GATES[name].copy()))
        for (a, b) in grid_edges(rows, cols, cyc % 4):
            if pg is not None:
                th, ph = (float(v) for v in pg.uniform(0.0, np.pi, size=2))
            else:
                th, ph = float(theta), float(phi)
            circ.gates.append(Gate("fsim", (a, b), fsim(th, ph), (th, ph)))
    return circ


def random_bitstrings(n_qubits: int, count: int, seed) -> np.ndarray:
    """``count`` random bitstrings as a (count, n_qubits) uint8 array;
    column q is the bit of qubit q."""
    g = _rng(seed)
    return g.integers(0, 2, size=(count, n_qubits), dtype=np.uint8)


def with_params(circ: Circuit, params: Sequence[Tuple[float, float]]) -> Circuit:
    """Copy of ``circ`` whose fSim gates take the given (theta, phi) list."""
    out = Circuit(circ.n_qubits, [], circ.rows, circ.cols, circ.depth)
    it = iter(params)
    for gt in circ.gates:
        if gt.name == "fsim":
            th, ph = next(it)
            out.gates.append(Gate("fsim", gt.qubits, fsim(th, ph), (float(th), float(ph))))
        else:
            out.gates.append(Gate(gt.name, gt.qubits, gt.matrix.copy(), gt.params))
    return out
