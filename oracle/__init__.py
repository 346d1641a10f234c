"""Plain, slow CPU oracle (FP64) for the emulated-CGEMM tensor-network path.

TEST INFRASTRUCTURE.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It shares no code with the CUDA library (``paper_2303_08989_gb300``)
and never imports it; both sides only share the seeded generators of
``qcs_inputs``.

What it computes, each following a passage of the paper (Ootomo et al. 2023):

* ``cgemm``: complex GEMM by the textbook triple loop (Section 3, the FP64
  reference of the CGEMM unit test), and a row-sampled OpenMP variant for
  large shapes.  ``sgemm`` / ``tcec_sgemm`` / ``exp_stats_real``: the same
  for real matrices (the SGEMM that Section 2.1 emulates).
* ``split`` / ``f32_to_f16`` / ``f32_to_tf32``: the hi/lo split of Eq. 1
  (Section 2.1) with IEEE round-to-nearest-even restated in C.
* ``exp_stats`` / ``stats_summary`` / ``select_mode``: the exponent statistics
  and the mode-selection rule of Section 4.1, and the size rule of
  Section 4.3.
* ``tcec_cgemm``: the emulated product of Eq. 1 with the complex expansion of
  Section 3, evaluated exactly in FP64; ``tcec_cgemm_3m`` the same with
  Gauss's three real products (a variant beyond the paper).
* ``rowcol_stats`` / ``select_rowcol`` / ``tcec_cgemm_rowcol``: Section 4.1's
  per-matrix scaling applied to every row of op(A) and column of op(B) (a
  variant beyond the paper), built from ``exp_stats`` / ``stats_summary`` per
  line and ``tcec_cgemm`` of the scaled operands.
* ``statevector`` / ``circuit_tn`` / ``amplitude``: the state-vector method and
  the tensor-network representation of a circuit (Section 2.2), the amplitude
  <x|U|0> of Eq. prob_dist (Section 5.3), with slicing (Section 5.3).
* ``loss_and_grad`` / ``fd_grad``: the FP64 gradient of sum_x log|a_x|^2 with
  respect to the fSim parameters (adjoint state vector and central
  differences).  The paper has no gradient; this is the reference for the
  differentiated contraction.

Parity pins that do not depend on this code live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qcs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Mode codes (the oracle's own numbering; they coincide with the C ABI's
# qcs_mode_t values so that tests can compare them directly).
MODE_AUTO, MODE_FP16X, MODE_FP16X_SCALED, MODE_TF32X, MODE_FP32, MODE_BF16X3 = range(6)
MODE_NAMES = {
    MODE_AUTO: "auto",
    MODE_FP16X: "fp16x",
    MODE_FP16X_SCALED: "fp16x_scaled",
    MODE_TF32X: "tf32x",
    MODE_FP32: "fp32",
    MODE_BF16X3: "bf16x3",
}
# FP16 emulation with one power-of-two scale per row of op(A) and per column
# of op(B) (a variant beyond the paper; the value the C ABI reports for it)
MODE_FP16X_ROWCOL = 6
MODE_NAMES[MODE_FP16X_ROWCOL] = "fp16x_rowcol"
OP_N, OP_T, OP_C = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile qcs_oracle.c with gcc (OpenMP) into oracle/_build/liboracle.so."""
    with _lock:
        os.makedirs(_BUILD, exist_ok=True)
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
            tmp = _SO + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
            subprocess.check_call(cmd)
            os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I = ctypes.c_int
        lib.oracle_cgemm_naive.argtypes = [I, I, I64, I64, I64, P, P, I64, P, I64, P, P, I64, P]
        lib.oracle_cgemm_rows.argtypes = [I, I, I64, I64, I64, P, P, I64, P, I64, P, P, I64, P, I64, P]
        lib.oracle_tcec_cgemm.argtypes = [I, I, I, I, I, I64, I64, I64, P, P, I64, P, I64, P, P, I64, P]
        D = ctypes.c_double
        lib.oracle_sgemm_rows.argtypes = [I, I, I64, I64, I64, D, P, I64, P, I64, D, P, I64, P,
                                          I64, P]
        lib.oracle_tcec_sgemm.argtypes = [I, I, I, I, I, I64, I64, I64, D, P, I64, P, I64, D, P,
                                          I64, P]
        lib.oracle_exp_stats_real.argtypes = [I64, I64, P, I64, P, P]
        lib.oracle_tcec_cgemm_3m.argtypes = [I, I, I, I, I, I64, I64, I64, P, P, I64, P, I64, P,
                                             P, I64, P]
        lib.oracle_f32_to_f16.argtypes = [ctypes.c_float]
        lib.oracle_f32_to_f16.restype = ctypes.c_uint16
        lib.oracle_f16_to_f32.argtypes = [ctypes.c_uint16]
        lib.oracle_f16_to_f32.restype = ctypes.c_float
        lib.oracle_f32_to_tf32.argtypes = [ctypes.c_float]
        lib.oracle_f32_to_tf32.restype = ctypes.c_float
        lib.oracle_f32_to_bf16.argtypes = [ctypes.c_float]
        lib.oracle_f32_to_bf16.restype = ctypes.c_float
        lib.oracle_split.argtypes = [I, I, I64, P, P, P]
        lib.oracle_exp_stats.argtypes = [I64, I64, P, I64, P, P]
        lib.oracle_contract_pair.argtypes = [I, P, P, P, I, P, P, P, I, P, P]
        lib.oracle_contract_pair.restype = I
        lib.oracle_num_threads.restype = I
        lib.oracle_sv_apply1.argtypes = [I, P, I, P]
        lib.oracle_sv_apply2.argtypes = [I, P, I, I, P]
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_L().oracle_num_threads())


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _mat_view(X: np.ndarray):
    """Column-major complex64 matrix -> (array, leading dim)."""
    assert X.dtype == np.complex64
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    assert X.flags.f_contiguous, "column-major (Fortran-ordered) input expected"
    return X, X.shape[0]


def _op_shape(X: np.ndarray, op: int, rows: int, cols: int):
    return (rows, cols) if op == OP_N else (cols, rows)


# ---------------------------------------------------------------------------
# CGEMM
# ---------------------------------------------------------------------------

def cgemm(opA: int, opB: int, m: int, n: int, k: int, alpha, A, B, beta=0.0, C=None,
          rows: Optional[Sequence[int]] = None) -> np.ndarray:
    """alpha * op(A) op(B) + beta * C in complex128 (Section 3 reference).

    A, B, C are Fortran-ordered complex64 arrays (their leading dimension is
    their first extent).  With ``rows`` given, only those output rows are
    computed (OpenMP, row-sampled); the result is then len(rows) x n.
    """
    A, lda = _mat_view(A)
    B, ldb = _mat_view(B)
    al = np.array([complex(alpha).real, complex(alpha).imag], dtype=np.float64)
    be = np.array([complex(beta).real, complex(beta).imag], dtype=np.float64)
    if C is not None:
        C, ldc = _mat_view(C)
        cp = _ptr(C)
    else:
        ldc, cp = 1, None
    if rows is None:
        out = np.zeros((m, n), dtype=np.complex128, order="F")
        _L().oracle_cgemm_naive(opA, opB, m, n, k, _ptr(al), _ptr(A), lda, _ptr(B), ldb,
                                _ptr(be), cp, ldc, _ptr(out))
        return out
    r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
    out = np.zeros((len(r), n), dtype=np.complex128, order="F")
    rc = _L().oracle_cgemm_rows(opA, opB, m, n, k, _ptr(al), _ptr(A), lda, _ptr(B), ldb,
                                _ptr(be), cp, ldc, _ptr(r), len(r), _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_cgemm_rows failed")
    return out


def tcec_cgemm(kind: int, sA: int, sB: int, opA: int, opB: int, m: int, n: int, k: int,
               alpha, A, B, beta=0.0, C=None) -> np.ndarray:
    """Exact (FP64) value of the emulated product, Eq. 1 + Section 3.
    kind: 0 FP16, 1 TF32, 2 BF16."""
    A, lda = _mat_view(A)
    B, ldb = _mat_view(B)
    al = np.array([complex(alpha).real, complex(alpha).imag], dtype=np.float64)
    be = np.array([complex(beta).real, complex(beta).imag], dtype=np.float64)
    if C is not None:
        C, ldc = _mat_view(C)
        cp = _ptr(C)
    else:
        ldc, cp = 1, None
    out = np.zeros((m, n), dtype=np.complex128, order="F")
    rc = _L().oracle_tcec_cgemm(kind, sA, sB, opA, opB, m, n, k, _ptr(al), _ptr(A), lda, _ptr(B),
                                ldb, _ptr(be), cp, ldc, _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_tcec_cgemm failed")
    return out


def _mat_view_real(X: np.ndarray):
    """Column-major float32 matrix -> (array, leading dim)."""
    assert X.dtype == np.float32
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    assert X.flags.f_contiguous, "column-major (Fortran-ordered) input expected"
    return X, X.shape[0]


def sgemm(opA: int, opB: int, m: int, n: int, k: int, alpha, A, B, beta=0.0, C=None,
          rows: Optional[Sequence[int]] = None) -> np.ndarray:
    """alpha * op(A) op(B) + beta * C in float64 for real matrices: the SGEMM
    that Section 2.1 emulates, by the textbook sum (OpenMP over columns).

    A, B, C are Fortran-ordered float32 arrays; op T and C both transpose.
    With ``rows`` only those output rows are computed (len(rows) x n)."""
    A, lda = _mat_view_real(A)
    B, ldb = _mat_view_real(B)
    if C is not None:
        C, ldc = _mat_view_real(C)
        cp = _ptr(C)
    else:
        ldc, cp = 1, None
    if rows is None:
        rp, nr = None, m
    else:
        r = np.ascontiguousarray(np.asarray(rows, dtype=np.int64))
        rp, nr = _ptr(r), len(r)
    out = np.zeros((nr, n), dtype=np.float64, order="F")
    _L().oracle_sgemm_rows(opA, opB, m, n, k, float(alpha), _ptr(A), lda, _ptr(B), ldb,
                           float(beta), cp, ldc, rp, nr, _ptr(out))
    return out


def tcec_sgemm(kind: int, sA: int, sB: int, opA: int, opB: int, m: int, n: int, k: int,
               alpha, A, B, beta=0.0, C=None) -> np.ndarray:
    """Exact (FP64) value of the emulated real product of Eq. 1.
    kind: 0 FP16, 1 TF32, 2 BF16."""
    A, lda = _mat_view_real(A)
    B, ldb = _mat_view_real(B)
    if C is not None:
        C, ldc = _mat_view_real(C)
        cp = _ptr(C)
    else:
        ldc, cp = 1, None
    out = np.zeros((m, n), dtype=np.float64, order="F")
    rc = _L().oracle_tcec_sgemm(kind, sA, sB, opA, opB, m, n, k, float(alpha), _ptr(A), lda,
                                _ptr(B), ldb, float(beta), cp, ldc, _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_tcec_sgemm failed")
    return out


def tcec_cgemm_3m(kind: int, sA: int, sB: int, opA: int, opB: int, m: int, n: int, k: int,
                  alpha, A, B, beta=0.0, C=None) -> np.ndarray:
    """Exact (FP64) value of Gauss's three-product form of the emulated
    complex product: T1 = Ar Br, T2 = Ai Bi, T3 = (Ar + Ai)(Br + Bi), each an
    Eq. 1 compensated product (operand sums in binary32, scaled by one binade
    less for FP16), Re = T1 - T2, Im = T3 - T1 - T2.  A variant beyond the
    paper.  kind: 0 FP16, 1 TF32, 2 BF16."""
    A, lda = _mat_view(A)
    B, ldb = _mat_view(B)
    al = np.array([complex(alpha).real, complex(alpha).imag], dtype=np.float64)
    be = np.array([complex(beta).real, complex(beta).imag], dtype=np.float64)
    if C is not None:
        C, ldc = _mat_view(C)
        cp = _ptr(C)
    else:
        ldc, cp = 1, None
    out = np.zeros((m, n), dtype=np.complex128, order="F")
    rc = _L().oracle_tcec_cgemm_3m(kind, sA, sB, opA, opB, m, n, k, _ptr(al), _ptr(A), lda,
                                   _ptr(B), ldb, _ptr(be), cp, ldc, _ptr(out))
    if rc != 0:
        raise MemoryError("oracle_tcec_cgemm_3m failed")
    return out


def rel_fro_error(C: np.ndarray, C64: np.ndarray) -> float:
    """Relative Frobenius error ||C - C64||_F / ||C64||_F (Section 3)."""
    C = np.asarray(C, dtype=np.complex128)
    C64 = np.asarray(C64, dtype=np.complex128)
    den = np.linalg.norm(C64)
    return float(np.linalg.norm(C - C64) / den) if den > 0 else float(np.linalg.norm(C - C64))


# ---------------------------------------------------------------------------
# Low-precision conversions and the split (Eq. 1)
# ---------------------------------------------------------------------------

def f32_to_f16_bits(x: float) -> int:
    return int(_L().oracle_f32_to_f16(ctypes.c_float(x)))


def f16_bits_to_f32(h: int) -> float:
    return float(_L().oracle_f16_to_f32(ctypes.c_uint16(h)))


def f32_to_tf32(x: float) -> float:
    return float(_L().oracle_f32_to_tf32(ctypes.c_float(x)))


def f32_to_bf16(x: float) -> float:
    return float(_L().oracle_f32_to_bf16(ctypes.c_float(x)))


def split(kind: int, s: int, x: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """hi, lo of Eq. 1 for every binary32 scalar in x, after scaling by 2^s.
    kind: 0 FP16, 1 TF32, 2 BF16.  Returns binary32 arrays holding the
    low-precision values."""
    xf = np.ascontiguousarray(np.asarray(x, dtype=np.float32).reshape(-1))
    hi = np.empty_like(xf)
    lo = np.empty_like(xf)
    _L().oracle_split(kind, int(s), xf.size, _ptr(xf), _ptr(hi), _ptr(lo))
    return hi.reshape(np.shape(x)), lo.reshape(np.shape(x))


# ---------------------------------------------------------------------------
# Exponent statistics and mode selection (Section 4.1, Section 4.3)
# ---------------------------------------------------------------------------

def exp_stats(X: np.ndarray, rows: Optional[int] = None, cols: Optional[int] = None):
    """Histogram of floor(log2|x|) + 127 over all real and imaginary scalars
    (bin 0: subnormal, bin 255: Inf/NaN; zeros apart).  Returns (hist, n_zero)."""
    X, ldx = _mat_view(X)
    rows = X.shape[0] if rows is None else rows
    cols = X.shape[1] if cols is None else cols
    hist = np.zeros(256, dtype=np.int64)
    nz = np.zeros(1, dtype=np.int64)
    _L().oracle_exp_stats(rows, cols, _ptr(X), ldx, _ptr(hist), _ptr(nz))
    return hist, int(nz[0])


def exp_stats_real(X: np.ndarray):
    """exp_stats over the scalars of a Fortran-ordered float32 matrix."""
    X, ldx = _mat_view_real(X)
    hist = np.zeros(256, dtype=np.int64)
    nz = np.zeros(1, dtype=np.int64)
    _L().oracle_exp_stats_real(X.shape[0], X.shape[1], _ptr(X), ldx, _ptr(hist), _ptr(nz))
    return hist, int(nz[0])


FP16_EMIN = -14   # least normal FP16 exponent: the "minimum value of FP16"
FP16_ETOP = 14    # the exponent the scaled maximum is moved to
WINDOW = FP16_ETOP - FP16_EMIN  # 28: binades below the maximum that survive


def stats_summary(hist: np.ndarray, n_zero: int) -> Dict[str, int]:
    """N, N1, N2, e_max of Section 4.1 from an exponent histogram.

    Readings taken where the paper is silent: zeros are representable in
    every mode and enter neither count nor total; "larger than the minimum
    value of FP16" means e >= -14 (least normal); the shifted window is
    [e_max - 28, e_max]; subnormal binary32 inputs (bin 0) always count as
    falling outside both windows.
    """
    hist = np.asarray(hist, dtype=np.int64)
    nonfinite = int(hist[255])
    finite = hist[:255]
    nnz = int(finite.sum())
    used = np.nonzero(finite)[0]
    e_max = int(used.max()) - 127 if used.size else None
    under1 = int(finite[: 127 + FP16_EMIN].sum())  # bins with e < -14 (bin 0 included)
    if e_max is None:
        under2 = 0
    else:
        lo_bin = e_max - WINDOW + 127  # bins below lo_bin fall outside the shifted window
        under2 = int(finite[1:max(lo_bin, 1)].sum()) + int(finite[0])
    return {
        "n": nnz + int(n_zero) + nonfinite,
        "nnz": nnz,
        "n_zero": int(n_zero),
        "nonfinite": nonfinite,
        "e_max": e_max,
        "n1": nnz - under1,
        "n2": nnz - under2,
        "under1": under1,
        "under2": under2,
    }


def select_mode(sa: Dict[str, int], sb: Dict[str, int], t: float = 0.0):
    """Mode selection rule of Section 4.1 for one GEMM.

    An operand tolerates FP16TCEC when its underflow count (nonzero scalars
    below 2^-14) is at most t * nnz and, because the tensors here are not
    bounded by 1 (the paper only checks underflow), its maximum exponent is
    at most 14.  It tolerates FP16TCEC with scaling when the count below the
    window shifted so that e_max becomes 14 is at most t * nnz.  Either
    operand failing both -> TF32TCEC; either failing the first -> FP16TCEC
    with scaling (each operand scaled by 2^(14 - e_max)); else FP16TCEC.
    Inf/NaN, or a maximum exponent of 127 (TF32 rounding could overflow),
    route the GEMM to plain FP32.  Returns (mode, sA, sB).
    """
    def ok1(s):
        return s["e_max"] is None or (s["e_max"] <= FP16_ETOP and s["under1"] <= t * s["nnz"])

    def ok2(s):
        return s["under2"] <= t * s["nnz"]

    for s in (sa, sb):
        if s["nonfinite"] > 0 or (s["e_max"] is not None and s["e_max"] >= 127):
            return MODE_FP32, 0, 0
    if not ok2(sa) or not ok2(sb):
        return MODE_TF32X, 0, 0
    if not ok1(sa) or not ok1(sb):
        scl = lambda s: 0 if s["e_max"] is None else FP16_ETOP - s["e_max"]
        return MODE_FP16X_SCALED, scl(sa), scl(sb)
    return MODE_FP16X, 0, 0


# ---------------------------------------------------------------------------
# Per-row / per-column scaling (a variant beyond the paper: Section 4.1's
# per-matrix scaling basis applied to each row of op(A) and column of op(B))
# ---------------------------------------------------------------------------

def _lines(X: np.ndarray, op: int, count: int, k: int, rows_of_op: bool):
    """The lines of op(X) as Fortran column vectors: rows of op(A)
    (rows_of_op) or columns of op(B).  Conjugation is left out: it does not
    change an exponent."""
    X, _ = _mat_view(X)
    out = []
    for i in range(count):
        if rows_of_op:   # row i of op(A): a stored row of A (N) or a stored column
            v = X[i, :k] if op == OP_N else X[:k, i]
        else:            # column j of op(B): a stored column of B (N) or a stored row
            v = X[:k, i] if op == OP_N else X[i, :k]
        out.append(np.asfortranarray(np.asarray(v, dtype=np.complex64).reshape(-1, 1)))
    return out


def rowcol_stats(A: np.ndarray, B: np.ndarray, opA: int, opB: int, m: int, n: int, k: int):
    """Per-line statistics of per-row / per-column scaling, each line taken as
    a matrix of its own through exp_stats and stats_summary (Section 4.1):
    the biased largest exponent of every row of op(A) (m) and column of
    op(B) (n), -1 for a line without a nonzero finite scalar, and the counts
    [under A, nonzero A, under B, nonzero B], "under" being the Stage 2 count
    of each line (below its window [e_max - 28, e_max]) summed over the lines."""
    res = []
    for X, op, cnt, rows_of_op in ((A, opA, m, True), (B, opB, n, False)):
        emax, under, nnz = [], 0, 0
        for v in _lines(X, op, cnt, k, rows_of_op):
            st = stats_summary(*exp_stats(v))
            emax.append(-1 if st["e_max"] is None else st["e_max"] + 127)
            under += st["under2"]
            nnz += st["nnz"]
        res.append((np.array(emax, dtype=np.int64), under, nnz))
    (ea, ua, na), (eb, ub, nb) = res
    return ea, eb, np.array([ua, na, ub, nb], dtype=np.int64)


def line_scale(emax_biased: int) -> int:
    """Scale exponent of a line: 14 - e_max moves its largest magnitude to
    [2^14, 2^15) as for a whole matrix in Section 4.1; 0 for a line without
    a nonzero finite scalar."""
    return 0 if emax_biased < 0 else FP16_ETOP - (int(emax_biased) - 127)


def select_rowcol(sa: Dict[str, int], sb: Dict[str, int], counts, t: float = 0.0):
    """Section 4.1's rule, then per-row / per-column scaling where the rule
    gives up on FP16 (TF32X): FP16 emulation with line scales when each
    operand's summed Stage 2 count over its lines is at most t times its
    nonzero count.  Returns (mode, sA, sB)."""
    mode = select_mode(sa, sb, t)
    if mode[0] == MODE_TF32X and counts[0] <= t * counts[1] and counts[2] <= t * counts[3]:
        return MODE_FP16X_ROWCOL, 0, 0
    return mode


def tcec_cgemm_rowcol(emaxA, emaxB, opA: int, opB: int, m: int, n: int, k: int, alpha, A, B,
                      beta=0.0, C=None) -> np.ndarray:
    """Exact (FP64) value of FP16 emulation with line scales: row i of op(A)
    multiplied by 2^sA_i and column j of op(B) by 2^sB_j in binary32 (the
    scaled matrices as stored), the Eq. 1 / Section 3 product of those
    (tcec_cgemm, FP16, no further scaling), element (i, j) multiplied back by
    2^-(sA_i + sB_j), then alpha and beta."""
    A32, _ = _mat_view(A)
    B32, _ = _mat_view(B)
    sa = [line_scale(e) for e in emaxA]
    sb = [line_scale(e) for e in emaxB]

    def scaled(X, op, scales, rows_of_op):
        Y = np.array(X, dtype=np.complex64, order="F", copy=True)
        for i, s in enumerate(scales):
            if rows_of_op:
                sl = (i, slice(0, k)) if op == OP_N else (slice(0, k), i)
            else:
                sl = (slice(0, k), i) if op == OP_N else (i, slice(0, k))
            v = Y[sl]
            re = np.ldexp(v.real.astype(np.float32), np.int32(s)).astype(np.float32)
            im = np.ldexp(v.imag.astype(np.float32), np.int32(s)).astype(np.float32)
            Y[sl] = re + 1j * im
        return Y

    As = scaled(A32, opA, sa, True)
    Bs = scaled(B32, opB, sb, False)
    prod = tcec_cgemm(0, 0, 0, opA, opB, m, n, k, 1.0, As, Bs)
    unscale = np.ldexp(1.0, -(np.array(sa)[:, None] + np.array(sb)[None, :]))
    out = complex(alpha) * (prod * unscale)
    if C is not None:
        C64, _ = _mat_view(C)
        out = out + complex(beta) * C64[:m, :n].astype(np.complex128)
    return np.asfortranarray(out)


def size_rule(m: int, n: int, k: int) -> Optional[int]:
    """Section 4.3: min(m, n, k) >= 2048 -> automatic selection (None);
    >= 512 -> TF32TCEC; else plain FP32."""
    s = min(m, n, k)
    if s >= 2048:
        return None
    if s >= 512:
        return MODE_TF32X
    return MODE_FP32


def emulated_kind(mode: int) -> int:
    return {MODE_FP16X: 0, MODE_FP16X_SCALED: 0, MODE_TF32X: 1, MODE_BF16X3: 2}[mode]


# ---------------------------------------------------------------------------
# Circuits: state vector and tensor network (Section 2.2, Section 5.3)
# ---------------------------------------------------------------------------

def apply_gate(psi: np.ndarray, mat: np.ndarray, qubits: Sequence[int]) -> np.ndarray:
    """psi has shape (2,)*n, axis q = qubit q.  Returns G psi."""
    k = len(qubits)
    g = np.asarray(mat, dtype=np.complex128).reshape((2,) * (2 * k))
    out = np.tensordot(g, psi, axes=(list(range(k, 2 * k)), list(qubits)))
    return np.moveaxis(out, list(range(k)), list(qubits))


def statevector(circ, gates=None) -> np.ndarray:
    """Apply every gate in order to |0...0> (state-vector method, Section 1)."""
    n = circ.n_qubits
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[(0,) * n] = 1.0
    for g in (circ.gates if gates is None else gates):
        psi = apply_gate(psi, g.matrix, g.qubits)
    return psi


def statevector_inplace(circ) -> np.ndarray:
    """The same state as ``statevector``, computed in place in C (one FP64
    vector of 2^n amplitudes, no copies), for circuits up to ~30 qubits.
    Returns a flat complex128 array in numpy C order over qubits 0..n-1."""
    n = circ.n_qubits
    psi = np.zeros(2 ** n, dtype=np.complex128)
    psi[0] = 1.0
    lib = _L()
    for g in circ.gates:
        m = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128))
        if len(g.qubits) == 1:
            lib.oracle_sv_apply1(n, _ptr(psi), int(g.qubits[0]), _ptr(m))
        else:
            lib.oracle_sv_apply2(n, _ptr(psi), int(g.qubits[0]), int(g.qubits[1]), _ptr(m))
    return psi


def bit_index(bits) -> int:
    """Basis index of a bitstring (qubit 0 most significant)."""
    idx = 0
    for b in bits:
        idx = 2 * idx + int(b)
    return idx


def sv_amplitudes(circ, bitstrings: np.ndarray) -> np.ndarray:
    psi = statevector(circ)
    return np.array([psi[tuple(int(b) for b in x)] for x in bitstrings], dtype=np.complex128)


def circuit_tn(circ, bits: Optional[Sequence[int]] = None):
    """Tensor network of <x|U|0> (Section 2.2): |0> as rank-1 tensors, each
    k-qubit gate as a rank-2k tensor (output legs first), <x| as rank-1
    tensors, wires as shared labels.  With bits None the output legs stay
    open; the returned output labels are then the final wire of each qubit.
    Returns (list of (array, labels), output_labels)."""
    n = circ.n_qubits
    tensors: List[Tuple[np.ndarray, List[int]]] = []
    wire = list(range(n))
    nxt = n
    for q in range(n):
        tensors.append((np.array([1.0, 0.0], dtype=np.complex128), [q]))
    for g in circ.gates:
        k = len(g.qubits)
        new = list(range(nxt, nxt + k))
        nxt += k
        t = np.asarray(g.matrix, dtype=np.complex128).reshape((2,) * (2 * k))
        tensors.append((t, new + [wire[q] for q in g.qubits]))
        for i, q in enumerate(g.qubits):
            wire[q] = new[i]
    if bits is None:
        return tensors, [wire[q] for q in range(n)]
    for q in range(n):
        v = np.zeros(2, dtype=np.complex128)
        v[int(bits[q])] = 1.0
        tensors.append((v, [wire[q]]))
    return tensors, []


def contract_pair_loops(A, la, B, lb, lc) -> np.ndarray:
    """Nested-loop contraction in C (no GEMM)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    B = np.ascontiguousarray(B, dtype=np.complex128)
    dims = {}
    for t, ls in ((A, la), (B, lb)):
        for d, l in zip(t.shape, ls):
            dims[l] = d
    shape_c = tuple(dims[l] for l in lc)
    C = np.zeros(shape_c, dtype=np.complex128)
    ia = np.array(la, dtype=np.int32)
    ib = np.array(lb, dtype=np.int32)
    ic = np.array(lc, dtype=np.int32) if len(lc) else np.zeros(1, dtype=np.int32)
    da = np.array(A.shape, dtype=np.int64) if A.ndim else np.zeros(1, dtype=np.int64)
    db = np.array(B.shape, dtype=np.int64) if B.ndim else np.zeros(1, dtype=np.int64)
    rc = _L().oracle_contract_pair(len(la), _ptr(ia), _ptr(da), _ptr(A), len(lb), _ptr(ib),
                                   _ptr(db), _ptr(B), len(lc), _ptr(ic), _ptr(C))
    if rc != 0:
        raise ValueError(f"oracle_contract_pair failed ({rc})")
    return C


def contract_pair_np(A, la, B, lb, lc) -> np.ndarray:
    """The same contraction with numpy.tensordot (a library matmul) as the step."""
    shared = [l for l in la if l in lb and l not in lc]
    ax_a = [la.index(l) for l in shared]
    ax_b = [lb.index(l) for l in shared]
    out = np.tensordot(A, B, axes=(ax_a, ax_b))
    rest = [l for l in la if l not in shared] + [l for l in lb if l not in shared]
    # labels present in both and kept in the output (hyperedges) are not used here
    assert len(rest) == len(set(rest)), "hyperedges are not supported by contract_pair_np"
    perm = [rest.index(l) for l in lc]
    return np.transpose(out, perm) if perm else out


def greedy_order(tensors, output_labels) -> List[Tuple[int, int]]:
    """The oracle's own contraction order: repeatedly contract the connected
    pair minimising size(result) - size(a) - size(b) (ties: lowest
    positions).  Returns pairs of positions in a growing list (each result
    is appended at the end)."""
    from collections import defaultdict

    labs = [list(ls) for _, ls in tensors]
    dims = {}
    for t, ls in tensors:
        for d, l in zip(np.shape(t), ls):
            dims[l] = d
    count = defaultdict(int)
    where = defaultdict(set)
    for i, ls in enumerate(labs):
        for l in ls:
            count[l] += 1
            where[l].add(i)
    for l in output_labels:
        count[l] += 1
    alive = set(range(len(labs)))

    def size(ls):
        s = 1
        for l in ls:
            s *= dims[l]
        return s

    def result(i, j):
        si = set(labs[i])
        sj = set(labs[j])
        return [l for l in dict.fromkeys(labs[i] + labs[j])
                if not (l in si and l in sj and count[l] == 2)]

    order = []
    while len(alive) > 1:
        best = None
        seen = set()
        for l, ws in where.items():
            if len(ws) < 2:
                continue
            ws = sorted(ws)
            for a in range(len(ws)):
                for b in range(a + 1, len(ws)):
                    i, j = ws[a], ws[b]
                    if (i, j) in seen:
                        continue
                    seen.add((i, j))
                    res = result(i, j)
                    key = (size(res) - size(labs[i]) - size(labs[j]), i, j)
                    if best is None or key < best[0]:
                        best = (key, i, j, res)
        if best is None:  # disconnected components: take the two lowest positions
            i, j = sorted(alive)[:2]
            res = result(i, j)
        else:
            _, i, j, res = best
        order.append((i, j))
        for u in (i, j):
            for l in labs[u]:
                count[l] -= 1
                where[l].discard(u)
            alive.discard(u)
        labs.append(res)
        nu = len(labs) - 1
        for l in res:
            count[l] += 1
            where[l].add(nu)
        alive.add(nu)
    return order


def order_cost(tensors, order, output_labels=()) -> Tuple[float, int]:
    """(flops of a pairwise order with 8 flops per complex multiply-add,
    log2 of the largest intermediate)."""
    from collections import Counter

    dims = {}
    for t, ls in tensors:
        for d, l in zip(np.shape(t), ls):
            dims[l] = d
    labs = [list(ls) for _, ls in tensors]
    cnt = Counter(l for ls in labs for l in ls)
    for l in output_labels:
        cnt[l] += 1
    flops, big = 0.0, 0
    for i, j in order:
        a, b = labs[i], labs[j]
        sh = set(a) & set(b)
        res = [l for l in dict.fromkeys(a + b) if not (l in sh and cnt[l] == 2)]
        flops += 8.0 * float(np.prod([dims[l] for l in set(a) | set(b)]))
        big = max(big, int(round(sum(np.log2(dims[l]) for l in res))))
        for l in a + b:
            cnt[l] -= 1
        for l in res:
            cnt[l] += 1
        labs.append(res)
    return flops, big


def random_greedy_order(tensors, output_labels, seeds=range(8)) -> List[Tuple[int, int]]:
    """Best (fewest flops) of several randomised greedy orders: like
    ``greedy_order`` but each candidate's cost is multiplied by a random
    factor in [1, 1.5) drawn per pair from a seeded generator, which breaks
    the many ties differently per seed."""
    from collections import defaultdict
    import heapq

    best = None
    for seed in seeds:
        rng = np.random.default_rng(seed)
        labs = [list(ls) for _, ls in tensors]
        dims = {}
        for t, ls in tensors:
            for d, l in zip(np.shape(t), ls):
                dims[l] = d
        count = defaultdict(int)
        where = defaultdict(set)
        for i, ls in enumerate(labs):
            for l in ls:
                count[l] += 1
                where[l].add(i)
        for l in output_labels:
            count[l] += 1
        alive = set(range(len(labs)))

        def size(ls):
            return float(np.prod([dims[l] for l in ls])) if ls else 1.0

        def result(i, j):
            si, sj = set(labs[i]), set(labs[j])
            return [l for l in dict.fromkeys(labs[i] + labs[j])
                    if not (l in si and l in sj and count[l] == 2)]

        heap = []

        def push(i, j):
            r = result(i, j)
            c = (size(r) - size(labs[i]) - size(labs[j])) * (1.0 + 0.5 * rng.random())
            heapq.heappush(heap, (c, i, j))

        for l, ws in list(where.items()):
            ws = sorted(ws)
            for a in range(len(ws)):
                for b in range(a + 1, len(ws)):
                    push(ws[a], ws[b])
        order = []
        while len(alive) > 1:
            pair = None
            while heap:
                _, i, j = heapq.heappop(heap)
                if i in alive and j in alive:
                    pair = (i, j)
                    break
            if pair is None:
                i, j = sorted(alive)[:2]
            else:
                i, j = pair
            res = result(i, j)
            order.append((i, j))
            for u in (i, j):
                for l in labs[u]:
                    count[l] -= 1
                    where[l].discard(u)
                alive.discard(u)
            labs.append(res)
            nu = len(labs) - 1
            for l in res:
                count[l] += 1
                where[l].add(nu)
            alive.add(nu)
            nb = set()
            for l in res:
                nb |= where[l]
            nb.discard(nu)
            for u in nb:
                push(min(u, nu), max(u, nu))
        cost = order_cost(tensors, order, output_labels)
        if best is None or cost[0] < best[0][0]:
            best = (cost, order)
    return best[1]


def slice_labels_by_weight(tensors, output_labels, order, count: int) -> List[int]:
    """Indices to slice: repeatedly the label that appears in the most of the
    largest intermediates of ``order`` (intermediate sizes recomputed after
    each choice)."""
    chosen: List[int] = []
    for _ in range(count):
        sub = slice_network(tensors, {l: 0 for l in chosen})
        labs = [list(ls) for _, ls in sub]
        from collections import Counter

        cnt = Counter(l for ls in labs for l in ls)
        for l in output_labels:
            cnt[l] += 1
        inter = []
        for i, j in order:
            a, b = labs[i], labs[j]
            sh = set(a) & set(b)
            res = [l for l in dict.fromkeys(a + b) if not (l in sh and cnt[l] == 2)]
            for l in a + b:
                cnt[l] -= 1
            for l in res:
                cnt[l] += 1
            labs.append(res)
            inter.append(res)
        top = max(len(r) for r in inter)
        weight: Dict[int, float] = {}
        for r in inter:
            if len(r) >= top - 2:
                for l in r:
                    if l not in output_labels:
                        weight[l] = weight.get(l, 0.0) + 2.0 ** (len(r) - top)
        chosen.append(min(weight, key=lambda l: (-weight[l], l)))
    return chosen


def contract_network(tensors, output_labels, order=None, use_loops: bool = False) -> np.ndarray:
    """Contract a whole network pairwise in ``order`` (default: greedy_order).
    A label is summed at the step after which no other tensor and not the
    output still carries it."""
    ts = [(np.asarray(t, dtype=np.complex128), list(ls)) for t, ls in tensors]
    if order is None:
        order = greedy_order(ts, output_labels)
    alive = set(range(len(ts)))
    keep = set(output_labels)
    f = contract_pair_loops if use_loops else contract_pair_np
    for (i, j) in order:
        (A, la), (B, lb) = ts[i], ts[j]
        alive -= {i, j}
        others = set()
        for u in alive:
            others |= set(ts[u][1])
        lc = [l for l in dict.fromkeys(la + lb) if not (l in la and l in lb) or l in keep or l in others]
        C = f(A, la, B, lb, lc)
        ts.append((C, lc))
        alive.add(len(ts) - 1)
    (res, lres), = [ts[u] for u in alive]
    perm = [lres.index(l) for l in output_labels]
    return np.transpose(res, perm) if perm else res


def slice_network(tensors, fixed: Dict[int, int]):
    """Fix the labels in ``fixed`` (label -> value) in every tensor that
    carries them (slicing, Section 5.3)."""
    out = []
    for t, ls in tensors:
        idx = tuple(fixed[l] if l in fixed else slice(None) for l in ls)
        out.append((np.asarray(t)[idx], [l for l in ls if l not in fixed]))
    return out


def amplitude(circ, bits, sliced: Sequence[int] = (), order=None) -> complex:
    """<x|U|0> by contracting the network; with ``sliced`` labels, the sum
    over all their values of the sliced networks."""
    tensors, outl = circuit_tn(circ, bits)
    if not sliced:
        return complex(contract_network(tensors, outl, order))
    dims = {}
    for t, ls in tensors:
        for d, l in zip(np.shape(t), ls):
            dims[l] = d
    total = 0.0 + 0.0j
    for val in np.ndindex(*[dims[l] for l in sliced]):
        sub = slice_network(tensors, dict(zip(sliced, val)))
        total += complex(contract_network(sub, outl, order))
    return total


# ---------------------------------------------------------------------------
# Gradient reference: L = sum_x log |a_x|^2 over the fSim parameters
# ---------------------------------------------------------------------------

def _dfsim(theta: float, phi: float):
    c, s = np.cos(theta), np.sin(theta)
    dth = np.zeros((4, 4), dtype=np.complex128)
    dth[1, 1] = dth[2, 2] = -s
    dth[1, 2] = dth[2, 1] = -1j * c
    dph = np.zeros((4, 4), dtype=np.complex128)
    dph[3, 3] = -1j * np.exp(-1j * phi)
    return dth, dph


def loss(circ, bitstrings) -> float:
    a = sv_amplitudes(circ, bitstrings)
    return float(np.sum(np.log(np.abs(a) ** 2)))


def loss_and_grad(circ, bitstrings):
    """Adjoint state-vector gradient.  Returns (L, grad) where grad has shape
    (n_fsim, 2) holding dL/dtheta, dL/dphi per fSim gate in circuit order."""
    psi = statevector(circ)
    n = circ.n_qubits
    lam = np.zeros_like(psi)
    L = 0.0
    for x in bitstrings:
        ix = tuple(int(b) for b in x)
        a = psi[ix]
        L += float(np.log(abs(a) ** 2))
        lam[ix] += a / abs(a) ** 2
    fs = circ.fsim_indices()
    grad = np.zeros((len(fs), 2))
    pos = {g: i for i, g in enumerate(fs)}
    for gi in range(len(circ.gates) - 1, -1, -1):
        g = circ.gates[gi]
        gh = np.conj(np.asarray(g.matrix)).T
        psi = apply_gate(psi, gh, g.qubits)  # state before this gate
        if g.name == "fsim":
            dth, dph = _dfsim(*g.params)
            grad[pos[gi], 0] = 2.0 * np.real(np.vdot(lam, apply_gate(psi, dth, g.qubits)))
            grad[pos[gi], 1] = 2.0 * np.real(np.vdot(lam, apply_gate(psi, dph, g.qubits)))
        lam = apply_gate(lam, gh, g.qubits)
    del n
    return L, grad


def fd_grad(circ, bitstrings, which: Sequence[Tuple[int, int]], h: float = 1e-6) -> np.ndarray:
    """Central differences (step h) of L for the listed (fsim number,
    parameter 0=theta/1=phi) pairs."""
    from qcs_inputs import with_params

    base = [g.params for g in circ.gates if g.name == "fsim"]
    out = np.zeros(len(which))
    for w, (fi, pi) in enumerate(which):
        vals = []
        for sgn in (+1, -1):
            p = [list(x) for x in base]
            p[fi][pi] += sgn * h
            vals.append(loss(with_params(circ, [tuple(x) for x in p]), bitstrings))
        out[w] = (vals[0] - vals[1]) / (2 * h)
    return out


def fidelity(a_ref: np.ndarray, a: np.ndarray) -> float:
    """|sum conj(a_ref) a|^2 / (sum |a_ref|^2 sum |a|^2) over computed
    amplitudes (the paper plots fidelity without defining it)."""
    a_ref = np.asarray(a_ref, dtype=np.complex128).ravel()
    a = np.asarray(a, dtype=np.complex128).ravel()
    num = abs(np.vdot(a_ref, a)) ** 2
    den = np.vdot(a_ref, a_ref).real * np.vdot(a, a).real
    return float(num / den) if den > 0 else 0.0
