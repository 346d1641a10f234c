"""CPU pins of the FP64 oracle against facts that do not come from the oracle:
values the paper prints, closed forms, library routines (numpy), exact
rational arithmetic and brute force.  A plausible slip in the oracle (a
dropped term, a sign, a transposed operand, a wrong rounding) fails one of
these."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from oracle import OP_C, OP_N, OP_T


# ---------------------------------------------------------------------------
# CGEMM (Section 3)
# ---------------------------------------------------------------------------

def F(a):
    return np.asfortranarray(np.asarray(a, dtype=np.complex64))


def test_cgemm_complex_product_sign():
    # (1+2i)(3+4i) = -5+10i fixes Im = Ar*Bi + Ai*Br (the printed formula is garbled).
    C = oracle.cgemm(OP_N, OP_N, 1, 1, 1, 1.0, F([[1 + 2j]]), F([[3 + 4j]]))
    assert C[0, 0] == -5 + 10j


def test_cgemm_hand_values_all_ops():
    A = F([[1 + 1j, 2], [0, 3 - 1j]])  # A[i, l]
    B = F([[1, 1j], [2 - 1j, 1]])
    # by hand: A @ B
    AB = np.array([[(1 + 1j) + 2 * (2 - 1j), (1 + 1j) * 1j + 2], [(3 - 1j) * (2 - 1j), 3 - 1j]])
    assert np.array_equal(oracle.cgemm(OP_N, OP_N, 2, 2, 2, 1, A, B), AB)
    # A^T B: (A^T)[i,l] = A[l,i]
    AtB = np.array([[(1 + 1j) * 1 + 0, (1 + 1j) * 1j + 0],
                    [2 * 1 + (3 - 1j) * (2 - 1j), 2 * 1j + (3 - 1j)]])
    assert np.array_equal(oracle.cgemm(OP_T, OP_N, 2, 2, 2, 1, A, B), AtB)
    # A^H B
    AhB = np.array([[(1 - 1j) * 1, (1 - 1j) * 1j],
                    [2 * 1 + (3 + 1j) * (2 - 1j), 2 * 1j + (3 + 1j)]])
    assert np.array_equal(oracle.cgemm(OP_C, OP_N, 2, 2, 2, 1, A, B), AhB)
    # A B^H
    ABh = np.array([[(1 + 1j) * 1 + 2 * (-1j), (1 + 1j) * (2 + 1j) + 2],
                    [(3 - 1j) * (-1j), 3 - 1j]])
    assert np.array_equal(oracle.cgemm(OP_N, OP_C, 2, 2, 2, 1, A, B), ABh)


def test_cgemm_identity_and_permutation():
    A = qi.cgemm_operand(5, 7, 3, seed=11)
    I7 = F(np.eye(7))
    assert np.array_equal(oracle.cgemm(OP_N, OP_N, 5, 7, 7, 1, A, I7), A.astype(np.complex128))
    P = F(np.eye(5)[[2, 0, 4, 1, 3]])
    assert np.array_equal(oracle.cgemm(OP_N, OP_N, 5, 7, 5, 1, P, A),
                          A[[2, 0, 4, 1, 3]].astype(np.complex128))


def test_cgemm_alpha_beta_and_ld():
    m, n, k = 6, 5, 4
    A = qi.cgemm_operand(m, k, 0, seed=1, ld=9)
    B = qi.cgemm_operand(k, n, 0, seed=2, ld=4)
    C = qi.cgemm_operand(m, n, 0, seed=3, ld=8)
    al, be = 0.5 - 2j, 1j
    got = oracle.cgemm(OP_N, OP_N, m, n, k, al, A, B, be, C)
    ref = al * (A[:m].astype(np.complex128) @ B[:k].astype(np.complex128)) + be * C[:m].astype(np.complex128)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("opA,opB", [(OP_N, OP_N), (OP_T, OP_C), (OP_C, OP_T), (OP_N, OP_C)])
def test_cgemm_vs_numpy(opA, opB):
    m, n, k = 13, 9, 17
    A = qi.cgemm_operand(m if opA == OP_N else k, k if opA == OP_N else m, 4, seed=(1, opA))
    B = qi.cgemm_operand(k if opB == OP_N else n, n if opB == OP_N else k, 4, seed=(2, opB))
    f = {OP_N: lambda X: X, OP_T: lambda X: X.T, OP_C: lambda X: X.conj().T}
    ref = f[opA](A.astype(np.complex128)) @ f[opB](B.astype(np.complex128))
    got = oracle.cgemm(opA, opB, m, n, k, 1, A, B)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_cgemm_rows_matches_naive():
    m, n, k = 40, 23, 31
    A = qi.cgemm_operand(k, m, 2, seed=5)
    B = qi.cgemm_operand(k, n, 2, seed=6)
    C = qi.cgemm_operand(m, n, 2, seed=7)
    full = oracle.cgemm(OP_C, OP_N, m, n, k, 2 - 1j, A, B, 0.25j, C)
    rows = [0, 7, 39, 12]
    part = oracle.cgemm(OP_C, OP_N, m, n, k, 2 - 1j, A, B, 0.25j, C, rows=rows)
    np.testing.assert_allclose(part, full[rows], rtol=1e-14, atol=1e-14)


# ---------------------------------------------------------------------------
# Rounding to the tensor-core input types (Eq. 1, toLow)
# ---------------------------------------------------------------------------

def _probe_floats():
    g = np.random.default_rng(0)
    xs = list(g.standard_normal(2000).astype(np.float32))
    xs += list((g.standard_normal(2000) * np.exp2(g.integers(-40, 40, 2000))).astype(np.float32))
    special = [0.0, -0.0, 1.0, -1.0, 65504.0, 65519.99, 65520.0, 65536.0, 1e9, -1e9, 2.0 ** -14,
               2.0 ** -24, 2.0 ** -25, 1.5 * 2.0 ** -25, 2.0 ** -26, 3 * 2.0 ** -25, 2.0 ** -15 * 1.0009765625,
               1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 1.0 + 2.0 ** -11 + 2.0 ** -20, 2.0 ** -130,
               np.float32(3.4028235e38), np.float32(1.1754944e-38), np.float32(1e-45)]
    xs += [np.float32(s) for s in special]
    # ties at the 11th significant bit in the subnormal FP16 range
    xs += [np.float32(k * 2.0 ** -25) for k in range(1, 80)]
    return [np.float32(x) for x in xs]


def test_f16_conversion_matches_numpy():
    for x in _probe_floats():
        want = int(np.array([x], dtype=np.float32).astype(np.float16).view(np.uint16)[0])
        assert oracle.f32_to_f16_bits(float(x)) == want, x
    for x in [np.inf, -np.inf]:
        want = int(np.array([x], dtype=np.float32).astype(np.float16).view(np.uint16)[0])
        assert oracle.f32_to_f16_bits(x) == want


def test_f16_decode_exhaustive():
    codes = np.arange(65536, dtype=np.uint16)
    ref = codes.view(np.float16).astype(np.float32)
    got = np.array([oracle.f16_bits_to_f32(int(c)) for c in codes], dtype=np.float32)
    fin = np.isfinite(ref)
    assert np.array_equal(got[fin], ref[fin])
    assert np.array_equal(np.isnan(got), np.isnan(ref))
    assert np.array_equal(np.isinf(got), np.isinf(ref))


def _rne_grid(x: float, frac_bits: int):
    """Round a binary32 value to frac_bits fraction bits, nearest-even, in
    exact rational arithmetic (binary32 exponent range)."""
    if x == 0 or not math.isfinite(x):
        return x
    e = 0
    ax = abs(x)
    while ax >= 2.0 ** (e + 1):
        e += 1
    while ax < 2.0 ** e:
        e -= 1
    q = Fraction(2) ** (max(e, -126) - frac_bits)
    r = Fraction(ax) / q
    n = math.floor(r)
    rem = r - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    v = n * q
    if v >= Fraction(2) ** 128:
        v = math.inf
    else:
        v = float(v)
    return math.copysign(v, x)


def test_tf32_and_bf16_rounding_exact():
    for x in _probe_floats():
        assert oracle.f32_to_tf32(float(x)) == _rne_grid(float(x), 10), x
        assert oracle.f32_to_bf16(float(x)) == _rne_grid(float(x), 7), x


def test_split_reconstructs_within_bound():
    g = np.random.default_rng(3)
    x = (g.standard_normal(4000) * np.exp2(g.integers(-12, 12, 4000))).astype(np.float32)
    for kind, bound in ((0, 2.0 ** -22), (1, 2.0 ** -22), (2, 2.0 ** -16)):
        hi, lo = oracle.split(kind, 0, x)
        rec = hi.astype(np.float64) + lo.astype(np.float64) * 2.0 ** -11
        ok = np.abs(x) >= 2.0 ** -13 if kind == 0 else np.ones(x.shape, bool)  # FP16 normal range
        assert ok.sum() > 3500
        assert np.all(np.abs(rec - x)[ok] <= bound * np.abs(x.astype(np.float64))[ok])
        if kind == 0:  # below the FP16 normal range the pair loses bits: the reason for scaling
            assert np.max((np.abs(rec - x) / np.abs(x))[~ok]) > bound
        # the hi part alone is off by about half an ulp of the low type
        assert np.max(np.abs(hi - x) / np.abs(x)) > 2.0 ** -14
    # values exact in FP16 have no residual
    xs = np.array([1.0, -0.5, 3.0, 1024.0, 2.0 ** -14], dtype=np.float32)
    hi, lo = oracle.split(0, 0, xs)
    assert np.array_equal(hi, xs) and np.all(lo == 0)


def test_split_scaling_is_a_power_of_two_shift():
    g = np.random.default_rng(4)
    x = (g.standard_normal(1000) * 2.0 ** -30).astype(np.float32)
    hi_s, lo_s = oracle.split(0, 30, x)
    hi_r, lo_r = oracle.split(0, 0, (x.astype(np.float64) * 2.0 ** 30).astype(np.float32))
    assert np.array_equal(hi_s, hi_r) and np.array_equal(lo_s, lo_r)
    # without the scaling these values underflow FP16 entirely
    hi0, _ = oracle.split(0, 0, x)
    assert np.all(hi0 == 0)


# ---------------------------------------------------------------------------
# Exponent statistics and the selection rule (Section 4.1, 4.3, 5.2)
# ---------------------------------------------------------------------------

def _floor_log2(v: float) -> int:
    e = 0
    a = abs(v)
    while a >= 2.0 ** (e + 1):
        e += 1
    while a < 2.0 ** e:
        e -= 1
    return e


def test_exp_stats_brute_force():
    g = np.random.default_rng(7)
    X = np.asfortranarray(((g.standard_normal((9, 6)) + 1j * g.standard_normal((9, 6)))
                           * np.exp2(g.integers(-30, 30, (9, 6)))).astype(np.complex64))
    X[0, 0] = 0
    X[1, 1] = complex(np.float32(1e-40), 0)   # subnormal real part, zero imaginary part
    X[2, 2] = complex(np.inf, 1)
    X[3, 3] = complex(np.nan, 2.0 ** -14)
    hist, nz = oracle.exp_stats(X)
    want = np.zeros(256, dtype=np.int64)
    wz = 0
    for v in np.concatenate([X.real.ravel(), X.imag.ravel()]):
        v = float(v)
        if not math.isfinite(v):
            want[255] += 1
        elif v == 0:
            wz += 1
        else:
            want[max(_floor_log2(v) + 127, 0)] += 1
    assert nz == wz and np.array_equal(hist, want)


def _modes(golden):
    out = []
    with open(os.path.join(golden, "selector_types.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                t, tol, mode = line.split()
                out.append((int(t), float(tol), mode))
    return out


def test_selector_types_golden(golden_dir):
    for kind, tol, mode in _modes(golden_dir):
        A = qi.typed_matrix(128, 128, kind, seed=(kind, 1))
        B = qi.typed_matrix(128, 128, 1, seed=(kind, 2))
        sa = oracle.stats_summary(*oracle.exp_stats(A))
        sb = oracle.stats_summary(*oracle.exp_stats(B))
        got, _, _ = oracle.select_mode(sa, sb, tol)
        assert oracle.MODE_NAMES[got] == mode, (kind, tol)


def _hist_of(values):
    X = np.asfortranarray(np.asarray(values, dtype=np.complex64).reshape(-1, 1))
    return oracle.stats_summary(*oracle.exp_stats(X))


def test_select_rule_cases():
    one = _hist_of([1.0, 0.5j, -0.25])
    assert oracle.select_mode(one, one, 0.0) == (oracle.MODE_FP16X, 0, 0)
    small = _hist_of([2.0 ** -20, 2.0 ** -30 * 1j])   # fits only after scaling
    assert oracle.select_mode(one, small, 0.0) == (oracle.MODE_FP16X_SCALED, 14, 14 + 20)
    big = _hist_of([2.0 ** 20, 1.0])                    # overflows unscaled FP16, fits scaled
    assert oracle.select_mode(big, one, 0.0) == (oracle.MODE_FP16X_SCALED, -6, 14)
    wide = _hist_of([2.0 ** 20, 2.0 ** -20])            # 40 binades: beyond the 29-binade window
    assert oracle.select_mode(wide, one, 0.0)[0] == oracle.MODE_TF32X
    assert oracle.select_mode(wide, one, 0.5)[0] == oracle.MODE_FP16X_SCALED
    nan = _hist_of([np.nan, 1.0])
    assert oracle.select_mode(one, nan, 0.0)[0] == oracle.MODE_FP32
    zero = _hist_of([0.0, 0.0])
    assert oracle.select_mode(zero, one, 0.0) == (oracle.MODE_FP16X, 0, 0)
    # exactly at the window's lower edge: e_max - 28 survives, e_max - 29 does not
    edge = _hist_of([1.0, 2.0 ** -28])
    assert edge["under2"] == 0
    edge2 = _hist_of([1.0, 2.0 ** -29])
    assert edge2["under2"] == 1


def test_size_rule():
    assert oracle.size_rule(2048, 4096, 2048) is None
    assert oracle.size_rule(512, 4096, 2047) == oracle.MODE_TF32X
    assert oracle.size_rule(511, 4096, 4096) == oracle.MODE_FP32


# ---------------------------------------------------------------------------
# The emulated product in exact arithmetic (Eq. 1 + Section 3)
# ---------------------------------------------------------------------------

def test_tcec_model_accuracy_uniform_inputs():
    # Section 3 prints relative errors of 1e-7 .. 1e-6 for U(-1,1) inputs.
    m, n, k = 24, 20, 64
    A = qi.uniform_operand(m, k, 1)
    B = qi.uniform_operand(k, n, 2)
    exact = oracle.cgemm(OP_N, OP_N, m, n, k, 1, A, B)
    for kind in (0, 1):
        err = oracle.rel_fro_error(oracle.tcec_cgemm(kind, 0, 0, OP_N, OP_N, m, n, k, 1, A, B), exact)
        assert 1e-9 < err < 1e-6, (kind, err)
    # one low-precision product without the correction is far off (Fig. 2)
    A16 = A.astype(np.complex64)
    hi_r, _ = oracle.split(0, 0, A16.real)
    hi_i, _ = oracle.split(0, 0, A16.imag)
    only_hi = np.asfortranarray((hi_r + 1j * hi_i).astype(np.complex64))
    err_hi = oracle.rel_fro_error(oracle.cgemm(OP_N, OP_N, m, n, k, 1, only_hi, B), exact)
    assert err_hi > 1e-5
    # BF16 pairs keep about 16 significant bits: above the FP32-level bar
    err_bf = oracle.rel_fro_error(oracle.tcec_cgemm(2, 0, 0, OP_N, OP_N, m, n, k, 1, A, B), exact)
    assert err_bf > 1e-6


def test_tcec_model_exact_on_small_integers_and_ops():
    g = np.random.default_rng(9)
    A = np.asfortranarray((g.integers(-8, 9, (7, 5)) + 1j * g.integers(-8, 9, (7, 5))).astype(np.complex64))
    B = np.asfortranarray((g.integers(-8, 9, (6, 7)) + 1j * g.integers(-8, 9, (6, 7))).astype(np.complex64))
    # op(A) = A^T (5 x 7), op(B) = B^H (7 x 6)
    ref = A.T.astype(np.complex128) @ B.conj().T.astype(np.complex128)
    for kind in (0, 1, 2):
        got = oracle.tcec_cgemm(kind, 0, 0, OP_T, OP_C, 5, 6, 7, 1, A, B)
        assert np.array_equal(got, ref), kind
    # scaling by 2^sA, 2^sB is undone exactly
    got = oracle.tcec_cgemm(0, 3, -2, OP_T, OP_C, 5, 6, 7, 1, A, B)
    assert np.array_equal(got, ref)


def test_tcec_model_scaled_recovers_tiny_inputs():
    m, n, k = 16, 16, 32
    A = np.asfortranarray((qi.uniform_operand(m, k, 3).astype(np.complex128) * 2.0 ** -40).astype(np.complex64))
    B = qi.uniform_operand(k, n, 4)
    exact = oracle.cgemm(OP_N, OP_N, m, n, k, 1, A, B)
    sa = oracle.stats_summary(*oracle.exp_stats(A))
    sb = oracle.stats_summary(*oracle.exp_stats(B))
    mode, sA, sB = oracle.select_mode(sa, sb, 0.0)
    assert mode == oracle.MODE_FP16X_SCALED
    err_scaled = oracle.rel_fro_error(oracle.tcec_cgemm(0, sA, sB, OP_N, OP_N, m, n, k, 1, A, B), exact)
    err_plain = oracle.rel_fro_error(oracle.tcec_cgemm(0, 0, 0, OP_N, OP_N, m, n, k, 1, A, B), exact)
    assert err_scaled < 1e-6 and err_plain > 0.5


def test_tcec_3m_model_exact_on_small_integers_and_ops():
    # integer parts and their sums are exact in every kind (also halved, for
    # FP16's one binade less of scaling): the three-product form then gives
    # the exact product, whatever the op -- a wrong sign or part fails here
    g = np.random.default_rng(12)
    A = np.asfortranarray((g.integers(-8, 9, (7, 5)) + 1j * g.integers(-8, 9, (7, 5))).astype(np.complex64))
    B = np.asfortranarray((g.integers(-8, 9, (6, 7)) + 1j * g.integers(-8, 9, (6, 7))).astype(np.complex64))
    for opA, opB, ra, rb in ((OP_T, OP_C, A.T, B.conj().T), (OP_C, OP_T, A.conj().T, B.T)):
        ref = ra.astype(np.complex128) @ rb.astype(np.complex128)
        for kind in (0, 1, 2):
            got = oracle.tcec_cgemm_3m(kind, 0, 0, opA, opB, 5, 6, 7, 1, A, B)
            assert np.array_equal(got, ref), (kind, opA)
        assert np.array_equal(oracle.tcec_cgemm_3m(0, 3, -2, opA, opB, 5, 6, 7, 1, A, B), ref)
    # alpha and beta as in the four-product model
    C = np.asfortranarray((g.integers(-4, 5, (5, 6)) + 1j * g.integers(-4, 5, (5, 6))).astype(np.complex64))
    ref = (0.5 - 1j) * (A.T.astype(np.complex128) @ B.conj().T.astype(np.complex128)) + 2j * C
    got = oracle.tcec_cgemm_3m(1, 0, 0, OP_T, OP_C, 5, 6, 7, 0.5 - 1j, A, B, 2j, C)
    assert np.array_equal(got, ref)


def test_tcec_3m_model_accuracy_uniform_inputs():
    # the three-product form stays at FP32 level on U(-1,1) parts, close to
    # the four-product model's error
    m, n, k = 24, 20, 64
    A = qi.uniform_operand(m, k, 1)
    B = qi.uniform_operand(k, n, 2)
    exact = oracle.cgemm(OP_N, OP_N, m, n, k, 1, A, B)
    for kind in (0, 1):
        e3 = oracle.rel_fro_error(oracle.tcec_cgemm_3m(kind, 0, 0, OP_N, OP_N, m, n, k, 1, A, B), exact)
        e4 = oracle.rel_fro_error(oracle.tcec_cgemm(kind, 0, 0, OP_N, OP_N, m, n, k, 1, A, B), exact)
        assert 1e-9 < e3 < 1e-6 and e3 < 4 * e4, (kind, e3, e4)


# ---------------------------------------------------------------------------
# Real matrices: the SGEMM of Section 2.1
# ---------------------------------------------------------------------------

def test_sgemm_hand_values_and_ops():
    A = np.asfortranarray(np.array([[1, 2, 3], [4, 5, 6]], dtype=np.float32))  # 2 x 3
    B = np.asfortranarray(np.array([[1, 0], [0, 1], [1, 1]], dtype=np.float32))  # 3 x 2
    # A B = [[4, 5], [10, 11]], by hand
    assert np.array_equal(oracle.sgemm(OP_N, OP_N, 2, 2, 3, 1.0, A, B), [[4, 5], [10, 11]])
    # op T: A^T A (3 x 3) = [[17, 22, 27], [22, 29, 36], [27, 36, 45]]
    assert np.array_equal(oracle.sgemm(OP_T, OP_N, 3, 3, 2, 1.0, A, A),
                          [[17, 22, 27], [22, 29, 36], [27, 36, 45]])
    # OP_C on a real matrix is the transpose
    assert np.array_equal(oracle.sgemm(OP_C, OP_N, 3, 3, 2, 1.0, A, A),
                          oracle.sgemm(OP_T, OP_N, 3, 3, 2, 1.0, A, A))
    # alpha, beta, C read through its leading dimension
    C = np.asfortranarray(np.array([[1, 1], [2, 2], [9, 9]], dtype=np.float32))  # ld 3
    got = oracle.sgemm(OP_N, OP_N, 2, 2, 3, 2.0, A, B, beta=-1.0, C=C)
    assert np.array_equal(got, [[7, 9], [18, 20]])


@pytest.mark.parametrize("opA,opB", [(OP_N, OP_N), (OP_T, OP_N), (OP_N, OP_T), (OP_T, OP_T)])
def test_sgemm_vs_numpy_and_complex_oracle(opA, opB):
    m, n, k = 13, 11, 17
    A = qi.sgemm_operand(*((m, k) if opA == OP_N else (k, m)), 4, (1, opA))
    B = qi.sgemm_operand(*((k, n) if opB == OP_N else (n, k)), 4, (2, opB))
    a = A.astype(np.float64) if opA == OP_N else A.T.astype(np.float64)
    b = B.astype(np.float64) if opB == OP_N else B.T.astype(np.float64)
    got = oracle.sgemm(opA, opB, m, n, k, 1.0, A, B)
    assert np.allclose(got, a @ b, rtol=1e-13, atol=1e-13)
    # a real matrix is a complex one with zero imaginary parts
    Ac = np.asfortranarray(A.astype(np.complex64))
    Bc = np.asfortranarray(B.astype(np.complex64))
    gc = oracle.cgemm(opA, opB, m, n, k, 1, Ac, Bc)
    assert np.array_equal(gc.imag, np.zeros_like(got)) and np.allclose(gc.real, got, rtol=1e-13)
    # sampled rows are those rows of the full product
    rows = [12, 0, 5]
    assert np.array_equal(oracle.sgemm(opA, opB, m, n, k, 1.0, A, B, rows=rows), got[rows])


def test_tcec_sgemm_reduces_to_the_complex_model_and_is_exact_on_integers():
    m, n, k = 9, 10, 40
    A = qi.sgemm_operand(m, k, 8, 5)
    B = qi.sgemm_operand(k, n, 8, 6)
    Ac = np.asfortranarray(A.astype(np.complex64))
    Bc = np.asfortranarray(B.astype(np.complex64))
    for kind, sA, sB in ((0, 0, 0), (0, 3, -2), (1, 0, 0), (2, 0, 0)):
        r = oracle.tcec_sgemm(kind, sA, sB, OP_N, OP_N, m, n, k, 1.0, A, B)
        c = oracle.tcec_cgemm(kind, sA, sB, OP_N, OP_N, m, n, k, 1, Ac, Bc)
        assert np.allclose(r, c.real, rtol=1e-14, atol=0), kind
    g = np.random.default_rng(3)
    Ai = np.asfortranarray(g.integers(-8, 9, (7, 5)).astype(np.float32))
    Bi = np.asfortranarray(g.integers(-8, 9, (6, 7)).astype(np.float32))
    ref = Ai.T.astype(np.float64) @ Bi.T.astype(np.float64)
    for kind in (0, 1, 2):
        assert np.array_equal(oracle.tcec_sgemm(kind, 0, 0, OP_T, OP_T, 5, 6, 7, 1.0, Ai, Bi), ref)
    assert np.array_equal(oracle.tcec_sgemm(0, 4, -3, OP_T, OP_T, 5, 6, 7, 1.0, Ai, Bi), ref)


def test_tcec_sgemm_accuracy_bound():
    # hi + lo carries 22 significant bits; the dropped lo*lo term is ~2^-22
    # relative, so the emulated product is FP32-accurate (Section 2.1)
    m, n, k = 32, 24, 256
    A = np.asfortranarray(np.random.default_rng(4).uniform(-1, 1, (m, k)).astype(np.float32))
    B = np.asfortranarray(np.random.default_rng(5).uniform(-1, 1, (k, n)).astype(np.float32))
    exact = oracle.sgemm(OP_N, OP_N, m, n, k, 1.0, A, B)
    for kind in (0, 1):
        err = oracle.rel_fro_error(oracle.tcec_sgemm(kind, 0, 0, OP_N, OP_N, m, n, k, 1.0, A, B),
                                   exact)
        assert 1e-9 < err < 1e-6, (kind, err)
    err_bf = oracle.rel_fro_error(oracle.tcec_sgemm(2, 0, 0, OP_N, OP_N, m, n, k, 1.0, A, B), exact)
    assert err_bf > 1e-6


def test_exp_stats_real_hand_values_and_complex_equivalence():
    x = np.array([1.0, 0.5, 0.0, 3.0, 2.0 ** -130, np.inf, -0.75, 2.0 ** 20], dtype=np.float32)
    hist, nz = oracle.exp_stats_real(np.asfortranarray(x.reshape(4, 2, order="F")))
    want = np.zeros(256, dtype=np.int64)
    for b in (127, 126, 128, 0, 255, 126, 147):
        want[b] += 1
    assert nz == 1 and np.array_equal(hist, want)
    X = qi.sgemm_operand(30, 20, 20, 8)
    h_r, z_r = oracle.exp_stats_real(X)
    h_c, z_c = oracle.exp_stats(np.asfortranarray(X.astype(np.complex64)))
    assert np.array_equal(h_r, h_c) and z_c == z_r + X.size


# ---------------------------------------------------------------------------
# Circuits, tensor networks, amplitudes (Section 2.2, Section 5.3)
# ---------------------------------------------------------------------------

def test_hadamard_example_golden(golden_dir):
    rows, state = [], []
    with open(os.path.join(golden_dir, "hadamard_example.txt")) as f:
        for line in f:
            if line.startswith("gate"):
                v = [float(x) for x in line.split()[1:]]
                rows.append([v[0] + 1j * v[1], v[2] + 1j * v[3]])
            elif line.startswith("state"):
                v = [float(x) for x in line.split()[1:]]
                state.append(v[0] + 1j * v[1])
    c = qi.Circuit(1, [qi.Gate("h", (0,), np.array(rows))])
    np.testing.assert_allclose(oracle.statevector(c).ravel(), state, atol=1e-15)
    tn, outl = oracle.circuit_tn(c, None)
    np.testing.assert_allclose(oracle.contract_network(tn, outl).ravel(), state, atol=1e-15)


def test_gate_closed_forms():
    X = np.array([[0, 1], [1, 0]])
    for name, P in (("sqrtX", X), ("sqrtY", np.array([[0, -1j], [1j, 0]]))):
        S = qi.SQRT_GATES[name]
        np.testing.assert_allclose(S @ S, P, atol=1e-15)
    c = qi.Circuit(1, [qi.Gate("sqrtX", (0,), qi.SQRT_GATES["sqrtX"])] * 2)
    np.testing.assert_allclose(oracle.statevector(c).ravel(), [0, 1], atol=1e-15)
    # fSim(pi/2, phi) sends |01> to -i|10>
    c = qi.Circuit(2, [qi.Gate("x", (1,), X.astype(complex)), qi.Gate("fsim", (0, 1), qi.fsim(np.pi / 2, 0.3))])
    psi = oracle.statevector(c)
    np.testing.assert_allclose(psi[1, 0], -1j, atol=1e-15)
    assert abs(psi[0, 1]) < 1e-15


def test_statevector_against_dense_kronecker():
    # the full 2^n unitary from np.kron (a library routine), n = 5
    circ = qi.random_grid_circuit(1, 5, 4, seed=21)
    n = 5
    U = np.eye(2 ** n, dtype=complex)
    I2 = np.eye(2)
    for g in circ.gates:
        if len(g.qubits) == 1:
            q = g.qubits[0]
            ops = [g.matrix if i == q else I2 for i in range(n)]
            full = ops[0]
            for o in ops[1:]:
                full = np.kron(full, o)
        else:
            a, b = g.qubits
            assert b == a + 1
            full = np.kron(np.kron(np.eye(2 ** a), g.matrix), np.eye(2 ** (n - b - 1)))
        U = full @ U
    np.testing.assert_allclose(oracle.statevector(circ).ravel(), U[:, 0], atol=1e-13)


def test_tn_amplitudes_match_statevector_small_grid():
    circ = qi.random_grid_circuit(3, 4, 8, seed=0)
    bits = qi.random_bitstrings(12, 64, seed=1)
    sv = oracle.sv_amplitudes(circ, bits)
    tn = np.array([oracle.amplitude(circ, b) for b in bits])
    np.testing.assert_allclose(tn, sv, rtol=0, atol=1e-13)
    assert oracle.fidelity(sv, tn) > 1 - 1e-12


def test_unitarity_open_network():
    circ = qi.random_grid_circuit(3, 4, 6, seed=5)
    tn, outl = oracle.circuit_tn(circ, None)
    psi = oracle.contract_network(tn, outl)
    assert abs(np.sum(np.abs(psi) ** 2) - 1.0) < 1e-12
    np.testing.assert_allclose(psi, oracle.statevector(circ), atol=1e-13)


def test_contraction_order_independence_and_loops():
    circ = qi.random_grid_circuit(2, 3, 5, seed=8)
    bits = [1, 0, 1, 1, 0, 0]
    tn, outl = oracle.circuit_tn(circ, bits)
    a1 = complex(oracle.contract_network(tn, outl))
    # a different, sequential order: always fold the next tensor into the running result
    order = [(0, 1)] + [(len(tn) + i, i + 2) for i in range(len(tn) - 2)]
    a2 = complex(oracle.contract_network(tn, outl, order))
    a3 = complex(oracle.contract_network(tn, outl, use_loops=True))
    assert abs(a1 - a2) < 1e-12 and abs(a1 - a3) < 1e-12


def test_pair_contraction_vs_einsum():
    g = np.random.default_rng(2)
    A = g.standard_normal((2, 3, 4, 2)) + 1j * g.standard_normal((2, 3, 4, 2))
    B = g.standard_normal((4, 2, 5)) + 1j * g.standard_normal((4, 2, 5))
    ref = np.einsum("abcd,cde->eab", A, B)
    got = oracle.contract_pair_loops(A, [0, 1, 2, 3], B, [2, 3, 4], [4, 0, 1])
    np.testing.assert_allclose(got, ref, atol=1e-12)
    got2 = oracle.contract_pair_np(A, [0, 1, 2, 3], B, [2, 3, 4], [4, 0, 1])
    np.testing.assert_allclose(got2, ref, atol=1e-12)


def test_slicing_sums_to_unsliced():
    circ = qi.random_grid_circuit(2, 3, 6, seed=9)
    bits = [0, 1, 1, 0, 1, 0]
    tn, _ = oracle.circuit_tn(circ, bits)
    labels = sorted({l for _, ls in tn for l in ls})
    sliced = labels[10:13]
    assert abs(oracle.amplitude(circ, bits, sliced) - oracle.amplitude(circ, bits)) < 1e-13


def test_closed_form_circuits():
    # no gates: <x|0> = delta(x, 0)
    c = qi.Circuit(4, [])
    assert oracle.amplitude(c, [0, 0, 0, 0]) == 1 and oracle.amplitude(c, [0, 1, 0, 0]) == 0
    # H on every qubit: |a|^2 = 2^-n for every x
    H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    c = qi.Circuit(5, [qi.Gate("h", (q,), H) for q in range(5)])
    for x in qi.random_bitstrings(5, 6, seed=3):
        assert abs(abs(oracle.amplitude(c, x)) ** 2 - 2.0 ** -5) < 1e-15


# ---------------------------------------------------------------------------
# Gradient reference
# ---------------------------------------------------------------------------

def test_adjoint_gradient_matches_central_differences():
    circ = qi.random_grid_circuit(2, 3, 4, seed=4, theta=None, phi=None, param_seed=5)
    bits = qi.random_bitstrings(6, 8, seed=6)
    L, grad = oracle.loss_and_grad(circ, bits)
    assert abs(L - oracle.loss(circ, bits)) < 1e-12
    which = [(i, p) for i in range(grad.shape[0]) for p in (0, 1)]
    fd = oracle.fd_grad(circ, bits, which, h=1e-6)
    want = np.array([grad[i, p] for i, p in which])
    np.testing.assert_allclose(want, fd, rtol=1e-5, atol=1e-6)


def test_fidelity_definition():
    a = np.array([1 + 1j, 0.5, -2j])
    assert abs(oracle.fidelity(a, a) - 1) < 1e-15
    assert abs(oracle.fidelity(a, a * np.exp(0.7j)) - 1) < 1e-15   # global phase invariant
    assert oracle.fidelity(np.array([1, 0]), np.array([0, 1])) == 0


def test_inplace_statevector_matches_tensordot_statevector():
    # two independent implementations of the same definition (C in place vs numpy tensordot)
    for rows, cols, depth, seed in ((3, 4, 8, 0), (2, 5, 6, 3), (1, 3, 3, 1)):
        circ = qi.random_grid_circuit(rows, cols, depth, seed=seed)
        a = oracle.statevector_inplace(circ)
        b = oracle.statevector(circ).ravel()
        np.testing.assert_allclose(a, b, atol=1e-13)
        x = qi.random_bitstrings(rows * cols, 1, seed=9)[0]
        assert a[oracle.bit_index(x)] == b[oracle.bit_index(x)] or abs(a[oracle.bit_index(x)] - b[oracle.bit_index(x)]) < 1e-14


def test_random_greedy_order_and_slice_chooser_preserve_the_amplitude():
    circ = qi.random_grid_circuit(3, 3, 6, seed=2)
    bits = qi.random_bitstrings(9, 1, seed=3)[0]
    tn, outl = oracle.circuit_tn(circ, bits)
    ref = oracle.statevector(circ)[tuple(int(b) for b in bits)]
    order = oracle.random_greedy_order(tn, outl, seeds=range(3))
    assert abs(complex(oracle.contract_network(tn, outl, order)) - ref) < 1e-13
    flops, big = oracle.order_cost(tn, order, outl)
    for seed in range(3):  # the best of the seeds is no worse than any one of them
        single = oracle.random_greedy_order(tn, outl, seeds=[seed])
        assert flops <= oracle.order_cost(tn, single, outl)[0]
    labels = oracle.slice_labels_by_weight(tn, outl, order, 3)
    assert len(set(labels)) == 3
    total = sum(complex(oracle.contract_network(oracle.slice_network(tn, dict(zip(labels, v))), outl))
                for v in np.ndindex(2, 2, 2))
    assert abs(total - ref) < 1e-13


# ---------------------------------------------------------------------------
# Per-row / per-column scaling (a variant beyond the paper, on Section 4.1's
# scaling basis): line statistics, selection, emulation model
# ---------------------------------------------------------------------------

def _op_lines(X, op, rows_of_op, r, c):
    """Lines of op(X) by numpy indexing: rows of op(A) / columns of op(B)."""
    M = np.asarray(X)[:r, :c]
    M = M if op == OP_N else M.T
    return [M[i, :] for i in range(M.shape[0])] if rows_of_op else [M[:, j] for j in range(M.shape[1])]


def _biased_exp_frexp(x: float) -> int:
    """floor(log2|x|) + 127 through frexp for normal binary32 numbers, 0 for
    subnormals, -1 for zero and Inf/NaN."""
    if x == 0 or not math.isfinite(x):
        return -1
    if abs(x) < 2.0 ** -126:
        return 0
    return math.frexp(x)[1] - 1 + 127


def _brute_rowcol(A, B, opA, opB, m, n, k):
    res = []
    for X, op, rows_of_op, r, c in ((A, opA, True, *((m, k) if opA == OP_N else (k, m))),
                                    (B, opB, False, *((k, n) if opB == OP_N else (n, k)))):
        emax, under, nnz = [], 0, 0
        for line in _op_lines(X, op, rows_of_op, r, c):
            bs = [_biased_exp_frexp(float(np.float32(v))) for z in line for v in (z.real, z.imag)]
            bs = [b for b in bs if b >= 0]
            E = max(bs) if bs else -1
            emax.append(E)
            nnz += len(bs)
            under += sum(1 for b in bs if b == 0 or b < E - 28)
        res.append((emax, under, nnz))
    return res


@pytest.mark.parametrize("opA,opB", [(OP_N, OP_N), (OP_T, OP_C), (OP_C, OP_T)])
def test_rowcol_stats_brute_force(opA, opB):
    m, n, k = 9, 7, 11
    ra, ca = (m, k) if opA == OP_N else (k, m)
    rb, cb = (k, n) if opB == OP_N else (n, k)
    A = qi.line_scaled_operand(ra, ca, 40, 0 if opA == OP_N else 1, seed=(opA, 1), ld=ra + 2)
    B = qi.line_scaled_operand(rb, cb, 40, 1 if opB == OP_N else 0, seed=(opB, 2))
    # a zero line, a subnormal-only line, a scalar 29 binades under its line
    if opA == OP_N:
        A[3, :k] = 0
        A[5, :k] = np.float32(3e-41)
        A[6, 2] = complex(A[6, 2].real * np.float32(2.0 ** -29), 0)
    else:
        A[:k, 3] = 0
        A[:k, 5] = np.float32(3e-41)
    ea, eb, cnt = oracle.rowcol_stats(A, B, opA, opB, m, n, k)
    (ba, ua, na), (bb, ub, nb) = _brute_rowcol(A, B, opA, opB, m, n, k)
    assert list(ea) == ba and list(eb) == bb
    assert list(cnt) == [ua, na, ub, nb]
    assert ea[3] == -1 and ea[5] == 0


def test_rowcol_stats_hand_window_edges():
    # each row: 2^a, 2^(a-28) (on the window's lower edge), 2^(a-29) (below), 0
    a = [-100, -3, 0, 17, 90]
    A = F([[2.0 ** e, 2.0 ** (e - 28), 2.0 ** (e - 29) * 1j, 0] for e in a])
    B = F(np.ones((4, 2)))
    ea, eb, cnt = oracle.rowcol_stats(A, B, OP_N, OP_N, 5, 2, 4)
    assert list(ea) == [e + 127 for e in a]
    assert list(eb) == [127, 127]
    # under: 2^(a-29) of every row, and 2^-128 of the first (a binary32 subnormal)
    assert list(cnt) == [6, 15, 0, 8]
    assert [oracle.line_scale(E) for E in ea] == [14 - e for e in a]
    assert oracle.line_scale(-1) == 0


def test_select_rowcol_cases():
    m = n = k = 48
    summ = lambda X: oracle.stats_summary(*oracle.exp_stats(X))
    # lines two to forty binades apart: the whole-matrix window fails, every line fits
    A = qi.line_scaled_operand(m, k, 20, 0, seed=5)
    B = qi.line_scaled_operand(k, n, 20, 1, seed=6)
    cnt = oracle.rowcol_stats(A, B, OP_N, OP_N, m, n, k)[2]
    assert oracle.select_mode(summ(A), summ(B), 0.1)[0] == oracle.MODE_TF32X
    assert oracle.select_rowcol(summ(A), summ(B), cnt, 0.1) == (oracle.MODE_FP16X_ROWCOL, 0, 0)
    # per-element spread: every line spans the whole range, TF32X stays
    A2 = qi.cgemm_operand(m, k, 20, seed=7)
    cnt2 = oracle.rowcol_stats(A2, B, OP_N, OP_N, m, n, k)[2]
    assert oracle.select_rowcol(summ(A2), summ(B), cnt2, 0.1)[0] == oracle.MODE_TF32X
    # what Section 4.1 already accepts is left as it is
    A3, B3 = qi.cgemm_operand(m, k, 0, seed=8), qi.cgemm_operand(k, n, 0, seed=9)
    cnt3 = oracle.rowcol_stats(A3, B3, OP_N, OP_N, m, n, k)[2]
    assert oracle.select_rowcol(summ(A3), summ(B3), cnt3, 0.1) == oracle.select_mode(summ(A3), summ(B3), 0.1)
    # Inf: plain FP32
    A4 = A.copy(order="F")
    A4[0, 0] = np.inf
    cnt4 = oracle.rowcol_stats(A4, B, OP_N, OP_N, m, n, k)[2]
    assert oracle.select_rowcol(summ(A4), summ(B), cnt4, 0.1)[0] == oracle.MODE_FP32


@pytest.mark.parametrize("opA,opB", [(OP_N, OP_N), (OP_T, OP_C), (OP_C, OP_N)])
def test_tcec_rowcol_model_exact_on_line_scaled_integers(opA, opB):
    g = np.random.default_rng(11)
    m, n, k = 6, 5, 7
    ra, ca = (m, k) if opA == OP_N else (k, m)
    rb, cb = (k, n) if opB == OP_N else (n, k)
    ints = lambda r, c: g.integers(-8, 9, (r, c)) + 1j * g.integers(-8, 9, (r, c))
    # op(A)'s rows and op(B)'s columns 2^-40 .. 2^40 apart
    fa = np.exp2(g.integers(-40, 41, m))
    fb = np.exp2(g.integers(-40, 41, n))
    A = ints(ra, ca) * (fa[:, None] if opA == OP_N else fa[None, :])
    B = ints(rb, cb) * (fb[None, :] if opB == OP_N else fb[:, None])
    A, B = F(A), F(B)
    opm = lambda X, op: X if op == OP_N else (X.T if op == OP_T else X.conj().T)
    ref = opm(A.astype(np.complex128), opA) @ opm(B.astype(np.complex128), opB)
    ea, eb, _ = oracle.rowcol_stats(A, B, opA, opB, m, n, k)
    got = oracle.tcec_cgemm_rowcol(ea, eb, opA, opB, m, n, k, 1.0, A, B)
    assert np.array_equal(got, ref)
    # one scale per matrix loses the rows far below the largest
    sa = oracle.stats_summary(*oracle.exp_stats(A))
    sb = oracle.stats_summary(*oracle.exp_stats(B))
    whole = oracle.tcec_cgemm(0, 14 - sa["e_max"], 14 - sb["e_max"], opA, opB, m, n, k, 1.0, A, B)
    assert not np.array_equal(whole, ref)
    # alpha and beta after the unscaling
    C0 = F(ints(m, n))
    got = oracle.tcec_cgemm_rowcol(ea, eb, opA, opB, m, n, k, 0.5 - 1j, A, B, 2.0, C0)
    assert np.array_equal(got, (0.5 - 1j) * ref + 2.0 * C0.astype(np.complex128))


def test_tcec_rowcol_model_accuracy_line_scaled_gaussian():
    m, n, k = 40, 36, 256
    A = qi.line_scaled_operand(m, k, 30, 0, seed=12)
    B = qi.line_scaled_operand(k, n, 30, 1, seed=13)
    exact = oracle.cgemm(OP_N, OP_N, m, n, k, 1.0, A, B)
    ea, eb, _ = oracle.rowcol_stats(A, B, OP_N, OP_N, m, n, k)
    err = oracle.rel_fro_error(oracle.tcec_cgemm_rowcol(ea, eb, OP_N, OP_N, m, n, k, 1.0, A, B), exact)
    # per element against the magnitudes: FP32-level, as Eq. 1 promises per line
    got = oracle.tcec_cgemm_rowcol(ea, eb, OP_N, OP_N, m, n, k, 1.0, A, B)
    mag = np.abs(A[:m, :k]).astype(np.float64) @ np.abs(B[:k, :n]).astype(np.float64)
    assert np.all(np.abs(got - exact) <= 2.0 ** -20 * mag)
    assert err < 1e-6
