"""Per-row / per-column power-of-two scaling (qcs_set_rowcol_scaling; a
variant beyond the paper on Section 4.1's scaling basis) against the FP64
oracle: the per-line statistics bit for bit, the selection, the product
element by element against the oracle's exact model of the emulation, and
every other outcome bit-identical to the call with the option off."""
import ctypes

import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import abs_bound, dev, host, lib, need_gpu, torch

pytestmark = pytest.mark.gpu

TOL = 0.1


@pytest.fixture(scope="module")
def handles():
    need_gpu()
    q = lib()
    on = q.Handle(tol=TOL, size_rule=False)
    on.set_rowcol_scaling(True)
    off = q.Handle(tol=TOL, size_rule=False)
    yield on, off
    on.close()
    off.close()


def _stored(op, r, c):
    return (r, c) if op == 0 else (c, r)


def _line_scaled(m, n, k, opA, opB, s, seed, pad=0):
    ra, ca = _stored(opA, m, k)
    rb, cb = _stored(opB, k, n)
    # the lines of op(A) are A's rows for N and its columns otherwise
    A = qi.line_scaled_operand(ra, ca, s, 0 if opA == 0 else 1, (seed, 1), ld=ra + pad)
    B = qi.line_scaled_operand(rb, cb, s, 1 if opB == 0 else 0, (seed, 2), ld=rb + pad)
    return A, B


def _summ(X, op, r, c):
    rows, cols = _stored(op, r, c)
    return oracle.stats_summary(*oracle.exp_stats(X, rows, cols))


def _run(h, m, n, k, opA, opB, A, B, alpha=1.0, beta=0.0, C0=None):
    q = lib()
    Ad = dev(A)[:(m if opA == 0 else k)]
    Bd = dev(B)[:(k if opB == 0 else n)]
    if C0 is not None:
        Cd = dev(C0)
    else:
        Cd = q.fortran_empty(m, n, ld=m + 2)
        Cd.fill_(complex(float("nan"), float("nan")))
    desc = torch.zeros(4, dtype=torch.int32, device="cuda")
    q.cgemm(h, Ad, Bd, Cd[:m], m=m, n=n, k=k, alpha=alpha, beta=beta, opA=opA, opB=opB,
            mode="auto", desc_out=desc)
    torch.cuda.synchronize()
    h.sync()
    return host(Cd)[:m, :n], desc.cpu().numpy()


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (37, 19, 40), (300, 200, 170), (64, 1000, 33)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (1, 2), (2, 1), (0, 1)])
def test_line_stats_bit_exact(handles, m, n, k, opA, opB):
    on, _ = handles
    A, B = _line_scaled(m, n, k, opA, opB, 40, (m, n, k, opA, opB), pad=3)
    # a zero line, a subnormal scalar, an Inf (none of which stop the statistics)
    if m > 3:
        if opA == 0:
            A[2, :k] = 0
        else:
            A[:k, 2] = 0
        A[0, 0] = complex(np.float32(3e-41), A[0, 0].imag)
    B[0, 0] = complex(np.inf, 0)
    ea, eb, cnt = lib().rowcol_stats(on, dev(A)[:_stored(opA, m, k)[0]], dev(B)[:_stored(opB, k, n)[0]],
                                     opA=opA, opB=opB)
    wa, wb, wc = oracle.rowcol_stats(A, B, opA, opB, m, n, k)
    assert np.array_equal(ea.cpu().numpy(), wa)
    assert np.array_equal(eb.cpu().numpy(), wb)
    assert np.array_equal(cnt.cpu().numpy(), wc)


@pytest.mark.parametrize("m,n,k", [(130, 70, 33), (257, 129, 100), (128, 256, 64), (9, 6, 700)])
@pytest.mark.parametrize("opA,opB", [(0, 0), (1, 0), (2, 1), (0, 2)])
def test_rowcol_selected_and_matches_model(handles, m, n, k, opA, opB):
    on, _ = handles
    A, B = _line_scaled(m, n, k, opA, opB, 24, (m, n, k, opA, opB), pad=1)
    C0 = qi.cgemm_operand(m, n, 0, seed=(m, 5), ld=m + 1)
    alpha, beta = 0.75 - 0.5j, 0.25 + 1j
    got, d = _run(on, m, n, k, opA, opB, A, B, alpha, beta, C0)
    ea, eb, cnt = oracle.rowcol_stats(A, B, opA, opB, m, n, k)
    want = oracle.select_rowcol(_summ(A, opA, m, k), _summ(B, opB, k, n), cnt, TOL)
    assert tuple(int(v) for v in d[:3]) == want
    assert want[0] == oracle.MODE_FP16X_ROWCOL
    model = oracle.tcec_cgemm_rowcol(ea, eb, opA, opB, m, n, k, alpha, A, B, beta, C0)
    bound = (2 * k + 8) * 2.0 ** -24 * (abs(alpha) * 2 * abs_bound(A, B, opA, opB, m, k, n)
                                        + abs(beta) * 2 * np.abs(C0[:m, :n]))
    bad = np.abs(got.astype(np.complex128) - model) > bound + 1e-30
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], model[bad][:5])


@pytest.mark.parametrize("case", ["fp16x", "fp16x_scaled", "tf32x", "fp32", "ksplit_tf32x"])
def test_other_outcomes_bit_identical(handles, case):
    on, off = handles
    m, n, k = (256, 256, 4096) if case == "ksplit_tf32x" else (200, 150, 96)
    if case == "fp16x":
        A, B = qi.typed_matrix(m, k, 1, 1), qi.typed_matrix(k, n, 1, 2)
    elif case == "fp16x_scaled":
        A, B = qi.typed_matrix(m, k, 2, 3), qi.typed_matrix(k, n, 1, 4)
    else:
        A, B = qi.cgemm_operand(m, k, 20, (len(case), 1)), qi.cgemm_operand(k, n, 20, (len(case), 2))
    if case == "fp32":
        A[3, 4] = complex(np.inf, 0)
    C0 = qi.cgemm_operand(m, n, 0, seed=9)
    got_on, d_on = _run(on, m, n, k, 0, 0, A, B, 0.5 + 0.25j, -1.0, C0)
    got_off, d_off = _run(off, m, n, k, 0, 0, A, B, 0.5 + 0.25j, -1.0, C0)
    name = case.replace("ksplit_", "")
    assert lib().MODE_NAME[int(d_on[0])] == name
    assert np.array_equal(d_on[:3], d_off[:3])
    assert np.array_equal(np.ascontiguousarray(got_on).view(np.uint32),
                          np.ascontiguousarray(got_off).view(np.uint32)) or (
        case == "fp32" and np.array_equal(got_on, got_off, equal_nan=True))


def test_rowcol_error_bar_and_against_tf32x(handles):
    """Line-scaled N(0, 1) at k = 1024: per-row / per-column scaling keeps
    the error at the FP32 level (<= 1e-6, <= 2x plain FP32 on the GPU) where
    Section 4.1 alone selects TF32X."""
    on, off = handles
    q = lib()
    m = n = k = 1024
    A, B = _line_scaled(m, n, k, 0, 0, 30, 77)
    rows = np.arange(0, m, 37)
    exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B, rows=rows)
    got, d = _run(on, m, n, k, 0, 0, A, B)
    assert int(d[0]) == q.MODE_FP16X_ROWCOL
    got_tf, d_tf = _run(off, m, n, k, 0, 0, A, B)
    assert q.MODE_NAME[int(d_tf[0])] == "tf32x"
    Cf = q.cgemm(off, dev(A), dev(B), mode="fp32")
    torch.cuda.synchronize()
    f32 = host(Cf)[rows]
    err = oracle.rel_fro_error(got[rows].astype(np.complex128), exact)
    err_f32 = oracle.rel_fro_error(f32.astype(np.complex128), exact)
    err_tf = oracle.rel_fro_error(got_tf[rows].astype(np.complex128), exact)
    assert err <= 1e-6 and err <= 2 * err_f32, (err, err_f32, err_tf)


def test_invalid_arguments_are_rejected(handles):
    on, _ = handles
    q = lib()
    L = q._lib
    f = on.lib.qcs_rowcol_stats
    buf = torch.zeros(64, dtype=torch.int64, device="cuda")
    P = buf.data_ptr()
    E = L.QCS_ERR_INVALID_ARG
    assert on.lib.qcs_set_rowcol_scaling(on.ptr, 2) == E
    assert on.lib.qcs_set_rowcol_scaling(None, 1) == E
    assert f(None, 0, 0, 2, 2, 2, P, 2, P, 2, P, P, P) == E
    assert f(on.ptr, 3, 0, 2, 2, 2, P, 2, P, 2, P, P, P) == E      # bad op
    assert f(on.ptr, 0, 0, 4, 2, 2, P, 3, P, 2, P, P, P) == E      # lda < m
    assert f(on.ptr, 0, 1, 2, 4, 2, P, 2, P, 3, P, P, P) == E      # ldb < n for op T
    assert f(on.ptr, 0, 0, 2, 2, 2, P, 2, P, 2, None, P, P) == E   # no emaxA
    assert f(on.ptr, 0, 0, 2, 2, 2, P, 2, P, 2, P, P, None) == E   # no counts
    assert f(on.ptr, 0, 0, -1, 2, 2, P, 2, P, 2, P, P, P) == E
    # a GEMM that reports the per-line mode takes no such mode as an argument
    one, zero = L.qcs_c32(1.0, 0.0), L.qcs_c32(0.0, 0.0)
    assert on.lib.qcs_cgemm(on.ptr, q.MODE_FP16X_ROWCOL, 0, 0, 2, 2, 2, ctypes.byref(one), P, 2,
                            P, 2, ctypes.byref(zero), P, 2, None) == E
