"""The counts of Section 4.1 that the GEMM path's own statistics kernels
(stats_pass1, stats_pass2, select2 -- the hot path, not the histogram of
qcs_exp_stats) hand to the selection, compared count by count with the
oracle's: e_max, nonzero, Inf/NaN, below 2^-14 (N - N1) and, when pass 2
runs, below the shifted window (N - N2); pass 2 must run exactly when the
pass-1 counts leave the mode undecided, and the descriptor must equal the
oracle's selection.  Inputs cover the sweep's exponent spreads, the paper's
Type-1/2/3 matrices, zeros, Inf/NaN, binary32 subnormals, magnitudes above
FP16's range, window edges, op T / op C and leading dimensions > rows."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import dev, lib, need_gpu, torch

pytestmark = pytest.mark.gpu


def _oracle_counts(X):
    return oracle.stats_summary(*oracle.exp_stats(X))


def _expect_stage2(sa, sb, tol):
    if sa["nonfinite"] or sb["nonfinite"]:
        return False
    if any(s["e_max"] is not None and s["e_max"] >= 127 for s in (sa, sb)):
        return False

    def ok1(s):
        return s["e_max"] is None or (s["e_max"] <= 14 and s["under1"] <= tol * s["nnz"])

    return not (ok1(sa) and ok1(sb))


def _check(A, B, opA, opB, tol, ldpad=0):
    q = lib()
    h = q.Handle(tol=tol, size_rule=False)
    try:
        def put(X):
            if ldpad == 0:
                return dev(X)
            ld, cols = X.shape
            base = torch.zeros((cols, ld + ldpad), dtype=torch.complex64, device="cuda")
            base[:, :ld] = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
            return base.t()[:ld]
        got, desc = q.selection_stats(h, put(A), put(B), opA=opA, opB=opB)
    finally:
        h.close()
    sa, sb = _oracle_counts(A), _oracle_counts(B)
    stage2 = _expect_stage2(sa, sb, tol)
    for g, s in zip(got, (sa, sb)):
        assert g["e_max"] == s["e_max"]
        assert g["n_nonzero"] == s["nnz"]
        assert g["n_nonfinite"] == s["nonfinite"]
        assert g["n_under_fp16"] == s["under1"]
        assert g["stage2"] == stage2
        if stage2:
            assert g["n_under_window"] == s["under2"]
    assert desc == oracle.select_mode(sa, sb, tol)
    return got, desc


@pytest.mark.parametrize("s", [0, 8, 20, 40])
@pytest.mark.parametrize("tol", [0.0, 0.1, 0.5])
def test_counts_on_the_sweep_distribution(s, tol):
    need_gpu()
    m, n, k = 300, 260, 333  # ragged: no multiple of the block sizes
    A = qi.cgemm_operand(m, k, s, seed=(41, s))
    B = qi.cgemm_operand(k, n, s, seed=(42, s))
    _check(A, B, 0, 0, tol)


@pytest.mark.parametrize("ops", [(1, 0), (2, 2), (0, 1)])
def test_counts_with_transposed_operands_and_padded_ld(ops):
    need_gpu()
    opA, opB = ops
    m, n, k = 129, 257, 77
    A = qi.cgemm_operand(k if opA else m, m if opA else k, 20, seed=(43, 1))
    B = qi.cgemm_operand(n if opB else k, k if opB else n, 20, seed=(43, 2))
    _check(A, B, opA, opB, 0.1, ldpad=3)


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_counts_on_the_papers_typed_matrices(kind):
    need_gpu()
    A = qi.typed_matrix(128, 96, kind, seed=(44, kind))
    B = qi.typed_matrix(96, 112, kind, seed=(45, kind))
    _, desc = _check(A, B, 0, 0, 0.1)
    assert desc[0] == {1: oracle.MODE_FP16X, 2: oracle.MODE_FP16X_SCALED, 3: oracle.MODE_TF32X}[kind]


def test_counts_with_zeros_specials_and_window_edges():
    need_gpu()
    rng = np.random.default_rng(46)
    m, n, k = 200, 150, 180
    A = qi.cgemm_operand(m, k, 4, seed=(46, 1))
    B = qi.cgemm_operand(k, n, 4, seed=(46, 2))
    A = np.asfortranarray(A)
    # zeros, binary32 subnormals, the edges of the FP16 window (2^-14 in,
    # just below out) and of the shifted window
    A.real[rng.integers(0, m, 50), rng.integers(0, k, 50)] = 0.0
    A.imag[:3, :3] = np.float32(2.0 ** -140)
    A.real[5, 5] = np.float32(2.0 ** -14)
    A.real[6, 6] = np.float32(np.nextafter(np.float32(2.0 ** -14), np.float32(0)))
    A.imag[7, 7] = np.float32(2.0 ** 14)
    _check(A, B, 0, 0, 0.0)
    _check(A, B, 0, 0, 0.5)
    # one operand above FP16's range: scaling decides
    B2 = np.asfortranarray(B.copy())
    B2.real[0, 0] = np.float32(2.0 ** 20)
    _check(A, B2, 0, 0, 0.1)
    # an all-zero operand, and a NaN / Inf (plain FP32)
    _check(np.zeros_like(A, order="F"), B, 0, 0, 0.0)
    B3 = np.asfortranarray(B.copy())
    B3.real[1, 1] = np.nan
    B3.imag[2, 2] = np.inf
    _, desc = _check(A, B3, 0, 0, 0.1)
    assert desc[0] == oracle.MODE_FP32


def test_counts_at_full_size():
    """16384^2 operands (2^29 scalars each), the bench's distribution."""
    need_gpu()
    q = lib()
    n = 16384
    g = torch.Generator(device="cuda").manual_seed(47)
    A = torch.randn((n, n), dtype=torch.complex64, device="cuda", generator=g).t()
    B = torch.randn((n, n), dtype=torch.complex64, device="cuda", generator=g).t()
    h = q.Handle(tol=0.0, size_rule=False)
    got, desc = q.selection_stats(h, A, B)
    h.close()
    for X, gs in ((A, got[0]), (B, got[1])):
        v = torch.view_as_real(X)
        mag = v.abs()
        nz = mag > 0
        assert gs["n_nonzero"] == int(nz.sum().item())
        assert gs["n_nonfinite"] == 0
        assert gs["n_under_fp16"] == int(((mag < 2.0 ** -14) & nz).sum().item())
        e_max = int(torch.frexp(mag.max())[1].item()) - 1  # exact floor(log2)
        assert gs["e_max"] == e_max
        if gs["stage2"]:
            assert gs["n_under_window"] == int(((mag < 2.0 ** (e_max - 28)) & nz).sum().item())
    del A, B
    torch.cuda.empty_cache()
