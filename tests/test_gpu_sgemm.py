"""GPU parity of the real GEMM (qcs_sgemm: the SGEMM emulation of Section 2.1
with the automatic selection of Section 4) against the FP64 oracle, through
the C ABI: statistics and selection (the decision compared exactly), the
plain FP32 kernel, the tensor-core kernel in every mode against the exact
emulation model, split K, and the edge cases."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import lib, need_gpu, torch

pytestmark = pytest.mark.gpu


def dev_r(x: np.ndarray):
    """numpy column-major float32 (ld, cols) -> device tensor with the same strides."""
    assert x.dtype == np.float32 and x.flags.f_contiguous
    ld, cols = x.shape
    base = torch.empty((cols, ld), dtype=torch.float32, device="cuda")
    base.copy_(torch.from_numpy(np.ascontiguousarray(x.T)))
    return base.t()


def host_r(t) -> np.ndarray:
    return np.asfortranarray(t.t().contiguous().cpu().numpy().T)


@pytest.fixture(scope="module")
def h():
    need_gpu()
    hd = lib().Handle(tol=0.0, size_rule=False)
    yield hd
    hd.close()


def _shape(op, r, c):
    return (r, c) if op == 0 else (c, r)


def _operands(m, n, k, opA, opB, s, seed, ldpad=0):
    ra, ca = _shape(opA, m, k)
    rb, cb = _shape(opB, k, n)
    A = qi.sgemm_operand(ra, ca, s, (seed, 1), ld=ra + ldpad)
    B = qi.sgemm_operand(rb, cb, s, (seed, 2), ld=rb + ldpad)
    return A, B


def _abs_bound(A, B, opA, opB, m, k, n):
    """(|op(A)| |op(B)|)_ij in FP64: bounds every product term of C_ij."""
    def op(X, o, r, c):
        X = np.abs(X.astype(np.float64))
        return X[:r, :c] if o == 0 else X[:c, :r].T
    return op(A, opA, m, k) @ op(B, opB, k, n)


def _run(h, mode, m, n, k, opA, opB, A, B, alpha=1.0, beta=0.0, C0=None):
    q = lib()
    Ad = dev_r(A)[:(m if opA == 0 else k)]
    Bd = dev_r(B)[:(k if opB == 0 else n)]
    if C0 is not None:
        Cd = dev_r(C0)
    else:
        Cd = q.fortran_empty_real(m, n, ld=m + 2)
        Cd.fill_(float("nan"))
    desc = torch.zeros(4, dtype=torch.int32, device="cuda")
    q.sgemm(h, Ad, Bd, Cd[:m], m=m, n=n, k=k, alpha=alpha, beta=beta, opA=opA, opB=opB,
            mode=mode, desc_out=desc)
    torch.cuda.synchronize()
    h.sync()
    return host_r(Cd)[:m, :n].astype(np.float64), desc.cpu().numpy()


def _want_mode(A, B, opA, opB, m, n, k, tol):
    ra, ca = _shape(opA, m, k)
    rb, cb = _shape(opB, k, n)
    sa = oracle.stats_summary(*oracle.exp_stats_real(np.asfortranarray(A[:ra, :ca])))
    sb = oracle.stats_summary(*oracle.exp_stats_real(np.asfortranarray(B[:rb, :cb])))
    return oracle.select_mode(sa, sb, tol)


# one and several 128-row tiles, one and several 256-column tiles, ragged tails
SHAPES = [(1, 1, 1), (13, 7, 5), (130, 70, 33), (257, 300, 100), (128, 256, 64), (200, 513, 96)]
OPPAIRS = [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0)]


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("opA,opB", OPPAIRS)
def test_sgemm_fp32_matches_oracle(h, m, n, k, opA, opB):
    A, B = _operands(m, n, k, opA, opB, 4, seed=(m, n, k, opA, opB), ldpad=3)
    C0 = qi.sgemm_operand(m, n, 0, seed=5, ld=m + 1)
    alpha, beta = 0.75, -1.25
    got, d = _run(h, "fp32", m, n, k, opA, opB, A, B, alpha, beta, C0)
    assert d[0] == oracle.MODE_FP32
    ref = oracle.sgemm(opA, opB, m, n, k, alpha, A, B, beta, C0)
    bound = (2 * k + 8) * 2.0 ** -24 * (abs(alpha) * _abs_bound(A, B, opA, opB, m, k, n)
                                        + abs(beta) * np.abs(C0[:m, :n]))
    assert np.all(np.abs(got - ref) <= bound + 1e-30)


@pytest.mark.parametrize("mode,kind", [("fp16x", 0), ("tf32x", 1), ("bf16x3", 2)])
@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("opA,opB", OPPAIRS)
def test_sgemm_tc_matches_emulation_model(h, mode, kind, m, n, k, opA, opB):
    A, B = _operands(m, n, k, opA, opB, 0, seed=(m, n, k, opA, opB, kind), ldpad=1)
    alpha = 1.0 if (m + n) % 2 else -0.5
    got, d = _run(h, mode, m, n, k, opA, opB, A, B, alpha)
    assert d[0] == {"fp16x": 1, "tf32x": 3, "bf16x3": 5}[mode]
    model = oracle.tcec_sgemm(kind, 0, 0, opA, opB, m, n, k, alpha, A, B)
    bound = (2 * k + 8) * 2.0 ** -24 * abs(alpha) * 2 * _abs_bound(A, B, opA, opB, m, k, n)
    bad = np.abs(got - model) > bound + 1e-30
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], model[bad][:5])


@pytest.mark.parametrize("m,n,k", [(130, 70, 33), (257, 300, 100)])
def test_sgemm_fp16x_scaled_and_beta(h, m, n, k):
    # tiny inputs that fit FP16 only after scaling; beta != 0 reads C
    A, B = _operands(m, n, k, 0, 1, 6, seed=(m, 7))
    A = np.asfortranarray((A.astype(np.float64) * 2.0 ** -40).astype(np.float32))
    C0 = qi.sgemm_operand(m, n, 0, seed=8)
    C0 = np.asfortranarray((C0.astype(np.float64) * 2.0 ** -40).astype(np.float32))
    got, d = _run(h, "fp16x_scaled", m, n, k, 0, 1, A, B, 1.0, -0.5, C0)
    sa = oracle.stats_summary(*oracle.exp_stats_real(A))
    sb = oracle.stats_summary(*oracle.exp_stats_real(B))
    assert d[0] == oracle.MODE_FP16X_SCALED
    assert (d[1], d[2]) == (14 - sa["e_max"], 14 - sb["e_max"])
    model = oracle.tcec_sgemm(0, int(d[1]), int(d[2]), 0, 1, m, n, k, 1.0, A, B, -0.5, C0)
    bound = (2 * k + 8) * 2.0 ** -24 * (2 * _abs_bound(A, B, 0, 1, m, k, n)
                                        + 0.5 * np.abs(C0[:m, :n]))
    assert np.all(np.abs(got - model) <= bound + 1e-45)
    exact = oracle.sgemm(0, 1, m, n, k, 1.0, A, B, -0.5, C0)
    assert oracle.rel_fro_error(got, exact) < 1e-6


@pytest.mark.parametrize("s", [0, 8, 20, 40])
@pytest.mark.parametrize("tol", [0.0, 0.5])
def test_sgemm_auto_picks_oracle_mode(h, s, tol):
    m, n, k = 200, 300, 96
    A, B = _operands(m, n, k, 0, 1, s, seed=(s, 11))
    h.set_tol(tol)
    try:
        got, d = _run(h, "auto", m, n, k, 0, 1, A, B)
    finally:
        h.set_tol(0.0)
    assert tuple(int(v) for v in d[:3]) == _want_mode(A, B, 0, 1, m, n, k, tol)
    exact = oracle.sgemm(0, 1, m, n, k, 1.0, A, B)
    assert oracle.rel_fro_error(got, exact) < 1e-6


@pytest.mark.parametrize("drain", [1, 4])
def test_sgemm_error_bars_unit_inputs(h, drain):
    """FP32-level accuracy on U(-1, 1) inputs with k = 4096: each emulated
    mode within 1e-6 relative of FP64 and within twice the plain FP32
    kernel's error (Section 2.1)."""
    m, n, k = 256, 512, 4096
    g = np.random.default_rng(21)
    A = np.asfortranarray(g.uniform(-1, 1, (m, k)).astype(np.float32))
    B = np.asfortranarray(g.uniform(-1, 1, (k, n)).astype(np.float32))
    exact = oracle.sgemm(0, 0, m, n, k, 1.0, A, B)
    h.set_drain_stages(drain)
    try:
        err32 = oracle.rel_fro_error(_run(h, "fp32", m, n, k, 0, 0, A, B)[0], exact)
        for mode in ("fp16x", "tf32x"):
            err = oracle.rel_fro_error(_run(h, mode, m, n, k, 0, 0, A, B)[0], exact)
            assert err < 1e-6 and err <= 2 * err32, (mode, err, err32)
    finally:
        h.set_drain_stages(4)


@pytest.mark.parametrize("splits", [2, 5])
def test_sgemm_split_k_matches_emulation_model(h, splits):
    m, n, k = 300, 520, 700
    A, B = _operands(m, n, k, 0, 0, 0, seed=(splits, 13))
    h.set_tc_splits(splits)
    try:
        got, d = _run(h, "fp16x", m, n, k, 0, 0, A, B, -0.5, 0.0)
        C0 = qi.sgemm_operand(m, n, 0, seed=14)
        got_b, _ = _run(h, "tf32x", m, n, k, 0, 0, A, B, 1.0, 0.25, C0)
    finally:
        h.set_tc_splits(0)
    model = oracle.tcec_sgemm(0, 0, 0, 0, 0, m, n, k, -0.5, A, B)
    bound = (2 * k + 8) * 2.0 ** -24 * 0.5 * 2 * _abs_bound(A, B, 0, 0, m, k, n)
    assert np.all(np.abs(got - model) <= bound)
    model_b = oracle.tcec_sgemm(1, 0, 0, 0, 0, m, n, k, 1.0, A, B, 0.25, C0)
    bound_b = (2 * k + 8) * 2.0 ** -24 * (2 * _abs_bound(A, B, 0, 0, m, k, n)
                                          + 0.25 * np.abs(C0[:m, :n]))
    assert np.all(np.abs(got_b - model_b) <= bound_b)


def test_sgemm_nonfinite_routes_to_fp32(h):
    m, n, k = 64, 300, 40
    A, B = _operands(m, n, k, 0, 0, 0, seed=15)
    A[3, 4] = np.inf
    got, d = _run(h, "auto", m, n, k, 0, 0, A, B)
    assert d[0] == oracle.MODE_FP32
    ref = oracle.sgemm(0, 0, m, n, k, 1.0, A, B)
    fin = np.isfinite(ref)
    assert np.allclose(got[fin], ref[fin], rtol=1e-5, atol=1e-4)
    assert np.array_equal(np.isinf(got), np.isinf(ref))


def test_sgemm_k_zero_and_empty_outputs(h):
    m, n = 70, 260
    C0 = qi.sgemm_operand(m, n, 0, seed=16)
    A = np.zeros((m, 1), dtype=np.float32, order="F")
    B = np.zeros((1, n), dtype=np.float32, order="F")
    for mode in ("auto", "fp16x", "fp32"):
        got, _ = _run(h, mode, m, n, 0, 0, 0, A, B, 1.0, -2.0, C0)
        assert np.array_equal(got, -2.0 * C0.astype(np.float64))
    q = lib()
    E = q.fortran_empty_real(0, 5)
    C = q.sgemm(h, E, dev_r(np.zeros((5, 3), dtype=np.float32, order="F")), mode="fp16x")
    assert tuple(C.shape) == (0, 3)


def test_sgemm_invalid_arguments_are_rejected(h):
    import ctypes

    from paper_2303_08989_gb300 import _lib as L

    q = lib()
    A = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    one = ctypes.c_float(1.0)
    P = ctypes.c_void_p(A.data_ptr())
    f = h.lib.qcs_sgemm
    ok = L.QCS_SUCCESS
    assert f(h.ptr, 9, 0, 0, 8, 8, 8, ctypes.byref(one), P, 8, P, 8, ctypes.byref(one), P, 8, None) == L.QCS_ERR_INVALID_ARG
    assert f(h.ptr, 0, 5, 0, 8, 8, 8, ctypes.byref(one), P, 8, P, 8, ctypes.byref(one), P, 8, None) == L.QCS_ERR_INVALID_ARG
    assert f(h.ptr, 0, 0, 0, 8, 8, 8, ctypes.byref(one), P, 4, P, 8, ctypes.byref(one), P, 8, None) == L.QCS_ERR_INVALID_ARG
    assert f(h.ptr, 0, 0, 0, -1, 8, 8, ctypes.byref(one), P, 8, P, 8, ctypes.byref(one), P, 8, None) == L.QCS_ERR_INVALID_ARG
    assert f(h.ptr, 0, 0, 0, 8, 8, 8, None, P, 8, P, 8, ctypes.byref(one), P, 8, None) == L.QCS_ERR_INVALID_ARG
    odd = ctypes.c_void_p(A.data_ptr() + 2)
    assert f(h.ptr, 0, 0, 0, 2, 2, 2, ctypes.byref(one), odd, 2, P, 2, ctypes.byref(one), P, 2, None) == L.QCS_ERR_UNSUPPORTED
    # m = 0: nothing to do, whatever the pointers
    assert f(h.ptr, 0, 0, 0, 0, 8, 8, ctypes.byref(one), None, 1, None, 8, ctypes.byref(one), None, 1, None) == ok
    with pytest.raises(TypeError):
        q.sgemm(h, A.to(torch.complex64), A)


def test_sgemm_full_size_sampled_rows(h):
    """8192^3 AUTO-0.1 under the paper's size rule: 64 sampled output rows
    against the FP64 oracle, and the selection against the oracle's."""
    m = n = k = 8192
    A = qi.sgemm_operand(m, k, 8, (8192, 1))
    B = qi.sgemm_operand(k, n, 8, (8192, 2))
    hd = lib().Handle(tol=0.1)
    try:
        q = lib()
        Ad, Bd = dev_r(A), dev_r(B)
        C = q.fortran_empty_real(m, n)
        desc = torch.zeros(4, dtype=torch.int32, device="cuda")
        q.sgemm(hd, Ad, Bd, C, mode="auto", desc_out=desc)
        torch.cuda.synchronize()
        hd.sync()
        d = desc.cpu().numpy()
        assert tuple(int(v) for v in d[:3]) == _want_mode(A, B, 0, 0, m, n, k, 0.1)
        rows = np.random.default_rng(17).choice(m, 64, replace=False)
        got = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
        ref = oracle.sgemm(0, 0, m, n, k, 1.0, A, B, rows=rows)
        assert oracle.rel_fro_error(got, ref) < 1e-6
    finally:
        hd.close()
