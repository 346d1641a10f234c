"""GPU parity of the emulated-CGEMM path (through the C ABI) against the
FP64 oracle: exponent statistics, selection, split (bit-exact), the plain
FP32 CGEMM and the tensor-core emulated CGEMM in every mode."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import abs_bound, dev, host, lib, need_gpu, torch

pytestmark = pytest.mark.gpu

OPS = {0: "N", 1: "T", 2: "C"}


@pytest.fixture(scope="module")
def h():
    need_gpu()
    q = lib()
    hd = q.Handle(tol=0.0, size_rule=False)
    yield hd
    hd.close()


def _shape(op, r, c):
    return (r, c) if op == 0 else (c, r)


def _operands(m, n, k, opA, opB, s, seed, ldpad=0, uniform=False):
    ra, ca = _shape(opA, m, k)
    rb, cb = _shape(opB, k, n)
    if uniform:
        A = qi.uniform_operand(ra, ca, (seed, 1))
        B = qi.uniform_operand(rb, cb, (seed, 2))
    else:
        A = qi.cgemm_operand(ra, ca, s, (seed, 1), ld=ra + ldpad)
        B = qi.cgemm_operand(rb, cb, s, (seed, 2), ld=rb + ldpad)
    return A, B


# ---------------------------------------------------------------------------
# statistics, selection, split: integer / bitwise results, compared exactly
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("rows,cols,ld,s", [(1, 1, 1, 0), (37, 19, 40, 8), (256, 300, 256, 20),
                                            (1000, 77, 1000, 40), (3, 0, 3, 0)])
def test_exp_stats_bit_exact(h, rows, cols, ld, s):
    X = qi.cgemm_operand(rows, cols, s, seed=(rows, cols), ld=ld)
    if rows * cols:
        X[0, 0] = 0
        X[rows - 1, cols - 1] = complex(np.float32(1e-41), np.inf)
    st = lib().exp_stats(h, dev(X)[:rows]).cpu().numpy()
    hist, nz = oracle.exp_stats(X, rows, cols)
    assert np.array_equal(st[:256], hist)
    assert st[256] == nz and st[257] == 2 * rows * cols


@pytest.mark.parametrize("tol", [0.0, 0.1, 0.5])
def test_select_matches_oracle(h, tol):
    q = lib()
    h.set_tol(tol)
    try:
        cases = [qi.typed_matrix(96, 80, t, (t, 9)) for t in (1, 2, 3)]
        cases += [qi.cgemm_operand(64, 48, s, (s, 3)) for s in (0, 8, 20, 40)]
        for A in cases:
            for B in cases[:3]:
                sa = q.exp_stats(h, dev(A))
                sb = q.exp_stats(h, dev(B))
                d = q.select(h, sa, sb).cpu().numpy()
                want = oracle.select_mode(oracle.stats_summary(*oracle.exp_stats(A)),
                                          oracle.stats_summary(*oracle.exp_stats(B)), tol)
                assert tuple(int(v) for v in d[:3]) == want
    finally:
        h.set_tol(0.0)


@pytest.mark.parametrize("mode,kind", [("fp16x", 0), ("fp16x_scaled", 0), ("tf32x", 1), ("bf16x3", 2)])
@pytest.mark.parametrize("which,op", [(0, 0), (0, 1), (1, 0), (1, 2)])
def test_split_bit_exact(h, mode, kind, which, op):
    q = lib()
    R, K = 70, 45
    rows, cols = (R, K) if (which == 0) == (op == 0) else (K, R)
    X = qi.cgemm_operand(rows, cols, 20 if mode == "fp16x_scaled" else 4, seed=(which, op), ld=rows + 3)
    sA = sB = 0
    if mode == "fp16x_scaled":
        sA, sB = 7, -5
    desc = torch.tensor([q.MODE_BY_NAME[mode], sA, sB, 0], dtype=torch.int32, device="cuda")
    planes = q.split(h, desc, which, op, dev(X)[:rows], R, K).cpu()
    # oracle: op(X) as an R x K array (which 0: op(A)[i, l]; which 1: op(B)[l, j] transposed)
    Xc = X[:rows, :cols].astype(np.complex64)
    if which == 0:
        M = Xc if op == 0 else (Xc.T if op == 1 else Xc.conj().T)
    else:
        M = Xc.T if op == 0 else (Xc if op == 1 else Xc.conj())
    s = sA if which == 0 else sB
    hr, lr = oracle.split(kind, s, np.ascontiguousarray(M.real))
    hi_, li = oracle.split(kind, s, np.ascontiguousarray(M.imag))
    if kind == 1:
        got = planes.numpy().astype(np.float32)
        want = np.stack([hr, hi_, lr, li])
        assert np.array_equal(got.view(np.uint32), want.astype(np.float32).view(np.uint32))
    else:
        got = planes.numpy().view(np.uint16)
        if kind == 0:
            enc = lambda v: v.astype(np.float16).view(np.uint16)
        else:
            enc = lambda v: (v.astype(np.float32).view(np.uint32) >> 16).astype(np.uint16)
        want = np.stack([enc(hr), enc(hi_), enc(lr), enc(li)])
        assert np.array_equal(got, want)


# ---------------------------------------------------------------------------
# CGEMM parity
# ---------------------------------------------------------------------------

SHAPES = [(1, 1, 1), (13, 7, 5), (130, 70, 33), (257, 129, 100), (128, 256, 64)]
OPPAIRS = [(0, 0), (1, 0), (2, 1), (0, 2), (1, 2)]


def _run(h, mode, m, n, k, opA, opB, A, B, alpha=1.0, beta=0.0, C0=None):
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
            mode=mode, desc_out=desc)
    torch.cuda.synchronize()
    h.sync()
    return host(Cd)[:m, :n].astype(np.complex128), desc.cpu().numpy()


@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("opA,opB", OPPAIRS)
def test_cgemm_fp32_matches_oracle(h, m, n, k, opA, opB):
    A, B = _operands(m, n, k, opA, opB, 4, seed=(m, n, k, opA, opB), ldpad=3)
    C0 = qi.cgemm_operand(m, n, 0, seed=5, ld=m + 1)
    alpha, beta = 0.75 - 0.5j, 0.25 + 1j
    got, d = _run(h, "fp32", m, n, k, opA, opB, A, B, alpha, beta, C0)
    assert d[0] == oracle.MODE_FP32
    ref = oracle.cgemm(opA, opB, m, n, k, alpha, A, B, beta, C0)
    bound = (2 * k + 8) * 2.0 ** -24 * (abs(alpha) * 2 * abs_bound(A, B, opA, opB, m, k, n)
                                        + abs(beta) * 2 * np.abs(C0[:m, :n]))
    assert np.all(np.abs(got - ref) <= bound + 1e-30)


@pytest.mark.parametrize("mode,kind", [("fp16x", 0), ("tf32x", 1), ("bf16x3", 2)])
@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("opA,opB", OPPAIRS)
def test_cgemm_tc_matches_emulation_model(h, mode, kind, m, n, k, opA, opB):
    A, B = _operands(m, n, k, opA, opB, 0, seed=(m, n, k, opA, opB, kind), ldpad=1)
    alpha, beta = (1.0, 0.0) if (m + n) % 2 else (0.5 + 0.25j, 0.0)
    got, d = _run(h, mode, m, n, k, opA, opB, A, B, alpha, beta)
    assert d[0] == {"fp16x": 1, "tf32x": 3, "bf16x3": 5}[mode]
    model = oracle.tcec_cgemm(kind, 0, 0, opA, opB, m, n, k, alpha, A, B)
    bound = (2 * k + 8) * 2.0 ** -24 * abs(alpha) * 2 * abs_bound(A, B, opA, opB, m, k, n)
    bad = np.abs(got - model) > bound + 1e-30
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], model[bad][:5])


@pytest.mark.parametrize("m,n,k", [(130, 70, 33), (257, 129, 100)])
def test_cgemm_fp16x_scaled_and_beta(h, m, n, k):
    # tiny inputs that only fit FP16 after scaling; beta != 0 exercises the C read
    A, B = _operands(m, n, k, 0, 1, 6, seed=(m, 7))
    A = np.asfortranarray((A.astype(np.complex128) * 2.0 ** -40).astype(np.complex64))
    C0 = qi.cgemm_operand(m, n, 0, seed=8)
    C0 = np.asfortranarray((C0.astype(np.complex128) * 2.0 ** -40).astype(np.complex64))
    got, d = _run(h, "fp16x_scaled", m, n, k, 0, 1, A, B, 1.0, -0.5j, C0)
    sa = oracle.stats_summary(*oracle.exp_stats(A))
    sb = oracle.stats_summary(*oracle.exp_stats(B))
    assert d[0] == oracle.MODE_FP16X_SCALED
    assert (d[1], d[2]) == (14 - sa["e_max"], 14 - sb["e_max"])
    exact = oracle.cgemm(0, 1, m, n, k, 1.0, A, B, -0.5j, C0)
    assert oracle.rel_fro_error(got, exact) < 1e-6


@pytest.mark.parametrize("s", [0, 8, 20, 40])
@pytest.mark.parametrize("tol", [0.0, 0.5])
def test_cgemm_auto_picks_oracle_mode(h, s, tol):
    m, n, k = 200, 150, 96
    A, B = _operands(m, n, k, 0, 0, s, seed=(s, 11))
    h.set_tol(tol)
    try:
        got, d = _run(h, "auto", m, n, k, 0, 0, A, B)
    finally:
        h.set_tol(0.0)
    want = oracle.select_mode(oracle.stats_summary(*oracle.exp_stats(A)),
                              oracle.stats_summary(*oracle.exp_stats(B)), tol)
    assert tuple(int(v) for v in d[:3]) == want
    exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
    assert oracle.rel_fro_error(got, exact) < 1e-6


@pytest.mark.parametrize("drain", [1, 2, 4])
def test_cgemm_error_bars_unit_inputs(h, drain):
    """FP32-level accuracy: U(-1,1) inputs, k = 4096 (Section 3 unit test):
    relative Frobenius error <= 1e-6 and <= 2x the plain FP32 GPU error, for
    every round-to-nearest drain interval."""
    m, n, k = 256, 192, 4096
    A, B = _operands(m, n, k, 0, 0, 0, seed=42, uniform=True)
    exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
    e32 = oracle.rel_fro_error(_run(h, "fp32", m, n, k, 0, 0, A, B)[0], exact)
    h.set_drain_stages(drain)
    try:
        for mode in ("fp16x", "tf32x", "auto"):
            e = oracle.rel_fro_error(_run(h, mode, m, n, k, 0, 0, A, B)[0], exact)
            assert e <= 1e-6 and e <= 2 * e32, (mode, e, e32)
    finally:
        h.set_drain_stages(4)


def test_nonfinite_inputs_route_to_fp32(h):
    m, n, k = 64, 64, 64
    A, B = _operands(m, n, k, 0, 0, 0, seed=3)
    A[5, 7] = complex(np.nan, 0)
    got, d = _run(h, "auto", m, n, k, 0, 0, A, B)
    assert d[0] == oracle.MODE_FP32
    assert np.isnan(got[5]).all() and np.isfinite(np.delete(got, 5, axis=0)).all()


def test_k_zero_scales_c(h):
    m, n = 9, 4
    C0 = qi.cgemm_operand(m, n, 0, seed=1)
    A = np.zeros((m, 1), np.complex64, order="F")
    B = np.zeros((1, n), np.complex64, order="F")
    got, _ = _run(h, "fp16x", m, n, 0, 0, 0, A, B, 1.0, 2.0, C0)
    assert np.array_equal(got, 2.0 * C0.astype(np.complex128))


def test_invalid_arguments_are_rejected(h):
    q = lib()
    import ctypes

    from paper_2303_08989_gb300 import _lib as L

    A = torch.zeros(16, dtype=torch.complex64, device="cuda")
    one = L.qcs_c32(1, 0)
    zero = L.qcs_c32(0, 0)
    P = ctypes.c_void_p(A.data_ptr())
    f = h.lib.qcs_cgemm
    assert f(h.ptr, 9, 0, 0, 2, 2, 2, ctypes.byref(one), P, 2, P, 2, ctypes.byref(zero), P, 2, None) == L.QCS_ERR_INVALID_ARG
    assert f(h.ptr, 0, 3, 0, 2, 2, 2, ctypes.byref(one), P, 2, P, 2, ctypes.byref(zero), P, 2, None) == L.QCS_ERR_INVALID_ARG
    assert f(h.ptr, 0, 0, 0, 4, 2, 2, ctypes.byref(one), P, 3, P, 2, ctypes.byref(zero), P, 4, None) == L.QCS_ERR_INVALID_ARG
    assert f(h.ptr, 0, 0, 0, -1, 2, 2, ctypes.byref(one), P, 3, P, 2, ctypes.byref(zero), P, 4, None) == L.QCS_ERR_INVALID_ARG
    assert f(h.ptr, 0, 0, 0, 2, 2, 2, None, P, 2, P, 2, ctypes.byref(zero), P, 2, None) == L.QCS_ERR_INVALID_ARG
    odd = ctypes.c_void_p(A.data_ptr() + 4)
    assert f(h.ptr, 0, 0, 0, 2, 2, 2, ctypes.byref(one), odd, 2, P, 2, ctypes.byref(zero), P, 2, None) == L.QCS_ERR_UNSUPPORTED
    assert h.lib.qcs_set_underflow_tol(h.ptr, 1.5) == L.QCS_ERR_INVALID_ARG
    del q


@pytest.mark.parametrize("m,n,k,opA,opB", [(1, 1, 100000, 0, 0), (4, 4, 50000, 1, 2),
                                           (16, 3, 70000, 2, 0), (64, 64, 4096, 0, 1)])
def test_cgemm_fp32_split_k_small_outputs(h, m, n, k, opA, opB):
    """End-of-tree reductions: few outputs, long k (split over warps)."""
    A, B = _operands(m, n, k, opA, opB, 2, seed=(m, n, k))
    C0 = qi.cgemm_operand(m, n, 0, seed=4)
    got, d = _run(h, "fp32", m, n, k, opA, opB, A, B, 1.5 - 0.5j, 0.5j, C0)
    ref = oracle.cgemm(opA, opB, m, n, k, 1.5 - 0.5j, A, B, 0.5j, C0)
    bound = (2 * k + 8) * 2.0 ** -24 * (1.6 * 2 * abs_bound(A, B, opA, opB, m, k, n)
                                        + 0.5 * 2 * np.abs(C0[:m, :n]))
    # the element-wise FP32 bound: a single long dot product cancels too much for a
    # relative-error bar to apply to it
    assert np.all(np.abs(got - ref) <= bound)


@pytest.mark.parametrize("m,n,k,opA,opB", [(2, 5000, 2, 0, 0), (5000, 2, 2, 0, 0), (3, 1000, 16, 1, 2),
                                           (1000, 16, 7, 2, 1), (16, 16, 16, 0, 1), (2048, 300, 8, 0, 0),
                                           (50, 60, 40, 1, 0), (300, 5000, 3, 1, 2), (40, 2000, 16, 2, 1),
                                           (100, 130, 12, 0, 1), (517, 4099, 5, 0, 0), (17, 700, 9, 1, 0),
                                           # 16 < k <= 32 with m <= 64: the small-k kernel's 32-register form
                                           (64, 4096, 32, 0, 0), (40, 5003, 17, 1, 2), (33, 2000, 24, 2, 1),
                                           (20, 9000, 31, 0, 1)])
def test_cgemm_fp32_skinny_and_per_element_shapes(h, m, n, k, opA, opB):
    """The bandwidth-bound FP32 kernels of Section 5.1.2's irregular shapes."""
    A, B = _operands(m, n, k, opA, opB, 3, seed=(m, n, k, 9), ldpad=2)
    C0 = qi.cgemm_operand(m, n, 0, seed=6, ld=m + 1)
    alpha, beta = 0.5 + 1j, -0.25
    got, d = _run(h, "fp32", m, n, k, opA, opB, A, B, alpha, beta, C0)
    ref = oracle.cgemm(opA, opB, m, n, k, alpha, A, B, beta, C0)
    bound = (2 * k + 8) * 2.0 ** -24 * (abs(alpha) * 2 * abs_bound(A, B, opA, opB, m, k, n)
                                        + abs(beta) * 2 * np.abs(C0[:m, :n]))
    assert np.all(np.abs(got - ref) <= bound + 1e-30)


@pytest.mark.parametrize("n", [1, 7, 5000, 65539])
@pytest.mark.parametrize("opA", [0, 1, 2])
def test_cgemm_fp32_two_by_n_columns(h, n, opA):
    """The (2, 2^N, 2) shape of Section 5.1.2 with B and C stored contiguous
    (a column of each is 16 bytes): the column-vector kernel."""
    m, k = 2, 2
    A = _operands(m, n, k, opA, 0, 3, seed=(n, opA, 1))[0]
    B = qi.cgemm_operand(k, n, 3, seed=(n, opA, 2))
    C0 = qi.cgemm_operand(m, n, 0, seed=(n, 6))
    alpha, beta = 0.5 + 0.25j, -1.0 + 0.5j
    q = lib()
    Cd = dev(C0)
    assert Cd.stride(1) == 2
    q.cgemm(h, dev(A)[:(m if opA == 0 else k)], dev(B), Cd, m=m, n=n, k=k, alpha=alpha,
            beta=beta, opA=opA, mode="fp32")
    torch.cuda.synchronize()
    h.sync()
    got = host(Cd).astype(np.complex128)
    ref = oracle.cgemm(opA, 0, m, n, k, alpha, A, B, beta, C0)
    bound = (2 * k + 8) * 2.0 ** -24 * (abs(alpha) * 2 * abs_bound(A, B, opA, 0, m, k, n)
                                        + abs(beta) * 2 * np.abs(C0[:m, :n]))
    assert np.all(np.abs(got - ref) <= bound + 1e-30)


@pytest.mark.parametrize("m", [2, 3, 7, 5000, 65539])
@pytest.mark.parametrize("opB", [0, 1, 2])
@pytest.mark.parametrize("pad", [0, 1])
def test_cgemm_fp32_n_by_two_rows(h, m, opB, pad):
    """The (2^N, 2, 2) shape of Section 5.1.2: A and C stored m x 2 with an
    even leading dimension (the paired-row kernel, odd m included: its last
    row is done alone) or an odd one (the per-row kernel), beta != 0."""
    n = k = 2
    ld = m + (m & 1)                       # even
    lda = m + 1 - (m & 1) if pad else ld   # odd with pad
    A = qi.cgemm_operand(m, k, 3, seed=(m, opB, 1), ld=lda)
    B = _operands(m, n, k, 0, opB, 3, seed=(m, opB, 2))[1]
    C0 = qi.cgemm_operand(m, n, 0, seed=(m, 6), ld=ld)
    alpha, beta = 0.5 + 0.25j, -1.0 + 0.5j
    got, _ = _run(h, "fp32", m, n, k, 0, opB, A, B, alpha, beta, C0)
    ref = oracle.cgemm(0, opB, m, n, k, alpha, A, B, beta, C0)
    bound = (2 * k + 8) * 2.0 ** -24 * (abs(alpha) * 2 * abs_bound(A, B, 0, opB, m, k, n)
                                        + abs(beta) * 2 * np.abs(C0[:m, :n]))
    assert np.all(np.abs(got - ref) <= bound + 1e-30)


# ---------------------------------------------------------------------------
# K ranges as separate work units (qcs_set_tc_splits)
# ---------------------------------------------------------------------------

def _model_bound(kind, sA, sB, m, n, k, opA, opB, A, B, alpha, beta, C0):
    model = oracle.tcec_cgemm(kind, sA, sB, opA, opB, m, n, k, alpha, A, B, beta, C0)
    bound = (2 * k + 8) * 2.0 ** -24 * (abs(alpha) * 2 * abs_bound(A, B, opA, opB, m, k, n)
                                        + abs(beta) * 2 * np.abs(C0[:m, :n]))
    return model, bound


@pytest.mark.parametrize("mode,kind", [("fp16x", 0), ("tf32x", 1), ("bf16x3", 2)])
@pytest.mark.parametrize("m,n,k,splits", [(257, 129, 100, 2), (130, 70, 1000, 5), (300, 40, 513, 16),
                                          (128, 256, 64, 3), (13, 7, 5, 4)])
def test_cgemm_tc_split_k_matches_emulation_model(h, mode, kind, m, n, k, splits):
    """Each K range's partial and their fixed-order sum stay inside the FP32
    bound of the emulation model; alpha and beta are applied once, by the
    reduction.  (128, 256, 64) asks for 3 ranges of 2 stages: capped at 2;
    (13, 7, 5) has one stage: no split."""
    opA, opB = (1, 2) if splits % 2 else (0, 0)
    A, B = _operands(m, n, k, opA, opB, 0, seed=(m, n, k, splits, kind), ldpad=1)
    C0 = qi.cgemm_operand(m, n, 0, seed=(splits, 3), ld=m + 1)
    alpha, beta = 0.5 + 0.25j, -0.75 + 0.5j
    h.set_tc_splits(splits)
    try:
        got, d = _run(h, mode, m, n, k, opA, opB, A, B, alpha, beta, C0)
    finally:
        h.set_tc_splits(0)
    assert d[0] == {"fp16x": 1, "tf32x": 3, "bf16x3": 5}[mode]
    model, bound = _model_bound(kind, 0, 0, m, n, k, opA, opB, A, B, alpha, beta, C0)
    bad = np.abs(got - model) > bound + 1e-30
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], model[bad][:5])


@pytest.mark.parametrize("s,tol,kind", [(0, 0.5, 0), (20, 0.0, 1), (8, 0.001, 0)])
def test_cgemm_tc_split_k_under_auto(h, s, tol, kind):
    """AUTO launches every candidate: with split K the selected kind writes the
    partials and the reduction (gated by the descriptor) forms C.  One output
    tile and long k: the per-shape choice splits (the count is not forced)."""
    m, n, k = 128, 96, 2048
    A, B = _operands(m, n, k, 0, 0, s, seed=(s, 21))
    C0 = qi.cgemm_operand(m, n, 0, seed=(s, 22))
    h.set_tol(tol)
    try:
        got, d = _run(h, "auto", m, n, k, 0, 0, A, B, 1.0, 0.5, C0)
    finally:
        h.set_tol(0.0)
    want = oracle.select_mode(oracle.stats_summary(*oracle.exp_stats(A)),
                              oracle.stats_summary(*oracle.exp_stats(B)), tol)
    assert tuple(int(v) for v in d[:3]) == want
    assert {1: 0, 2: 0, 3: 1}[int(d[0])] == kind
    model, bound = _model_bound(kind, int(d[1]), int(d[2]), m, n, k, 0, 0, A, B, 1.0, 0.5, C0)
    assert np.all(np.abs(got - model) <= bound + 1e-30)


def test_cgemm_tc_split_k_leaves_fp32_result(h):
    """A GEMM that AUTO sends to FP32 (a NaN input): the gated reduction must
    not overwrite the SIMT kernel's output."""
    m, n, k = 128, 64, 1024
    A, B = _operands(m, n, k, 0, 0, 0, seed=23)
    A[3, 9] = complex(np.nan, 0)
    h.set_tc_splits(8)
    try:
        got, d = _run(h, "auto", m, n, k, 0, 0, A, B)
    finally:
        h.set_tc_splits(0)
    assert d[0] == oracle.MODE_FP32
    assert np.isnan(got[3]).all() and np.isfinite(np.delete(got, 3, axis=0)).all()
    ref = oracle.cgemm(0, 0, m, n, k, 1.0, np.where(np.isnan(A), 0, A), B)
    keep = np.delete(np.arange(m), 3)
    assert oracle.rel_fro_error(got[keep], ref[keep]) < 1e-5


def test_set_tc_splits_rejects_out_of_range(h):
    from paper_2303_08989_gb300 import _lib as L

    assert h.lib.qcs_set_tc_splits(h.ptr, -1) == L.QCS_ERR_INVALID_ARG
    assert h.lib.qcs_set_tc_splits(h.ptr, 17) == L.QCS_ERR_INVALID_ARG
    assert h.lib.qcs_set_tc_splits(h.ptr, 0) == 0
