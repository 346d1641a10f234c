"""GPU parity of Gauss's three-product CGEMM (qcs_set_complex_products 3, a
variant beyond the paper: three emulated real GEMMs T1 = Ar Br, T2 = Ai Bi,
T3 = (Ar + Ai)(Br + Bi) in one grouped tensor-core launch, Re = T1 - T2,
Im = T3 - T1 - T2) against the oracle's exact three-product model and FP64,
through the C ABI."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import abs_bound, dev, host, lib, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    need_gpu()
    hd = lib().Handle(tol=0.0, size_rule=False)
    hd.set_complex_products(3)
    yield hd
    hd.close()


def _shape(op, r, c):
    return (r, c) if op == 0 else (c, r)


def _operands(m, n, k, opA, opB, s, seed, ldpad=0):
    ra, ca = _shape(opA, m, k)
    rb, cb = _shape(opB, k, n)
    A = qi.cgemm_operand(ra, ca, s, (seed, 1), ld=ra + ldpad)
    B = qi.cgemm_operand(rb, cb, s, (seed, 2), ld=rb + ldpad)
    return A, B


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


SHAPES = [(1, 1, 1), (13, 7, 5), (130, 70, 33), (257, 300, 100), (200, 513, 96)]
OPPAIRS = [(0, 0), (1, 0), (2, 1), (0, 2), (1, 2)]
KIND = {"fp16x": 0, "fp16x_scaled": 0, "tf32x": 1, "bf16x3": 2}


@pytest.mark.parametrize("mode", ["fp16x", "tf32x", "bf16x3"])
@pytest.mark.parametrize("m,n,k", SHAPES)
@pytest.mark.parametrize("opA,opB", OPPAIRS)
def test_3m_matches_three_product_model(h, mode, m, n, k, opA, opB):
    A, B = _operands(m, n, k, opA, opB, 0, seed=(m, n, k, opA, opB, KIND[mode], 3), ldpad=1)
    alpha = 1.0 if (m + n) % 2 else 0.5 + 0.25j
    got, d = _run(h, mode, m, n, k, opA, opB, A, B, alpha)
    assert d[0] == {"fp16x": 1, "tf32x": 3, "bf16x3": 5}[mode]
    model = oracle.tcec_cgemm_3m(KIND[mode], 0, 0, opA, opB, m, n, k, alpha, A, B)
    # T1, T2, T3 each within k truncating adds of their |.| sums (all bounded
    # by the |re| + |im| product), then three binary32 combination steps
    bound = (2 * k + 16) * 2.0 ** -24 * abs(alpha) * 4 * abs_bound(A, B, opA, opB, m, k, n)
    bad = np.abs(got - model) > bound + 1e-30
    assert not bad.any(), (np.argwhere(bad)[:5], got[bad][:5], model[bad][:5])


@pytest.mark.parametrize("m,n,k", [(130, 70, 33), (257, 300, 100)])
def test_3m_fp16x_scaled_and_beta(h, m, n, k):
    A, B = _operands(m, n, k, 0, 1, 6, seed=(m, 17))
    A = np.asfortranarray((A.astype(np.complex128) * 2.0 ** -40).astype(np.complex64))
    C0 = qi.cgemm_operand(m, n, 0, seed=18)
    C0 = np.asfortranarray((C0.astype(np.complex128) * 2.0 ** -40).astype(np.complex64))
    got, d = _run(h, "fp16x_scaled", m, n, k, 0, 1, A, B, 1.0, -0.5j, C0)
    sa = oracle.stats_summary(*oracle.exp_stats(A))
    sb = oracle.stats_summary(*oracle.exp_stats(B))
    assert d[0] == oracle.MODE_FP16X_SCALED
    assert (d[1], d[2]) == (14 - sa["e_max"], 14 - sb["e_max"])
    model = oracle.tcec_cgemm_3m(0, int(d[1]), int(d[2]), 0, 1, m, n, k, 1.0, A, B, -0.5j, C0)
    bound = (2 * k + 16) * 2.0 ** -24 * (4 * abs_bound(A, B, 0, 1, m, k, n)
                                         + 2 * 0.5 * np.abs(C0[:m, :n]))
    assert np.all(np.abs(got - model) <= bound + 1e-45)
    exact = oracle.cgemm(0, 1, m, n, k, 1.0, A, B, -0.5j, C0)
    assert oracle.rel_fro_error(got, exact) < 1e-6


@pytest.mark.parametrize("s", [0, 8, 20])
def test_3m_auto_selection_and_error(h, s):
    m, n, k = 200, 300, 96
    A, B = _operands(m, n, k, 0, 0, s, seed=(s, 19))
    h.set_tol(0.5)
    try:
        got, d = _run(h, "auto", m, n, k, 0, 0, A, B)
    finally:
        h.set_tol(0.0)
    want = oracle.select_mode(oracle.stats_summary(*oracle.exp_stats(A)),
                              oracle.stats_summary(*oracle.exp_stats(B)), 0.5)
    assert tuple(int(v) for v in d[:3]) == want
    exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
    assert oracle.rel_fro_error(got, exact) < 1e-6


def test_3m_error_bars_unit_inputs(h):
    """U(-1,1) parts, k = 4096: each emulated mode within 1e-6 of FP64 and
    within twice the plain FP32 kernel's error, as the four-product form."""
    m, n, k = 256, 256, 4096
    A = qi.uniform_operand(m, k, 22)
    B = qi.uniform_operand(k, n, 23)
    exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
    err32 = oracle.rel_fro_error(_run(h, "fp32", m, n, k, 0, 0, A, B)[0], exact)
    for mode in ("fp16x", "tf32x"):
        err = oracle.rel_fro_error(_run(h, mode, m, n, k, 0, 0, A, B)[0], exact)
        assert err < 1e-6 and err <= 2 * err32, (mode, err, err32)


def test_3m_split_k_matches_model(h):
    m, n, k = 300, 260, 900
    A, B = _operands(m, n, k, 0, 0, 0, seed=24)
    h.set_tc_splits(3)
    try:
        got, _ = _run(h, "tf32x", m, n, k, 0, 0, A, B)
    finally:
        h.set_tc_splits(0)
    model = oracle.tcec_cgemm_3m(1, 0, 0, 0, 0, m, n, k, 1.0, A, B)
    bound = (2 * k + 16) * 2.0 ** -24 * 4 * abs_bound(A, B, 0, 0, m, k, n)
    assert np.all(np.abs(got - model) <= bound)


def test_3m_fp32_mode_nonfinite_and_k_zero(h):
    m, n, k = 64, 80, 40
    A, B = _operands(m, n, k, 0, 0, 0, seed=25)
    # FP32 mode keeps the complex SIMT kernel
    got, d = _run(h, "fp32", m, n, k, 0, 0, A, B)
    assert d[0] == oracle.MODE_FP32
    assert oracle.rel_fro_error(got, oracle.cgemm(0, 0, m, n, k, 1.0, A, B)) < 5e-6
    # Inf routes AUTO to FP32 (the three products do not run)
    A[3, 4] = np.inf
    got, d = _run(h, "auto", m, n, k, 0, 0, A, B)
    assert d[0] == oracle.MODE_FP32
    ref = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
    fin = np.isfinite(ref)
    assert np.allclose(got[fin], ref[fin], rtol=1e-5, atol=1e-4)
    # k = 0: C = beta C
    C0 = qi.cgemm_operand(m, n, 0, seed=26)
    got, _ = _run(h, "fp16x", m, n, 0, 0, 0, A, B, 1.0, 2.0 - 1j, C0)
    assert np.allclose(got, (2.0 - 1j) * C0.astype(np.complex128), rtol=1e-6)


def test_set_complex_products_rejects_other_values(h):
    from paper_2303_08989_gb300 import _lib as L

    for bad in (0, 2, 5):
        assert h.lib.qcs_set_complex_products(h.ptr, bad) == L.QCS_ERR_INVALID_ARG
    assert h.lib.qcs_set_complex_products(h.ptr, 3) == L.QCS_SUCCESS


def test_3m_full_size_sampled_rows():
    """8192^3 AUTO-0.1 with three products under the paper's size rule: 16
    sampled rows against FP64 and the error of the four-product form on the
    same inputs."""
    q = lib()
    n = 8192
    A = qi.cgemm_operand(n, n, 0, (8192, 31))
    B = qi.cgemm_operand(n, n, 0, (8192, 32))
    rows = np.random.default_rng(33).choice(n, 16, replace=False)
    ref = oracle.cgemm(0, 0, n, n, n, 1.0, A, B, rows=rows)
    Ad, Bd = dev(A), dev(B)
    errs = {}
    for products in (4, 3):
        hd = q.Handle(tol=0.1)
        hd.set_complex_products(products)
        try:
            C = q.fortran_empty(n, n)
            q.cgemm(hd, Ad, Bd, C, mode="auto")
            torch.cuda.synchronize()
            hd.sync()
            got = C[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.complex128)
            errs[products] = oracle.rel_fro_error(got, ref)
        finally:
            hd.close()
    assert errs[3] < 1e-6 and errs[3] < 3 * errs[4], errs
