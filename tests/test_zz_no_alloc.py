"""qcs_cgemm_noalloc -- the CGEMM entry point that needs no handle and
allocates no device memory, for callers whose device memory belongs to
another allocator with a fixed budget, or whose loops cannot afford
cudaMalloc's device-wide synchronisation -- checked through the C ABI
against qcs_cgemm on the same inputs, on two calls in a row.

The file name sorts last so that a run stopping at the first failure has
already run every other test; it passes alone in a fresh process too.
"""
import ctypes

import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import abs_bound, dev, host, lib, need_gpu, torch

pytestmark = pytest.mark.gpu

MODES = {"auto": 0, "fp16x": 1, "fp16x_scaled": 2, "tf32x": 3, "fp32": 4}


def _noalloc(L, stream, mode, tol, m, n, k, Ad, Bd, Cd, desc=None, opA=0, opB=0):
    one = L.qcs_c32(1.0, 0.0)
    zero = L.qcs_c32(0.0, 0.0)
    return L.load().qcs_cgemm_noalloc(
        ctypes.c_void_p(stream), MODES[mode], tol, opA, opB, m, n, k, ctypes.byref(one),
        ctypes.c_void_p(Ad.data_ptr()), Ad.stride(1), ctypes.c_void_p(Bd.data_ptr()), Bd.stride(1),
        ctypes.byref(zero), ctypes.c_void_p(Cd.data_ptr()), Cd.stride(1),
        ctypes.c_void_p(desc.data_ptr()) if desc is not None else None)


@pytest.mark.parametrize("mode", ["auto", "fp16x", "tf32x", "fp16x_scaled", "fp32"])
def test_noalloc_matches_cgemm_on_two_calls(mode):
    need_gpu()
    q = lib()
    from paper_2303_08989_gb300 import _lib as L

    tol = 0.1
    h = q.Handle(tol=tol, size_rule=False)
    stream = torch.cuda.current_stream().cuda_stream
    m, n, k = 300, 260, 200
    # two calls in a row on different data: nothing of the first may leak into the second
    for call, (s, seed) in enumerate([(8, 11), (0, 12)]):
        A = qi.cgemm_operand(m, k, s, seed=(seed, 1))
        B = qi.cgemm_operand(k, n, s, seed=(seed, 2))
        Ad, Bd = dev(A), dev(B)
        C_ref = q.fortran_empty(m, n)
        d_ref = torch.zeros(4, dtype=torch.int32, device="cuda")
        q.cgemm(h, Ad, Bd, C_ref, mode=mode, desc_out=d_ref)
        C_na = q.fortran_empty(m, n)
        C_na.fill_(complex(float("nan"), float("nan")))
        d_na = torch.zeros(4, dtype=torch.int32, device="cuda")
        rc = _noalloc(L, stream, mode, tol, m, n, k, Ad, Bd, C_na, d_na)
        assert rc == L.QCS_SUCCESS, (call, L.status_string(rc))
        torch.cuda.synchronize()
        h.sync()
        assert torch.equal(d_na, d_ref), (call, d_na, d_ref)
        got, ref = host(C_na).astype(np.complex128), host(C_ref).astype(np.complex128)
        # the tolerance of the CGEMM parity tests: FP32 accumulation over 2k terms
        bound = (2 * k + 8) * 2.0 ** -24 * 2 * abs_bound(A, B, 0, 0, m, k, n)
        assert np.all(np.abs(got - ref) <= bound), call
        exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
        assert oracle.rel_fro_error(got, exact) < 1e-6, call
    h.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    need_gpu()
    from paper_2303_08989_gb300 import _lib as L

    stream = torch.cuda.current_stream().cuda_stream
    m = n = k = 2048  # AUTO planes alone: 16 B x (2048 + 2048) x 2048 = 128 MiB > 64 MiB
    A = torch.zeros((k, m), dtype=torch.complex64, device="cuda").t()
    B = torch.zeros((n, k), dtype=torch.complex64, device="cuda").t()
    C = torch.full((n, m), 3.0 + 0j, dtype=torch.complex64, device="cuda").t()
    rc = _noalloc(L, stream, "auto", 0.0, m, n, k, A, B, C)
    assert rc == L.QCS_ERR_SCRATCH_TOO_SMALL
    torch.cuda.synchronize()
    assert bool((C == 3.0).all())  # nothing was launched
    # the same problem in plain FP32 needs no planes and fits
    rc = _noalloc(L, stream, "fp32", 0.0, m, n, k, A, B, C)
    assert rc == L.QCS_SUCCESS
    torch.cuda.synchronize()
    assert bool((C == 0).all())


def _status(L, stream, reset=0):
    return L.load().qcs_cgemm_noalloc_status(ctypes.c_void_p(stream), reset)


def test_noalloc_transposed_and_conjugated_operands_allocate_nothing():
    """op(A) = A^T and op(B) = B^H against qcs_cgemm, in every mode; after
    one round that loads every kernel, a second round of calls leaves the
    device's free memory unchanged, and the status word stays clear."""
    need_gpu()
    q = lib()
    from paper_2303_08989_gb300 import _lib as L

    tol = 0.1
    h = q.Handle(tol=tol, size_rule=False)
    stream = torch.cuda.current_stream().cuda_stream
    m, n, k = 200, 264, 136
    A = qi.cgemm_operand(k, m, 8, seed=(21, 1))  # stored k x m: op T
    B = qi.cgemm_operand(n, k, 8, seed=(21, 2))  # stored n x k: op C
    Ad, Bd = dev(A), dev(B)
    exact = oracle.cgemm(1, 2, m, n, k, 1.0, A, B)
    bound = (2 * k + 8) * 2.0 ** -24 * 2 * abs_bound(A, B, 1, 2, m, k, n)
    outs = {mode: (q.fortran_empty(m, n), q.fortran_empty(m, n),
                   torch.zeros(4, dtype=torch.int32, device="cuda"),
                   torch.zeros(4, dtype=torch.int32, device="cuda")) for mode in MODES}
    for rnd in range(2):
        if rnd == 1:
            torch.cuda.synchronize()
            free0 = torch.cuda.mem_get_info()[0]
        for mode, (C_ref, C_na, d_ref, d_na) in outs.items():
            if rnd == 0:
                q.cgemm(h, Ad, Bd, C_ref, opA=1, opB=2, mode=mode, desc_out=d_ref)
            C_na.fill_(complex(float("nan"), float("nan")))
            rc = _noalloc(L, stream, mode, tol, m, n, k, Ad, Bd, C_na, d_na, opA=1, opB=2)
            assert rc == L.QCS_SUCCESS, (mode, L.status_string(rc))
        torch.cuda.synchronize()
        h.sync()
        if rnd == 1:
            assert torch.cuda.mem_get_info()[0] == free0
    assert _status(L, stream) == L.QCS_SUCCESS
    for mode, (C_ref, C_na, d_ref, d_na) in outs.items():
        assert torch.equal(d_na, d_ref), mode
        got, ref = host(C_na).astype(np.complex128), host(C_ref).astype(np.complex128)
        assert np.all(np.abs(got - ref) <= bound), mode
        assert oracle.rel_fro_error(got, exact) < 1e-6, mode
    h.close()


def test_noalloc_status_is_clear_after_normal_calls():
    need_gpu()
    from paper_2303_08989_gb300 import _lib as L

    stream = torch.cuda.current_stream().cuda_stream
    m = n = k = 256
    A = dev(qi.cgemm_operand(m, k, 0, seed=(22, 1)))
    B = dev(qi.cgemm_operand(k, n, 0, seed=(22, 2)))
    C = torch.empty((n, m), dtype=torch.complex64, device="cuda").t()
    for _ in range(2):
        assert _noalloc(L, stream, "auto", 0.0, m, n, k, A, B, C) == L.QCS_SUCCESS
        assert _status(L, stream, reset=1) == L.QCS_SUCCESS
        assert _status(L, stream) == L.QCS_SUCCESS
