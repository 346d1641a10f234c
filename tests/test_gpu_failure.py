"""Failure detection on the GPU without a fault: the tensor-core kernels'
bounded waits.  A test hook (qcs_debug_stall_producer) keeps the TMA producer
from issuing any load, so that the MMA issuer's wait for the first stage runs
out after a short budget (qcs_set_wait_budget); the kernel records a timeout
in the handle's error word, releases its tensor memory and returns.  Checked:
qcs_sync reports QCS_ERR_TIMEOUT once (the word is then clear), and the same
handle computes correct results afterwards."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import dev, host, lib, need_gpu, torch

pytestmark = pytest.mark.gpu


def _expect_timeout(q, h):
    from paper_2303_08989_gb300 import _lib as L

    torch.cuda.synchronize()
    with pytest.raises(L.QcsError) as e:
        h.sync()
    assert e.value.code == L.QCS_ERR_TIMEOUT
    h.sync()  # reported once: the word was cleared


@pytest.mark.parametrize("mode,splits", [("fp16x", 0), ("tf32x", 0), ("fp16x", 4)])
def test_stalled_producer_times_out_and_the_handle_recovers(mode, splits):
    need_gpu()
    q = lib()
    m, n, k = 384, 256, 512
    A = qi.cgemm_operand(m, k, 0, seed=(31, 1))
    B = qi.cgemm_operand(k, n, 0, seed=(31, 2))
    Ad, Bd = dev(A), dev(B)
    exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
    h = q.Handle(tol=0.0, size_rule=False)
    if splits:
        h.set_tc_splits(splits)
    h.set_wait_budget(2_000_000)  # 2 ms
    h.debug_stall_producer(True)
    C = q.cgemm(h, Ad, Bd, mode=mode)
    _expect_timeout(q, h)
    h.debug_stall_producer(False)
    h.set_wait_budget(2_000_000_000)
    for _ in range(2):
        C = q.cgemm(h, Ad, Bd, mode=mode)
        torch.cuda.synchronize()
        h.sync()
        assert oracle.rel_fro_error(host(C).astype(np.complex128), exact) < 1e-6
    h.close()


def test_stalled_producer_in_the_real_and_three_product_kernels():
    need_gpu()
    q = lib()
    m, n, k = 256, 512, 256
    h = q.Handle(tol=0.0, size_rule=False)
    h.set_wait_budget(2_000_000)
    Ar = qi.sgemm_operand(m, k, 0, seed=(32, 1))
    Br = qi.sgemm_operand(k, n, 0, seed=(32, 2))
    Ard = torch.from_numpy(np.ascontiguousarray(Ar.T)).cuda().t()
    Brd = torch.from_numpy(np.ascontiguousarray(Br.T)).cuda().t()
    h.debug_stall_producer(True)
    q.sgemm(h, Ard, Brd, mode="fp16x")
    _expect_timeout(q, h)
    h.set_complex_products(3)
    A = dev(qi.cgemm_operand(m, k, 0, seed=(32, 3)))
    B = dev(qi.cgemm_operand(k, n, 0, seed=(32, 4)))
    q.cgemm(h, A, B, mode="fp16x")
    _expect_timeout(q, h)
    h.debug_stall_producer(False)
    Cr = q.sgemm(h, Ard, Brd, mode="fp16x")
    torch.cuda.synchronize()
    h.sync()
    exact = oracle.sgemm(0, 0, m, n, k, 1.0, Ar, Br)
    assert oracle.rel_fro_error(Cr.cpu().numpy().astype(np.float64), exact) < 1e-6
    h.close()


def test_wait_budget_rejects_out_of_range_values():
    need_gpu()
    q = lib()
    from paper_2303_08989_gb300 import _lib as L

    h = q.Handle()
    for bad in (0, 999, 10_000_000_001):
        with pytest.raises(L.QcsError):
            h.set_wait_budget(bad)
    h.close()
