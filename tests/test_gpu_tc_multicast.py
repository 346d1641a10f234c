"""The complex tensor-core kernel in clusters of two CTAs that share each
op(B) box by TMA multicast (qcs_set_tc_multicast): the same MMAs per tile
in the same order, so C equals the one-CTA kernel's bit for bit, in every
kind, op pair, group and K-range setting; odd tile-row counts fall back to
the one-CTA kernel; a stalled producer times out in both CTAs and the
handle recovers."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import dev, host, lib, need_gpu, torch

pytestmark = pytest.mark.gpu


def _pair(q, A, B, mode, opA=0, opB=0, alpha=1.0, beta=0.0, C0=None, splits=0, tol=0.0):
    outs = []
    for mc in (False, True):
        h = q.Handle(tol=tol, size_rule=False)
        try:
            h.set_tc_multicast(mc)
            if splits:
                h.set_tc_splits(splits)
            Cd = dev(C0) if C0 is not None else None
            C = q.cgemm(h, dev(A), dev(B), Cd, alpha=alpha, beta=beta, opA=opA, opB=opB,
                        mode=mode)
            torch.cuda.synchronize()
            h.sync()
            outs.append(host(C))
        finally:
            h.close()
    return outs


@pytest.mark.parametrize("m,n,k,mode,opA,opB", [
    (256, 256, 256, "fp16x", 0, 0),
    (1024, 384, 512, "fp16x", 1, 0),
    (512, 1000, 320, "tf32x", 0, 2),        # ragged n
    (768, 640, 1000, "bf16x3", 2, 1),       # ragged k
    (2048, 2048, 1024, "fp16x_scaled", 0, 0),
    (256, 129, 64, "auto", 1, 2),
])
def test_clusters_are_bit_identical(m, n, k, mode, opA, opB):
    need_gpu()
    q = lib()
    s = 8 if mode in ("fp16x_scaled", "auto") else 0
    shapeA = (m, k) if opA == 0 else (k, m)
    shapeB = (k, n) if opB == 0 else (n, k)
    A = qi.cgemm_operand(*shapeA, s, seed=(m, n, k, 1))
    B = qi.cgemm_operand(*shapeB, s, seed=(m, n, k, 2))
    C0 = qi.cgemm_operand(m, n, 0, seed=(m, n, k, 3))
    one, mc = _pair(q, A, B, mode, opA, opB, alpha=0.5 - 1j, beta=0.25j, C0=C0, tol=0.1)
    assert np.array_equal(one, mc)
    ref = oracle.cgemm(opA, opB, m, n, k, 0.5 - 1j, A, B, 0.25j, C0)
    assert oracle.rel_fro_error(mc.astype(np.complex128), ref) < 1e-5


@pytest.mark.parametrize("splits", [2, 5])
def test_clusters_with_k_ranges(splits):
    need_gpu()
    q = lib()
    m, n, k = 512, 256, 2048
    A = qi.cgemm_operand(m, k, 0, seed=(5, 1))
    B = qi.cgemm_operand(k, n, 0, seed=(5, 2))
    one, mc = _pair(q, A, B, "fp16x", splits=splits)
    assert np.array_equal(one, mc)


def test_odd_tile_rows_fall_back():
    need_gpu()
    q = lib()
    m, n, k = 384, 256, 256  # three tile rows
    A = qi.cgemm_operand(m, k, 0, seed=(6, 1))
    B = qi.cgemm_operand(k, n, 0, seed=(6, 2))
    one, mc = _pair(q, A, B, "fp16x")
    assert np.array_equal(one, mc)


def test_clusters_in_a_contraction_group():
    """A grouped tree run (instances with their own selected modes in one
    tensor-core launch per kind) with clusters on and off: the same amplitudes."""
    need_gpu()
    import paper_2303_08989_gb300.tn as tn

    q = lib()
    circ = qi.random_grid_circuit(4, 4, 10, seed=8)
    bits = qi.random_bitstrings(16, 6, seed=9)
    plan = tn.plan_circuit(circ, bits, seed=4, n_slices=2)
    for st in plan.steps:
        if st.m >= 256 and st.n >= 64:
            st.mode = q.MODE_AUTO
    res = []
    for mc in (False, True):
        h = q.Handle(tol=0.1, size_rule=False)
        try:
            h.set_instance_batch(6)
            h.set_tc_multicast(mc)
            cp = tn.CompiledPlan(plan)
            out = cp.forward(h)
            torch.cuda.synchronize()
            h.sync()
            res.append(out.cpu().numpy())
        finally:
            h.close()
    assert np.array_equal(res[0], res[1])


def test_stalled_producer_times_out_in_both_ctas():
    need_gpu()
    from paper_2303_08989_gb300 import _lib as L

    q = lib()
    m, n, k = 512, 256, 512
    A = qi.cgemm_operand(m, k, 0, seed=(7, 1))
    B = qi.cgemm_operand(k, n, 0, seed=(7, 2))
    exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
    h = q.Handle(tol=0.0, size_rule=False)
    try:
        h.set_tc_multicast(True)
        h.set_wait_budget(2_000_000)  # 2 ms
        h.debug_stall_producer(True)
        q.cgemm(h, dev(A), dev(B), mode="fp16x")
        torch.cuda.synchronize()
        with pytest.raises(L.QcsError) as e:
            h.sync()
        assert e.value.code == L.QCS_ERR_TIMEOUT
        h.debug_stall_producer(False)
        h.set_wait_budget(2_000_000_000)
        C = q.cgemm(h, dev(A), dev(B), mode="fp16x")
        torch.cuda.synchronize()
        h.sync()
        assert oracle.rel_fro_error(host(C).astype(np.complex128), exact) < 1e-6
    finally:
        h.close()


def test_setter_rejects_bad_values():
    need_gpu()
    q = lib()
    h = q.Handle()
    try:
        assert h.lib.qcs_set_tc_multicast(h._h, 2) == -1
    finally:
        h.close()
