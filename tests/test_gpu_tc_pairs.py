"""The tensor-core kernels as CTA pairs (qcs_set_tc_pairs): a cluster of two
CTAs runs one 256-row tile with tcgen05 MMAs of cta_group::2, each CTA
holding its 128 rows of op(A) and half of every op(B) operand.  Every output
element is the same sequence of tensor-core products as in one CTA, so C
equals the one-CTA kernel's bit for bit in every kind, op pair, group and
K-range setting, for the complex and the real kernel and Gauss's
three-product form; shapes with an odd number of tile rows, and other drain
lengths, fall back to the one-CTA kernel; a stalled producer times out in
both CTAs and the handle recovers."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import dev, host, lib, need_gpu, torch

pytestmark = pytest.mark.gpu


def _handles(q, tol, **kw):
    out = []
    for pairs in (False, True):
        h = q.Handle(tol=tol, size_rule=False)
        h.set_tc_pairs(pairs)
        if kw.get("splits"):
            h.set_tc_splits(kw["splits"])
        if kw.get("products"):
            h.set_complex_products(kw["products"])
        if kw.get("drain"):
            h.set_drain_stages(kw["drain"])
        out.append(h)
    return out


def _cgemm_pair(q, A, B, mode, opA=0, opB=0, alpha=1.0, beta=0.0, C0=None, tol=0.0, **kw):
    outs = []
    for h in _handles(q, tol, **kw):
        try:
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
    (2048, 8192, 32, "tf32x", 0, 0),        # one stage per tile
])
def test_pairs_are_bit_identical(m, n, k, mode, opA, opB):
    need_gpu()
    q = lib()
    s = 8 if mode in ("fp16x_scaled", "auto") else 0
    shapeA = (m, k) if opA == 0 else (k, m)
    shapeB = (k, n) if opB == 0 else (n, k)
    A = qi.cgemm_operand(*shapeA, s, seed=(m, n, k, 11))
    B = qi.cgemm_operand(*shapeB, s, seed=(m, n, k, 12))
    C0 = qi.cgemm_operand(m, n, 0, seed=(m, n, k, 13))
    one, pr = _cgemm_pair(q, A, B, mode, opA, opB, alpha=0.5 - 1j, beta=0.25j, C0=C0, tol=0.1)
    ref = oracle.cgemm(opA, opB, m, n, k, 0.5 - 1j, A, B, 0.25j, C0)
    assert oracle.rel_fro_error(pr.astype(np.complex128), ref) < 1e-5
    assert np.array_equal(one, pr)


@pytest.mark.parametrize("splits", [2, 5])
def test_pairs_with_k_ranges(splits):
    need_gpu()
    q = lib()
    m, n, k = 512, 256, 2048
    A = qi.cgemm_operand(m, k, 0, seed=(15, 1))
    B = qi.cgemm_operand(k, n, 0, seed=(15, 2))
    one, pr = _cgemm_pair(q, A, B, "fp16x", splits=splits)
    assert np.array_equal(one, pr)
    exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
    assert oracle.rel_fro_error(pr.astype(np.complex128), exact) < 1e-6


@pytest.mark.parametrize("m,drain", [(384, 4), (512, 2), (512, 1)])
def test_odd_tile_rows_and_other_drains_fall_back(m, drain):
    need_gpu()
    q = lib()
    n, k = 256, 512
    A = qi.cgemm_operand(m, k, 0, seed=(16, m, 1))
    B = qi.cgemm_operand(k, n, 0, seed=(16, m, 2))
    one, pr = _cgemm_pair(q, A, B, "fp16x", drain=drain)
    assert np.array_equal(one, pr)


def test_pairs_in_gauss_three_products():
    """The three real GEMMs of the three-product form as one grouped launch
    of the real kernel in pairs."""
    need_gpu()
    q = lib()
    m, n, k = 768, 512, 384
    A = qi.cgemm_operand(m, k, 0, seed=(17, 1))
    B = qi.cgemm_operand(k, n, 0, seed=(17, 2))
    one, pr = _cgemm_pair(q, A, B, "fp16x", products=3)
    assert np.array_equal(one, pr)
    exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
    assert oracle.rel_fro_error(pr.astype(np.complex128), exact) < 1e-6


def _dev_r(x):
    base = torch.empty((x.shape[1], x.shape[0]), dtype=torch.float32, device="cuda")
    base.copy_(torch.from_numpy(np.ascontiguousarray(x.T)))
    return base.t()


def _host_r(t):
    return np.asfortranarray(t.t().contiguous().cpu().numpy().T)


@pytest.mark.parametrize("m,n,k,mode,opA,opB", [
    (512, 512, 512, "fp16x", 0, 0),
    (1024, 700, 300, "tf32x", 1, 0),        # ragged n, k
    (256, 256, 1024, "bf16x3", 0, 1),
    (768, 1024, 512, "auto", 1, 1),
])
def test_real_pairs_are_bit_identical(m, n, k, mode, opA, opB):
    need_gpu()
    q = lib()
    s = 8 if mode == "auto" else 0
    ra, ca = (m, k) if opA == 0 else (k, m)
    rb, cb = (k, n) if opB == 0 else (n, k)
    A = qi.sgemm_operand(ra, ca, s, (m, n, k, 21))
    B = qi.sgemm_operand(rb, cb, s, (m, n, k, 22))
    outs = []
    for h in _handles(q, 0.1):
        try:
            C = q.sgemm(h, _dev_r(A), _dev_r(B), m=m, n=n, k=k, opA=opA, opB=opB, mode=mode)
            torch.cuda.synchronize()
            h.sync()
            outs.append(_host_r(C)[:m, :n])
        finally:
            h.close()
    exact = oracle.sgemm(opA, opB, m, n, k, 1.0, A, B)
    err = np.linalg.norm(outs[1] - exact) / np.linalg.norm(exact)
    assert err < 1e-5
    assert np.array_equal(outs[0], outs[1])


def test_pairs_in_a_contraction_group():
    """A grouped tree run (instances with their own selected modes in one
    tensor-core launch per kind) with pairs on and off: the same amplitudes."""
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
    for pairs in (False, True):
        h = q.Handle(tol=0.1, size_rule=False)
        try:
            h.set_instance_batch(6)
            h.set_tc_pairs(pairs)
            cp = tn.CompiledPlan(plan)
            out = cp.forward(h)
            torch.cuda.synchronize()
            h.sync()
            res.append(out.cpu().numpy())
        finally:
            h.close()
    assert np.array_equal(res[0], res[1])


@pytest.mark.parametrize("real", [False, True])
def test_stalled_producer_times_out_in_both_ctas(real):
    need_gpu()
    from paper_2303_08989_gb300 import _lib as L

    q = lib()
    m, n, k = 512, 512, 512
    if real:
        A = qi.sgemm_operand(m, k, 0, (27, 1))
        B = qi.sgemm_operand(k, n, 0, (27, 2))
        exact = oracle.sgemm(0, 0, m, n, k, 1.0, A, B)
        run = lambda h: _host_r(q.sgemm(h, _dev_r(A), _dev_r(B), mode="fp16x"))  # noqa: E731
    else:
        A = qi.cgemm_operand(m, k, 0, seed=(27, 1))
        B = qi.cgemm_operand(k, n, 0, seed=(27, 2))
        exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
        run = lambda h: host(q.cgemm(h, dev(A), dev(B), mode="fp16x"))  # noqa: E731
    h = q.Handle(tol=0.0, size_rule=False)
    try:
        h.set_tc_pairs(True)
        h.set_wait_budget(2_000_000)  # 2 ms
        h.debug_stall_producer(True)
        run(h)
        torch.cuda.synchronize()
        with pytest.raises(L.QcsError) as e:
            h.sync()
        assert e.value.code == L.QCS_ERR_TIMEOUT
        h.debug_stall_producer(False)
        h.set_wait_budget(2_000_000_000)
        C = run(h)
        torch.cuda.synchronize()
        h.sync()
        got = C.astype(np.complex128 if not real else np.float64)
        assert np.linalg.norm(got - exact) / np.linalg.norm(exact) < 1e-6
    finally:
        h.close()


def test_pair_setter_rejects_bad_values():
    need_gpu()
    q = lib()
    h = q.Handle()
    try:
        assert h.lib.qcs_set_tc_pairs(h._h, 2) == -1
        h.set_tc_pairs(True)
        h.set_tc_pairs(False)
    finally:
        h.close()
