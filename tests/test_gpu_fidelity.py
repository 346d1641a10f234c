"""qcs_fidelity_stats: the FP64 norms, overlap and error sums on the GPU
(Section 5.3's fidelity and error of amplitudes against an exact
reference) against numpy FP64 and the oracle's fidelity."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import lib, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    need_gpu()
    hd = lib().Handle()
    yield hd
    hd.close()


def _pair(n, seed):
    rng = np.random.default_rng(seed)
    ref = (rng.standard_normal(n) + 1j * rng.standard_normal(n)) * 2.0 ** rng.integers(-30, 30, n)
    a = ref + 1e-6 * np.abs(ref) * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
    return a, ref


@pytest.mark.parametrize("n", [1, 7, 256, 257, 100003, (1 << 20) + 3])
def test_sums_match_numpy_fp64(h, n):
    q = lib()
    a, ref = _pair(n, n)
    da = torch.from_numpy(a).cuda()
    dr = torch.from_numpy(ref).cuda()
    got = q.fidelity_stats(h, da, dr)
    assert got["norm2"] == pytest.approx(float(np.sum(np.abs(a) ** 2)), rel=1e-12)
    assert got["ref_norm2"] == pytest.approx(float(np.sum(np.abs(ref) ** 2)), rel=1e-12)
    ov = np.vdot(ref, a)
    assert got["overlap"].real == pytest.approx(ov.real, rel=1e-12)
    # the imaginary part cancels to about 1e-6 of |ov|: compare it against the
    # scale of its terms (FP64 rounding of a sum in another order)
    scale = float(np.sum(np.abs(ref) * np.abs(a)))
    assert abs(got["overlap"].imag - ov.imag) <= 1e-12 * scale
    d = np.abs(a - ref)
    assert got["err2"] == pytest.approx(float(np.sum(d ** 2)), rel=1e-10)
    assert got["max_abs_err"] == pytest.approx(float(np.max(d)), rel=1e-12)
    assert got["fidelity"] == pytest.approx(oracle.fidelity(ref, a), rel=1e-12)
    assert got["rel_l2_err"] == pytest.approx(
        float(np.linalg.norm(a - ref) / np.linalg.norm(ref)), rel=1e-10)
    # fixed summation order: the same bits twice
    again = q.fidelity_stats(h, da, dr)
    assert again == got


def test_complex64_result_and_norm_only(h):
    q = lib()
    a, ref = _pair(4099, 3)
    a32 = a.astype(np.complex64)
    got = q.fidelity_stats(h, torch.from_numpy(a32).cuda(), torch.from_numpy(ref).cuda())
    a64 = a32.astype(np.complex128)
    assert got["fidelity"] == pytest.approx(oracle.fidelity(ref, a64), rel=1e-12)
    assert got["err2"] == pytest.approx(float(np.sum(np.abs(a64 - ref) ** 2)), rel=1e-9)
    only = q.fidelity_stats(h, torch.from_numpy(a32).cuda())
    assert set(only) == {"norm2"}
    assert only["norm2"] == pytest.approx(float(np.sum(np.abs(a64) ** 2)), rel=1e-12)


def test_empty_and_invalid(h):
    import ctypes

    q = lib()
    out = torch.full((6,), 7.0, dtype=torch.float64, device="cuda")
    buf = torch.zeros(8, dtype=torch.complex128, device="cuda")
    rc = h.lib.qcs_fidelity_stats(h.ptr, ctypes.c_void_p(buf.data_ptr()), 0, None, 0,
                                  ctypes.c_void_p(out.data_ptr()))
    assert rc == 0
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0] * 6
    assert h.lib.qcs_fidelity_stats(h.ptr, None, 0, None, 4, ctypes.c_void_p(out.data_ptr())) == -1
    assert h.lib.qcs_fidelity_stats(h.ptr, ctypes.c_void_p(buf.data_ptr() + 8), 0, None, 4,
                                    ctypes.c_void_p(out.data_ptr())) == -1  # complex128 misaligned
    assert h.lib.qcs_fidelity_stats(h.ptr, ctypes.c_void_p(buf.data_ptr()), 2, None, 4,
                                    ctypes.c_void_p(out.data_ptr())) == -1
    assert h.lib.qcs_fidelity_stats(h.ptr, ctypes.c_void_p(buf.data_ptr()), 0, None, -1,
                                    ctypes.c_void_p(out.data_ptr())) == -1


def test_tree_amplitudes_fidelity_on_the_gpu(h):
    """The 12-qubit amplitudes from the contraction tree (FP64 slice sums on
    the device) reduced against the oracle's state-vector amplitudes on the
    GPU give the oracle's own fidelity of the same numbers."""
    import paper_2303_08989_gb300.tn as tn

    q = lib()
    circ = qi.random_grid_circuit(3, 4, 8, seed=0)
    bits = qi.random_bitstrings(12, 64, seed=1)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=2)
    cp = tn.CompiledPlan(plan)
    hd = q.Handle(tol=0.0, size_rule=True)
    try:
        out = cp.forward(hd)
        torch.cuda.synchronize()
        hd.sync()
    finally:
        hd.close()
    ref = oracle.sv_amplitudes(circ, bits)
    got = q.fidelity_stats(h, out[:, 0].contiguous(), torch.from_numpy(ref).cuda())
    a = out[:, 0].cpu().numpy()
    assert got["fidelity"] == pytest.approx(oracle.fidelity(ref, a), rel=1e-12)
    assert got["fidelity"] >= 1 - 1e-5
