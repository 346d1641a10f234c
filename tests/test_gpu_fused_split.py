"""The TF32X CGEMM with the Eq. 1 split inside the tensor-core kernel's
staging (qcs_set_fused_split): the kernel reads A and B as stored and splits
each staged tile in shared memory.  Its tensor-core inputs and their order
are those of the two-pass path, so C must equal the two-pass result bit for
bit, for every operand op, ragged shapes (TMA zero fill at every edge),
alpha / beta and ldc > m; AUTO calls that select TF32X take it, those that
select FP16X are untouched; unsupported layouts fall back; a stalled
producer times out and the handle recovers.  Every result also meets the
FP32-level bound against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import dev, host, lib, need_gpu, torch

pytestmark = pytest.mark.gpu

OPS = {"N": 0, "T": 1, "C": 2}


def _operands(opA, opB, m, n, k, s, seed):
    A = qi.cgemm_operand(m if opA == 0 else k, k if opA == 0 else m, s, seed=(seed, 1))
    B = qi.cgemm_operand(k if opB == 0 else n, n if opB == 0 else k, s, seed=(seed, 2))
    return A, B


def _pair(mode, opA, opB, m, n, k, s=0, seed=1, alpha=1.0, beta=0.0, ldc=None, tol=0.0):
    """(fused C, two-pass C, A, B, C0) on the same inputs."""
    q = lib()
    A, B = _operands(opA, opB, m, n, k, s, seed)
    Ad, Bd = dev(A), dev(B)
    rng = np.random.default_rng(seed + 7)
    C0 = (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))).astype(np.complex64)
    outs = []
    for fused in (True, False):
        h = q.Handle(tol=tol, size_rule=False)
        h.set_fused_split(fused)
        C = q.fortran_empty(m, n, ld=ldc)
        C.copy_(torch.from_numpy(C0).cuda())
        desc = torch.zeros(4, dtype=torch.int32, device="cuda")
        q.cgemm(h, Ad, Bd, C, alpha=alpha, beta=beta, opA=opA, opB=opB, mode=mode, desc_out=desc)
        torch.cuda.synchronize()
        h.sync()
        outs.append((host(C).astype(np.complex128), q.MODE_NAME[int(desc[0].item())]))
        h.close()
    return outs[0], outs[1], A, B, C0


@pytest.mark.parametrize("ops", ["NN", "TN", "CN", "NT", "NC", "CC", "TT"])
@pytest.mark.parametrize("shape", [(300, 260, 200), (128, 128, 16), (257, 129, 48), (96, 520, 1000)])
def test_fused_tf32x_is_bit_identical_to_two_pass(ops, shape):
    need_gpu()
    m, n, k = shape
    opA, opB = OPS[ops[0]], OPS[ops[1]]
    (cf, mf), (cu, mu), A, B, _ = _pair("tf32x", opA, opB, m, n, k, s=8, seed=3)
    assert mf == mu == "tf32x"
    assert np.array_equal(cf, cu)
    exact = oracle.cgemm(opA, opB, m, n, k, 1.0, A, B)
    assert oracle.rel_fro_error(cf, exact) < 1e-6


def test_fused_with_alpha_beta_and_padded_ldc():
    need_gpu()
    m, n, k = 333, 190, 260
    alpha, beta = complex(0.75, -1.25), complex(-0.5, 0.25)
    (cf, _), (cu, _), A, B, C0 = _pair("tf32x", 0, 1, m, n, k, s=4, seed=5, alpha=alpha,
                                       beta=beta, ldc=352)
    assert np.array_equal(cf, cu)
    want = alpha * oracle.cgemm(0, 1, m, n, k, 1.0, A, B) + beta * C0.astype(np.complex128)
    assert oracle.rel_fro_error(cf, want) < 1e-6


@pytest.mark.parametrize("s,picked", [(40, "tf32x"), (0, "fp16x")])
def test_fused_under_auto(s, picked):
    """AUTO-0.1: inputs spread over 2^+-40 select TF32X (the fused kernel
    runs); N(0, 1) inputs select FP16X (the fused kernel exits, the FP16
    planes are split as before)."""
    need_gpu()
    (cf, mf), (cu, mu), A, B, _ = _pair("auto", 0, 0, 384, 256, 512, s=s, seed=9, tol=0.1)
    assert mf == mu == picked
    assert np.array_equal(cf, cu)
    assert oracle.rel_fro_error(cf, oracle.cgemm(0, 0, 384, 256, 512, 1.0, A, B)) < 1e-6


def test_fused_falls_back_on_odd_leading_dimension():
    """lda odd: TMA cannot read the rows, the two-pass path runs."""
    need_gpu()
    q = lib()
    m, n, k = 131, 140, 96
    A, B = _operands(0, 0, m, n, k, 0, 11)
    # rows of m + 2 = 133 elements: an odd leading dimension
    base = torch.zeros((k, m + 2), dtype=torch.complex64, device="cuda")
    base[:, :m] = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    Ad = base.t()[:m]
    assert Ad.stride(1) % 2 == 1
    res = []
    for fused in (True, False):
        h = q.Handle(tol=0.0, size_rule=False)
        h.set_fused_split(fused)
        C = q.cgemm(h, Ad, dev(B), mode="tf32x")
        torch.cuda.synchronize()
        h.sync()
        res.append(host(C))
        h.close()
    assert np.array_equal(res[0], res[1])
    assert oracle.rel_fro_error(res[0].astype(np.complex128),
                                oracle.cgemm(0, 0, m, n, k, 1.0, A, B)) < 1e-6


def test_fused_full_size_tile_grid():
    """2048^3: 256 tiles over the SMs, 128 stages per tile, whole C compared
    bit for bit on the device."""
    need_gpu()
    q = lib()
    n = 2048
    g = torch.Generator(device="cuda").manual_seed(13)
    A = torch.randn((n, n), dtype=torch.complex64, device="cuda", generator=g).t()
    B = torch.randn((n, n), dtype=torch.complex64, device="cuda", generator=g).t()
    res = []
    for fused in (True, False):
        h = q.Handle(tol=0.0, size_rule=False)
        h.set_fused_split(fused)
        res.append(q.cgemm(h, A, B, mode="tf32x"))
        torch.cuda.synchronize()
        h.sync()
        h.close()
    assert torch.equal(res[0], res[1])


def test_fused_stalled_producer_times_out_and_recovers():
    need_gpu()
    q = lib()
    m, n, k = 256, 256, 256
    A, B = _operands(0, 0, m, n, k, 0, 17)
    Ad, Bd = dev(A), dev(B)
    h = q.Handle(tol=0.0, size_rule=False)
    h.set_fused_split(True)
    h.set_wait_budget(2_000_000)
    h.debug_stall_producer(True)
    q.cgemm(h, Ad, Bd, mode="tf32x")
    torch.cuda.synchronize()
    from paper_2303_08989_gb300 import _lib as L

    with pytest.raises(L.QcsError) as e:
        h.sync()
    assert e.value.code == L.QCS_ERR_TIMEOUT
    h.debug_stall_producer(False)
    h.set_wait_budget(2_000_000_000)
    C = q.cgemm(h, Ad, Bd, mode="tf32x")
    torch.cuda.synchronize()
    h.sync()
    assert oracle.rel_fro_error(host(C).astype(np.complex128),
                                oracle.cgemm(0, 0, m, n, k, 1.0, A, B)) < 1e-6
    h.close()
