"""Accumulation rounding of tcgen05 MMA (FP16/TF32 inputs, FP32 accumulator
in tensor memory), measured through qcs_cgemm on crafted inputs.

Section 2.1 notes that the A100 tensor cores round toward zero inside the
accumulation, so the method adds the hi*hi products outside the tensor core
with round-to-nearest.  Whether that is needed on sm_103a is decided by this
measurement: 1 + 0.75 ulp(1) must round to 1 + ulp(1) under
round-to-nearest and to 1 under truncation.
"""
import numpy as np
import pytest

from gpu_helpers import dev, host, lib, need_gpu, torch

pytestmark = pytest.mark.gpu

ULP1 = 2.0 ** -23


def _dot(h, mode, pairs, k):
    """C (1x1) = sum_l a_l b_l with a, b given at positions l."""
    q = lib()
    A = np.zeros((1, k), np.complex64, order="F")
    B = np.zeros((k, 1), np.complex64, order="F")
    for l, a, b in pairs:
        A[0, l] = a
        B[l, 0] = b
    C = q.fortran_empty(1, 1)
    q.cgemm(h, dev(A), dev(B), C, alpha=1.0, beta=0.0, mode=mode)
    torch.cuda.synchronize()
    return host(C)[0, 0]


@pytest.fixture(scope="module")
def h():
    need_gpu()
    hd = lib().Handle(size_rule=False)
    # one unbroken K loop, so that the drain groups start at k = 0 (the
    # per-shape choice would cut these one-tile GEMMs into K ranges)
    hd.set_tc_splits(1)
    yield hd
    hd.close()


@pytest.mark.parametrize("drain", [1, 4])
@pytest.mark.parametrize("mode", ["fp16x", "tf32x"])
def test_accumulation_rounding(h, mode, drain, capsys):
    """Inside one drain group the sum stays in tensor memory and is truncated
    by the hardware (1 + 0.75 ulp -> 1); across groups it goes through the
    epilogue's round-to-nearest FP32 adds (-> 1 + 1 ulp).  A drain setting of
    d groups 2 d MMA K steps (32 d values of k for FP16, 16 d for TF32)."""
    h.set_drain_stages(drain)
    k_mma = 16 if mode == "fp16x" else 8
    k_group = 2 * k_mma * drain
    small_a, small_b = 2.0 ** -12, 1.5 * 2.0 ** -12  # product 0.75 ulp(1)
    cases = {
        "within one MMA": ([(0, 1.0, 1.0), (1, small_a, small_b)], 0.0),
        "across MMAs of one group": ([(0, 1.0, 1.0), (k_mma, small_a, small_b)], 0.0),
        "small first, one group": ([(0, small_a, small_b), (k_mma, 1.0, 1.0)], 0.0),
        "last K step of the group": ([(0, 1.0, 1.0), (k_group - 1, small_a, small_b)], 0.0),
        "across drain groups": ([(0, 1.0, 1.0), (k_group, small_a, small_b)], ULP1),
        "across drain groups, small first": ([(0, small_a, small_b), (k_group, 1.0, 1.0)], ULP1),
    }
    try:
        for name, (pairs, want) in cases.items():
            c = _dot(h, mode, pairs, 2 * k_group)
            assert c.imag == 0.0
            got = float(c.real) - 1.0
            with capsys.disabled():
                print(f"[tcgen05 {mode} drain {drain}] {name}: result - 1 = {got / ULP1:+.3f} ulp")
            assert got == want, name
    finally:
        h.set_drain_stages(4)
