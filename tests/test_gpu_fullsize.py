"""Parity at the CGEMM sweep's full sizes, in the launch configuration
bench.py times (AUTO-0.1, size rule on, column-major, alpha = 1, beta = 0):
the selected mode against the oracle's rule on the full operands, and the
result on sampled output rows against the FP64 oracle, row by row.  The
accuracy bar is the one the method is held to: relative Frobenius error at
most twice that of the plain FP32 GPU CGEMM on the same inputs (and at most
1e-6 where k <= 4096 on unit-scaled inputs)."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import dev, lib, need_gpu, torch

pytestmark = pytest.mark.gpu

N_ROWS = 16


@pytest.fixture(scope="module")
def h():
    need_gpu()
    hd = lib().Handle(tol=0.1, size_rule=True)
    yield hd
    hd.close()


def _rows(n, seed):
    g = np.random.default_rng(seed)
    return sorted(set(g.choice(n, size=N_ROWS - 1, replace=False).tolist()) | {n - 1})


def _sampled(h, mode, A, B, n, rows):
    """Run the n^3 CGEMM on the device; return (sampled rows of C, descriptor)."""
    q = lib()
    Ad, Bd = dev(A), dev(B)
    C = q.fortran_empty(n, n)
    desc = torch.zeros(4, dtype=torch.int32, device="cuda")
    q.cgemm(h, Ad, Bd, C, mode=mode, desc_out=desc)
    torch.cuda.synchronize()
    h.sync()
    got = C[torch.tensor(rows, device="cuda")].cpu().numpy().astype(np.complex128)
    del Ad, Bd, C
    torch.cuda.empty_cache()
    return got, desc.cpu().numpy()


def _check(h, n, s, modes, seed):
    A = qi.cgemm_operand(n, n, s, seed=(n, s, 1))
    B = qi.cgemm_operand(n, n, s, seed=(n, s, 2))
    rows = _rows(n, seed)
    exact = oracle.cgemm(0, 0, n, n, n, 1.0, A, B, rows=rows)
    e32 = oracle.rel_fro_error(_sampled(h, "fp32", A, B, n, rows)[0], exact)
    want = oracle.select_mode(oracle.stats_summary(*oracle.exp_stats(A)),
                              oracle.stats_summary(*oracle.exp_stats(B)), 0.1)
    out = {}
    for mode in modes:
        got, d = _sampled(h, mode, A, B, n, rows)
        if mode == "auto":
            assert tuple(int(v) for v in d[:3]) == want
        e = oracle.rel_fro_error(got, exact)
        assert e <= 2 * e32, (mode, e, e32)
        out[mode] = (e, int(d[0]))
    return out, e32


@pytest.mark.parametrize("s", [0, 8, 20, 40])
def test_sweep_16384_auto_sampled_rows(h, s):
    """The bench's workload: m = n = k = 16384, parts N(0,1) 2^e, e ~ U[-s, s]."""
    (res, e32) = _check(h, 16384, s, ["auto"], seed=s)
    print(f"[16384 s={s}] auto err {res['auto'][0]:.3e} (mode {res['auto'][1]}), fp32 err {e32:.3e}")


@pytest.mark.parametrize("s,modes", [(0, ["fp16x", "tf32x"]), (8, ["fp16x_scaled", "tf32x"])])
def test_sweep_8192_forced_modes_sampled_rows(h, s, modes):
    res, e32 = _check(h, 8192, s, modes + ["auto"], seed=100 + s)
    for m, (e, _) in res.items():
        print(f"[8192 s={s}] {m} err {e:.3e}, fp32 err {e32:.3e}")


def test_unit_inputs_4096_error_below_1e6(h):
    """Section 3's unit test at the sweep's 4096 point: U(-1, 1) parts,
    relative Frobenius error <= 1e-6 on sampled rows in every emulated mode."""
    n = 4096
    A = qi.uniform_operand(n, n, (n, 7, 1))
    B = qi.uniform_operand(n, n, (n, 7, 2))
    rows = _rows(n, 7)
    exact = oracle.cgemm(0, 0, n, n, n, 1.0, A, B, rows=rows)
    for mode in ("fp16x", "tf32x", "auto"):
        e = oracle.rel_fro_error(_sampled(h, mode, A, B, n, rows)[0], exact)
        assert e <= 1e-6, (mode, e)
