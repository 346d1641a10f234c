"""The drop-in route of the paper's library (Section 3): an unmodified
application's cuBLAS GEMMs, redirected by libqcs_cublas.so loaded ahead of
cuBLAS, run as emulated GEMMs.  Here the application is PyTorch in a child
process started with LD_PRELOAD: torch.matmul (cublasCgemm, cublasSgemm) and
torch.bmm (cublasCgemmStridedBatched, cublasSgemmStridedBatched) on complex64
and float32 CUDA tensors.  Results are
checked against the FP64 oracle, and the library's own counters show which
calls it took and which it passed to cuBLAS."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import need_gpu

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SHIM = os.path.join(ROOT, "paper_2303_08989_gb300", "_build", "libqcs_cublas.so")

CHILD = r"""
import ctypes, json, sys
import numpy as np
import torch
d = np.load(sys.argv[1])
A = torch.from_numpy(d["A"]).cuda()
B = torch.from_numpy(d["B"]).cuda()
Ab = torch.from_numpy(d["Ab"]).cuda()
Bb = torch.from_numpy(d["Bb"]).cuda()
C = torch.matmul(A, B)
Cb = torch.bmm(Ab, Bb)
torch.backends.cuda.matmul.allow_tf32 = False
R = torch.matmul(A.real.contiguous(), B.real.contiguous())
Rb = torch.bmm(Ab.real.contiguous(), Bb.real.contiguous())
torch.cuda.synchronize()
shim = ctypes.CDLL(sys.argv[2])
taken, passed = ctypes.c_longlong(), ctypes.c_longlong()
shim.qcs_cublas_shim_counts(ctypes.byref(taken), ctypes.byref(passed))
np.savez(sys.argv[3], C=C.cpu().numpy(), Cb=Cb.cpu().numpy(), R=R.cpu().numpy(),
         Rb=Rb.cpu().numpy())
print(json.dumps({"taken": taken.value, "passed": passed.value}))
"""


def _run_child(tmp_path, env_extra):
    rng_seed = 17
    m, k, n, batch = 640, 576, 704, 3
    # row-major torch operands; torch hands cuBLAS the column-major transposes
    A = qi.cgemm_operand(m, k, 0, seed=(rng_seed, 1))
    B = qi.cgemm_operand(k, n, 0, seed=(rng_seed, 2))
    Ab = np.stack([qi.cgemm_operand(m // 2, k, 4, seed=(rng_seed, 3, b)) for b in range(batch)])
    Bb = np.stack([qi.cgemm_operand(k, n // 2, 4, seed=(rng_seed, 4, b)) for b in range(batch)])
    inp = tmp_path / "in.npz"
    out = tmp_path / "out.npz"
    np.savez(inp, A=np.ascontiguousarray(A), B=np.ascontiguousarray(B),
             Ab=np.ascontiguousarray(Ab), Bb=np.ascontiguousarray(Bb))
    env = dict(os.environ)
    env["LD_PRELOAD"] = SHIM + (":" + env["LD_PRELOAD"] if env.get("LD_PRELOAD") else "")
    env.update(env_extra)
    r = subprocess.run([sys.executable, "-c", CHILD, str(inp), SHIM, str(out)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    counts = json.loads(r.stdout.strip().splitlines()[-1])
    res = np.load(out)
    A64, B64 = A.astype(np.complex128), B.astype(np.complex128)
    errs = {"matmul": oracle.rel_fro_error(res["C"], A64 @ B64),
            "bmm": max(oracle.rel_fro_error(res["Cb"][b], Ab[b].astype(np.complex128)
                                            @ Bb[b].astype(np.complex128))
                       for b in range(batch)),
            "smatmul": oracle.rel_fro_error(res["R"], A64.real @ B64.real),
            "sbmm": max(oracle.rel_fro_error(res["Rb"][b], Ab[b].real.astype(np.float64)
                                             @ Bb[b].real.astype(np.float64))
                        for b in range(batch))}
    return counts, errs


def test_cublas_complex_gemms_run_emulated(tmp_path):
    """QCS_CUBLAS_MODE=auto with the size rule off: all four calls run
    through qcs_cgemm / qcs_sgemm (statistics, selection, tensor-core
    emulation) at FP32-level error."""
    need_gpu()
    assert os.path.exists(SHIM), "build() makes libqcs_cublas.so"
    counts, errs = _run_child(tmp_path, {"QCS_CUBLAS_MODE": "auto", "QCS_SIZE_RULE": "0",
                                         "QCS_UNDERFLOW_TOL": "0.1"})
    assert counts == {"taken": 4, "passed": 0}, counts
    assert max(errs.values()) < 1e-6, errs


@pytest.mark.parametrize("mode", ["tf32x", "fp32"])
def test_cublas_shim_forced_modes(tmp_path, mode):
    need_gpu()
    counts, errs = _run_child(tmp_path, {"QCS_CUBLAS_MODE": mode})
    assert counts == {"taken": 4, "passed": 0}, counts
    bar = 1e-6 if mode == "tf32x" else 5e-6
    assert max(errs.values()) < bar, errs


def test_cublas_shim_passes_through_when_asked(tmp_path):
    """QCS_CUBLAS_MODE=cublas: every call goes to the next cuBLAS definition."""
    need_gpu()
    counts, errs = _run_child(tmp_path, {"QCS_CUBLAS_MODE": "cublas"})
    assert counts == {"taken": 0, "passed": 4}, counts
    assert max(errs.values()) < 1e-4, errs
