"""GB300-native emulated-CGEMM tensor-network quantum circuit simulation.

Python face of libqcs (include/qcs.h).  Every numerical step runs in the CUDA
library; this module only passes device pointers, sizes and the current torch
stream.  Matrices are column-major: a torch tensor ``X`` of shape (rows, cols)
with ``X.stride() == (1, ld)`` (``ld >= rows``), complex64 (float32 for
``sgemm``), on the GPU.
"""
from __future__ import annotations

import ctypes
from typing import Optional

from . import _lib
from ._lib import (MODE_AUTO, MODE_BF16X3, MODE_BY_NAME, MODE_FP16X, MODE_FP16X_ROWCOL,
                   MODE_FP16X_SCALED, MODE_FP32, MODE_NAME, MODE_TF32X, OP_C, OP_N, OP_T,
                   SIZE_RULE_OFF, SIZE_RULE_PAPER,
                   SIZE_RULE_TUNED, QcsError)

__all__ = [
    "Handle", "cgemm", "sgemm", "fortran_empty_real", "exp_stats", "select", "split", "permute", "fortran_empty", "to_fortran",
    "MODE_AUTO", "MODE_FP16X", "MODE_FP16X_SCALED", "MODE_TF32X", "MODE_FP32", "MODE_BF16X3",
    "MODE_FP16X_ROWCOL", "rowcol_stats",
    "MODE_BY_NAME", "MODE_NAME", "OP_N", "OP_T", "OP_C", "QcsError",
    "SIZE_RULE_OFF", "SIZE_RULE_PAPER", "SIZE_RULE_TUNED",
]


def _torch():
    import torch

    return torch


def _mode(mode) -> int:
    if isinstance(mode, str):
        return MODE_BY_NAME[mode]
    return int(mode)


def _ld(X, rows: int) -> int:
    """Leading dimension of a column-major tensor view."""
    if X.dim() != 2:
        raise ValueError("expected a 2-D column-major tensor")
    if X.shape[1] <= 1:
        return max(rows, X.stride(1) if X.shape[1] == 1 else rows, 1)
    if X.stride(0) != 1:
        raise ValueError("tensor is not column-major (stride(0) must be 1)")
    return X.stride(1)


def fortran_empty(rows: int, cols: int, ld: Optional[int] = None, device="cuda"):
    """Uninitialised column-major complex64 (rows x cols) with leading dim ld."""
    torch = _torch()
    ld = rows if ld is None else ld
    base = torch.empty((cols, ld), dtype=torch.complex64, device=device)
    return base.t()[:rows]


def fortran_empty_real(rows: int, cols: int, ld: Optional[int] = None, device="cuda"):
    """Uninitialised column-major float32 (rows x cols) with leading dim ld."""
    torch = _torch()
    ld = rows if ld is None else ld
    base = torch.empty((cols, ld), dtype=torch.float32, device=device)
    return base.t()[:rows]


def to_fortran(x, device="cuda"):
    """Copy a 2-D array/tensor into a column-major complex64 device tensor."""
    torch = _torch()
    t = torch.as_tensor(x)
    if t.dim() == 1:
        t = t.reshape(-1, 1)
    out = fortran_empty(t.shape[0], t.shape[1], device=device)
    out.copy_(t.to(torch.complex64))
    return out


class Handle:
    """Owns a qcs handle (workspace, tolerance, size rule, tuning table)
    bound to a stream.  ``size_rule``: True/1 the paper's cut-offs, False/0
    none, 2 (SIZE_RULE_TUNED) the per-shape decisions of ``autotune_*``."""

    def __init__(self, stream=None, tol: float = 0.0, size_rule=True):
        torch = _torch()
        self.lib = _lib.load()
        self._h = ctypes.c_void_p()
        s = stream if stream is not None else torch.cuda.current_stream()
        _lib.check(self.lib.qcs_create(ctypes.byref(self._h), ctypes.c_void_p(s.cuda_stream)),
                   "qcs_create")
        self.stream = s
        self.set_tol(tol)
        self.set_size_rule(size_rule)

    @property
    def ptr(self):
        return self._h

    def set_stream(self, stream):
        _lib.check(self.lib.qcs_set_stream(self._h, ctypes.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def set_tol(self, t: float):
        _lib.check(self.lib.qcs_set_underflow_tol(self._h, float(t)), "qcs_set_underflow_tol")
        self.tol = float(t)

    def set_size_rule(self, rule):
        rule = int(rule) if not isinstance(rule, bool) else (SIZE_RULE_PAPER if rule else SIZE_RULE_OFF)
        _lib.check(self.lib.qcs_set_size_rule(self._h, rule))
        self.size_rule = rule

    def auto_counts(self, reset: bool = True, flops: bool = False):
        """{mode name: count} of what AUTO GEMMs on this handle selected on the
        device (qcs_get_auto_counts); synchronizes the stream.  With
        ``flops`` returns (counts, {mode name: summed 8 m n k})."""
        c = (ctypes.c_int64 * _lib.NUM_MODES)()
        f = (ctypes.c_double * _lib.NUM_MODES)()
        _lib.check(self.lib.qcs_get_auto_counts(self._h, c, f, 1 if reset else 0),
                   "qcs_get_auto_counts")
        counts = {MODE_NAME[i]: int(c[i]) for i in range(_lib.NUM_MODES)}
        if flops:
            return counts, {MODE_NAME[i]: float(f[i]) for i in range(_lib.NUM_MODES)}
        return counts

    def autotune_gemm(self, m: int, n: int, k: int, opA: int = OP_N, opB: int = OP_N,
                      reps: int = 3) -> dict:
        """Time AUTO / TF32X / FP32 for one shape and record the fastest in the
        handle's table (qcs_autotune_gemm)."""
        e = _lib.qcs_tune_entry_t()
        _lib.check(self.lib.qcs_autotune_gemm(self._h, int(opA), int(opB), int(m), int(n), int(k),
                                              int(reps), ctypes.byref(e)), "qcs_autotune_gemm")
        return _tune_dict(e)

    def tuning(self) -> list:
        """The handle's tuning table as a list of dicts (qcs_get_tuning)."""
        cnt = ctypes.c_int64()
        _lib.check(self.lib.qcs_get_tuning(self._h, None, 0, ctypes.byref(cnt)), "qcs_get_tuning")
        arr = (_lib.qcs_tune_entry_t * max(cnt.value, 1))()
        _lib.check(self.lib.qcs_get_tuning(self._h, arr, cnt.value, ctypes.byref(cnt)),
                   "qcs_get_tuning")
        return [_tune_dict(arr[i]) for i in range(cnt.value)]

    def set_tuning(self, entries: list):
        """Load entries (dicts as returned by ``tuning``) into the table."""
        arr = (_lib.qcs_tune_entry_t * max(len(entries), 1))()
        for i, d in enumerate(entries):
            e = arr[i]
            e.m, e.n, e.k, e.opA, e.opB = d["m"], d["n"], d["k"], d["opA"], d["opB"]
            for j in range(_lib.NUM_MODES):
                e.ms[j] = d["ms"].get(MODE_NAME[j], -1.0)
            e.best = MODE_BY_NAME[d["best"]]
            e.reps = d.get("reps", 0)
            e.splits = d.get("splits", 0)
            e.group_m = d.get("group_m", 0)
        _lib.check(self.lib.qcs_set_tuning(self._h, arr, len(entries)), "qcs_set_tuning")

    def set_instance_batch(self, instances: int):
        """Contraction-tree instances (slices / bitstrings) per group: plain
        FP32 steps become one batched launch per group (qcs_set_instance_batch)."""
        _lib.check(self.lib.qcs_set_instance_batch(self._h, int(instances)), "qcs_set_instance_batch")
        self.instance_batch = int(instances)

    def set_tc_schedule(self, group_m: int = 8, l2_promotion: int = 256):
        """Raster group and L2 promotion of the tensor-core kernels
        (qcs_set_tc_schedule); a performance knob only."""
        _lib.check(self.lib.qcs_set_tc_schedule(self._h, int(group_m), int(l2_promotion)),
                   "qcs_set_tc_schedule")

    def set_tc_splits(self, splits: int = 0):
        """K ranges per tensor-core GEMM (qcs_set_tc_splits): 0 chooses per
        shape, 1..16 forces the count."""
        _lib.check(self.lib.qcs_set_tc_splits(self._h, int(splits)), "qcs_set_tc_splits")

    def set_complex_products(self, products: int = 4):
        """Real products per emulated complex product of cgemm
        (qcs_set_complex_products): 4, the paper's expansion, or 3, Gauss's."""
        _lib.check(self.lib.qcs_set_complex_products(self._h, int(products)),
                   "qcs_set_complex_products")

    def set_group_budget(self, nbytes: int):
        """Bytes a grouped GPU-filling tree step may hold for its instances
        (qcs_set_group_budget; default 32 GiB, 0 = such steps per instance)."""
        _lib.check(self.lib.qcs_set_group_budget(self._h, int(nbytes)), "qcs_set_group_budget")

    def set_tc_multicast(self, enabled: bool):
        """Run the complex tensor-core kernel in clusters of two CTAs that share
        each op(B) box by TMA multicast (qcs_set_tc_multicast; off by default)."""
        _lib.check(self.lib.qcs_set_tc_multicast(self._h, int(bool(enabled))),
                   "qcs_set_tc_multicast")

    def set_rowcol_scaling(self, enabled: bool):
        """AUTO falls back to FP16 emulation with per-row (op(A)) and
        per-column (op(B)) power-of-two scaling before TF32X
        (qcs_set_rowcol_scaling; off by default)."""
        _lib.check(self.lib.qcs_set_rowcol_scaling(self._h, int(bool(enabled))),
                   "qcs_set_rowcol_scaling")

    def set_tc_pairs(self, enabled: bool):
        """Run the tensor-core kernels as CTA pairs on 256-row tiles, each CTA
        holding half of every op(B) operand (tcgen05 cta_group::2;
        qcs_set_tc_pairs; off by default)."""
        _lib.check(self.lib.qcs_set_tc_pairs(self._h, int(bool(enabled))), "qcs_set_tc_pairs")

    def set_tree_levels(self, enabled: bool):
        """Run a contraction tree level by level, the small plain-FP32 steps
        of each level as one launch (qcs_set_tree_levels; on by default)."""
        _lib.check(self.lib.qcs_set_tree_levels(self._h, int(bool(enabled))),
                   "qcs_set_tree_levels")

    def set_fused_split(self, enabled: bool):
        """TF32X split inside the tensor-core kernel's staging
        (qcs_set_fused_split) instead of a separate pass."""
        _lib.check(self.lib.qcs_set_fused_split(self._h, int(bool(enabled))),
                   "qcs_set_fused_split")

    def set_wait_budget(self, ns: int):
        """Bound of every device-side wait in the tensor-core kernels
        (qcs_set_wait_budget), in nanoseconds."""
        _lib.check(self.lib.qcs_set_wait_budget(self._h, int(ns)), "qcs_set_wait_budget")

    def debug_stall_producer(self, enabled: bool):
        """Test hook (qcs_debug_stall_producer): the tensor-core kernels'
        TMA producer issues no loads, so their waits run out."""
        _lib.check(self.lib.qcs_debug_stall_producer(self._h, int(bool(enabled))),
                   "qcs_debug_stall_producer")

    def measure_fma_peak(self) -> float:
        """FP32 FMA rate of the CUDA cores in TFLOP/s (qcs_measure_fma_peak):
        the roofline of the plain FP32 CGEMM."""
        out = ctypes.c_double()
        _lib.check(self.lib.qcs_measure_fma_peak(self._h, ctypes.byref(out)),
                   "qcs_measure_fma_peak")
        return out.value

    def set_drain_stages(self, stages: int):
        _lib.check(self.lib.qcs_set_drain_stages(self._h, int(stages)), "qcs_set_drain_stages")
        self.drain_stages = int(stages)

    def set_profiling(self, on: bool):
        _lib.check(self.lib.qcs_set_profiling(self._h, 1 if on else 0))

    def get_profile(self):
        """{stage: (milliseconds, event pairs)} accumulated since the last read."""
        n = len(_lib.PROFILE_STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        _lib.check(self.lib.qcs_get_profile(self._h, ms, cnt, n), "qcs_get_profile")
        return {name: (ms[i], cnt[i]) for i, name in enumerate(_lib.PROFILE_STAGES)}

    def sync(self):
        _lib.check(self.lib.qcs_sync(self._h), "qcs_sync")

    def close(self):
        if self._h:
            self.lib.qcs_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _tune_dict(e) -> dict:
    return {"m": e.m, "n": e.n, "k": e.k, "opA": e.opA, "opB": e.opB,
            "ms": {MODE_NAME[j]: e.ms[j] for j in range(_lib.NUM_MODES) if e.ms[j] >= 0},
            "best": MODE_NAME[e.best], "reps": e.reps, "splits": e.splits, "group_m": e.group_m}


def cgemm(h: Handle, A, B, C=None, *, m=None, n=None, k=None, alpha=1.0, beta=0.0,
          opA=OP_N, opB=OP_N, mode="auto", desc_out=None):
    """C = alpha op(A) op(B) + beta C with qcs_cgemm; returns C.

    A, B, C are column-major complex64 device tensors (see module doc).  If C
    is None a new m x n tensor is allocated (beta must then be 0).
    ``desc_out``: optional int32 device tensor with 4 elements receiving the
    descriptor (mode, sA, sB, 0) the GEMM ran with.
    """
    torch = _torch()
    rA, cA = A.shape
    rB, cB = B.shape
    m = (rA if opA == OP_N else cA) if m is None else m
    k = (cA if opA == OP_N else rA) if k is None else k
    n = (cB if opB == OP_N else rB) if n is None else n
    if C is None:
        if complex(beta) != 0:
            raise ValueError("beta != 0 needs C")
        C = fortran_empty(m, n, device=A.device)
    lda = _ld(A, rA)
    ldb = _ld(B, rB)
    ldc = _ld(C, C.shape[0])
    al = _lib.qcs_c32(complex(alpha).real, complex(alpha).imag)
    be = _lib.qcs_c32(complex(beta).real, complex(beta).imag)
    dp = ctypes.c_void_p(desc_out.data_ptr()) if desc_out is not None else None
    rc = h.lib.qcs_cgemm(h.ptr, _mode(mode), int(opA), int(opB), m, n, k, ctypes.byref(al),
                         ctypes.c_void_p(A.data_ptr()), lda, ctypes.c_void_p(B.data_ptr()), ldb,
                         ctypes.byref(be), ctypes.c_void_p(C.data_ptr()), ldc, dp)
    _lib.check(rc, "qcs_cgemm")
    del torch
    return C


def selection_stats(h: Handle, A, B, *, opA=OP_N, opB=OP_N):
    """The Section 4.1 counts AUTO's selection takes for op(A) op(B)
    (qcs_selection_stats): a list of two dicts (op(A), op(B)) with e_max
    (None if no finite nonzero scalar), stage2, n_nonzero, n_nonfinite,
    n_under_fp16, n_under_window, and the descriptor (mode, sA, sB)."""
    rA, cA = A.shape
    rB, cB = B.shape
    m = rA if opA == OP_N else cA
    k = cA if opA == OP_N else rA
    n = cB if opB == OP_N else rB
    out = (_lib.qcs_selection_stats_t * 2)()
    d = _lib.qcs_gemm_desc_t()
    _lib.check(h.lib.qcs_selection_stats(h.ptr, int(opA), int(opB), m, n, k,
                                         ctypes.c_void_p(A.data_ptr()), _ld(A, rA),
                                         ctypes.c_void_p(B.data_ptr()), _ld(B, rB), out,
                                         ctypes.byref(d)), "qcs_selection_stats")
    res = []
    for o in out:
        res.append({"e_max": None if o.e_max == -128 else int(o.e_max), "stage2": bool(o.stage2),
                    "n_nonzero": int(o.n_nonzero), "n_nonfinite": int(o.n_nonfinite),
                    "n_under_fp16": int(o.n_under_fp16), "n_under_window": int(o.n_under_window)})
    return res, (int(d.mode), int(d.sA), int(d.sB))


def rowcol_stats(h: Handle, A, B, *, opA=OP_N, opB=OP_N):
    """The per-line statistics of per-row / per-column scaling
    (qcs_rowcol_stats): (emaxA, emaxB, counts) as CUDA int32 tensors of m
    and n biased exponents (-1: no nonzero finite scalar) and an int64
    tensor [under A, nonzero A, under B, nonzero B]."""
    torch = _torch()
    rA, cA = A.shape
    rB, cB = B.shape
    m = rA if opA == OP_N else cA
    k = cA if opA == OP_N else rA
    n = cB if opB == OP_N else rB
    ea = torch.empty(m, dtype=torch.int32, device=A.device)
    eb = torch.empty(n, dtype=torch.int32, device=A.device)
    cnt = torch.empty(4, dtype=torch.int64, device=A.device)
    _lib.check(h.lib.qcs_rowcol_stats(h.ptr, int(opA), int(opB), m, n, k,
                                      ctypes.c_void_p(A.data_ptr()), _ld(A, rA),
                                      ctypes.c_void_p(B.data_ptr()), _ld(B, rB),
                                      ctypes.c_void_p(ea.data_ptr()), ctypes.c_void_p(eb.data_ptr()),
                                      ctypes.c_void_p(cnt.data_ptr())), "qcs_rowcol_stats")
    return ea, eb, cnt


def fidelity_stats(h: Handle, a, ref=None) -> dict:
    """FP64 sums on the GPU (qcs_fidelity_stats) of a (complex128 or
    complex64 CUDA tensor) against ref (complex128 CUDA tensor of the same
    number of elements, or None): norms, overlap, error; with ref also the
    fidelity |<ref|a>|^2 / (<a|a><ref|ref>) and the relative L2 error.
    Synchronises to return host floats."""
    import torch

    a = a.contiguous()
    if a.dtype not in (torch.complex128, torch.complex64):
        raise TypeError("a must be complex128 or complex64")
    n = a.numel()
    r = None
    if ref is not None:
        r = ref.contiguous()
        if r.dtype != torch.complex128 or r.numel() != n:
            raise ValueError("ref must be complex128 with as many elements as a")
    out = torch.zeros(6, dtype=torch.float64, device=a.device)
    _lib.check(h.lib.qcs_fidelity_stats(h.ptr, ctypes.c_void_p(a.data_ptr()),
                                        1 if a.dtype == torch.complex64 else 0,
                                        ctypes.c_void_p(r.data_ptr()) if r is not None else None,
                                        n, ctypes.c_void_p(out.data_ptr())),
               "qcs_fidelity_stats")
    v = out.cpu().tolist()
    res = {"norm2": v[0]}
    if r is not None:
        res.update({"ref_norm2": v[1], "overlap": complex(v[2], v[3]), "err2": v[4],
                    "max_abs_err": v[5],
                    "fidelity": (v[2] ** 2 + v[3] ** 2) / (v[0] * v[1]) if v[0] * v[1] > 0 else 0.0,
                    "rel_l2_err": (v[4] / v[1]) ** 0.5 if v[1] > 0 else float("inf")})
    return res


def sgemm(h: Handle, A, B, C=None, *, m=None, n=None, k=None, alpha=1.0, beta=0.0,
          opA=OP_N, opB=OP_N, mode="auto", desc_out=None):
    """C = alpha op(A) op(B) + beta C for real matrices with qcs_sgemm;
    returns C.  A, B, C are column-major float32 device tensors; OP_C acts
    as OP_T.  If C is None a new m x n tensor is allocated (beta must then
    be 0).  ``desc_out`` as for cgemm."""
    rA, cA = A.shape
    rB, cB = B.shape
    m = (rA if opA == OP_N else cA) if m is None else m
    k = (cA if opA == OP_N else rA) if k is None else k
    n = (cB if opB == OP_N else rB) if n is None else n
    for X in (A, B) + ((C,) if C is not None else ()):
        if X.dtype != _torch().float32:
            raise TypeError("sgemm takes float32 tensors")
    if C is None:
        if float(beta) != 0:
            raise ValueError("beta != 0 needs C")
        C = fortran_empty_real(m, n, device=A.device)
    al = ctypes.c_float(float(alpha))
    be = ctypes.c_float(float(beta))
    dp = ctypes.c_void_p(desc_out.data_ptr()) if desc_out is not None else None
    rc = h.lib.qcs_sgemm(h.ptr, _mode(mode), int(opA), int(opB), m, n, k, ctypes.byref(al),
                         ctypes.c_void_p(A.data_ptr()), _ld(A, rA), ctypes.c_void_p(B.data_ptr()),
                         _ld(B, rB), ctypes.byref(be), ctypes.c_void_p(C.data_ptr()),
                         _ld(C, C.shape[0]), dp)
    _lib.check(rc, "qcs_sgemm")
    return C


def exp_stats(h: Handle, X, out=None):
    """Exponent statistics of a column-major matrix into an int64 device
    tensor of 258 entries (hist[256], n_zero, n)."""
    torch = _torch()
    rows, cols = X.shape
    if out is None:
        out = torch.zeros(258, dtype=torch.int64, device=X.device)
    _lib.check(h.lib.qcs_exp_stats(h.ptr, rows, cols, ctypes.c_void_p(X.data_ptr()), _ld(X, rows),
                                   ctypes.c_void_p(out.data_ptr())), "qcs_exp_stats")
    return out


def select(h: Handle, statsA, statsB, desc=None):
    """Mode selection from two statistics tensors; returns an int32 device
    tensor (mode, sA, sB, 0)."""
    torch = _torch()
    if desc is None:
        desc = torch.zeros(4, dtype=torch.int32, device=statsA.device)
    _lib.check(h.lib.qcs_select(h.ptr, ctypes.c_void_p(statsA.data_ptr()),
                                ctypes.c_void_p(statsB.data_ptr()), ctypes.c_void_p(desc.data_ptr())),
               "qcs_select")
    return desc


def split(h: Handle, desc, which: int, op: int, X, R: int, K: int):
    """The split stage alone: returns the 4 planes (hi.re, hi.im, lo.re,
    lo.im) as a (4, R, K) int16 tensor (16-bit modes) or float32 tensor
    (TF32X)."""
    torch = _torch()
    mode = int(desc[0].item())
    dt = torch.float32 if mode == MODE_TF32X else torch.int16
    planes = torch.zeros((4, R, K), dtype=dt, device=X.device)
    rows = (R if op == OP_N else K) if which == 0 else (K if op == OP_N else R)
    _lib.check(h.lib.qcs_split(h.ptr, ctypes.c_void_p(desc.data_ptr()), which, op, R, K,
                               ctypes.c_void_p(X.data_ptr()), _ld(X, rows),
                               ctypes.c_void_p(planes.data_ptr()), K, R * K), "qcs_split")
    return planes


def permute(h: Handle, src, dims, strides, offset: int = 0, out=None):
    """Strided gather (first index fastest) of a complex64 device tensor."""
    torch = _torch()
    total = 1
    for d in dims:
        total *= int(d)
    if out is None:
        out = torch.empty(total, dtype=torch.complex64, device=src.device)
    r = len(dims)
    D = (ctypes.c_int64 * max(r, 1))(*[int(d) for d in dims])
    S = (ctypes.c_int64 * max(r, 1))(*[int(s) for s in strides])
    _lib.check(h.lib.qcs_permute(h.ptr, r, D, S, int(offset), ctypes.c_void_p(src.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), None), "qcs_permute")
    return out
