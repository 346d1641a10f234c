"""Shared helpers of the GPU tests (device setup, layout conversions)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lib():
    import paper_2303_08989_gb300 as q

    return q


def dev(x: np.ndarray):
    """numpy column-major complex64 (ld, cols) -> device tensor with the same strides."""
    assert x.dtype == np.complex64 and x.flags.f_contiguous
    ld, cols = x.shape
    base = torch.empty((cols, ld), dtype=torch.complex64, device="cuda")
    base.copy_(torch.from_numpy(np.ascontiguousarray(x.T)))
    return base.t()


def host(t) -> np.ndarray:
    """device column-major tensor -> numpy Fortran complex64 of the same shape."""
    a = t.t().contiguous().cpu().numpy().T
    return np.asfortranarray(a)


def abs_bound(A: np.ndarray, B: np.ndarray, opA: int, opB: int, m: int, k: int, n: int) -> np.ndarray:
    """(|op(A)| |op(B)|)_ij in FP64 with |z| = |re| + |im| (bounds every real
    product term that enters C_ij)."""
    def op(X, o, r, c):
        X = X.astype(np.complex128)
        M = X[:r, :c] if o == 0 else (X[:c, :r].T if o == 1 else X[:c, :r].conj().T)
        return np.abs(M.real) + np.abs(M.imag)

    return op(A, opA, m, k) @ op(B, opB, k, n)
