"""GPU tests of the measured size rule (qcs_autotune_gemm / qcs_autotune_tree,
QCS_SIZE_RULE_TUNED) and of the device-side count of what the automatic
selection chose (qcs_get_auto_counts).  Results stay checked against the
FP64 oracle: a tuned decision only moves a GEMM between paths of the same
accuracy level."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import dev, host, lib, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture()
def h():
    need_gpu()
    hd = lib().Handle(tol=0.1, size_rule=False)
    yield hd
    hd.close()


def _gemm(h, mode, A, B, m, n, k):
    q = lib()
    C = q.fortran_empty(m, n)
    desc = torch.zeros(4, dtype=torch.int32, device="cuda")
    q.cgemm(h, dev(A), dev(B), C, mode=mode, desc_out=desc)
    torch.cuda.synchronize()
    h.sync()
    return host(C).astype(np.complex128), desc.cpu().numpy()


def test_auto_counts_follow_the_device_selection(h):
    m = n = k = 96
    A = qi.cgemm_operand(m, k, 0, seed=(1, 1))
    B = qi.cgemm_operand(k, n, 0, seed=(1, 2))
    T3 = qi.typed_matrix(k, n, 3, seed=(1, 3))
    bad = A.copy(order="F")
    bad[3, 4] = complex(np.inf, 0)
    assert h.auto_counts(reset=True) == {name: 0 for name in lib().MODE_BY_NAME}
    _gemm(h, "auto", A, B, m, n, k)
    _gemm(h, "auto", A, T3, m, n, k)
    _gemm(h, "auto", bad, B, m, n, k)
    _gemm(h, "fp32", A, B, m, n, k)  # forced modes do not count
    want = {name: 0 for name in lib().MODE_BY_NAME}
    for X, Y in ((A, B), (A, T3), (bad, B)):
        mode = oracle.select_mode(oracle.stats_summary(*oracle.exp_stats(X)),
                                  oracle.stats_summary(*oracle.exp_stats(Y)), 0.1)[0]
        want[lib().MODE_NAME[mode]] += 1
    counts, flops = h.auto_counts(reset=True, flops=True)
    assert counts == want
    assert flops == {mode: 8.0 * m * n * k * cnt for mode, cnt in want.items()}
    assert sum(h.auto_counts(reset=False).values()) == 0


def test_autotune_prunes_and_picks():
    """A tiny GEMM cannot repay the statistics and split launches (FP32
    wins); a large square one cannot lose on the tensor cores (FP32 is
    pruned without being run)."""
    need_gpu()
    hd = lib().Handle(tol=0.1, size_rule=False)
    try:
        tiny = hd.autotune_gemm(8, 8, 8, reps=5)
        assert set(tiny["ms"]) == {"auto", "tf32x", "fp32"}
        assert all(v > 0 for v in tiny["ms"].values())
        assert tiny["best"] == "fp32"
        big = hd.autotune_gemm(4096, 4096, 4096, reps=2)
        assert "fp32" not in big["ms"]
        assert big["best"] in ("auto", "tf32x")
        keys = [(e["m"], e["n"], e["k"]) for e in hd.tuning()]
        assert keys == sorted(keys) and (8, 8, 8) in keys and (4096, 4096, 4096) in keys
    finally:
        hd.close()


@pytest.mark.parametrize("best", ["auto", "tf32x", "fp32"])
def test_tuned_rule_applies_the_table(h, best):
    """QCS_SIZE_RULE_TUNED runs the recorded decision for the exact key
    (m, n, k, opA, opB); other shapes fall back to the paper's cut-offs."""
    q = lib()
    m, n, k = 160, 96, 64
    A = qi.cgemm_operand(m, k, 0, seed=(2, 1))
    B = qi.cgemm_operand(k, n, 0, seed=(2, 2))
    h.set_tuning([{"m": m, "n": n, "k": k, "opA": 0, "opB": 0, "ms": {}, "best": best}])
    h.set_size_rule(q.SIZE_RULE_TUNED)
    got, d = _gemm(h, "auto", A, B, m, n, k)
    sel = oracle.select_mode(oracle.stats_summary(*oracle.exp_stats(A)),
                             oracle.stats_summary(*oracle.exp_stats(B)), 0.1)[0]
    want = {"auto": sel, "tf32x": q.MODE_TF32X, "fp32": q.MODE_FP32}[best]
    assert d[0] == want
    exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
    assert oracle.rel_fro_error(got, exact) < 1e-6
    # a shape that was never tuned: the paper's rule (min(m, n, k) < 512 -> FP32)
    _, d2 = _gemm(h, "auto", A[:m - 1].copy(order="F"), B, m - 1, n, k)
    assert d2[0] == q.MODE_FP32


def test_set_tuning_rejects_bad_entries(h):
    q = lib()
    with pytest.raises(q.QcsError):
        h.set_tuning([{"m": 4, "n": 4, "k": 4, "opA": 0, "opB": 0, "ms": {}, "best": "fp16x"}])
    with pytest.raises(q.QcsError):
        h.set_tuning([{"m": 0, "n": 4, "k": 4, "opA": 0, "opB": 0, "ms": {}, "best": "fp32"}])
    assert h.tuning() == []


def test_autotuned_tree_matches_oracle():
    """Tune every AUTO shape of a contraction plan (forward and adjoint),
    then contract under the tuned rule: amplitudes and gradients stay at the
    FP32 level against the FP64 oracle."""
    need_gpu()
    import paper_2303_08989_gb300.tn as tn

    q = lib()
    hd = q.Handle(tol=0.1, size_rule=q.SIZE_RULE_TUNED)
    try:
        circ = qi.random_grid_circuit(3, 4, 8, seed=0)
        bits = qi.random_bitstrings(12, 16, seed=1)
        plan = tn.plan_circuit(circ, bits, seed=2, mode=q.MODE_AUTO)
        cp = tn.CompiledPlan(plan)
        n1 = cp.autotune(hd, backward=True, reps=1)
        shapes = {(s.m, s.n, s.k) for s in plan.steps}
        assert 0 < n1 <= 3 * len(plan.steps)
        assert {(e["m"], e["n"], e["k"]) for e in hd.tuning()} >= shapes
        assert cp.autotune(hd, backward=True, reps=1) == 0  # all shapes known now
        out = cp.forward(hd)
        torch.cuda.synchronize()
        hd.sync()
        ref = oracle.sv_amplitudes(circ, bits)
        a = out.cpu().numpy()[:, 0]
        assert oracle.fidelity(ref, a) >= 1 - 1e-5
        assert np.max(np.abs(a - ref)) <= 1e-5 * np.max(np.abs(ref))
    finally:
        hd.close()


def test_autotune_measures_the_k_range_count():
    """One output tile and a long k: the tuner also times the faster emulated
    candidate at several K-range counts and records the fastest in
    ``splits``; under the tuned rule that count runs.  A table entry's count
    round-trips through qcs_get_tuning / qcs_set_tuning, is validated, and
    results stay at the FP32 level against the FP64 oracle."""
    need_gpu()
    q = lib()
    m, n, k = 128, 96, 4096
    hd = q.Handle(tol=0.1, size_rule=False)
    try:
        e = hd.autotune_gemm(m, n, k, reps=2)
        assert 1 <= e["splits"] <= 16
        big = hd.autotune_gemm(4096, 2048, 64, reps=1)  # 512 tiles >= 2 x 152: not measured
        assert big["splits"] == 0
        A = qi.cgemm_operand(m, k, 0, seed=(5, 1))
        B = qi.cgemm_operand(k, n, 0, seed=(5, 2))
        exact = oracle.cgemm(0, 0, m, n, k, 1.0, A, B)
        hd.set_size_rule(q.SIZE_RULE_TUNED)
        for splits in (e["splits"], 3, 1):
            entry = dict(e, splits=splits, best="auto")
            hd.set_tuning([entry])
            assert [x["splits"] for x in hd.tuning() if x["k"] == k] == [splits]
            got, d = _gemm(hd, "auto", A, B, m, n, k)
            assert d[0] == q.MODE_FP16X
            assert oracle.rel_fro_error(got, exact) < 1e-6, splits
        with pytest.raises(q.QcsError):
            hd.set_tuning([dict(e, splits=17)])
    finally:
        hd.close()


def test_tuner_measures_the_raster_and_results_do_not_depend_on_it():
    """Shapes with at least twice as many output tiles as SMs get a raster
    group measured by the tuner; under the tuned rule the table's raster is
    used, and changing it only reorders tiles (the same bits)."""
    need_gpu()
    q = lib()
    hd = q.Handle(tol=0.1, size_rule=False)
    try:
        e = hd.autotune_gemm(4096, 4096, 1024, reps=1)  # 1024 tiles of 128 x 128
        assert e["group_m"] in (2, 4, 8, 16), e
        small = hd.autotune_gemm(1024, 1024, 1024, reps=1)  # 64 tiles: K ranges instead
        assert small["group_m"] == 0
        m, n, k = 2048, 2304, 256
        A = dev(qi.cgemm_operand(m, k, 0, seed=(61, 1)))
        B = dev(qi.cgemm_operand(k, n, 0, seed=(61, 2)))
        outs = []
        hd.set_size_rule(q.SIZE_RULE_TUNED)
        for gm in (1, 3, 16):
            hd.set_tuning([{"m": m, "n": n, "k": k, "opA": 0, "opB": 0, "ms": {}, "best": "auto",
                            "splits": 1, "group_m": gm}])
            assert [t["group_m"] for t in hd.tuning() if (t["m"], t["n"], t["k"]) == (m, n, k)] == [gm]
            outs.append(q.cgemm(hd, A, B, mode="auto"))
            torch.cuda.synchronize()
            hd.sync()
        assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
        from paper_2303_08989_gb300 import _lib as L

        with pytest.raises(L.QcsError):
            hd.set_tuning([{"m": m, "n": n, "k": k, "opA": 0, "opB": 0, "ms": {}, "best": "auto",
                            "group_m": 65}])
    finally:
        hd.close()
