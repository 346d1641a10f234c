"""Level launches of the contraction-tree executor (qcs_set_tree_levels):
the small plain-FP32 steps of each tree level run as one launch over all
of them and all instances of a group, reading their operands through
offset tables.  Against the FP64 oracle and against the step-by-step
executor (levels off), eagerly, in groups, from CUDA graphs, and through
the adjoint."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import lib, need_gpu, torch

pytestmark = pytest.mark.gpu


def _tn():
    import paper_2303_08989_gb300.tn as tn

    return tn


def _forward(hd, plan):
    tn = _tn()
    cp = tn.CompiledPlan(plan)
    out = cp.forward(hd)
    torch.cuda.synchronize()
    hd.sync()
    return out.cpu().numpy(), cp.last_info


def _both(plan, G=1, size_rule=True, tol=0.0):
    """(levels on, levels off) results and infos of one plan."""
    q = lib()
    hd = q.Handle(tol=tol, size_rule=size_rule)
    try:
        hd.set_instance_batch(G)
        on, info_on = _forward(hd, plan)
        hd.set_tree_levels(False)
        off, info_off = _forward(hd, plan)
    finally:
        hd.close()
    return on, info_on, off, info_off


CASES = [
    # (rows, cols, depth, circuit seed, bitstrings, slices, absorb, G)
    (3, 4, 8, 0, 64, 0, False, 1),
    (3, 4, 8, 0, 64, 0, False, 16),
    (3, 4, 8, 3, 4, 3, True, 5),
    (4, 4, 10, 8, 6, 2, False, 24),
    (4, 5, 10, 1, 3, 4, True, 7),
]


@pytest.mark.parametrize("rows,cols,depth,cseed,nb,n_slices,absorb,G", CASES)
def test_levels_match_oracle_and_step_by_step(rows, cols, depth, cseed, nb, n_slices, absorb,
                                              G):
    """Amplitudes of random grid circuits (bitstring batches, sliced indices
    with per-instance leaf offsets, directly read leaves, absorbed gates,
    ragged last groups) with level launches against the FP64 state vector
    and against the step-by-step run: the same GEMM count, level launches
    covering most GEMMs, and agreement at FP32 rounding."""
    need_gpu()
    tn = _tn()
    n = rows * cols
    circ = qi.random_grid_circuit(rows, cols, depth, seed=cseed)
    bits = qi.random_bitstrings(n, nb, seed=cseed + 1)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=n_slices, absorb=absorb)
    on, info_on, off, info_off = _both(plan, G=G)
    assert info_on.gemm_count == info_off.gemm_count == plan.n_instances * len(plan.steps)
    assert info_off.level_launches == 0 and info_off.level_gemms == 0
    assert info_on.level_launches > 0
    assert info_on.level_gemms >= info_on.gemm_count // 2
    # at most one level launch per level and group (plus one per level and instance
    # after the batched part)
    assert info_on.level_launches < info_on.level_gemms
    ref = oracle.sv_amplitudes(circ, bits)
    for got in (on, off):
        assert oracle.fidelity(ref, got[:, 0]) >= 1 - 1e-5
        assert np.max(np.abs(got[:, 0] - ref)) <= 1e-5 * np.max(np.abs(ref))
    scale = np.max(np.abs(off))
    assert np.max(np.abs(on - off)) <= 2e-6 * scale


def test_levels_in_groups_and_graphs_are_bit_identical():
    """With level launches, group sizes 1, 6 and 32 and a CUDA-graph replay
    give the same bits: each output element is one FP32 FMA chain in a fixed
    order, whatever the launch it runs in."""
    need_gpu()
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(4, 4, 10, seed=8)
    bits = qi.random_bitstrings(16, 6, seed=9)
    plan = tn.plan_circuit(circ, bits, seed=4, n_slices=2)
    hd = q.Handle(tol=0.0, size_rule=True)
    try:
        one, _ = _forward(hd, plan)
        for G in (6, 32):
            hd.set_instance_batch(G)
            got, _ = _forward(hd, plan)
            assert np.array_equal(got, one), G
            cp = tn.CompiledPlan(plan)
            g, out = cp.graph(hd)
            out.zero_()
            g.launch()
            torch.cuda.synchronize()
            hd.sync()
            assert np.array_equal(out.cpu().numpy(), one), G
            g.close()
    finally:
        hd.close()


def test_levels_with_emulated_steps_between():
    """Every third step emulated (FP16X) and the others plain FP32: the level
    schedule interleaves level launches with the emulated steps' own launch
    sequences; the results match the step-by-step run and the FP64 oracle."""
    need_gpu()
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(3, 4, 8, seed=3)
    bits = qi.random_bitstrings(12, 4, seed=4)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=3)
    for i, st in enumerate(plan.steps):
        st.mode = q.MODE_FP16X if i % 3 == 2 else q.MODE_FP32
    on, info_on, off, _ = _both(plan, G=4, size_rule=False)
    assert info_on.level_launches > 0
    n_fp16x = sum(1 for st in plan.steps if st.mode == q.MODE_FP16X)
    assert info_on.mode_count[q.MODE_FP16X] == plan.n_instances * n_fp16x
    ref = oracle.sv_amplitudes(circ, bits)
    for got in (on, off):
        assert oracle.fidelity(ref, got[:, 0]) >= 1 - 1e-5
    assert np.max(np.abs(on - off)) <= 1e-5 * np.max(np.abs(off))


@pytest.mark.parametrize("n_slices", [0, 2])
def test_adjoint_with_level_launches(n_slices):
    """The adjoint recomputes each instance's forward pass with level
    launches; the gradient of sum log|a|^2 matches the FP64 adjoint and the
    step-by-step run."""
    need_gpu()
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(2, 3, 4, seed=4, theta=None, phi=None, param_seed=5)
    bits = qi.random_bitstrings(6, 8, seed=6)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=n_slices, mode=q.MODE_FP32)
    params0 = np.array([g.params for g in circ.gates if g.name == "fsim"], dtype=np.float64)
    grads = []
    hd = q.Handle(tol=0.0, size_rule=True)
    try:
        for levels in (True, False):
            hd.set_tree_levels(levels)
            params = torch.tensor(params0, dtype=torch.float32, device="cuda",
                                  requires_grad=True)
            cp = tn.CompiledPlan(plan, leaf_data=[])
            leaves = tn.torch_leaves(plan.net, circ, params)
            amps = tn.contract(cp, hd, leaves)
            loss = torch.log(amps.abs() ** 2).sum()
            loss.backward()
            torch.cuda.synchronize()
            hd.sync()
            grads.append(params.grad.double().cpu().numpy())
            info = cp.last_info  # the backward call's
            if levels:
                # forward recompute and adjoint: most GEMMs inside level launches
                assert info.level_launches > 0
                assert info.level_gemms >= info.gemm_count // 2
            else:
                assert info.level_launches == 0
    finally:
        hd.close()
    _, g_ref = oracle.loss_and_grad(circ, bits)
    for g in grads:
        assert np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref) < 1e-4
    assert np.linalg.norm(grads[0] - grads[1]) / np.linalg.norm(grads[1]) < 1e-5


def test_level_setter_rejects_bad_values():
    need_gpu()
    q = lib()
    hd = q.Handle()
    try:
        rc = hd.lib.qcs_set_tree_levels(hd._h, 2)
        assert rc == -1
        hd.set_tree_levels(False)
        hd.set_tree_levels(True)
    finally:
        hd.close()


def test_adjoint_rejects_overlapping_leaf_gradients():
    """The adjoints of a level's steps add into their leaves' gradients at
    the same time, so gradient buffers that overlap are an argument error,
    found on the host before any launch."""
    import ctypes

    need_gpu()
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(2, 3, 4, seed=4)
    bits = qi.random_bitstrings(6, 2, seed=6)
    plan = tn.plan_circuit(circ, bits, seed=2, mode=q.MODE_FP32)
    cp = tn.CompiledPlan(plan)
    hd = q.Handle(tol=0.0, size_rule=True)
    try:
        sizes = [t.numel() for t in cp.leaves]
        g_out = torch.zeros((plan.n_slots, plan.out_size), dtype=torch.complex128, device="cuda")
        buf = torch.zeros(sum(sizes), dtype=torch.complex64, device="cuda")
        ok = list(buf.split(sizes))
        bad = list(ok)
        bad[1] = buf[: sizes[1]]  # overlaps leaf 0's gradient
        info = q._lib.qcs_run_info_t()
        rc = hd.lib.qcs_contract_tree_backward(
            hd.ptr, ctypes.byref(cp.tree), cp._ptrs(cp.leaves), ctypes.c_void_p(g_out.data_ptr()),
            cp._ptrs(bad), ctypes.byref(info))
        assert rc == -1
        rc = hd.lib.qcs_contract_tree_backward(
            hd.ptr, ctypes.byref(cp.tree), cp._ptrs(cp.leaves), ctypes.c_void_p(g_out.data_ptr()),
            cp._ptrs(ok), ctypes.byref(info))
        assert rc == 0
        torch.cuda.synchronize()
        hd.sync()
    finally:
        hd.close()
