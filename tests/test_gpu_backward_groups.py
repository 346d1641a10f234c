"""The adjoint in groups of instances (qcs_set_instance_batch applies to
qcs_contract_tree_backward too): every step's adjoint GEMMs, gathers and
scatters for the whole group in one launch each, the small steps' adjoints
of a level in one launch, each instance's leaf gradients in its own buffer,
added into the caller's in instance order.  The gradient equals the
one-instance-at-a-time gradient bit for bit and matches the FP64 adjoint."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import lib, need_gpu, torch

pytestmark = pytest.mark.gpu


def _tn():
    import paper_2303_08989_gb300.tn as tn

    return tn


def _grad(hd, tn, plan, circ, params0):
    params = torch.tensor(params0, dtype=torch.float32, device="cuda", requires_grad=True)
    cp = tn.CompiledPlan(plan, leaf_data=[])
    leaves = tn.torch_leaves(plan.net, circ, params)
    amps = tn.contract(cp, hd, leaves)
    loss = torch.log(amps.abs() ** 2).sum()
    loss.backward()
    torch.cuda.synchronize()
    hd.sync()
    return loss.item(), params.grad.double().cpu().numpy(), cp.last_info


@pytest.mark.parametrize("mode,size_rule,n_slices,G", [
    ("fp32", True, 2, 3),        # 8 bitstrings x 4 slices: groups of 3, a ragged last group
    ("fp32", True, 0, 8),
    ("auto", True, 1, 16),
    ("tf32x", False, 2, 5),      # every adjoint GEMM emulated: grouped tensor-core launches
    ("fp16x", False, 1, 4),
])
def test_grouped_adjoint_is_bit_identical(mode, size_rule, n_slices, G):
    need_gpu()
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(2, 3, 4, seed=4, theta=None, phi=None, param_seed=5)
    bits = qi.random_bitstrings(6, 8, seed=6)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=n_slices, mode=q.MODE_BY_NAME[mode])
    p0 = np.array([g.params for g in circ.gates if g.name == "fsim"], dtype=np.float64)
    hd = q.Handle(tol=0.0, size_rule=size_rule)
    try:
        l1, g1, _ = _grad(hd, tn, plan, circ, p0)
        hd.set_instance_batch(G)
        lg, gg, info = _grad(hd, tn, plan, circ, p0)
    finally:
        hd.close()
    assert lg == l1
    assert np.array_equal(gg, g1)
    assert info.gemm_count >= 2 * plan.n_instances * len(plan.steps)
    L_ref, g_ref = oracle.loss_and_grad(circ, bits)
    assert np.linalg.norm(gg - g_ref) / np.linalg.norm(g_ref) < 1e-4


def test_grouped_adjoint_with_sliced_leaves_and_levels_off():
    """Sliced leaves (each instance writes its own part of a leaf's
    gradient) with level launches off: the grouped gathers and scatters of
    every step, bit-identical to one instance at a time."""
    need_gpu()
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(3, 3, 6, seed=7, theta=None, phi=None, param_seed=8)
    bits = qi.random_bitstrings(9, 3, seed=9)
    plan = tn.plan_circuit(circ, bits, seed=3, n_slices=3, mode=q.MODE_FP32)
    p0 = np.array([g.params for g in circ.gates if g.name == "fsim"], dtype=np.float64)
    hd = q.Handle(tol=0.0, size_rule=True)
    try:
        hd.set_tree_levels(False)
        l1, g1, _ = _grad(hd, tn, plan, circ, p0)
        hd.set_instance_batch(6)
        lg, gg, info = _grad(hd, tn, plan, circ, p0)
    finally:
        hd.close()
    assert info.level_launches == 0
    assert lg == l1
    assert np.array_equal(gg, g1)
    L_ref, g_ref = oracle.loss_and_grad(circ, bits)
    assert np.linalg.norm(gg - g_ref) / np.linalg.norm(g_ref) < 1e-4


def test_a_lone_leaf_forward_and_backward_in_groups():
    """A plan without steps (the root is the leaf itself, read at each
    instance's offset): the forward copies, the backward seeds the leaf's
    gradient at each instance's offset; a group size above 1 falls back to
    one instance at a time and gives the same result."""
    import ctypes

    need_gpu()
    q = lib()
    L = q._lib
    n_inst, out_size = 3, 4
    leaf = torch.arange(12, dtype=torch.float32, device="cuda").to(torch.complex64) * (1 + 2j)
    t = L.qcs_tree_t()
    sizes = (ctypes.c_int64 * 1)(12)
    offs = (ctypes.c_int64 * 3)(0, 4, 8)
    slots = (ctypes.c_int32 * 3)(0, 1, 2)
    t.n_leaves, t.n_steps, t.n_instances, t.n_slots = 1, 0, n_inst, n_inst
    t.leaf_size, t.instance_offset, t.instance_slot = sizes, offs, slots
    t.steps, t.out_size, t.out_index = None, out_size, None
    leaves = (ctypes.c_void_p * 1)(leaf.data_ptr())
    g_out = torch.zeros((n_inst, out_size), dtype=torch.complex128, device="cuda")
    g_out += torch.arange(n_inst * out_size, dtype=torch.float64, device="cuda").reshape(
        n_inst, out_size).to(torch.complex128) * (0.5 - 1j)
    grads = []
    for G in (1, 3):
        hd = q.Handle()
        try:
            hd.set_instance_batch(G)
            out = torch.zeros((n_inst, out_size), dtype=torch.complex128, device="cuda")
            info = L.qcs_run_info_t()
            assert hd.lib.qcs_contract_tree(hd.ptr, ctypes.byref(t), leaves,
                                            ctypes.c_void_p(out.data_ptr()), ctypes.byref(info)) == 0
            gl = torch.zeros(12, dtype=torch.complex64, device="cuda")
            gp = (ctypes.c_void_p * 1)(gl.data_ptr())
            assert hd.lib.qcs_contract_tree_backward(hd.ptr, ctypes.byref(t), leaves,
                                                     ctypes.c_void_p(g_out.data_ptr()), gp,
                                                     ctypes.byref(info)) == 0
            torch.cuda.synchronize()
            hd.sync()
            assert torch.equal(out.cpu(), leaf.cpu().to(torch.complex128).reshape(n_inst, out_size))
            grads.append(gl.cpu())
        finally:
            hd.close()
    assert torch.equal(grads[0], grads[1])
    assert torch.equal(grads[0], g_out.reshape(-1).cpu().to(torch.complex64))
