"""GPU parity of the contraction-tree executor and its adjoint (through the
C ABI) against the FP64 oracle: amplitudes of random grid circuits (closed,
sliced, batched bitstrings, open), and the gradient of sum log|a|^2 with
respect to the fSim parameters."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import lib, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def h():
    need_gpu()
    hd = lib().Handle(tol=0.0, size_rule=True)
    yield hd
    hd.close()


def _tn():
    import paper_2303_08989_gb300.tn as tn

    return tn


def _run(h, plan):
    tn = _tn()
    cp = tn.CompiledPlan(plan)
    out = cp.forward(h)
    torch.cuda.synchronize()
    h.sync()
    return out.cpu().numpy(), cp.last_info


def test_plain_method_small_grid_fp32(h):
    """3x4 grid, depth 8, 64 random bitstrings, greedy order; the size rule
    sends these small GEMMs to plain FP32 on the GPU."""
    tn = _tn()
    circ = qi.random_grid_circuit(3, 4, 8, seed=0)
    bits = qi.random_bitstrings(12, 64, seed=1)
    plan = tn.plan_circuit(circ, bits, seed=2)
    got, info = _run(h, plan)
    ref = oracle.sv_amplitudes(circ, bits)
    a = got[:, 0]
    assert oracle.fidelity(ref, a) >= 1 - 1e-5
    assert np.max(np.abs(a - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert info.gemm_count == 64 * len(plan.steps)
    assert info.mode_count[4] == info.gemm_count  # all plain FP32 under the size rule


def test_plain_method_small_grid_with_absorbed_gates(h):
    """The same 12-qubit workload with the single-qubit gates contracted into
    their neighbours on the host (a third of the steps), against the FP64
    state vector."""
    tn = _tn()
    circ = qi.random_grid_circuit(3, 4, 8, seed=0)
    bits = qi.random_bitstrings(12, 64, seed=1)
    plan = tn.plan_circuit(circ, bits, seed=2, absorb=True)
    assert len(plan.steps) < len(tn.plan_circuit(circ, bits, seed=2).steps) // 2
    got, _ = _run(h, plan)
    ref = oracle.sv_amplitudes(circ, bits)
    assert oracle.fidelity(ref, got[:, 0]) >= 1 - 1e-5
    assert np.max(np.abs(got[:, 0] - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("mode", ["fp16x", "tf32x", "fp16x_scaled", "auto"])
def test_emulated_modes_on_every_step(h, mode):
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(3, 4, 8, seed=0)
    bits = qi.random_bitstrings(12, 8, seed=1)
    plan = tn.plan_circuit(circ, bits, seed=2, mode=q.MODE_BY_NAME[mode])
    h.set_size_rule(False)
    try:
        got, info = _run(h, plan)
    finally:
        h.set_size_rule(True)
    ref = oracle.sv_amplitudes(circ, bits)
    assert oracle.fidelity(ref, got[:, 0]) >= 1 - 1e-5
    assert np.max(np.abs(got[:, 0] - ref)) <= 1e-5 * np.max(np.abs(ref))


def test_sliced_amplitudes(h):
    tn = _tn()
    circ = qi.random_grid_circuit(3, 4, 8, seed=3)
    bits = qi.random_bitstrings(12, 4, seed=4)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=3)
    assert plan.n_instances == 4 * 8
    got, _ = _run(h, plan)
    ref = oracle.sv_amplitudes(circ, bits)
    assert oracle.fidelity(ref, got[:, 0]) >= 1 - 1e-5
    # the oracle's own sliced contraction agrees
    net = tn.circuit_network(circ, bits[:1])
    assert abs(oracle.amplitude(circ, bits[0], sliced=plan.sliced) - ref[0]) < 1e-12


def test_open_network_state_vector(h):
    tn = _tn()
    circ = qi.random_grid_circuit(2, 3, 6, seed=5)
    plan = tn.plan_circuit(circ, None, seed=1, n_slices=1)
    got, _ = _run(h, plan)
    ref = oracle.statevector(circ).ravel()
    assert oracle.fidelity(ref, got[0]) >= 1 - 1e-5
    assert abs(np.sum(np.abs(got[0]) ** 2) - 1.0) < 1e-5


def _grad_check(h, mode, n_slices, size_rule):
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(2, 3, 4, seed=4, theta=None, phi=None, param_seed=5)
    bits = qi.random_bitstrings(6, 8, seed=6)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=n_slices, mode=q.MODE_BY_NAME[mode])
    params0 = np.array([g.params for g in circ.gates if g.name == "fsim"], dtype=np.float64)
    params = torch.tensor(params0, dtype=torch.float32, device="cuda", requires_grad=True)
    cp = tn.CompiledPlan(plan, leaf_data=[])
    h.set_size_rule(size_rule)
    try:
        leaves = tn.torch_leaves(plan.net, circ, params)
        amps = tn.contract(cp, h, leaves)
        loss = torch.log(amps.abs() ** 2).sum()
        loss.backward()
        torch.cuda.synchronize()
        h.sync()
    finally:
        h.set_size_rule(True)
    L_ref, g_ref = oracle.loss_and_grad(circ, bits)
    g = params.grad.double().cpu().numpy()
    assert abs(loss.item() - L_ref) < 1e-4 * abs(L_ref)
    rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    assert rel < 1e-4, rel
    return rel


@pytest.mark.parametrize("mode,n_slices,size_rule", [("auto", 0, True), ("fp32", 2, True),
                                                     ("tf32x", 1, False), ("fp16x", 0, False)])
def test_backward_matches_oracle_gradient(h, mode, n_slices, size_rule):
    _grad_check(h, mode, n_slices, size_rule)


def test_invalid_plan_is_rejected_before_launch(h):
    tn = _tn()
    from paper_2303_08989_gb300 import _lib as L

    circ = qi.random_grid_circuit(2, 2, 2, seed=1)
    plan = tn.plan_circuit(circ, qi.random_bitstrings(4, 2, seed=1))
    cp = tn.CompiledPlan(plan)
    cp._steps[0].map_a.strides[0] = 10 ** 6  # reads far outside the leaf
    out = torch.zeros((plan.n_slots, 1), dtype=torch.complex128, device="cuda")
    import ctypes

    rc = h.lib.qcs_contract_tree(h.ptr, ctypes.byref(cp.tree), cp._ptrs(cp.leaves),
                                 ctypes.c_void_p(out.data_ptr()), None)
    assert rc == L.QCS_ERR_INVALID_ARG
    cp2 = tn.CompiledPlan(plan)
    cp2._steps[1].a = len(plan.net.leaves) + 5  # refers to a later step
    rc = h.lib.qcs_contract_tree(h.ptr, ctypes.byref(cp2.tree), cp2._ptrs(cp2.leaves),
                                 ctypes.c_void_p(out.data_ptr()), None)
    assert rc == L.QCS_ERR_INVALID_ARG


def _golden_amplitudes(path):
    bits, amps = [], []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            b, re, im = line.split()
            bits.append([int(c) for c in b])
            amps.append(float(re) + 1j * float(im))
    return np.array(bits, dtype=np.uint8), np.array(amps)


def test_full_size_30_qubit_sliced_amplitudes_vs_fp64_golden(h, golden_dir):
    """The contraction workload at full size: 5x6 grid, depth 14, 6 sliced
    indices (64 slices), AUTO-0.1 per GEMM, against FP64 amplitudes the
    oracle's state vector wrote to tests/golden (the oracle cannot contract
    this network itself in reasonable time)."""
    import os

    tn = _tn()
    bits_all, ref_all = _golden_amplitudes(os.path.join(golden_dir, "grid5x6_d14_amplitudes.txt"))
    assert np.array_equal(bits_all, qi.random_bitstrings(30, 8, seed=1))
    circ = qi.random_grid_circuit(5, 6, 14, seed=0)
    bits, ref = bits_all[:2], ref_all[:2]
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=6)
    assert plan.n_instances == 2 * 64
    h.set_tol(0.1)
    try:
        got, info = _run(h, plan)
    finally:
        h.set_tol(0.0)
    a = got[:, 0]
    assert oracle.fidelity(ref, a) >= 1 - 1e-5
    assert np.all(np.abs(a - ref) <= 1e-4 * np.abs(ref)), (a, ref)
    assert info.mode_count[0] > 0  # some GEMMs took the statistics-based selection


@pytest.mark.parametrize("absorb", [False, True])
def test_full_size_30_qubit_in_the_bench_configuration_vs_fp64_golden(golden_dir, absorb):
    """The contraction in bench.py's configuration: the cheapest of many
    seeded greedy orders (256 here), 6 sliced indices, instances in groups
    of 16 (grouped tensor-core launches, also for the steps that fill the
    GPU alone; batched FP32 steps), AUTO-0.1 under the measured size rule with
    K ranges from the tuner; two bitstrings x 64 slices against the FP64
    amplitudes of tests/golden, eagerly, replayed from a CUDA graph, and with
    the GPU-filling steps one instance at a time (bit-identical)."""
    import os

    need_gpu()
    tn = _tn()
    q = lib()
    bits_all, ref_all = _golden_amplitudes(os.path.join(golden_dir, "grid5x6_d14_amplitudes.txt"))
    circ = qi.random_grid_circuit(5, 6, 14, seed=0)
    bits, ref = (bits_all[4:6], ref_all[4:6]) if absorb else (bits_all[2:4], ref_all[2:4])
    plan = tn.plan_circuit(circ, bits, seed=0, n_slices=6, mode=q.MODE_AUTO, trials=256,
                           absorb=absorb, workers=8)
    if absorb:  # the single-qubit gates are part of their neighbours' tensors
        assert len(plan.steps) < len(tn.circuit_network(circ, bits).leaves) // 2
    assert plan.n_instances == 2 * 64 and plan.max_log2_size <= 25
    hd = q.Handle(tol=0.1, size_rule=q.SIZE_RULE_TUNED)
    try:
        hd.set_instance_batch(16)
        cp = tn.CompiledPlan(plan)
        assert cp.autotune(hd, reps=2) > 0
        eager = cp.forward(hd)
        torch.cuda.synchronize()
        hd.sync()
        info = cp.last_info
        g, out = cp.graph(hd)
        out.zero_()
        g.launch()
        torch.cuda.synchronize()
        hd.sync()
        replay = out.cpu().numpy()
        g.close()
        # the steps that fill the GPU alone one instance at a time (group budget 0)
        hd.set_group_budget(0)
        per_instance = cp.forward(hd).cpu().numpy()
        hd.sync()
        info0 = cp.last_info
    finally:
        hd.close()
    a = eager.cpu().numpy()[:, 0]
    assert np.array_equal(replay[:, 0], a)
    assert np.array_equal(per_instance[:, 0], a)
    assert info0.workspace_bytes < info.workspace_bytes  # the default grouped those steps
    assert oracle.fidelity(ref, a) >= 1 - 1e-5
    assert np.all(np.abs(a - ref) <= 1e-4 * np.abs(ref)), (a, ref)
    assert info.mode_count[q.MODE_FP32] > 0 and info.mode_count[q.MODE_FP32] < info.gemm_count


@pytest.mark.parametrize("mode,n_slices", [("auto", 0), ("tf32x", 2)])
def test_graph_replay_equals_eager(h, mode, n_slices):
    """qcs_tree_graph_*: the captured launch sequence replays to the same bits as
    the eager call, also after the leaf buffers were overwritten in place."""
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(3, 4, 8, seed=0)
    bits = qi.random_bitstrings(12, 16, seed=1)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=n_slices, mode=q.MODE_BY_NAME[mode])
    h.set_size_rule(False)
    try:
        cp = tn.CompiledPlan(plan)
        eager = cp.forward(h).clone()
        g, out = cp.graph(h)
        g.launch()
        torch.cuda.synchronize()
        h.sync()
        assert torch.equal(out, eager)
        # new gate values in the same buffers: the replay reads the current contents
        circ2 = qi.random_grid_circuit(3, 4, 8, seed=7)
        for t, lf in zip(cp.leaves, tn.circuit_network(circ2, bits).leaves):
            t.copy_(torch.from_numpy(lf.data))
        g.launch()
        eager2 = cp.forward(h)
        torch.cuda.synchronize()
        assert torch.equal(out, eager2)
        ref = oracle.sv_amplitudes(circ2, bits)
        assert oracle.fidelity(ref, out.cpu().numpy()[:, 0]) >= 1 - 1e-5
        g.close()
    finally:
        h.set_size_rule(True)


def _golden_slices(path):
    labels, rows = None, []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            if line.startswith("sliced"):
                labels = [int(v) for v in line.split()[1:]]
                continue
            v, re, im = line.split()
            rows.append((v, float(re) + 1j * float(im)))
    return labels, rows


def sampled_slice_plan(tn, circ, bits, labels, values, seed=5):
    """The plan restricted to the given slice assignments, one output slot each."""
    import copy

    net = tn.circuit_network(circ, bits)
    order = tn.greedy_order(net, seed=seed, skip=[tn.BATCH] + labels)
    plan = tn.build_plan(net, order, labels)
    idx = [int(v, 2) for v in values]  # the first sliced index varies slowest
    sub = copy.copy(plan)
    sub.instance_offset = np.ascontiguousarray(plan.instance_offset[idx])
    sub.instance_slot = np.arange(len(idx), dtype=np.int32)
    sub.n_slots = len(idx)
    return plan, sub


def test_40_qubit_sampled_slices_vs_fp64_golden(h, golden_dir):
    """Precision at scale: a 40-qubit 5x8 grid circuit (depth 12), sliced on
    8 indices (256 slices); four sampled slices, contracted with AUTO-0.1 per
    GEMM, against the oracle's FP64 contraction of the same slices."""
    import os

    path = os.path.join(golden_dir, "slices5x8_d12.txt")
    if not os.path.exists(path):
        pytest.skip("golden file not written")
    tn = _tn()
    labels, rows = _golden_slices(path)
    circ = qi.random_grid_circuit(5, 8, 12, seed=0)
    bits = qi.random_bitstrings(40, 1, seed=1)
    plan, sub = sampled_slice_plan(tn, circ, bits, labels, [v for v, _ in rows])
    assert plan.n_instances == 256 and plan.max_log2_size <= 30
    h.set_tol(0.1)
    try:
        got, info = _run(h, sub)
    finally:
        h.set_tol(0.0)
    ref = np.array([a for _, a in rows])
    a = got[:, 0]
    assert oracle.fidelity(ref, a) >= 1 - 1e-5
    assert np.all(np.abs(a - ref) <= 1e-4 * np.abs(ref)), (a, ref)


@pytest.mark.parametrize("G", [2, 5, 32])
def test_instance_groups_are_bit_identical(G):
    """qcs_set_instance_batch: plain-FP32 steps run as one batched launch per
    group of G instances (slices x bitstrings), the emulated steps loop over
    the group; every GEMM computes exactly what it computes alone, so the
    result equals the one-instance-at-a-time result bit for bit, eagerly and
    replayed from a CUDA graph, and matches the FP64 oracle."""
    need_gpu()
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(3, 4, 8, seed=3)
    bits = qi.random_bitstrings(12, 4, seed=4)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=3)
    # every third step emulated on the tensor cores, the rest plain FP32
    for i, st in enumerate(plan.steps):
        st.mode = q.MODE_FP16X if i % 3 == 2 else q.MODE_FP32
    hd = q.Handle(tol=0.0, size_rule=False)
    try:
        one, _ = _run(hd, plan)
        hd.set_instance_batch(G)
        cp = tn.CompiledPlan(plan)
        grouped = cp.forward(hd)
        torch.cuda.synchronize()
        hd.sync()
        info = cp.last_info
        assert info.gemm_count == plan.n_instances * len(plan.steps)
        g, out = cp.graph(hd)
        out.zero_()
        g.launch()
        torch.cuda.synchronize()
        hd.sync()
        replay = out.cpu().numpy()
        g.close()
    finally:
        hd.close()
    assert np.array_equal(grouped.cpu().numpy(), one)
    assert np.array_equal(replay, one)
    ref = oracle.sv_amplitudes(circ, bits)
    assert oracle.fidelity(ref, one[:, 0]) >= 1 - 1e-5


def test_instance_groups_with_direct_and_split_k_steps():
    """Groups over a network whose last step reduces a long k into one output
    (the split-K FP32 path, one partial buffer per instance) and whose steps
    read leaves directly: bit-identical to one instance at a time."""
    need_gpu()
    tn = _tn()
    q = lib()
    circ = qi.random_grid_circuit(4, 4, 10, seed=8)
    bits = qi.random_bitstrings(16, 6, seed=9)
    plan = tn.plan_circuit(circ, bits, seed=4, n_slices=2, mode=q.MODE_FP32)
    assert any(s.m * s.n <= 4096 and s.k >= 1024 for s in plan.steps)
    assert any(st.direct_a != -1 or st.direct_b != -1 for st in plan.steps)
    hd = q.Handle(tol=0.0, size_rule=False)
    try:
        one, _ = _run(hd, plan)
        for G in (3, 24):
            hd.set_instance_batch(G)
            got, _ = _run(hd, plan)
            assert np.array_equal(got, one), G
    finally:
        hd.close()
    ref = oracle.sv_amplitudes(circ, bits)
    assert oracle.fidelity(ref, one[:, 0]) >= 1 - 1e-5


@pytest.mark.parametrize("mode", ["fp16x", "tf32x", "auto", "bf16x3", "fp16x_scaled"])
def test_split_through_the_map_equals_gather_then_split(mode):
    """An emulated step whose operand is a permuted intermediate is split
    straight from the intermediate through its gather map (no gather pass;
    statistics read the intermediate as stored).  The result must equal, bit
    for bit, gathering the operand first and running qcs_cgemm on it."""
    need_gpu()
    tn = _tn()
    q = lib()
    rng = np.random.default_rng(11)

    def leaf(labels, dims):
        x = (rng.standard_normal(int(np.prod(dims))) + 1j * rng.standard_normal(int(np.prod(dims))))
        return tn.Leaf(x.astype(np.complex64), list(labels), list(dims))

    I, J, P, Q, R = 0, 1, 2, 3, 4
    d = {I: 128, J: 8, P: 16, Q: 32, R: 256}
    L0 = leaf([J, I, P], [d[J], d[I], d[P]])
    L1 = leaf([P, Q], [d[P], d[Q]])
    L2 = leaf([J, Q, R], [d[J], d[Q], d[R]])
    net = tn.Network([L0, L1, L2], [I, R], d)
    plan = tn.build_plan(net, [(0, 1), (3, 2)], mode=q.MODE_FP32)
    s1 = plan.steps[1]
    assert s1.direct_a == -1 and (s1.m, s1.n, s1.k) == (128, 256, 256)
    s1.mode = q.MODE_BY_NAME[mode]
    hd = q.Handle(tol=0.0, size_rule=False)
    try:
        cp = tn.CompiledPlan(plan)
        got = cp.forward(hd)
        torch.cuda.synchronize()
        hd.sync()
        got = got.cpu().numpy()[0]
        # the same two GEMMs by hand: step 0 in FP32, gather with torch, qcs_cgemm
        s0 = plan.steps[0]
        A0 = torch.as_strided(torch.from_numpy(L0.data).cuda(), tuple(s0.map_a[0][::-1]),
                              tuple(s0.map_a[1][::-1])).reshape(s0.k, s0.m).t()
        B0 = torch.as_strided(torch.from_numpy(L1.data).cuda(), tuple(s0.map_b[0][::-1]),
                              tuple(s0.map_b[1][::-1])).reshape(s0.n, s0.k).t()
        T = q.cgemm(hd, q.to_fortran(A0), q.to_fortran(B0), mode="fp32")
        Tflat = T.t().reshape(-1)  # column-major storage of the intermediate
        A1 = torch.as_strided(Tflat, tuple(s1.map_a[0][::-1]), tuple(s1.map_a[1][::-1]))
        A1 = q.to_fortran(A1.reshape(s1.k, s1.m).t())
        B1 = torch.as_strided(torch.from_numpy(L2.data).cuda(), tuple(s1.map_b[0][::-1]),
                              tuple(s1.map_b[1][::-1])).reshape(s1.n, s1.k).t()
        C1 = q.cgemm(hd, A1, q.to_fortran(B1), mode=mode)
        torch.cuda.synchronize()
        want = C1.cpu().numpy().astype(np.complex128)  # [i, r]
    finally:
        hd.close()
    # the open result is ordered like numpy C order over the output labels (I, R)
    assert np.array_equal(got.reshape(d[I], d[R]), want)


@pytest.mark.parametrize("splits", [1, 3])
def test_grouped_emulated_step_with_a_mode_per_instance(splits):
    """One emulated step over a group of 4 instances whose operands select
    four different modes (FP16X, TF32X, FP16X_SCALED and, for an operand with
    a NaN, FP32): the grouped tensor-core launches run only the units of the
    instances that selected their kind, with each instance's scales, the
    FP32 candidates and the split-K reduction are gated per instance, and
    every instance equals, bit for bit, its result when run alone."""
    need_gpu()
    tn = _tn()
    q = lib()
    B_, I, K, J = tn.BATCH, 0, 1, 2
    d = {B_: 4, I: 256, K: 192, J: 160}
    rng = np.random.default_rng(31)

    def normal(shape):
        return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)

    a = normal((4, d[I], d[K]))  # [b, i, k]
    a[1] *= 2.0 ** rng.integers(-40, 41, size=(d[I], d[K]))
    a[2] *= 2.0 ** -30
    a[3, 5, 7] = complex(np.nan, 0)
    b = normal((d[K], d[J]))
    # leaves store their labels first-index-fastest
    L0 = tn.Leaf(np.ascontiguousarray(a.transpose(2, 1, 0).ravel()).astype(np.complex64),
                 [B_, I, K], [d[B_], d[I], d[K]])
    L1 = tn.Leaf(np.ascontiguousarray(b.T.ravel()).astype(np.complex64), [K, J], [d[K], d[J]])
    net = tn.Network([L0, L1], [I, J], d, batch=4)
    plan = tn.build_plan(net, [(0, 1)], mode=q.MODE_AUTO)
    assert plan.n_instances == 4 and plan.steps[0].direct_a == -1
    hd = q.Handle(tol=1e-3, size_rule=False)
    try:
        hd.set_tc_splits(splits)
        hd.auto_counts()
        one, _ = _run(hd, plan)
        assert hd.auto_counts() == {"auto": 0, "fp16x": 1, "fp16x_scaled": 1, "tf32x": 1,
                                    "fp32": 1, "bf16x3": 0}
        hd.set_instance_batch(4)
        grouped, info = _run(hd, plan)
        assert info.gemm_count == 4
    finally:
        hd.close()
    np.testing.assert_array_equal(grouped, one)  # NaN where NaN
    a64 = a.astype(np.complex64).astype(np.complex128)
    b64 = b.astype(np.complex64).astype(np.complex128)
    for inst in range(4):
        got = one[inst].reshape(d[I], d[J])
        if inst == 3:
            assert np.isnan(got[5]).all() and np.isfinite(np.delete(got, 5, axis=0)).all()
            got, want = np.delete(got, 5, axis=0), np.delete(a64[3], 5, axis=0) @ b64
        else:
            want = a64[inst] @ b64
        assert oracle.rel_fro_error(got, want) < (1e-5 if inst == 3 else 2e-6), inst
