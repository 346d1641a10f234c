"""Host logic of the contraction planner (no GPU): the plan, interpreted
with numpy, must give the oracle's amplitudes, for closed and open networks,
with slicing and bitstring batches; the maps must be bijections."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from plan_sim import gather_index, run

tn = pytest.importorskip("paper_2303_08989_gb300.tn")


def _leaves(plan):
    return [lf.data for lf in plan.net.leaves]


def test_closed_amplitudes_batched_bitstrings():
    circ = qi.random_grid_circuit(3, 4, 8, seed=0)
    bits = qi.random_bitstrings(12, 16, seed=1)
    plan = tn.plan_circuit(circ, bits, seed=2)
    got = run(plan, _leaves(plan))[:, 0]
    ref = oracle.sv_amplitudes(circ, bits)
    np.testing.assert_allclose(got, ref, atol=1e-6)  # complex64 leaves, FP64 arithmetic
    assert plan.n_instances == 16 and plan.n_slots == 16


def test_sliced_plan_sums_to_the_amplitude():
    circ = qi.random_grid_circuit(3, 3, 6, seed=4)
    bits = qi.random_bitstrings(9, 3, seed=5)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=3)
    assert len(plan.sliced) == 3 and plan.n_instances == 3 * 8
    got = run(plan, _leaves(plan))[:, 0]
    np.testing.assert_allclose(got, oracle.sv_amplitudes(circ, bits), atol=1e-6)


def test_open_network_gives_the_state_vector():
    circ = qi.random_grid_circuit(2, 3, 5, seed=6)
    plan = tn.plan_circuit(circ, None, seed=3)
    got = run(plan, _leaves(plan))[0]
    np.testing.assert_allclose(got, oracle.statevector(circ).ravel(), atol=1e-6)
    # bitstring gather from the open result
    bits = qi.random_bitstrings(6, 5, seed=7)
    net = tn.circuit_network(circ, None)
    order = tn.greedy_order(net, seed=3)
    p2 = tn.build_plan(net, order, outputs=bits)
    np.testing.assert_allclose(run(p2, _leaves(p2))[0], oracle.sv_amplitudes(circ, bits), atol=1e-6)


def test_open_network_sliced():
    circ = qi.random_grid_circuit(2, 3, 6, seed=8)
    net = tn.circuit_network(circ, None)
    order = tn.greedy_order(net, seed=1)
    sliced = tn.choose_slices(net, order, n_labels=2)
    plan = tn.build_plan(net, order, sliced)
    np.testing.assert_allclose(run(plan, _leaves(plan))[0], oracle.statevector(circ).ravel(),
                               atol=1e-6)


def test_maps_are_bijections_and_within_bounds():
    circ = qi.random_grid_circuit(3, 4, 8, seed=0)
    plan = tn.plan_circuit(circ, qi.random_bitstrings(12, 4, seed=1), n_slices=2)
    sizes = [lf.data.size for lf in plan.net.leaves]
    for st in plan.steps:
        sizes.append(st.m * st.n)
    for st in plan.steps:
        for mp, src, elems in ((st.map_a, st.a, st.m * st.k), (st.map_b, st.b, st.k * st.n)):
            idx = gather_index(*mp)
            assert idx.size == elems and len(np.unique(idx)) == elems
            base = plan.instance_offset[:, src].max() if src < len(plan.net.leaves) else 0
            assert base + idx.max() < sizes[src]


def test_greedy_order_is_seeded_and_contracts_everything():
    circ = qi.random_grid_circuit(4, 5, 12, seed=3)
    net = tn.circuit_network(circ, None)
    o1 = tn.greedy_order(net, seed=2)
    o2 = tn.greedy_order(net, seed=2)
    assert o1 == o2
    assert len(o1) == len(net.leaves) - 1
    inter = tn.intermediates(net, o1)
    assert sorted(inter[-1]) == sorted(net.output)


def test_slicer_bounds_the_largest_intermediate():
    circ = qi.random_grid_circuit(4, 5, 12, seed=3)
    net = tn.circuit_network(circ, None)
    order = tn.greedy_order(net, seed=2)
    base = max(len(r) for r in tn.intermediates(net, order))
    sliced = tn.choose_slices(net, order, max_log2_size=base - 3)
    after = max(len(r) for r in tn.intermediates(net, order, sliced))
    assert after <= base - 3 and len(sliced) >= 3


def test_open_network_sliced_with_bitstring_gather():
    # the differentiation workload's plan shape: open legs, sliced, amplitudes gathered
    circ = qi.random_grid_circuit(3, 3, 6, seed=2, theta=None, phi=None, param_seed=3)
    bits = qi.random_bitstrings(9, 12, seed=1)
    net = tn.circuit_network(circ, None)
    order = tn.greedy_order(net, seed=2)
    sliced = tn.choose_slices(net, order, n_labels=2)
    plan = tn.build_plan(net, order, sliced, outputs=bits)
    assert plan.n_instances == 4 and plan.n_slots == 1 and plan.out_size == 12
    got = run(plan, _leaves(plan))[0]
    np.testing.assert_allclose(got, oracle.sv_amplitudes(circ, bits), atol=1e-6)


def test_best_greedy_order_is_the_cheapest_seed():
    """best_greedy_order returns the order (and slicing) with the fewest
    flops per instance among its seeds; order_cost agrees with the plan's
    own count; the chosen plan still contracts to the oracle's amplitudes."""
    circ = qi.random_grid_circuit(3, 4, 8, seed=0)
    bits = qi.random_bitstrings(12, 2, seed=1)
    net = tn.circuit_network(circ, bits)
    skip = [tn.BATCH]
    costs = {}
    for seed in range(8):
        order = tn.greedy_order(net, seed=seed, skip=skip)
        sliced = tn.choose_slices(net, order, n_labels=2, skip=skip)
        flops, big = tn.order_cost(net, order, skip + sliced)
        plan = tn.build_plan(net, order, sliced)
        assert flops == pytest.approx(plan.flops) and big == plan.max_log2_size
        costs[seed] = (flops, big, seed)
    order, sliced, seed = tn.best_greedy_order(net, range(8), skip=skip, n_slices=2)
    assert costs[seed] == min(costs.values())
    plan = tn.plan_circuit(circ, bits, seed=0, n_slices=2, trials=8)
    assert plan.flops == pytest.approx(costs[seed][0])
    got = run(plan, _leaves(plan))[:, 0]
    np.testing.assert_allclose(got, oracle.sv_amplitudes(circ, bits), atol=1e-6)


def test_best_greedy_order_in_worker_processes_matches_serial():
    """Costing the seeds in spawned worker processes picks the same order,
    slicing and seed as the serial search."""
    circ = qi.random_grid_circuit(4, 4, 10, seed=3)
    bits = qi.random_bitstrings(16, 1, seed=4)
    net = tn.circuit_network(circ, bits)
    skip = [tn.BATCH]
    serial = tn.best_greedy_order(net, range(5, 29), skip=skip, n_slices=3)
    parallel = tn.best_greedy_order(net, range(5, 29), skip=skip, n_slices=3, workers=3)
    assert serial == parallel


def test_absorbing_single_qubit_gates_keeps_the_amplitudes():
    """Single-qubit gates contracted into their neighbours on the host: a
    third of the leaves remain, and the plan interpreter's amplitudes equal
    those of the full network and the oracle's state vector (up to the
    complex64 rounding of the merged tensors)."""
    import oracle

    circ = qi.random_grid_circuit(3, 3, 8, seed=4)
    bits = qi.random_bitstrings(9, 6, seed=5)
    net = tn.circuit_network(circ, bits)
    small = tn.absorb_single_qubit_gates(net)
    n1 = sum(1 for g in circ.gates if len(g.qubits) == 1)
    assert len(small.leaves) == len(net.leaves) - n1
    assert not [lf for lf in small.leaves if lf.kind == "gate" and len(lf.labels) == 2]
    ref = oracle.sv_amplitudes(circ, bits)
    for nw in (net, small):
        order = tn.greedy_order(nw, seed=1, skip=[tn.BATCH])
        plan = tn.build_plan(nw, order, tn.choose_slices(nw, order, n_labels=2, skip=[tn.BATCH]))
        got = run(plan, [lf.data for lf in plan.net.leaves])[:, 0]
        np.testing.assert_allclose(got, ref, atol=2e-6)


def test_absorption_respects_frozen_gates_and_kept_labels():
    circ = qi.random_grid_circuit(2, 3, 6, seed=4, theta=None, phi=None, param_seed=5)
    net = tn.circuit_network(circ, None)
    fs = set(circ.fsim_indices())
    small = tn.absorb_single_qubit_gates(net, frozen_gates=fs)
    before = {lf.gate: lf for lf in net.leaves if lf.kind == "gate" and lf.gate in fs}
    after = {lf.gate: lf for lf in small.leaves if lf.kind == "gate" and lf.gate in fs}
    assert before.keys() == after.keys()
    for g, lf in after.items():  # parametric leaves untouched
        assert lf.labels == before[g].labels and np.array_equal(lf.data, before[g].data)
    assert len(small.leaves) < len(net.leaves)
    # the same network, frozen or not, gives the same state
    import oracle

    ref = oracle.statevector(circ).ravel()
    order = tn.greedy_order(small, seed=1)
    plan = tn.build_plan(small, order, [])
    got = run(plan, [lf.data for lf in plan.net.leaves])[0]
    np.testing.assert_allclose(got, ref, atol=2e-6)
    # kept labels survive
    lab = [lf.labels[1] for lf in net.leaves if lf.kind == "gate" and len(lf.labels) == 2][:3]
    kept = tn.absorb_single_qubit_gates(net, keep_labels=lab)
    present = {l for lf in kept.leaves for l in lf.labels}
    assert set(lab) <= present


def test_torch_leaves_keep_constant_copies_and_follow_params():
    """The leaf tensors of a differentiated network (CPU tensors here): fSim
    leaves are the gate's matrix at the given parameters in first-index-
    fastest order; the constant leaves are copied once and reused, and a new
    leaf list is copied again."""
    torch = pytest.importorskip("torch")
    circ = qi.random_grid_circuit(2, 2, 4, seed=0, theta=None, phi=None, param_seed=3)
    net = tn.circuit_network(circ, None)
    p0 = np.array([g.params for g in circ.gates if g.name == "fsim"])
    params = torch.tensor(p0, dtype=torch.float64)
    first = tn.torch_leaves(net, circ, params, device="cpu")
    second = tn.torch_leaves(net, circ, params * 0.5, device="cpu")
    fs = {g: i for i, g in enumerate(circ.fsim_indices())}
    for i, lf in enumerate(net.leaves):
        if lf.kind == "gate" and lf.gate in fs:
            th, ph = (p0[fs[lf.gate]] * 0.5)
            want = qi.fsim(th, ph).reshape(2, 2, 2, 2).transpose(3, 2, 1, 0).ravel()
            np.testing.assert_allclose(second[i].numpy(), want, atol=1e-6)
        else:
            assert second[i] is first[i]
            assert np.array_equal(second[i].numpy(), lf.data)
    net.leaves = list(net.leaves)
    third = tn.torch_leaves(net, circ, params, device="cpu")
    assert all(third[i] is not first[i] for i, lf in enumerate(net.leaves)
               if not (lf.kind == "gate" and lf.gate in fs))
