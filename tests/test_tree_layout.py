"""Host logic of the contraction-tree executor, on the CPU: the schedule
(level by level, or plan order) and the workspace layout that
qcs_tree_layout_info reports for real plans.  Every step is issued once,
after the steps that produce its operands; steps that may run at the same
time (equal times) or whose outputs are live at once never share memory;
the level launches hold exactly the small plain-FP32 steps."""
import ctypes

import numpy as np
import pytest

import qcs_inputs as qi


def _mods():
    import paper_2303_08989_gb300._lib as L
    import paper_2303_08989_gb300.tn as tn

    return L, tn


def _layout(tree, backward=0, G=1, levels=1, sms=152, budget=32 << 30):
    L, _ = _mods()
    lib = L.load()
    ns = tree.n_steps
    off, by = (ctypes.c_int64 * ns)(), (ctypes.c_int64 * ns)()
    tm, sm, order = (ctypes.c_int32 * ns)(), (ctypes.c_int32 * ns)(), (ctypes.c_int32 * ns)()
    out = L.qcs_tree_layout_t()
    rc = lib.qcs_tree_layout_info(ctypes.byref(tree), backward, G, levels, sms, budget, off, by,
                                  tm, sm, order, ctypes.byref(out))
    assert rc == 0
    return (np.array(off[:]), np.array(by[:]), np.array(tm[:]), np.array(sm[:]),
            np.array(order[:]), out)


def _plans():
    _, tn = _mods()
    res = []
    c = qi.random_grid_circuit(3, 4, 8, seed=0)
    res.append(("12q, 64 bitstrings", tn.plan_circuit(c, qi.random_bitstrings(12, 64, seed=1),
                                                      seed=2)))
    c = qi.random_grid_circuit(4, 4, 10, seed=8)
    res.append(("16q sliced", tn.plan_circuit(c, qi.random_bitstrings(16, 6, seed=9), seed=4,
                                              n_slices=2)))
    c = qi.random_grid_circuit(5, 6, 14, seed=0)
    net = tn.absorb_single_qubit_gates(tn.circuit_network(c, qi.random_bitstrings(30, 1, seed=1)))
    _, order, sliced, _ = tn.cheapest_network_order([net], [844], skip=[tn.BATCH], n_slices=6)
    res.append(("30q absorbed", tn.build_plan(net, order, sliced, mode=0)))
    return res


PLANS = None


def plans():
    global PLANS
    if PLANS is None:
        PLANS = _plans()
    return PLANS


def _check(plan, tree, G, levels):
    nl = tree.n_leaves
    ns = tree.n_steps
    off, by, tm, sm, order, out = _layout(tree, G=G, levels=levels)
    steps = plan.steps
    # a permutation, each step after its producers
    assert sorted(order.tolist()) == list(range(ns))
    pos = np.empty(ns, dtype=int)
    pos[order] = np.arange(ns)
    P = out.batched_steps
    for s, st in enumerate(steps):
        for o in (st.a, st.b):
            if o >= nl:
                assert pos[o - nl] < pos[s]
                assert tm[o - nl] < tm[s]
    # liveness: [time, last reader's time] (the root and batched outputs read
    # by per-instance steps: to the end); overlapping intervals, disjoint bytes
    INF = 1 << 40
    last = np.full(ns, -1, dtype=np.int64)
    last[ns - 1] = INF
    for s, st in enumerate(steps):
        for o in (st.a, st.b):
            if o >= nl:
                p = o - nl
                last[p] = max(last[p], INF if (s >= P and p < P) else tm[s])
    for i in range(ns):
        for j in range(i + 1, ns):
            if tm[i] <= last[j] and tm[j] <= last[i]:
                assert off[i] + by[i] <= off[j] or off[j] + by[j] <= off[i], (i, j)
    # the small steps and the level launches
    if levels:
        for s, st in enumerate(steps):
            if sm[s]:
                assert st.m * st.k <= 1024 and st.k * st.n <= 1024 and st.m * st.n <= 4096
        lv = {}
        for s in range(ns):
            if sm[s]:
                lv.setdefault((s >= P, tm[s]), []).append(s)
        assert out.level_launches == len(lv)
        # a launch's steps are issued together
        for grp in lv.values():
            p = sorted(pos[grp])
            assert p[-1] - p[0] == len(p) - 1
    else:
        assert order.tolist() == list(range(ns))
        assert tm.tolist() == list(range(ns))
        assert not sm.any() and out.level_launches == 0
    assert out.group == min(G, tree.n_instances)
    assert out.total_bytes >= max(off + by)
    return out


@pytest.mark.parametrize("G", [1, 16])
@pytest.mark.parametrize("levels", [1, 0])
def test_schedule_and_liveness(G, levels):
    _, tn = _mods()
    for name, plan in plans():
        cp = tn.CompiledPlan(plan, device="cpu", leaf_data=[])
        out = _check(plan, cp.tree, G, levels)
        if levels:
            assert out.level_launches > 0, name


def test_backward_layout_keeps_every_output_and_groups():
    _, tn = _mods()
    name, plan = plans()[1]
    cp = tn.CompiledPlan(plan, device="cpu", leaf_data=[])
    for G in (1, 4):
        off, by, tm, sm, order, out = _layout(cp.tree, backward=1, G=G)
        assert out.group == min(G, plan.n_instances)
        idx = np.argsort(off)
        assert np.all(off[idx][1:] >= off[idx][:-1] + by[idx][:-1])  # no sharing at all
        if G > 1:
            assert out.batched_steps == len(plan.steps)  # every step once per group


def test_group_budget_moves_the_per_instance_boundary():
    """With a zero group budget the steps that fill the GPU alone (and every
    later one) run per instance; with the default they stay in the group."""
    _, tn = _mods()
    name, plan = plans()[2]
    for st in plan.steps:
        st.mode = 1 if st.m * st.n >= 152 * 128 * 128 else st.mode  # emulated where it fills
    cp = tn.CompiledPlan(plan, device="cpu", leaf_data=[])
    *_, out_def = _layout(cp.tree, G=16)
    *_, out_zero = _layout(cp.tree, G=16, budget=0)
    assert out_def.batched_steps == len(plan.steps)
    assert out_zero.batched_steps < len(plan.steps)
    assert out_zero.total_bytes < out_def.total_bytes


def test_invalid_plan_rejected():
    L, tn = _mods()
    name, plan = plans()[0]
    cp = tn.CompiledPlan(plan, device="cpu", leaf_data=[])
    lib = L.load()
    out = L.qcs_tree_layout_t()
    assert lib.qcs_tree_layout_info(ctypes.byref(cp.tree), 0, 0, 1, 152, 0, None, None, None,
                                    None, None, ctypes.byref(out)) == -1
    assert lib.qcs_tree_layout_info(ctypes.byref(cp.tree), 0, 1, 2, 152, 0, None, None, None,
                                    None, None, ctypes.byref(out)) == -1
    cp.tree.steps[0].a = cp.tree.steps[0].b  # a step reading the same tensor twice
    assert lib.qcs_tree_layout_info(ctypes.byref(cp.tree), 0, 1, 1, 152, 0, None, None, None,
                                    None, None, ctypes.byref(out)) == -1


@pytest.mark.parametrize("offsets,index,ok", [
    ((0, 4, 8), None, True),          # each instance reads its own 4 elements
    ((0, 4, 9), None, False),         # the last window runs past the leaf
    ((0, 4, 8), (0, 1, 2, 3), True),
    ((0, 4, 9), (0, 1, 2, 3), False),  # index 3 at offset 9 is element 12 of 12
    ((0, 0, 0), (11, 0, 5, 5), True),
    ((0, 0, 1), (11, 0, 5, 5), False),
])
def test_a_lone_leaf_is_read_at_every_instance_offset(offsets, index, ok):
    """A plan without steps: the root of an instance is leaf 0 from that
    instance's offset on, so the output (the first out_size elements, or the
    out_index entries) must lie inside the leaf at every offset."""
    L, _ = _mods()
    lib = L.load()
    t = L.qcs_tree_t()
    sizes = (ctypes.c_int64 * 1)(12)
    offs = (ctypes.c_int64 * 3)(*offsets)
    slots = (ctypes.c_int32 * 3)(0, 1, 2)
    t.n_leaves, t.n_steps, t.n_instances, t.n_slots = 1, 0, 3, 3
    t.leaf_size, t.instance_offset, t.instance_slot = sizes, offs, slots
    t.steps, t.out_size = None, 4
    idx = (ctypes.c_int64 * 4)(*index) if index is not None else None
    t.out_index = idx
    out = L.qcs_tree_layout_t()
    for backward in (0, 1):
        rc = lib.qcs_tree_layout_info(ctypes.byref(t), backward, 1, 1, 152, 32 << 30, None, None,
                                      None, None, None, ctypes.byref(out))
        assert rc == (0 if ok else L.QCS_ERR_INVALID_ARG), backward
