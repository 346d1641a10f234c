"""A plain numpy interpreter of executor plans (complex128), to test the
planner's host logic on the CPU: gathers by index arithmetic, GEMM with
numpy.matmul."""
import numpy as np


def gather_index(dims, strides):
    """Source offsets of a column-major matrix's elements in order t = 0, 1, ..."""
    total = int(np.prod(dims)) if dims else 1
    t = np.arange(total, dtype=np.int64)
    off = np.zeros(total, dtype=np.int64)
    for d, s in zip(dims, strides):
        off += (t % d) * s
        t //= d
    return off


def run(plan, leaves):
    """Returns (n_slots, out_size) complex128 like qcs_contract_tree."""
    nl = len(plan.net.leaves)
    out = np.zeros((plan.n_slots, plan.out_size), dtype=np.complex128)
    for inst in range(plan.n_instances):
        tens = []
        def src(i):
            if i < nl:
                return np.asarray(leaves[i], dtype=np.complex128)[plan.instance_offset[inst, i]:]
            return tens[i - nl]
        for st in plan.steps:
            A = src(st.a)[gather_index(*st.map_a)].reshape(st.m, st.k, order="F")
            B = src(st.b)[gather_index(*st.map_b)].reshape(st.k, st.n, order="F")
            if st.direct_a == 0:
                assert np.array_equal(A.ravel(order="F"), src(st.a)[: st.m * st.k])
            if st.direct_a == 1:
                assert np.array_equal(A.T.ravel(order="F"), src(st.a)[: st.m * st.k])
            if st.direct_b == 0:
                assert np.array_equal(B.ravel(order="F"), src(st.b)[: st.k * st.n])
            if st.direct_b == 1:
                assert np.array_equal(B.T.ravel(order="F"), src(st.b)[: st.k * st.n])
            tens.append((A @ B).ravel(order="F"))
        root = tens[-1] if plan.steps else src(0)
        vals = root[plan.out_index] if plan.out_index is not None else root[: plan.out_size]
        out[plan.instance_slot[inst]] += vals
    return out


def run_backward(plan, leaves, grad_out):
    """Leaf gradients (list of complex128 arrays, torch convention dL/dRe +
    i dL/dIm) for dL/d(out) = grad_out ((n_slots, out_size)), the adjoint of
    ``run``: per instance the forward recomputed, the root seeded from its
    slot's gradient, grad_A = grad_C B^H and grad_B = A^H grad_C per step,
    scattered back through the maps (leaves at the instance's offsets)."""
    nl = len(plan.net.leaves)
    grads = [np.zeros(np.asarray(lf).size, dtype=np.complex128) for lf in leaves]
    for inst in range(plan.n_instances):
        offs = plan.instance_offset[inst]
        tens = []

        def src(i):
            if i < nl:
                return np.asarray(leaves[i], dtype=np.complex128)[offs[i]:]
            return tens[i - nl]

        mats = []
        for st in plan.steps:
            A = src(st.a)[gather_index(*st.map_a)].reshape(st.m, st.k, order="F")
            B = src(st.b)[gather_index(*st.map_b)].reshape(st.k, st.n, order="F")
            mats.append((A, B))
            tens.append((A @ B).ravel(order="F"))
        root_size = tens[-1].size if plan.steps else np.asarray(leaves[0]).size - offs[0]
        groot = np.zeros(root_size, dtype=np.complex128)
        idx = plan.out_index if plan.out_index is not None else np.arange(plan.out_size)
        np.add.at(groot, idx, grad_out[plan.instance_slot[inst]])
        if not plan.steps:
            grads[0][offs[0]:offs[0] + root_size] += groot
            continue
        tgrad = [None] * len(plan.steps)
        tgrad[-1] = groot
        for s in range(len(plan.steps) - 1, -1, -1):
            st = plan.steps[s]
            A, B = mats[s]
            gC = tgrad[s].reshape(st.m, st.n, order="F")
            gA = (gC @ B.conj().T).ravel(order="F")
            gB = (A.conj().T @ gC).ravel(order="F")
            for opnd, g, mp in ((st.a, gA, st.map_a), (st.b, gB, st.map_b)):
                where = gather_index(*mp)
                if opnd < nl:
                    np.add.at(grads[opnd], offs[opnd] + where, g)
                else:
                    j = opnd - nl
                    if tgrad[j] is None:
                        tgrad[j] = np.zeros(tens[j].size, dtype=np.complex128)
                    np.add.at(tgrad[j], where, g)
    return grads
