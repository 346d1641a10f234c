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
