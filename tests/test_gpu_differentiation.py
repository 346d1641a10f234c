"""The differentiated workload at its full size: a 20-qubit 4 x 5 grid
circuit of depth 12 whose fSim (theta, phi) are free parameters drawn from
U[0, pi] (parameter seed 3), loss L = sum over 256 bitstrings of
log |a_x|^2, contracted as an open network with 2 sliced indices (recomputed
per slice in the backward) in the cheapest of 64 seeded greedy orders,
AUTO-0.1 under the size rule measured on this GPU.

The gradient that qcs_contract_tree_backward returns through the
torch.autograd.Function is compared with the FP64 adjoint state-vector
gradient of the oracle (itself pinned against FP64 central differences on
the CPU), and the GPU loss is differentiated numerically along a few
parameters (central differences, h = 1e-3) as a convention-free check."""
import numpy as np
import pytest

import oracle
import qcs_inputs as qi
from gpu_helpers import lib, need_gpu, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def workload():
    need_gpu()
    import paper_2303_08989_gb300.tn as tn

    q = lib()
    circ = qi.random_grid_circuit(4, 5, 12, seed=0, theta=None, phi=None, param_seed=3)
    bits = qi.random_bitstrings(20, 256, seed=1)
    net = tn.circuit_network(circ, None)
    order, sliced, _ = tn.best_greedy_order(net, range(64), n_slices=2, workers=8)
    plan = tn.build_plan(net, order, sliced, mode=q.MODE_AUTO, outputs=bits)
    assert plan.n_instances == 4
    L_ref, g_ref = oracle.loss_and_grad(circ, bits)
    p0 = np.array([g.params for g in circ.gates if g.name == "fsim"], dtype=np.float64)
    return tn, q, circ, bits, plan, p0, L_ref, g_ref


def _loss(tn, cp, h, circ, plan, params):
    leaves = tn.torch_leaves(plan.net, circ, params)
    amps = tn.contract(cp, h, leaves)
    return torch.log(amps.abs() ** 2).sum()


def test_gradient_at_the_differentiation_workload(workload):
    tn, q, circ, bits, plan, p0, L_ref, g_ref = workload
    h = q.Handle(tol=0.1, size_rule=q.SIZE_RULE_TUNED)
    try:
        cp = tn.CompiledPlan(plan, leaf_data=[])
        cp.autotune(h, backward=True, reps=1)
        params = torch.tensor(p0, dtype=torch.float32, device="cuda", requires_grad=True)
        loss = _loss(tn, cp, h, circ, plan, params)
        loss.backward()
        torch.cuda.synchronize()
        h.sync()
        g = params.grad.double().cpu().numpy()
        assert abs(loss.item() - L_ref) < 1e-5 * abs(L_ref), (loss.item(), L_ref)
        rel = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
        print(f"[differentiation 4x5 d12] loss rel err {abs(loss.item() - L_ref) / abs(L_ref):.2e}, "
              f"gradient rel L2 vs FP64 adjoint {rel:.2e}")
        assert rel < 1e-4, rel
        # central differences of the GPU loss along three parameters
        rng = np.random.default_rng(7)
        hstep = 1e-3
        for gi in rng.choice(len(p0), 3, replace=False):
            for j in (0, 1):
                vals = []
                for sgn in (1.0, -1.0):
                    p = p0.copy()
                    p[gi, j] += sgn * hstep
                    with torch.no_grad():
                        pt = torch.tensor(p, dtype=torch.float32, device="cuda")
                        vals.append(_loss(tn, cp, h, circ, plan, pt).item())
                fd = (vals[0] - vals[1]) / (2 * hstep)
                assert abs(fd - g[gi, j]) <= 2e-3 + 1e-2 * abs(g[gi, j]), (gi, j, fd, g[gi, j])
    finally:
        h.close()


def test_graphed_forward_and_backward_equal_eager(workload):
    """The same forward + backward replayed as two CUDA graphs (both grouped
    over the 4 slices: the adjoint's steps for all slices at once, each
    slice's leaf gradients in its own buffer, added in slice order): loss and
    gradient bit-identical to the eager one-slice-at-a-time calls, on two
    replays in a row."""
    import time

    tn, q, circ, bits, plan, p0, L_ref, g_ref = workload
    h = q.Handle(tol=0.1, size_rule=q.SIZE_RULE_TUNED)
    try:
        cp = tn.CompiledPlan(plan, leaf_data=[])
        cp.autotune(h, backward=True, reps=1)
        params = torch.tensor(p0, dtype=torch.float32, device="cuda", requires_grad=True)

        def step():
            params.grad = None
            loss = _loss(tn, cp, h, circ, plan, params)
            loss.backward()
            torch.cuda.synchronize()
            h.sync()
            return loss.item(), params.grad.clone()

        step()
        t0 = time.perf_counter()
        l_eager, g_eager = step()
        t_eager = time.perf_counter() - t0
        h.set_instance_batch(4)
        cp.use_graphs(h)
        step()
        t0 = time.perf_counter()
        l_graph, g_graph = step()
        t_graph = time.perf_counter() - t0
        print(f"[differentiation 4x5 d12] forward + backward: eager {t_eager * 1e3:.1f} ms, "
              f"graphs {t_graph * 1e3:.1f} ms")
        assert l_graph == l_eager
        assert torch.equal(g_graph, g_eager)
        cp.graphed.close()
    finally:
        h.close()
