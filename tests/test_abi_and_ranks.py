"""CPU tests of the C ABI's presence (no compute calls) and of the
multi-rank host logic (instance sharding + FP64 all-reduce over gloo)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qcs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|const\s+char\s*\*)\s*(qcs_\w+)\s*\(", src)))


def test_library_loads_and_exports_every_declared_symbol():
    from paper_2303_08989_gb300 import _lib, build

    build.build()
    lib = ctypes.CDLL(_lib.LIB_PATH)
    names = _declared()
    assert len(names) >= 17
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(_lib.EXPORTED) == names


def test_header_is_plain_c_and_cpp():
    """include/qcs.h is a C ABI: it compiles on its own as C11 and as C++."""
    import shutil
    import subprocess

    hdr = os.path.join(ROOT, "include", "qcs.h")
    for cc, lang, std in (("gcc", "c", "-std=c11"), ("g++", "c++", "-std=c++17")):
        if shutil.which(cc) is None:
            pytest.skip(f"{cc} not installed")
        r = subprocess.run([cc, "-fsyntax-only", "-Wall", "-Werror", "-x", lang, std, hdr],
                           capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def test_cublas_interception_library_exports_its_entry_points():
    """libqcs_cublas.so (the drop-in route) defines the cuBLAS GEMMs it
    intercepts and its counter, and finds libqcs.so next to itself."""
    from paper_2303_08989_gb300 import build

    build.build()
    shim = ctypes.CDLL(build.SHIM)
    for name in ("cublasCgemm_v2", "cublasCgemmStridedBatched", "cublasCgemmBatched",
                 "cublasSgemm_v2", "cublasSgemmStridedBatched", "qcs_cublas_shim_counts"):
        assert hasattr(shim, name), name
    taken, passed = ctypes.c_longlong(-1), ctypes.c_longlong(-1)
    shim.qcs_cublas_shim_counts(ctypes.byref(taken), ctypes.byref(passed))
    assert (taken.value, passed.value) == (0, 0)


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import qcs_inputs as qi
    import paper_2303_08989_gb300.tn as tn
    from plan_sim import run

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    circ = qi.random_grid_circuit(3, 3, 6, seed=4)
    bits = qi.random_bitstrings(9, 3, seed=5)
    plan = tn.plan_circuit(circ, bits, seed=2, n_slices=3)
    sub = tn.shard_plan(plan, rank, world)
    part = torch.from_numpy(run(sub, [lf.data for lf in plan.net.leaves]))
    tn.allreduce_slots(part)
    q.put((rank, part.numpy()))
    dist.destroy_process_group()


def test_instance_sharding_with_gloo_allreduce():
    import socket

    import torch.multiprocessing as mp

    import oracle
    import qcs_inputs as qi

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    circ = qi.random_grid_circuit(3, 3, 6, seed=4)
    ref = oracle.sv_amplitudes(circ, qi.random_bitstrings(9, 3, seed=5))
    for r in (0, 1):
        np.testing.assert_allclose(res[r][:, 0], ref, atol=1e-6)


def _grad_out(plan, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((plan.n_slots, plan.out_size))
            + 1j * rng.standard_normal((plan.n_slots, plan.out_size)))


def _grad_plan():
    import qcs_inputs as qi
    import paper_2303_08989_gb300.tn as tn

    circ = qi.random_grid_circuit(2, 3, 4, seed=4, theta=None, phi=None, param_seed=5)
    bits = qi.random_bitstrings(6, 5, seed=6)
    net = tn.circuit_network(circ, None)
    order = tn.greedy_order(net, seed=2)
    sliced = tn.choose_slices(net, order, n_labels=2)
    return tn.build_plan(net, order, sliced, mode=0, outputs=bits)


def test_backward_interpreter_matches_central_differences():
    """The CPU adjoint of the plan interpreter (the reference the sharded
    backward is compared with): L = sum Re(conj(w) out) has torch gradient
    w with respect to out; its leaf gradients must match central
    differences of L along random complex directions of random leaves."""
    from plan_sim import run, run_backward

    plan = _grad_plan()
    leaves = [lf.data.astype(np.complex128) for lf in plan.net.leaves]
    w = _grad_out(plan, 3)
    grads = run_backward(plan, leaves, w)

    def L(lv):
        return float(np.sum(np.real(np.conj(w) * run(plan, lv))))

    rng = np.random.default_rng(4)
    for li in rng.choice(len(leaves), 4, replace=False):
        d = rng.standard_normal(leaves[li].size) + 1j * rng.standard_normal(leaves[li].size)
        h = 1e-6
        lp = [x.copy() for x in leaves]
        lm = [x.copy() for x in leaves]
        lp[li] = lp[li] + h * d
        lm[li] = lm[li] - h * d
        fd = (L(lp) - L(lm)) / (2 * h)
        an = float(np.real(np.vdot(grads[li], d)))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (li, fd, an)


def _grad_rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import paper_2303_08989_gb300.tn as tn
    from plan_sim import run_backward

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    plan = _grad_plan()
    sub = tn.shard_plan(plan, rank, world)
    leaves = [lf.data.astype(np.complex128) for lf in plan.net.leaves]
    grads = [torch.from_numpy(g) for g in run_backward(sub, leaves, _grad_out(plan, 3))]
    tn.allreduce_leaf_grads(grads)
    q.put((rank, [g.numpy() for g in grads]))
    dist.destroy_process_group()


def test_backward_sharding_with_gloo_allreduce_of_leaf_gradients():
    """Each of two ranks runs the adjoint on its round-robin share of the
    instances (slices); one all-reduce of the packed leaf gradients gives
    every rank the gradient of the whole plan."""
    import socket

    import torch.multiprocessing as mp

    from plan_sim import run_backward

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_grad_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    plan = _grad_plan()
    assert plan.n_instances == 4
    leaves = [lf.data.astype(np.complex128) for lf in plan.net.leaves]
    full = run_backward(plan, leaves, _grad_out(plan, 3))
    for r in (0, 1):
        for got, want in zip(res[r], full):
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)
