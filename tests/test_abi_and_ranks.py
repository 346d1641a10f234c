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
