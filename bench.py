#!/usr/bin/env python
"""Emulated CGEMM throughput at FP32-level error, against plain FP32.

One step = one AUTO-mode qcs_cgemm on the CGEMM-sweep workload: exponent
statistics of A and B, device-side mode selection, the Eq. 1 split of both
operands, the tcgen05 error-corrected GEMM (and the candidate kernels that
exit because they were not selected).  Inputs are resident in HBM when the
timed region starts; they are larger than L2 (2 GiB per operand at 16384),
so no flush is needed between steps.

Printed JSON line (rank 0): the contract's keys plus
  e2e           the same metric through the public API with host buffers:
                per step, pinned-host -> device copies of A and B, the GEMM,
                and the device -> host copy of C;
  roofline      the tcgen05 GEMM kernel's tensor throughput (3 products per
                real product: 24 m n k flops) against the measured peak;
  cpu_baseline  the FP64 CPU oracle timed on a row sample of the same GEMM
                (its output also gives the error of the GPU result);
  fp32          the plain FP32 SIMT CGEMM and cuBLAS CGEMM (torch) on the same
                inputs, for the "vs plain FP32" part of the metric.

  --impl reference   times the FP64 CPU oracle alone (rank 0), same metric.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "emulated CGEMM TFLOP/s & contraction s/slice vs plain FP32 at FP32-level error"
UNIT = "TFLOP/s"


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--size", type=int, default=16384)
    p.add_argument("--s", type=int, default=0, help="exponent spread of the inputs")
    p.add_argument("--tol", type=float, default=0.1, help="AUTO-t underflow tolerance")
    p.add_argument("--mode", default="auto")
    p.add_argument("--sample-rows", type=int, default=16)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--no-tree", action="store_true", help="skip the contraction-tree legs")
    p.add_argument("--tree-slices", type=int, default=16,
                   help="slices of the 30-qubit network timed per mode")
    p.add_argument("--no-sweep", action="store_true", help="skip the CGEMM-sweep leg")
    p.add_argument("--no-sgemm", action="store_true", help="skip the real-GEMM leg")
    p.add_argument("--sgemm-sizes", type=int, nargs="+", default=[8192, 16384])
    p.add_argument("--rowcol-sizes", type=int, nargs="*", default=[8192],
                   help="sizes of the per-row/per-column scaling leg (none: skip it)")
    p.add_argument("--greedy-trials", type=int, default=1024,
                   help="seeded greedy orders tried per network (the cheapest is contracted)")
    p.add_argument("--greedy-workers", type=int, default=min(16, os.cpu_count() or 1),
                   help="host processes that cost the seeded orders")
    p.add_argument("--sweep-sizes", type=int, nargs="+", default=[1024, 2048, 4096, 8192, 16384])
    p.add_argument("--profile", choices=["slice", "slice_seed2", "gather", "gemm", "sgemm",
                                         "scaling", "contraction", "precision",
                                         "differentiation"],
                   default=None,
                   help="run one workload for an ncu capture (NVTX range 'measure') and exit: "
                        "'slice' one group of 16 slices of the 30-qubit network in the cheapest "
                        "of --greedy-trials greedy orders (AUTO-t, tuned rule), 'slice_seed2' one "
                        "slice in the "
                        "order of seed 2, 'gather' a random permutation of 2^26 elements, 'gemm' "
                        "ten qcs_cgemm calls of --gemm-shape in --mode, 'sgemm' ten qcs_sgemm "
                        "calls of --gemm-shape in --mode, 'scaling' the exponent spread of the "
                        "large GEMM operands of the 5x6 depth-14 network (order of seed 2) under "
                        "one scale per matrix, per row of op(A) and per column of op(B); "
                        "'differentiation' one forward + backward of the differentiated "
                        "workload in its cheapest order (--mode auto or fp32)")
    p.add_argument("--rowcol", action="store_true",
                   help="with --profile gemm: line-scaled operands and per-row/column scaling on")
    p.add_argument("--complex-products", type=int, choices=[3, 4], default=4,
                   help="with --profile gemm: real products per complex product (3: Gauss)")
    p.add_argument("--gemm-shape", type=int, nargs=3, default=[2048, 8192, 32],
                   metavar=("M", "N", "K"), help="the GEMM of --profile gemm")
    p.add_argument("--tuning-file", default=None,
                   help="with --profile slice*|contraction|precision|differentiation: load the "
                        "size-rule tuning table from this JSON "
                        "file if it exists, else measure it and write it there (a run under ncu "
                        "would measure distorted times: ncu slows every launch)")
    p.add_argument("--no-absorb", action="store_true",
                   help="contract the networks with their single-qubit gates as separate leaves "
                        "(default: absorbed into their neighbours on the host first)")
    p.add_argument("--no-levels", action="store_true",
                   help="run contraction trees step by step in plan order (default: level "
                        "launches of the small plain-FP32 steps, qcs_set_tree_levels)")
    p.add_argument("--group-budget-mb", type=int, default=None,
                   help="bytes (MiB) a grouped GPU-filling tree step may hold (qcs_set_group_budget; "
                        "default: the library's 32 GiB; 0: such steps one instance at a time)")
    p.add_argument("--instance-batch", type=int, default=16,
                   help="contraction instances per group (plain-FP32 steps batched)")
    p.add_argument("--legs-file", default=None,
                   help="also write every leg's full result to this JSON file (each leg is "
                        "printed to stderr as one JSON line in any case)")
    return p.parse_args(argv)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="qcs_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_operand(torch, n: int, s: int, seed: int, device):
    """n x n column-major complex64; parts N(0,1) * 2^e, e ~ U_int[-s, s]."""
    g = torch.Generator(device=device).manual_seed(seed)
    base = torch.empty((n, n), dtype=torch.complex64, device=device)  # (cols, rows) storage
    re = torch.randn((n, n), generator=g, device=device, dtype=torch.float32)
    im = torch.randn((n, n), generator=g, device=device, dtype=torch.float32)
    if s > 0:
        re.mul_(torch.exp2(torch.randint(-s, s + 1, (n, n), generator=g, device=device).float()))
        im.mul_(torch.exp2(torch.randint(-s, s + 1, (n, n), generator=g, device=device).float()))
    base.copy_(torch.complex(re, im))
    del re, im
    return base.t()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            mp = json.load(f)
        return mp.get("bf16_tflops"), mp.get("bf16_tflops_sustained"), "measured"
    except (OSError, ValueError):
        return 1900.0, 1700.0, "fallback"


def oracle_sample(A_rows_np, B_np, n: int, rows: int):
    """FP64 oracle on ``rows`` output rows: (seconds, result, threads)."""
    import numpy as np

    import oracle

    Asub = np.asfortranarray(A_rows_np[:rows])
    t0 = time.perf_counter()
    ref = oracle.cgemm(0, 0, rows, n, n, 1.0, Asub, B_np, rows=list(range(rows)))
    return time.perf_counter() - t0, ref, oracle.num_threads()


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle as it stands
# ---------------------------------------------------------------------------

TC_SOURCES = ["paper_2303_08989_gb300/csrc/gemm_tc.cu", "paper_2303_08989_gb300/csrc/ptx.cuh",
              "paper_2303_08989_gb300/csrc/internal.h"]
TC_TRAFFIC_PROFILE = "profiles/cgemm_tc_fp16x_16384_dram.md"


TC_CONSTANTS = ("kBM", "kBN", "kRowBytes", "kStages", "kPlanes", "kPlanesB", "kTileBytes",
                "kAStageBytes", "kBStageBytes", "kTcThreads", "kTmemCols")


def tc_sources_sha256() -> str:
    """SHA-256 of what the tensor-core kernel's DRAM traffic depends on: its
    source, its PTX wrappers and the tile constants it takes from the
    internal header (the header's other declarations do not count)."""
    import re

    h = hashlib.sha256()
    for rel in TC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            data = f.read()
        if rel.endswith("internal.h"):
            pat = re.compile(r"^constexpr\s+\w+\s+(%s)\s*=.*$" % "|".join(TC_CONSTANTS))
            data = "\n".join(ln for ln in data.decode().splitlines() if pat.match(ln)).encode()
        h.update(data)
    return h.hexdigest()


def tc_traffic(mode_used: str, n: int):
    """DRAM bytes per launch of the tensor-core kernel from the committed ncu
    capture (read + write), or None when that capture does not describe this
    launch: another workload, or kernel sources changed since."""
    if mode_used != "fp16x" or n != 16384:
        return None
    try:
        with open(os.path.join(ROOT, TC_TRAFFIC_PROFILE)) as f:
            fields = dict(line.strip("- \n").split(": ", 1) for line in f
                          if line.startswith("- ") and ": " in line)
        if fields.get("kernel_source_sha256") != tc_sources_sha256():
            return None
        return int(fields["traffic_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def gemm_config(args, world: int) -> dict:
    """The workload both arms report (the CGEMM-sweep point bench.py times)."""
    n = args.size
    return {"workload": f"CGEMM m=n=k={n}, parts N(0,1)*2^e, e~U_int[-{args.s},{args.s}], "
                        f"AUTO-{args.tol:g} (size rule on)",
            "m": n, "n": n, "k": n, "s": args.s, "tol": args.tol, "mode": args.mode,
            "l2": "operands 8*n^2 bytes each, larger than L2; no flush",
            "parallelism": f"{world} independent GEMMs (one per GPU)"}


def run_reference(args, rank: int):
    if rank != 0:
        return
    import numpy as np

    import oracle
    import qcs_inputs as qi

    n = args.size
    rows = 4
    A = qi.cgemm_operand(rows, n, args.s, seed=(1, n))
    B = qi.cgemm_operand(n, n, args.s, seed=(2, n))
    flops = 8.0 * rows * n * n
    for _ in range(args.warmup):
        oracle.cgemm(0, 0, rows, n, n, 1.0, A, B, rows=list(range(rows)))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.cgemm(0, 0, rows, n, n, 1.0, A, B, rows=list(range(rows)))
    dt = (time.perf_counter() - t0) / args.steps
    val = flops / dt / 1e12
    sample = f"{rows} output rows of the m=n=k={n} CGEMM per step (FP64 OpenMP oracle)"
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic",
        "config": dict(gemm_config(args, 1), sample=sample),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    del np


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def scaling_probe(args):
    """Per-row / per-column power-of-two scaling (a variant beyond Section
    4.1's one scale per matrix) on the operands a contraction feeds its large
    GEMMs.  Instance 0 of the 5x6 depth-14 network in the greedy order of
    seed 2 is contracted step by step with qcs_cgemm in plain FP32 (the
    intermediates carry FP32 rounding, as on the emulated path); for every
    step with m n k >= 2^33 it prints the fraction of op(A)'s and op(B)'s
    nonzero scalars below the window [e_max - 28, e_max] that scaling keeps,
    with e_max taken over the whole matrix (the paper), over each row of
    op(A) and over each column of op(B) (scales that the epilogue can undo
    exactly, 2^-(r_i + c_j))."""
    import torch

    import paper_2303_08989_gb300 as q
    import paper_2303_08989_gb300.tn as tn
    import qcs_inputs as qi

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)

    def fractions(X, per_row):
        v = torch.view_as_real(X).abs()
        nz = v > 0
        e = torch.frexp(v)[1].to(torch.int32) - 1  # floor(log2 |x|) of the nonzero scalars
        e = torch.where(nz, e, torch.full_like(e, -1000))
        n = max(int(nz.sum()), 1)
        emax = int(e.max())
        local = e.amax(dim=(1, 2) if per_row else (0, 2), keepdim=True)
        return (emax, int(((e < emax - 28) & nz).sum()) / n,
                int(((e < local - 28) & nz).sum()) / n)

    circ = qi.random_grid_circuit(5, 6, 14, seed=0)
    bits = qi.random_bitstrings(30, 1, seed=1)
    net = tn.circuit_network(circ, bits)
    order = tn.greedy_order(net, seed=2, skip=[tn.BATCH])
    plan = tn.build_plan(net, order, tn.choose_slices(net, order, n_labels=6, skip=[tn.BATCH]))
    h = q.Handle(size_rule=False)
    nl = len(plan.net.leaves)
    leaves = [torch.from_numpy(lf.data).to(dev) for lf in plan.net.leaves]
    tens = []

    def src(i):
        return leaves[i][int(plan.instance_offset[0, i]):] if i < nl else tens[i - nl]

    rows = []
    for s, st in enumerate(plan.steps):
        A = torch.as_strided(src(st.a), tuple(st.map_a[0][::-1]), tuple(st.map_a[1][::-1]))
        B = torch.as_strided(src(st.b), tuple(st.map_b[0][::-1]), tuple(st.map_b[1][::-1]))
        A = q.to_fortran(A.reshape(st.k, st.m).t(), device=dev)
        B = q.to_fortran(B.reshape(st.n, st.k).t(), device=dev)
        C = q.cgemm(h, A, B, mode="fp32")
        if st.m * st.n * st.k >= 2 ** 33:
            ea, ga, la = fractions(A, True)
            eb, gb, lb = fractions(B, False)
            rows.append({"step": s, "m": st.m, "n": st.n, "k": st.k,
                         "A": {"e_max": ea, "below_window_per_matrix": ga, "per_row": la},
                         "B": {"e_max": eb, "below_window_per_matrix": gb, "per_column": lb}})
        tens.append(C.t().reshape(-1))
        del A, B
    h.close()
    print(json.dumps({"profile": "scaling", "steps": rows}), flush=True)


def contraction_network(args, tn, qi):
    """The 30-qubit network of the contraction leg: 5x6 grid, depth 14, one
    bitstring, in the cheapest of --greedy-trials seeded greedy orders over
    the network with and without its single-qubit gates absorbed, 6 sliced
    indices.  Returns (circuit, bits, networks, index used, order, sliced, seed)."""
    circ = qi.random_grid_circuit(5, 6, 14, seed=0)
    bits = qi.random_bitstrings(30, 1, seed=1)
    net_full = tn.circuit_network(circ, bits)
    nets = [net_full] + ([] if args.no_absorb else [tn.absorb_single_qubit_gates(net_full)])
    which, order, sliced, seed_used = tn.cheapest_network_order(
        nets, range(args.greedy_trials), skip=[tn.BATCH], n_slices=6, workers=args.greedy_workers)
    return circ, bits, nets, which, order, sliced, seed_used


def precision_network(args, tn, qi):
    """The 40-qubit network of the precision leg: 5x8 grid, depth 12, one
    bitstring, sliced on the 8 indices of tests/golden/slices5x8_d12.txt, in
    the cheapest of --greedy-trials orders.  Returns (labels, golden rows,
    circuit, bits, networks, index used, order, seed), or None without the file."""
    path = os.path.join(ROOT, "tests", "golden", "slices5x8_d12.txt")
    if not os.path.exists(path):
        return None
    labels, rows = None, []
    with open(path) as f:
        for line in f:
            if line.startswith("sliced"):
                labels = [int(v) for v in line.split()[1:]]
            elif line.strip() and not line.startswith("#"):
                v, re, im = line.split()
                rows.append((v, float(re) + 1j * float(im)))
    circ = qi.random_grid_circuit(5, 8, 12, seed=0)
    bits = qi.random_bitstrings(40, 1, seed=1)
    net_full = tn.circuit_network(circ, bits)
    # absorbed or not, the oracle's sliced labels survive
    nets = [net_full] + ([] if args.no_absorb else
                         [tn.absorb_single_qubit_gates(net_full, keep_labels=labels)])
    which, order, _, seed_used = tn.cheapest_network_order(
        nets, range(args.greedy_trials), skip=[tn.BATCH] + labels, workers=args.greedy_workers)
    return labels, rows, circ, bits, nets, which, order, seed_used


def differentiation_network(args, tn, qi):
    """The differentiated workload (4x5 grid, depth 12, free fSim parameters,
    256 bitstrings) and its two contraction orders: the greedy order of seed 2
    (4.2e11 flops per slice: the adjoint GEMMs are large enough for the tensor
    cores) and the cheapest of --greedy-trials orders over the network with and
    without its frozen single-qubit gates absorbed."""
    import numpy as np

    c4 = qi.random_grid_circuit(4, 5, 12, seed=0, theta=None, phi=None, param_seed=3)
    b4 = qi.random_bitstrings(20, 256, seed=1)
    p0s = np.array([g.params for g in c4.gates if g.name == "fsim"])
    net4_full = tn.circuit_network(c4, None)
    # the parametric fSim leaves stay as they are
    nets4 = [net4_full] + ([] if args.no_absorb else
                           [tn.absorb_single_qubit_gates(net4_full, frozen_gates=c4.fsim_indices())])
    o_s2 = tn.greedy_order(net4_full, seed=2)
    orders = {"seed2": (net4_full, o_s2, tn.choose_slices(net4_full, o_s2, n_labels=2))}
    w4, o_b, sl_b, _ = tn.cheapest_network_order(nets4, range(args.greedy_trials), n_slices=2,
                                                 workers=args.greedy_workers)
    orders["cheapest"] = (nets4[w4], o_b, sl_b)
    return c4, b4, p0s, orders, w4


def differentiation_setup(q, tn, torch, dev, hd, c4, b4, p0s, net_order, mode, rule,
                          tuning_file=None):
    """Plan, compiled plan, parameters and the forward + backward closure of
    the differentiated workload in one order (the loss is the sum of
    log|a|^2 over the bitstrings).  Under the tuned rule the size-rule table
    is measured, or loaded from ``tuning_file`` when that file exists (and
    written there otherwise)."""
    net4, order, sliced = net_order
    plan = tn.build_plan(net4, order, sliced, mode=q.MODE_BY_NAME[mode], outputs=b4)
    cp = tn.CompiledPlan(plan, device=dev, leaf_data=[])
    if rule == q.SIZE_RULE_TUNED:
        if tuning_file and os.path.exists(tuning_file):
            with open(tuning_file) as f:
                hd.set_tuning(json.load(f))
        else:
            cp.autotune(hd, backward=True, reps=2)
            if tuning_file:
                with open(tuning_file, "w") as f:
                    json.dump(hd.tuning(), f)
    params = torch.tensor(p0s, dtype=torch.float32, device=dev, requires_grad=True)

    def fwd_bwd():
        params.grad = None
        leaves = tn.torch_leaves(plan.net, c4, params, device=dev)
        amps = tn.contract(cp, hd, leaves)
        loss = torch.log(amps.abs() ** 2).sum()
        loss.backward()
        return loss
    return plan, cp, params, fwd_bwd


def profile_run(args):
    """One workload between torch.cuda.nvtx range 'measure' (after one
    untimed run), for ``ncu --nvtx --nvtx-include "measure/"``; prints a
    short JSON line with the CUDA-event time of the measured run."""
    import torch

    import paper_2303_08989_gb300 as q
    import paper_2303_08989_gb300.tn as tn
    import qcs_inputs as qi

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.profile == "differentiation":
        c4, b4, p0s, orders, w4 = differentiation_network(args, tn, qi)
        rule = q.SIZE_RULE_PAPER if args.mode == "fp32" else q.SIZE_RULE_TUNED
        h = q.Handle(tol=args.tol, size_rule=rule)
        plan, cp, params, run = differentiation_setup(q, tn, torch, dev, h, c4, b4, p0s,
                                                      orders["cheapest"], args.mode, rule,
                                                      args.tuning_file)
        h.set_instance_batch(plan.n_instances)
        cp.use_graphs(h)
        fwd_bwd = run

        def run():
            # the backward on this thread (not autograd's device thread), so
            # that ncu's NVTX filter on the range "measure" sees its launches
            with torch.autograd.set_multithreading_enabled(False):
                return fwd_bwd()

        def phases():
            """The same forward + backward with CUDA events and host clocks
            between its parts: leaf tensors, forward replay, loss, backward."""
            params.grad = None
            marks = []

            def mark(name):
                ev = torch.cuda.Event(enable_timing=True)
                ev.record()
                marks.append((name, ev, time.perf_counter()))
            mark("start")
            leaves = tn.torch_leaves(plan.net, c4, params, device=dev)
            mark("leaves")
            amps = tn.contract(cp, h, leaves)
            mark("forward")
            loss = torch.log(amps.abs() ** 2).sum()
            mark("loss")
            with torch.autograd.set_multithreading_enabled(False):
                loss.backward()
            mark("backward")
            torch.cuda.synchronize()
            return {b[0]: {"event_ms": a[1].elapsed_time(b[1]), "wall_ms": (b[2] - a[2]) * 1e3}
                    for a, b in zip(marks, marks[1:])}
        what = ("forward + backward of the differentiated 4x5 depth-12 workload (256 "
                "bitstrings, 4 slices) in the cheapest of %d orders, %s, two CUDA-graph "
                "replays" % (args.greedy_trials, args.mode))
    elif args.profile in ("slice", "slice_seed2", "contraction", "precision"):
        circ = qi.random_grid_circuit(5, 6, 14, seed=0)
        bits = qi.random_bitstrings(30, 1, seed=1)
        if args.profile == "contraction":
            _, _, nets, which, order, sliced, seed_used = contraction_network(args, tn, qi)
            plan = tn.build_plan(nets[which], order, sliced, mode=q.MODE_AUTO)
            ni, what = 16, ("16 slices (one group) of the contraction leg's 30-qubit network "
                            "(seed %d of %d, single-qubit gates %s), AUTO-%g, tuned rule"
                            % (seed_used, args.greedy_trials,
                               "absorbed" if which == 1 else "apart", args.tol))
        elif args.profile == "precision":
            labels, _, _, _, nets, which, order, seed_used = precision_network(args, tn, qi)
            plan = tn.build_plan(nets[which], order, labels, mode=q.MODE_AUTO)
            ni, what = 16, ("16 slices (one group) of the precision leg's 40-qubit network "
                            "(seed %d of %d), AUTO-%g, tuned rule"
                            % (seed_used, args.greedy_trials, args.tol))
        elif args.profile == "slice":
            plan = tn.plan_circuit(circ, bits, seed=0, n_slices=6, mode=q.MODE_AUTO,
                                   trials=args.greedy_trials, workers=args.greedy_workers)
            ni, what = 16, ("16 slices (one group) of the 5x6 depth-14 network in the cheapest "
                            "of %d greedy orders, AUTO-%g, tuned rule"
                            % (args.greedy_trials, args.tol))
        else:
            plan = tn.plan_circuit(circ, bits, seed=2, n_slices=6, mode=q.MODE_AUTO)
            ni, what = 1, ("one slice of the 5x6 depth-14 network in the greedy order of "
                           "seed 2, AUTO-%g, tuned rule" % args.tol)
        cp = tn.CompiledPlan(plan, device=dev)
        cp.tree.n_instances = ni
        h = q.Handle(tol=args.tol, size_rule=q.SIZE_RULE_TUNED)
        h.set_instance_batch(ni)
        if args.tuning_file and os.path.exists(args.tuning_file):
            with open(args.tuning_file) as f:
                h.set_tuning(json.load(f))
        else:
            cp.autotune(h)
            if args.tuning_file:
                with open(args.tuning_file, "w") as f:
                    json.dump(h.tuning(), f)
        run = lambda: cp.forward(h)
    elif args.profile == "gemm":
        m, n, k = args.gemm_shape
        h = q.Handle(tol=args.tol, size_rule=False)
        h.set_complex_products(args.complex_products)
        if args.rowcol:
            if not (m == n == k):
                raise SystemExit("--rowcol takes a square --gemm-shape")
            A = make_line_operand(torch, m, 30, 0, 41 * m, dev)
            B = make_line_operand(torch, m, 30, 1, 43 * m, dev)
            h.set_rowcol_scaling(True)
        else:
            g = torch.Generator(device=dev).manual_seed(9)
            A = torch.randn((k, m), dtype=torch.complex64, device=dev, generator=g).t()
            B = torch.randn((n, k), dtype=torch.complex64, device=dev, generator=g).t()
        C = q.fortran_empty(m, n, device=dev)

        def run():
            for _ in range(10):
                q.cgemm(h, A, B, C, mode=args.mode)
        what = "10 x qcs_cgemm (%d, %d, %d), mode %s, %s, %d real products" % (
            m, n, k, args.mode,
            "lines N(0,1)*2^e, e~U_int[-30,30], per-row/column scaling on" if args.rowcol
            else "parts N(0,1)", args.complex_products)
    elif args.profile == "sgemm":
        m, n, k = args.gemm_shape
        g = torch.Generator(device=dev).manual_seed(9)
        A = torch.randn((k, m), dtype=torch.float32, device=dev, generator=g).t()
        B = torch.randn((n, k), dtype=torch.float32, device=dev, generator=g).t()
        C = q.fortran_empty_real(m, n, device=dev)
        h = q.Handle(tol=args.tol, size_rule=False)

        def run():
            for _ in range(10):
                q.sgemm(h, A, B, C, mode=args.mode)
        what = "10 x qcs_sgemm (%d, %d, %d), mode %s, entries N(0,1)" % (m, n, k, args.mode)
    else:
        r = 26
        g = torch.Generator(device="cpu").manual_seed(5)
        perm = torch.randperm(r, generator=g).tolist()
        src = torch.empty(2 ** r, dtype=torch.complex64, device=dev)
        out = torch.empty_like(src)
        h = q.Handle()
        strides = [2 ** p for p in perm]
        run = lambda: q.permute(h, src, [2] * r, strides, out=out)
        what = "permutation of 2^26 complex64 (26 binary indices, seeded)"
    run()
    torch.cuda.synchronize()
    with torch.cuda.nvtx.range("measure"):
        t0 = time.perf_counter()
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    h.sync()
    res = {"profile": args.profile, "workload": what, "ms": e0.elapsed_time(e1),
           "wall_ms": wall * 1e3}
    if args.profile == "differentiation":
        res["phases"] = phases()
    print(json.dumps(res), flush=True)
    if args.profile == "differentiation":
        cp.graphed.close()
    h.close()


def main():
    args = parse()
    if args.no_levels:
        os.environ["QCS_TREE_LEVELS"] = "0"  # read by every handle at creation
    if args.group_budget_mb is not None:
        os.environ["QCS_GROUP_BUDGET_MB"] = str(args.group_budget_mb)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.profile == "scaling":
        scaling_probe(args)
        return
    if args.profile:
        profile_run(args)
        return

    import numpy as np
    import torch

    import paper_2303_08989_gb300 as q

    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    n = args.size
    flops = 8.0 * n * n * n
    h = q.Handle(tol=args.tol, size_rule=True)
    A = make_operand(torch, n, args.s, 1000 + rank, dev)
    B = make_operand(torch, n, args.s, 2000 + rank, dev)
    C = q.fortran_empty(n, n, device=dev)
    desc = torch.zeros(4, dtype=torch.int32, device=dev)

    # ---- warm-up ----
    for _ in range(args.warmup):
        q.cgemm(h, A, B, C, mode=args.mode, desc_out=desc)
    torch.cuda.synchronize()
    mode_used = q.MODE_NAME[int(desc[0].item())]

    # ---- timed region: device-resident inputs ----
    clocks = ClockSampler(dev.index if world == 1 else local)
    h.set_profiling(True)
    h.get_profile()  # clear
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        q.cgemm(h, A, B, C, mode=args.mode)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    prof = h.get_profile()
    h.set_profiling(False)
    ms = max_over_ranks(ms)
    value = world * flops / (ms * 1e-3) / 1e12
    # statistics pass 1 and 2, selection, split x2, tcgen05 FP16, tcgen05 TF32, SIMT (gated)
    launches_per_step = 8

    # ---- dominant kernel roofline (live CUDA-event timing of the tcgen05 GEMM) ----
    tc_ms, tc_n = prof["gemm_tc"]
    tc_avg = tc_ms / max(tc_n, 1)
    burst, sustained, src = peaks()
    kind_ratio = {"fp16x": 1.0, "fp16x_scaled": 1.0, "bf16x3": 1.0, "tf32x": 1.1 / 2.25}.get(mode_used)
    roofline = None
    if kind_ratio is not None and tc_avg > 0:
        achieved = 24.0 * n * n * n / (tc_avg * 1e-3) / 1e12
        peak = sustained * kind_ratio
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": tc_traffic(mode_used, n),
                    "kernel": f"cgemm_tc_kernel ({mode_used}), 3 tensor products per real product",
                    "peak_source": f"{src} bf16 sustained" + (" x TF32/BF16 nominal ratio 1.1/2.25"
                                                              if kind_ratio != 1.0 else "")}
    stages = {k: {"ms_per_step": v[0] / args.steps, "launches": v[1]} for k, v in prof.items() if v[1]}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64",
        "data": "synthetic (seeded torch.randn on the device)",
        "config": dict(gemm_config(args, world), mode_selected=mode_used),
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clk,
        "stages": stages,
        "roofline": roofline,
    }

    legs = {}

    # ---- error of the GPU result against the FP64 oracle (row sample) + CPU baseline ----
    if rank == 0:
        rows = args.sample_rows
        A_rows = A[:rows].cpu().numpy().astype(np.complex64)
        B_np = B.cpu().numpy()
        C_rows = C[:rows].cpu().numpy().astype(np.complex128)
        secs, ref, threads = oracle_sample(A_rows, B_np, n, rows)
        import oracle

        out["error"] = {"rel_fro_vs_fp64": oracle.rel_fro_error(C_rows, ref),
                        "sample": f"{rows} output rows"}
        if world == 1:  # the oracle's rate is reported at N = 1 only
            out["cpu_baseline"] = {"value": 8.0 * rows * n * n / secs / 1e12, "unit": UNIT,
                                   "cores": threads, "kind": "oracle",
                                   "sample": f"{rows} of {n} output rows of the same GEMM "
                                             "(FP64, OpenMP)",
                                   "seconds": secs}
        del B_np

    # ---- plain FP32 on the same inputs ----
    if not args.no_extras:
        reps = 2
        C2 = q.fortran_empty(n, n, device=dev)
        q.cgemm(h, A, B, C2, mode="fp32")
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            q.cgemm(h, A, B, C2, mode="fp32")
        e1.record(stream)
        torch.cuda.synchronize()
        simt = flops / (e0.elapsed_time(e1) / reps * 1e-3) / 1e12
        torch.matmul(A, B)  # cuBLAS CGEMM on the column-major views (default math mode)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            torch.matmul(A, B)
        e1.record(stream)
        torch.cuda.synchronize()
        cublas = flops / (e0.elapsed_time(e1) / reps * 1e-3) / 1e12
        # the CUDA cores' FP32 FMA rate right after: the SIMT kernel's roofline
        fma_peak = h.measure_fma_peak()
        out["fp32"] = {"simt_tflops": simt, "cublas_cgemm_tflops": cublas,
                       "fma_peak_tflops": fma_peak, "simt_frac_of_fma_peak": simt / fma_peak}
        if rank == 0:
            C2r = C2[:args.sample_rows].cpu().numpy().astype(np.complex128)
            import oracle

            out["fp32"]["rel_fro_vs_fp64"] = oracle.rel_fro_error(C2r, ref)
        # the other emulated paths on the same inputs, forced: TF32X (AUTO's
        # fallback) and BF16X3 (a measured candidate AUTO never selects)
        legs["candidates"] = {}
        for mode in ("tf32x", "bf16x3"):
            q.cgemm(h, A, B, C2, mode=mode)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                q.cgemm(h, A, B, C2, mode=mode)
            e1.record(stream)
            torch.cuda.synchronize()
            entry = {"tflops": flops / (e0.elapsed_time(e1) / reps * 1e-3) / 1e12}
            if rank == 0:
                entry["rel_fro_vs_fp64"] = oracle.rel_fro_error(
                    C2[:args.sample_rows].cpu().numpy().astype(np.complex128), ref)
            legs["candidates"][mode] = entry
        # Gauss's three-product form (a variant beyond the paper): AUTO-t and
        # forced FP16X on the same inputs, nominal 8 m n k flops
        h3 = q.Handle(tol=args.tol, size_rule=True)
        h3.set_complex_products(3)
        for mode in ("auto", "fp16x"):
            q.cgemm(h3, A, B, C2, mode=mode)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(reps):
                q.cgemm(h3, A, B, C2, mode=mode)
            e1.record(stream)
            torch.cuda.synchronize()
            entry = {"tflops": flops / (e0.elapsed_time(e1) / reps * 1e-3) / 1e12,
                     "complex_products": 3}
            if rank == 0:
                entry["rel_fro_vs_fp64"] = oracle.rel_fro_error(
                    C2[:args.sample_rows].cpu().numpy().astype(np.complex128), ref)
            legs["candidates"][mode + "_3m"] = entry
        h3.close()
        del C2

    # ---- end to end through the public API, host buffers ----
    if not args.no_e2e:
        hA = torch.empty((n, n), dtype=torch.complex64, pin_memory=True)
        hB = torch.empty((n, n), dtype=torch.complex64, pin_memory=True)
        hC = torch.empty((n, n), dtype=torch.complex64, pin_memory=True)
        hA.copy_(A.t())
        hB.copy_(B.t())
        Ad = torch.empty((n, n), dtype=torch.complex64, device=dev)
        Bd = torch.empty((n, n), dtype=torch.complex64, device=dev)
        Cd = torch.empty((n, n), dtype=torch.complex64, device=dev)

        def e2e_step():
            Ad.copy_(hA, non_blocking=True)
            Bd.copy_(hB, non_blocking=True)
            q.cgemm(h, Ad.t(), Bd.t(), Cd.t(), mode=args.mode)
            hC.copy_(Cd, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        # as many steps as the timed region, so that the pipeline's fill (the
        # first step's copies in) and drain (the last copy out) weigh little
        ek = max(4, args.steps)
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(ek):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ems_serial = max_over_ranks(e0.elapsed_time(e1) / ek)

        # The same steps pipelined: two device buffer sets and three streams,
        # so that step i+1's host->device copies and step i-1's device->host
        # copy overlap step i's GEMM.  Every step still copies its own inputs
        # in and its own result out inside the timed region.
        sets = [(Ad, Bd, Cd)] + [tuple(torch.empty((n, n), dtype=torch.complex64, device=dev)
                                       for _ in range(3))]
        s_in, s_cmp, s_out = (torch.cuda.Stream(device=dev) for _ in range(3))
        ev = {key: [torch.cuda.Event() for _ in range(2)] for key in ("in", "gemm", "out")}
        h.set_stream(s_cmp)

        def e2e_pipelined(steps):
            for i in range(steps):
                b = i % 2
                A_, B_, C_ = sets[b]
                with torch.cuda.stream(s_in):
                    if i >= 2:
                        s_in.wait_event(ev["gemm"][b])
                    A_.copy_(hA, non_blocking=True)
                    B_.copy_(hB, non_blocking=True)
                    ev["in"][b].record(s_in)
                with torch.cuda.stream(s_cmp):
                    s_cmp.wait_event(ev["in"][b])
                    if i >= 2:
                        s_cmp.wait_event(ev["out"][b])
                    q.cgemm(h, A_.t(), B_.t(), C_.t(), mode=args.mode)
                    ev["gemm"][b].record(s_cmp)
                with torch.cuda.stream(s_out):
                    s_out.wait_event(ev["gemm"][b])
                    hC.copy_(C_, non_blocking=True)
                    ev["out"][b].record(s_out)

        e2e_pipelined(2)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(s_in)
        s_cmp.wait_event(p0)
        s_out.wait_event(p0)
        e2e_pipelined(ek)
        p1.record(s_out)  # after the last copy out, which waited for everything before it
        torch.cuda.synchronize()
        barrier()
        h.set_stream(stream)
        ems = max_over_ranks(p0.elapsed_time(p1) / ek)
        out["e2e"] = {"value": world * flops / (ems * 1e-3) / 1e12, "unit": UNIT,
                      "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": n * n * 8,
                      "ms_per_step": ems, "steps": ek,
                      "pipelined": "2 buffer sets, 3 streams",
                      "serial_value": world * flops / (ems_serial * 1e-3) / 1e12,
                      "serial_ms_per_step": ems_serial}
        del hA, hB, hC, Ad, Bd, Cd, sets

    # The legs after the timed step report beside the headline; one that
    # raises is recorded as {"error": ...} and the line is still printed.
    def leg(key, fn):
        try:
            res = fn()
        except Exception as e:  # noqa: BLE001 -- reported in the JSON line
            import traceback

            traceback.print_exc()
            legs[key or "tree_legs"] = {"error": f"{type(e).__name__}: {e}"[:500]}
            return
        legs.update(res if key is None else {key: res})

    if not args.no_extras:
        leg("hbm_kernels", lambda: hbm_legs(q, torch, dev, h, stages, n))
    if not args.no_extras and not args.no_sweep:
        leg("sweep", lambda: sweep_leg(args, q, torch, dev, rank))
    if not args.no_extras and not args.no_sgemm:
        leg("sgemm", lambda: sgemm_leg(args, q, torch, dev, rank))
    if not args.no_extras and args.rowcol_sizes:
        leg("rowcol", lambda: rowcol_leg(args, q, torch, dev, rank))

    if not args.no_tree:
        leg(None, lambda: tree_legs(args, q, torch, dev, rank, world, dist))

    if rank == 0:
        emit_legs(legs, args.legs_file)
        print(json.dumps(contract_line(out, legs)), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# output: the legs in full on stderr (and optionally a file), one short line
# on stdout
# ---------------------------------------------------------------------------

LINE_LIMIT = 2800  # bytes; the contract line stays well inside what a log tail keeps


def _sig(x, digits=4):
    """``x`` rounded to ``digits`` significant digits (other types unchanged)."""
    if isinstance(x, float):
        import math

        if not math.isfinite(x) or x == 0.0:
            return x if math.isfinite(x) else None
        return float(f"{x:.{digits}g}")
    if isinstance(x, dict):
        return {k: _sig(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [_sig(v, digits) for v in x]
    return x


def emit_legs(legs: dict, path=None):
    """Every leg as one JSON line on stderr, tagged with its name, and all of
    them in one JSON object at ``path`` when given."""
    for key, val in legs.items():
        print(json.dumps({"leg": key, "result": val}, default=str), file=sys.stderr, flush=True)
    if path:
        d = os.path.dirname(os.path.abspath(path))
        os.makedirs(d, exist_ok=True)
        with open(path, "w") as f:
            json.dump(legs, f, indent=1, default=str)


def legs_summary(legs: dict) -> dict:
    """A few numbers per leg for the contract line: seconds per slice of the
    contractions (AUTO against all-FP32) with their errors against FP64, the
    differentiated workload, the sweep's range of AUTO speed-ups, and the
    memory-bound kernels' fractions of copy bandwidth; a leg that failed
    keeps the start of its error message."""
    s = {}

    def ms(entry):
        return None if not isinstance(entry, dict) or "s_per_slice" not in entry \
            else entry["s_per_slice"] * 1e3

    for key, name in (("contraction", "contraction_5x6_d14"),
                      ("precision_at_scale", "precision_5x8_d12"),
                      ("contraction_seed2_order", "contraction_5x6_d14_seed2_order")):
        c = legs.get(key)
        if not isinstance(c, dict):
            continue
        if "error" in c or "skipped" in c:
            s[name] = {"error": str(c.get("error", c.get("skipped")))[:120]}
            continue
        e = {"auto_ms_per_slice": ms(c.get("auto")), "auto_t0.5_ms_per_slice": ms(c.get("auto_t0.5")),
             "fp32_ms_per_slice": ms(c.get("fp32")), "speedup_vs_fp32": c.get("speedup_vs_fp32")}
        auto = c.get("auto") or {}
        if "amplitude_rel_err_vs_fp64" in auto:
            e["auto_amp_rel_err_vs_fp64"] = auto["amplitude_rel_err_vs_fp64"]
            e["fp32_amp_rel_err_vs_fp64"] = (c.get("fp32") or {}).get("amplitude_rel_err_vs_fp64")
        if "sampled_slices_fidelity_vs_fp64" in c:
            e["auto_infidelity_4_slices_vs_fp64"] = 1.0 - c["sampled_slices_fidelity_vs_fp64"]
        ff = ((auto.get("routing") or {}).get("flops_fraction"))
        if ff:
            e["auto_flops_fraction"] = {k: v for k, v in ff.items() if v}
        s[name] = e
    d = legs.get("differentiation")
    if isinstance(d, dict):
        if "error" in d:
            s["differentiation_4x5_d12"] = {"error": str(d["error"])[:120]}
        else:
            s["differentiation_4x5_d12"] = {
                k: d.get(k) for k in ("auto_s", "fp32_s", "speedup_vs_fp32",
                                      "auto_grad_rel_l2_vs_fp64", "fp32_grad_rel_l2_vs_fp64")}
            if isinstance(d.get("cheapest_order"), dict):
                co = d["cheapest_order"]
                s["differentiation_4x5_d12"]["cheapest_order_auto_s"] = co.get("auto_s")
                s["differentiation_4x5_d12"]["cheapest_order_fp32_s"] = co.get("fp32_s")
    sh = legs.get("contraction_sharded")
    if isinstance(sh, dict) and "error" not in sh:
        s["contraction_5x6_d14_sharded"] = {k: sh.get(k) for k in
                                            ("ranks", "s_per_slice", "amplitude_rel_err_vs_fp64")}
    p = legs.get("plain_small")
    if isinstance(p, dict) and "error" not in p:
        s["plain_3x4_d8"] = {"ms_per_64_bitstrings_graph": (p.get("s_per_batch_grouped_cuda_graph")
                                                            or 0) * 1e3,
                             "infidelity_vs_fp64": (None if p.get("fidelity_vs_fp64") is None
                                                    else 1.0 - p["fidelity_vs_fp64"])}
    sw = legs.get("sweep")
    if isinstance(sw, dict):
        if "error" in sw:
            s["sweep"] = {"error": str(sw["error"])[:120]}
        else:
            sp = [pt["auto_speedup_vs_fp32"] for pt in sw.get("points", [])
                  if "auto_speedup_vs_fp32" in pt]
            er = [pt["auto_err_ratio_vs_fp32"] for pt in sw.get("points", [])
                  if "auto_err_ratio_vs_fp32" in pt]
            s["sweep"] = {"points": len(sw.get("points", [])),
                          "auto_speedup_vs_fp32_min_max": [min(sp), max(sp)] if sp else None,
                          "auto_err_over_fp32_err_min_max": [min(er), max(er)] if er else None}
    hb = legs.get("hbm_kernels")
    if isinstance(hb, dict) and "error" not in hb:
        s["hbm_frac"] = {k: v["frac"] for k, v in hb.items() if isinstance(v, dict) and "frac" in v}
    for key, val in legs.items():
        if isinstance(val, dict) and "error" in val and key not in s:
            s[key] = {"error": str(val["error"])[:120]}
    return _sig(s)


def contract_line(out: dict, legs: dict) -> dict:
    """The one JSON line of the contract: the headline step's keys from
    ``out`` and a short summary of the legs, trimmed to ``LINE_LIMIT``
    bytes (the longest summaries go first)."""
    line = _sig(dict(out), 6)
    line["legs"] = legs_summary(legs)
    line["legs_detail"] = "one JSON line per leg on stderr (--legs-file writes them to a file)"
    keep = ["contraction_5x6_d14", "contraction_5x6_d14_sharded", "precision_5x8_d12",
            "differentiation_4x5_d12", "sweep",
            "contraction_5x6_d14_seed2_order", "plain_3x4_d8", "hbm_frac"]
    order = sorted(line["legs"], key=lambda k: -keep.index(k) if k in keep else -len(keep))
    while len(json.dumps(line)) > LINE_LIMIT and order:
        line["legs"].pop(order.pop(0))
    for key in ("stages", "fp32", "error"):
        if len(json.dumps(line)) > LINE_LIMIT:
            line.pop(key, None)
    return line


def hbm_legs(q, torch, dev, h, stages, n):
    """Bandwidth of the memory-bound kernels of the path, against the
    measured HBM copy bandwidth: statistics and split (from the CGEMM
    step's live stage timings), a standalone gather (a random permutation
    of a 2^28-element tensor of 28 binary indices, the shape of the
    contraction's reshapes) and the skinny CGEMMs of Section 5.1.2."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            hbm, src = float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        hbm, src = 6800.0, "fallback"
    res = {"peak_gbs": hbm, "peak_source": src}

    def entry(bytes_, ms):
        gbs = bytes_ / (ms * 1e-3) / 1e9
        return {"GB/s": gbs, "frac": gbs / hbm, "ms": ms, "bytes": bytes_}

    if "stats" in stages:
        res["exp_stats"] = entry(2 * 8 * n * n, stages["stats"]["ms_per_step"])
        res["exp_stats"]["note"] = "pass 1 over A and B (pass 2 not needed by this input)"
    if "split" in stages:
        # A: 8 B read + 4 FP16 planes (8 B) written; B: 8 B read + 5 planes (10 B)
        res["split"] = entry((8 + 8 + 8 + 10) * n * n, stages["split"]["ms_per_step"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # gather: random permutation of 28 binary indices
    r = 28
    g = torch.Generator(device="cpu").manual_seed(5)
    perm = torch.randperm(r, generator=g).tolist()
    src = torch.empty(2 ** r, dtype=torch.complex64, device=dev)
    out = torch.empty_like(src)
    dims = [2] * r
    strides = [2 ** p for p in perm]
    ms = timed(lambda: q.permute(h, src, dims, strides, out=out))
    res["gather_perm_2^28"] = entry(2 * 8 * 2 ** r, ms)
    del src, out
    # skinny CGEMMs (FP32 path): (2, 2^26, 2) and (2^26, 2, 2)
    N = 2 ** 26
    A = torch.zeros((2, 2), dtype=torch.complex64, device=dev).t()
    B = torch.zeros((N, 2), dtype=torch.complex64, device=dev).t()  # 2 x N column-major
    C = torch.empty((N, 2), dtype=torch.complex64, device=dev).t()   # 2 x N
    ms = timed(lambda: q.cgemm(h, A, B, C, mode="fp32"))
    res["skinny_2xNx2"] = entry(8 * (2 * 2 + 2 * N + 2 * N), ms)
    A2 = torch.zeros((2, N), dtype=torch.complex64, device=dev).t()   # N x 2
    B2 = torch.zeros((2, 2), dtype=torch.complex64, device=dev).t()
    C2 = torch.empty((2, N), dtype=torch.complex64, device=dev).t()   # N x 2
    ms = timed(lambda: q.cgemm(h, A2, B2, C2, mode="fp32"))
    res["skinny_Nx2x2"] = entry(8 * (N * 2 + 4 + N * 2), ms)
    return res


def _finite_or_none(x: float):
    import math

    return x if math.isfinite(x) else None


def sweep_leg(args, q, torch, dev, rank):
    """The whole CGEMM sweep: m = n = k in ``args.sweep_sizes``, parts
    N(0,1) 2^e with e ~ U_int[-s, s] for s in {0, 8, 20, 40}; per point the
    TFLOP/s of FP32 (SIMT), TF32X, FP16X, FP16X_SCALED, AUTO-t (t =
    ``args.tol``, the paper's size rule on) and AUTO-t under the size rule
    measured for the shape (qcs_autotune_gemm) on the same inputs, cuBLAS
    CGEMM (torch, default math mode), the relative Frobenius error of each
    against the FP64 oracle on ``args.sample_rows`` output rows, and the mode
    the device-side selection picks at t in {0, 1e-3, 0.1, 0.5} (statistics
    and selection alone, no size rule)."""
    import numpy as np

    import oracle

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        # one untimed call, then enough calls for ~0.2 s (at least 2)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        first = e0.elapsed_time(e1)
        reps = int(max(2, min(50, 200.0 / max(first, 1e-3))))
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    h = q.Handle(tol=args.tol, size_rule=True)
    ht = q.Handle(tol=args.tol, size_rule=q.SIZE_RULE_TUNED)
    hsel = q.Handle(tol=0.0, size_rule=False)
    rows = args.sample_rows
    points = []
    for n in args.sweep_sizes:
        flops = 8.0 * n * n * n
        for s in (0, 8, 20, 40):
            A = make_operand(torch, n, s, 31 * n + s, dev)
            B = make_operand(torch, n, s, 37 * n + s, dev)
            C = q.fortran_empty(n, n, device=dev)
            pt = {"size": n, "s": s, "modes": {}}
            ref = None
            if rank == 0:
                _, ref, _ = oracle_sample(A[:rows].cpu().numpy().astype(np.complex64),
                                          B.cpu().numpy(), n, rows)
            desc = torch.zeros(4, dtype=torch.int32, device=dev)
            if s == 0:
                ht.autotune_gemm(n, n, n, reps=3)  # the measured size rule for this shape
            for mode in ("fp32", "tf32x", "fp16x", "fp16x_scaled", "auto", "auto_tuned"):
                hh, mm = (ht, "auto") if mode == "auto_tuned" else (h, mode)
                ms = timed(lambda: q.cgemm(hh, A, B, C, mode=mm))
                entry = {"tflops": flops / (ms * 1e-3) / 1e12, "ms": ms}
                if mm == "auto":
                    q.cgemm(hh, A, B, C, mode=mm, desc_out=desc)
                    entry["selected"] = q.MODE_NAME[int(desc[0].item())]
                if rank == 0:
                    got = C[:rows].cpu().numpy().astype(np.complex128)
                    entry["rel_fro_vs_fp64"] = (_finite_or_none(oracle.rel_fro_error(got, ref))
                                                if np.isfinite(got).all() else None)
                pt["modes"][mode] = entry
            ms = timed(lambda: torch.matmul(A, B))
            pt["cublas_cgemm_tflops"] = flops / (ms * 1e-3) / 1e12
            sA, sB = q.exp_stats(hsel, A), q.exp_stats(hsel, B)
            picks = {}
            for t in (0.0, 1e-3, 0.1, 0.5):
                hsel.set_tol(t)
                picks[f"{t:g}"] = q.MODE_NAME[int(q.select(hsel, sA, sB)[0].item())]
            pt["auto_pick_by_tol"] = picks
            fp32 = pt["modes"]["fp32"]
            auto = pt["modes"]["auto"]
            pt["auto_speedup_vs_fp32"] = auto["tflops"] / fp32["tflops"]
            if auto.get("rel_fro_vs_fp64") is not None and fp32.get("rel_fro_vs_fp64"):
                pt["auto_err_ratio_vs_fp32"] = auto["rel_fro_vs_fp64"] / fp32["rel_fro_vs_fp64"]
            points.append(pt)
            del A, B, C
            torch.cuda.empty_cache()
    h.close()
    ht.close()
    hsel.close()
    return {"workload": "CGEMM m=n=k, column-major, alpha=1, beta=0; parts N(0,1)*2^e, "
                        "e~U_int[-s,s] per real scalar; forced modes, AUTO-"
                        f"{args.tol:g} with the paper's size rule and with the size rule "
                        "measured on this GPU (auto_tuned)",
            "error_sample": f"{rows} output rows vs the FP64 oracle",
            "points": points}


def make_line_operand(torch, n: int, s: int, axis: int, seed: int, device):
    """n x n column-major complex64 whose rows (axis 0) or columns (axis 1)
    each carry one binade: parts N(0,1) * 2^e_line, e_line ~ U_int[-s, s]."""
    g = torch.Generator(device=device).manual_seed(seed)
    base = torch.empty((n, n), dtype=torch.complex64, device=device)  # (cols, rows) storage
    re = torch.randn((n, n), generator=g, device=device, dtype=torch.float32)
    im = torch.randn((n, n), generator=g, device=device, dtype=torch.float32)
    f = torch.exp2(torch.randint(-s, s + 1, (n,), generator=g, device=device).float())
    # storage is (column, row): a row of the matrix is a storage column
    f = f[None, :] if axis == 0 else f[:, None]
    base.copy_(torch.complex(re * f, im * f))
    del re, im
    return base.t()


def rowcol_leg(args, q, torch, dev, rank):
    """Per-row / per-column scaling (qcs_set_rowcol_scaling) on line-scaled
    operands: op(A)'s rows and op(B)'s columns N(0,1) * 2^e_line with
    e_line ~ U_int[-30, 30], m = n = k in ``args.rowcol_sizes``.  Section 4.1
    alone selects TF32X here (the lines span 61 binades); with the option
    AUTO-t runs FP16 emulation with line scales.  TFLOP/s and the error
    against the FP64 oracle on ``args.sample_rows`` rows for AUTO-t without
    and with the option and for plain FP32."""
    import numpy as np

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    h = q.Handle(tol=args.tol, size_rule=False)
    hr = q.Handle(tol=args.tol, size_rule=False)
    hr.set_rowcol_scaling(True)
    rows = args.sample_rows
    points = []
    for n in args.rowcol_sizes:
        flops = 8.0 * n * n * n
        A = make_line_operand(torch, n, 30, 0, 41 * n, dev)
        B = make_line_operand(torch, n, 30, 1, 43 * n, dev)
        C = q.fortran_empty(n, n, device=dev)
        ref = None
        if rank == 0:
            _, ref, _ = oracle_sample(A[:rows].cpu().numpy().astype(np.complex64),
                                      B.cpu().numpy(), n, rows)
        pt = {"size": n}
        desc = torch.zeros(4, dtype=torch.int32, device=dev)
        for name, hh, mode in (("auto", h, "auto"), ("auto_rowcol", hr, "auto"),
                               ("fp32", h, "fp32")):
            ms = timed(lambda: q.cgemm(hh, A, B, C, mode=mode))
            q.cgemm(hh, A, B, C, mode=mode, desc_out=desc)
            entry = {"tflops": flops / (ms * 1e-3) / 1e12, "ms": ms,
                     "selected": q.MODE_NAME[int(desc[0].item())]}
            if rank == 0:
                got = C[:rows].cpu().numpy().astype(np.complex128)
                import oracle

                entry["rel_fro_vs_fp64"] = (_finite_or_none(oracle.rel_fro_error(got, ref))
                                            if np.isfinite(got).all() else None)
            pt[name] = entry
        pt["rowcol_speedup_vs_auto"] = pt["auto_rowcol"]["tflops"] / pt["auto"]["tflops"]
        points.append(pt)
        del A, B, C
        torch.cuda.empty_cache()
    h.close()
    hr.close()
    return {"workload": "CGEMM m=n=k, rows of A and columns of B N(0,1)*2^e_line, "
                        f"e_line~U_int[-30,30]; AUTO-{args.tol:g} (size rule off) without and "
                        "with per-row/per-column scaling, and plain FP32",
            "error_sample": f"{rows} output rows vs the FP64 oracle", "points": points}


def sgemm_leg(args, q, torch, dev, rank):
    """Real GEMMs through qcs_sgemm (the SGEMM emulation of Section 2.1):
    m = n = k in ``args.sgemm_sizes``, entries N(0,1) 2^e with e ~ U_int[-s, s]
    for s in {0, 20}; per point the TFLOP/s (2 m n k) of the plain FP32
    kernel, TF32X, FP16X and AUTO-t under the paper's size rule, cuBLAS SGEMM
    through torch (TF32 off), the relative Frobenius error of each against
    the FP64 oracle on ``args.sample_rows`` output rows, and the tensor-core
    work 6 m n k of the FP16X call as a fraction of the sustained bf16 peak
    (the whole call: statistics-free split + tensor-core kernel)."""
    import numpy as np

    import oracle

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        first = e0.elapsed_time(e1)
        reps = int(max(2, min(50, 200.0 / max(first, 1e-3))))
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def operand(n, s, seed):
        g = torch.Generator(device=dev).manual_seed(seed)
        x = torch.randn((n, n), generator=g, device=dev, dtype=torch.float32)
        if s > 0:
            x.mul_(torch.exp2(torch.randint(-s, s + 1, (n, n), generator=g, device=dev).float()))
        return x.t()  # column-major view

    _, sustained, src = peaks()
    h = q.Handle(tol=args.tol, size_rule=True)
    rows = args.sample_rows
    points = []
    allow = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for n in args.sgemm_sizes:
            flops = 2.0 * n * n * n
            for s in (0, 20):
                A = operand(n, s, 41 * n + s)
                B = operand(n, s, 43 * n + s)
                C = q.fortran_empty_real(n, n, device=dev)
                pt = {"size": n, "s": s, "modes": {}}
                ref = None
                if rank == 0:
                    pick = np.random.default_rng(n + s).choice(n, rows, replace=False)
                    At = np.asfortranarray(A[torch.from_numpy(pick).to(dev)].cpu().numpy().T)
                    ref = oracle.sgemm(oracle.OP_T, oracle.OP_N, rows, n, n, 1.0, At,
                                       np.asfortranarray(B.cpu().numpy()))
                desc = torch.zeros(4, dtype=torch.int32, device=dev)
                for mode in ("fp32", "tf32x", "fp16x", "auto"):
                    ms = timed(lambda: q.sgemm(h, A, B, C, mode=mode))
                    entry = {"tflops": flops / (ms * 1e-3) / 1e12, "ms": ms}
                    if mode == "auto":
                        q.sgemm(h, A, B, C, mode=mode, desc_out=desc)
                        entry["selected"] = q.MODE_NAME[int(desc[0].item())]
                    if mode == "fp16x":
                        entry["tensor_frac_of_sustained_bf16"] = (
                            3 * flops / (ms * 1e-3) / 1e12 / sustained)
                    if rank == 0:
                        got = C[torch.from_numpy(pick).to(dev)].cpu().numpy().astype(np.float64)
                        entry["rel_fro_vs_fp64"] = (_finite_or_none(oracle.rel_fro_error(got, ref))
                                                    if np.isfinite(got).all() else None)
                    pt["modes"][mode] = entry
                Ar, Br = A.t().contiguous(), B.t().contiguous()  # row-major copies: C^T = B^T A^T
                ms = timed(lambda: torch.matmul(Br, Ar))
                pt["cublas_sgemm_tflops"] = flops / (ms * 1e-3) / 1e12
                if rank == 0:
                    got = torch.matmul(Br, Ar).t()[torch.from_numpy(pick).to(dev)]
                    pt["cublas_sgemm_rel_fro_vs_fp64"] = _finite_or_none(
                        oracle.rel_fro_error(got.cpu().numpy().astype(np.float64), ref))
                pt["auto_speedup_vs_fp32"] = (pt["modes"]["auto"]["tflops"]
                                              / pt["modes"]["fp32"]["tflops"])
                points.append(pt)
                del A, B, C, Ar, Br
                torch.cuda.empty_cache()
    finally:
        torch.backends.cuda.matmul.allow_tf32 = allow
        h.close()
    return {"workload": "real GEMM m=n=k, column-major, alpha=1, beta=0; entries N(0,1)*2^e, "
                        f"e~U_int[-s,s]; forced modes and AUTO-{args.tol:g} with the paper's "
                        "size rule",
            "flops": "2 m n k",
            "peak_source": src,
            "error_sample": f"{rows} output rows vs the FP64 oracle",
            "points": points}


MODE_KEYS = ["auto", "fp16x", "fp16x_scaled", "tf32x", "fp32", "bf16x3"]


def _time_plan(torch, cp, h, instances=None, reps=1):
    """Seconds per call of qcs_contract_tree (CUDA events), optionally on the
    first ``instances`` instances of the plan only."""
    if instances is not None:
        cp.tree.n_instances = instances
    cp.forward(h)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        out = cp.forward(h)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps * 1e-3, out


def _time_graph(torch, cp, h, reps=2):
    """Seconds per replay of the plan's forward captured in a CUDA graph."""
    g, out = cp.graph(h)
    g.launch()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.launch()
    e1.record()
    torch.cuda.synchronize()
    g.close()
    return e0.elapsed_time(e1) / reps * 1e-3, out


def _gpu_fidelity(q, torch, dev, got, ref):
    """Fidelity, relative L2 and largest absolute error of ``got`` against the
    FP64 reference ``ref`` (complex arrays), summed in FP64 on the GPU
    (qcs_fidelity_stats)."""
    import numpy as np

    h = q.Handle()
    try:
        a = torch.from_numpy(np.ascontiguousarray(np.asarray(got, dtype=np.complex128))).to(dev)
        r = torch.from_numpy(np.ascontiguousarray(np.asarray(ref, dtype=np.complex128))).to(dev)
        return q.fidelity_stats(h, a.reshape(-1), r.reshape(-1))
    finally:
        h.close()


def _routing(info, counts, flops):
    """GEMMs per mode that actually ran in one call, by count and by nominal
    flops: the host-decided modes of qcs_run_info_t, with the AUTO ones
    replaced by what the device selected."""
    host = dict(zip(MODE_KEYS, info["mode_count"]))
    hostf = dict(zip(MODE_KEYS, info["mode_flops"]))
    ran = {k: host[k] + counts.get(k, 0) for k in MODE_KEYS[1:]}
    ranf = {k: hostf[k] + flops.get(k, 0.0) for k in MODE_KEYS[1:]}
    total = max(sum(ran.values()), 1)
    totalf = max(sum(ranf.values()), 1.0)
    return {"gemms": ran, "fraction": {k: round(v / total, 4) for k, v in ran.items()},
            "flops_fraction": {k: round(v / totalf, 4) for k, v in ranf.items()}}


def _contract_variants(args, q, tn, torch, dev, make_plan, ns, variants, full=False):
    """Seconds per instance (slice) of one plan under several (mode, size
    rule, tolerance) variants, each on its own handle: eager calls and a
    CUDA-graph replay of ``ns`` instances, the routing of the GEMMs, for the
    tuned rule the tuning cost and decisions, and with ``full`` the result of
    all instances (``_full``)."""
    res = {}
    for name, mode, rule, tol in variants:
        h = q.Handle(tol=tol, size_rule=rule)
        h.set_instance_batch(args.instance_batch)
        plan = make_plan(q.MODE_BY_NAME[mode])
        cp = tn.CompiledPlan(plan, device=dev)
        n_all = cp.tree.n_instances
        cp.tree.n_instances = ns
        e = {}
        if rule == q.SIZE_RULE_TUNED:
            t0 = time.perf_counter()
            e["shapes_tuned"] = cp.autotune(h, reps=2)
            e["tuning_s"] = time.perf_counter() - t0
            best = {}
            for t in h.tuning():
                best[t["best"]] = best.get(t["best"], 0) + 1
            e["tuned_decisions"] = best
        secs, _ = _time_plan(torch, cp, h)
        h.auto_counts(reset=True)
        out = cp.forward(h)
        counts, cflops = h.auto_counts(reset=True, flops=True)
        info = tn.info_dict(cp.last_info)
        gsecs, gout = _time_graph(torch, cp, h)
        e.update({"s_per_slice": gsecs / ns, "s_per_slice_eager": secs / ns, "slices_timed": ns,
                  "instance_batch": args.instance_batch,
                  "workspace_gb": info["workspace_bytes"] / 1e9,
                  "tflops": info["flops"] / gsecs / 1e12, "gemms_per_slice": info["gemm_count"] / ns,
                  "level_launches_per_slice": info["level_launches"] / ns,
                  "level_gemm_fraction": round(info["level_gemms"] / max(info["gemm_count"], 1), 4),
                  "routing": _routing(info, counts, cflops)})
        if name == variants[0][0] and not args.no_levels:
            # the same variant step by step (one launch sequence per step, plan order)
            h.set_tree_levels(False)
            e["s_per_slice_step_by_step"] = _time_graph(torch, cp, h)[0] / ns
            h.set_tree_levels(True)
        e["_out"] = out.cpu().numpy()
        if full:
            cp.tree.n_instances = n_all
            e["_full"] = cp.forward(h).cpu().numpy()
        res[name] = e
        h.close()
        del cp
        torch.cuda.empty_cache()
    return res


def tree_legs(args, q, torch, dev, rank, world=1, dist=None):
    """The contraction half of the metric (s/slice, AUTO vs all-FP32), the
    plain small-grid amplitudes and the differentiated workload."""
    import numpy as np

    import paper_2303_08989_gb300.tn as tn
    import qcs_inputs as qi

    res = {}
    variants = [("auto", "auto", q.SIZE_RULE_TUNED, args.tol),
                ("auto_t0.5", "auto", q.SIZE_RULE_TUNED, 0.5),
                ("auto_paper_rule", "auto", q.SIZE_RULE_PAPER, args.tol),
                ("fp32", "fp32", q.SIZE_RULE_PAPER, 0.0)]
    # 30-qubit 5x6 grid, depth 14, sliced on 6 indices (64 slices), one bitstring,
    # contracted in the cheapest of --greedy-trials seeded greedy orders
    t0 = time.perf_counter()
    circ, bits, nets, which, order, sliced, seed_used = contraction_network(args, tn, qi)
    net, net_full = nets[which], nets[0]
    planning_s = time.perf_counter() - t0
    plans = {}

    def make_plan(mode):
        plans[mode] = tn.build_plan(net, order, sliced, mode=mode)
        return plans[mode]

    ns = min(args.tree_slices, 64)
    per = _contract_variants(args, q, tn, torch, dev, make_plan, ns, variants, full=True)
    p = plans[q.MODE_AUTO]
    # the FP64 amplitude of this bitstring (oracle state vector, tests/golden)
    ref = None
    gpath = os.path.join(ROOT, "tests", "golden", "grid5x6_d14_amplitudes.txt")
    want = "".join(str(int(v)) for v in bits[0])
    if os.path.exists(gpath):
        with open(gpath) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 3 and parts[0] == want:
                    ref = float(parts[1]) + 1j * float(parts[2])
    for v in per.values():
        v.pop("_out")
        amp = complex(v.pop("_full")[0, 0])
        if ref is not None:
            # |amp - ref| / |ref|, in FP64 on the GPU
            v["amplitude_rel_err_vs_fp64"] = _gpu_fidelity(q, torch, dev, [amp], [ref])["rel_l2_err"]
    res["contraction"] = {
        "workload": "5x6 grid random circuit, depth 14, the cheapest of %d seeded greedy orders "
                    "(seeds 0-%d), 6 sliced indices (64 slices), 1 bitstring; AUTO-%g (measured "
                    "size rule) vs all-FP32, CUDA-graph replays of %d slices; amplitude over all "
                    "64 slices vs the FP64 state vector"
                    % (args.greedy_trials, args.greedy_trials - 1, args.tol, ns),
        "greedy_seed": seed_used, "planning_s": planning_s,
        "single_qubit_gates_absorbed": which == 1, "steps": len(p.steps),
        "slices_total": p.n_instances, "flops_per_slice": p.flops,
        "max_intermediate_log2": p.max_log2_size,
        "auto": per["auto"], "auto_t0.5": per["auto_t0.5"],
        "auto_paper_rule": per["auto_paper_rule"], "fp32": per["fp32"],
        "speedup_vs_fp32": per["fp32"]["s_per_slice"] / per["auto"]["s_per_slice"],
        "speedup_vs_fp32_t0.5": per["fp32"]["s_per_slice"] / per["auto_t0.5"]["s_per_slice"],
    }
    if world > 1:
        res["contraction_sharded"] = sharded_leg(args, q, tn, torch, dev, p, ref, rank, world, dist)
    # the same network in the order of greedy seed 2 alone: 12x the flops per
    # slice, in larger GEMMs (the regime where one large GEMM dominates)
    order2 = tn.greedy_order(net_full, seed=2, skip=[tn.BATCH])
    sliced2 = tn.choose_slices(net_full, order2, n_labels=6, skip=[tn.BATCH])
    plans2 = {}

    def make_plan2(mode):
        plans2[mode] = tn.build_plan(net_full, order2, sliced2, mode=mode)
        return plans2[mode]

    per2 = _contract_variants(args, q, tn, torch, dev, make_plan2, 4,
                              [v for v in variants if v[0] != "auto_paper_rule"])
    for v in per2.values():
        v.pop("_out")
    p2 = plans2[q.MODE_AUTO]
    res["contraction_seed2_order"] = {
        "workload": "the same network in the greedy order of seed 2 alone, 6 sliced indices; "
                    "CUDA-graph replays of 4 slices",
        "flops_per_slice": p2.flops, "max_intermediate_log2": p2.max_log2_size,
        "auto": per2["auto"], "auto_t0.5": per2["auto_t0.5"], "fp32": per2["fp32"],
        "speedup_vs_fp32": per2["fp32"]["s_per_slice"] / per2["auto"]["s_per_slice"],
        "speedup_vs_fp32_t0.5": per2["fp32"]["s_per_slice"] / per2["auto_t0.5"]["s_per_slice"],
    }
    h = q.Handle(tol=args.tol, size_rule=True)
    # plain method, smallest size: 3x4 grid, depth 8, 64 bitstrings (FP32 path by the size rule)
    c0 = qi.random_grid_circuit(3, 4, 8, seed=0)
    b0 = qi.random_bitstrings(12, 64, seed=1)
    p0 = tn.plan_circuit(c0, b0, seed=2, absorb=not args.no_absorb)
    cp0 = tn.CompiledPlan(p0, device=dev)
    secs0, out0 = _time_plan(torch, cp0, h, reps=3)
    secs_g, _ = _time_graph(torch, cp0, h, reps=3)
    # all 64 bitstrings as one group: every step one batched launch
    h.set_instance_batch(64)
    secs_b, out_b = _time_plan(torch, cp0, h, reps=3)
    secs_bg, _ = _time_graph(torch, cp0, h, reps=3)
    res["plain_small"] = {"workload": "3x4 grid, depth 8, 64 bitstrings, greedy order",
                          "s_per_batch": secs0, "s_per_batch_cuda_graph": secs_g,
                          "s_per_batch_grouped": secs_b, "s_per_batch_grouped_cuda_graph": secs_bg,
                          "grouped_bit_identical": bool(torch.equal(out0, out_b)),
                          "gemms": cp0.last_info.gemm_count}
    if rank == 0:
        import oracle

        ref = oracle.sv_amplitudes(c0, b0)
        res["plain_small"]["fidelity_vs_fp64"] = _gpu_fidelity(
            q, torch, dev, out0.cpu().numpy()[:, 0], ref)["fidelity"]
    h.close()
    # differentiation: 4x5 grid, depth 12, free fSim parameters, 256 bitstrings
    c4, b4, p0s, orders, w4 = differentiation_network(args, tn, qi)
    diff = {}
    for mode, rule, which in (("auto", q.SIZE_RULE_TUNED, "seed2"),
                              ("fp32", q.SIZE_RULE_PAPER, "seed2"),
                              ("auto_cheapest_order", q.SIZE_RULE_TUNED, "cheapest"),
                              ("fp32_cheapest_order", q.SIZE_RULE_PAPER, "cheapest")):
        hd = q.Handle(tol=args.tol, size_rule=rule)
        plan, cp, params, fwd_bwd = differentiation_setup(q, tn, torch, dev, hd, c4, b4, p0s,
                                                          orders[which], mode.split("_")[0],
                                                          rule)

        def timed_fwd_bwd():
            fwd_bwd()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            loss = fwd_bwd()
            torch.cuda.synchronize()
            return time.perf_counter() - t0, loss

        t_eager, _ = timed_fwd_bwd()
        # the same as two CUDA-graph replays, the forward grouped over the slices
        hd.set_instance_batch(plan.n_instances)
        cp.use_graphs(hd)
        t_graph, loss = timed_fwd_bwd()
        diff[mode] = {"s_fwd_bwd": t_graph, "s_fwd_bwd_eager": t_eager,
                      "loss": float(loss.item()), "grad": params.grad.double().cpu().numpy()}
        cp.graphed.close()
        hd.close()
    out4 = {"workload": "4x5 grid, depth 12, fSim(theta, phi) ~ U[0, pi], loss sum log|a|^2 "
                        "over 256 bitstrings; open network, 2 sliced indices (4 slices, "
                        "recomputed in the backward); AUTO with the measured size rule; forward "
                        "(grouped) and backward as CUDA-graph replays, eager beside",
            "auto_s": diff["auto"]["s_fwd_bwd"], "fp32_s": diff["fp32"]["s_fwd_bwd"],
            "auto_s_eager": diff["auto"]["s_fwd_bwd_eager"],
            "fp32_s_eager": diff["fp32"]["s_fwd_bwd_eager"],
            "speedup_vs_fp32": diff["fp32"]["s_fwd_bwd"] / diff["auto"]["s_fwd_bwd"],
            "cheapest_order": {"auto_s": diff["auto_cheapest_order"]["s_fwd_bwd"],
                               "fp32_s": diff["fp32_cheapest_order"]["s_fwd_bwd"],
                               "auto_s_eager": diff["auto_cheapest_order"]["s_fwd_bwd_eager"],
                               "fp32_s_eager": diff["fp32_cheapest_order"]["s_fwd_bwd_eager"],
                               "note": "the cheapest of %d seeded greedy orders: 100x and more "
                                       "fewer flops, GEMMs too small for emulation to matter"
                                       % args.greedy_trials,
                               "single_qubit_gates_absorbed": w4 == 1}}
    if rank == 0:
        import oracle

        L_ref, g_ref = oracle.loss_and_grad(c4, b4)
        for mode in ("auto", "fp32", "auto_cheapest_order", "fp32_cheapest_order"):
            g = diff[mode]["grad"]
            out4[f"{mode}_grad_rel_l2_vs_fp64"] = float(np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref))
            out4[f"{mode}_loss_rel_vs_fp64"] = abs(diff[mode]["loss"] - L_ref) / abs(L_ref)
    res["differentiation"] = out4
    res["precision_at_scale"] = scale_leg(args, q, torch, dev, tn, qi, rank)
    return res


def sharded_leg(args, q, tn, torch, dev, plan, ref, rank, world, dist):
    """All 64 slices of the 30-qubit network split over the ranks (Section
    5.3: slices are independent): rank r contracts instances r, r + world, ...
    (tn.shard_plan) as one CUDA-graph replay, then one all-reduce of the
    FP64 output slots (NCCL) gives every rank the amplitude.  Timed from a
    barrier to the end of the all-reduce, max over ranks; seconds per slice
    over all 64 slices; the amplitude against the FP64 state vector."""
    sub = tn.shard_plan(plan, rank, world)
    h = q.Handle(tol=args.tol, size_rule=q.SIZE_RULE_TUNED)
    h.set_instance_batch(args.instance_batch)
    cp = tn.CompiledPlan(sub, device=dev)
    cp.autotune(h, reps=2)
    g, out = cp.graph(h)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for timed in (False, True):
        dist.barrier()
        torch.cuda.synchronize()
        e0.record()
        g.launch()
        tn.allreduce_slots(out)
        e1.record()
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    amp = complex(out[0, 0].item())
    g.close()
    h.close()
    res = {"workload": "5x6 grid, depth 14, 64 slices dealt round-robin over %d ranks, AUTO-%g "
                       "(measured size rule), one graph replay per rank + NCCL all-reduce of the "
                       "FP64 slots" % (world, args.tol),
           "ranks": world, "slices_per_rank": int(sub.n_instances),
           "s_per_slice": float(t.item()) * 1e-3 / plan.n_instances}
    if ref is not None:
        res["amplitude_rel_err_vs_fp64"] = abs(amp - ref) / abs(ref)
    return res


def scale_leg(args, q, torch, dev, tn, qi, rank):
    """40-qubit 5x8 grid, depth 12 (the depth a seeded greedy order slices to
    <= 2^30 with 256 slices), sliced on the 8 indices the oracle chose for its
    FP64 sample: AUTO vs all-FP32 seconds per slice on a sample of slices, the
    fraction of GEMMs routed to each mode, and the four FP64-checked slices."""
    import copy

    import numpy as np

    found = precision_network(args, tn, qi)
    if found is None:
        return {"skipped": "tests/golden/slices5x8_d12.txt missing"}
    labels, rows, circ, bits, nets, which, order, seed_used = found
    net = nets[which]
    plans = {}

    def make_plan(mode):
        plans[mode] = tn.build_plan(net, order, labels, mode=mode)
        return plans[mode]

    variants = [("auto", "auto", q.SIZE_RULE_TUNED, args.tol),
                ("auto_t0.5", "auto", q.SIZE_RULE_TUNED, 0.5),
                ("fp32", "fp32", q.SIZE_RULE_PAPER, 0.0)]
    per = _contract_variants(args, q, tn, torch, dev, make_plan, 16, variants)
    plan = plans[q.MODE_AUTO]
    out = {"workload": "5x8 grid (40 qubits), depth 12, 8 sliced indices (256 slices), the "
                       "cheapest of %d seeded greedy orders of the sliced network, 1 bitstring; "
                       "AUTO-%g (measured size rule) vs all-FP32, CUDA-graph replays of 16 "
                       "slices" % (args.greedy_trials, args.tol),
           "greedy_seed": seed_used, "single_qubit_gates_absorbed": which == 1,
           "steps": len(plan.steps),
           "flops_per_slice": plan.flops, "max_intermediate_log2": plan.max_log2_size}
    idx = [int(v, 2) for v, _ in rows]
    sub = copy.copy(plan)
    sub.instance_offset = np.ascontiguousarray(plan.instance_offset[idx])
    sub.instance_slot = np.arange(len(idx), dtype=np.int32)
    sub.n_slots = len(idx)
    cps = tn.CompiledPlan(sub, device=dev)
    for tol, key in ((args.tol, ""), (0.5, "_t0.5")):
        h = q.Handle(tol=tol, size_rule=q.SIZE_RULE_TUNED)
        cps.autotune(h, reps=2)
        got = cps.forward(h).cpu().numpy()[:, 0]
        h.close()
        if rank == 0:
            ref = np.array([a for _, a in rows])
            fs = _gpu_fidelity(q, torch, dev, got, ref)
            out["sampled_slices_fidelity_vs_fp64" + key] = fs["fidelity"]
            out["sampled_slices_max_rel_err_vs_fp64" + key] = float(
                np.max(np.abs(got - ref) / np.abs(ref)))
    b = per["fp32"]["_out"][0, 0]
    for v in per.values():
        a = v.pop("_out")[0, 0]
        v["partial_sum_rel_diff_vs_fp32"] = float(abs(a - b) / abs(b))
    out["auto"], out["auto_t0.5"], out["fp32"] = per["auto"], per["auto_t0.5"], per["fp32"]
    out["speedup_vs_fp32"] = per["fp32"]["s_per_slice"] / per["auto"]["s_per_slice"]
    out["speedup_vs_fp32_t0.5"] = per["fp32"]["s_per_slice"] / per["auto_t0.5"]["s_per_slice"]
    return out


if __name__ == "__main__":
    main()
