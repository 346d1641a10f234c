"""Tensor-network planning for qcs_contract_tree (host side).

circuit -> tensor network (Section 2.2: |0> and <x| as rank-1 tensors, a
k-qubit gate as a rank-2k tensor, wires as shared indices) -> seeded greedy
contraction order -> slicing (Section 5.3: fixed values of chosen indices,
results summed) -> a TTGT plan (Section 1: each pairwise contraction
reshaped to one CGEMM) that libqcs executes.  Nothing numerical happens here
beyond building the leaf tensors; every contraction runs in the CUDA library.

Storage convention: every tensor is stored first-index-fastest (Fortran
order) over its label list; a tensor whose labels are (M..., K...) is the
column-major M x K matrix.

Instances.  Sliced indices and the bitstring index of a batch of closed
amplitudes are "instance labels": they are not contracted; each instance
fixes their values, which moves each leaf's base by a constant offset, and
the executor adds the root of every instance into its output slot (one slot
per bitstring; the slices of a bitstring share it).
"""
from __future__ import annotations

import ctypes
import heapq
import itertools
import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import _lib

BATCH = -1  # label of the bitstring index of batched <x| leaves


@dataclass
class Leaf:
    data: np.ndarray          # complex64, 1-D, first-index-fastest over ``labels``
    labels: List[int]
    dims: List[int]
    kind: str = "gate"        # "init", "gate", "final"
    gate: int = -1            # index of the gate in the circuit, for gate leaves


@dataclass
class Network:
    leaves: List[Leaf]
    output: List[int]         # open labels, in the order of the returned result
    dims: Dict[int, int]
    batch: int = 0            # number of bitstrings in the BATCH label (0: none)


def _fortran_flat(t: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(t).ravel(order="F")).astype(np.complex64)


def circuit_network(circ, bitstrings: Optional[np.ndarray] = None) -> Network:
    """The network of <x|U|0> for a circuit (qcs_inputs.Circuit).

    bitstrings None: output legs open (the result is the state U|0>, ordered
    as numpy's C order over qubits 0..n-1).  Otherwise a (B, n) array: the <x|
    leaves carry the BATCH label with one column per bitstring.
    """
    n = circ.n_qubits
    leaves: List[Leaf] = []
    dims: Dict[int, int] = {}
    wire = list(range(n))
    for q in range(n):
        dims[q] = 2
        leaves.append(Leaf(np.array([1, 0], np.complex64), [q], [2], "init"))
    nxt = n
    for gi, g in enumerate(circ.gates):
        k = len(g.qubits)
        new = list(range(nxt, nxt + k))
        nxt += k
        for l in new:
            dims[l] = 2
        t = np.asarray(g.matrix, dtype=np.complex128).reshape((2,) * (2 * k))
        labels = new + [wire[q] for q in g.qubits]
        leaves.append(Leaf(_fortran_flat(t), labels, [2] * (2 * k), "gate", gi))
        for i, q in enumerate(g.qubits):
            wire[q] = new[i]
    if bitstrings is None:
        return Network(leaves, [wire[q] for q in range(n)], dims)
    bs = np.asarray(bitstrings, dtype=np.int64).reshape(-1, n)
    B = bs.shape[0]
    dims[BATCH] = B
    for q in range(n):
        v = np.zeros((2, B), np.complex64)
        v[bs[:, q], np.arange(B)] = 1.0
        leaves.append(Leaf(_fortran_flat(v), [wire[q], BATCH], [2, B], "final"))
    return Network(leaves, [], dims, batch=B)


def _merge_gate(T: Leaf, g: Leaf, elim: int) -> Leaf:
    """T contracted with the single-qubit gate leaf g (labels [out, in]) over
    label ``elim`` of T: elim = in (T produces the gate's input) gives
    T'[..., out, ...] = sum_in g[out, in] T[..., in, ...]; elim = out (T
    consumes its output) gives T'[..., in, ...] = sum_out T[..., out, ...]
    g[out, in].  The label keeps its position; arithmetic in complex128."""
    out_l, in_l = g.labels
    G = g.data.astype(np.complex128).reshape((2, 2), order="F")  # G[out, in]
    t = T.data.astype(np.complex128).reshape(T.dims, order="F")
    ax = T.labels.index(elim)
    if elim == in_l:
        t = np.moveaxis(np.tensordot(G, t, axes=([1], [ax])), 0, ax)
        new = out_l
    else:
        t = np.moveaxis(np.tensordot(G, t, axes=([0], [ax])), 0, ax)
        new = in_l
    labels = list(T.labels)
    labels[ax] = new
    return Leaf(_fortran_flat(t), labels, list(T.dims), T.kind, T.gate)


def absorb_single_qubit_gates(net: Network, frozen_gates: Sequence[int] = (),
                              keep_labels: Sequence[int] = ()) -> Network:
    """The same network with every single-qubit gate contracted, on the host,
    into the tensor that produces its input wire (or, when that is not
    allowed, the tensor that consumes its output): chains of single-qubit
    gates between two multi-qubit gates become part of the multi-qubit gate's
    tensor, and those at the start of a wire part of its |0> leaf.  The tree
    then has none of the (2, 2^N, 2)-shaped steps that contract a 2 x 2 gate
    into a large intermediate.  ``frozen_gates``: circuit gate indices whose
    leaves must stay as they are (parametric gates of a differentiated
    circuit); ``keep_labels``: labels that must survive (e.g. sliced
    indices; output and bitstring labels always do).  Exact up to complex64
    rounding of the merged tensors."""
    leaves = [Leaf(lf.data.copy(), list(lf.labels), list(lf.dims), lf.kind, lf.gate)
              for lf in net.leaves]
    frozen = set(frozen_gates)
    keep = set(keep_labels) | set(net.output) | {BATCH}
    alive = [True] * len(leaves)
    holders: Dict[int, set] = {}
    for i, lf in enumerate(leaves):
        for l in lf.labels:
            holders.setdefault(l, set()).add(i)

    def other(label, i):
        h = [j for j in holders.get(label, ()) if j != i and alive[j]]
        return h[0] if h else None

    def mutable(j):
        return not (leaves[j].kind == "gate" and leaves[j].gate in frozen)

    for i, lf in enumerate(leaves):
        if not (lf.kind == "gate" and len(lf.labels) == 2 and lf.gate not in frozen):
            continue
        out_l, in_l = lf.labels
        p, c = other(in_l, i), other(out_l, i)
        if p is not None and in_l not in keep and mutable(p):
            tgt, elim, new = p, in_l, out_l
        elif c is not None and out_l not in keep and mutable(c):
            tgt, elim, new = c, out_l, in_l
        else:
            continue
        leaves[tgt] = _merge_gate(leaves[tgt], lf, elim)
        holders[elim].discard(tgt)
        holders[elim].discard(i)
        holders[new].discard(i)
        holders[new].add(tgt)
        alive[i] = False
    return Network([lf for lf, a in zip(leaves, alive) if a], list(net.output), dict(net.dims),
                   net.batch)


# ---------------------------------------------------------------------------
# contraction order
# ---------------------------------------------------------------------------

def greedy_order(net: Network, seed: int = 2, skip: Sequence[int] = ()) -> List[Tuple[int, int]]:
    """Seeded greedy order: repeatedly contract the connected pair with the
    smallest size(result) - size(a) - size(b) (log-sizes, a random jitter
    breaks ties).  Labels in ``skip`` (instance labels) are ignored.
    Returns SSA pairs: tensor ids, each contraction appending a new id."""
    rng = np.random.default_rng(seed)
    skip = set(skip)
    labs: List[frozenset] = [frozenset(l for l in lf.labels if l not in skip) for lf in net.leaves]
    keep = set(net.output)
    count: Dict[int, int] = {}
    where: Dict[int, set] = {}
    for i, ls in enumerate(labs):
        for l in ls:
            count[l] = count.get(l, 0) + 1
            where.setdefault(l, set()).add(i)
    alive = set(range(len(labs)))
    logd = {l: math.log2(d) for l, d in net.dims.items()}

    def lsize(ls):
        return sum(logd[l] for l in ls)

    def result(i, j):
        a, b = labs[i], labs[j]
        return frozenset(l for l in a | b
                         if not (l in a and l in b and count[l] == 2 and l not in keep))

    def score(i, j):
        r = result(i, j)
        return (2.0 ** lsize(r) - 2.0 ** lsize(labs[i]) - 2.0 ** lsize(labs[j])) \
            * (1.0 + 1e-6 * rng.random()), r

    heap = []
    for l, ws in where.items():
        for i, j in itertools.combinations(sorted(ws), 2):
            sc, _ = score(i, j)
            heapq.heappush(heap, (sc, i, j))
    order = []
    while len(alive) > 1:
        pair = None
        while heap:
            sc, i, j = heapq.heappop(heap)
            if i in alive and j in alive:
                pair = (i, j)
                break
        if pair is None:  # disconnected components: join the two smallest
            i, j = sorted(alive, key=lambda u: (lsize(labs[u]), u))[:2]
            pair = (min(i, j), max(i, j))
        i, j = pair
        r = result(i, j)
        for u in (i, j):
            for l in labs[u]:
                count[l] -= 1
                where[l].discard(u)
            alive.discard(u)
        new = len(labs)
        labs.append(r)
        for l in r:
            count[l] = count.get(l, 0) + 1
            where.setdefault(l, set()).add(new)
        alive.add(new)
        order.append((i, j))
        nb = set()
        for l in r:
            nb |= where[l]
        nb.discard(new)
        for u in nb:
            sc, _ = score(min(u, new), max(u, new))
            heapq.heappush(heap, (sc, min(u, new), max(u, new)))
    return order


def intermediates(net: Network, order, skip: Sequence[int] = ()) -> List[frozenset]:
    """Label sets of every intermediate of an SSA order (instance labels removed)."""
    skip = set(skip)
    labs = [frozenset(l for l in lf.labels if l not in skip) for lf in net.leaves]
    count: Dict[int, int] = {}
    for ls in labs:
        for l in ls:
            count[l] = count.get(l, 0) + 1
    keep = set(net.output)
    out = []
    for i, j in order:
        a, b = labs[i], labs[j]
        r = frozenset(l for l in a | b if not (l in a and l in b and count[l] == 2 and l not in keep))
        for l in a:
            count[l] -= 1
        for l in b:
            count[l] -= 1
        for l in r:
            count[l] = count.get(l, 0) + 1
        labs.append(r)
        out.append(r)
    return out


def choose_slices(net: Network, order, n_labels: Optional[int] = None,
                  max_log2_size: Optional[float] = None, skip: Sequence[int] = ()) -> List[int]:
    """Pick indices to slice (Section 5.3): repeatedly the index that
    removes the most work -- the one carried by the largest intermediates,
    weighted by their sizes -- until ``n_labels`` are chosen or the largest
    intermediate is at most 2**max_log2_size elements."""
    sliced: List[int] = []
    keep = set(net.output) | set(skip)
    while True:
        inter = intermediates(net, order, list(skip) + sliced)
        logs = [sum(math.log2(net.dims[l]) for l in r) for r in inter]
        biggest = max(logs) if logs else 0.0
        if n_labels is not None and len(sliced) >= n_labels:
            break
        if n_labels is None and (max_log2_size is None or biggest <= max_log2_size):
            break
        weight: Dict[int, float] = {}
        for r, lg in zip(inter, logs):
            if lg < biggest - 2:
                continue
            for l in r:
                if l not in keep:
                    weight[l] = weight.get(l, 0.0) + 2.0 ** (lg - biggest)
        if not weight:
            break
        sliced.append(min(weight, key=lambda l: (-weight[l], l)))
    return sliced


def order_cost(net: Network, order, skip: Sequence[int] = ()) -> Tuple[float, float]:
    """(flops, log2 of the largest intermediate) of one instance of an SSA
    order with the labels in ``skip`` fixed: each pairwise contraction costs
    8 x the product of the dims of all its labels (the CGEMM's 8 m n k)."""
    skip = set(skip)
    labs = [frozenset(l for l in lf.labels if l not in skip) for lf in net.leaves]
    logd = {l: math.log2(d) for l, d in net.dims.items()}
    flops, big = 0.0, 0.0
    for r, (i, j) in zip(intermediates(net, order, skip), order):
        labs.append(r)
        flops += 8.0 * 2.0 ** sum(logd[l] for l in labs[i] | labs[j])
        big = max(big, sum(logd[l] for l in r))
    return flops, big


def _seeded_order(net: Network, seed: int, skip, n_slices: int, max_log2_size):
    order = greedy_order(net, seed=seed, skip=skip)
    sliced = []
    if n_slices or max_log2_size is not None:
        sliced = choose_slices(net, order, n_labels=n_slices or None,
                               max_log2_size=max_log2_size, skip=skip)
    return order, sliced


def _seed_keys(net: Network, seeds: Sequence[int], skip, n_slices: int, max_log2_size):
    """(flops per instance, largest intermediate, seed) of each seeded order."""
    keys = []
    for seed in seeds:
        order, sliced = _seeded_order(net, seed, skip, n_slices, max_log2_size)
        flops, big = order_cost(net, order, list(skip) + sliced)
        keys.append((flops, big, seed))
    return keys


def best_greedy_order(net: Network, seeds: Sequence[int], skip: Sequence[int] = (),
                      n_slices: int = 0, max_log2_size: Optional[float] = None,
                      workers: int = 1):
    """The seeded greedy order (and its slicing) with the fewest flops per
    instance over ``seeds``; ties go to the smaller largest intermediate, then
    the smaller seed.  The greedy choice breaks ties between equal scores at
    random, and on grid circuits the seed alone moves the cost of a slice by
    10x and more.  ``workers`` > 1 costs the seeds in that many worker
    processes (started with spawn, so a process that already uses CUDA can
    call it); the result is the same.  Returns (order, sliced labels, seed)."""
    seeds = list(seeds)
    skip = list(skip)
    if workers > 1 and len(seeds) > 1:
        import concurrent.futures as cf
        import multiprocessing as mp

        chunks = [seeds[i::workers] for i in range(workers) if seeds[i::workers]]
        with cf.ProcessPoolExecutor(max_workers=len(chunks),
                                    mp_context=mp.get_context("spawn")) as ex:
            futs = [ex.submit(_seed_keys, net, c, skip, n_slices, max_log2_size) for c in chunks]
            keys = [k for f in futs for k in f.result()]
    else:
        keys = _seed_keys(net, seeds, skip, n_slices, max_log2_size)
    seed = min(keys)[2]
    order, sliced = _seeded_order(net, seed, skip, n_slices, max_log2_size)
    return order, sliced, seed


# ---------------------------------------------------------------------------
# TTGT plan
# ---------------------------------------------------------------------------

def _fortran_strides(dims: Sequence[int]) -> List[int]:
    st, acc = [], 1
    for d in dims:
        st.append(acc)
        acc *= d
    return st


def _compress(dims: List[int], strides: List[int]) -> Tuple[List[int], List[int]]:
    """Merge adjacent dims that are contiguous in the source; drop size 1."""
    od, os_ = [], []
    for d, s in zip(dims, strides):
        if d == 1:
            continue
        if od and os_[-1] * od[-1] == s:
            od[-1] *= d
        else:
            od.append(d)
            os_.append(s)
    return od, os_


@dataclass
class Step:
    a: int
    b: int
    direct_a: int
    direct_b: int
    m: int
    n: int
    k: int
    map_a: Tuple[List[int], List[int]]
    map_b: Tuple[List[int], List[int]]
    labels_out: List[int]
    mode: int = 0


@dataclass
class Plan:
    net: Network
    steps: List[Step]
    sliced: List[int]
    instance_offset: np.ndarray   # (n_instances, n_leaves) int64
    instance_slot: np.ndarray     # (n_instances,) int32
    n_slots: int
    out_size: int
    out_index: Optional[np.ndarray]
    root_labels: List[int]
    max_log2_size: float = 0.0
    flops: float = 0.0

    @property
    def n_instances(self) -> int:
        return int(self.instance_slot.shape[0])


def build_plan(net: Network, order, sliced: Sequence[int] = (), mode: int = 0,
               outputs: Optional[np.ndarray] = None) -> Plan:
    """Turn an SSA order into executor steps.

    outputs: for an open network, an optional (B, n_out) array of values of
    the output labels to gather (e.g. bitstrings); default: the whole
    result in numpy C order over ``net.output``.
    """
    sliced = list(sliced)
    inst = set(sliced) | ({BATCH} if net.batch else set())
    nl = len(net.leaves)
    labels: List[List[int]] = [list(lf.labels) for lf in net.leaves]   # storage labels
    strides: List[Dict[int, int]] = [dict(zip(lf.labels, _fortran_strides(lf.dims)))
                                     for lf in net.leaves]
    contiguous = [not (set(lf.labels) & inst) for lf in net.leaves]
    count: Dict[int, int] = {}
    for ls in labels:
        for l in ls:
            if l not in inst:
                count[l] = count.get(l, 0) + 1
    keep = set(net.output)
    steps: List[Step] = []
    max_log2 = 0.0
    flops = 0.0
    for (i, j) in order:
        la = [l for l in labels[i] if l not in inst]
        lb = [l for l in labels[j] if l not in inst]
        shared = [l for l in la if l in lb]
        hyper = [l for l in shared if count[l] > 2 or l in keep]
        if hyper:
            raise ValueError(f"hyperedge labels {hyper} are not supported")
        K_a = shared
        K_b = [l for l in lb if l in shared]
        M = [l for l in la if l not in shared]
        N = [l for l in lb if l not in shared]
        a_dir = {"N": contiguous[i] and la == M + K_a, "T": contiguous[i] and la == K_a + M}
        b_dir = {"N": contiguous[j] and lb == K_b + N, "T": contiguous[j] and lb == N + K_b}
        if (a_dir["N"] or a_dir["T"]):
            K = K_a
            if K_b != K:
                b_dir = {"N": False, "T": False}
        elif (b_dir["N"] or b_dir["T"]):
            K = K_b
        else:
            K = K_a
            b_dir = {"N": contiguous[j] and lb == K + N, "T": contiguous[j] and lb == N + K}
        d = net.dims
        m = int(np.prod([d[l] for l in M], dtype=np.int64)) if M else 1
        n = int(np.prod([d[l] for l in N], dtype=np.int64)) if N else 1
        k = int(np.prod([d[l] for l in K], dtype=np.int64)) if K else 1
        map_a = _compress([d[l] for l in M + K], [strides[i][l] for l in M + K])
        map_b = _compress([d[l] for l in K + N], [strides[j][l] for l in K + N])
        if len(map_a[0]) > _lib.MAX_RANK or len(map_b[0]) > _lib.MAX_RANK:
            raise ValueError("operand rank beyond QCS_MAX_RANK after compression")
        direct_a = 0 if a_dir["N"] else (1 if a_dir["T"] else -1)
        direct_b = 0 if b_dir["N"] else (1 if b_dir["T"] else -1)
        out_labels = M + N
        steps.append(Step(i, j, direct_a, direct_b, m, n, k, map_a, map_b, out_labels, mode))
        for l in la + lb:
            count[l] -= 1
        for l in out_labels:
            count[l] = count.get(l, 0) + 1
        labels.append(out_labels)
        strides.append(dict(zip(out_labels, _fortran_strides([d[l] for l in out_labels]))))
        contiguous.append(True)
        max_log2 = max(max_log2, math.log2(m * n))
        flops += 8.0 * m * n * k
    root = len(labels) - 1 if order else 0
    root_labels = [l for l in labels[root] if l not in inst]
    if sorted(root_labels) != sorted(net.output):
        raise ValueError("the order does not contract the network to its output labels")
    rs = strides[root]
    if net.output:
        if outputs is None:
            nout = len(net.output)
            vals = np.array(list(itertools.product(*[range(net.dims[l]) for l in net.output])),
                            dtype=np.int64).reshape(-1, nout)
        else:
            vals = np.asarray(outputs, dtype=np.int64)
        out_index = vals @ np.array([rs[l] for l in net.output], dtype=np.int64)
        out_size = int(out_index.shape[0])
    else:
        out_index = None
        out_size = 1
    # instances: bitstring x slice assignment
    slice_vals = list(itertools.product(*[range(net.dims[l]) for l in sliced])) or [()]
    B = net.batch if net.batch else 1
    offs = np.zeros((B * len(slice_vals), nl), dtype=np.int64)
    slots = np.zeros(B * len(slice_vals), dtype=np.int32)
    leaf_strides = strides[:nl]
    r = 0
    for b in range(B):
        for sv in slice_vals:
            val = dict(zip(sliced, sv))
            if net.batch:
                val[BATCH] = b
            for li in range(nl):
                offs[r, li] = sum(val[l] * leaf_strides[li][l] for l in net.leaves[li].labels
                                  if l in val)
            slots[r] = b
            r += 1
    return Plan(net, steps, sliced, offs, slots, B, out_size, out_index, root_labels,
                max_log2, flops)


# ---------------------------------------------------------------------------
# device side: leaves, ctypes plan, forward / backward through libqcs
# ---------------------------------------------------------------------------

class CompiledPlan:
    """A plan marshalled into qcs_tree_t, with its leaves on the device."""

    def __init__(self, plan: Plan, device="cuda", leaf_data: Optional[List] = None):
        import torch

        self.plan = plan
        self.device = torch.device(device)
        L = _lib
        steps = (L.qcs_step_t * max(len(plan.steps), 1))()
        for s, st in enumerate(plan.steps):
            c = steps[s]
            c.a, c.b, c.direct_a, c.direct_b = st.a, st.b, st.direct_a, st.direct_b
            c.m, c.n, c.k, c.mode = st.m, st.n, st.k, st.mode
            for mp, dst in ((st.map_a, c.map_a), (st.map_b, c.map_b)):
                dst.rank = len(mp[0])
                for q, (dd, ss) in enumerate(zip(*mp)):
                    dst.dims[q] = dd
                    dst.strides[q] = ss
        self._steps = steps
        nl = len(plan.net.leaves)
        self._leaf_size = (ctypes.c_int64 * nl)(*[lf.data.size for lf in plan.net.leaves])
        offs = np.ascontiguousarray(plan.instance_offset.reshape(-1), dtype=np.int64)
        self._offs = offs
        slots = np.ascontiguousarray(plan.instance_slot, dtype=np.int32)
        self._slots = slots
        self._out_index = (np.ascontiguousarray(plan.out_index, dtype=np.int64)
                           if plan.out_index is not None else None)
        t = L.qcs_tree_t()
        t.n_leaves = nl
        t.n_steps = len(plan.steps)
        t.n_instances = plan.n_instances
        t.n_slots = plan.n_slots
        t.leaf_size = self._leaf_size
        t.instance_offset = offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
        t.instance_slot = slots.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        t.steps = steps
        t.out_size = plan.out_size
        t.out_index = (self._out_index.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
                       if self._out_index is not None else None)
        self.tree = t
        if leaf_data is None:
            leaf_data = [torch.from_numpy(lf.data).to(self.device) for lf in plan.net.leaves]
        self.leaves = leaf_data

    def _ptrs(self, tensors):
        return (ctypes.c_void_p * len(tensors))(*[ctypes.c_void_p(t.data_ptr()) for t in tensors])

    def forward(self, h, leaves=None):
        """Contract every instance; returns complex128 (n_slots, out_size)."""
        import torch

        leaves = self.leaves if leaves is None else leaves
        out = torch.empty((self.plan.n_slots, self.plan.out_size), dtype=torch.complex128,
                          device=self.device)
        info = _lib.qcs_run_info_t()
        ptrs = self._ptrs([t.contiguous() for t in leaves])
        _lib.check(h.lib.qcs_contract_tree(h.ptr, ctypes.byref(self.tree), ptrs,
                                           ctypes.c_void_p(out.data_ptr()), ctypes.byref(info)),
                   "qcs_contract_tree")
        self.last_info = info
        return out

    def graph(self, h, out=None):
        """Capture this plan's forward call into a CUDA graph (qcs_tree_graph_*);
        returns (graph, out).  ``graph.launch()`` recomputes ``out`` from the
        current contents of ``self.leaves``."""
        import torch

        if out is None:
            out = torch.empty((self.plan.n_slots, self.plan.out_size), dtype=torch.complex128,
                              device=self.device)
        g = TreeGraph(h, self, out)
        return g, out

    def backward(self, h, grad_out, leaves=None):
        """Leaf gradients (list of complex64 tensors) for dL/d out = grad_out
        (torch convention: dL/dRe + i dL/dIm)."""
        import torch

        leaves = [t.contiguous() for t in (self.leaves if leaves is None else leaves)]
        # every leaf gradient is a slice of one zeroed buffer (one memset)
        sizes = [t.numel() for t in leaves]
        grads = list(torch.zeros(sum(sizes), dtype=torch.complex64,
                                 device=self.device).split(sizes))
        g = grad_out.to(torch.complex128).contiguous()
        info = _lib.qcs_run_info_t()
        _lib.check(h.lib.qcs_contract_tree_backward(
            h.ptr, ctypes.byref(self.tree), self._ptrs(leaves), ctypes.c_void_p(g.data_ptr()),
            self._ptrs(grads), ctypes.byref(info)), "qcs_contract_tree_backward")
        self.last_info = info
        return grads

    def use_graphs(self, h):
        """From now on, contract() runs this plan's forward and backward as two
        CUDA-graph replays on ``h`` (GraphedPlan) instead of launching every
        kernel from the host.  Call after any autotuning and with the
        instance batch already set; returns the GraphedPlan."""
        self.graphed = GraphedPlan(self, h)
        return self.graphed

    def autotune(self, h, backward: bool = False, reps: int = 3) -> int:
        """Time the candidate modes of every AUTO GEMM shape this plan issues
        (qcs_autotune_tree) and record them in ``h``'s table; returns the
        number of shapes timed.  Use with ``h.set_size_rule(SIZE_RULE_TUNED)``."""
        n = ctypes.c_int64()
        _lib.check(h.lib.qcs_autotune_tree(h.ptr, ctypes.byref(self.tree), 1 if backward else 0,
                                           int(reps), ctypes.byref(n)), "qcs_autotune_tree")
        return int(n.value)


class TreeGraph:
    """An instantiated CUDA graph of one plan's forward call."""

    def __init__(self, h, cp: CompiledPlan, out):
        self.h = h
        self.cp = cp
        self.out = out
        self._leaves = [t.contiguous() for t in cp.leaves]
        self._ptrs = cp._ptrs(self._leaves)
        self._g = ctypes.c_void_p()
        _lib.check(h.lib.qcs_tree_graph_create(h.ptr, ctypes.byref(cp.tree), self._ptrs,
                                               ctypes.c_void_p(out.data_ptr()),
                                               ctypes.byref(self._g)), "qcs_tree_graph_create")

    def launch(self):
        _lib.check(self.h.lib.qcs_tree_graph_launch(self._g), "qcs_tree_graph_launch")
        return self.out

    def close(self):
        if self._g:
            self.h.lib.qcs_tree_graph_destroy(self._g)
            self._g = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GraphedPlan:
    """A plan's forward and backward captured as two CUDA graphs over
    persistent device buffers: the leaves packed into one buffer, the output,
    the output gradient and the packed leaf gradients.  ``forward(leaves)``
    copies the leaves in (one kernel) and replays the forward graph;
    ``backward(leaves, grad_out)`` copies the leaves and the output gradient
    in, clears the gradients and replays the backward graph.  Both return
    fresh tensors, so the buffers may be reused by the next call."""

    def __init__(self, cp: "CompiledPlan", h):
        import torch

        self.cp, self.h = cp, h
        plan, dev = cp.plan, cp.device
        self.sizes = [lf.data.size for lf in plan.net.leaves]
        self.leaf_buf = torch.zeros(sum(self.sizes), dtype=torch.complex64, device=dev)
        self.grad_buf = torch.zeros_like(self.leaf_buf)
        self.leaves = list(self.leaf_buf.split(self.sizes))
        self.grads = list(self.grad_buf.split(self.sizes))
        self.out = torch.zeros((plan.n_slots, plan.out_size), dtype=torch.complex128, device=dev)
        self.gout = torch.zeros_like(self.out)
        lp, gp = cp._ptrs(self.leaves), cp._ptrs(self.grads)
        self._keep = (lp, gp)
        self._fwd, self._bwd = ctypes.c_void_p(), ctypes.c_void_p()
        _lib.check(h.lib.qcs_tree_graph_create(h.ptr, ctypes.byref(cp.tree), lp,
                                               ctypes.c_void_p(self.out.data_ptr()),
                                               ctypes.byref(self._fwd)), "qcs_tree_graph_create")
        _lib.check(h.lib.qcs_tree_backward_graph_create(
            h.ptr, ctypes.byref(cp.tree), lp, ctypes.c_void_p(self.gout.data_ptr()), gp,
            ctypes.byref(self._bwd)), "qcs_tree_backward_graph_create")

    def _load(self, leaves):
        import torch

        torch.cat([t.reshape(-1) for t in leaves], out=self.leaf_buf)

    def forward(self, leaves):
        self._load(leaves)
        _lib.check(self.h.lib.qcs_tree_graph_launch(self._fwd), "qcs_tree_graph_launch")
        return self.out.clone()

    def backward(self, leaves, grad_out):
        self._load(leaves)
        self.gout.copy_(grad_out)
        self.grad_buf.zero_()
        _lib.check(self.h.lib.qcs_tree_graph_launch(self._bwd), "qcs_tree_graph_launch")
        return list(self.grad_buf.clone().split(self.sizes))

    def close(self):
        for g in ("_fwd", "_bwd"):
            if getattr(self, g, None):
                self.h.lib.qcs_tree_graph_destroy(getattr(self, g))
                setattr(self, g, ctypes.c_void_p())

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def info_dict(info) -> dict:
    return {"seconds": info.seconds, "gemm_count": info.gemm_count,
            "gather_count": info.gather_count, "mode_count": list(info.mode_count),
            "workspace_bytes": info.workspace_bytes, "flops": info.flops,
            "mode_flops": list(info.mode_flops), "level_launches": info.level_launches,
            "level_gemms": info.level_gemms}


# ---------------------------------------------------------------------------
# differentiation: torch.autograd.Function over qcs_contract_tree
# ---------------------------------------------------------------------------

def _torch_fsim_leaves(theta, phi):
    """First-index-fastest flat complex64 fSim(theta_g, phi_g) tensors, one row
    per gate (shape (n, 16)), built with a handful of batched torch ops so
    that autograd reaches theta and phi."""
    import torch

    c = torch.cos(theta).to(torch.complex64)
    s = torch.sin(theta).to(torch.complex64)
    e = torch.exp(-1j * phi.to(torch.complex64))
    one = torch.ones_like(c)
    zero = torch.zeros_like(c)
    G = torch.stack([one, zero, zero, zero,
                     zero, c, -1j * s, zero,
                     zero, -1j * s, c, zero,
                     zero, zero, zero, e], dim=-1)  # (n, 16): row-major 4 x 4
    return G.reshape(-1, 2, 2, 2, 2).permute(0, 4, 3, 2, 1).reshape(-1, 16)


def torch_leaves(net: Network, circ, params, device="cuda"):
    """Device leaf tensors of ``net``; the fSim leaves are functions of
    ``params`` ((n_fsim, 2) real tensor: theta, phi per fSim gate in circuit
    order), every other leaf is constant.  The fSim leaves come from one
    batched evaluation (rows of one tensor).  The constant ones come from one
    host-to-device copy, made on the first call for a (network, circuit,
    device) and kept on the network for later calls, with the index rows of
    the fSim gates; replacing ``net.leaves`` drops the kept copy."""
    import torch

    key = (id(circ), str(torch.device(device)), str(params.device))
    kept = net.__dict__.get("_torch_leaf_cache")
    if kept is None or kept[0] != key or kept[1] is not net.leaves:
        fs = {g: i for i, g in enumerate(circ.fsim_indices())}
        var = [i for i, lf in enumerate(net.leaves) if lf.kind == "gate" and lf.gate in fs]
        const = [i for i in range(len(net.leaves)) if i not in set(var)]
        rows = (torch.tensor([fs[net.leaves[i].gate] for i in var], device=params.device)
                if var else None)
        consts = []
        if const:
            flat = np.concatenate([net.leaves[i].data.ravel() for i in const]).astype(np.complex64)
            dev = torch.from_numpy(flat).to(device)
            consts = list(dev.split([net.leaves[i].data.size for i in const]))
        kept = (key, net.leaves, var, rows, const, consts)
        net.__dict__["_torch_leaf_cache"] = kept
    _, _, var, rows, const, consts = kept
    out = [None] * len(net.leaves)
    if var:
        P = params[rows].to(device)
        for i, t in zip(var, _torch_fsim_leaves(P[:, 0], P[:, 1]).unbind(0)):
            out[i] = t
    for i, t in zip(const, consts):
        out[i] = t
    return out


def _make_function():
    import torch

    class ContractTree(torch.autograd.Function):
        """out = qcs_contract_tree(plan, leaves); the backward runs
        qcs_contract_tree_backward (adjoint emulated CGEMMs, recompute per
        instance)."""

        @staticmethod
        def forward(ctx, cp, h, *leaves):
            ctx.cp = cp
            ctx.h = h
            ctx.save_for_backward(*leaves)
            gp = getattr(cp, "graphed", None)
            if gp is not None and gp.h is h:
                return gp.forward(list(leaves))
            return cp.forward(h, list(leaves))

        @staticmethod
        def backward(ctx, grad_out):
            leaves = ctx.saved_tensors
            gp = getattr(ctx.cp, "graphed", None)
            if gp is not None and gp.h is ctx.h:
                grads = gp.backward(list(leaves), grad_out)
            else:
                grads = ctx.cp.backward(ctx.h, grad_out, list(leaves))
            return (None, None, *[g if t.requires_grad else None for g, t in zip(grads, leaves)])

    return ContractTree


_FN = None


def contract(cp: CompiledPlan, h, leaves):
    """Differentiable contraction of ``leaves`` (complex64 device tensors)."""
    global _FN
    if _FN is None:
        _FN = _make_function()
    return _FN.apply(cp, h, *leaves)


def cheapest_network_order(nets: Sequence[Network], seeds: Sequence[int],
                           skip: Sequence[int] = (), n_slices: int = 0,
                           max_log2_size: Optional[float] = None, workers: int = 1):
    """best_greedy_order over each of several equivalent networks (e.g. a
    circuit's network with and without absorb_single_qubit_gates); returns
    (index of the network, order, sliced labels, seed) of the one whose best
    order has the fewest flops per instance (ties: the earlier network)."""
    best = None
    for i, nw in enumerate(nets):
        order, sliced, seed = best_greedy_order(nw, seeds, skip=skip, n_slices=n_slices,
                                                max_log2_size=max_log2_size, workers=workers)
        flops, _ = order_cost(nw, order, skip=list(skip) + list(sliced))
        if best is None or flops < best[0]:
            best = (flops, i, order, sliced, seed)
    return best[1:]


def plan_circuit(circ, bitstrings=None, seed: int = 2, n_slices: int = 0,
                 max_log2_size: Optional[float] = None, mode: int = 0, trials: int = 1,
                 workers: int = 1, absorb: bool = False) -> Plan:
    """circuit -> network -> greedy order (seeded) -> slices -> plan.
    ``n_slices``: number of sliced indices (2**n_slices slices).  ``trials``
    > 1: the cheapest of the greedy orders of seeds seed .. seed + trials - 1
    (best_greedy_order, costed in ``workers`` processes).  ``absorb``: the
    single-qubit gates contracted into their neighbours first
    (absorb_single_qubit_gates)."""
    net = circuit_network(circ, bitstrings)
    if absorb:
        net = absorb_single_qubit_gates(net)
    skip = [BATCH] if net.batch else []
    if trials > 1:
        order, sliced, _ = best_greedy_order(net, range(seed, seed + trials), skip=skip,
                                             n_slices=n_slices, max_log2_size=max_log2_size,
                                             workers=workers)
        return build_plan(net, order, sliced, mode=mode)
    order = greedy_order(net, seed=seed, skip=skip)
    sliced = []
    if n_slices or max_log2_size is not None:
        sliced = choose_slices(net, order, n_labels=n_slices or None,
                               max_log2_size=max_log2_size, skip=skip)
    return build_plan(net, order, sliced, mode=mode)


# ---------------------------------------------------------------------------
# several GPUs: instances (slices, bitstrings) are independent (Section 5.3)
# ---------------------------------------------------------------------------

def shard_plan(plan: Plan, rank: int, world: int) -> Plan:
    """The instances of ``plan`` that rank ``rank`` of ``world`` runs
    (round-robin).  Summing every rank's output slots gives the full result."""
    import copy

    idx = np.arange(rank, plan.n_instances, world)
    sub = copy.copy(plan)
    sub.instance_offset = np.ascontiguousarray(plan.instance_offset[idx])
    sub.instance_slot = np.ascontiguousarray(plan.instance_slot[idx])
    return sub


def allreduce_slots(out, group=None):
    """Sum complex128 output slots over the ranks of ``group`` in place."""
    import torch
    import torch.distributed as dist

    dist.all_reduce(torch.view_as_real(out), op=dist.ReduceOp.SUM, group=group)
    return out


def allreduce_leaf_grads(grads, group=None):
    """Sum leaf gradients (complex tensors, e.g. from CompiledPlan.backward on
    a shard of the instances) over the ranks of ``group`` in place: every
    rank then holds the gradient of the whole plan.  One collective over one
    packed buffer."""
    import torch
    import torch.distributed as dist

    flat = torch.cat([torch.view_as_real(g).reshape(-1) for g in grads])
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for g in grads:
        n = 2 * g.numel()
        torch.view_as_real(g).reshape(-1).copy_(flat[off:off + n])
        off += n
    return grads
