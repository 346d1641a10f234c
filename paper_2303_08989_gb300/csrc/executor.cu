// Contraction-tree executor (qcs_contract_tree, qcs_contract_tree_backward).
//
// A plan is a list of pairwise contractions, each reshaped to one CGEMM
// (TTGT: gather the operands into matrices, GEMM; Section 1, Section 2.2).
// The executor runs the plan once per instance -- one assignment of the
// sliced indices and/or one bitstring (Section 5.3) -- on the handle's
// stream: per step an optional gather of each operand (the permute /
// slice-gather kernel), then qcs_cgemm's launch sequence (statistics,
// selection, split, tensor-core or FP32 GEMM), writing the step's output
// into its own slot of the tree workspace.  The root of each instance is
// accumulated in FP64 into its output slot.  Instances run in groups
// (qcs_set_instance_batch): the steps up to the first emulated one that
// fills the GPU alone run once for the group, their GEMMs as one batched
// FP32 launch or one grouped tensor-core launch.
//
// The adjoint recomputes an instance's forward pass, then walks the steps
// backwards: grad_A = grad_out B_mat^H and grad_B = A_mat^H grad_out as two
// emulated CGEMMs with conjugate-transpose flags, and scatters each operand
// gradient back through the same map that gathered the operand (adding into
// the caller's leaf gradients at the instance's offset).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <set>
#include <tuple>
#include <vector>

#include "internal.h"

namespace qcs {
namespace {

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// One entry of a step sequence: a single step, or (step < 0) the level
// launch of small steps small_order[first .. first + count).
struct Item {
    int step = -1;
    int first = 0, count = 0;
    int smem_elems = 0;  // level launch: shared memory per warp (complex values)
    int smem_bwd = 0;    // ... of its adjoint launch
};

struct Layout {
    int G = 1;                      // instances per group
    std::vector<size_t> inter_off;  // byte offset of each step's output ([G][m n])
    std::vector<size_t> grad_off;   // byte offset of each step's output gradient (backward)
    std::vector<char> batched;      // step runs as one batched launch per group
    int P = 0;                      // steps [0, P): batched; [P, ns): one instance at a time
    std::vector<int> eff;           // effective mode of each step's forward GEMM
    std::vector<char> small;        // step runs inside its level's launch
    std::vector<Item> seq_b, seq_i; // order of the steps before P (once per group), from P on
    std::vector<int> small_order;   // the small steps, grouped by launch
    std::vector<int> time;          // when each step runs (equal times may overlap)
    std::vector<int32_t> tab;       // element-offset tables of the small steps' operands
    std::vector<int32_t> tab_a, tab_b;  // start of each small step's tables in ``tab``
    size_t out_index = 0, offsets = 0, bufA = 0, bufB = 0, tmpA = 0, tmpB = 0, gemm = 0, total = 0;
    size_t small_desc = 0, small_tab = 0, small_bwd = 0;
    // backward in groups (G > 1): each instance's leaf gradients in its own
    // zeroed buffer of lgrad_stride elements (leaf i at lgrad_off[i]), added
    // into the caller's in instance order after the group (leaf_tab)
    size_t lgrad = 0, leaf_tab = 0;
    int64_t lgrad_stride = 0, max_leaf = 0;
    std::vector<int64_t> lgrad_off;
    size_t gemm_bytes = 0, inter_bytes = 0;
};

int64_t root_size(const qcs_tree_t *t, const std::vector<int64_t> &size_of) {
    return t->n_steps > 0 ? size_of[t->n_leaves + t->n_steps - 1] : size_of[0];
}

// Largest offset (relative to the tensor start) a map reads; strides >= 0.
bool map_span(const qcs_gather_t &g, int64_t expect_elems, int64_t &span) {
    if (g.rank < 0 || g.rank > QCS_MAX_RANK) return false;
    int64_t prod = 1;
    span = 0;
    for (int d = 0; d < g.rank; ++d) {
        if (g.dims[d] < 1 || g.strides[d] < 0) return false;
        prod *= g.dims[d];
        span += (g.dims[d] - 1) * g.strides[d];
    }
    return prod == expect_elems;
}

// Host-side validation of the whole plan: ids, shapes, and that every
// element a map, a direct operand or the output gather reads lies inside its
// tensor (for leaves, at every instance offset).
int validate(const qcs_tree_t *t, std::vector<int64_t> &size_of, bool need_tree) {
    if (!t || t->n_leaves < 1 || t->n_steps < 0 || t->n_instances < 1 || t->n_slots < 1 ||
        !t->leaf_size || !t->instance_offset || !t->instance_slot || t->out_size < 1 ||
        (t->n_steps > 0 && !t->steps))
        return QCS_ERR_INVALID_ARG;
    const int nl = t->n_leaves, ns = t->n_steps, ni = t->n_instances;
    size_of.assign(nl + ns, 0);
    for (int i = 0; i < nl; ++i) {
        if (t->leaf_size[i] < 1) return QCS_ERR_INVALID_ARG;
        size_of[i] = t->leaf_size[i];
    }
    std::vector<int64_t> max_off(nl, 0);
    for (int inst = 0; inst < ni; ++inst) {
        if (t->instance_slot[inst] < 0 || t->instance_slot[inst] >= t->n_slots) return QCS_ERR_INVALID_ARG;
        for (int i = 0; i < nl; ++i) {
            const int64_t o = t->instance_offset[(int64_t)inst * nl + i];
            if (o < 0) return QCS_ERR_INVALID_ARG;
            max_off[i] = std::max(max_off[i], o);
        }
    }
    std::vector<int> uses(nl + ns, 0);
    for (int s = 0; s < ns; ++s) {
        const qcs_step_t &st = t->steps[s];
        const int self = nl + s;
        if (st.a < 0 || st.b < 0 || st.a >= self || st.b >= self || st.a == st.b) return QCS_ERR_INVALID_ARG;
        if (st.m < 1 || st.n < 1 || st.k < 1) return QCS_ERR_INVALID_ARG;
        if (st.mode < QCS_MODE_AUTO || st.mode > QCS_MODE_BF16X3) return QCS_ERR_INVALID_ARG;
        uses[st.a]++;
        uses[st.b]++;
        const int ids[2] = {st.a, st.b};
        const qcs_gather_t *maps[2] = {&st.map_a, &st.map_b};
        const int direct[2] = {st.direct_a, st.direct_b};
        const int64_t elems[2] = {st.m * st.k, st.k * st.n};
        for (int o = 0; o < 2; ++o) {
            int64_t span;
            if (!map_span(*maps[o], elems[o], span)) return QCS_ERR_INVALID_ARG;
            const int id = ids[o];
            const int64_t base = id < nl ? max_off[id] : 0;
            if (base + span >= size_of[id]) return QCS_ERR_INVALID_ARG;
            if (direct[o] != -1) {
                if (direct[o] != QCS_OP_N && direct[o] != QCS_OP_T) return QCS_ERR_INVALID_ARG;
                if (size_of[id] != elems[o] || base != 0) return QCS_ERR_INVALID_ARG;
            }
        }
        size_of[self] = st.m * st.n;
    }
    // The root as every instance sees it: the last step's output, or (no
    // steps) leaf 0 from the instance's offset on.
    const int64_t rs = ns > 0 ? root_size(t, size_of) : size_of[0] - max_off[0];
    if (t->out_index) {
        for (int64_t j = 0; j < t->out_size; ++j)
            if (t->out_index[j] < 0 || t->out_index[j] >= rs) return QCS_ERR_INVALID_ARG;
    } else if (ns > 0 ? rs != t->out_size : rs < t->out_size) {
        return QCS_ERR_INVALID_ARG;
    }
    if (need_tree) {
        for (int i = 0; i < nl + ns - 1; ++i)
            if (uses[i] != 1) return QCS_ERR_INVALID_ARG;
        if (ns > 0 && uses[nl + ns - 1] != 0) return QCS_ERR_INVALID_ARG;
    }
    return QCS_SUCCESS;
}

inline int fwd_op(int direct) { return direct == QCS_OP_T ? QCS_OP_T : QCS_OP_N; }

// Offsets of the step outputs when intermediates may share memory: the
// output of step s is live from step s until its last reader (the root until
// the end), and is placed first-fit among the blocks live at step s.  A
// step's output never overlaps its operands, which are still live then.
// Steps from P on run once per instance of the group, so an output of an
// earlier step that one of them reads stays live to the end.
// time[s] orders the steps as they run: steps of equal time may run at once
// (one level launch, or steps of a level issued back to back), so an output
// is live from its step's time to its last reader's time, inclusive.
size_t place_by_liveness(const qcs_tree_t *t, const std::vector<size_t> &bytes, int P,
                         const std::vector<int> &time, std::vector<size_t> &off) {
    const int nl = t->n_leaves, ns = t->n_steps;
    constexpr int kEnd = INT32_MAX;
    std::vector<int> last(ns);  // time of the last reader of each output; the root: the end
    for (int s = 0; s < ns; ++s) last[s] = (s == ns - 1) ? kEnd : -1;
    for (int s = 0; s < ns; ++s) {
        const qcs_step_t &st = t->steps[s];
        for (const int id : {st.a, st.b}) {
            if (id < nl) continue;
            const int p = id - nl;
            last[p] = std::max(last[p], (s >= P && p < P) ? kEnd : time[s]);
        }
    }
    std::vector<int> order(ns);
    for (int s = 0; s < ns; ++s) order[s] = s;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return time[x] < time[y]; });
    struct Block {
        size_t off, size;
        int id;
    };
    std::vector<Block> live;  // sorted by offset
    size_t peak = 0;
    off.assign(ns, 0);
    for (const int s : order) {
        live.erase(std::remove_if(live.begin(), live.end(),
                                  [&](const Block &b) { return last[b.id] < time[s]; }),
                   live.end());
        size_t at = 0;
        for (const Block &b : live) {
            if (b.off >= at + bytes[s]) break;
            at = std::max(at, b.off + b.size);
        }
        off[s] = at;
        live.insert(std::upper_bound(live.begin(), live.end(), at,
                                     [](size_t v, const Block &b) { return v < b.off; }),
                    Block{at, bytes[s], s});
        peak = std::max(peak, at + bytes[s]);
    }
    return peak;
}

// Element offsets of op(X) (rows x cols, element e = i + l rows) inside its
// tensor: through the gather map (e split by the map's dims, first fastest),
// or the tensor itself in N or T layout.  False if an offset exceeds int32.
bool operand_table(int direct, const qcs_gather_t &g, int64_t rows, int64_t cols,
                   std::vector<int32_t> &tab) {
    const int64_t count = rows * cols;
    for (int64_t e = 0; e < count; ++e) {
        int64_t o;
        if (direct == QCS_OP_N) {
            o = e;
        } else if (direct == QCS_OP_T) {
            o = (e / rows) + (e % rows) * cols;
        } else {
            o = 0;
            int64_t rest = e;
            for (int d = 0; d < g.rank; ++d) {
                o += (rest % g.dims[d]) * g.strides[d];
                rest /= g.dims[d];
            }
        }
        if (o > INT32_MAX) return false;
        tab.push_back((int32_t)o);
    }
    return true;
}

// The steps [lo, hi) in the order they run, into ``items``.  Level
// launches on: level by level (a step's level is one more than the highest
// level of its operands produced in [lo, hi)), the small steps of a level
// first as one launch, then its other steps in plan order; every step of a
// level gets the time base + level - 1.  Off: plan order, time = step.
// Returns the next free time.
int schedule(const qcs_tree_t *t, Layout &L, int lo, int hi, int base, bool levels,
             std::vector<Item> &items, std::vector<int> &time) {
    const int nl = t->n_leaves;
    if (!levels) {
        for (int s = lo; s < hi; ++s) {
            Item it;
            it.step = s;
            items.push_back(it);
            time[s] = s;
        }
        return hi;
    }
    std::vector<int> level(hi > lo ? hi - lo : 0, 1);
    int top = 0;
    for (int s = lo; s < hi; ++s) {
        const qcs_step_t &st = t->steps[s];
        for (const int id : {st.a, st.b})
            if (id >= nl + lo) level[s - lo] = std::max(level[s - lo], level[id - nl - lo] + 1);
        top = std::max(top, level[s - lo]);
    }
    for (int d = 1; d <= top; ++d) {
        Item lv;
        lv.first = (int)L.small_order.size();
        for (int s = lo; s < hi; ++s) {
            if (level[s - lo] != d || !L.small[s]) continue;
            const qcs_step_t &st = t->steps[s];
            L.small_order.push_back(s);
            lv.smem_elems = std::max<int>(lv.smem_elems, (int)(st.m * st.k + st.k * st.n));
            lv.smem_bwd =
                std::max<int>(lv.smem_bwd, (int)(st.m * st.n + st.m * st.k + st.k * st.n));
        }
        lv.count = (int)L.small_order.size() - lv.first;
        if (lv.count > 0) items.push_back(lv);
        for (int s = lo; s < hi; ++s) {
            if (level[s - lo] != d) continue;
            time[s] = base + d - 1;
            if (L.small[s]) continue;
            Item it;
            it.step = s;
            items.push_back(it);
        }
    }
    return base + top;
}

// Workspace of one call.  Forward: the instances run in groups of G that
// share the buffers.  The steps before P run once per group: a plain-FP32
// step as one batched gather and one batched GEMM launch, an emulated step as
// one grouped sequence (run_cgemm_group: one tensor-core launch per kind over
// the tiles of all G instances), outputs holding G instances.  P is the first
// emulated step with at least one output tile per SM whose planes and output
// for G instances exceed the handle's group budget: from there on (in a tree
// from a greedy order, the few largest contractions at the end) the steps run
// one instance after another, outputs holding one instance.  Steps run level
// by level when level launches are on (schedule()).  Outputs reuse memory by
// liveness.  Backward (G = 1): every output is kept.
Layout plan_layout(qcs_handle_t h, const qcs_tree_t *t, bool backward, int G) {
    Layout L;
    L.G = G;
    const int ns = t->n_steps;
    size_t p = 0;
    L.out_index = p;
    p += align256(sizeof(int64_t) * (t->out_index ? t->out_size : 1));
    L.offsets = p;
    p += align256(sizeof(int64_t) * (size_t)t->n_instances * t->n_leaves);
    int64_t maxA = 1, maxB = 1;
    size_t gemm = 0;
    L.eff.resize(ns);
    L.batched.assign(ns, 0);
    std::vector<size_t> bytes(ns);
    for (int s = 0; s < ns; ++s) {
        const qcs_step_t &st = t->steps[s];
        L.eff[s] = effective_mode(h, st.mode, fwd_op(st.direct_a), fwd_op(st.direct_b), st.m, st.n,
                                  st.k);
        // An emulated step whose output tiles fill the GPU alone still gains
        // from one launch over its instances (full tile waves, one pipeline
        // ramp), but a group holds G copies of its planes and output: when
        // those exceed the handle's budget it and every later step run per
        // instance.
        const int64_t tiles = ((st.m + kBM - 1) / kBM) * ((st.n + kBN - 1) / kBN);
        bool fills = L.eff[s] != QCS_MODE_FP32 && tiles >= h->num_sms;
        if (fills) {
            const size_t grouped =
                gemm_workspace_bytes(L.eff[s], st.m, st.n, st.k, h->num_sms,
                                     gemm_splits(h, fwd_op(st.direct_a), fwd_op(st.direct_b), st.m,
                                                 st.n, st.k),
                                     G) +
                sizeof(float2) * (size_t)(st.m * st.n) * G;
            fills = grouped > h->group_budget;
        }
        L.batched[s] = (G > 1 && !fills) ? 1 : 0;
    }
    L.P = 0;
    while (L.P < ns && L.batched[L.P]) ++L.P;
    for (int s = L.P; s < ns; ++s) L.batched[s] = 0;
    // small plain-FP32 steps: run inside their level's launch, operands read
    // through element-offset tables
    L.small.assign(ns, 0);
    L.tab_a.assign(ns, 0);
    L.tab_b.assign(ns, 0);
    for (int s = 0; s < ns && h->tree_levels; ++s) {
        const qcs_step_t &st = t->steps[s];
        if (L.eff[s] != QCS_MODE_FP32 || st.m * st.k > kTreeSmallOperand ||
            st.k * st.n > kTreeSmallOperand || st.m * st.n > kTreeSmallOutput)
            continue;
        // the adjoint's level launch too: both adjoint GEMMs plain FP32, and
        // grad_out with both operands in one warp's shared memory
        if (backward && (st.m * st.n + st.m * st.k + st.k * st.n > kTreeSmallBwdElems ||
                         effective_mode(h, st.mode, QCS_OP_N, QCS_OP_C, st.m, st.k, st.n) !=
                             QCS_MODE_FP32 ||
                         effective_mode(h, st.mode, QCS_OP_C, QCS_OP_N, st.k, st.n, st.m) !=
                             QCS_MODE_FP32))
            continue;
        const size_t at = L.tab.size();
        L.tab_a[s] = (int32_t)at;
        bool ok = operand_table(st.direct_a, st.map_a, st.m, st.k, L.tab);
        L.tab_b[s] = (int32_t)L.tab.size();
        ok = ok && operand_table(st.direct_b, st.map_b, st.k, st.n, L.tab);
        if (ok && L.tab.size() <= (size_t)INT32_MAX) {
            L.small[s] = 1;
        } else {
            L.tab.resize(at);
        }
    }
    L.time.assign(ns, 0);
    std::vector<int> &time = L.time;
    const int tb = schedule(t, L, 0, L.P, 0, h->tree_levels != 0, L.seq_b, time);
    schedule(t, L, L.P, ns, tb, h->tree_levels != 0, L.seq_i, time);
    for (int s = 0; s < ns; ++s) {
        const qcs_step_t &st = t->steps[s];
        const int64_t gb = L.batched[s] ? G : 1;
        bytes[s] = align256(sizeof(float2) * st.m * st.n * gb);
        if (L.eff[s] == QCS_MODE_FP32) {
            // a batched plain-FP32 GEMM reads the gathered operands of the whole
            // group and keeps a split-K partial buffer per instance, at the end
            // of its workspace
            maxA = std::max(maxA, st.m * st.k * gb);
            maxB = std::max(maxB, st.k * st.n * gb);
            gemm = std::max(gemm, gemm_workspace_bytes(QCS_MODE_FP32, st.m, st.n, st.k, h->num_sms,
                                                       0) +
                                      (size_t)(gb - 1) * kSplitKBytes);
        } else {
            // an emulated step gathers one instance at a time; its planes and
            // descriptors hold the whole group
            maxA = std::max(maxA, st.m * st.k);
            maxB = std::max(maxB, st.k * st.n);
            gemm = std::max(gemm, gemm_workspace_bytes(
                                      L.eff[s], st.m, st.n, st.k, h->num_sms,
                                      gemm_splits(h, fwd_op(st.direct_a), fwd_op(st.direct_b),
                                                  st.m, st.n, st.k),
                                      (int)gb));
        }
        if (backward) {
            // the two adjoint GEMMs, for the whole group (batched FP32 with a
            // split-K buffer per instance, or grouped emulated)
            const int eA = effective_mode(h, st.mode, QCS_OP_N, QCS_OP_C, st.m, st.k, st.n);
            const int eB = effective_mode(h, st.mode, QCS_OP_C, QCS_OP_N, st.k, st.n, st.m);
            gemm = std::max(gemm, gemm_workspace_bytes(
                                      eA, st.m, st.k, st.n, h->num_sms,
                                      gemm_splits(h, QCS_OP_N, QCS_OP_C, st.m, st.k, st.n),
                                      (int)gb) +
                                      (eA == QCS_MODE_FP32 ? (size_t)(gb - 1) * kSplitKBytes : 0));
            gemm = std::max(gemm, gemm_workspace_bytes(
                                      eB, st.k, st.n, st.m, h->num_sms,
                                      gemm_splits(h, QCS_OP_C, QCS_OP_N, st.k, st.n, st.m),
                                      (int)gb) +
                                      (eB == QCS_MODE_FP32 ? (size_t)(gb - 1) * kSplitKBytes : 0));
            // its gathers and scatters handle the whole group at once
            maxA = std::max(maxA, st.m * st.k * gb);
            maxB = std::max(maxB, st.k * st.n * gb);
        }
    }
    L.inter_off.resize(ns);
    if (backward) {
        for (int s = 0; s < ns; ++s) {
            L.inter_off[s] = p;
            p += bytes[s];
        }
    } else {
        std::vector<size_t> rel;
        const size_t inter = place_by_liveness(t, bytes, L.P, time, rel);
        for (int s = 0; s < ns; ++s) L.inter_off[s] = p + rel[s];
        p += align256(inter);
    }
    L.inter_bytes = p - L.offsets;
    L.bufA = p;
    p += align256(sizeof(float2) * maxA);
    L.bufB = p;
    p += align256(sizeof(float2) * maxB);
    if (backward) {
        L.grad_off.resize(ns);
        for (int s = 0; s < ns; ++s) {
            L.grad_off[s] = p;
            p += align256(sizeof(float2) * t->steps[s].m * t->steps[s].n * (L.batched[s] ? G : 1));
        }
        L.tmpA = p;
        p += align256(sizeof(float2) * maxA);
        L.tmpB = p;
        p += align256(sizeof(float2) * maxB);
        if (G > 1) {
            L.lgrad_off.resize(t->n_leaves);
            int64_t q = 0;
            for (int i = 0; i < t->n_leaves; ++i) {
                L.lgrad_off[i] = q;
                q += (t->leaf_size[i] + 31) / 32 * 32;  // 256-byte aligned per leaf
                L.max_leaf = std::max(L.max_leaf, t->leaf_size[i]);
            }
            L.lgrad_stride = q;
            L.lgrad = p;
            p += align256(sizeof(float2) * (size_t)q * G);
            L.leaf_tab = p;
            p += align256(sizeof(LeafGradRef) * t->n_leaves);
        }
    }
    L.gemm = p;
    L.gemm_bytes = gemm;
    p += align256(gemm);
    L.small_desc = p;
    p += align256(sizeof(TreeSmallStep) * L.small_order.size());
    L.small_tab = p;
    p += align256(sizeof(int32_t) * L.tab.size());
    if (backward) {
        L.small_bwd = p;
        p += align256(sizeof(TreeSmallBwd) * L.small_order.size());
    }
    L.total = p;
    return L;
}

struct Ctx {
    qcs_handle_t h;
    const qcs_tree_t *t;
    const qcs_c32 *const *leaves;
    uint8_t *ws;
    Layout L;
    std::vector<int64_t> size_of;  // elements of every tensor (leaves, then step outputs)
    qcs_run_info_t *info;
    qcs_c32 *const *grad_leaves = nullptr;  // backward: the caller's leaf gradients
};

float2 *inter_ptr(const Ctx &c, int s) { return reinterpret_cast<float2 *>(c.ws + c.L.inter_off[s]); }
float2 *grad_ptr(const Ctx &c, int s) { return reinterpret_cast<float2 *>(c.ws + c.L.grad_off[s]); }

// Tensor ``id`` as seen by instance ``inst`` at position g of its group
// (outputs of batched steps hold the whole group, the others one instance).
const float2 *tensor_ptr(const Ctx &c, int id, int inst, int g = 0) {
    const int nl = c.t->n_leaves;
    if (id < nl)
        return reinterpret_cast<const float2 *>(c.leaves[id]) +
               c.t->instance_offset[(int64_t)inst * nl + id];
    return inter_ptr(c, id - nl) + (c.L.batched[id - nl] ? (int64_t)g * c.size_of[id] : 0);
}

void count_gemm(const Ctx &c, int eff, int64_t m, int64_t n, int64_t k, int64_t count = 1) {
    if (!c.info) return;
    c.info->gemm_count += count;
    const double f = 8.0 * (double)m * (double)n * (double)k * (double)count;
    if (eff >= 0 && eff < 6) {
        c.info->mode_count[eff] += count;
        c.info->mode_flops[eff] += f;
    }
    c.info->flops += f;
}

int gather(const Ctx &c, const qcs_gather_t &g, const float2 *src, float2 *dst,
           const CopyBatch &cb = CopyBatch{}) {
    if (c.info) c.info->gather_count += cb.count;
    ProfScope ps(c.h, kProfPermute);
    return launch_permute(g.rank, g.dims, g.strides, 0, src, dst, nullptr, 0, c.h->stream, cb) ==
                   cudaSuccess
               ? QCS_SUCCESS
               : QCS_ERR_CUDA;
}

int gemm(const Ctx &c, int mode, int opA, int opB, int64_t m, int64_t n, int64_t k,
         const float2 *A, int64_t lda, const float2 *B, int64_t ldb, float2 *C) {
    const int eff = effective_mode(c.h, mode, opA, opB, m, n, k);
    count_gemm(c, eff, m, n, k);
    return run_cgemm(c.h, c.ws + c.L.gemm, eff, opA, opB, m, n, k, make_float2(1.f, 0.f), A, lda,
                     B, ldb, make_float2(0.f, 0.f), C, m, nullptr, nullptr);
}

// One operand of a batched step: the gathered matrices of the group in
// ``buf`` (stride rows x cols), or the tensor itself (a leaf shared by every
// instance: stride 0; an intermediate: stride of its instance slots).
int batched_operand(const Ctx &c, int id, int direct, const qcs_gather_t &map, int inst0, int G,
                    int64_t elems, float2 *buf, const float2 *&X, int64_t &stride) {
    const int nl = c.t->n_leaves;
    if (direct != -1) {
        X = tensor_ptr(c, id, inst0, 0);
        stride = id < nl ? 0 : c.size_of[id];
        return QCS_SUCCESS;
    }
    CopyBatch cb;
    cb.count = G;
    cb.out_stride = elems;
    const float2 *src;
    if (id < nl) {
        src = reinterpret_cast<const float2 *>(c.leaves[id]);
        cb.off = reinterpret_cast<const int64_t *>(c.ws + c.L.offsets) + (int64_t)inst0 * nl + id;
        cb.off_stride = nl;
    } else {
        src = inter_ptr(c, id - nl);
        cb.in_stride = c.size_of[id];
    }
    X = buf;
    stride = elems;
    return gather(c, map, src, buf, cb);
}

// Does the map read every element of a tensor of ``size`` elements exactly
// once (a permutation of the whole tensor, as for every intermediate)?
bool whole_permutation(const qcs_gather_t &g, int64_t size) {
    int64_t st[QCS_MAX_RANK], dm[QCS_MAX_RANK];
    int r = 0;
    for (int d = 0; d < g.rank; ++d)
        if (g.dims[d] > 1) {
            st[r] = g.strides[d];
            dm[r++] = g.dims[d];
        }
    for (int i = 1; i < r; ++i)  // insertion sort by stride
        for (int j = i; j > 0 && st[j] < st[j - 1]; --j) {
            std::swap(st[j], st[j - 1]);
            std::swap(dm[j], dm[j - 1]);
        }
    int64_t expect = 1;
    for (int i = 0; i < r; ++i) {
        if (st[i] != expect) return false;
        expect *= dm[i];
    }
    return expect == size;
}

// The view of one operand of a step: the tensor through its map when the GEMM
// is emulated and the operand is an intermediate permuted as a whole (the
// split then reads through the map: no gather), else the gathered matrix or
// the directly usable tensor.
int operand_view(const Ctx &c, int s, int id, int direct, const qcs_gather_t &map, int inst, int g,
                 int64_t rows, int64_t ld_direct, float2 *buf, OperandView &v) {
    const float2 *X = tensor_ptr(c, id, inst, g);
    if (direct != -1) {
        v.X = X;
        v.ld = ld_direct;
        return QCS_SUCCESS;
    }
    if (c.L.eff[s] != QCS_MODE_FP32 && id >= c.t->n_leaves && whole_permutation(map, c.size_of[id])) {
        v.X = X;
        v.map = &map;
        v.flat = c.size_of[id];
        v.buf = buf;
        return QCS_SUCCESS;
    }
    if (int r = gather(c, map, X, buf)) return r;
    v.X = buf;
    v.ld = rows;
    return QCS_SUCCESS;
}

// One step for one instance (position g of its group): operand views (gathers
// where needed), then qcs_cgemm's launch sequence, output into the step's slot.
int step_instance(const Ctx &c, int s, int inst, int g) {
    const qcs_step_t &st = c.t->steps[s];
    float2 *bufA = reinterpret_cast<float2 *>(c.ws + c.L.bufA);
    float2 *bufB = reinterpret_cast<float2 *>(c.ws + c.L.bufB);
    const int opA = fwd_op(st.direct_a), opB = fwd_op(st.direct_b);
    const int64_t lda = opA == QCS_OP_T ? st.k : st.m, ldb = opB == QCS_OP_T ? st.n : st.k;
    OperandView va, vb;
    if (int r = operand_view(c, s, st.a, st.direct_a, st.map_a, inst, g, st.m, lda, bufA, va))
        return r;
    if (int r = operand_view(c, s, st.b, st.direct_b, st.map_b, inst, g, st.k, ldb, bufB, vb))
        return r;
    float2 *C = inter_ptr(c, s) + (c.L.batched[s] ? (int64_t)g * st.m * st.n : 0);
    count_gemm(c, c.L.eff[s], st.m, st.n, st.k);
    return run_cgemm_views(c.h, c.ws + c.L.gemm, c.L.eff[s], opA, opB, st.m, st.n, st.k,
                           make_float2(1.f, 0.f), va, vb, make_float2(0.f, 0.f), C, st.m, nullptr,
                           nullptr);
}

// One emulated step for the G instances of a group: per instance the
// operand views (mapped operands are read through their maps or gathered
// inside the GEMM sequence, one instance at a time), then run_cgemm_group:
// statistics, selection and split per instance, one tensor-core launch per
// kind over the tiles of all G instances.
int step_grouped(const Ctx &c, int s, int inst0, int G) {
    const qcs_step_t &st = c.t->steps[s];
    float2 *bufA = reinterpret_cast<float2 *>(c.ws + c.L.bufA);
    float2 *bufB = reinterpret_cast<float2 *>(c.ws + c.L.bufB);
    const int opA = fwd_op(st.direct_a), opB = fwd_op(st.direct_b);
    const int64_t lda = opA == QCS_OP_T ? st.k : st.m, ldb = opB == QCS_OP_T ? st.n : st.k;
    std::vector<OperandView> va(G), vb(G);
    const int ids[2] = {st.a, st.b};
    const int direct[2] = {st.direct_a, st.direct_b};
    const qcs_gather_t *maps[2] = {&st.map_a, &st.map_b};
    const int64_t lds[2] = {lda, ldb};
    float2 *bufs[2] = {bufA, bufB};
    for (int o = 0; o < 2; ++o) {
        const int id = ids[o];
        const bool whole = id >= c.t->n_leaves && whole_permutation(*maps[o], c.size_of[id]);
        for (int g = 0; g < G; ++g) {
            OperandView &v = (o == 0 ? va : vb)[g];
            v.X = tensor_ptr(c, id, inst0 + g, g);
            if (direct[o] != -1) {
                v.ld = lds[o];
                continue;
            }
            v.map = maps[o];
            v.flat = whole ? c.size_of[id] : 0;
            v.buf = bufs[o];
            if (c.info && !whole) c.info->gather_count++;
        }
    }
    count_gemm(c, c.L.eff[s], st.m, st.n, st.k, G);
    return run_cgemm_group(c.h, c.ws + c.L.gemm, c.L.eff[s], opA, opB, st.m, st.n, st.k,
                           make_float2(1.f, 0.f), va.data(), vb.data(), G, make_float2(0.f, 0.f),
                           inter_ptr(c, s), st.m, st.m * st.n, nullptr, nullptr);
}

// One batched step for the G instances of a group: batched gathers, one
// batched plain-FP32 GEMM launch.
int step_batched(const Ctx &c, int s, int inst0, int G) {
    const qcs_step_t &st = c.t->steps[s];
    float2 *bufA = reinterpret_cast<float2 *>(c.ws + c.L.bufA);
    float2 *bufB = reinterpret_cast<float2 *>(c.ws + c.L.bufB);
    const int opA = fwd_op(st.direct_a), opB = fwd_op(st.direct_b);
    const int64_t lda = opA == QCS_OP_T ? st.k : st.m, ldb = opB == QCS_OP_T ? st.n : st.k;
    const float2 *A, *B;
    GemmBatch bt;
    bt.count = G;
    bt.sC = st.m * st.n;
    if (int r = batched_operand(c, st.a, st.direct_a, st.map_a, inst0, G, st.m * st.k, bufA, A,
                                bt.sA))
        return r;
    if (int r = batched_operand(c, st.b, st.direct_b, st.map_b, inst0, G, st.k * st.n, bufB, B,
                                bt.sB))
        return r;
    count_gemm(c, c.L.eff[s], st.m, st.n, st.k, G);
    return run_cgemm(c.h, c.ws + c.L.gemm, c.L.eff[s], opA, opB, st.m, st.n, st.k,
                     make_float2(1.f, 0.f), A, lda, B, ldb, make_float2(0.f, 0.f), inter_ptr(c, s),
                     st.m, nullptr, nullptr, bt);
}

const int64_t *dev_index(const Ctx &c) {
    return c.t->out_index ? reinterpret_cast<const int64_t *>(c.ws + c.L.out_index) : nullptr;
}

const float2 *root_ptr(const Ctx &c, int inst, int g = 0) {
    return c.t->n_steps > 0 ? tensor_ptr(c, c.t->n_leaves + c.t->n_steps - 1, inst, g)
                            : tensor_ptr(c, 0, inst);
}

int accumulate_root(const Ctx &c, int inst, int g, double *d_out) {
    ProfScope ps(c.h, kProfReduce);
    const int64_t slot = c.t->instance_slot[inst];
    return launch_accumulate_gather_c128(root_ptr(c, inst, g), dev_index(c),
                                         d_out + 2 * slot * c.t->out_size, c.t->out_size,
                                         c.h->stream) == cudaSuccess
               ? QCS_SUCCESS
               : QCS_ERR_CUDA;
}

// One level launch: the small steps of ``it`` for G instances (instances
// inst0 .. inst0 + G - 1 at group positions g0 .. g0 + G - 1).
int level_small(const Ctx &c, const Item &it, int inst0, int g0, int G) {
    for (int q = it.first; q < it.first + it.count; ++q) {
        const qcs_step_t &st = c.t->steps[c.L.small_order[q]];
        count_gemm(c, QCS_MODE_FP32, st.m, st.n, st.k, G);
    }
    if (c.info) {
        c.info->level_launches++;
        c.info->level_gemms += (int64_t)it.count * G;
    }
    ProfScope ps(c.h, kProfGemmSimt);
    const auto *desc = reinterpret_cast<const TreeSmallStep *>(c.ws + c.L.small_desc) + it.first;
    return launch_tree_small(desc, it.count, G, inst0, g0,
                             reinterpret_cast<const int64_t *>(c.ws + c.L.offsets),
                             c.t->n_leaves, reinterpret_cast<const int32_t *>(c.ws + c.L.small_tab),
                             it.smem_elems, c.h->stream) == cudaSuccess
               ? QCS_SUCCESS
               : QCS_ERR_CUDA;
}

// Forward pass of the G instances inst0 .. inst0 + G - 1: the batched steps
// once for the group, then the remaining steps instance by instance, each
// root added into its output slot (when d_out is not NULL).
int forward_group(const Ctx &c, int inst0, int G, double *d_out) {
    for (const Item &it : c.L.seq_b) {
        if (it.step < 0) {
            if (int r = level_small(c, it, inst0, 0, G)) return r;
            continue;
        }
        const int s = it.step;
        if (G > 1) {
            if (int r = (c.L.eff[s] == QCS_MODE_FP32 ? step_batched(c, s, inst0, G)
                                                     : step_grouped(c, s, inst0, G)))
                return r;
        } else if (int r = step_instance(c, s, inst0, 0)) {
            return r;
        }
    }
    for (int g = 0; g < G; ++g) {
        for (const Item &it : c.L.seq_i) {
            if (int r = (it.step < 0 ? level_small(c, it, inst0 + g, g, 1)
                                     : step_instance(c, it.step, inst0 + g, g)))
                return r;
        }
        if (d_out)
            if (int r = accumulate_root(c, inst0 + g, g, d_out)) return r;
    }
    return QCS_SUCCESS;
}

// The level launches' step table (device pointers of this call's workspace
// and leaves) and offset tables, uploaded once per call.
int upload_leaf_tab(const Ctx &c);

int upload_small(const Ctx &c) {
    const Layout &L = c.L;
    if (L.small_order.empty()) return upload_leaf_tab(c);
    const int nl = c.t->n_leaves;
    std::vector<TreeSmallStep> desc(L.small_order.size());
    for (size_t q = 0; q < desc.size(); ++q) {
        const int s = L.small_order[q];
        const qcs_step_t &st = c.t->steps[s];
        TreeSmallStep &d = desc[q];
        const int ids[2] = {st.a, st.b};
        const float2 **base[2] = {&d.a, &d.b};
        int64_t *istride[2] = {&d.a_istride, &d.b_istride};
        int32_t *leaf[2] = {&d.a_leaf, &d.b_leaf};
        for (int o = 0; o < 2; ++o) {
            const int id = ids[o];
            if (id < nl) {
                *base[o] = reinterpret_cast<const float2 *>(c.leaves[id]);
                *leaf[o] = id;
                *istride[o] = 0;
            } else {
                *base[o] = inter_ptr(c, id - nl);
                *leaf[o] = -1;
                *istride[o] = L.batched[id - nl] ? c.size_of[id] : 0;
            }
        }
        d.c = inter_ptr(c, s);
        d.c_istride = L.batched[s] ? st.m * st.n : 0;
        d.m = (int32_t)st.m;
        d.n = (int32_t)st.n;
        d.k = (int32_t)st.k;
        d.a_tab = L.tab_a[s];
        d.b_tab = L.tab_b[s];
        d.pad = 0;
    }
    cudaStream_t st = c.h->stream;
    if (cudaMemcpyAsync(c.ws + L.small_desc, desc.data(), sizeof(TreeSmallStep) * desc.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(c.ws + L.small_tab, L.tab.data(), sizeof(int32_t) * L.tab.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    if (!c.grad_leaves) return QCS_SUCCESS;
    // the adjoint's table: operands and their gradients (leaf gradients at
    // offset 0 here; the kernel adds the instance offset to both).  In groups
    // a leaf's gradient goes to the instance's own buffer of the group.
    const bool grp = L.G > 1;
    float2 *lgrad = reinterpret_cast<float2 *>(c.ws + L.lgrad);
    std::vector<TreeSmallBwd> bwd(L.small_order.size());
    for (size_t q = 0; q < bwd.size(); ++q) {
        const int s = L.small_order[q];
        const qcs_step_t &sp = c.t->steps[s];
        TreeSmallBwd &d = bwd[q];
        const int ids[2] = {sp.a, sp.b};
        const float2 **x[2] = {&d.a, &d.b};
        float2 **gx[2] = {&d.ga, &d.gb};
        int64_t *xs[2] = {&d.a_istride, &d.b_istride};
        int64_t *gxs[2] = {&d.ga_istride, &d.gb_istride};
        int32_t *leaf[2] = {&d.a_leaf, &d.b_leaf};
        for (int o = 0; o < 2; ++o) {
            const int id = ids[o];
            if (id < nl) {
                *x[o] = reinterpret_cast<const float2 *>(c.leaves[id]);
                *gx[o] = grp ? lgrad + L.lgrad_off[id] : reinterpret_cast<float2 *>(c.grad_leaves[id]);
                *xs[o] = 0;
                *gxs[o] = grp ? L.lgrad_stride : 0;
                *leaf[o] = id;
            } else {
                *x[o] = inter_ptr(c, id - nl);
                *gx[o] = grad_ptr(c, id - nl);
                *xs[o] = *gxs[o] = L.batched[id - nl] ? c.size_of[id] : 0;
                *leaf[o] = -1;
            }
        }
        d.gc = grad_ptr(c, s);
        d.gc_istride = L.batched[s] ? sp.m * sp.n : 0;
        d.m = (int32_t)sp.m;
        d.n = (int32_t)sp.n;
        d.k = (int32_t)sp.k;
        d.a_tab = L.tab_a[s];
        d.b_tab = L.tab_b[s];
        d.pad = 0;
    }
    if (cudaMemcpyAsync(c.ws + L.small_bwd, bwd.data(), sizeof(TreeSmallBwd) * bwd.size(),
                        cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    return upload_leaf_tab(c);
}

// The caller's leaf gradients and where each instance's buffer of a group
// holds them (backward in groups).
int upload_leaf_tab(const Ctx &c) {
    const Layout &L = c.L;
    if (L.G <= 1 || !c.grad_leaves) return QCS_SUCCESS;
    std::vector<LeafGradRef> tab(c.t->n_leaves);
    for (int i = 0; i < c.t->n_leaves; ++i)
        tab[i] = LeafGradRef{reinterpret_cast<float2 *>(c.grad_leaves[i]), c.t->leaf_size[i],
                             L.lgrad_off[i]};
    if (cudaMemcpyAsync(c.ws + L.leaf_tab, tab.data(), sizeof(LeafGradRef) * tab.size(),
                        cudaMemcpyHostToDevice, c.h->stream) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    return QCS_SUCCESS;
}

int begin(qcs_handle_t h, const qcs_tree_t *t, bool backward, Ctx &c, Workspace *own = nullptr) {
    if (int r = validate(t, c.size_of, backward)) return r;
    c.h = h;
    c.t = t;
    // the backward runs in groups too when every step can hold the group
    const int G = std::max(1, std::min(h->instance_batch, t->n_instances));
    c.L = plan_layout(h, t, backward, G);
    if (backward && G > 1 && (t->n_steps == 0 || c.L.P < t->n_steps))
        c.L = plan_layout(h, t, backward, 1);
    Workspace &w = own ? *own : h->tree_ws;
    if (int r = ensure_workspace(w, c.L.total)) return r;
    c.ws = static_cast<uint8_t *>(w.ptr);
    if (t->out_index) {
        if (cudaMemcpyAsync(c.ws + c.L.out_index, t->out_index, sizeof(int64_t) * t->out_size,
                            cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
            cudaGetLastError();
            return QCS_ERR_CUDA;
        }
    }
    if ((c.L.G > 1 || !c.L.small_order.empty()) &&
        cudaMemcpyAsync(c.ws + c.L.offsets, t->instance_offset,
                        sizeof(int64_t) * (size_t)t->n_instances * t->n_leaves,
                        cudaMemcpyHostToDevice, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    if (int r = upload_small(c)) return r;
    if (c.info) c.info->workspace_bytes = (int64_t)c.L.total;
    return QCS_SUCCESS;
}

// Every launch of a forward call after begin(): clear d_out, then per group
// of instances the steps and the FP64 accumulation of each root.
int forward_all(const Ctx &c, double *d_out) {
    const qcs_tree_t *tree = c.t;
    qcs_handle_t h = c.h;
    if (cudaMemsetAsync(d_out, 0, sizeof(double) * 2 * tree->n_slots * tree->out_size, h->stream) !=
        cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    for (int inst0 = 0; inst0 < tree->n_instances; inst0 += c.L.G) {
        const int G = std::min(c.L.G, tree->n_instances - inst0);
        if (int r = forward_group(c, inst0, G, d_out)) return r;
    }
    return QCS_SUCCESS;
}

// Every launch of a backward call after begin(): per instance the forward
// recomputed, the root's gradient seeded from its slot, then per step (last
// to first) the two adjoint GEMMs and the scatters of the operand gradients
// through the maps that gathered the operands.
int backward_all(Ctx &c, const double *d_grad_out, qcs_c32 *const *d_grad_leaves) {
    const qcs_tree_t *tree = c.t;
    qcs_handle_t h = c.h;
    qcs_run_info_t *info = c.info;
    const Layout &L = c.L;
    const std::vector<int64_t> &size_of = c.size_of;
    const int nl = tree->n_leaves, ns = tree->n_steps;
    cudaStream_t s = h->stream;
    // G > 1: a group's instances at once; their intermediates and gradients
    // at one stride, each one's leaf gradients in its own buffer (lgrad)
    const int G = L.G;
    const bool grp = G > 1;
    const std::vector<Item> &seq = grp ? L.seq_b : L.seq_i;
    const int64_t *offs = reinterpret_cast<const int64_t *>(c.ws + L.offsets);
    float2 *lgrad = reinterpret_cast<float2 *>(c.ws + L.lgrad);
    float2 *Am = reinterpret_cast<float2 *>(c.ws + L.bufA);
    float2 *Bm = reinterpret_cast<float2 *>(c.ws + L.bufB);
    float2 *gA = reinterpret_cast<float2 *>(c.ws + L.tmpA);
    float2 *gB = reinterpret_cast<float2 *>(c.ws + L.tmpB);
    // operand ``id`` of the instances inst0 .. inst0 + Gc - 1 gathered into
    // buf, elems complex apart
    auto gather_op = [&](int id, const qcs_gather_t &map, int inst0, int Gc, int64_t elems,
                         float2 *buf) -> int {
        if (!grp) return gather(c, map, tensor_ptr(c, id, inst0), buf);
        CopyBatch cb;
        cb.count = Gc;
        cb.out_stride = elems;
        const float2 *src;
        if (id < nl) {
            src = reinterpret_cast<const float2 *>(c.leaves[id]);
            cb.off = offs + (int64_t)inst0 * nl + id;
            cb.off_stride = nl;
        } else {
            src = inter_ptr(c, id - nl);
            cb.in_stride = size_of[id];
        }
        return gather(c, map, src, buf, cb);
    };
    // an operand gradient scattered back through the map that gathered the
    // operand: added into a leaf's gradient (alone) or stored into the
    // instance's own leaf buffer (groups); stored into an intermediate's
    auto scatter_op = [&](int id, const qcs_gather_t &g, int inst0, int Gc, const float2 *src,
                          int64_t elems) -> int {
        if (info) info->gather_count += Gc;
        ProfScope ps(h, kProfPermute);
        cudaError_t e;
        CopyBatch cb;
        cb.count = Gc;
        cb.in_stride = elems;
        if (!grp && id < nl) {
            float2 *dst = reinterpret_cast<float2 *>(d_grad_leaves[id]) +
                          tree->instance_offset[(int64_t)inst0 * nl + id];
            e = launch_scatter(g.rank, g.dims, g.strides, 0, src, dst, 1, s);
        } else if (id < nl) {
            cb.out_stride = L.lgrad_stride;
            cb.out_off = offs + (int64_t)inst0 * nl + id;
            cb.out_off_stride = nl;
            e = launch_scatter(g.rank, g.dims, g.strides, 0, src, lgrad + L.lgrad_off[id], 0, s, cb);
        } else {
            cb.out_stride = size_of[id];
            e = launch_scatter(g.rank, g.dims, g.strides, 0, src, grad_ptr(c, id - nl), 0, s, cb);
        }
        return e == cudaSuccess ? QCS_SUCCESS : QCS_ERR_CUDA;
    };
    // one adjoint GEMM for the group: a batched plain-FP32 launch, or one
    // grouped emulated sequence; operands and results sA, sB, sC apart
    auto adj_gemm = [&](int mode, int opA, int opB, int64_t m, int64_t n, int64_t k,
                        const float2 *A, int64_t lda, int64_t sA, const float2 *B, int64_t ldb,
                        int64_t sB, float2 *C, int64_t sC, int Gc) -> int {
        if (!grp) return gemm(c, mode, opA, opB, m, n, k, A, lda, B, ldb, C);
        const int eff = effective_mode(h, mode, opA, opB, m, n, k);
        count_gemm(c, eff, m, n, k, Gc);
        if (eff == QCS_MODE_FP32) {
            GemmBatch bt;
            bt.count = Gc;
            bt.sA = sA;
            bt.sB = sB;
            bt.sC = sC;
            return run_cgemm(h, c.ws + L.gemm, eff, opA, opB, m, n, k, make_float2(1.f, 0.f), A,
                             lda, B, ldb, make_float2(0.f, 0.f), C, m, nullptr, nullptr, bt);
        }
        std::vector<OperandView> va(Gc), vb(Gc);
        for (int g = 0; g < Gc; ++g) {
            va[g].X = A + g * sA;
            va[g].ld = lda;
            vb[g].X = B + g * sB;
            vb[g].ld = ldb;
        }
        return run_cgemm_group(h, c.ws + L.gemm, eff, opA, opB, m, n, k, make_float2(1.f, 0.f),
                               va.data(), vb.data(), Gc, make_float2(0.f, 0.f), C, m, sC, nullptr,
                               nullptr);
    };
    for (int inst0 = 0; inst0 < tree->n_instances; inst0 += G) {
        const int Gc = std::min(G, tree->n_instances - inst0);
        if (grp && cudaMemsetAsync(lgrad, 0, sizeof(float2) * (size_t)L.lgrad_stride * Gc, s) !=
                       cudaSuccess) {
            cudaGetLastError();
            return QCS_ERR_CUDA;
        }
        if (int r = forward_group(c, inst0, Gc, nullptr)) return r;
        // seed the roots' gradients
        if (ns > 0) {
            const int64_t rs = size_of[nl + ns - 1];
            float2 *groot = grad_ptr(c, ns - 1);
            if (cudaMemsetAsync(groot, 0, sizeof(float2) * rs * Gc, s) != cudaSuccess) {
                cudaGetLastError();
                return QCS_ERR_CUDA;
            }
            for (int r = 0; r < Gc; ++r) {
                const int64_t slot = tree->instance_slot[inst0 + r];
                if (launch_seed_grad(d_grad_out + 2 * slot * tree->out_size, dev_index(c),
                                     groot + r * rs, tree->out_size, s) != cudaSuccess)
                    return QCS_ERR_CUDA;
            }
        } else {  // a lone leaf (groups need a step)
            float2 *groot = reinterpret_cast<float2 *>(d_grad_leaves[0]) +
                            tree->instance_offset[(int64_t)inst0 * nl];
            const int64_t slot = tree->instance_slot[inst0];
            if (launch_seed_grad(d_grad_out + 2 * slot * tree->out_size, dev_index(c), groot,
                                 tree->out_size, s) != cudaSuccess)
                return QCS_ERR_CUDA;
        }
        // the steps in the reverse of the order the forward ran them: a
        // step's output gradient is complete once its consumer (a later step,
        // at a higher level) has run
        for (auto it = seq.rbegin(); it != seq.rend(); ++it) {
            if (it->step < 0) {
                if (info) {
                    info->level_launches++;
                    for (int q = it->first; q < it->first + it->count; ++q) {
                        const qcs_step_t &sp = tree->steps[L.small_order[q]];
                        count_gemm(c, QCS_MODE_FP32, sp.m, sp.k, sp.n, Gc);
                        count_gemm(c, QCS_MODE_FP32, sp.k, sp.n, sp.m, Gc);
                        info->level_gemms += 2 * Gc;
                    }
                }
                ProfScope ps(h, kProfGemmSimt);
                const auto *desc = reinterpret_cast<const TreeSmallBwd *>(c.ws + L.small_bwd) + it->first;
                if (launch_tree_small_bwd(desc, it->count, Gc, inst0, offs, nl,
                                          reinterpret_cast<const int32_t *>(c.ws + L.small_tab),
                                          it->smem_bwd, s) != cudaSuccess)
                    return QCS_ERR_CUDA;
                continue;
            }
            const qcs_step_t &st = tree->steps[it->step];
            const float2 *gC = grad_ptr(c, it->step);
            const int64_t mk = st.m * st.k, kn = st.k * st.n, mn = st.m * st.n;
            if (int r = gather_op(st.a, st.map_a, inst0, Gc, mk, Am)) return r;
            if (int r = gather_op(st.b, st.map_b, inst0, Gc, kn, Bm)) return r;
            // grad_A (m x k) = grad_out (m x n) B_mat^H ; grad_B (k x n) = A_mat^H grad_out
            if (int r = adj_gemm(st.mode, QCS_OP_N, QCS_OP_C, st.m, st.k, st.n, gC, st.m, mn, Bm,
                                 st.k, kn, gA, mk, Gc))
                return r;
            if (int r = adj_gemm(st.mode, QCS_OP_C, QCS_OP_N, st.k, st.n, st.m, Am, st.m, mk, gC,
                                 st.m, mn, gB, kn, Gc))
                return r;
            if (int r = scatter_op(st.a, st.map_a, inst0, Gc, gA, mk)) return r;
            if (int r = scatter_op(st.b, st.map_b, inst0, Gc, gB, kn)) return r;
        }
        // the group's leaf gradients into the caller's, in instance order
        if (grp && launch_leaf_grad_reduce(reinterpret_cast<const LeafGradRef *>(c.ws + L.leaf_tab),
                                           nl, L.max_leaf, lgrad, L.lgrad_stride, Gc, s) !=
                       cudaSuccess)
            return QCS_ERR_CUDA;
    }
    return QCS_SUCCESS;
}

// Pointers present and 8-byte aligned, and the leaf gradients pairwise
// disjoint (the adjoints of independent steps add into them at once).
bool backward_args_ok(const qcs_tree_t *tree, const qcs_c32 *const *leaves,
                      qcs_c32 *const *d_grad_leaves) {
    if (!tree->leaf_size) return false;
    std::vector<std::pair<uintptr_t, uintptr_t>> spans;
    for (int i = 0; i < tree->n_leaves; ++i) {
        if (!leaves[i] || !d_grad_leaves[i] || (reinterpret_cast<uintptr_t>(leaves[i]) & 7u) ||
            (reinterpret_cast<uintptr_t>(d_grad_leaves[i]) & 7u) || tree->leaf_size[i] < 1)
            return false;
        const uintptr_t lo = reinterpret_cast<uintptr_t>(d_grad_leaves[i]);
        spans.emplace_back(lo, lo + sizeof(qcs_c32) * (uintptr_t)tree->leaf_size[i]);
    }
    std::sort(spans.begin(), spans.end());
    for (size_t i = 1; i < spans.size(); ++i)
        if (spans[i].first < spans[i - 1].second) return false;
    return true;
}

}  // namespace
}  // namespace qcs

struct qcs_tree_graph_s {
    qcs_handle_t h = nullptr;
    qcs::Workspace ws;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

using namespace qcs;

extern "C" {

int qcs_contract_tree(qcs_handle_t h, const qcs_tree_t *tree, const qcs_c32 *const *leaves,
                      double *d_out, qcs_run_info_t *info) {
    if (!h || !tree || !leaves || !d_out) return QCS_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    if (info) *info = qcs_run_info_t{};
    for (int i = 0; i < tree->n_leaves; ++i)
        if (!leaves[i] || (reinterpret_cast<uintptr_t>(leaves[i]) & 7u)) return QCS_ERR_INVALID_ARG;
    Ctx c;
    c.leaves = leaves;
    c.info = info;
    if (int r = begin(h, tree, false, c)) return r;
    if (int r = forward_all(c, d_out)) return r;
    if (info)
        info->seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return QCS_SUCCESS;
}

int qcs_contract_tree_backward(qcs_handle_t h, const qcs_tree_t *tree,
                               const qcs_c32 *const *leaves, const double *d_grad_out,
                               qcs_c32 *const *d_grad_leaves, qcs_run_info_t *info) {
    if (!h || !tree || !leaves || !d_grad_out || !d_grad_leaves) return QCS_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    if (info) *info = qcs_run_info_t{};
    if (tree->n_leaves >= 1 && !backward_args_ok(tree, leaves, d_grad_leaves))
        return QCS_ERR_INVALID_ARG;
    Ctx c;
    c.leaves = leaves;
    c.grad_leaves = d_grad_leaves;
    c.info = info;
    if (int r = begin(h, tree, true, c)) return r;
    if (int r = backward_all(c, d_grad_out, d_grad_leaves)) return r;
    if (info)
        info->seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return QCS_SUCCESS;
}

int qcs_tree_backward_graph_create(qcs_handle_t h, const qcs_tree_t *tree,
                                   const qcs_c32 *const *leaves, const double *d_grad_out,
                                   qcs_c32 *const *d_grad_leaves, qcs_tree_graph_t *out) {
    if (!h || !tree || !leaves || !d_grad_out || !d_grad_leaves || !out) return QCS_ERR_INVALID_ARG;
    *out = nullptr;
    if (tree->n_leaves >= 1 && !backward_args_ok(tree, leaves, d_grad_leaves))
        return QCS_ERR_INVALID_ARG;
    qcs_tree_graph_s *g = new (std::nothrow) qcs_tree_graph_s;
    if (!g) return QCS_ERR_ALLOC;
    g->h = h;
    Ctx c;
    c.leaves = leaves;
    c.grad_leaves = d_grad_leaves;
    c.info = nullptr;
    int r = begin(h, tree, true, c, &g->ws);
    if (r == QCS_SUCCESS && cudaStreamSynchronize(h->stream) != cudaSuccess) r = QCS_ERR_CUDA;
    const int profiling = h->profiling;
    cudaStream_t user = h->stream, cap = nullptr;
    h->profiling = 0;
    if (r == QCS_SUCCESS && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
        r = QCS_ERR_CUDA;
    if (r == QCS_SUCCESS) {
        h->stream = cap;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            r = QCS_ERR_CUDA;
        } else {
            const int rb = backward_all(c, d_grad_out, d_grad_leaves);
            const cudaError_t e = cudaStreamEndCapture(cap, &g->graph);
            r = rb ? rb : (e == cudaSuccess ? QCS_SUCCESS : QCS_ERR_CUDA);
        }
    }
    h->stream = user;
    h->profiling = profiling;
    if (cap) cudaStreamDestroy(cap);
    if (r == QCS_SUCCESS && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess)
        r = QCS_ERR_CUDA;
    if (r != QCS_SUCCESS) {
        cudaGetLastError();
        if (g->graph) cudaGraphDestroy(g->graph);
        if (g->ws.ptr) cudaFree(g->ws.ptr);
        delete g;
        return r;
    }
    *out = g;
    return QCS_SUCCESS;
}

int qcs_tree_layout_info(const qcs_tree_t *tree, int backward, int instance_batch, int levels,
                         int num_sms, uint64_t group_budget, int64_t *step_offset,
                         int64_t *step_bytes, int32_t *step_time, int32_t *step_small,
                         int32_t *step_order, qcs_tree_layout_t *out) {
    if (!tree || !out || instance_batch < 1 || num_sms < 1 || (levels != 0 && levels != 1))
        return QCS_ERR_INVALID_ARG;
    std::vector<int64_t> size_of;
    if (int r = validate(tree, size_of, backward != 0)) return r;
    // a handle that never touches a device: the paper's size rule, no tuning
    qcs_handle_s h;
    h.num_sms = num_sms;
    h.tree_levels = levels;
    h.group_budget = (size_t)group_budget;
    const int ns = tree->n_steps;
    const int G = std::max(1, std::min(instance_batch, tree->n_instances));
    Layout L = plan_layout(&h, tree, backward != 0, G);
    if (backward && G > 1 && (ns == 0 || L.P < ns)) L = plan_layout(&h, tree, true, 1);
    for (int s = 0; s < ns; ++s) {
        if (step_offset) step_offset[s] = (int64_t)L.inter_off[s];
        if (step_bytes)
            step_bytes[s] = (int64_t)(sizeof(float2) * tree->steps[s].m * tree->steps[s].n *
                                      (L.batched[s] ? L.G : 1));
        if (step_time) step_time[s] = L.time[s];
        if (step_small) step_small[s] = L.small[s];
    }
    if (step_order) {
        int q = 0;
        for (const std::vector<Item> *seq : {&L.seq_b, &L.seq_i})
            for (const Item &it : *seq) {
                if (it.step >= 0) {
                    step_order[q++] = it.step;
                } else {
                    for (int i = it.first; i < it.first + it.count; ++i)
                        step_order[q++] = L.small_order[i];
                }
            }
    }
    *out = qcs_tree_layout_t{};
    out->total_bytes = (int64_t)L.total;
    out->group = L.G;
    out->batched_steps = L.P;
    int launches = 0;
    for (const std::vector<Item> *seq : {&L.seq_b, &L.seq_i})
        for (const Item &it : *seq) launches += it.step < 0 ? 1 : 0;
    out->level_launches = launches;
    return QCS_SUCCESS;
}

int qcs_autotune_tree(qcs_handle_t h, const qcs_tree_t *tree, int backward, int reps,
                      int64_t *n_tuned) {
    if (n_tuned) *n_tuned = 0;
    if (!h || !tree || reps < 1) return QCS_ERR_INVALID_ARG;
    std::vector<int64_t> size_of;
    if (int r = validate(tree, size_of, backward != 0)) return r;
    // The (m, n, k, opA, opB) of every AUTO GEMM the executor issues: the
    // forward GEMM of each step (op T for a direct transposed operand,
    // else N) and, for the adjoint, grad_A = grad_out B_mat^H and
    // grad_B = A_mat^H grad_out on gathered operands.
    std::set<std::tuple<int64_t, int64_t, int64_t, int, int>> keys;
    for (int s = 0; s < tree->n_steps; ++s) {
        const qcs_step_t &st = tree->steps[s];
        if (st.mode != QCS_MODE_AUTO) continue;
        keys.insert(std::make_tuple(st.m, st.n, st.k,
                                    st.direct_a == QCS_OP_T ? (int)QCS_OP_T : (int)QCS_OP_N,
                                    st.direct_b == QCS_OP_T ? (int)QCS_OP_T : (int)QCS_OP_N));
        if (backward) {
            keys.insert(std::make_tuple(st.m, st.k, st.n, (int)QCS_OP_N, (int)QCS_OP_C));
            keys.insert(std::make_tuple(st.k, st.n, st.m, (int)QCS_OP_C, (int)QCS_OP_N));
        }
    }
    int64_t count = 0;
    for (const auto &key : keys) {
        if (h->tuned.count(key)) continue;
        const int64_t m = std::get<0>(key), n = std::get<1>(key), k = std::get<2>(key);
        if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) continue;
        if (int r = tune_shape(h, std::get<3>(key), std::get<4>(key), m, n, k, reps, nullptr))
            return r;
        ++count;
    }
    if (n_tuned) *n_tuned = count;
    return QCS_SUCCESS;
}

int qcs_tree_graph_create(qcs_handle_t h, const qcs_tree_t *tree, const qcs_c32 *const *leaves,
                          double *d_out, qcs_tree_graph_t *out) {
    if (!h || !tree || !leaves || !d_out || !out) return QCS_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < tree->n_leaves; ++i)
        if (!leaves[i] || (reinterpret_cast<uintptr_t>(leaves[i]) & 7u)) return QCS_ERR_INVALID_ARG;
    qcs_tree_graph_s *g = new (std::nothrow) qcs_tree_graph_s;
    if (!g) return QCS_ERR_ALLOC;
    g->h = h;
    Ctx c;
    c.leaves = leaves;
    c.info = nullptr;
    // begin() validates, allocates the graph's workspace and uploads the
    // output index, all before the capture starts.
    int r = begin(h, tree, false, c, &g->ws);
    if (r == QCS_SUCCESS && cudaStreamSynchronize(h->stream) != cudaSuccess) r = QCS_ERR_CUDA;
    // Capture on a private stream (the legacy default stream cannot be
    // captured); the instantiated graph then launches on the handle's stream.
    const int profiling = h->profiling;
    cudaStream_t user = h->stream, cap = nullptr;
    h->profiling = 0;
    if (r == QCS_SUCCESS && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
        r = QCS_ERR_CUDA;
    if (r == QCS_SUCCESS) {
        h->stream = cap;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            r = QCS_ERR_CUDA;
        } else {
            const int rf = forward_all(c, d_out);
            const cudaError_t e = cudaStreamEndCapture(cap, &g->graph);
            r = rf ? rf : (e == cudaSuccess ? QCS_SUCCESS : QCS_ERR_CUDA);
        }
    }
    h->stream = user;
    h->profiling = profiling;
    if (cap) cudaStreamDestroy(cap);
    if (r == QCS_SUCCESS && cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess)
        r = QCS_ERR_CUDA;
    if (r != QCS_SUCCESS) {
        cudaGetLastError();
        if (g->graph) cudaGraphDestroy(g->graph);
        if (g->ws.ptr) cudaFree(g->ws.ptr);
        delete g;
        return r;
    }
    *out = g;
    return QCS_SUCCESS;
}

int qcs_tree_graph_launch(qcs_tree_graph_t g) {
    if (!g || !g->exec) return QCS_ERR_INVALID_ARG;
    return cudaGraphLaunch(g->exec, g->h->stream) == cudaSuccess ? QCS_SUCCESS : QCS_ERR_CUDA;
}

int qcs_tree_graph_destroy(qcs_tree_graph_t g) {
    if (!g) return QCS_ERR_INVALID_ARG;
    cudaStreamSynchronize(g->h->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->ws.ptr) cudaFree(g->ws.ptr);
    delete g;
    return QCS_SUCCESS;
}

}  // extern "C"
