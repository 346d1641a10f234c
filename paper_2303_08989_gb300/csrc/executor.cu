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
// accumulated in FP64 into its output slot.
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

struct Layout {
    std::vector<size_t> inter_off;  // byte offset of each step's output
    std::vector<size_t> grad_off;   // byte offset of each step's output gradient (backward)
    size_t out_index = 0, bufA = 0, bufB = 0, tmpA = 0, tmpB = 0, gemm = 0, total = 0;
    size_t gemm_bytes = 0;
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
    const int64_t rs = root_size(t, size_of);
    if (t->out_index) {
        for (int64_t j = 0; j < t->out_size; ++j)
            if (t->out_index[j] < 0 || t->out_index[j] >= rs) return QCS_ERR_INVALID_ARG;
    } else if (rs != t->out_size) {
        return QCS_ERR_INVALID_ARG;
    }
    if (ns == 0 && max_off[0] + t->out_size > size_of[0] && !t->out_index) return QCS_ERR_INVALID_ARG;
    if (need_tree) {
        for (int i = 0; i < nl + ns - 1; ++i)
            if (uses[i] != 1) return QCS_ERR_INVALID_ARG;
        if (ns > 0 && uses[nl + ns - 1] != 0) return QCS_ERR_INVALID_ARG;
    }
    return QCS_SUCCESS;
}

Layout plan_layout(qcs_handle_t h, const qcs_tree_t *t, bool backward) {
    Layout L;
    const int nl = t->n_leaves, ns = t->n_steps;
    size_t p = 0;
    L.out_index = p;
    p += align256(sizeof(int64_t) * (t->out_index ? t->out_size : 1));
    int64_t maxA = 1, maxB = 1;
    size_t gemm = 0;
    L.inter_off.resize(ns);
    for (int s = 0; s < ns; ++s) {
        const qcs_step_t &st = t->steps[s];
        L.inter_off[s] = p;
        p += align256(sizeof(float2) * st.m * st.n);
        maxA = std::max(maxA, st.m * st.k);
        maxB = std::max(maxB, st.k * st.n);
        const int opA = st.direct_a == QCS_OP_T ? QCS_OP_T : QCS_OP_N;
        const int opB = st.direct_b == QCS_OP_T ? QCS_OP_T : QCS_OP_N;
        gemm = std::max(gemm, gemm_workspace_bytes(effective_mode(h, st.mode, opA, opB, st.m, st.n,
                                                                  st.k),
                                                   st.m, st.n, st.k, h->num_sms));
        if (backward) {
            gemm = std::max(gemm, gemm_workspace_bytes(effective_mode(h, st.mode, QCS_OP_N,
                                                                      QCS_OP_C, st.m, st.k, st.n),
                                                       st.m, st.k, st.n, h->num_sms));
            gemm = std::max(gemm, gemm_workspace_bytes(effective_mode(h, st.mode, QCS_OP_C,
                                                                      QCS_OP_N, st.k, st.n, st.m),
                                                       st.k, st.n, st.m, h->num_sms));
        }
    }
    (void)nl;
    L.bufA = p;
    p += align256(sizeof(float2) * maxA);
    L.bufB = p;
    p += align256(sizeof(float2) * maxB);
    if (backward) {
        L.grad_off.resize(ns);
        for (int s = 0; s < ns; ++s) {
            L.grad_off[s] = p;
            p += align256(sizeof(float2) * t->steps[s].m * t->steps[s].n);
        }
        L.tmpA = p;
        p += align256(sizeof(float2) * maxA);
        L.tmpB = p;
        p += align256(sizeof(float2) * maxB);
    }
    L.gemm = p;
    L.gemm_bytes = gemm;
    p += align256(gemm);
    L.total = p;
    return L;
}

struct Ctx {
    qcs_handle_t h;
    const qcs_tree_t *t;
    const qcs_c32 *const *leaves;
    uint8_t *ws;
    Layout L;
    qcs_run_info_t *info;
};

float2 *inter_ptr(const Ctx &c, int s) { return reinterpret_cast<float2 *>(c.ws + c.L.inter_off[s]); }
float2 *grad_ptr(const Ctx &c, int s) { return reinterpret_cast<float2 *>(c.ws + c.L.grad_off[s]); }

const float2 *tensor_ptr(const Ctx &c, int id, int inst) {
    const int nl = c.t->n_leaves;
    if (id < nl)
        return reinterpret_cast<const float2 *>(c.leaves[id]) +
               c.t->instance_offset[(int64_t)inst * nl + id];
    return inter_ptr(c, id - nl);
}

void count_gemm(const Ctx &c, int eff, int64_t m, int64_t n, int64_t k) {
    if (!c.info) return;
    c.info->gemm_count++;
    if (eff >= 0 && eff < 6) c.info->mode_count[eff]++;
    c.info->flops += 8.0 * (double)m * (double)n * (double)k;
}

int gather(const Ctx &c, const qcs_gather_t &g, const float2 *src, float2 *dst) {
    if (c.info) c.info->gather_count++;
    ProfScope ps(c.h, kProfPermute);
    return launch_permute(g.rank, g.dims, g.strides, 0, src, dst, nullptr, 0, c.h->stream) ==
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

// Forward pass of one instance: every step's output into its slot.
int forward_instance(const Ctx &c, int inst) {
    const qcs_tree_t *t = c.t;
    for (int s = 0; s < t->n_steps; ++s) {
        const qcs_step_t &st = t->steps[s];
        const float2 *A = tensor_ptr(c, st.a, inst);
        const float2 *B = tensor_ptr(c, st.b, inst);
        int opA = QCS_OP_N, opB = QCS_OP_N;
        int64_t lda = st.m, ldb = st.k;
        if (st.direct_a == -1) {
            float2 *buf = reinterpret_cast<float2 *>(c.ws + c.L.bufA);
            if (int r = gather(c, st.map_a, A, buf)) return r;
            A = buf;
        } else if (st.direct_a == QCS_OP_T) {
            opA = QCS_OP_T;
            lda = st.k;
        }
        if (st.direct_b == -1) {
            float2 *buf = reinterpret_cast<float2 *>(c.ws + c.L.bufB);
            if (int r = gather(c, st.map_b, B, buf)) return r;
            B = buf;
        } else if (st.direct_b == QCS_OP_T) {
            opB = QCS_OP_T;
            ldb = st.n;
        }
        if (int r = gemm(c, st.mode, opA, opB, st.m, st.n, st.k, A, lda, B, ldb, inter_ptr(c, s)))
            return r;
    }
    return QCS_SUCCESS;
}

const float2 *root_ptr(const Ctx &c, int inst) {
    return c.t->n_steps > 0 ? inter_ptr(c, c.t->n_steps - 1) : tensor_ptr(c, 0, inst);
}

int begin(qcs_handle_t h, const qcs_tree_t *t, bool backward, std::vector<int64_t> &size_of,
          Ctx &c, Workspace *own = nullptr) {
    if (int r = validate(t, size_of, backward)) return r;
    c.h = h;
    c.t = t;
    c.L = plan_layout(h, t, backward);
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
    if (c.info) c.info->workspace_bytes = (int64_t)c.L.total;
    return QCS_SUCCESS;
}

const int64_t *dev_index(const Ctx &c) {
    return c.t->out_index ? reinterpret_cast<const int64_t *>(c.ws + c.L.out_index) : nullptr;
}

// Every launch of a forward call after begin(): clear d_out, then per
// instance the steps and the FP64 accumulation of the root.
int forward_all(const Ctx &c, double *d_out) {
    const qcs_tree_t *tree = c.t;
    qcs_handle_t h = c.h;
    if (cudaMemsetAsync(d_out, 0, sizeof(double) * 2 * tree->n_slots * tree->out_size, h->stream) !=
        cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    for (int inst = 0; inst < tree->n_instances; ++inst) {
        if (int r = forward_instance(c, inst)) return r;
        ProfScope ps(h, kProfReduce);
        const int64_t slot = tree->instance_slot[inst];
        if (launch_accumulate_gather_c128(root_ptr(c, inst), dev_index(c),
                                          d_out + 2 * slot * tree->out_size, tree->out_size,
                                          h->stream) != cudaSuccess)
            return QCS_ERR_CUDA;
    }
    return QCS_SUCCESS;
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
    std::vector<int64_t> size_of;
    Ctx c;
    c.leaves = leaves;
    c.info = info;
    if (int r = begin(h, tree, false, size_of, c)) return r;
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
    for (int i = 0; i < tree->n_leaves; ++i)
        if (!leaves[i] || !d_grad_leaves[i] || (reinterpret_cast<uintptr_t>(leaves[i]) & 7u) ||
            (reinterpret_cast<uintptr_t>(d_grad_leaves[i]) & 7u))
            return QCS_ERR_INVALID_ARG;
    std::vector<int64_t> size_of;
    Ctx c;
    c.leaves = leaves;
    c.info = info;
    if (int r = begin(h, tree, true, size_of, c)) return r;
    const int nl = tree->n_leaves, ns = tree->n_steps;
    cudaStream_t s = h->stream;
    auto scatter_into = [&](int id, int inst, const qcs_gather_t &g, const float2 *src) -> int {
        if (info) info->gather_count++;
        ProfScope ps(h, kProfPermute);
        cudaError_t e;
        if (id < nl) {
            float2 *dst = reinterpret_cast<float2 *>(d_grad_leaves[id]) +
                          tree->instance_offset[(int64_t)inst * nl + id];
            e = launch_scatter(g.rank, g.dims, g.strides, 0, src, dst, 1, s);
        } else {
            e = launch_scatter(g.rank, g.dims, g.strides, 0, src, grad_ptr(c, id - nl), 0, s);
        }
        return e == cudaSuccess ? QCS_SUCCESS : QCS_ERR_CUDA;
    };
    for (int inst = 0; inst < tree->n_instances; ++inst) {
        if (int r = forward_instance(c, inst)) return r;
        const int64_t slot = tree->instance_slot[inst];
        const double *g = d_grad_out + 2 * slot * tree->out_size;
        // seed the root's gradient
        float2 *groot;
        if (ns > 0) {
            groot = grad_ptr(c, ns - 1);
            if (cudaMemsetAsync(groot, 0, sizeof(float2) * size_of[nl + ns - 1], s) != cudaSuccess) {
                cudaGetLastError();
                return QCS_ERR_CUDA;
            }
        } else {
            groot = reinterpret_cast<float2 *>(d_grad_leaves[0]) + tree->instance_offset[(int64_t)inst * nl];
        }
        if (launch_seed_grad(g, dev_index(c), groot, tree->out_size, s) != cudaSuccess)
            return QCS_ERR_CUDA;
        for (int st_i = ns - 1; st_i >= 0; --st_i) {
            const qcs_step_t &st = tree->steps[st_i];
            const float2 *gC = grad_ptr(c, st_i);
            float2 *Am = reinterpret_cast<float2 *>(c.ws + c.L.bufA);
            float2 *Bm = reinterpret_cast<float2 *>(c.ws + c.L.bufB);
            float2 *gA = reinterpret_cast<float2 *>(c.ws + c.L.tmpA);
            float2 *gB = reinterpret_cast<float2 *>(c.ws + c.L.tmpB);
            if (int r = gather(c, st.map_a, tensor_ptr(c, st.a, inst), Am)) return r;
            if (int r = gather(c, st.map_b, tensor_ptr(c, st.b, inst), Bm)) return r;
            // grad_A (m x k) = grad_out (m x n) B_mat^H ; grad_B (k x n) = A_mat^H grad_out
            if (int r = gemm(c, st.mode, QCS_OP_N, QCS_OP_C, st.m, st.k, st.n, gC, st.m, Bm, st.k, gA))
                return r;
            if (int r = gemm(c, st.mode, QCS_OP_C, QCS_OP_N, st.k, st.n, st.m, Am, st.m, gC, st.m, gB))
                return r;
            if (int r = scatter_into(st.a, inst, st.map_a, gA)) return r;
            if (int r = scatter_into(st.b, inst, st.map_b, gB)) return r;
        }
    }
    if (info)
        info->seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
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
    std::vector<int64_t> size_of;
    Ctx c;
    c.leaves = leaves;
    c.info = nullptr;
    // begin() validates, allocates the graph's workspace and uploads the
    // output index, all before the capture starts.
    int r = begin(h, tree, false, size_of, c, &g->ws);
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
