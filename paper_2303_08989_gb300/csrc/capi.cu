// C ABI (include/qcs.h): argument validation, workspace, tensor-map encoding
// and the launch sequence of one emulated CGEMM:
//
//   stats(A) + stats(B)  -- one launch, one HBM pass over each operand
//   select               -- mode flag / scale descriptor on the device
//   split(A), split(B)   -- Eq. 1 planes (kernel exits for mode FP32)
//   tcgen05 FP16 kernel  -- exits unless FP16X / FP16X_SCALED was selected
//   tcgen05 TF32 kernel  -- exits unless TF32X was selected
//   SIMT FP32 kernel     -- exits unless FP32 was selected
//
// i.e. the host never learns the mode: every candidate is launched and the
// ones not selected return at once (Section 4.2).
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <new>

#include "internal.h"

using namespace qcs;

namespace qcs {

int ensure_workspace(Workspace &w, size_t bytes) {
    if (bytes <= w.bytes) return QCS_SUCCESS;
    if (w.ptr) {
        cudaFree(w.ptr);
        w.ptr = nullptr;
        w.bytes = 0;
    }
    // grow with some headroom so that a sweep of sizes does not reallocate each call
    const size_t want = bytes + bytes / 8;
    if (cudaMalloc(&w.ptr, want) != cudaSuccess) {
        cudaGetLastError();
        w.ptr = nullptr;
        return QCS_ERR_ALLOC;
    }
    w.bytes = want;
    return QCS_SUCCESS;
}

static cudaEvent_t pool_get(qcs_handle_s *h) {
    if (!h->event_pool.empty()) {
        cudaEvent_t e = h->event_pool.back();
        h->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

ProfScope::ProfScope(qcs_handle_s *h, int stage) : h_(h) {
    if (!h_->profiling) return;
    ProfEvent pe{stage, pool_get(h_), pool_get(h_)};
    if (!pe.start || !pe.stop) return;
    cudaEventRecord(pe.start, h_->stream);
    h_->prof.push_back(pe);
    idx_ = static_cast<int>(h_->prof.size()) - 1;
}

ProfScope::~ProfScope() {
    if (idx_ >= 0) cudaEventRecord(h_->prof[idx_].stop, h_->stream);
}

}  // namespace qcs

namespace {

inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int cuda_status(cudaError_t e) { return e == cudaSuccess ? QCS_SUCCESS : QCS_ERR_CUDA; }

// Number of stats blocks for a matrix of ``nel`` complex values.
int stats_blocks(int64_t nel, int num_sms) {
    const int64_t per_block = int64_t(kStatsThreads) * 64;  // complex values per block, minimum
    int64_t g = (nel + per_block - 1) / per_block;
    g = std::max<int64_t>(1, std::min<int64_t>(g, num_sms));
    return static_cast<int>(g);
}

}  // namespace

// Blocks of the two-stage statistics for ``nel`` complex values: up to four
// 256-thread blocks per SM, at least 2048 complex values per block.
int qcs::stats2_blocks(int64_t nel, int num_sms) {
    int64_t g = (nel + 2047) / 2048;
    g = std::max<int64_t>(1, std::min<int64_t>(g, 4 * (int64_t)num_sms));
    return static_cast<int>(g);
}

namespace {

// Tensor map of one operand's planes: {K, R, nplanes}, box = one stage of all
// planes (kRowBytes of K x 128 rows), 64-byte swizzle (the layout the
// kernel's shared-memory descriptors describe).
int encode_planes(qcs_handle_t h, CUtensorMap *map, void *base, int64_t R_pad, int64_t K_pad,
                  int esz, int nplanes, int box_rows = kBM, int box_planes = 0) {
    const CUtensorMapDataType dt =
        esz == 2 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t gdim[3] = {(cuuint64_t)K_pad, (cuuint64_t)R_pad, (cuuint64_t)nplanes};
    cuuint64_t gstride[2] = {(cuuint64_t)(K_pad * esz), (cuuint64_t)(K_pad * R_pad * esz)};
    cuuint32_t box[3] = {(cuuint32_t)(kRowBytes / esz), (cuuint32_t)box_rows,
                         (cuuint32_t)(box_planes > 0 ? box_planes : nplanes)};
    cuuint32_t estride[3] = {1, 1, 1};
    const CUtensorMapL2promotion promo =
        h->tc_l2_promotion >= 256 ? CU_TENSOR_MAP_L2_PROMOTION_L2_256B
        : h->tc_l2_promotion >= 128 ? CU_TENSOR_MAP_L2_PROMOTION_L2_128B
        : h->tc_l2_promotion >= 64  ? CU_TENSOR_MAP_L2_PROMOTION_L2_64B
                                    : CU_TENSOR_MAP_L2_PROMOTION_NONE;
    CUresult r = h->encode(map, dt, 3, base, gdim, gstride, box, estride,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, promo,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? QCS_SUCCESS : QCS_ERR_CUDA;
}

bool valid_op(int op) { return op == QCS_OP_N || op == QCS_OP_T || op == QCS_OP_C; }
bool valid_mode(int m) { return m >= QCS_MODE_AUTO && m <= QCS_MODE_BF16X3; }

// Plane strides of op(X) for the split: element (r, c) of the plane is
// X[r * sr + c * sc].  For the A operand r = i, c = l (op(A) is m x k);
// for the B operand r = j, c = l (op(B) is k x n).
void plane_strides(int which, int op, int64_t ld, int64_t &sr, int64_t &sc) {
    if (which == 0) {
        if (op == QCS_OP_N) { sr = 1; sc = ld; } else { sr = ld; sc = 1; }
    } else {
        if (op == QCS_OP_N) { sr = ld; sc = 1; } else { sr = 1; sc = ld; }
    }
}

}  // namespace

// Effective mode after the size rule (host side, sizes are known on the host).
int qcs::effective_mode(qcs_handle_t h, int mode, int opA, int opB, int64_t m, int64_t n,
                        int64_t k) {
    if (mode != QCS_MODE_AUTO || h->size_rule == QCS_SIZE_RULE_OFF) return mode;
    if (h->size_rule == QCS_SIZE_RULE_TUNED) {
        const auto it = h->tuned.find(std::make_tuple(m, n, k, opA, opB));
        if (it != h->tuned.end()) return it->second.best;
    }
    const int64_t s = std::min(m, std::min(n, k));
    if (s >= 2048) return QCS_MODE_AUTO;
    if (s >= 512) return QCS_MODE_TF32X;
    return QCS_MODE_FP32;
}

// K ranges of a tensor-core GEMM of this shape: the count qcs_set_tc_splits
// forces, else the count the tuner measured for the shape (under the tuned
// size rule), else 0 (tc_split_count's per-shape rule).
int qcs::gemm_splits(qcs_handle_t h, int opA, int opB, int64_t m, int64_t n, int64_t k) {
    if (h->tc_splits > 0) return h->tc_splits;
    if (h->size_rule == QCS_SIZE_RULE_TUNED) {
        const auto it = h->tuned.find(std::make_tuple(m, n, k, opA, opB));
        if (it != h->tuned.end() && it->second.splits > 0) return it->second.splits;
    }
    return 0;
}

// Raster of a tensor-core GEMM of this shape: the group the tuner measured
// for it (under the tuned size rule), else the handle's schedule.
int qcs::gemm_group_m(qcs_handle_t h, int opA, int opB, int64_t m, int64_t n, int64_t k) {
    if (h->size_rule == QCS_SIZE_RULE_TUNED) {
        const auto it = h->tuned.find(std::make_tuple(m, n, k, opA, opB));
        if (it != h->tuned.end() && it->second.group_m > 0) return it->second.group_m;
    }
    return h->tc_group_m;
}

// The whole emulated CGEMM on the handle's stream.  desc_ws/partials/planes
// come from ``ws`` (a device buffer of at least gemm_workspace_bytes()).
namespace qcs {

namespace {

// Byte offsets, from the start of the plane area, of the split planes of a
// group of G GEMMs and of the K-range partials.  A group whose instances may
// select different kinds (AUTO, G > 1) keeps 2-byte and 4-byte planes apart
// (instance g's rows sit at the same element offset in either, which in
// bytes depends on the kind); otherwise one region serves the selected kind.
struct PlaneLayout {
    size_t a16 = 0, b16 = 0, a32 = 0, b32 = 0, partials = 0, total = 0;
};

PlaneLayout plane_layout(int eff, int64_t m, int64_t n, int64_t k, int G, int S) {
    PlaneLayout L;
    const bool need16 = (eff == QCS_MODE_AUTO || eff == QCS_MODE_FP16X ||
                         eff == QCS_MODE_FP16X_SCALED || eff == QCS_MODE_BF16X3);
    const bool need32 = (eff == QCS_MODE_AUTO || eff == QCS_MODE_TF32X);
    const int64_t kp = round_up(k, 32), mp = round_up(m, kBM), np = round_up(n, kBN);
    size_t off = 0;
    auto region = [&](int esz, int planes, int64_t rows) {
        const size_t o = off;
        off += align256(size_t(planes) * G * rows * kp * esz);
        return o;
    };
    if (G > 1 && need16 && need32) {
        L.a16 = region(2, kPlanes, mp);
        L.b16 = region(2, kPlanesB, np);
        L.a32 = region(4, kPlanes, mp);
        L.b32 = region(4, kPlanesB, np);
    } else {
        const int esz = need32 ? 4 : 2;
        L.a16 = L.a32 = region(esz, kPlanes, mp);
        L.b16 = L.b32 = region(esz, kPlanesB, np);
    }
    if (S > 1) {
        L.partials = off;
        off += align256(sizeof(float2) * S * G * m * n);
    }
    L.total = off;
    return L;
}

}  // namespace

size_t gemm_workspace_bytes(int eff, int64_t m, int64_t n, int64_t k, int num_sms, int splits,
                            int G) {
    size_t bytes = align256(sizeof(qcs_gemm_desc_t) * G);  // descriptors
    bytes += align256(size_t(2) * num_sms * kPartialStride * sizeof(int64_t));
    bytes += align256(kSplitKBytes);
    if (eff != QCS_MODE_FP32)
        bytes += plane_layout(eff, m, n, k, G, tc_split_count(m, n, k, 1, num_sms, splits)).total;
    return bytes;
}

int run_cgemm(qcs_handle_t h, void *ws, int eff, int opA, int opB, int64_t m, int64_t n, int64_t k,
              float2 alpha, const float2 *A, int64_t lda, const float2 *B, int64_t ldb, float2 beta,
              float2 *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out, const qcs_gemm_desc_t *d_desc_in,
              const GemmBatch &bt) {
    OperandView va, vb;
    va.X = A;
    va.ld = lda;
    vb.X = B;
    vb.ld = ldb;
    return run_cgemm_views(h, ws, eff, opA, opB, m, n, k, alpha, va, vb, beta, C, ldc, d_desc_out,
                           d_desc_in, bt);
}

namespace {

// Gather op(X) of a mapped view into its buffer (only if the GEMM selected
// FP32 when gate is not NULL); the view then reads it as a matrix.
int gather_view(qcs_handle_t h, OperandView &v, int64_t rows, const qcs_gemm_desc_t *gate) {
    ProfScope ps(h, kProfPermute);
    CopyBatch cb;
    cb.gate = gate;
    if (launch_permute(v.map->rank, v.map->dims, v.map->strides, 0, v.X, v.buf, nullptr, 0,
                       h->stream, cb) != cudaSuccess)
        return QCS_ERR_CUDA;
    v.X = v.buf;
    v.ld = rows;
    v.map = nullptr;
    return QCS_SUCCESS;
}

// The split of one operand (which 0: op(A), R = m; 1: op(B), R = n) into
// its planes: through its map (fused), or from the matrix.  The split
// writes with the selected kind's element size; the pitch is kp elements
// either way, so both tensor maps of the GEMM describe it.  Instance g of a
// group owns rows [g R_pad, (g + 1) R_pad) of every plane.
int split_operand(qcs_handle_t h, int which, const qcs_gemm_desc_t *dg, const OperandView &X,
                  int op, int64_t R, int64_t k, int64_t R_pad, int64_t kp, void *planes,
                  int64_t plane_stride, int64_t plane_off, void *planes32, bool fused,
                  bool tf32_fused, const SplitBatch &sb) {
    ProfScope ps(h, kProfSplit);
    cudaError_t e;
    if (fused) {
        e = launch_split_gather(dg, which, X.map->rank, X.map->dims, X.map->strides, X.X,
                                which == 0 ? R : k, planes, kp, plane_stride, h->stream, which,
                                plane_off, planes32, sb);
    } else {
        int64_t sr, sc;
        plane_strides(which, op, X.ld, sr, sc);
        e = launch_split(dg, which, X.X, sr, sc, op == QCS_OP_C, R, k, R_pad, kp, planes, kp,
                         plane_stride, h->stream, which, plane_off, planes32, tf32_fused ? 1 : 0,
                         sb, h->line_emax[which]);
    }
    return e == cudaSuccess ? QCS_SUCCESS : QCS_ERR_CUDA;
}

}  // namespace

int run_cgemm_views(qcs_handle_t h, void *ws, int eff, int opA, int opB, int64_t m, int64_t n,
                    int64_t k, float2 alpha, const OperandView &A_in, const OperandView &B_in,
                    float2 beta, float2 *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out,
                    const qcs_gemm_desc_t *d_desc_in, const GemmBatch &bt) {
    return run_cgemm_group(h, ws, eff, opA, opB, m, n, k, alpha, &A_in, &B_in, 1, beta, C, ldc, 0,
                           d_desc_out, d_desc_in, bt);
}

int run_cgemm_group(qcs_handle_t h, void *ws, int eff, int opA, int opB, int64_t m, int64_t n,
                    int64_t k, float2 alpha, const OperandView *A_in, const OperandView *B_in,
                    int G, float2 beta, float2 *C, int64_t ldc, int64_t c_stride,
                    qcs_gemm_desc_t *d_desc_out, const qcs_gemm_desc_t *d_desc_in,
                    const GemmBatch &bt) {
    cudaStream_t s = h->stream;
    if (G < 1) return QCS_ERR_INVALID_ARG;
    const int gm = gemm_group_m(h, opA, opB, m, n, k);
    if (bt.count != 1 && (eff != QCS_MODE_FP32 || k == 0 || d_desc_out || d_desc_in || G != 1 ||
                          A_in[0].map || B_in[0].map))
        return QCS_ERR_UNSUPPORTED;
    if (G > 1 && (eff == QCS_MODE_FP32 || k == 0 || d_desc_out || d_desc_in))
        return QCS_ERR_UNSUPPORTED;
    for (int g = 0; g < G; ++g)
        if ((A_in[g].map && (opA != QCS_OP_N || !A_in[g].buf)) ||
            (B_in[g].map && (opB != QCS_OP_N || !B_in[g].buf)))
            return QCS_ERR_INVALID_ARG;
    uint8_t *p = static_cast<uint8_t *>(ws);
    qcs_gemm_desc_t *desc = reinterpret_cast<qcs_gemm_desc_t *>(p);
    p += align256(sizeof(qcs_gemm_desc_t) * G);
    int64_t *partials = reinterpret_cast<int64_t *>(p);
    p += align256(size_t(2) * h->num_sms * kPartialStride * sizeof(int64_t));
    float2 *splitk = reinterpret_cast<float2 *>(p);  // kSplitKBytes per batch entry (FP32 batches
    p += align256(kSplitKBytes);                      // run without planes, so the rest follows)
    cudaError_t e = cudaSuccess;
    const int64_t kp = round_up(k, 32), mp = round_up(m, kBM), np = round_up(n, kBN);
    if (G > 1 && (G * mp > INT32_MAX || G * np > INT32_MAX)) return QCS_ERR_UNSUPPORTED;

    // A mapped operand is split straight from its tensor when the emulated
    // path runs, the map permutes that tensor as a whole (``flat``) and tiles
    // with no plane padding; otherwise it is gathered here and read as a
    // matrix (for G = 1 once, and the FP32 candidate reuses it; for a group
    // per instance into the one buffer, and the FP32 candidate gathers again,
    // only if it was selected).
    std::vector<OperandView> Av(A_in, A_in + G), Bv(B_in, B_in + G);
    const bool emulated = (eff != QCS_MODE_FP32 && k > 0);
    const OperandView &A0 = Av[0], &B0 = Bv[0];
    const bool fusedA = A0.map && A0.flat > 0 && emulated && mp == m && kp == k &&
                        split_gather_supported(0, A0.map->rank, A0.map->dims, A0.map->strides, m, kp);
    const bool fusedB = B0.map && B0.flat > 0 && emulated && np == n && kp == k &&
                        split_gather_supported(1, B0.map->rank, B0.map->dims, B0.map->strides, k, kp);
    // TF32 selection split inside the tensor-core kernel (qcs_set_fused_split):
    // one GEMM on matrices as stored, one K range, the default drain
    const bool tf32_fused =
        h->fused_split && emulated && G == 1 && bt.count == 1 && !A0.map && !B0.map &&
        (eff == QCS_MODE_TF32X || eff == QCS_MODE_AUTO) && h->drain_stages == 4 &&
        tc_split_count(m, n, k, 1, h->num_sms, gemm_splits(h, opA, opB, m, n, k)) == 1 &&
        tc_fused_supported(opA, opB, m, n, k, A0.X, A0.ld, B0.X, B0.ld);

    // The per-instance front of the sequence: gathers, statistics and
    // selection (or the constant descriptor), the split of both operands.
    const bool need16 = (eff == QCS_MODE_AUTO || eff == QCS_MODE_FP16X ||
                         eff == QCS_MODE_FP16X_SCALED || eff == QCS_MODE_BF16X3);
    const bool need32 = (eff == QCS_MODE_AUTO || eff == QCS_MODE_TF32X);
    TcWork w;
    w.wait_ns = h->wait_ns;
    w.stall = h->debug_stall;
    w.G = G;
    w.a_rows = mp;
    w.b_rows = np;
    w.c_stride = c_stride;
    // K ranges are chosen per GEMM, not per group, so that an instance's
    // result does not depend on the group it ran in
    w.S = emulated ? tc_split_count(m, n, k, 1, h->num_sms, gemm_splits(h, opA, opB, m, n, k)) : 1;
    const PlaneLayout PL = plane_layout(eff, m, n, k, G, w.S);
    uint8_t *planesA = p + PL.a16, *planesB = p + PL.b16;
    uint8_t *planesA32 = p + PL.a32, *planesB32 = p + PL.b32;
    void *sepA32 = (PL.a32 != PL.a16) ? planesA32 : nullptr;
    void *sepB32 = (PL.b32 != PL.b16) ? planesB32 : nullptr;
    if (w.S > 1) w.P = reinterpret_cast<float2 *>(p + PL.partials);
    // One split launch for an operand of the whole group when the instances'
    // operands lie one stride apart and are read the same way (a matrix, or
    // the same whole-tensor map): the intermediates of a grouped step.
    auto one_stride = [&](const std::vector<OperandView> &V, bool mapped_ok, int64_t &stride) {
        if (G < 2 || !emulated || (V[0].map && !mapped_ok)) return false;
        const intptr_t d = reinterpret_cast<intptr_t>(V[1].X) - reinterpret_cast<intptr_t>(V[0].X);
        if (d % (intptr_t)sizeof(float2) != 0) return false;
        for (int g = 1; g < G; ++g)
            if (reinterpret_cast<intptr_t>(V[g].X) - reinterpret_cast<intptr_t>(V[0].X) !=
                    (intptr_t)g * d ||
                V[g].map != V[0].map || V[g].ld != V[0].ld || V[g].flat != V[0].flat)
                return false;
        stride = (int64_t)(d / (intptr_t)sizeof(float2));
        return true;
    };
    int64_t dxA = 0, dxB = 0;
    const bool batchA = !(tf32_fused && eff == QCS_MODE_TF32X) && one_stride(Av, fusedA, dxA);
    const bool batchB = !(tf32_fused && eff == QCS_MODE_TF32X) && one_stride(Bv, fusedB, dxB);
    // constant descriptors of the whole group in one launch
    const bool const_desc = !d_desc_in && eff != QCS_MODE_AUTO && eff != QCS_MODE_FP16X_SCALED &&
                            (eff != QCS_MODE_FP32 || d_desc_out);
    if (const_desc) {
        e = launch_set_desc(desc, eff, s, G);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    }
    // The statistics and selection of all instances in one launch each, when
    // every operand is read as stored (a matrix, or a whole-tensor map) with
    // the instances' operands one stride apart
    bool stats_done = false;
    if (!d_desc_in && G > 1 && (eff == QCS_MODE_AUTO || eff == QCS_MODE_FP16X_SCALED) &&
        (!A0.map || fusedA) && (!B0.map || fusedB)) {
        auto stride_of = [&](const std::vector<OperandView> &V, int64_t &stride) {
            const intptr_t d = reinterpret_cast<intptr_t>(V[1].X) - reinterpret_cast<intptr_t>(V[0].X);
            if (d % (intptr_t)sizeof(float2) != 0) return false;
            for (int g = 1; g < G; ++g)
                if (reinterpret_cast<intptr_t>(V[g].X) - reinterpret_cast<intptr_t>(V[0].X) !=
                        (intptr_t)g * d ||
                    V[g].map != V[0].map || V[g].ld != V[0].ld || V[g].flat != V[0].flat)
                    return false;
            stride = (int64_t)(d / (intptr_t)sizeof(float2));
            return true;
        };
        int64_t sxA = 0, sxB = 0;
        const int64_t ra = fusedA ? A0.flat : ((opA == QCS_OP_N) ? m : k);
        const int64_t ca = fusedA ? 1 : ((opA == QCS_OP_N) ? k : m);
        const int64_t rb = fusedB ? B0.flat : ((opB == QCS_OP_N) ? k : n);
        const int64_t cb = fusedB ? 1 : ((opB == QCS_OP_N) ? n : k);
        // per-instance blocks so that the whole batch fills the GPU about as
        // one instance does; the partials of all instances fit the buffer
        const int share = std::max(1, (4 * h->num_sms + G - 1) / G);
        const int gA = std::min(stats2_blocks(ra * ca, h->num_sms), share);
        const int gB = std::min(stats2_blocks(rb * cb, h->num_sms), share);
        const int64_t need = (int64_t)6 * G * (gA + gB);
        if (G <= 65535 && need <= (int64_t)2 * h->num_sms * kPartialStride &&
            stride_of(Av, sxA) && stride_of(Bv, sxB)) {
            ProfScope ps(h, kProfStats);
            e = launch_stats_select_2stage_batch(
                A0.X, ra, ca, fusedA ? A0.flat : A0.ld, gA, sxA, B0.X, rb, cb,
                fusedB ? B0.flat : B0.ld, gB, sxB, G, h->tol, eff, partials,
                partials + (int64_t)5 * G * (gA + gB), desc, h->d_counts,
                8.0 * (double)m * (double)n * (double)k, s);
            if (e != cudaSuccess) return QCS_ERR_CUDA;
            stats_done = true;
        }
    }
    for (int g = 0; g < G; ++g) {
        OperandView &A = Av[g], &B = Bv[g];
        qcs_gemm_desc_t *dg = desc + g;
        if (A.map && !fusedA)
            if (int r = gather_view(h, A, m, nullptr)) return r;
        if (B.map && !fusedB)
            if (int r = gather_view(h, B, k, nullptr)) return r;
        if (d_desc_in) {
            dg = const_cast<qcs_gemm_desc_t *>(d_desc_in);
            desc = dg;
        } else if (!stats_done && (eff == QCS_MODE_AUTO || eff == QCS_MODE_FP16X_SCALED)) {
            // Statistics of both operands as stored (a transpose or a
            // whole-tensor permutation does not change the multiset).
            const int64_t ra = fusedA ? A.flat : ((opA == QCS_OP_N) ? m : k);
            const int64_t ca = fusedA ? 1 : ((opA == QCS_OP_N) ? k : m);
            const int64_t rb = fusedB ? B.flat : ((opB == QCS_OP_N) ? k : n);
            const int64_t cb = fusedB ? 1 : ((opB == QCS_OP_N) ? n : k);
            const int64_t lda = fusedA ? A.flat : A.ld, ldb = fusedB ? B.flat : B.ld;
            const int gA = stats2_blocks(ra * ca, h->num_sms), gB = stats2_blocks(rb * cb, h->num_sms);
            ProfScope ps(h, kProfStats);
            e = launch_stats_select_2stage(A.X, ra, ca, lda, gA, B.X, rb, cb, ldb, gB, h->tol, eff,
                                           partials, partials + 5 * (gA + gB), dg, h->d_counts,
                                           8.0 * (double)m * (double)n * (double)k, s);
            if (e != cudaSuccess) return QCS_ERR_CUDA;
        }
        // (a plain FP32 GEMM runs ungated; it needs a descriptor only to report it)
        if (!emulated || (tf32_fused && eff == QCS_MODE_TF32X)) continue;
        if (!batchA)
            if (int r = split_operand(h, 0, dg, A, opA, m, k, mp, kp, planesA, G * mp * kp,
                                      g * mp * kp, sepA32, fusedA, tf32_fused, SplitBatch{}))
                return r;
        if (!batchB)
            if (int r = split_operand(h, 1, dg, B, opB, n, k, np, kp, planesB, G * np * kp,
                                      g * np * kp, sepB32, fusedB, tf32_fused, SplitBatch{}))
                return r;
    }
    if (batchA)
        if (int r = split_operand(h, 0, desc, Av[0], opA, m, k, mp, kp, planesA, G * mp * kp, 0,
                                  sepA32, fusedA, tf32_fused, SplitBatch{G, dxA, mp * kp}))
            return r;
    if (batchB)
        if (int r = split_operand(h, 1, desc, Bv[0], opB, n, k, np, kp, planesB, G * np * kp, 0,
                                  sepB32, fusedB, tf32_fused, SplitBatch{G, dxB, np * kp}))
            return r;

    if (k == 0) {
        // C = beta C: the SIMT kernel with k = 0 does exactly that (no desc gate).
        e = launch_cgemm_simt(nullptr, opA, opB, m, n, 0, alpha, Av[0].X, Av[0].ld, Bv[0].X,
                              Bv[0].ld, beta, C, ldc, nullptr, s);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    } else if (emulated) {
        {
            // One launch per kind over the tiles of all G instances.
            ProfScope ps_tc(h, kProfGemmTc);
            if (need16) {
                CUtensorMap ma, mb, mc[2], pc[2];
                if (encode_planes(h, &ma, planesA, G * mp, kp, 2, kPlanes) ||
                    encode_planes(h, &mb, planesB, G * np, kp, 2, kPlanesB) ||
                    (h->tc_multicast &&
                     (encode_planes(h, &mc[0], planesB, G * np, kp, 2, kPlanesB, kBM, 3) ||
                      encode_planes(h, &mc[1], planesB, G * np, kp, 2, kPlanesB, kBM, 2))) ||
                    (h->tc_pairs &&
                     (encode_planes(h, &pc[0], planesB, G * np, kp, 2, kPlanesB, kBM, 2) ||
                      encode_planes(h, &pc[1], planesB, G * np, kp, 2, kPlanesB, kBN / 2, 2))))
                    return QCS_ERR_CUDA;
                const int kind = (eff == QCS_MODE_BF16X3) ? 2 : 0;
                e = launch_cgemm_tc(kind, h->drain_stages, desc, &ma, &mb, m, n, kp, alpha, beta, C,
                                    ldc, h->d_err, h->num_sms, gm, s, w,
                                    h->tc_multicast ? mc : nullptr, h->tc_pairs ? pc : nullptr);
                if (e != cudaSuccess) return QCS_ERR_CUDA;
            }
            if (need32 && tf32_fused) {
                e = launch_cgemm_tc_fused(h->encode, desc, opA, opB, m, n, k, alpha, A0.X, A0.ld,
                                          B0.X, B0.ld, beta, C, ldc, h->d_err, h->num_sms,
                                          gm, w, s);
                if (e != cudaSuccess) return QCS_ERR_CUDA;
            } else if (need32) {
                CUtensorMap ma, mb, mc[2], pc[2];
                if (encode_planes(h, &ma, planesA32, G * mp, kp, 4, kPlanes) ||
                    encode_planes(h, &mb, planesB32, G * np, kp, 4, kPlanesB) ||
                    (h->tc_multicast &&
                     (encode_planes(h, &mc[0], planesB32, G * np, kp, 4, kPlanesB, kBM, 3) ||
                      encode_planes(h, &mc[1], planesB32, G * np, kp, 4, kPlanesB, kBM, 2))) ||
                    (h->tc_pairs &&
                     (encode_planes(h, &pc[0], planesB32, G * np, kp, 4, kPlanesB, kBM, 2) ||
                      encode_planes(h, &pc[1], planesB32, G * np, kp, 4, kPlanesB, kBN / 2, 2))))
                    return QCS_ERR_CUDA;
                e = launch_cgemm_tc(1, h->drain_stages, desc, &ma, &mb, m, n, kp, alpha, beta, C,
                                    ldc, h->d_err, h->num_sms, gm, s, w,
                                    h->tc_multicast ? mc : nullptr, h->tc_pairs ? pc : nullptr);
                if (e != cudaSuccess) return QCS_ERR_CUDA;
            }
            e = launch_tc_reduce(desc, m, n, alpha, beta, C, ldc, h->num_sms, w, s);
            if (e != cudaSuccess) return QCS_ERR_CUDA;
        }
        if (eff == QCS_MODE_AUTO) {
            // the FP32 candidate of each instance: mapped operands are
            // gathered only if it was selected
            for (int g = 0; g < G; ++g) {
                OperandView &A = Av[g], &B = Bv[g];
                const bool regatherA = fusedA || (G > 1 && A_in[g].map);
                const bool regatherB = fusedB || (G > 1 && B_in[g].map);
                if (regatherA) {
                    A = A_in[g];
                    if (int r = gather_view(h, A, m, desc + g)) return r;
                }
                if (regatherB) {
                    B = B_in[g];
                    if (int r = gather_view(h, B, k, desc + g)) return r;
                }
                ProfScope ps(h, kProfGemmSimt);
                e = launch_cgemm_simt(desc + g, opA, opB, m, n, k, alpha, A.X, A.ld, B.X, B.ld,
                                      beta, C + g * c_stride, ldc, splitk, s);
                if (e != cudaSuccess) return QCS_ERR_CUDA;
            }
        }
    } else {
        ProfScope ps(h, kProfGemmSimt);
        e = launch_cgemm_simt(nullptr, opA, opB, m, n, k, alpha, Av[0].X, Av[0].ld, Bv[0].X,
                              Bv[0].ld, beta, C, ldc, splitk, s, bt);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    }
    if (d_desc_out) {
        e = cudaMemcpyAsync(d_desc_out, desc, sizeof(qcs_gemm_desc_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    }
    return QCS_SUCCESS;
}

// ---- real GEMM --------------------------------------------------------------

namespace {

// Plane areas of one real GEMM: A two planes of mp rows, B two planes of
// np rows (n rounded up to the real tile's 256 columns), then the partials.
struct RealLayout {
    int64_t kp = 0, mp = 0, np = 0;
    size_t a = 0, b = 0, partials = 0, total = 0;
};

RealLayout real_layout(int eff, int64_t m, int64_t n, int64_t k, int S) {
    RealLayout L;
    L.kp = round_up(k, 32);
    L.mp = round_up(m, kBM);
    L.np = round_up(n, 2 * kBN);
    const int esz = (eff == QCS_MODE_AUTO || eff == QCS_MODE_TF32X) ? 4 : 2;
    L.a = 0;
    L.b = align256(size_t(2) * L.mp * L.kp * esz);
    L.partials = L.b + align256(size_t(2) * L.np * L.kp * esz);
    L.total = L.partials + (S > 1 ? align256(sizeof(float) * S * m * n) : 0);
    return L;
}

// The size rule for a real GEMM: the paper's cut-offs (the tuned table
// holds complex shapes).
int effective_mode_real(qcs_handle_t h, int mode, int64_t m, int64_t n, int64_t k) {
    if (mode != QCS_MODE_AUTO || h->size_rule == QCS_SIZE_RULE_OFF) return mode;
    const int64_t s = std::min(m, std::min(n, k));
    if (s >= 2048) return QCS_MODE_AUTO;
    if (s >= 512) return QCS_MODE_TF32X;
    return QCS_MODE_FP32;
}

}  // namespace

size_t sgemm_workspace_bytes(int eff, int64_t m, int64_t n, int64_t k, int num_sms, int splits) {
    size_t bytes = align256(sizeof(qcs_gemm_desc_t));
    bytes += align256(size_t(2) * num_sms * kPartialStride * sizeof(int64_t));
    if (eff != QCS_MODE_FP32 && k > 0)
        bytes += real_layout(eff, m, n, k, tc_split_count(m, n, k, 1, num_sms, splits, true)).total;
    return bytes;
}

int run_sgemm(qcs_handle_t h, void *ws, int eff, int opA, int opB, int64_t m, int64_t n, int64_t k,
              float alpha, const float *A, int64_t lda, const float *B, int64_t ldb, float beta,
              float *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out) {
    cudaStream_t s = h->stream;
    uint8_t *p = static_cast<uint8_t *>(ws);
    qcs_gemm_desc_t *desc = reinterpret_cast<qcs_gemm_desc_t *>(p);
    p += align256(sizeof(qcs_gemm_desc_t));
    int64_t *partials = reinterpret_cast<int64_t *>(p);
    p += align256(size_t(2) * h->num_sms * kPartialStride * sizeof(int64_t));
    cudaError_t e = cudaSuccess;
    const bool emulated = (eff != QCS_MODE_FP32 && k > 0);
    if (eff == QCS_MODE_AUTO || eff == QCS_MODE_FP16X_SCALED) {
        // statistics of both operands as stored (a transpose keeps the multiset)
        const int64_t ra = (opA == QCS_OP_N) ? m : k, ca = (opA == QCS_OP_N) ? k : m;
        const int64_t rb = (opB == QCS_OP_N) ? k : n, cb = (opB == QCS_OP_N) ? n : k;
        const int gA = stats2_blocks((ra * ca + 1) / 2, h->num_sms);
        const int gB = stats2_blocks((rb * cb + 1) / 2, h->num_sms);
        ProfScope ps(h, kProfStats);
        e = launch_stats_select_2stage_real(A, ra, ca, lda, gA, B, rb, cb, ldb, gB, h->tol, eff,
                                            partials, partials + 5 * (gA + gB), desc, h->d_counts,
                                            2.0 * (double)m * (double)n * (double)k, s);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    } else if (eff != QCS_MODE_FP32 || d_desc_out) {
        e = launch_set_desc(desc, eff, s);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    }
    if (!emulated) {
        ProfScope ps(h, kProfGemmSimt);
        e = launch_sgemm_simt(nullptr, opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    } else {
        TcWork w;
        w.wait_ns = h->wait_ns;
        w.stall = h->debug_stall;
        w.S = tc_split_count(m, n, k, 1, h->num_sms, h->tc_splits, true);
        const RealLayout L = real_layout(eff, m, n, k, w.S);
        uint8_t *planesA = p + L.a, *planesB = p + L.b;
        if (w.S > 1) w.P = reinterpret_cast<float2 *>(p + L.partials);
        w.a_rows = L.mp;
        w.b_rows = L.np;
        {
            int64_t sr, sc;
            ProfScope ps(h, kProfSplit);
            plane_strides(0, opA, lda, sr, sc);
            e = launch_split_real(desc, 0, A, sr, sc, m, k, L.mp, L.kp, planesA, L.kp, L.mp * L.kp, s);
            if (e == cudaSuccess) {
                plane_strides(1, opB, ldb, sr, sc);
                e = launch_split_real(desc, 1, B, sr, sc, n, k, L.np, L.kp, planesB, L.kp,
                                      L.np * L.kp, s);
            }
            if (e != cudaSuccess) return QCS_ERR_CUDA;
        }
        const bool need16 = (eff == QCS_MODE_AUTO || eff == QCS_MODE_FP16X ||
                             eff == QCS_MODE_FP16X_SCALED || eff == QCS_MODE_BF16X3);
        const bool need32 = (eff == QCS_MODE_AUTO || eff == QCS_MODE_TF32X);
        {
            ProfScope ps_tc(h, kProfGemmTc);
            for (int esz = 2; esz <= 4; esz += 2) {
                if ((esz == 2 && !need16) || (esz == 4 && !need32)) continue;
                CUtensorMap ma, mb, pb;
                if (encode_planes(h, &ma, planesA, L.mp, L.kp, esz, 2, kBM) ||
                    encode_planes(h, &mb, planesB, L.np, L.kp, esz, 2, 2 * kBN) ||
                    (h->tc_pairs && encode_planes(h, &pb, planesB, L.np, L.kp, esz, 2, kBM)))
                    return QCS_ERR_CUDA;
                const int kind = (esz == 4) ? 1 : (eff == QCS_MODE_BF16X3 ? 2 : 0);
                e = launch_sgemm_tc(kind, h->drain_stages, desc, &ma, &mb, m, n, L.kp, alpha, beta,
                                    C, ldc, h->d_err, h->num_sms, h->tc_group_m, s, w,
                                    h->tc_pairs ? &pb : nullptr);
                if (e != cudaSuccess) return QCS_ERR_CUDA;
            }
            e = launch_tc_reduce_real(desc, m, n, alpha, beta, C, ldc, h->num_sms, w, s);
            if (e != cudaSuccess) return QCS_ERR_CUDA;
        }
        if (eff == QCS_MODE_AUTO) {
            ProfScope ps(h, kProfGemmSimt);
            e = launch_sgemm_simt(desc, opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, s);
            if (e != cudaSuccess) return QCS_ERR_CUDA;
        }
    }
    if (d_desc_out) {
        e = cudaMemcpyAsync(d_desc_out, desc, sizeof(qcs_gemm_desc_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    }
    return QCS_SUCCESS;
}

// ---- Gauss's three-product CGEMM --------------------------------------------

namespace {

// The three real operands of each side (Ar, Ai, Ar + Ai) as instances 0, 1,
// 2 of a group: two planes each, instance g's rows after those of g - 1;
// then the three real products T (m x n floats each) and the partials.
struct Gauss3Layout {
    int64_t kp = 0, mp = 0, np = 0;
    size_t a = 0, b = 0, t = 0, partials = 0, total = 0;
};

Gauss3Layout gauss3_layout(int eff, int64_t m, int64_t n, int64_t k, int S) {
    Gauss3Layout L;
    L.kp = round_up(k, 32);
    L.mp = round_up(m, kBM);
    L.np = round_up(n, 2 * kBN);
    const int esz = (eff == QCS_MODE_AUTO || eff == QCS_MODE_TF32X) ? 4 : 2;
    L.a = 0;
    L.b = align256(size_t(2) * 3 * L.mp * L.kp * esz);
    L.t = L.b + align256(size_t(2) * 3 * L.np * L.kp * esz);
    L.partials = L.t + align256(sizeof(float) * 3 * m * n);
    L.total = L.partials + (S > 1 ? align256(sizeof(float) * S * 3 * m * n) : 0);
    return L;
}

}  // namespace

// The per-line statistics of op(A)'s rows and op(B)'s columns: each line's
// largest biased exponent (emaxA: m, emaxB: n) and counts[4] = {below the
// shifted windows in op(A), nonzero in op(A), the same for op(B)}.
cudaError_t rowcol_line_stats(cudaStream_t s, int opA, int opB, int64_t m, int64_t n, int64_t k,
                              const float2 *A, int64_t lda, const float2 *B, int64_t ldb,
                              int *emaxA, int *emaxB, unsigned long long *counts) {
    // a row of op(A) is a stored row of A (N) or a stored column (T, C); a
    // column of op(B) is a stored column of B (N) or a stored row (T, C)
    const int64_t ra = (opA == QCS_OP_N) ? m : k, ca = (opA == QCS_OP_N) ? k : m;
    const int64_t rb = (opB == QCS_OP_N) ? k : n, cb = (opB == QCS_OP_N) ? n : k;
    const int rowsA = (opA == QCS_OP_N) ? 1 : 0, rowsB = (opB == QCS_OP_N) ? 0 : 1;
    cudaError_t e = cudaMemsetAsync(counts, 0, 4 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = launch_line_emax(A, ra, ca, lda, rowsA, emaxA, s);
    if (e == cudaSuccess) e = launch_line_emax(B, rb, cb, ldb, rowsB, emaxB, s);
    if (e == cudaSuccess) e = launch_line_under(A, ra, ca, lda, rowsA, emaxA, counts, s);
    if (e == cudaSuccess) e = launch_line_under(B, rb, cb, ldb, rowsB, emaxB, counts + 2, s);
    return e;
}

namespace {

struct RowcolLayout {
    size_t desc, partials, counts, emaxA, emaxB, P, total;
};

RowcolLayout rowcol_layout(int64_t m, int64_t n, int num_sms) {
    RowcolLayout L;
    size_t off = 0;
    L.desc = off;  // desc0, descK, descOut
    off += align256(3 * sizeof(qcs_gemm_desc_t));
    L.partials = off;
    off += align256(size_t(2) * num_sms * kPartialStride * sizeof(int64_t));
    L.counts = off;
    off += align256(4 * sizeof(unsigned long long));
    L.emaxA = off;
    off += align256(sizeof(int) * (size_t)m);
    L.emaxB = off;
    off += align256(sizeof(int) * (size_t)n);
    L.P = off;
    off += align256(sizeof(float2) * (size_t)m * (size_t)n);
    L.total = off;
    return L;
}

}  // namespace

size_t rowcol_workspace_bytes(int64_t m, int64_t n, int64_t k, int num_sms, int splits) {
    return rowcol_layout(m, n, num_sms).total +
           gemm_workspace_bytes(QCS_MODE_AUTO, m, n, k, num_sms, splits, 1);
}

int run_cgemm_rowcol(qcs_handle_t h, void *ws, int opA, int opB, int64_t m, int64_t n, int64_t k,
                     float2 alpha, const float2 *A, int64_t lda, const float2 *B, int64_t ldb,
                     float2 beta, float2 *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out) {
    if (k == 0 || m == 0 || n == 0) return QCS_ERR_UNSUPPORTED;
    cudaStream_t s = h->stream;
    uint8_t *p = static_cast<uint8_t *>(ws);
    const RowcolLayout L = rowcol_layout(m, n, h->num_sms);
    qcs_gemm_desc_t *desc0 = reinterpret_cast<qcs_gemm_desc_t *>(p + L.desc);
    qcs_gemm_desc_t *descK = desc0 + 1, *descOut = desc0 + 2;
    int64_t *partials = reinterpret_cast<int64_t *>(p + L.partials);
    unsigned long long *counts = reinterpret_cast<unsigned long long *>(p + L.counts);
    int *emaxA = reinterpret_cast<int *>(p + L.emaxA);
    int *emaxB = reinterpret_cast<int *>(p + L.emaxB);
    float2 *P = reinterpret_cast<float2 *>(p + L.P);
    {
        // Section 4.1 on the whole matrices, as qcs_cgemm's AUTO
        const int64_t ra = (opA == QCS_OP_N) ? m : k, ca = (opA == QCS_OP_N) ? k : m;
        const int64_t rb = (opB == QCS_OP_N) ? k : n, cb = (opB == QCS_OP_N) ? n : k;
        const int gA = stats2_blocks(ra * ca, h->num_sms), gB = stats2_blocks(rb * cb, h->num_sms);
        ProfScope ps(h, kProfStats);
        if (launch_stats_select_2stage(A, ra, ca, lda, gA, B, rb, cb, ldb, gB, h->tol,
                                       QCS_MODE_AUTO, partials, partials + 5 * (gA + gB), desc0,
                                       h->d_counts, 8.0 * (double)m * (double)n * (double)k,
                                       s) != cudaSuccess ||
            rowcol_line_stats(s, opA, opB, m, n, k, A, lda, B, ldb, emaxA, emaxB, counts) !=
                cudaSuccess ||
            launch_rowcol_select(desc0, counts, h->tol, descK, descOut, s) != cudaSuccess)
            return QCS_ERR_CUDA;
    }
    // the GEMM on the selected descriptor into P (alpha 1, beta 0); the
    // split reads the line exponents when descK says so
    h->line_emax[0] = emaxA;
    h->line_emax[1] = emaxB;
    const int r = run_cgemm(h, p + L.total, QCS_MODE_AUTO, opA, opB, m, n, k, make_float2(1.f, 0.f),
                            A, lda, B, ldb, make_float2(0.f, 0.f), P, m, nullptr, descK);
    h->line_emax[0] = h->line_emax[1] = nullptr;
    if (r != QCS_SUCCESS) return r;
    if (launch_rowcol_combine(descK, emaxA, emaxB, P, m, n, alpha, beta, C, ldc, h->num_sms, s) !=
        cudaSuccess)
        return QCS_ERR_CUDA;
    if (d_desc_out &&
        cudaMemcpyAsync(d_desc_out, descOut, sizeof(qcs_gemm_desc_t), cudaMemcpyDeviceToDevice,
                        s) != cudaSuccess)
        return QCS_ERR_CUDA;
    return QCS_SUCCESS;
}

size_t cgemm3m_workspace_bytes(int eff, int64_t m, int64_t n, int64_t k, int num_sms, int splits) {
    size_t bytes = align256(3 * sizeof(qcs_gemm_desc_t));
    bytes += align256(size_t(2) * num_sms * kPartialStride * sizeof(int64_t));
    bytes += align256(kSplitKBytes);
    bytes += gauss3_layout(eff, m, n, k, tc_split_count(m, n, k, 1, num_sms, splits, true)).total;
    return bytes;
}

// C = alpha op(A) op(B) + beta C with T1 = Ar Br, T2 = Ai Bi,
// T3 = (Ar + Ai)(Br + Bi) as three emulated real GEMMs in one grouped
// tensor-core launch (Ar, Ai: the parts of op(A), conjugation applied), then
// Re = T1 - T2, Im = T3 - T1 - T2.  Statistics and selection are those of A
// and B (Section 4.1); T3 runs with desc[2] (launch_derive_3m_desc).  Only
// emulated modes (eff != FP32, k > 0); AUTO's FP32 candidate is the complex
// SIMT kernel, gated as in run_cgemm.
int run_cgemm_3m(qcs_handle_t h, void *ws, int eff, int opA, int opB, int64_t m, int64_t n,
                 int64_t k, float2 alpha, const float2 *A, int64_t lda, const float2 *B,
                 int64_t ldb, float2 beta, float2 *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out) {
    if (eff == QCS_MODE_FP32 || k == 0) return QCS_ERR_UNSUPPORTED;
    cudaStream_t s = h->stream;
    uint8_t *p = static_cast<uint8_t *>(ws);
    qcs_gemm_desc_t *desc = reinterpret_cast<qcs_gemm_desc_t *>(p);
    p += align256(3 * sizeof(qcs_gemm_desc_t));
    int64_t *partials = reinterpret_cast<int64_t *>(p);
    p += align256(size_t(2) * h->num_sms * kPartialStride * sizeof(int64_t));
    float2 *splitk = reinterpret_cast<float2 *>(p);
    p += align256(kSplitKBytes);
    cudaError_t e = cudaSuccess;
    if (eff == QCS_MODE_AUTO || eff == QCS_MODE_FP16X_SCALED) {
        const int64_t ra = (opA == QCS_OP_N) ? m : k, ca = (opA == QCS_OP_N) ? k : m;
        const int64_t rb = (opB == QCS_OP_N) ? k : n, cb = (opB == QCS_OP_N) ? n : k;
        const int gA = stats2_blocks(ra * ca, h->num_sms), gB = stats2_blocks(rb * cb, h->num_sms);
        ProfScope ps(h, kProfStats);
        e = launch_stats_select_2stage(A, ra, ca, lda, gA, B, rb, cb, ldb, gB, h->tol, eff,
                                       partials, partials + 5 * (gA + gB), desc, h->d_counts,
                                       8.0 * (double)m * (double)n * (double)k, s);
    } else {
        e = launch_set_desc(desc, eff, s);
    }
    if (e == cudaSuccess) e = launch_derive_3m_desc(desc, s);
    if (e != cudaSuccess) return QCS_ERR_CUDA;

    TcWork w;
    w.wait_ns = h->wait_ns;
    w.stall = h->debug_stall;
    w.G = 3;
    w.S = tc_split_count(m, n, k, 1, h->num_sms, h->tc_splits, true);
    const Gauss3Layout L = gauss3_layout(eff, m, n, k, w.S);
    uint8_t *planesA = p + L.a, *planesB = p + L.b;
    float *T = reinterpret_cast<float *>(p + L.t);
    if (w.S > 1) w.P = reinterpret_cast<float2 *>(p + L.partials);
    w.a_rows = L.mp;
    w.b_rows = L.np;
    w.c_stride = m * n;
    {
        ProfScope ps(h, kProfSplit);
        // one pass over each complex operand writes the planes of its three
        // real operands (parts 0, 1, 2 = instances 0, 1, 2)
        for (int which = 0; which < 2 && e == cudaSuccess; ++which) {
            const int op = which == 0 ? opA : opB;
            int64_t sr, sc;
            plane_strides(which, op, which == 0 ? lda : ldb, sr, sc);
            const int64_t R = which == 0 ? m : n, Rp = which == 0 ? L.mp : L.np;
            e = launch_split_gauss(desc, which, which == 0 ? A : B, sr, sc, op == QCS_OP_C, R, k, Rp,
                                   L.kp, which == 0 ? planesA : planesB, L.kp, 3 * Rp * L.kp,
                                   Rp * L.kp, s);
        }
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    }
    const bool need16 = (eff == QCS_MODE_AUTO || eff == QCS_MODE_FP16X ||
                         eff == QCS_MODE_FP16X_SCALED || eff == QCS_MODE_BF16X3);
    const bool need32 = (eff == QCS_MODE_AUTO || eff == QCS_MODE_TF32X);
    {
        ProfScope ps_tc(h, kProfGemmTc);
        for (int esz = 2; esz <= 4; esz += 2) {
            if ((esz == 2 && !need16) || (esz == 4 && !need32)) continue;
            CUtensorMap ma, mb, pb;
            if (encode_planes(h, &ma, planesA, 3 * L.mp, L.kp, esz, 2, kBM) ||
                encode_planes(h, &mb, planesB, 3 * L.np, L.kp, esz, 2, 2 * kBN) ||
                (h->tc_pairs && encode_planes(h, &pb, planesB, 3 * L.np, L.kp, esz, 2, kBM)))
                return QCS_ERR_CUDA;
            const int kind = (esz == 4) ? 1 : (eff == QCS_MODE_BF16X3 ? 2 : 0);
            e = launch_sgemm_tc(kind, h->drain_stages, desc, &ma, &mb, m, n, L.kp, 1.0f, 0.0f, T, m,
                                h->d_err, h->num_sms, h->tc_group_m, s, w,
                                h->tc_pairs ? &pb : nullptr);
            if (e != cudaSuccess) return QCS_ERR_CUDA;
        }
        e = launch_tc_reduce_real(desc, m, n, 1.0f, 0.0f, T, m, h->num_sms, w, s);
        if (e == cudaSuccess) e = launch_combine_3m(desc, m, n, T, alpha, beta, C, ldc, h->num_sms, s);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    }
    if (eff == QCS_MODE_AUTO) {
        ProfScope ps(h, kProfGemmSimt);
        e = launch_cgemm_simt(desc, opA, opB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, splitk, s);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    }
    if (d_desc_out) {
        e = cudaMemcpyAsync(d_desc_out, desc, sizeof(qcs_gemm_desc_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return QCS_ERR_CUDA;
    }
    return QCS_SUCCESS;
}

int validate_cgemm(int mode, int opA, int opB, int64_t m, int64_t n, int64_t k, const void *alpha,
                   const void *A, int64_t lda, const void *B, int64_t ldb, const void *beta,
                   const void *C, int64_t ldc) {
    if (!valid_mode(mode) || !valid_op(opA) || !valid_op(opB)) return QCS_ERR_INVALID_ARG;
    if (m < 0 || n < 0 || k < 0) return QCS_ERR_INVALID_ARG;
    if (!alpha || !beta) return QCS_ERR_INVALID_ARG;
    const int64_t rowsA = (opA == QCS_OP_N) ? m : k;
    const int64_t rowsB = (opB == QCS_OP_N) ? k : n;
    if (lda < std::max<int64_t>(1, rowsA) || ldb < std::max<int64_t>(1, rowsB) ||
        ldc < std::max<int64_t>(1, m))
        return QCS_ERR_INVALID_ARG;
    if (m == 0 || n == 0) return QCS_SUCCESS;
    if (!C) return QCS_ERR_INVALID_ARG;
    if (k > 0 && (!A || !B)) return QCS_ERR_INVALID_ARG;
    auto mis = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 7u) != 0; };
    if (mis(A) || mis(B) || mis(C)) return QCS_ERR_UNSUPPORTED;
    return QCS_SUCCESS;
}

}  // namespace qcs

extern "C" {

int qcs_create(qcs_handle_t *out, void *cuda_stream) {
    if (!out) return QCS_ERR_INVALID_ARG;
    *out = nullptr;
    qcs_handle_s *h = new (std::nothrow) qcs_handle_s;
    if (!h) return QCS_ERR_ALLOC;
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete h;
        return QCS_ERR_CUDA;
    }
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    // One block: the error word at byte 0, the selection counters at byte 8.
    if (cudaMalloc(&h->d_err, kStatusBlockBytes) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return QCS_ERR_ALLOC;
    }
    cudaMemset(h->d_err, 0, kStatusBlockBytes);
    h->d_counts = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(h->d_err) + 8);
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        cudaFree(h->d_err);
        delete h;
        return QCS_ERR_CUDA;
    }
    h->encode = reinterpret_cast<EncodeTiledFn>(fn);
    if (const char *t = std::getenv("QCS_UNDERFLOW_TOL")) h->tol = std::atof(t);
    if (const char *r = std::getenv("QCS_SIZE_RULE")) {
        const int v = std::atoi(r);
        h->size_rule = (v == QCS_SIZE_RULE_OFF || v == QCS_SIZE_RULE_TUNED) ? v : QCS_SIZE_RULE_PAPER;
    }
    if (const char *g = std::getenv("QCS_TC_GROUP_M")) h->tc_group_m = std::max(1, std::atoi(g));
    if (const char *p = std::getenv("QCS_TC_L2_PROMOTION")) h->tc_l2_promotion = std::atoi(p);
    if (const char *c = std::getenv("QCS_COMPLEX_PRODUCTS"))
        h->complex_products = (std::atoi(c) == 3) ? 3 : 4;
    if (const char *f = std::getenv("QCS_FUSED_SPLIT")) h->fused_split = std::atoi(f) != 0;
    if (const char *l = std::getenv("QCS_TREE_LEVELS")) h->tree_levels = std::atoi(l) != 0;
    if (const char *c = std::getenv("QCS_TC_MULTICAST")) h->tc_multicast = std::atoi(c) != 0;
    if (const char *c = std::getenv("QCS_TC_PAIRS")) h->tc_pairs = std::atoi(c) != 0;
    if (const char *b = std::getenv("QCS_GROUP_BUDGET_MB"))
        h->group_budget = (size_t)std::max(0LL, std::atoll(b)) << 20;
    if (const char *k = std::getenv("QCS_TC_SPLITS"))
        h->tc_splits = std::min(kMaxSplits, std::max(0, std::atoi(k)));
    if (const char *d = std::getenv("QCS_DRAIN_STAGES")) {
        const int v = std::atoi(d);
        h->drain_stages = (v >= 4) ? 4 : (v == 2 ? 2 : 1);
    }
    *out = h;
    return QCS_SUCCESS;
}

int qcs_destroy(qcs_handle_t h) {
    if (!h) return QCS_ERR_INVALID_ARG;
    cudaStreamSynchronize(h->stream);
    if (h->ws.ptr) cudaFree(h->ws.ptr);
    if (h->tree_ws.ptr) cudaFree(h->tree_ws.ptr);
    if (h->d_err) cudaFree(h->d_err);
    for (const ProfEvent &pe : h->prof) {
        cudaEventDestroy(pe.start);
        cudaEventDestroy(pe.stop);
    }
    for (cudaEvent_t e : h->event_pool) cudaEventDestroy(e);
    delete h;
    return QCS_SUCCESS;
}

int qcs_set_stream(qcs_handle_t h, void *cuda_stream) {
    if (!h) return QCS_ERR_INVALID_ARG;
    h->stream = static_cast<cudaStream_t>(cuda_stream);
    return QCS_SUCCESS;
}

int qcs_set_underflow_tol(qcs_handle_t h, double t) {
    if (!h || !(t >= 0.0 && t <= 1.0)) return QCS_ERR_INVALID_ARG;
    h->tol = t;
    return QCS_SUCCESS;
}

int qcs_set_drain_stages(qcs_handle_t h, int stages) {
    if (!h || (stages != 1 && stages != 2 && stages != 4)) return QCS_ERR_INVALID_ARG;
    h->drain_stages = stages;
    return QCS_SUCCESS;
}

int qcs_set_tc_schedule(qcs_handle_t h, int group_m, int l2_promotion) {
    if (!h || group_m < 1 || group_m > 1024 ||
        (l2_promotion != 0 && l2_promotion != 64 && l2_promotion != 128 && l2_promotion != 256))
        return QCS_ERR_INVALID_ARG;
    h->tc_group_m = group_m;
    h->tc_l2_promotion = l2_promotion;
    return QCS_SUCCESS;
}

int qcs_set_tc_splits(qcs_handle_t h, int splits) {
    if (!h || splits < 0 || splits > kMaxSplits) return QCS_ERR_INVALID_ARG;
    h->tc_splits = splits;
    return QCS_SUCCESS;
}

int qcs_set_complex_products(qcs_handle_t h, int products) {
    if (!h || (products != 3 && products != 4)) return QCS_ERR_INVALID_ARG;
    h->complex_products = products;
    return QCS_SUCCESS;
}

int qcs_selection_stats(qcs_handle_t h, qcs_op_t transA, qcs_op_t transB, int64_t m, int64_t n,
                        int64_t k, const qcs_c32 *A, int64_t lda, const qcs_c32 *B, int64_t ldb,
                        qcs_selection_stats_t *out, qcs_gemm_desc_t *desc_out) {
    if (!h || !out) return QCS_ERR_INVALID_ARG;
    const qcs_c32 one{1.f, 0.f}, zero{0.f, 0.f};
    if (int r = validate_cgemm(QCS_MODE_AUTO, transA, transB, m, n, k, &one, A, lda, B, ldb, &zero,
                               A, std::max<int64_t>(m, 1)))
        return r;
    if (m == 0 || n == 0 || k == 0) return QCS_ERR_INVALID_ARG;
    const int64_t ra = (transA == QCS_OP_N) ? m : k, ca = (transA == QCS_OP_N) ? k : m;
    const int64_t rb = (transB == QCS_OP_N) ? k : n, cb = (transB == QCS_OP_N) ? n : k;
    const int gA = stats2_blocks(ra * ca, h->num_sms), gB = stats2_blocks(rb * cb, h->num_sms);
    const size_t p1b = align256(sizeof(int64_t) * 5 * (gA + gB));
    const size_t p2b = align256(sizeof(int64_t) * (gA + gB));
    const size_t bytes = p1b + p2b + align256(sizeof(qcs_gemm_desc_t)) + align256(10 * sizeof(int64_t));
    if (int r = ensure_workspace(h->ws, bytes)) return r;
    uint8_t *p = static_cast<uint8_t *>(h->ws.ptr);
    int64_t *p1 = reinterpret_cast<int64_t *>(p);
    int64_t *p2 = reinterpret_cast<int64_t *>(p + p1b);
    qcs_gemm_desc_t *desc = reinterpret_cast<qcs_gemm_desc_t *>(p + p1b + p2b);
    int64_t *summary =
        reinterpret_cast<int64_t *>(p + p1b + p2b + align256(sizeof(qcs_gemm_desc_t)));
    cudaError_t e = launch_stats_select_2stage(
        reinterpret_cast<const float2 *>(A), ra, ca, lda, gA, reinterpret_cast<const float2 *>(B),
        rb, cb, ldb, gB, h->tol, QCS_MODE_AUTO, p1, p2, desc, nullptr, 0.0, h->stream, summary);
    int64_t hs[10];
    qcs_gemm_desc_t hd;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs, summary, sizeof(hs), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&hd, desc, sizeof(hd), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    for (int o = 0; o < 2; ++o) {
        const int64_t *v = hs + 5 * o;
        out[o].e_max = v[0] < 0 ? -128 : (int32_t)(v[0] - 127);
        out[o].stage2 = v[4] >= 0 ? 1 : 0;
        out[o].n_nonzero = v[1];
        out[o].n_nonfinite = v[2];
        out[o].n_under_fp16 = v[3];
        out[o].n_under_window = v[4] >= 0 ? v[4] : 0;
    }
    if (desc_out) *desc_out = hd;
    return QCS_SUCCESS;
}

int qcs_set_group_budget(qcs_handle_t h, uint64_t bytes) {
    if (!h) return QCS_ERR_INVALID_ARG;
    h->group_budget = (size_t)bytes;
    return QCS_SUCCESS;
}

int qcs_fidelity_stats(qcs_handle_t h, const void *a, int a_c64, const double *ref, int64_t n,
                       double *d_out) {
    if (!h || !a || !d_out || n < 0 || (a_c64 != 0 && a_c64 != 1)) return QCS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(a) & (a_c64 ? 7u : 15u)) ||
        (ref && (reinterpret_cast<uintptr_t>(ref) & 15u)) ||
        (reinterpret_cast<uintptr_t>(d_out) & 7u))
        return QCS_ERR_INVALID_ARG;
    // a fixed block count for a given n, so the summation order depends on n alone
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((n + 255) / 256, std::min(kFidBlocksMax, 4 * h->num_sms)));
    if (int r = ensure_workspace(h->ws, sizeof(double) * 6 * (size_t)blocks)) return r;
    return launch_fidelity_stats(a, a_c64, ref, n, static_cast<double *>(h->ws.ptr), blocks,
                                 d_out, h->stream) == cudaSuccess
               ? QCS_SUCCESS
               : QCS_ERR_CUDA;
}

int qcs_set_tc_multicast(qcs_handle_t h, int enabled) {
    if (!h || (enabled != 0 && enabled != 1)) return QCS_ERR_INVALID_ARG;
    h->tc_multicast = enabled;
    return QCS_SUCCESS;
}

int qcs_set_tc_pairs(qcs_handle_t h, int enabled) {
    if (!h || (enabled != 0 && enabled != 1)) return QCS_ERR_INVALID_ARG;
    h->tc_pairs = enabled;
    return QCS_SUCCESS;
}

int qcs_set_rowcol_scaling(qcs_handle_t h, int enabled) {
    if (!h || (enabled != 0 && enabled != 1)) return QCS_ERR_INVALID_ARG;
    h->rowcol = enabled;
    return QCS_SUCCESS;
}

int qcs_rowcol_stats(qcs_handle_t h, qcs_op_t transA, qcs_op_t transB, int64_t m, int64_t n,
                     int64_t k, const qcs_c32 *A, int64_t lda, const qcs_c32 *B, int64_t ldb,
                     int32_t *d_emaxA, int32_t *d_emaxB, int64_t *d_counts) {
    if (!h || !valid_op(transA) || !valid_op(transB) || m < 0 || n < 0 || k < 0 || !d_counts)
        return QCS_ERR_INVALID_ARG;
    if ((m > 0 && !d_emaxA) || (n > 0 && !d_emaxB)) return QCS_ERR_INVALID_ARG;
    const int64_t ra = (transA == QCS_OP_N) ? m : k, rb = (transB == QCS_OP_N) ? k : n;
    if ((m * k > 0 && !A) || (n * k > 0 && !B) || lda < std::max<int64_t>(1, ra) ||
        ldb < std::max<int64_t>(1, rb))
        return QCS_ERR_INVALID_ARG;
    return cuda_status(rowcol_line_stats(
        h->stream, transA, transB, m, n, k, reinterpret_cast<const float2 *>(A), lda,
        reinterpret_cast<const float2 *>(B), ldb, reinterpret_cast<int *>(d_emaxA),
        reinterpret_cast<int *>(d_emaxB), reinterpret_cast<unsigned long long *>(d_counts)));
}

int qcs_set_tree_levels(qcs_handle_t h, int enabled) {
    if (!h || (enabled != 0 && enabled != 1)) return QCS_ERR_INVALID_ARG;
    h->tree_levels = enabled;
    return QCS_SUCCESS;
}

int qcs_set_fused_split(qcs_handle_t h, int enabled) {
    if (!h) return QCS_ERR_INVALID_ARG;
    h->fused_split = enabled ? 1 : 0;
    return QCS_SUCCESS;
}

int qcs_set_wait_budget(qcs_handle_t h, uint64_t ns) {
    if (!h || ns < 1000ull || ns > 10000000000ull) return QCS_ERR_INVALID_ARG;
    h->wait_ns = ns;
    return QCS_SUCCESS;
}

int qcs_debug_stall_producer(qcs_handle_t h, int enabled) {
    if (!h) return QCS_ERR_INVALID_ARG;
    h->debug_stall = enabled ? 1 : 0;
    return QCS_SUCCESS;
}

int qcs_set_instance_batch(qcs_handle_t h, int instances) {
    if (!h || instances < 1 || instances > 65535) return QCS_ERR_INVALID_ARG;
    h->instance_batch = instances;
    return QCS_SUCCESS;
}

int qcs_set_size_rule(qcs_handle_t h, int rule) {
    if (!h) return QCS_ERR_INVALID_ARG;
    h->size_rule = (rule == QCS_SIZE_RULE_OFF || rule == QCS_SIZE_RULE_TUNED) ? rule
                                                                              : QCS_SIZE_RULE_PAPER;
    return QCS_SUCCESS;
}

int qcs_exp_stats(qcs_handle_t h, int64_t rows, int64_t cols, const qcs_c32 *X, int64_t ldx,
                  qcs_stats_t *d_stats) {
    if (!h || !d_stats || rows < 0 || cols < 0 || ldx < std::max<int64_t>(1, rows))
        return QCS_ERR_INVALID_ARG;
    if (rows * cols > 0 && !X) return QCS_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(X) & 7u) != 0) return QCS_ERR_UNSUPPORTED;
    const size_t bytes = align256(size_t(2) * h->num_sms * kPartialStride * sizeof(int64_t)) + 256;
    if (int r = ensure_workspace(h->ws, bytes)) return r;
    int64_t *partials = reinterpret_cast<int64_t *>(static_cast<uint8_t *>(h->ws.ptr) + 256);
    const int g = stats_blocks(rows * cols, h->num_sms);
    cudaError_t e = launch_stats2(reinterpret_cast<const float2 *>(X), rows, cols, ldx, g, nullptr,
                                  0, 0, 1, 0, partials, h->stream);
    if (e != cudaSuccess) return QCS_ERR_CUDA;
    return cuda_status(launch_stats_finalize(partials, g, 2 * rows * cols, d_stats, h->stream));
}

int qcs_select(qcs_handle_t h, const qcs_stats_t *d_statsA, const qcs_stats_t *d_statsB,
               qcs_gemm_desc_t *d_desc) {
    if (!h || !d_statsA || !d_statsB || !d_desc) return QCS_ERR_INVALID_ARG;
    return cuda_status(launch_select_from_stats(d_statsA, d_statsB, h->tol, d_desc, h->stream));
}

int qcs_cgemm(qcs_handle_t h, qcs_mode_t mode, qcs_op_t transA, qcs_op_t transB, int64_t m,
              int64_t n, int64_t k, const qcs_c32 *alpha, const qcs_c32 *A, int64_t lda,
              const qcs_c32 *B, int64_t ldb, const qcs_c32 *beta, qcs_c32 *C, int64_t ldc,
              qcs_gemm_desc_t *d_desc_out) {
    if (!h) return QCS_ERR_INVALID_ARG;
    if (int r = validate_cgemm(mode, transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc))
        return r;
    if (m == 0 || n == 0) return QCS_SUCCESS;
    if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) return QCS_ERR_UNSUPPORTED;
    const int eff = effective_mode(h, mode, transA, transB, m, n, k);
    const float2 al = make_float2(alpha->x, alpha->y), be = make_float2(beta->x, beta->y);
    if (h->complex_products == 3 && eff != QCS_MODE_FP32 && k > 0) {
        if (int r = ensure_workspace(h->ws, cgemm3m_workspace_bytes(eff, m, n, k, h->num_sms,
                                                                   h->tc_splits)))
            return r;
        return run_cgemm_3m(h, h->ws.ptr, eff, transA, transB, m, n, k, al,
                            reinterpret_cast<const float2 *>(A), lda,
                            reinterpret_cast<const float2 *>(B), ldb, be,
                            reinterpret_cast<float2 *>(C), ldc, d_desc_out);
    }
    if (h->rowcol && eff == QCS_MODE_AUTO && k > 0) {
        if (int r = ensure_workspace(h->ws, rowcol_workspace_bytes(
                                                m, n, k, h->num_sms,
                                                gemm_splits(h, transA, transB, m, n, k))))
            return r;
        return run_cgemm_rowcol(h, h->ws.ptr, transA, transB, m, n, k, al,
                                reinterpret_cast<const float2 *>(A), lda,
                                reinterpret_cast<const float2 *>(B), ldb, be,
                                reinterpret_cast<float2 *>(C), ldc, d_desc_out);
    }
    if (int r = ensure_workspace(h->ws, gemm_workspace_bytes(eff, m, n, k, h->num_sms,
                                                            gemm_splits(h, transA, transB, m, n, k), 1)))
        return r;
    return run_cgemm(h, h->ws.ptr, eff, transA, transB, m, n, k, al,
                     reinterpret_cast<const float2 *>(A), lda, reinterpret_cast<const float2 *>(B),
                     ldb, be, reinterpret_cast<float2 *>(C), ldc, d_desc_out, nullptr);
}

int qcs_sgemm(qcs_handle_t h, qcs_mode_t mode, qcs_op_t transA, qcs_op_t transB, int64_t m,
              int64_t n, int64_t k, const float *alpha, const float *A, int64_t lda,
              const float *B, int64_t ldb, const float *beta, float *C, int64_t ldc,
              qcs_gemm_desc_t *d_desc_out) {
    if (!h) return QCS_ERR_INVALID_ARG;
    if (!valid_mode(mode) || !valid_op(transA) || !valid_op(transB)) return QCS_ERR_INVALID_ARG;
    if (m < 0 || n < 0 || k < 0 || !alpha || !beta) return QCS_ERR_INVALID_ARG;
    const int64_t rowsA = (transA == QCS_OP_N) ? m : k;
    const int64_t rowsB = (transB == QCS_OP_N) ? k : n;
    if (lda < std::max<int64_t>(1, rowsA) || ldb < std::max<int64_t>(1, rowsB) ||
        ldc < std::max<int64_t>(1, m))
        return QCS_ERR_INVALID_ARG;
    if (m == 0 || n == 0) return QCS_SUCCESS;
    if (!C || (k > 0 && (!A || !B))) return QCS_ERR_INVALID_ARG;
    auto mis = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 3u) != 0; };
    if (mis(A) || mis(B) || mis(C)) return QCS_ERR_UNSUPPORTED;
    if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) return QCS_ERR_UNSUPPORTED;
    const int eff = effective_mode_real(h, mode, m, n, k);
    if (int r = ensure_workspace(h->ws, sgemm_workspace_bytes(eff, m, n, k, h->num_sms,
                                                             h->tc_splits)))
        return r;
    return run_sgemm(h, h->ws.ptr, eff, transA, transB, m, n, k, *alpha, A, lda, B, ldb, *beta, C,
                     ldc, d_desc_out);
}

int qcs_split(qcs_handle_t h, const qcs_gemm_desc_t *d_desc, int which, qcs_op_t op, int64_t R,
              int64_t K, const qcs_c32 *X, int64_t ldx, void *planes, int64_t pitch,
              int64_t plane_stride) {
    if (!h || !d_desc || !X || !planes || (which != 0 && which != 1) || !valid_op(op))
        return QCS_ERR_INVALID_ARG;
    if (R < 0 || K < 0 || pitch < K || plane_stride < R * pitch) return QCS_ERR_INVALID_ARG;
    const int64_t rows = (which == 0) ? ((op == QCS_OP_N) ? R : K) : ((op == QCS_OP_N) ? K : R);
    if (ldx < std::max<int64_t>(1, rows)) return QCS_ERR_INVALID_ARG;
    int64_t sr, sc;
    plane_strides(which, op, ldx, sr, sc);
    return cuda_status(launch_split(d_desc, which, reinterpret_cast<const float2 *>(X), sr, sc,
                                    op == QCS_OP_C, R, K, R, K, planes, pitch, plane_stride,
                                    h->stream));
}

int qcs_permute(qcs_handle_t h, int rank, const int64_t *dims, const int64_t *strides,
                int64_t offset, const qcs_c32 *in, qcs_c32 *out, qcs_stats_t *d_stats) {
    if (!h || rank < 0 || rank > QCS_MAX_RANK || (rank > 0 && (!dims || !strides)) || !in || !out)
        return QCS_ERR_INVALID_ARG;
    int64_t total = 1;
    for (int d = 0; d < rank; ++d) {
        if (dims[d] < 0) return QCS_ERR_INVALID_ARG;
        total *= dims[d];
    }
    cudaError_t e = launch_permute(rank, dims, strides, offset, reinterpret_cast<const float2 *>(in),
                                   reinterpret_cast<float2 *>(out), nullptr, 0, h->stream);
    if (e != cudaSuccess) return QCS_ERR_CUDA;
    if (d_stats) return qcs_exp_stats(h, total, 1, out, std::max<int64_t>(1, total), d_stats);
    return QCS_SUCCESS;
}

int qcs_set_profiling(qcs_handle_t h, int enabled) {
    if (!h) return QCS_ERR_INVALID_ARG;
    h->profiling = enabled ? 1 : 0;
    return QCS_SUCCESS;
}

int qcs_get_profile(qcs_handle_t h, double *ms, int64_t *counts, int n) {
    if (!h || !ms || n < 0) return QCS_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    for (int i = 0; i < n; ++i) {
        ms[i] = 0.0;
        if (counts) counts[i] = 0;
    }
    int rc = QCS_SUCCESS;
    for (const ProfEvent &pe : h->prof) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, pe.start, pe.stop) != cudaSuccess) {
            cudaGetLastError();
            rc = QCS_ERR_CUDA;
        } else if (pe.stage < n) {
            ms[pe.stage] += t;
            if (counts) counts[pe.stage] += 1;
        }
        h->event_pool.push_back(pe.start);
        h->event_pool.push_back(pe.stop);
    }
    h->prof.clear();
    return rc;
}

int qcs_sync(qcs_handle_t h) {
    if (!h) return QCS_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    int err = 0;
    if (cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return QCS_ERR_CUDA;
    if (err != 0) {
        cudaMemset(h->d_err, 0, sizeof(int));
        return QCS_ERR_TIMEOUT;
    }
    return QCS_SUCCESS;
}

int qcs_get_auto_counts(qcs_handle_t h, int64_t *counts, double *flops, int reset) {
    if (!h || !counts) return QCS_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    struct {
        unsigned long long c[QCS_NUM_MODES];
        double f[QCS_NUM_MODES];
    } d;
    static_assert(sizeof(d) + 8 <= kStatusBlockBytes, "status block");
    if (cudaMemcpy(&d, h->d_counts, sizeof(d), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    for (int i = 0; i < QCS_NUM_MODES; ++i) {
        counts[i] = (int64_t)d.c[i];
        if (flops) flops[i] = d.f[i];
    }
    if (reset && cudaMemset(h->d_counts, 0, sizeof(d)) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    return QCS_SUCCESS;
}

const char *qcs_status_string(int status) {
    switch (status) {
        case QCS_SUCCESS: return "success";
        case QCS_ERR_INVALID_ARG: return "invalid argument";
        case QCS_ERR_UNSUPPORTED: return "unsupported";
        case QCS_ERR_ALLOC: return "workspace allocation failed";
        case QCS_ERR_CUDA: return "CUDA runtime error";
        case QCS_ERR_TIMEOUT: return "device-side wait timed out";
        case QCS_ERR_SCRATCH_TOO_SMALL:
            return "problem needs more than the fixed scratch of qcs_cgemm_noalloc";
        default: return "unknown status";
    }
}

}  // extern "C"
