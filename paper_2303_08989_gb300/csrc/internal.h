// Internal declarations shared by the translation units of libqcs.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <map>
#include <tuple>
#include <vector>

#include "../../include/qcs.h"

namespace qcs {

// Error word codes written by kernels into the handle's device error word.
enum : int {
    kErrNone = 0,
    kErrTimeoutProducer = 1,
    kErrTimeoutMma = 2,
    kErrTimeoutEpilogue = 3,
};

// Wait budget of a device-side bounded wait (nanoseconds).  No legitimate
// wait inside one launch comes near it.
constexpr uint64_t kWaitBudgetNs = 2000000000ull;

// Tile geometry of the tensor-core GEMM.
constexpr int kBM = 128;          // complex rows of C per tile (TMEM lanes)
constexpr int kBN = 128;          // complex columns of C per tile
constexpr int kRowBytes = 64;     // K bytes of one smem operand row per stage (two MMA K steps)
constexpr int kStages = 3;
constexpr int kPlanes = 4;        // planes of op(A), and of op(B) in qcs_split: hi.re, hi.im, lo.re, lo.im
// op(B) in the GEMM path: five planes, so that the hi planes pair up as the
// 256-row B operands [-Bi; Br] and [Br; Bi] of N = 256 MMAs.
constexpr int kPlanesB = 5;       // -hi.im, hi.re, hi.im, lo.re, lo.im
constexpr int kTileBytes = kBM * kRowBytes;                // one plane tile: 8 KB
constexpr int kAStageBytes = kPlanes * kTileBytes;         // 32 KB
constexpr int kBStageBytes = kPlanesB * kTileBytes;        // 40 KB
constexpr int kStageBytes = kAStageBytes + kBStageBytes;   // 72 KB
constexpr int kTcThreads = 320;   // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int kTmemCols = 512;    // acc0 [re | im], acc1 [re | im] x 128 columns

// Split-K FP32 path for small outputs with long k: at most this many
// outputs, and at most this many (output, k chunk) partials in the scratch.
constexpr int64_t kSplitKMaxOutputs = 4096;
constexpr int64_t kSplitKMaxPartials = 16384;
constexpr size_t kSplitKBytes = size_t(kSplitKMaxPartials) * 8;

// Stats grid: blocks x threads, per-block partial histograms of 257 int64
// (256 bins + zero count).
constexpr int kStatsThreads = 128;
constexpr int kPartialStride = 257;
// handle's device status block: error word at byte 0, AUTO selection
// counts (6 uint64) at byte 8, their flops (6 doubles) at byte 56
constexpr size_t kStatusBlockBytes = 128;

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace qcs

namespace qcs {
enum ProfStage : int {
    kProfStats = 0,
    kProfSelect = 1,
    kProfSplit = 2,
    kProfGemmTc = 3,
    kProfGemmSimt = 4,
    kProfPermute = 5,
    kProfReduce = 6,
};
struct ProfEvent {
    int stage;
    cudaEvent_t start, stop;
};
}  // namespace qcs

struct qcs_handle_s {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    double tol = 0.0;
    int size_rule = 1;
    int drain_stages = 4;            // stages per RN drain of the tensor-core hi*hi sum
    int instance_batch = 1;          // contraction-tree instances per group (forward)
    int tc_group_m = 8;              // tensor-core raster: tile rows per group
    int tc_l2_promotion = 256;       // L2 promotion of the plane loads (bytes; 0 = none)
    int tc_splits = 0;               // K ranges per tensor-core GEMM (0 = chosen per shape)
    int complex_products = 4;        // real products per emulated complex product (4, or 3: Gauss)
    int fused_split = 0;             // TF32X: split inside the tensor-core kernel's staging
    int tree_levels = 1;             // tree executor: small FP32 steps of a level in one launch
    int tc_multicast = 0;            // complex tensor-core kernel in clusters of two sharing B
    int tc_pairs = 0;                // tensor-core kernels as CTA pairs (cta_group::2)
    int rowcol = 0;                  // AUTO: per-row / per-column scaling before TF32X
    const int *line_emax[2] = {nullptr, nullptr};  // set only inside run_cgemm_rowcol
    size_t group_budget = size_t(32) << 30;  // tree executor: bytes a grouped GPU-filling step may hold
    uint64_t wait_ns = qcs::kWaitBudgetNs;  // bound of the tensor-core kernels' device waits
    int debug_stall = 0;             // test hook: the TMA producer issues no loads
    int *d_err = nullptr;            // device error word (start of a 64-byte block)
    unsigned long long *d_counts = nullptr;  // in that block: AUTO selections per mode, flops
    qcs::Workspace ws;               // GEMM workspace (planes, partials, descriptor)
    qcs::Workspace tree_ws;          // contraction-tree intermediates
    qcs::EncodeTiledFn encode = nullptr;
    int profiling = 0;
    std::vector<qcs::ProfEvent> prof;     // recorded, not yet read
    std::vector<cudaEvent_t> event_pool;  // reusable events
    // (m, n, k, opA, opB) -> measured decision (QCS_SIZE_RULE_TUNED)
    std::map<std::tuple<int64_t, int64_t, int64_t, int, int>, qcs_tune_entry_t> tuned;
};

namespace qcs {
// Records a start event on construction and a stop event on destruction
// when the handle's profiling is on.
class ProfScope {
   public:
    ProfScope(qcs_handle_s *h, int stage);
    ~ProfScope();

   private:
    qcs_handle_s *h_;
    int idx_ = -1;
};
}  // namespace qcs

namespace qcs {

int ensure_workspace(Workspace &w, size_t bytes);

// A batch of equal-shape CGEMMs in one launch: entry g reads A + g sA,
// B + g sB and writes C + g sC (a stride of 0 shares the operand).
struct GemmBatch {
    int64_t count = 1;
    int64_t sA = 0, sB = 0, sC = 0;
};

// A batch of equal-shape copies in one launch: copy g reads from
// in + off[g * off_stride] (a device table; or in + g in_stride when off is
// NULL) and writes to out + g out_stride.
struct CopyBatch {
    int64_t count = 1;
    const int64_t *off = nullptr;
    int64_t off_stride = 0;
    int64_t in_stride = 0, out_stride = 0;
    // not NULL: copy g also writes out_off[g * out_off_stride] elements further
    const int64_t *out_off = nullptr;
    int64_t out_off_stride = 0;
    const qcs_gemm_desc_t *gate = nullptr;  // not NULL: copy only if that GEMM selected FP32
};

// ---- launchers (kernels.cu) ----------------------------------------------
// Exponent statistics of ``count_cols`` columns of ``rows`` complex values
// (leading dim ld) into per-block partials.  Two matrices in one launch:
// blocks [0, gA) take X0, [gA, gA+gB) take X1.
cudaError_t launch_stats2(const float2 *X0, int64_t rows0, int64_t cols0, int64_t ld0, int gA,
                          const float2 *X1, int64_t rows1, int64_t cols1, int64_t ld1, int gB,
                          int64_t *partials, cudaStream_t s);
// Reduce partials into qcs_stats_t (optional) and select the mode.
cudaError_t launch_select(const int64_t *partials, int gA, int gB, int64_t nA, int64_t nB,
                          double tol, int forced_mode, qcs_stats_t *statsA, qcs_stats_t *statsB,
                          qcs_gemm_desc_t *desc, cudaStream_t s);
// Two-stage statistics + selection for the GEMM path: pass 1 (e_max,
// zeros, Inf/NaN, count below 2^-14), pass 2 only when needed (count below
// the shifted window), final selection.  gA / gB blocks of 256 threads per
// matrix; p1 holds 5 int64 per block, p2 one.  ``counts`` (optional: 6
// uint64 indexed by qcs_mode_t, then 6 doubles) gets one increment and
// ``work`` (the GEMM's 8 m n k) added for the selected mode.  ``summary``
// (optional, 10 int64): the counts the selection used (qcs_selection_stats).
cudaError_t launch_stats_select_2stage(const float2 *X0, int64_t rows0, int64_t cols0, int64_t ld0,
                                       int gA, const float2 *X1, int64_t rows1, int64_t cols1,
                                       int64_t ld1, int gB, double tol, int forced, int64_t *p1,
                                       int64_t *p2, qcs_gemm_desc_t *desc,
                                       unsigned long long *counts, double work, cudaStream_t s,
                                       int64_t *summary = nullptr);
// The same for G instances in one launch each: instance g reads X0 + g dx0
// and X1 + g dx1, uses partials p1 + 5 g (gA + gB), p2 + g (gA + gB) and
// writes desc[g]; the counts are integers, so a decision does not depend on
// the batch or the block counts.
cudaError_t launch_stats_select_2stage_batch(const float2 *X0, int64_t rows0, int64_t cols0,
                                             int64_t ld0, int gA, int64_t dx0, const float2 *X1,
                                             int64_t rows1, int64_t cols1, int64_t ld1, int gB,
                                             int64_t dx1, int G, double tol, int forced,
                                             int64_t *p1, int64_t *p2, qcs_gemm_desc_t *desc,
                                             unsigned long long *counts, double work,
                                             cudaStream_t s);
int stats2_blocks(int64_t nel, int num_sms);
// Select from two finished qcs_stats_t.
cudaError_t launch_select_from_stats(const qcs_stats_t *a, const qcs_stats_t *b, double tol,
                                     qcs_gemm_desc_t *desc, cudaStream_t s);
// FP64 sums of a result against a reference (qcs_fidelity_stats): per-block
// partials (6 doubles per block, ``blocks`` blocks) then one block.
constexpr int kFidBlocksMax = 1024;
cudaError_t launch_fidelity_stats(const void *a, int a_c64, const double *ref, int64_t n,
                                  double *partials, int blocks, double *out, cudaStream_t s);

// Write a constant descriptor (forced mode).
cudaError_t launch_set_desc(qcs_gemm_desc_t *desc, int mode, cudaStream_t s, int count = 1);

// The splits of the same operand of ``count`` equal-shape GEMMs in one
// launch: instance g reads its operand in_stride elements after that of
// instance g - 1, takes descriptor desc + g, and writes its rows
// off_stride elements after those of instance g - 1 in every plane.
struct SplitBatch {
    int count = 1;
    int64_t in_stride = 0;
    int64_t off_stride = 0;
};

// Split op(X) into 4 planes (R x K, row pitch ``pitch`` elements, planes
// ``plane_stride`` elements apart); rows >= R or columns >= K up to
// R_pad x K_pad are zero-filled.  (sr, sc): element strides of X for a step
// in r and in c; conj: negate imaginary parts.  planes6 (the name predates
// the layout): the kPlanesB-plane op(B) layout of the tensor-core GEMM
// (-hi.im, hi.re, hi.im, lo.re, lo.im).  plane_off: element offset of row 0
// in every plane (instance g of a group of equal-shape GEMMs writes its rows
// after those of instances 0 .. g-1); elements are those of the kind the
// descriptor selected.  planes32 (not NULL): where a TF32 selection writes
// instead of ``planes`` -- a group whose instances may select different
// kinds keeps the 2-byte and 4-byte planes in separate regions.  skip_tf32:
// write nothing for a TF32 selection (the fused TF32X kernel splits itself).
// qcs_gemm_desc_t::reserved value of a descriptor whose FP16 split scales
// every row of op(A) and every column of op(B) by its own power of two (the
// per-line exponents passed to launch_split / launch_rowcol_combine).
constexpr int kDescLineScales = 1;

// Per-row / per-column power-of-two scaling (qcs_set_rowcol_scaling).
// launch_line_emax: for each row (per_row = 1) or column (0) of the stored
// rows x cols matrix X (column-major, ld), the largest biased binary32
// exponent over its nonzero finite real and imaginary scalars, -1 if none
// (emax is cleared first).  launch_line_under: counts[0] += scalars below the
// line's shifted window (biased exponent 0, or below emax - 28), counts[1] +=
// nonzero finite scalars (counts must be cleared by the caller).
cudaError_t launch_line_emax(const float2 *X, int64_t rows, int64_t cols, int64_t ld, int per_row,
                             int *emax, cudaStream_t s);
cudaError_t launch_line_under(const float2 *X, int64_t rows, int64_t cols, int64_t ld,
                              int per_row, const int *emax, unsigned long long *counts,
                              cudaStream_t s);
// descK (for the kernels) and descOut (reported) from the Section 4.1
// selection desc0 and counts[4] = {under A, nonzero A, under B, nonzero B}.
cudaError_t launch_rowcol_select(const qcs_gemm_desc_t *desc0, const unsigned long long *counts,
                                 double tol, qcs_gemm_desc_t *descK, qcs_gemm_desc_t *descOut,
                                 cudaStream_t s);
// C = alpha D_A^-1 P D_B^-1 + beta C (D: the per-line scales when descK
// carries kDescLineScales, else the identity); P is m x n with ld m.
cudaError_t launch_rowcol_combine(const qcs_gemm_desc_t *descK, const int *emaxA,
                                  const int *emaxB, const float2 *P, int64_t m, int64_t n,
                                  float2 alpha, float2 beta, float2 *C, int64_t ldc, int num_sms,
                                  cudaStream_t s);

cudaError_t launch_split(const qcs_gemm_desc_t *desc, int which, const float2 *X, int64_t sr,
                         int64_t sc, int conj, int64_t R, int64_t K, int64_t R_pad, int64_t K_pad,
                         void *planes, int64_t pitch, int64_t plane_stride, cudaStream_t s,
                         int planes6 = 0, int64_t plane_off = 0, void *planes32 = nullptr,
                         int skip_tf32 = 0, const SplitBatch &sb = SplitBatch{},
                         const int *line_emax = nullptr);

// The split stage reading its operand through a gather map (the reshape of
// a contraction folded into the split pass): op(X) is the rows x cols
// column-major matrix whose element t = i + l rows is
// src[sum_d x_d strides[d]] with t decomposed over dims (first fastest), as
// qcs_gather_t describes it; ``which`` 0 writes it as the A planes (R = rows,
// K = cols), 1 as the B planes (R = cols, K = rows).  No padding is written:
// the caller needs R and K to be the padded sizes.  NotSupported (nothing
// launched) when the map does not tile; split_gather_supported tells first.
bool split_gather_supported(int which, int rank, const int64_t *dims, const int64_t *strides,
                            int64_t rows, int64_t pitch);
cudaError_t launch_split_gather(const qcs_gemm_desc_t *desc, int which, int rank,
                                const int64_t *dims, const int64_t *strides, const float2 *src,
                                int64_t rows, void *planes, int64_t pitch, int64_t plane_stride,
                                cudaStream_t s, int planes6 = 0, int64_t plane_off = 0,
                                void *planes32 = nullptr, const SplitBatch &sb = SplitBatch{});
cudaError_t launch_permute(int rank, const int64_t *dims, const int64_t *strides, int64_t offset,
                           const float2 *in, float2 *out, int64_t *stats_partials, int gstats,
                           cudaStream_t s, const CopyBatch &cb = CopyBatch{});
cudaError_t launch_stats_finalize(const int64_t *partials, int g, int64_t n, qcs_stats_t *out,
                                  cudaStream_t s);
cudaError_t launch_accumulate_c128(const float2 *src, double *dst, int64_t count, int overwrite,
                                   cudaStream_t s);
cudaError_t launch_scatter(int rank, const int64_t *dims, const int64_t *strides, int64_t offset,
                           const float2 *src, float2 *dst, int accumulate, cudaStream_t s,
                           const CopyBatch &cb = CopyBatch{});
cudaError_t launch_accumulate_gather_c128(const float2 *src, const int64_t *index, double *dst,
                                          int64_t count, cudaStream_t s);
cudaError_t launch_seed_grad(const double *g, const int64_t *index, float2 *grad_root,
                             int64_t count, cudaStream_t s);

// One small plain-FP32 contraction step of a tree level, as the level launch
// reads it.  op(A) (m x k) and op(B) (k x n) are read element by element
// through offset tables (element e = i + l m of op(A) lies at
// a[tab[a_tab + e]], likewise op(B) with e = l + j k), which fold the step's
// gather map (or its direct N / T layout) into the load; C (m x n) is written
// dense.  Instance r of the launch (position g0 + r of its group, instance
// inst0 + r of the plan) reads a leaf operand at its per-instance offset
// off[inst nl + leaf] and an intermediate at g istride.
struct TreeSmallStep {
    const float2 *a, *b;
    float2 *c;
    int64_t a_istride, b_istride, c_istride;
    int32_t a_leaf, b_leaf;  // leaf index, or -1 for an intermediate
    int32_t m, n, k;
    int32_t a_tab, b_tab;
    int32_t pad;
};
constexpr int64_t kTreeSmallOperand = 1024;  // max elements of op(A) and of op(B)
constexpr int64_t kTreeSmallOutput = 4096;   // max elements of C
// steps[0 .. n_steps) for G instances each: one warp per (step, instance),
// smem_elems complex values of shared memory per warp (>= m k + k n).
cudaError_t launch_tree_small(const TreeSmallStep *steps, int n_steps, int G, int inst0, int g0,
                              const int64_t *off, int nl, const int32_t *tab, int smem_elems,
                              cudaStream_t s);

// The adjoint of one small step: from the output gradient gc (m x n, dense)
// grad_A = gc op(B)^H and grad_B = op(A)^H gc, written through the operands'
// offset tables into their gradients: ga[tab[a_tab + e]] (added for a leaf,
// at its instance offset; stored for an intermediate, whose map covers it
// once), likewise gb.  Instance r of the launch (position r of its group,
// instance inst0 + r) reads an intermediate operand r a_istride further,
// writes its gradients r ga_istride further (for a leaf too: its own
// gradient buffer of the group), and takes gc r gc_istride further.
struct TreeSmallBwd {
    const float2 *a, *b, *gc;
    float2 *ga, *gb;
    int64_t a_istride, b_istride, ga_istride, gb_istride, gc_istride;
    int32_t a_leaf, b_leaf;  // leaf index, or -1 for an intermediate
    int32_t m, n, k;
    int32_t a_tab, b_tab;
    int32_t pad;
};
constexpr int64_t kTreeSmallBwdElems = 2048;  // max m n + m k + k n of a step's adjoint
cudaError_t launch_tree_small_bwd(const TreeSmallBwd *steps, int n_steps, int G, int inst0,
                                  const int64_t *off, int nl, const int32_t *tab, int smem_elems,
                                  cudaStream_t s);

// grad[i][e] += scratch[g stride + leaf_off[i] + e] for g = 0 .. G-1 in
// order, for every leaf i (the leaf gradients of a group of instances of
// the adjoint, each instance's in its own buffer, added in instance order).
struct LeafGradRef {
    float2 *grad;
    int64_t size, scratch_off;
};
cudaError_t launch_leaf_grad_reduce(const LeafGradRef *leaves, int nl, int64_t max_size,
                                    const float2 *scratch, int64_t stride, int G, cudaStream_t s);

// ---- shared with the executor (capi.cu) ------------------------------------
int effective_mode(qcs_handle_t h, int mode, int opA, int opB, int64_t m, int64_t n, int64_t k);
// K-range setting for a GEMM of this shape: forced, tuned, or 0 (per-shape rule).
int gemm_splits(qcs_handle_t h, int opA, int opB, int64_t m, int64_t n, int64_t k);
// Raster group of the tensor-core GEMMs of this shape (tuned, else the handle's).
int gemm_group_m(qcs_handle_t h, int opA, int opB, int64_t m, int64_t n, int64_t k);
// Time the candidate modes of one shape (qcs_autotune_gemm without validation).
int tune_shape(qcs_handle_t h, int opA, int opB, int64_t m, int64_t n, int64_t k, int reps,
               qcs_tune_entry_t *out);
// ``splits``: the handle's K-range setting (0 = chosen per shape); ``G``:
// equal-shape GEMMs run as one group (run_cgemm_group).
size_t gemm_workspace_bytes(int eff, int64_t m, int64_t n, int64_t k, int num_sms, int splits,
                            int G = 1);
// ``bt``: a batch of equal-shape GEMMs (plain FP32 only; UNSUPPORTED otherwise).
// Host-side argument checks of qcs_cgemm (QCS_SUCCESS or an error code).
int validate_cgemm(int mode, int opA, int opB, int64_t m, int64_t n, int64_t k, const void *alpha,
                   const void *A, int64_t lda, const void *B, int64_t ldb, const void *beta,
                   const void *C, int64_t ldc);

int run_cgemm(qcs_handle_t h, void *ws, int eff, int opA, int opB, int64_t m, int64_t n, int64_t k,
              float2 alpha, const float2 *A, int64_t lda, const float2 *B, int64_t ldb, float2 beta,
              float2 *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out, const qcs_gemm_desc_t *d_desc_in,
              const GemmBatch &bt = GemmBatch{});

// An operand of run_cgemm_views: the column-major matrix X (leading
// dimension ld, the GEMM's op applied), or -- when ``map`` is set -- op(X)
// (op must be N) read through that gather map from the tensor X, whose
// ``flat`` elements the map permutes as a whole (``flat`` = 0: the map reads
// part of X, for instance one slice, and op(X) is always gathered).  ``buf``
// (room for the gathered matrix) receives op(X) when a kernel needs it as a
// matrix: the FP32 path, or a split that cannot read through the map.
struct OperandView {
    const float2 *X = nullptr;
    int64_t ld = 0;
    const qcs_gather_t *map = nullptr;
    int64_t flat = 0;
    float2 *buf = nullptr;
};
// run_cgemm with operand views: a mapped operand of an emulated GEMM is never
// gathered -- its statistics read the tensor as stored (a permutation keeps
// the multiset of exponents), its split reads through the map, and only the
// FP32 candidate of AUTO gathers it, when (and only when) that candidate was
// selected.
int run_cgemm_views(qcs_handle_t h, void *ws, int eff, int opA, int opB, int64_t m, int64_t n,
                    int64_t k, float2 alpha, const OperandView &A, const OperandView &B,
                    float2 beta, float2 *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out,
                    const qcs_gemm_desc_t *d_desc_in, const GemmBatch &bt = GemmBatch{});
// G equal-shape emulated GEMMs as one group (the instances of a contraction
// step): instance g reads A[g], B[g] and writes C + g c_stride.  Per instance
// the gathers, statistics, selection (its own descriptor) and split; then one
// tensor-core launch per kind over the tiles of every instance (each unit
// runs only if its instance selected that kind), and for AUTO the FP32
// candidate of each instance, gated by its descriptor.  G = 1 is
// run_cgemm_views.  ``ws``: gemm_workspace_bytes(..., G) bytes.
int run_cgemm_group(qcs_handle_t h, void *ws, int eff, int opA, int opB, int64_t m, int64_t n,
                    int64_t k, float2 alpha, const OperandView *A, const OperandView *B, int G,
                    float2 beta, float2 *C, int64_t ldc, int64_t c_stride,
                    qcs_gemm_desc_t *d_desc_out, const qcs_gemm_desc_t *d_desc_in,
                    const GemmBatch &bt = GemmBatch{});

// ---- GEMM launchers -------------------------------------------------------
// Plain FP32 SIMT CGEMM (runs only when desc->mode == FP32, or always when
// desc is NULL).
cudaError_t launch_cgemm_simt(const qcs_gemm_desc_t *desc, int opA, int opB, int64_t m,
                              int64_t n, int64_t k, float2 alpha, const float2 *A, int64_t lda,
                              const float2 *B, int64_t ldb, float2 beta, float2 *C, int64_t ldc,
                              float2 *splitk, cudaStream_t s, const GemmBatch &bt = GemmBatch{});
// Work of one tensor-core launch: G equal-shape GEMMs, each with its K loop
// split into S ranges.  Instance g reads its A planes from row g * a_rows of
// the A tensor map (its B planes from row g * b_rows), its descriptor from
// desc[g], and writes C + g * c_stride.  S > 1: every range writes its
// partial into P ([r][g] blocks of m x n complex, column-major, ld m) and
// launch_tc_reduce then forms C.
// ``wait_ns`` bounds every device-side wait of the launch; ``stall`` (a test
// hook, qcs_debug_stall_producer) makes the TMA producer issue no loads, so
// that the MMA issuer's first wait runs out and the launch records a timeout.
struct TcWork {
    int G = 1, S = 1;
    int64_t a_rows = 0, b_rows = 0, c_stride = 0;
    float2 *P = nullptr;
    uint64_t wait_ns = kWaitBudgetNs;
    int stall = 0;
};
constexpr int kMaxSplits = 16;
// K ranges for a launch over G GEMMs of m x n x k: ``forced`` > 0 is taken
// (at most one range per 32 k), 0 chooses from the wave count and the cost
// of the partials.
// ``real``: the real kernel's 128 x 256 tiles and 4-byte outputs.
int tc_split_count(int64_t m, int64_t n, int64_t k, int64_t G, int num_sms, int forced,
                   bool real = false);

// TF32X CGEMM with the Eq. 1 split in the tensor-core kernel's staging: the
// kernel reads A and B as stored (op N / T / C), one GEMM, one K range; it
// runs only if desc->mode is TF32X.  tc_fused_supported: the TMA limits
// (even lda, ldb; 16-byte aligned A, B; sizes within int).
bool tc_fused_supported(int opA, int opB, int64_t m, int64_t n, int64_t k, const float2 *A,
                        int64_t lda, const float2 *B, int64_t ldb);
cudaError_t launch_cgemm_tc_fused(EncodeTiledFn encode, const qcs_gemm_desc_t *desc, int opA,
                                  int opB, int64_t m, int64_t n, int64_t k, float2 alpha,
                                  const float2 *A, int64_t lda, const float2 *B, int64_t ldb,
                                  float2 beta, float2 *C, int64_t ldc, int *d_err, int num_sms,
                                  int group_m, const TcWork &w, cudaStream_t s);

// Tensor-core emulated CGEMM over split planes.  ``kind``: 0 FP16 (modes
// FP16X, FP16X_SCALED), 1 TF32, 2 BF16; the kernel returns at once unless
// desc->mode belongs to its kind (per instance when w.G > 1).
// ``drain``: pipeline stages per round-to-nearest drain of the hi*hi
// accumulator (1, 2 or 4).  When the output has an even number of tile
// rows: pairB not NULL (and drain 4) runs CTA pairs on M = 256 tiles
// (pairB[0]: the B planes in boxes of 128 rows x 2 planes, pairB[1]: 64 rows
// x 2 planes); else mcB not NULL runs clusters of two CTAs sharing the B
// boxes (mcB[0]: planes 0-2 of each box, mcB[1]: planes 3-4).  Otherwise
// mapB (all five planes of a box).
cudaError_t launch_cgemm_tc(int kind, int drain, const qcs_gemm_desc_t *desc,
                            const CUtensorMap *mapA, const CUtensorMap *mapB, int64_t m,
                            int64_t n, int64_t k_pad, float2 alpha, float2 beta, float2 *C,
                            int64_t ldc, int *d_err, int num_sms, int group_m, cudaStream_t s,
                            const TcWork &w = TcWork{}, const CUtensorMap *mcB = nullptr,
                            const CUtensorMap *pairB = nullptr);
// C = alpha sum_r P_r + beta C after a split-K launch (nothing when w.S == 1),
// for the instances whose descriptor did not select FP32.
cudaError_t launch_tc_reduce(const qcs_gemm_desc_t *desc, int64_t m, int64_t n, float2 alpha,
                             float2 beta, float2 *C, int64_t ldc, int num_sms, const TcWork &w,
                             cudaStream_t s);

// ---- real GEMM (qcs_sgemm) ------------------------------------------------
// The two-stage statistics + selection over real matrices (one scalar per
// element); otherwise as launch_stats_select_2stage.
cudaError_t launch_stats_select_2stage_real(const float *X0, int64_t rows0, int64_t cols0,
                                            int64_t ld0, int gA, const float *X1, int64_t rows1,
                                            int64_t cols1, int64_t ld1, int gB, double tol,
                                            int forced, int64_t *p1, int64_t *p2,
                                            qcs_gemm_desc_t *desc, unsigned long long *counts,
                                            double work, cudaStream_t s);
// Split a real op(X) (element (r, c) at X[r sr + c sc]) into the planes hi
// and lo (R_pad x K_pad, pitch elements per row, plane_stride apart), zero
// beyond R x K; elements of the kind the descriptor selected.
cudaError_t launch_split_real(const qcs_gemm_desc_t *desc, int which, const float *X, int64_t sr,
                              int64_t sc, int64_t R, int64_t K, int64_t R_pad, int64_t K_pad,
                              void *planes, int64_t pitch, int64_t plane_stride, cudaStream_t s);
// Gauss's three-product CGEMM: desc[1], desc[2] from the selected desc[0]
// (the T3 operand sums lose one binade of FP16 scaling), and the final
// combination C = alpha (T1 - T2 + i (T3 - T1 - T2)) + beta C.
cudaError_t launch_derive_3m_desc(qcs_gemm_desc_t *desc, cudaStream_t s);
// The three real operands of a Gauss product (real parts, imaginary parts,
// their binary32 sum) split in one pass over the complex op(X) (complex
// strides sr, sc; conj negates imaginary parts): part p's planes at element
// offset p part_off; desc[0]'s scale for parts 0 and 1, desc[2]'s for part 2.
cudaError_t launch_split_gauss(const qcs_gemm_desc_t *desc, int which, const float2 *X, int64_t sr,
                               int64_t sc, int conj, int64_t R, int64_t K, int64_t R_pad,
                               int64_t K_pad, void *planes, int64_t pitch, int64_t plane_stride,
                               int64_t part_off, cudaStream_t s);
cudaError_t launch_combine_3m(const qcs_gemm_desc_t *desc, int64_t m, int64_t n, const float *T,
                              float2 alpha, float2 beta, float2 *C, int64_t ldc, int num_sms,
                              cudaStream_t s);
// Plain FP32 real GEMM (runs only when desc->mode == FP32, or always when
// desc is NULL).
cudaError_t launch_sgemm_simt(const qcs_gemm_desc_t *desc, int opA, int opB, int64_t m,
                              int64_t n, int64_t k, float alpha, const float *A, int64_t lda,
                              const float *B, int64_t ldb, float beta, float *C, int64_t ldc,
                              cudaStream_t s);
// The tensor-core kernel on real planes: A two planes (hi, lo) read in
// 128-row boxes, B two planes in 256-row boxes, tiles of 128 x 256 floats of
// C; w.P (when w.S > 1) holds S G m n floats.  pairB not NULL (the B planes
// in 128-row boxes; drain 4, an even number of tile rows): CTA pairs on
// 256 x 256 tiles.
cudaError_t launch_sgemm_tc(int kind, int drain, const qcs_gemm_desc_t *desc,
                            const CUtensorMap *mapA, const CUtensorMap *mapB, int64_t m,
                            int64_t n, int64_t k_pad, float alpha, float beta, float *C,
                            int64_t ldc, int *d_err, int num_sms, int group_m, cudaStream_t s,
                            const TcWork &w = TcWork{}, const CUtensorMap *pairB = nullptr);
cudaError_t launch_tc_reduce_real(const qcs_gemm_desc_t *desc, int64_t m, int64_t n, float alpha,
                                  float beta, float *C, int64_t ldc, int num_sms, const TcWork &w,
                                  cudaStream_t s);
// Gauss's three-product form of one emulated CGEMM (qcs_set_complex_products 3).
// AUTO with per-row / per-column scaling (qcs_set_rowcol_scaling): the
// Section 4.1 selection, the per-line statistics and the decision, then
// run_cgemm on the selected descriptor into a scratch product, then the
// combine with the line scales, alpha and beta.
size_t rowcol_workspace_bytes(int64_t m, int64_t n, int64_t k, int num_sms, int splits);
cudaError_t rowcol_line_stats(cudaStream_t s, int opA, int opB, int64_t m, int64_t n, int64_t k,
                              const float2 *A, int64_t lda, const float2 *B, int64_t ldb,
                              int *emaxA, int *emaxB, unsigned long long *counts);
int run_cgemm_rowcol(qcs_handle_t h, void *ws, int opA, int opB, int64_t m, int64_t n, int64_t k,
                     float2 alpha, const float2 *A, int64_t lda, const float2 *B, int64_t ldb,
                     float2 beta, float2 *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out);
size_t cgemm3m_workspace_bytes(int eff, int64_t m, int64_t n, int64_t k, int num_sms, int splits);
int run_cgemm_3m(qcs_handle_t h, void *ws, int eff, int opA, int opB, int64_t m, int64_t n,
                 int64_t k, float2 alpha, const float2 *A, int64_t lda, const float2 *B,
                 int64_t ldb, float2 beta, float2 *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out);
// Workspace of one real GEMM and its launch sequence (as run_cgemm, G = 1).
size_t sgemm_workspace_bytes(int eff, int64_t m, int64_t n, int64_t k, int num_sms, int splits);
int run_sgemm(qcs_handle_t h, void *ws, int eff, int opA, int opB, int64_t m, int64_t n, int64_t k,
              float alpha, const float *A, int64_t lda, const float *B, int64_t ldb, float beta,
              float *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out);

}  // namespace qcs
