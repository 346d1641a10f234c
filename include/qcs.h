/*
 * qcs.h -- C ABI of the GB300 (sm_103a) library for tensor-network quantum
 * circuit simulation by error-corrected SGEMM emulation on tensor cores with
 * automatic precision selection (Ootomo, Manabe, Harada, Yokota, 2023).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Matrices are BLAS column-major.  A complex number is qcs_c32 (two
 *   floats, real then imaginary: layout-compatible with cuComplex and
 *   torch.complex64).  Element (i, j) of a matrix X with leading dimension
 *   ldx is X[i + j * ldx].
 * - op(X): QCS_OP_N uses X as stored, QCS_OP_T its transpose, QCS_OP_C its
 *   conjugate transpose.
 * - Pointers marked "device" are CUDA device pointers owned by the caller;
 *   the library never frees or keeps them beyond the call's stream work.
 *   Pointers marked "host" are read during the call only.
 * - Every call is asynchronous on the handle's stream and never waits for
 *   the GPU (Section 4.2: the statistics never travel to the host).
 *   Argument errors are found on the host and returned before any launch.
 *   Errors raised on the device (a bounded wait that ran out) are recorded
 *   in a device error word and returned by the next qcs_sync().
 * - Return value: QCS_SUCCESS (0) or a negative QCS_ERR_* code.
 * - No call takes or returns ownership of memory: the handle owns its
 *   workspace (allocated with cudaMalloc on first need, grown on demand,
 *   freed by qcs_destroy).
 */
#ifndef QCS_H
#define QCS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QCS_SUCCESS 0
#define QCS_ERR_INVALID_ARG (-1) /* bad pointer, size, leading dimension, enum or plan */
#define QCS_ERR_UNSUPPORTED (-2) /* valid request this build cannot run (e.g. alignment) */
#define QCS_ERR_ALLOC (-3)       /* cudaMalloc of the workspace failed */
#define QCS_ERR_CUDA (-4)        /* a CUDA runtime call failed */
#define QCS_ERR_TIMEOUT (-5)     /* a device-side bounded wait ran out (see qcs_sync) */
#define QCS_ERR_SCRATCH_TOO_SMALL (-6) /* qcs_cgemm_noalloc: problem needs more than its fixed scratch */

typedef struct qcs_handle_s *qcs_handle_t;

/* GEMM computing modes.  Section 2.1 / Table 1 define FP16TCEC and TF32TCEC,
 * Section 4 adds FP16TCEC with scaling and the automatic choice between them;
 * FP32 is the plain single-precision SIMT baseline; BF16X3 is a measured
 * candidate with the same split on bfloat16 parts (not chosen by AUTO). */
typedef enum {
    QCS_MODE_AUTO = 0,
    QCS_MODE_FP16X = 1,
    QCS_MODE_FP16X_SCALED = 2,
    QCS_MODE_TF32X = 3,
    QCS_MODE_FP32 = 4,
    QCS_MODE_BF16X3 = 5
} qcs_mode_t;
#define QCS_NUM_MODES 6
/* Reported only (in a qcs_cgemm call's d_desc_out, never accepted as an
 * argument): FP16 emulation with every row of op(A) and every column of
 * op(B) scaled by its own power of two (qcs_set_rowcol_scaling). */
#define QCS_MODE_FP16X_ROWCOL 6

typedef enum { QCS_OP_N = 0, QCS_OP_T = 1, QCS_OP_C = 2 } qcs_op_t;

typedef struct {
    float x, y;
} qcs_c32;

/* Exponent statistics of one matrix (Section 4.1), device-resident.
 * Every real and every imaginary scalar x counts once.  For x != 0,
 * e = floor(log2 |x|); hist[e + 127] counts normal binary32 numbers,
 * hist[0] subnormal ones and hist[255] Inf/NaN.  Zeros enter no bin and are
 * counted in n_zero.  n is the total number of scalars (2 * rows * cols). */
typedef struct {
    int64_t hist[256];
    int64_t n_zero;
    int64_t n;
} qcs_stats_t;

/* Per-GEMM mode descriptor written on the device by the selector (the
 * "mode flag buffer" of Section 4.2): the chosen qcs_mode_t and the
 * power-of-two exponents sA, sB applied to op(A), op(B) before the split
 * (zero unless mode is FP16X_SCALED; the product is multiplied by
 * 2^-(sA+sB) in the epilogue). */
typedef struct {
    int32_t mode;
    int32_t sA;
    int32_t sB;
    int32_t reserved;
} qcs_gemm_desc_t;

/* Create a handle bound to the current CUDA device and to ``cuda_stream``
 * (a cudaStream_t; NULL = legacy default stream).  Returns INVALID_ARG if
 * ``out`` is NULL, CUDA if no device is usable. */
int qcs_create(qcs_handle_t *out, void *cuda_stream);

/* Destroy a handle: synchronizes its stream, frees its workspace. */
int qcs_destroy(qcs_handle_t h);

/* Rebind the handle to another stream (subsequent calls only). */
int qcs_set_stream(qcs_handle_t h, void *cuda_stream);

/* Underflow tolerance t of Section 4.1 (the "underflow admissibility
 * threshold", AUTO-t of Section 5.2), in [0, 1].  An operand tolerates a
 * mode when at most t * (number of nonzero finite scalars) of its scalars
 * fall outside that mode's exponent window.  Default 0 (no underflow). */
int qcs_set_underflow_tol(qcs_handle_t h, double t);

/* Size rule for QCS_MODE_AUTO (Section 4.3: small GEMMs do not repay the
 * statistics and split passes):
 *   QCS_SIZE_RULE_OFF    AUTO always selects from the statistics;
 *   QCS_SIZE_RULE_PAPER  the paper's cut-offs, measured on its GPU:
 *                        min(m,n,k) >= 2048 -> automatic selection, >= 512 ->
 *                        TF32X, else FP32 (default);
 *   QCS_SIZE_RULE_TUNED  the decision measured on this GPU for the shape by
 *                        qcs_autotune_gemm / qcs_autotune_tree (or loaded
 *                        with qcs_set_tuning); shapes never tuned fall back
 *                        to the PAPER cut-offs.
 * Any other nonzero value means PAPER. */
#define QCS_SIZE_RULE_OFF 0
#define QCS_SIZE_RULE_PAPER 1
#define QCS_SIZE_RULE_TUNED 2
int qcs_set_size_rule(qcs_handle_t h, int rule);

/* Round-to-nearest drain interval of the tensor-core kernels: the hi*hi
 * products are summed in tensor memory over groups of 2 x ``stages``
 * tensor-core K steps (32 x ``stages`` complex k for FP16/BF16, 16 x
 * ``stages`` for TF32), where the hardware accumulation truncates, then
 * added to round-to-nearest FP32 sums (Section 2.1's remedy for the tensor
 * core's rounding toward zero, applied per group of MMAs).  1, 2 or 4;
 * default 4 (environment override QCS_DRAIN_STAGES).  Larger groups are
 * faster and slightly less accurate. */
int qcs_set_drain_stages(qcs_handle_t h, int stages);

/* Schedule of the tensor-core kernels (a performance knob; results do not
 * depend on it): output tiles are processed in a raster of groups of
 * ``group_m`` tile rows (1 to 1024; default 8), column after column inside a
 * group, so that tiles in flight share operand panels in L2; the split
 * planes are loaded with an L2 promotion of ``l2_promotion`` bytes (0, 64,
 * 128 or 256; default 256).  Environment overrides QCS_TC_GROUP_M and
 * QCS_TC_L2_PROMOTION. */
int qcs_set_tc_schedule(qcs_handle_t h, int group_m, int l2_promotion);

/* Clusters of the complex tensor-core kernel (a schedule; results do not
 * depend on it).  While ``enabled`` is 1 the kernel runs as clusters of two
 * CTAs on pairs of tile rows of the same tile column, in lockstep: each
 * loads part of the shared op(B) box of a stage and multicasts it to both
 * (TMA multicast within the cluster), so each CTA reads half as much of B
 * from L2; a stage is released when the MMAs of both CTAs have read it.
 * Used when the output has an even number of 128-row tile rows.  Default 0;
 * environment override QCS_TC_MULTICAST.  QCS_ERR_INVALID_ARG for other
 * values. */
int qcs_set_tc_multicast(qcs_handle_t h, int enabled);

/* CTA pairs for the tensor-core kernels (a schedule; each output element is
 * the same sequence of tensor-core products in the same order either way).
 * While ``enabled`` is 1 the complex and real kernels run in clusters of two
 * CTAs, each cluster on one 256-row tile (two 128-row tile rows of the same
 * tile column) with tcgen05 MMAs of cta_group::2: each CTA holds its 128
 * rows of op(A) and half of every op(B) operand of a stage, and one thread
 * of the even CTA issues the MMAs of both, so each tensor core reads half as
 * many op(B) bytes per MMA from shared memory.  Used when the output has an
 * even number of 128-row tile rows and the drain is 4 stages (the default);
 * takes precedence over qcs_set_tc_multicast.  Default 0; environment
 * override QCS_TC_PAIRS.  QCS_ERR_INVALID_ARG for other values. */
int qcs_set_tc_pairs(qcs_handle_t h, int enabled);

/* K ranges of the tensor-core kernels.  A GEMM with few 128 x 128 output
 * tiles for its K (for example m = n = 1024: 64 tiles on 152 SMs) leaves
 * SMs idle; its K loop can be cut into ``splits`` equal ranges that run as
 * separate work units.  Each range writes its partial product (FP32, in the
 * handle's workspace: splits x m x n complex) and one more kernel adds the
 * ranges in a fixed order and applies alpha and beta, so results are
 * deterministic but differ from the unsplit GEMM by FP32 rounding of the
 * partial sums.  ``splits`` = 0 (default) chooses the count per shape from
 * the number of tile waves and the partials' memory traffic; 1 to 16 forces
 * it (at most one range per 32 k).  Environment override QCS_TC_SPLITS.
 * This is a schedule of Section 2.1's emulation, not a step of the paper.
 * Returns QCS_ERR_INVALID_ARG for other values. */
int qcs_set_tc_splits(qcs_handle_t h, int splits);

/* Per-row / per-column power-of-two scaling for AUTO (a variant beyond the
 * paper: the scaling basis of Section 4.1, where one power of two per
 * matrix moves its largest exponent to 14, applied to each row of op(A) and
 * each column of op(B) instead).  While ``enabled`` is 1, a qcs_cgemm call
 * whose mode after the size rule is AUTO (k > 0, four real products) first
 * selects as Section 4.1 does.  If that selection is TF32X, row i of op(A)
 * is scaled by 2^(14 - e_max(i)) and column j of op(B) by 2^(14 - e_max(j))
 * (e_max over the nonzero finite real and imaginary scalars of the line; a
 * line without any keeps scale 1), and the GEMM runs as FP16 emulation when
 * each operand's count of nonzero scalars below its lines' shifted windows
 * [e_max - 28, e_max] (binary32 subnormals included) is at most t times its
 * nonzero count, t the underflow tolerance; the product is multiplied back
 * by 2^-(sA_i + sB_j), then alpha and beta are applied.  d_desc_out then
 * reports QCS_MODE_FP16X_ROWCOL with sA = sB = 0; otherwise the call gives
 * what it gives with the option off.  The call takes a further m x n complex
 * product and the line statistics (two passes over A and B) from the
 * handle's workspace.  Default 0; QCS_ERR_INVALID_ARG for other values. */
int qcs_set_rowcol_scaling(qcs_handle_t h, int enabled);

/* The per-line statistics of qcs_set_rowcol_scaling for op(A) (m x k) and
 * op(B) (k x n) as stored (A: lda, B: ldb, column-major, device): the
 * largest biased binary32 exponent of every row of op(A) into d_emaxA[m] and
 * of every column of op(B) into d_emaxB[n] (-1 for a line without a nonzero
 * finite scalar; real and imaginary parts count separately), and into
 * d_counts[4]: op(A)'s nonzero scalars below their row's shifted window
 * (biased exponent 0, or below e_max - 28), op(A)'s nonzero finite scalars,
 * and the same two for op(B)'s columns.  Device buffers, caller-owned;
 * asynchronous on the handle's stream.  QCS_ERR_INVALID_ARG on bad
 * arguments. */
int qcs_rowcol_stats(qcs_handle_t h, qcs_op_t transA, qcs_op_t transB, int64_t m, int64_t n,
                     int64_t k, const qcs_c32 *A, int64_t lda, const qcs_c32 *B, int64_t ldb,
                     int32_t *d_emaxA, int32_t *d_emaxB, int64_t *d_counts);

/* Real products per emulated complex product of qcs_cgemm: 4 (default; the
 * complex expansion of Section 3, Re = ArBr - AiBi, Im = ArBi + AiBr) or 3
 * (Gauss's form, a variant beyond the paper: T1 = Ar Br, T2 = Ai Bi,
 * T3 = (Ar + Ai)(Br + Bi) as three emulated real GEMMs, Re = T1 - T2,
 * Im = T3 - T1 - T2; 9 tensor-core products instead of 12).  With 3 the
 * statistics and selection are still those of A and B; the operand sums of
 * T3 are formed in binary32 and, for the FP16 kind, split with one binade
 * less of scaling (2^(s-1)) so that they cannot overflow.  Applies to
 * qcs_cgemm calls whose mode (after the size rule) is emulated and k > 0;
 * the FP32 mode, the contraction tree and qcs_cgemm_noalloc keep 4.  The
 * error differs from the four-product form (the imaginary part is a
 * difference of products); the parity tests bound it against the exact
 * three-product model and FP64.  Environment override QCS_COMPLEX_PRODUCTS.
 * Returns QCS_ERR_INVALID_ARG for other values. */
int qcs_set_complex_products(qcs_handle_t h, int products);

/* The counts of Section 4.1 that AUTO's selection takes for one GEMM, as the
 * GEMM path computes them (pass 1: e_max, zeros, Inf/NaN, the count below
 * FP16's least normal 2^-14, i.e. N - N1; pass 2, only when pass 1 does not
 * decide: the count below the window [e_max - 28, e_max] that scaling by
 * 2^(14 - e_max) keeps, i.e. N - N2).  Real and imaginary parts count as
 * separate scalars; zeros are in neither count nor total. */
typedef struct {
    int32_t e_max;          /* largest exponent floor(log2|x|) of a finite nonzero scalar; -128 if none */
    int32_t stage2;         /* 1 if the pass-2 count was taken */
    int64_t n_nonzero;      /* finite nonzero scalars */
    int64_t n_nonfinite;    /* Inf / NaN scalars */
    int64_t n_under_fp16;   /* finite nonzero scalars with exponent < -14 (subnormals included) */
    int64_t n_under_window; /* finite nonzero scalars below 2^(e_max - 28); 0 unless stage2 */
} qcs_selection_stats_t;

/* Run the statistics and selection of an AUTO qcs_cgemm of op(A) (m x k) and
 * op(B) (k x n) -- the same kernels, the handle's tolerance, no size rule --
 * and return their counts for op(A) in out[0] and op(B) in out[1] (host)
 * and the descriptor the selection wrote in *desc_out (host, optional).
 * Arguments as qcs_cgemm (m, n, k >= 1).  Synchronizes the handle's stream. */
int qcs_selection_stats(qcs_handle_t h, qcs_op_t transA, qcs_op_t transB, int64_t m, int64_t n,
                        int64_t k, const qcs_c32 *A, int64_t lda, const qcs_c32 *B, int64_t ldb,
                        qcs_selection_stats_t *out, qcs_gemm_desc_t *desc_out);

/* Where the Eq. 1 split of a TF32X selection runs (Section 2.1).  0
 * (default): a separate pass writes the hi / lo TF32 planes of op(A) and
 * op(B) to the handle's workspace in HBM and the tensor-core kernel reads
 * them back.  1: the tensor-core kernel reads A and B as stored and its
 * epilogue warps split each staged tile in shared memory between their
 * accumulator drains, so the planes never leave the SM; the MMAs and their
 * order are the same, so the result is bit-identical.  Applies to qcs_cgemm
 * calls whose mode (after the size rule) is TF32X or AUTO, on matrices (not
 * gather views of the contraction tree), when the tensor-core GEMM runs as
 * one K range with the default drain of 4 stages and the TMA limits hold
 * (lda, ldb even; A, B 16-byte aligned); other calls keep the separate
 * pass.  Environment override QCS_FUSED_SPLIT. */
int qcs_set_fused_split(qcs_handle_t h, int enabled);

/* Failure detection (not a step of the paper).  Every wait inside the
 * tensor-core kernels (a TMA stage landing, the MMAs freeing a stage, the
 * epilogue draining an accumulator) gives up after ``ns`` nanoseconds of the
 * GPU's global timer; the kernel then records QCS_ERR_TIMEOUT in the
 * handle's device error word (read by qcs_sync), releases its tensor
 * memory, waits (bounded) for its copies in flight and returns, leaving C
 * partly written.  Default 2 s, far above any legitimate wait inside one
 * launch.  ``ns`` from 1000 to 10^10; QCS_ERR_INVALID_ARG otherwise. */
int qcs_set_wait_budget(qcs_handle_t h, uint64_t ns);

/* Test hook for failure detection.  While ``enabled`` != 0 the TMA producer
 * warp of every tensor-core kernel launched on this handle issues no loads,
 * so the MMA issuer's first wait for a stage never completes and runs out
 * after the wait budget (qcs_set_wait_budget): the launch takes that path
 * of a real stall (a lost copy) without any fault.  Results of such calls
 * are garbage; qcs_sync reports QCS_ERR_TIMEOUT.  Off by default. */
int qcs_debug_stall_producer(qcs_handle_t h, int enabled);

/* Exponent statistics (Section 4.1, Stage 1 and Stage 2 in one pass) of the
 * rows x cols complex matrix X (device, leading dim ldx >= rows), written
 * to d_stats (device, caller-owned).  rows or cols may be 0. */
int qcs_exp_stats(qcs_handle_t h, int64_t rows, int64_t cols, const qcs_c32 *X, int64_t ldx,
                  qcs_stats_t *d_stats);

/* Mode selection rule of Section 4.1 from the statistics of op(A) and
 * op(B) (both device), with the handle's tolerance.  Writes the descriptor
 * to d_desc (device).  Either operand out of both FP16 windows -> TF32X;
 * either out of the unscaled window -> FP16X_SCALED with sA, sB moving each
 * maximum exponent to 14; otherwise FP16X.  Inf/NaN or a maximum exponent
 * of 127 -> FP32. */
int qcs_select(qcs_handle_t h, const qcs_stats_t *d_statsA, const qcs_stats_t *d_statsB,
               qcs_gemm_desc_t *d_desc);

/* C = alpha * op(A) * op(B) + beta * C (Section 3: the complex product as
 * four real products, each emulated with Eq. 1 of Section 2.1).
 *   op(A) is m x k, op(B) is k x n, C is m x n; all device pointers.
 *   lda >= rows of A as stored (m for OP_N, k otherwise), likewise ldb, and
 *   ldc >= m.  alpha and beta are host pointers.  m, n, k >= 0.
 *   mode AUTO runs statistics + selection on the device (Section 4); a forced
 *   mode skips them.  d_desc_out (device, optional) receives the descriptor
 *   the GEMM ran with.  C must not overlap A or B.
 *   The tensor-core modes need A, B, C 8-byte aligned (always true for
 *   cudaMalloc'd complex64); otherwise UNSUPPORTED. */
int qcs_cgemm(qcs_handle_t h, qcs_mode_t mode, qcs_op_t transA, qcs_op_t transB, int64_t m,
              int64_t n, int64_t k, const qcs_c32 *alpha, const qcs_c32 *A, int64_t lda,
              const qcs_c32 *B, int64_t ldb, const qcs_c32 *beta, qcs_c32 *C, int64_t ldc,
              qcs_gemm_desc_t *d_desc_out);

/* C = alpha * op(A) * op(B) + beta * C for real FP32 matrices: the SGEMM
 * emulation of Section 2.1 (Eq. 1: one real product as hi*hi + (lo*hi +
 * hi*lo) / 2^11 on the tensor cores, the hi*hi sum added with
 * round-to-nearest) with the automatic selection of Section 4.
 *   op(A) is m x k, op(B) is k x n, C is m x n, column-major, all device
 *   pointers (4-byte aligned); lda >= rows of A as stored (m for OP_N, k
 *   otherwise), likewise ldb, and ldc >= m.  OP_C is OP_T.  alpha and beta
 *   are host pointers.  m, n, k >= 0 (each at most 2^31 - 1, else
 *   UNSUPPORTED).  C must not overlap A or B.
 *   mode AUTO runs statistics (every scalar of A and B as stored) and the
 *   selection rule on the device; the size rule of the handle applies with
 *   the paper's cut-offs (Section 4.3) -- QCS_SIZE_RULE_TUNED acts as
 *   QCS_SIZE_RULE_PAPER here, the tuned table holding complex shapes.  The
 *   K-range count set by qcs_set_tc_splits applies.  d_desc_out (device,
 *   optional) receives the descriptor the GEMM ran with; the selection
 *   counters of qcs_get_auto_counts add 2 m n k flops per AUTO call. */
int qcs_sgemm(qcs_handle_t h, qcs_mode_t mode, qcs_op_t transA, qcs_op_t transB, int64_t m,
              int64_t n, int64_t k, const float *alpha, const float *A, int64_t lda,
              const float *B, int64_t ldb, const float *beta, float *C, int64_t ldc,
              qcs_gemm_desc_t *d_desc_out);

/* The split stage of qcs_cgemm alone (Eq. 1 of Section 2.1 after the
 * scaling of Section 4.2), for inspection: op(X) (R x K for which == 0, i.e.
 * the A operand; K x R for which == 1, the B operand) is split under the
 * mode and scale held in d_desc (device) into four planes
 * hi.re, hi.im, lo.re, lo.im, each R x K row-major (K contiguous) with row
 * pitch ``pitch`` elements, stored as IEEE binary16 bit patterns (FP16X,
 * FP16X_SCALED), bfloat16 bit patterns (BF16X3) or binary32 (TF32X).  Planes
 * are consecutive, ``plane_stride`` elements apart.  Nothing is written for
 * mode FP32. */
int qcs_split(qcs_handle_t h, const qcs_gemm_desc_t *d_desc, int which, qcs_op_t op, int64_t R,
              int64_t K, const qcs_c32 *X, int64_t ldx, void *planes, int64_t pitch,
              int64_t plane_stride);

/* Tensor permutation with fixed (sliced) indices: the reshaping step of the
 * TTGT contraction (Section 1, Section 2.2).  out (device, contiguous,
 * first index fastest) has ``rank`` dims ``dims[0..rank)``; its element
 * (i_0, ..., i_{r-1}) is in[offset + sum_d i_d * strides[d]] (element
 * strides of the input, device).  dims/strides are host arrays, rank <= QCS_MAX_RANK.
 * When d_stats is not NULL, the exponent statistics of the output are also
 * written there (fused, Section 4.1). */
int qcs_permute(qcs_handle_t h, int rank, const int64_t *dims, const int64_t *strides,
                int64_t offset, const qcs_c32 *in, qcs_c32 *out, qcs_stats_t *d_stats);

/* ---- contraction tree (Section 2.2, Section 5.3) ---------------------- */

#define QCS_MAX_RANK 32

/* Where the elements of a column-major matrix live in a source tensor:
 * element (i, l) of an R x K matrix has column-major index t = i + l R;
 * decomposing t first-index-fastest over dims[0..rank) gives (x_0, ...),
 * and the element is at source offset sum_d x_d strides[d] (plus the
 * instance offset when the source is a leaf).  prod(dims) = R K. */
typedef struct {
    int32_t rank;
    int32_t pad_;
    int64_t dims[QCS_MAX_RANK];
    int64_t strides[QCS_MAX_RANK];
} qcs_gather_t;

/* One pairwise contraction, reshaped to a CGEMM (TTGT, Section 1):
 *   out (m x n, column-major, stored contiguous) = A_mat (m x k) B_mat (k x n)
 * where A_mat is read from tensor ``a`` through map_a and B_mat from tensor
 * ``b`` through map_b.  Tensors are numbered: leaves 0 .. n_leaves-1, then
 * step s produces tensor n_leaves + s (m n elements).  direct_a is a
 * qcs_op_t when tensor a, as stored, already is A_mat (QCS_OP_N, leading
 * dimension m) or its transpose (QCS_OP_T, leading dimension k) and its
 * instance offsets are all zero; otherwise -1 and A_mat is gathered
 * first.  Likewise direct_b (QCS_OP_N: ld k; QCS_OP_T: ld n). */
typedef struct {
    int32_t a, b;
    int32_t direct_a, direct_b;
    int64_t m, n, k;
    qcs_gather_t map_a;
    qcs_gather_t map_b;
    int32_t mode;  /* qcs_mode_t of this GEMM (AUTO: size rule + per-GEMM selection) */
    int32_t pad_;
} qcs_step_t;

/* A contraction plan run for n_instances instances.  An instance is one
 * assignment of the sliced indices (Section 5.3) and/or one bitstring: it
 * reads leaf i at element offset instance_offset[inst * n_leaves + i] of the
 * caller's leaf tensor, contracts all steps, and adds the root tensor (the
 * last step's output, or leaf 0 when n_steps == 0) -- gathered at out_index
 * -- into output slot instance_slot[inst], in FP64.  Slices of one bitstring
 * share a slot, so their sum is the amplitude. */
typedef struct {
    int32_t n_leaves;
    int32_t n_steps;
    int32_t n_instances;
    int32_t n_slots;
    const int64_t *leaf_size;        /* host, n_leaves: elements of each full leaf tensor */
    const int64_t *instance_offset;  /* host, n_instances * n_leaves */
    const int32_t *instance_slot;    /* host, n_instances, each in [0, n_slots) */
    const qcs_step_t *steps;         /* host, n_steps */
    int64_t out_size;                /* results per slot */
    const int64_t *out_index;        /* host, out_size indices into the root, or NULL:
                                        the root itself (then root size == out_size;
                                        n_steps == 0: the out_size elements of leaf 0
                                        from the instance's offset on) */
} qcs_tree_t;

typedef struct {
    double seconds;           /* host wall time of the call (launch side) */
    int64_t gemm_count;       /* CGEMMs issued (all instances) */
    int64_t gather_count;     /* gathers / scatters issued */
    int64_t mode_count[6];    /* GEMMs per effective mode after the size rule (AUTO counted in [0]) */
    int64_t workspace_bytes;  /* bytes of the tree workspace */
    double flops;             /* nominal 8 m n k summed over the GEMMs */
    double mode_flops[6];     /* the same per effective mode (as mode_count) */
    int64_t level_launches;   /* level launches issued (qcs_set_tree_levels) */
    int64_t level_gemms;      /* GEMMs they covered (all instances; part of gemm_count) */
} qcs_run_info_t;

/* Instances per group of qcs_contract_tree and qcs_tree_graph_create (1 to
 * 65535; default 1).  With G > 1 the forward pass runs the instances in
 * groups of G (Section 5.3: slices and bitstrings are independent instances
 * of one step sequence).  Each step up to the first emulated step that
 * fills the GPU alone (at least one 128 x 128 output tile per SM) AND whose
 * split planes and output for the G instances exceed the group budget
 * (qcs_set_group_budget) runs once per group: a step whose
 * GEMM runs in plain FP32 (after the size rule) as one batched gather and
 * one batched GEMM launch; an emulated step as per-instance statistics,
 * selection and split followed by one persistent tensor-core launch per
 * kind over the output tiles of all G instances (each instance keeps its
 * own selected mode; for AUTO the FP32 candidate of each instance is
 * launched gated).  Their outputs hold G instances each (intermediates share
 * memory by liveness).  The later steps loop over the group.  Results do
 * not depend on G.  The backward runs in groups of G as well when every
 * step can hold the group (else one instance at a time): the recomputed
 * forward, then per step the gathers, the two adjoint GEMMs and the
 * scatters of all G instances, each instance's leaf gradients in a buffer
 * of its own that is added into d_grad_leaves in instance order -- the same
 * sums in the same order as one instance at a time.  Its launches can be
 * captured in a graph (qcs_tree_backward_graph_create). */
int qcs_set_instance_batch(qcs_handle_t h, int instances);

/* The tree executor's plan for a call, computed on the host only (no device
 * is touched; for inspection and tests): with ``instance_batch`` instances
 * per group, level launches on or off, ``num_sms`` SMs, the given group
 * budget, the paper's size rule and no tuning table.  Per step (host arrays
 * of n_steps, each optional): the byte offset of its output in the tree
 * workspace (step_offset) and its size (step_bytes, all instances of a
 * group), the time it runs at (step_time: steps of equal time may run at
 * once, so their outputs must not overlap; an output is live from its
 * step's time to its last reader's), whether it runs inside a level
 * launch (step_small), and the order the steps are issued in (step_order,
 * a permutation; a level launch's steps consecutive).  *out gets the
 * workspace size, the group size used, the steps that run once per group
 * and the level launches per group.  QCS_ERR_INVALID_ARG as
 * qcs_contract_tree for a bad plan. */
typedef struct {
    int64_t total_bytes;
    int32_t group;
    int32_t batched_steps;
    int32_t level_launches;
    int32_t reserved;
} qcs_tree_layout_t;
int qcs_tree_layout_info(const qcs_tree_t *tree, int backward, int instance_batch, int levels,
                         int num_sms, uint64_t group_budget, int64_t *step_offset,
                         int64_t *step_bytes, int32_t *step_time, int32_t *step_small,
                         int32_t *step_order, qcs_tree_layout_t *out);

/* Memory a grouped step of the tree executor may hold (bytes; default
 * 32 GiB; environment override QCS_GROUP_BUDGET_MB): an emulated step that
 * fills the GPU alone still runs once for its group of G instances -- full
 * tile waves and one pipeline ramp for all of them -- unless its split planes
 * and output for the G instances exceed this; then it and every later step
 * run per instance (qcs_set_instance_batch).  0: every step that fills the
 * GPU alone runs per instance.  Results do not depend on it. */
int qcs_set_group_budget(qcs_handle_t h, uint64_t bytes);

/* Level launches of the tree executor (Section 2.2: the steps of one level
 * of the contraction tree are independent).  While ``enabled`` is 1 (the
 * default; environment override QCS_TREE_LEVELS) the executor runs the
 * steps of a group level by level (a step's level: one more than its
 * operands' highest), and the steps of a level whose GEMM runs in plain FP32
 * (after the size rule) with op(A) and op(B) of at most 1024 elements and C
 * of at most 4096 -- the gate-sized contractions that make up most of a
 * circuit's tree -- run as ONE launch for all of them and all instances of
 * the group, their gathers folded into the operand loads.  Each output
 * element is the same FP32 sum, term order l = 0 .. k-1 with one FMA per
 * real product, as the plain-FP32 per-element kernels form.  0: one step
 * after another in plan order.  QCS_ERR_INVALID_ARG for other values. */
int qcs_set_tree_levels(qcs_handle_t h, int enabled);

/* Contract the plan for every instance and accumulate into d_out (device,
 * complex128 as interleaved doubles, n_slots * out_size values, slot-major;
 * overwritten).  leaves: host array of n_leaves device pointers (complex64).
 * info: optional host out.  The plan is validated on the host (ids, ranks,
 * and every read offset within its tensor) before anything is launched.
 * Intermediates live in the handle's tree workspace. */
int qcs_contract_tree(qcs_handle_t h, const qcs_tree_t *tree, const qcs_c32 *const *leaves,
                      double *d_out, qcs_run_info_t *info);

/* The launches of one qcs_contract_tree call, captured into a CUDA graph
 * (Section 5.3's slices are independent instances of one step sequence, so
 * the whole sequence replays with one launch).  qcs_tree_graph_create
 * validates the plan, allocates the graph's own workspace (cudaMalloc; not
 * during a capture), records every kernel the call would launch for these
 * leaves and this d_out into a graph and instantiates it; nothing is
 * computed.  qcs_tree_graph_launch replays it on the handle's current
 * stream: the same result qcs_contract_tree would write to d_out, from the
 * current contents of the same leaf buffers.  The leaf and output buffers
 * and the handle must outlive the graph.  qcs_tree_graph_destroy
 * synchronizes the handle's stream and frees the graph and its workspace. */
typedef struct qcs_tree_graph_s *qcs_tree_graph_t;
int qcs_tree_graph_create(qcs_handle_t h, const qcs_tree_t *tree, const qcs_c32 *const *leaves,
                          double *d_out, qcs_tree_graph_t *out);
int qcs_tree_graph_launch(qcs_tree_graph_t g);
int qcs_tree_graph_destroy(qcs_tree_graph_t g);

/* The launches of one qcs_contract_tree_backward call captured into a CUDA
 * graph, the same way: qcs_tree_backward_graph_create validates the plan,
 * allocates the graph's own workspace (cudaMalloc; not during a capture) and
 * records every kernel the call would launch for these leaves, this
 * d_grad_out and these d_grad_leaves; nothing is computed.  Each
 * qcs_tree_graph_launch of it then adds the leaf gradients to
 * d_grad_leaves, from the current contents of the leaf and d_grad_out
 * buffers, exactly as qcs_contract_tree_backward would (the caller clears
 * d_grad_leaves between replays if it wants the gradient alone).  The
 * buffers and the handle must outlive the graph; qcs_tree_graph_destroy
 * frees it.  Replaying removes the host cost of the backward's launches
 * (two gathers, two GEMMs and two scatters per step and instance), which
 * dominates on trees of many small contractions. */
int qcs_tree_backward_graph_create(qcs_handle_t h, const qcs_tree_t *tree,
                                   const qcs_c32 *const *leaves, const double *d_grad_out,
                                   qcs_c32 *const *d_grad_leaves, qcs_tree_graph_t *out);

/* Adjoint of qcs_contract_tree.  Given d_grad_out (device complex128,
 * n_slots * out_size values: dL/dRe + i dL/dIm of each output), adds to
 * d_grad_leaves[i] (host array of device complex64 pointers, each the size
 * of the caller's full leaf tensor; not cleared) the gradient of L with
 * respect to every leaf element in the same convention.  Each forward GEMM
 * out = A_mat B_mat has two adjoint GEMMs, grad_A = grad_out B_mat^H and
 * grad_B = A_mat^H grad_out, run as emulated CGEMMs in the step's mode
 * (op C flags); the forward intermediates are recomputed per instance
 * (slice) rather than kept across instances.  Every tensor of the plan must
 * be used by exactly one step (a tree), and the gradients of different leaves
 * must not overlap in memory (QCS_ERR_INVALID_ARG otherwise): with level
 * launches (qcs_set_tree_levels) the adjoints of a level's small steps run
 * at once and add into them concurrently. */
int qcs_contract_tree_backward(qcs_handle_t h, const qcs_tree_t *tree,
                               const qcs_c32 *const *leaves, const double *d_grad_out,
                               qcs_c32 *const *d_grad_leaves, qcs_run_info_t *info);

/* FP64 reductions of a result against a reference (Section 5.3 measures
 * amplitudes by their fidelity and error against an exact reference; these
 * are the only FP64 arithmetic on the GPU besides the slice sums).  a
 * (device, n complex: complex128 as interleaved doubles, or complex64 when
 * a_c64 is 1) and ref (device, n complex128, or NULL: then only the norm of
 * a) give, in d_out (device, 6 doubles):
 *   [0] sum |a_j|^2        [1] sum |ref_j|^2
 *   [2] Re sum conj(ref_j) a_j   [3] Im of the same
 *   [4] sum |a_j - ref_j|^2     [5] max_j |a_j - ref_j|
 * so that the fidelity is (d[2]^2 + d[3]^2) / (d[0] d[1]) and the relative
 * L2 error sqrt(d[4] / d[1]); entries that need ref are 0 without it.  Every
 * sum is formed in FP64 in a fixed order (per-block partials, then one block
 * in a fixed tree), so the result does not depend on scheduling.
 * Asynchronous on the handle's stream; n >= 0; QCS_ERR_INVALID_ARG for NULL
 * a or d_out, or misaligned pointers (8-byte for complex64, 16 for
 * complex128). */
int qcs_fidelity_stats(qcs_handle_t h, const void *a, int a_c64, const double *ref, int64_t n,
                       double *d_out);

/* qcs_cgemm without a handle and without allocating device memory.  (The
 * paper has no counterpart: this serves callers that must not allocate at
 * call time -- their device memory is owned by another allocator with a
 * fixed budget, such as a framework's caching allocator or a pre-sized
 * arena, or they run latency-critical loops that cannot afford cudaMalloc /
 * cudaFree, which may synchronise the whole device.)
 *
 * Same operation, arguments and semantics as qcs_cgemm, on the stream
 * ``cuda_stream`` (a cudaStream_t; NULL = legacy default stream) of the
 * current device, with underflow tolerance ``underflow_tol`` (as
 * qcs_set_underflow_tol) and the size rule that qcs_set_size_rule controls
 * switched off, so that AUTO always selects from the statistics.  The
 * caller still passes A, B, C (and the optional d_desc_out); the workspace
 * lives in a fixed device array of QCS_NOALLOC_SCRATCH_BYTES (64 MiB) that
 * every GPU which loads this part of the library keeps until the process
 * exits.  The workspace of a call is 256 bytes, the statistics partials,
 * the split planes -- for op(A) 16 bytes per element of
 * ceil(m/128)*128 x ceil(k/32)*32 and for op(B) 20 bytes per element of
 * ceil(n/128)*128 x ceil(k/32)*32 in AUTO and TF32X, half that in the
 * 16-bit modes, none in FP32 -- and, when the library splits the
 * tensor-core GEMM along K (chosen from the shape, up to 16 ranges), 8 bytes
 * per range per element of m x n for the partial products.  A problem whose
 * workspace does not fit is rejected with QCS_ERR_SCRATCH_TOO_SMALL before
 * anything is launched; that return code, not this estimate, is
 * authoritative (m = n = k = 1024 fits in every mode).
 *
 * Set-up: the first call on a device, with that device current, resolves
 * the array's device address (cudaGetSymbolAddress).  Under CUDA's lazy
 * module loading that is also the moment the driver commits the 64 MiB on
 * the device, outside any caller's allocator, and it can fail there with
 * QCS_ERR_CUDA when the device is full: make that first call at start-up,
 * and before any stream capture on the device.  Later calls allocate and
 * free nothing.  All calls on a device share the one array and it keeps the
 * last call's contents (what must start at zero is cleared): calls that
 * overlap on the GPU, e.g. on two concurrent streams, race and corrupt each
 * other's results; serialise them.  A device-side wait that times out
 * (see qcs_set_wait_budget; default 2 s) leaves C partly written and sets
 * an error word in the array that stays set until qcs_cgemm_noalloc_status
 * clears it. */
#define QCS_NOALLOC_SCRATCH_BYTES (64u << 20)
int qcs_cgemm_noalloc(void *cuda_stream, qcs_mode_t mode, double underflow_tol, qcs_op_t transA,
                      qcs_op_t transB, int64_t m, int64_t n, int64_t k, const qcs_c32 *alpha,
                      const qcs_c32 *A, int64_t lda, const qcs_c32 *B, int64_t ldb,
                      const qcs_c32 *beta, qcs_c32 *C, int64_t ldc, qcs_gemm_desc_t *d_desc_out);

/* The device-side status of qcs_cgemm_noalloc on the current device (the
 * paper has no counterpart; a no-allocation caller has no handle to pass to
 * qcs_sync).  Waits for ``cuda_stream``, then returns QCS_ERR_TIMEOUT if a
 * wait inside a tensor-core kernel of any qcs_cgemm_noalloc call on this
 * device gave up since the word was last cleared, QCS_SUCCESS if none did
 * (or no call has run on the device yet), QCS_ERR_CUDA on a runtime error.
 * ``reset`` != 0 clears the word after reading it.  Allocates nothing. */
int qcs_cgemm_noalloc_status(void *cuda_stream, int reset);

/* ---- autotuning: the size rule re-derived on this GPU ------------------ */

/* One tuned shape.  The key is (m, n, k, opA, opB) as qcs_cgemm receives
 * them.  ms[mode] is the measured time of one call in that forced mode
 * (QCS_MODE_AUTO: statistics + selection + the selected path), negative
 * when the candidate was not run (pruned: an FP32 call that cannot win).
 * best is what QCS_SIZE_RULE_TUNED then runs for an AUTO GEMM of this shape:
 * QCS_MODE_AUTO (statistics decide), QCS_MODE_TF32X (no statistics: TF32
 * has FP32's exponent range) or QCS_MODE_FP32.  splits is the tensor-core
 * schedule measured for the shape: the number of K ranges (see
 * qcs_set_tc_splits) that ran the faster emulated candidate fastest; under
 * QCS_SIZE_RULE_TUNED the tensor-core GEMMs of this shape use it unless
 * qcs_set_tc_splits forces a count.  0: not measured (the per-shape rule
 * applies); ms[] of the emulated candidate is its time at that count.
 * group_m is the tensor-core raster measured for the shape (tile rows per
 * raster group, see qcs_set_tc_schedule) for shapes with at least twice as
 * many 128 x 128 output tiles as SMs; under QCS_SIZE_RULE_TUNED the
 * tensor-core GEMMs of this shape use it.  0: not measured (the handle's
 * schedule applies).  The raster only orders the tiles: results do not
 * depend on it. */
typedef struct {
    int64_t m, n, k;
    int32_t opA, opB;
    float ms[QCS_NUM_MODES];
    int32_t best;
    int32_t reps;
    int32_t splits;
    int32_t group_m;
} qcs_tune_entry_t;

/* Time the candidates for one shape on the handle's stream and record the
 * fastest in the handle's table (replacing an earlier entry for the key).
 * Operands are synthetic, allocated by this call (cudaMalloc of op(A),
 * op(B) and C) and freed before it returns: parts of magnitude in [1, 2)
 * with random signs, so that the statistics select FP16X.  Each candidate
 * runs once untimed, then ``reps`` (>= 1) times between CUDA events;
 * FP32 is not run when 8 m n k / 45 TFLOP/s is above 4x the faster
 * emulated candidate.  Ties go to the earlier of AUTO, TF32X, FP32.  For a
 * shape with fewer 128 x 128 output tiles than twice the SM count, the
 * faster emulated candidate is also timed at 1, 2, 4, 8 and 16 K ranges
 * (at most one per 32 k; not when qcs_set_tc_splits forces a count) and the
 * fastest count is recorded in ``splits``; for a shape with more tiles, it
 * is timed with raster groups of 2, 4, 8 and 16 tile rows and the fastest is
 * recorded in ``group_m``.
 * Synchronizes the stream; not during a stream capture.  out (host,
 * optional) receives the entry.  m, n, k >= 1. */
int qcs_autotune_gemm(qcs_handle_t h, qcs_op_t transA, qcs_op_t transB, int64_t m, int64_t n,
                      int64_t k, int reps, qcs_tune_entry_t *out);

/* qcs_autotune_gemm for every distinct AUTO GEMM shape that
 * qcs_contract_tree (and, with backward != 0, qcs_contract_tree_backward)
 * issues for the plan, skipping shapes already in the table.  n_tuned
 * (host, optional) receives the number of shapes timed.  The plan is
 * validated as qcs_contract_tree validates it. */
int qcs_autotune_tree(qcs_handle_t h, const qcs_tree_t *tree, int backward, int reps,
                      int64_t *n_tuned);

/* Read the handle's table: up to ``capacity`` entries (in key order) into
 * ``entries`` (host); *count receives the table's size. */
int qcs_get_tuning(qcs_handle_t h, qcs_tune_entry_t *entries, int64_t capacity, int64_t *count);

/* Add entries (host) to the handle's table, e.g. decisions saved from an
 * earlier process on the same GPU; each replaces the entry of its key.
 * best must be AUTO, TF32X or FP32. */
int qcs_set_tuning(qcs_handle_t h, const qcs_tune_entry_t *entries, int64_t count);

/* Measurement aid (not a step of the paper): the FP32 FMA rate of the CUDA
 * cores, the roofline of the plain FP32 CGEMM (QCS_MODE_FP32 and the
 * baseline of Section 5).  Runs a kernel of independent FMA chains on every
 * SM (64 warps each, about 50 ms) on the handle's stream and writes
 * 2 x FMAs / second / 1e12 to *tflops (host).  Synchronizes the stream; not
 * during a stream capture.  The rate depends on the clock the GPU runs at
 * under this load. */
int qcs_measure_fma_peak(qcs_handle_t h, double *tflops);

/* Stage timing (tracing aid, off by default).  While enabled, every call
 * records a pair of CUDA events on the handle's stream around each stage
 * it launches.  qcs_get_profile() synchronizes the stream, writes the
 * milliseconds accumulated per stage since the previous read into ms[0..n)
 * -- [0] exponent statistics, [1] selection, [2] split, [3] tensor-core
 * GEMM, [4] FP32 SIMT GEMM, [5] permute/gather, [6] FP64 reductions -- and
 * the number of event pairs per stage into counts (optional), then clears
 * them.  Enabling it adds no synchronisation to the calls themselves. */
#define QCS_PROFILE_STAGES 7
int qcs_set_profiling(qcs_handle_t h, int enabled);
int qcs_get_profile(qcs_handle_t h, double *ms, int64_t *counts, int n);

/* What the automatic selection (Section 4.1) chose: counts[i] (host array of
 * QCS_NUM_MODES) receives how many GEMMs of mode AUTO on this handle -- after
 * the size rule, so only those that ran the statistics -- selected
 * qcs_mode_t i on the device since the handle was created or last reset,
 * and flops[i] (host, optional) their nominal 8 m n k summed.  (The
 * selection happens on the device, so the host-side counts of
 * qcs_run_info_t only know that such a GEMM was AUTO.)  Synchronizes the
 * handle's stream.  reset != 0 clears the counters afterwards.  Graph
 * replays count too. */
int qcs_get_auto_counts(qcs_handle_t h, int64_t *counts, double *flops, int reset);

/* Wait for the handle's stream; return TIMEOUT if a device-side bounded
 * wait gave up since the last qcs_sync (the word is then cleared), CUDA on
 * a runtime error, else SUCCESS. */
int qcs_sync(qcs_handle_t h);

/* Static string for a status code. */
const char *qcs_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* QCS_H */
