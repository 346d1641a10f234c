// Drop-in interception of cuBLAS single-precision GEMMs (libqcs_cublas.so).
//
// The paper's library is used by linking it in front of cuBLAS: calls to the
// cuBLAS GEMM routines of an unmodified application are redirected to the
// emulated GEMM, and an environment variable picks the mode (Section 3).
// This library does the same for the single-precision GEMMs: loaded before
// cuBLAS (LD_PRELOAD, or linked ahead of it), it defines
//   cublasCgemm_v2, cublasCgemmStridedBatched, cublasCgemmBatched,
//   cublasSgemm_v2, cublasSgemmStridedBatched
// and runs them through qcs_cgemm / qcs_sgemm on the cuBLAS handle's
// stream.  Calls it cannot take -- alpha/beta in device memory
// (CUBLAS_POINTER_MODE_DEVICE), an argument qcs_cgemm / qcs_sgemm rejects,
// the batched form with device pointer arrays, or QCS_CUBLAS_MODE=cublas --
// go to the next definition in the link order, the real cuBLAS.
//
// Environment:
//   QCS_CUBLAS_MODE    auto (default) | fp16x | fp16x_scaled | tf32x | fp32 |
//                      bf16x3 | cublas (pass every call through)
//   QCS_UNDERFLOW_TOL  AUTO-t of the qcs handles (read by qcs_create)
//   QCS_SIZE_RULE      0 off, 1 the paper's cut-offs (default), 2 tuned
//   QCS_COMPLEX_PRODUCTS  3: complex GEMMs as Gauss's three real products
//
// One qcs handle per CUDA stream, created on first use and kept until exit.
// The calls of one handle are serialised by a lock, as cuBLAS requires of
// one cuBLAS handle anyway.
#include <cublas_v2.h>
#include <dlfcn.h>

#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "../../include/qcs.h"

namespace {

typedef cublasStatus_t (*GetStreamFn)(cublasHandle_t, cudaStream_t *);
typedef cublasStatus_t (*GetPointerModeFn)(cublasHandle_t, cublasPointerMode_t *);
typedef cublasStatus_t (*CgemmFn)(cublasHandle_t, cublasOperation_t, cublasOperation_t, int, int,
                                  int, const cuComplex *, const cuComplex *, int,
                                  const cuComplex *, int, const cuComplex *, cuComplex *, int);
typedef cublasStatus_t (*CgemmStridedFn)(cublasHandle_t, cublasOperation_t, cublasOperation_t,
                                         int, int, int, const cuComplex *, const cuComplex *, int,
                                         long long, const cuComplex *, int, long long,
                                         const cuComplex *, cuComplex *, int, long long, int);
typedef cublasStatus_t (*SgemmFn)(cublasHandle_t, cublasOperation_t, cublasOperation_t, int, int,
                                  int, const float *, const float *, int, const float *, int,
                                  const float *, float *, int);
typedef cublasStatus_t (*SgemmStridedFn)(cublasHandle_t, cublasOperation_t, cublasOperation_t,
                                         int, int, int, const float *, const float *, int,
                                         long long, const float *, int, long long, const float *,
                                         float *, int, long long, int);
typedef cublasStatus_t (*CgemmBatchedFn)(cublasHandle_t, cublasOperation_t, cublasOperation_t, int,
                                         int, int, const cuComplex *, const cuComplex *const[],
                                         int, const cuComplex *const[], int, const cuComplex *,
                                         cuComplex *const[], int, int);

std::atomic<long long> g_taken{0}, g_passed{0};
std::mutex g_lock;
std::map<cudaStream_t, qcs_handle_t> g_handles;

// cuBLAS's own definition of ``name``.  RTLD_NEXT finds it when cuBLAS is
// in the global scope; an application that loads cuBLAS as the dependency of
// a library opened with RTLD_LOCAL (Python extensions) keeps it out of that
// scope, so the already-loaded cuBLAS is then looked up by its soname.
template <typename F>
F next_symbol(const char *name) {
    if (void *p = dlsym(RTLD_NEXT, name)) return reinterpret_cast<F>(p);
    static void *lib = [] {
        for (const char *so : {"libcublas.so.13", "libcublas.so.12", "libcublas.so"})
            if (void *h = dlopen(so, RTLD_NOW | RTLD_LOCAL | RTLD_NOLOAD)) return h;
        for (const char *so : {"libcublas.so.13", "libcublas.so.12", "libcublas.so"})
            if (void *h = dlopen(so, RTLD_NOW | RTLD_LOCAL)) return h;
        return static_cast<void *>(nullptr);
    }();
    return lib ? reinterpret_cast<F>(dlsym(lib, name)) : nullptr;
}

// -1: pass every call to cuBLAS; otherwise the qcs mode.
int shim_mode() {
    static const int mode = [] {
        const char *v = std::getenv("QCS_CUBLAS_MODE");
        if (!v || !*v || !std::strcmp(v, "auto")) return (int)QCS_MODE_AUTO;
        if (!std::strcmp(v, "fp16x")) return (int)QCS_MODE_FP16X;
        if (!std::strcmp(v, "fp16x_scaled")) return (int)QCS_MODE_FP16X_SCALED;
        if (!std::strcmp(v, "tf32x")) return (int)QCS_MODE_TF32X;
        if (!std::strcmp(v, "fp32")) return (int)QCS_MODE_FP32;
        if (!std::strcmp(v, "bf16x3")) return (int)QCS_MODE_BF16X3;
        return -1;  // "cublas" or anything else: do not intercept
    }();
    return mode;
}

qcs_op_t to_op(cublasOperation_t t) {
    return t == CUBLAS_OP_N ? QCS_OP_N : (t == CUBLAS_OP_T ? QCS_OP_T : QCS_OP_C);
}

// The stream of a cuBLAS handle when the call can run through qcs (host
// alpha/beta); false otherwise.
bool takeable(cublasHandle_t handle, cudaStream_t *stream) {
    if (shim_mode() < 0) return false;
    static GetStreamFn get_stream = next_symbol<GetStreamFn>("cublasGetStream_v2");
    static GetPointerModeFn get_pm = next_symbol<GetPointerModeFn>("cublasGetPointerMode_v2");
    if (!get_stream || !get_pm) return false;
    cublasPointerMode_t pm;
    if (get_pm(handle, &pm) != CUBLAS_STATUS_SUCCESS || pm != CUBLAS_POINTER_MODE_HOST) return false;
    return get_stream(handle, stream) == CUBLAS_STATUS_SUCCESS;
}

// The qcs handle of ``stream`` (created on first use); call with g_lock held.
int handle_of(cudaStream_t stream, qcs_handle_t *out) {
    qcs_handle_t &h = g_handles[stream];
    if (!h) {
        if (int r = qcs_create(&h, stream)) {
            h = nullptr;
            return r;
        }
    }
    *out = h;
    return QCS_SUCCESS;
}

// qcs_sgemm on ``stream`` under the lock of its handle; QCS status.
int run_real(cudaStream_t stream, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k,
             const float *alpha, const float *A, int lda, const float *B, int ldb,
             const float *beta, float *C, int ldc) {
    std::lock_guard<std::mutex> guard(g_lock);
    qcs_handle_t h;
    if (int r = handle_of(stream, &h)) return r;
    return qcs_sgemm(h, (qcs_mode_t)shim_mode(), to_op(ta), to_op(tb), m, n, k, alpha, A, lda, B,
                     ldb, beta, C, ldc, nullptr);
}

// qcs_cgemm on ``stream`` under the lock of its handle; QCS status.
int run(cudaStream_t stream, cublasOperation_t ta, cublasOperation_t tb, int m, int n, int k,
        const cuComplex *alpha, const cuComplex *A, int lda, const cuComplex *B, int ldb,
        const cuComplex *beta, cuComplex *C, int ldc) {
    std::lock_guard<std::mutex> guard(g_lock);
    qcs_handle_t h;
    if (int r = handle_of(stream, &h)) return r;
    static_assert(sizeof(cuComplex) == sizeof(qcs_c32), "complex layouts differ");
    return qcs_cgemm(h, (qcs_mode_t)shim_mode(), to_op(ta), to_op(tb), m, n, k,
                     reinterpret_cast<const qcs_c32 *>(alpha), reinterpret_cast<const qcs_c32 *>(A),
                     lda, reinterpret_cast<const qcs_c32 *>(B), ldb,
                     reinterpret_cast<const qcs_c32 *>(beta), reinterpret_cast<qcs_c32 *>(C), ldc,
                     nullptr);
}

}  // namespace

extern "C" {

cublasStatus_t cublasCgemm_v2(cublasHandle_t handle, cublasOperation_t transa,
                              cublasOperation_t transb, int m, int n, int k,
                              const cuComplex *alpha, const cuComplex *A, int lda,
                              const cuComplex *B, int ldb, const cuComplex *beta, cuComplex *C,
                              int ldc) {
    cudaStream_t stream;
    if (takeable(handle, &stream) &&
        run(stream, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc) == QCS_SUCCESS) {
        g_taken++;
        return CUBLAS_STATUS_SUCCESS;
    }
    static CgemmFn real = next_symbol<CgemmFn>("cublasCgemm_v2");
    if (!real) return CUBLAS_STATUS_NOT_SUPPORTED;
    g_passed++;
    return real(handle, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

cublasStatus_t cublasCgemmStridedBatched(cublasHandle_t handle, cublasOperation_t transa,
                                         cublasOperation_t transb, int m, int n, int k,
                                         const cuComplex *alpha, const cuComplex *A, int lda,
                                         long long strideA, const cuComplex *B, int ldb,
                                         long long strideB, const cuComplex *beta, cuComplex *C,
                                         int ldc, long long strideC, int batchCount) {
    cudaStream_t stream;
    if (batchCount >= 0 && takeable(handle, &stream)) {
        int r = QCS_SUCCESS, b = 0;
        for (; b < batchCount && r == QCS_SUCCESS; ++b)
            r = run(stream, transa, transb, m, n, k, alpha, A + b * strideA, lda, B + b * strideB,
                    ldb, beta, C + b * strideC, ldc);
        if (r == QCS_SUCCESS) {
            g_taken++;
            return CUBLAS_STATUS_SUCCESS;
        }
        // Arguments are checked before anything is launched, and every entry
        // has the same sizes: a rejection of the first entry hands the whole
        // call to cuBLAS.  A failure after entries ran cannot be handed over
        // (with beta != 0 they would be applied twice).
        if (b > 1 || (r != QCS_ERR_UNSUPPORTED && r != QCS_ERR_INVALID_ARG))
            return CUBLAS_STATUS_EXECUTION_FAILED;
    }
    static CgemmStridedFn real = next_symbol<CgemmStridedFn>("cublasCgemmStridedBatched");
    if (!real) return CUBLAS_STATUS_NOT_SUPPORTED;
    g_passed++;
    return real(handle, transa, transb, m, n, k, alpha, A, lda, strideA, B, ldb, strideB, beta, C,
                ldc, strideC, batchCount);
}

cublasStatus_t cublasCgemmBatched(cublasHandle_t handle, cublasOperation_t transa,
                                  cublasOperation_t transb, int m, int n, int k,
                                  const cuComplex *alpha, const cuComplex *const Aarray[], int lda,
                                  const cuComplex *const Barray[], int ldb, const cuComplex *beta,
                                  cuComplex *const Carray[], int ldc, int batchCount) {
    // The pointer arrays live in device memory (cuBLAS's contract): reading
    // them would synchronise the stream, so these calls go to cuBLAS.
    static CgemmBatchedFn real = next_symbol<CgemmBatchedFn>("cublasCgemmBatched");
    if (!real) return CUBLAS_STATUS_NOT_SUPPORTED;
    g_passed++;
    return real(handle, transa, transb, m, n, k, alpha, Aarray, lda, Barray, ldb, beta, Carray, ldc,
                batchCount);
}

cublasStatus_t cublasSgemm_v2(cublasHandle_t handle, cublasOperation_t transa,
                              cublasOperation_t transb, int m, int n, int k, const float *alpha,
                              const float *A, int lda, const float *B, int ldb, const float *beta,
                              float *C, int ldc) {
    cudaStream_t stream;
    if (takeable(handle, &stream) &&
        run_real(stream, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc) ==
            QCS_SUCCESS) {
        g_taken++;
        return CUBLAS_STATUS_SUCCESS;
    }
    static SgemmFn real = next_symbol<SgemmFn>("cublasSgemm_v2");
    if (!real) return CUBLAS_STATUS_NOT_SUPPORTED;
    g_passed++;
    return real(handle, transa, transb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

cublasStatus_t cublasSgemmStridedBatched(cublasHandle_t handle, cublasOperation_t transa,
                                         cublasOperation_t transb, int m, int n, int k,
                                         const float *alpha, const float *A, int lda,
                                         long long strideA, const float *B, int ldb,
                                         long long strideB, const float *beta, float *C, int ldc,
                                         long long strideC, int batchCount) {
    cudaStream_t stream;
    if (batchCount >= 0 && takeable(handle, &stream)) {
        int r = QCS_SUCCESS, b = 0;
        for (; b < batchCount && r == QCS_SUCCESS; ++b)
            r = run_real(stream, transa, transb, m, n, k, alpha, A + b * strideA, lda,
                         B + b * strideB, ldb, beta, C + b * strideC, ldc);
        if (r == QCS_SUCCESS) {
            g_taken++;
            return CUBLAS_STATUS_SUCCESS;
        }
        // as for cublasCgemmStridedBatched: only a rejection of the first
        // entry can be handed to cuBLAS
        if (b > 1 || (r != QCS_ERR_UNSUPPORTED && r != QCS_ERR_INVALID_ARG))
            return CUBLAS_STATUS_EXECUTION_FAILED;
    }
    static SgemmStridedFn real = next_symbol<SgemmStridedFn>("cublasSgemmStridedBatched");
    if (!real) return CUBLAS_STATUS_NOT_SUPPORTED;
    g_passed++;
    return real(handle, transa, transb, m, n, k, alpha, A, lda, strideA, B, ldb, strideB, beta, C,
                ldc, strideC, batchCount);
}

// Calls this library ran through qcs_cgemm / qcs_sgemm (*taken) and passed to cuBLAS
// (*passed) since it was loaded.
void qcs_cublas_shim_counts(long long *taken, long long *passed) {
    if (taken) *taken = g_taken.load();
    if (passed) *passed = g_passed.load();
}

}  // extern "C"
