// qcs_cgemm_noalloc: the emulated CGEMM for callers that must not allocate
// device memory when they call it.
//
// Such callers own all device memory through another allocator with a fixed
// budget (a framework's caching allocator, a pre-sized arena), or run
// latency-critical loops that cannot afford cudaMalloc / cudaFree, which may
// synchronise the whole device.  qcs_cgemm needs a handle, and the handle
// allocates its workspace with cudaMalloc on first need; this entry point
// needs no handle and allocates nothing: the workspace (mode descriptor,
// statistics partials, split planes) and the device error word live in the
// fixed array below, and the launch sequence is the one qcs_cgemm runs.
#include <cuda_runtime.h>

#include <mutex>

#include "internal.h"

namespace qcs {

// Fixed scratch, QCS_NOALLOC_SCRATCH_BYTES.  Every GPU that loads this part of
// the library keeps it until the process exits.  Host code must not use the
// symbol as an address: it is a host-side stand-in.  The device address comes
// from cudaGetSymbolAddress (see noalloc_setup).
constexpr size_t kNoallocBytes = QCS_NOALLOC_SCRATCH_BYTES;
constexpr size_t kNoallocHeader = 256;  // device error word, then unused bytes
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {

constexpr int kMaxDevices = 64;

struct DeviceSetup {
    bool ready = false;
    unsigned char *scratch = nullptr;  // device address of g_noalloc_scratch
    int num_sms = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];
EncodeTiledFn g_encode = nullptr;

// Once per device, with that device current: resolve the scratch array's
// device address and the SM count, and clear the error word on ``s`` (the
// first caller's stream, ahead of its launches).  Returns QCS_SUCCESS or an
// error code.
int noalloc_setup(int dev, cudaStream_t s, DeviceSetup *&out) {
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &d = g_setup[dev];
    if (!d.ready) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return QCS_ERR_CUDA;
        }
        if (cudaMemsetAsync(ptr, 0, kNoallocHeader, s) != cudaSuccess) {
            cudaGetLastError();
            return QCS_ERR_CUDA;
        }
        if (cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return QCS_ERR_CUDA;
        }
        if (!g_encode) {
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                 cudaEnableDefault, &q) != cudaSuccess ||
                q != cudaDriverEntryPointSuccess || !fn) {
                cudaGetLastError();
                return QCS_ERR_CUDA;
            }
            g_encode = reinterpret_cast<EncodeTiledFn>(fn);
        }
        d.scratch = static_cast<unsigned char *>(ptr);
        d.ready = true;
    }
    out = &d;
    return QCS_SUCCESS;
}

}  // namespace
}  // namespace qcs

using namespace qcs;

extern "C" int qcs_cgemm_noalloc(void *cuda_stream, qcs_mode_t mode, double underflow_tol,
                                 qcs_op_t transA, qcs_op_t transB, int64_t m, int64_t n, int64_t k,
                                 const qcs_c32 *alpha, const qcs_c32 *A, int64_t lda,
                                 const qcs_c32 *B, int64_t ldb, const qcs_c32 *beta, qcs_c32 *C,
                                 int64_t ldc, qcs_gemm_desc_t *d_desc_out) {
    if (!(underflow_tol >= 0.0 && underflow_tol <= 1.0)) return QCS_ERR_INVALID_ARG;
    if (int r = validate_cgemm(mode, transA, transB, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc))
        return r;
    if (m == 0 || n == 0) return QCS_SUCCESS;
    if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) return QCS_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return QCS_ERR_UNSUPPORTED;
    DeviceSetup *d = nullptr;
    if (int r = noalloc_setup(dev, static_cast<cudaStream_t>(cuda_stream), d)) return r;

    // A stack handle: no workspace of its own, the caller's stream and
    // tolerance, and the size rule off, so that AUTO selects from the
    // statistics as qcs_cgemm does with the size rule off; the error word is
    // the scratch's (sticky until qcs_cgemm_noalloc_status clears it).
    qcs_handle_s h;
    h.device = dev;
    h.num_sms = d->num_sms;
    h.stream = static_cast<cudaStream_t>(cuda_stream);
    h.tol = underflow_tol;
    h.size_rule = 0;
    h.d_err = reinterpret_cast<int *>(d->scratch);
    h.encode = g_encode;
    const int eff = mode;
    if (kNoallocHeader + gemm_workspace_bytes(eff, m, n, k, d->num_sms, 0) > kNoallocBytes)
        return QCS_ERR_SCRATCH_TOO_SMALL;
    // The error word was cleared at set-up and is only ever raised by a
    // timed-out wait; everything else in the scratch is overwritten by the
    // launches below before it is read.
    const float2 al = make_float2(alpha->x, alpha->y), be = make_float2(beta->x, beta->y);
    return run_cgemm(&h, d->scratch + kNoallocHeader, eff, transA, transB, m, n, k, al,
                     reinterpret_cast<const float2 *>(A), lda, reinterpret_cast<const float2 *>(B),
                     ldb, be, reinterpret_cast<float2 *>(C), ldc, d_desc_out, nullptr);
}

extern "C" int qcs_cgemm_noalloc_status(void *cuda_stream, int reset) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return QCS_ERR_UNSUPPORTED;
    unsigned char *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (g_setup[dev].ready) scratch = g_setup[dev].scratch;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    if (!scratch) return QCS_SUCCESS;  // no call has run on this device
    int word = 0;
    if (cudaMemcpy(&word, scratch, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    if (word != 0 && reset) {
        if (cudaMemsetAsync(scratch, 0, sizeof(int), s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return QCS_ERR_CUDA;
        }
    }
    return word != 0 ? QCS_ERR_TIMEOUT : QCS_SUCCESS;
}
