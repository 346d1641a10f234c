// Autotuning of the AUTO size rule (qcs_autotune_gemm, qcs_get_tuning,
// qcs_set_tuning; qcs_autotune_tree lives with the executor).
//
// Section 4.3 decides from min(m, n, k) alone whether a GEMM is worth the
// statistics and split passes, with cut-offs measured on the paper's GPU.
// Here the decision is measured per shape on this GPU: the candidates AUTO
// (statistics + selection + the selected emulated path), TF32X (split +
// tensor-core GEMM, no statistics) and FP32 (SIMT) run on synthetic operands
// of the shape and the fastest is recorded in the handle's table, which
// QCS_SIZE_RULE_TUNED consults.  Every candidate keeps the FP32 accuracy
// level, so the choice is about time only.  For shapes with few output tiles
// the tensor-core schedule is measured too: the K-range count (split K) that
// runs the faster emulated candidate fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <tuple>

#include "internal.h"

namespace qcs {
namespace {

// Complex parts of magnitude in [1, 2) with random signs: every exponent is
// 0, so the statistics select FP16X whatever the tolerance.  The bits come
// from SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
// number generators", 2014) of the element index.
__global__ void fill_unit_binade(float2 *__restrict__ x, int64_t n, uint64_t seed) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const uint32_t a = (uint32_t)z, b = (uint32_t)(z >> 32);
        x[i] = make_float2(__uint_as_float(0x3F800000u | (a & 0x807FFFFFu)),
                           __uint_as_float(0x3F800000u | (b & 0x807FFFFFu)));
    }
}

// Above the SIMT CGEMM's rate: the CUDA cores' FP32 FMA peak at the maximum
// clock is 152 SMs x 128 lanes x 2 flops x 2.07 GHz = 80.5 TFLOP/s.
constexpr double kFp32BoundFlops = 90e12;
constexpr float kFp32Prune = 4.0f;
const int kCandidates[3] = {QCS_MODE_AUTO, QCS_MODE_TF32X, QCS_MODE_FP32};

// FP32 FMA throughput of the CUDA cores: each thread runs 16 independent
// chains x <- x a + b (a, b are arguments, so nothing folds), 128 FMAs per
// loop trip.  The sum is stored only if it equals -1, which it never does
// for a in (0, 1), b > 0, so the chains stay live.
__global__ void __launch_bounds__(256) fma_peak_kernel(float a, float b, int iters, float *sink) {
    float x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = threadIdx.x * 1e-3f + (float)j;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int j = 0; j < 16; ++j) x[j] = fmaf(x[j], a, b);
    }
    float sum = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) sum += x[j];
    if (sum == -1.0f) sink[blockIdx.x] = sum;
}

struct DeviceBuffer {
    void *p = nullptr;
    ~DeviceBuffer() {
        if (p) cudaFree(p);
    }
};

}  // namespace

int tune_shape(qcs_handle_t h, int opA, int opB, int64_t m, int64_t n, int64_t k, int reps,
               qcs_tune_entry_t *out) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return QCS_ERR_UNSUPPORTED;
    const int64_t ra = (opA == QCS_OP_N) ? m : k, ca = (opA == QCS_OP_N) ? k : m;
    const int64_t rb = (opB == QCS_OP_N) ? k : n, cb = (opB == QCS_OP_N) ? n : k;
    // the largest K-range count any timing below uses
    size_t ws = 0;
    for (int c : kCandidates)
        ws = std::max(ws, gemm_workspace_bytes(c, m, n, k, h->num_sms, kMaxSplits));
    if (int r = ensure_workspace(h->ws, ws)) return r;
    DeviceBuffer A, B, C;
    if (cudaMalloc(&A.p, sizeof(float2) * ra * ca) != cudaSuccess ||
        cudaMalloc(&B.p, sizeof(float2) * rb * cb) != cudaSuccess ||
        cudaMalloc(&C.p, sizeof(float2) * m * n) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_ALLOC;
    }
    float2 *dA = static_cast<float2 *>(A.p), *dB = static_cast<float2 *>(B.p);
    float2 *dC = static_cast<float2 *>(C.p);
    const unsigned grid = (unsigned)(4 * h->num_sms);
    fill_unit_binade<<<grid, 256, 0, h->stream>>>(dA, ra * ca, 0x5151ull);
    fill_unit_binade<<<grid, 256, 0, h->stream>>>(dB, rb * cb, 0xA2A2ull);
    if (cudaGetLastError() != cudaSuccess) return QCS_ERR_CUDA;

    // a new measurement replaces the table's entry, which must not steer it
    h->tuned.erase(std::make_tuple(m, n, k, opA, opB));
    qcs_tune_entry_t e{};
    e.m = m;
    e.n = n;
    e.k = k;
    e.opA = opA;
    e.opB = opB;
    e.reps = reps;
    for (float &v : e.ms) v = -1.f;

    // Tuning calls are not the caller's work: no profile records, no
    // selection counts.  The emulated candidates run at the per-shape K-range
    // count (or the one qcs_set_tc_splits forces) unless a count is being
    // measured.
    const int profiling = h->profiling;
    unsigned long long *counts = h->d_counts;
    const int forced_splits = h->tc_splits;
    h->profiling = 0;
    h->d_counts = nullptr;
    h->tc_splits = forced_splits > 0 ? forced_splits
                                     : tc_split_count(m, n, k, 1, h->num_sms, 0);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = QCS_SUCCESS;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = QCS_ERR_CUDA;
    auto run = [&](int mode) {
        return run_cgemm(h, h->ws.ptr, mode, opA, opB, m, n, k, make_float2(1.f, 0.f), dA, ra, dB,
                         rb, make_float2(0.f, 0.f), dC, m, nullptr, nullptr);
    };
    auto time_mode = [&](int mode) -> int {
        if (int r = run(mode)) return r;  // untimed first call
        if (cudaEventRecord(e0, h->stream) != cudaSuccess) return QCS_ERR_CUDA;
        for (int i = 0; i < reps; ++i)
            if (int r = run(mode)) return r;
        if (cudaEventRecord(e1, h->stream) != cudaSuccess ||
            cudaEventSynchronize(e1) != cudaSuccess)
            return QCS_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) return QCS_ERR_CUDA;
        e.ms[mode] = ms / (float)reps;
        return QCS_SUCCESS;
    };
    if (rc == QCS_SUCCESS) rc = time_mode(QCS_MODE_AUTO);
    if (rc == QCS_SUCCESS) rc = time_mode(QCS_MODE_TF32X);
    // The tensor-core schedule: with few output tiles, time the faster
    // emulated candidate at other K-range counts and keep the fastest.
    const int64_t tiles = ((m + kBM - 1) / kBM) * ((n + kBN - 1) / kBN);
    if (rc == QCS_SUCCESS && forced_splits == 0 && tiles < 2 * (int64_t)h->num_sms) {
        const int emu = e.ms[QCS_MODE_TF32X] < e.ms[QCS_MODE_AUTO] ? QCS_MODE_TF32X : QCS_MODE_AUTO;
        const int heuristic = h->tc_splits;
        int best_s = heuristic;
        float best_ms = e.ms[emu];
        const int64_t nkb = (k + 31) / 32;
        for (int S : {1, 2, 4, 8, 16}) {
            if (S == heuristic || S > nkb) continue;
            h->tc_splits = S;
            if ((rc = time_mode(emu)) != QCS_SUCCESS) break;
            if (e.ms[emu] < best_ms) {
                best_ms = e.ms[emu];
                best_s = S;
            }
        }
        e.ms[emu] = best_ms;
        e.splits = best_s;
    }
    // The raster: with many output tiles, time the faster emulated candidate
    // with groups of 2, 4, 8 and 16 tile rows and keep the fastest.
    if (rc == QCS_SUCCESS && tiles >= 2 * (int64_t)h->num_sms) {
        const int emu = e.ms[QCS_MODE_TF32X] < e.ms[QCS_MODE_AUTO] ? QCS_MODE_TF32X : QCS_MODE_AUTO;
        const int handle_gm = h->tc_group_m;
        int best_g = handle_gm;
        float best_ms = e.ms[emu];
        for (int g : {2, 4, 8, 16}) {
            if (g == handle_gm) continue;
            h->tc_group_m = g;
            if ((rc = time_mode(emu)) != QCS_SUCCESS) break;
            if (e.ms[emu] < best_ms) {
                best_ms = e.ms[emu];
                best_g = g;
            }
        }
        h->tc_group_m = handle_gm;
        e.ms[emu] = best_ms;
        e.group_m = best_g;
    }
    h->tc_splits = forced_splits;
    if (rc == QCS_SUCCESS) {
        const float emulated = std::min(e.ms[QCS_MODE_AUTO], e.ms[QCS_MODE_TF32X]);
        const double fp32_bound_ms = 8.0 * (double)m * (double)n * (double)k / kFp32BoundFlops * 1e3;
        if (fp32_bound_ms <= kFp32Prune * emulated) rc = time_mode(QCS_MODE_FP32);
    }
    h->profiling = profiling;
    h->d_counts = counts;
    h->tc_splits = forced_splits;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (rc != QCS_SUCCESS) {
        cudaGetLastError();
        return rc;
    }
    e.best = QCS_MODE_AUTO;
    for (int c : kCandidates)
        if (e.ms[c] >= 0.f && e.ms[c] < e.ms[e.best]) e.best = c;
    h->tuned[std::make_tuple(m, n, k, opA, opB)] = e;
    if (out) *out = e;
    return QCS_SUCCESS;
}

}  // namespace qcs

using namespace qcs;

namespace {
bool valid_tune_op(int op) { return op == QCS_OP_N || op == QCS_OP_T || op == QCS_OP_C; }
}  // namespace

extern "C" {

int qcs_autotune_gemm(qcs_handle_t h, qcs_op_t transA, qcs_op_t transB, int64_t m, int64_t n,
                      int64_t k, int reps, qcs_tune_entry_t *out) {
    if (!h || !valid_tune_op(transA) || !valid_tune_op(transB) || m < 1 || n < 1 || k < 1 ||
        reps < 1)
        return QCS_ERR_INVALID_ARG;
    if (m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) return QCS_ERR_UNSUPPORTED;
    return tune_shape(h, transA, transB, m, n, k, reps, out);
}

int qcs_get_tuning(qcs_handle_t h, qcs_tune_entry_t *entries, int64_t capacity, int64_t *count) {
    if (!h || capacity < 0 || (capacity > 0 && !entries)) return QCS_ERR_INVALID_ARG;
    int64_t i = 0;
    for (const auto &kv : h->tuned) {
        if (i >= capacity) break;
        entries[i++] = kv.second;
    }
    if (count) *count = (int64_t)h->tuned.size();
    return QCS_SUCCESS;
}

int qcs_set_tuning(qcs_handle_t h, const qcs_tune_entry_t *entries, int64_t count) {
    if (!h || count < 0 || (count > 0 && !entries)) return QCS_ERR_INVALID_ARG;
    for (int64_t i = 0; i < count; ++i) {
        const qcs_tune_entry_t &e = entries[i];
        if (e.m < 1 || e.n < 1 || e.k < 1 || !valid_tune_op(e.opA) || !valid_tune_op(e.opB) ||
            (e.best != QCS_MODE_AUTO && e.best != QCS_MODE_TF32X && e.best != QCS_MODE_FP32) ||
            e.splits < 0 || e.splits > kMaxSplits || e.group_m < 0 || e.group_m > 64)
            return QCS_ERR_INVALID_ARG;
    }
    for (int64_t i = 0; i < count; ++i) {
        const qcs_tune_entry_t &e = entries[i];
        h->tuned[std::make_tuple(e.m, e.n, e.k, (int)e.opA, (int)e.opB)] = e;
    }
    return QCS_SUCCESS;
}

}  // extern "C"


int qcs_measure_fma_peak(qcs_handle_t h, double *tflops) {
    if (!h || !tflops) return QCS_ERR_INVALID_ARG;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    if (cs != cudaStreamCaptureStatusNone) return QCS_ERR_UNSUPPORTED;
    const int blocks = 8 * h->num_sms;  // 64 warps per SM
    const int iters = 4096;             // 2^19 FMAs per thread: about 50 ms
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return QCS_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return QCS_ERR_CUDA;
    }
    float *sink = static_cast<float *>(h->ws.ptr);  // never written (see the kernel)
    fma_peak_kernel<<<blocks, 256, 0, h->stream>>>(0.999999f, 1e-6f, iters / 8, sink);
    cudaEventRecord(e0, h->stream);
    fma_peak_kernel<<<blocks, 256, 0, h->stream>>>(0.999999f, 1e-6f, iters, sink);
    cudaEventRecord(e1, h->stream);
    float ms = 0.f;
    const bool ok = cudaGetLastError() == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms > 0.f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!ok) {
        cudaGetLastError();
        return QCS_ERR_CUDA;
    }
    const double flops = 2.0 * 128.0 * iters * 256.0 * blocks;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return QCS_SUCCESS;
}
