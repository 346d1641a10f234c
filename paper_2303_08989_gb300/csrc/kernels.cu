// Memory-bound kernels of the emulated-CGEMM path and the plain FP32 CGEMM.
//
//   stats2_kernel     exponent statistics (Section 4.1) of one or two
//                     matrices in one HBM pass: a histogram of biased
//                     exponents over every real and imaginary scalar,
//                     counted in lane-private shared-memory bins (no bank
//                     conflicts, no contended atomics).
//   select_kernel     the mode-selection rule of Section 4.1 on the device
//                     (the statistics never go to the host, Section 4.2).
//   split_kernel      Eq. 1 of Section 2.1 after the power-of-two scaling of
//                     Section 4.2: op(X) -> four planes hi.re, hi.im, lo.re,
//                     lo.im in the K-contiguous layout the tensor-core kernel
//                     loads with TMA (transposing through shared memory when
//                     the source is contiguous along the other index).
//   permute_kernel    strided gather of a tensor (TTGT reshaping, slicing).
//   cgemm_simt_kernel plain FP32 complex GEMM on the CUDA cores (the FP32
//                     baseline and mode).
//   cgemm_skinny_kernel  bandwidth-bound CGEMM for very small m, n or k
//                     (Section 5.3.2 irregular shapes).
//   split_real_kernel, sgemm_simt_kernel, the statistics on float input:
//                     the same stages for real operands (qcs_sgemm).
//   split_gauss_kernel, derive_3m_desc_kernel, combine_3m_kernel: the
//                     three-product (Gauss) form of an emulated CGEMM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "internal.h"
#include "ptx.cuh"

namespace qcs {

// ===========================================================================
// Exponent statistics
// ===========================================================================

namespace {

constexpr int kStatsWarps = kStatsThreads / 32;
constexpr size_t kStatsSmem = size_t(kStatsWarps) * 256 * 32 * sizeof(uint32_t);  // 128 KB

__device__ __forceinline__ void count_scalar(uint32_t *h, int lane, float x, uint32_t &nz) {
    const uint32_t u = __float_as_uint(x);
    if ((u & 0x7FFFFFFFu) == 0u) {
        ++nz;
    } else {
        atomicAdd(&h[((u >> 23) & 0xFFu) * 32u + lane], 1u);
    }
}

__global__ void __launch_bounds__(kStatsThreads) stats2_kernel(
    const float2 *__restrict__ X0, int64_t rows0, int64_t cols0, int64_t ld0, int gA,
    const float2 *__restrict__ X1, int64_t rows1, int64_t cols1, int64_t ld1, int gB,
    int64_t *__restrict__ partials) {
    extern __shared__ uint32_t hist[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kStatsWarps * 256 * 32; i += kStatsThreads) hist[i] = 0u;
    __syncthreads();
    uint32_t *h = hist + warp * 256 * 32;

    const bool first = blockIdx.x < gA;
    const float2 *X = first ? X0 : X1;
    const int64_t rows = first ? rows0 : rows1, cols = first ? cols0 : cols1;
    const int64_t ld = first ? ld0 : ld1;
    const int64_t blk = first ? blockIdx.x : blockIdx.x - gA;
    const int64_t nblk = first ? gA : gB;
    uint32_t nz = 0;

    const int64_t nel = rows * cols;  // complex elements
    if (nel > 0) {
        const int64_t gtid = blk * kStatsThreads + tid;
        const int64_t gstride = nblk * kStatsThreads;
        if (ld == rows && (reinterpret_cast<uintptr_t>(X) & 15u) == 0) {
            // contiguous: two complex values per 16-byte load, 16 loads in
            // flight per thread (4 warps per SM must cover the HBM latency)
            const float4 *p = reinterpret_cast<const float4 *>(X);
            const int64_t n4 = nel >> 1;
            constexpr int U = 16;
            int64_t i = gtid;
            for (; i + (U - 1) * gstride < n4; i += U * gstride) {
                float4 v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) v[u] = __ldcs(p + i + u * gstride);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    count_scalar(h, lane, v[u].x, nz);
                    count_scalar(h, lane, v[u].y, nz);
                    count_scalar(h, lane, v[u].z, nz);
                    count_scalar(h, lane, v[u].w, nz);
                }
            }
            for (; i < n4; i += gstride) {
                const float4 v = __ldcs(p + i);
                count_scalar(h, lane, v.x, nz);
                count_scalar(h, lane, v.y, nz);
                count_scalar(h, lane, v.z, nz);
                count_scalar(h, lane, v.w, nz);
            }
            if ((nel & 1) && gtid == 0) {
                const float2 v = X[nel - 1];
                count_scalar(h, lane, v.x, nz);
                count_scalar(h, lane, v.y, nz);
            }
        } else {
            for (int64_t i = gtid; i < nel; i += gstride) {
                const int64_t c = i / rows, r = i - c * rows;
                const float2 v = X[r + c * ld];
                count_scalar(h, lane, v.x, nz);
                count_scalar(h, lane, v.y, nz);
            }
        }
    }
    __syncthreads();
    int64_t *out = partials + static_cast<int64_t>(blockIdx.x) * kPartialStride;
    for (int bin = tid; bin < 256; bin += kStatsThreads) {
        uint64_t s = 0;
        for (int w = 0; w < kStatsWarps; ++w)
            for (int l = 0; l < 32; ++l) {
                const int ll = (l + tid) & 31;  // rotate lanes: conflict-free reads
                s += hist[(w * 256 + bin) * 32 + ll];
            }
        out[bin] = static_cast<int64_t>(s);
    }
    // zero count: block reduction
    __shared__ uint32_t zsum[kStatsWarps];
    uint32_t z = nz;
    for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
    if (lane == 0) zsum[warp] = z;
    __syncthreads();
    if (tid == 0) {
        uint64_t t = 0;
        for (int w = 0; w < kStatsWarps; ++w) t += zsum[w];
        out[256] = static_cast<int64_t>(t);
    }
}

// Section 4.1 readings: zeros enter no count; "larger than the minimum value
// of FP16" is e >= -14; the scaled window is [e_max - 28, e_max]; binary32
// subnormals (bin 0) count as outside both windows.
struct Summary {
    int64_t nnz, nonfinite, under1, under2;
    int bmax;  // highest finite bin in use, -1 if none
};

__device__ Summary summarize(const int64_t *h) {
    Summary s;
    s.nonfinite = h[255];
    s.nnz = 0;
    s.bmax = -1;
    s.under1 = 0;
    for (int b = 0; b < 255; ++b) {
        s.nnz += h[b];
        if (h[b] > 0) s.bmax = b;
        if (b < 127 - 14) s.under1 += h[b];
    }
    s.under2 = h[0];
    for (int b = 1; b < s.bmax - 28; ++b) s.under2 += h[b];
    return s;
}

__device__ void select_rule(const Summary &a, const Summary &b, double tol, int forced,
                            qcs_gemm_desc_t *desc) {
    auto ok1 = [&](const Summary &s) {
        return s.bmax < 0 || (s.bmax - 127 <= 14 && (double)s.under1 <= tol * (double)s.nnz);
    };
    auto ok2 = [&](const Summary &s) { return (double)s.under2 <= tol * (double)s.nnz; };
    auto scale = [&](const Summary &s) { return s.bmax < 0 ? 0 : 14 - (s.bmax - 127); };
    int mode;
    int sA = 0, sB = 0;
    if (forced == QCS_MODE_FP16X_SCALED) {
        mode = QCS_MODE_FP16X_SCALED;
        sA = scale(a);
        sB = scale(b);
    } else if (a.nonfinite > 0 || b.nonfinite > 0 || a.bmax >= 254 || b.bmax >= 254) {
        mode = QCS_MODE_FP32;
    } else if (!ok2(a) || !ok2(b)) {
        mode = QCS_MODE_TF32X;
    } else if (!ok1(a) || !ok1(b)) {
        mode = QCS_MODE_FP16X_SCALED;
        sA = scale(a);
        sB = scale(b);
    } else {
        mode = QCS_MODE_FP16X;
    }
    desc->mode = mode;
    desc->sA = sA;
    desc->sB = sB;
    desc->reserved = 0;
}

__global__ void __launch_bounds__(256) select_kernel(const int64_t *__restrict__ partials, int gA,
                                                     int gB, int64_t nA, int64_t nB, double tol,
                                                     int forced, qcs_stats_t *statsA,
                                                     qcs_stats_t *statsB, qcs_gemm_desc_t *desc) {
    __shared__ int64_t hA[257], hB[257];
    for (int bin = threadIdx.x; bin < 257; bin += blockDim.x) {
        int64_t sa = 0, sb = 0;
        for (int b = 0; b < gA; ++b) sa += partials[(int64_t)b * kPartialStride + bin];
        for (int b = 0; b < gB; ++b) sb += partials[(int64_t)(gA + b) * kPartialStride + bin];
        hA[bin] = sa;
        hB[bin] = sb;
    }
    __syncthreads();
    for (int bin = threadIdx.x; bin < 256; bin += blockDim.x) {
        if (statsA) statsA->hist[bin] = hA[bin];
        if (statsB) statsB->hist[bin] = hB[bin];
    }
    if (threadIdx.x == 0) {
        if (statsA) {
            statsA->n_zero = hA[256];
            statsA->n = nA;
        }
        if (statsB) {
            statsB->n_zero = hB[256];
            statsB->n = nB;
        }
        if (desc) select_rule(summarize(hA), summarize(hB), tol, forced, desc);
    }
}

__global__ void select_from_stats_kernel(const qcs_stats_t *a, const qcs_stats_t *b, double tol,
                                         qcs_gemm_desc_t *desc) {
    __shared__ int64_t hA[256], hB[256];
    for (int bin = threadIdx.x; bin < 256; bin += blockDim.x) {
        hA[bin] = a->hist[bin];
        hB[bin] = b->hist[bin];
    }
    __syncthreads();
    if (threadIdx.x == 0) select_rule(summarize(hA), summarize(hB), tol, QCS_MODE_AUTO, desc);
}

__global__ void set_desc_kernel(qcs_gemm_desc_t *desc, int mode, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        desc[i].mode = mode;
        desc[i].sA = 0;
        desc[i].sB = 0;
        desc[i].reserved = 0;
    }
}

__global__ void stats_finalize_kernel(const int64_t *__restrict__ partials, int g, int64_t n,
                                      qcs_stats_t *out) {
    for (int bin = threadIdx.x; bin < 257; bin += blockDim.x) {
        int64_t s = 0;
        for (int b = 0; b < g; ++b) s += partials[(int64_t)b * kPartialStride + bin];
        if (bin < 256)
            out->hist[bin] = s;
        else
            out->n_zero = s;
    }
    if (threadIdx.x == 0) out->n = n;
}

}  // namespace

// ---------------------------------------------------------------------------
// Two-stage statistics for the GEMM path (Section 4.1 Stage 1 / Stage 2),
// register-only so that every SM runs at full occupancy.
//   pass 1: e_max (largest biased exponent of a finite nonzero scalar), the
//           number of zeros, of Inf/NaN and of finite nonzero scalars below
//           2^-14 (N - N1).
//   pass 2: only when the Stage 1 outcome does not decide the mode: the
//           number below the window shifted so that e_max becomes 14 (N - N2).
// Per-block partials: pass 1 five int64 (bmax, 0, zeros, nonfinite, under1),
// pass 2 one int64.
// ---------------------------------------------------------------------------

constexpr int kS2Threads = 256;

struct Acc1 {
    uint32_t bmax;
    uint32_t zeros, nonfinite, under1;
};

__device__ __forceinline__ void acc1_scalar(Acc1 &a, float x) {
    const uint32_t mag = __float_as_uint(x) & 0x7FFFFFFFu;
    const uint32_t be = mag >> 23;
    const bool zero = mag == 0u;
    const bool nonfin = be == 255u;
    const bool fin_nz = !zero && !nonfin;
    a.bmax = fin_nz ? max(a.bmax, be) : a.bmax;
    a.zeros += zero;
    a.nonfinite += nonfin;
    a.under1 += (fin_nz && be < 113u);  // e < -14 (binary32 subnormals included)
}

template <class F>
__device__ __forceinline__ void for_each_scalar(const float2 *X, int64_t rows, int64_t cols,
                                                int64_t ld, int64_t gtid, int64_t gstride, F f) {
    const int64_t nel = rows * cols;
    if (nel <= 0) return;
    if (ld == rows && (reinterpret_cast<uintptr_t>(X) & 15u) == 0) {
        const float4 *p = reinterpret_cast<const float4 *>(X);
        const int64_t n4 = nel >> 1;
        constexpr int U = 8;
        int64_t i = gtid;
        for (; i + (U - 1) * gstride < n4; i += U * gstride) {
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = __ldcs(p + i + u * gstride);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                f(v[u].x);
                f(v[u].y);
                f(v[u].z);
                f(v[u].w);
            }
        }
        for (; i < n4; i += gstride) {
            const float4 v = __ldcs(p + i);
            f(v.x);
            f(v.y);
            f(v.z);
            f(v.w);
        }
        if ((nel & 1) && gtid == 0) {
            const float2 v = X[nel - 1];
            f(v.x);
            f(v.y);
        }
    } else {
        for (int64_t i = gtid; i < nel; i += gstride) {
            const int64_t c = i / rows, r = i - c * rows;
            const float2 v = X[r + c * ld];
            f(v.x);
            f(v.y);
        }
    }
}

// The same walk over a real matrix (one scalar per element).
template <class F>
__device__ __forceinline__ void for_each_scalar(const float *X, int64_t rows, int64_t cols,
                                                int64_t ld, int64_t gtid, int64_t gstride, F f) {
    const int64_t nel = rows * cols;
    if (nel <= 0) return;
    if (ld == rows && (reinterpret_cast<uintptr_t>(X) & 15u) == 0) {
        const float4 *p = reinterpret_cast<const float4 *>(X);
        const int64_t n4 = nel >> 2;
        constexpr int U = 8;
        int64_t i = gtid;
        for (; i + (U - 1) * gstride < n4; i += U * gstride) {
            float4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = __ldcs(p + i + u * gstride);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                f(v[u].x);
                f(v[u].y);
                f(v[u].z);
                f(v[u].w);
            }
        }
        for (; i < n4; i += gstride) {
            const float4 v = __ldcs(p + i);
            f(v.x);
            f(v.y);
            f(v.z);
            f(v.w);
        }
        if (gtid == 0)
            for (int64_t t = n4 << 2; t < nel; ++t) f(X[t]);
    } else {
        for (int64_t i = gtid; i < nel; i += gstride) {
            const int64_t c = i / rows, r = i - c * rows;
            f(X[r + c * ld]);
        }
    }
}

// Scalars per element: 2 for complex64, 1 for float.
template <class T>
__host__ __device__ constexpr int64_t scalars_per() { return (int64_t)(sizeof(T) / sizeof(float)); }

__device__ __forceinline__ uint32_t block_max(uint32_t v, uint32_t *sh) {
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    uint32_t r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = max(r, sh[w]);
    return r;
}

__device__ __forceinline__ uint64_t block_sum(uint64_t v, uint64_t *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    uint64_t r = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    return r;
}

template <class T>
__global__ void __launch_bounds__(kS2Threads) stats_pass1_kernel(
    const T *__restrict__ X0, int64_t rows0, int64_t cols0, int64_t ld0, int gA,
    const T *__restrict__ X1, int64_t rows1, int64_t cols1, int64_t ld1, int gB,
    int64_t *__restrict__ p1, int64_t dx0, int64_t dx1) {
    __shared__ uint32_t shm[kS2Threads / 32];
    __shared__ uint64_t shs[kS2Threads / 32];
    // instance blockIdx.y of a batch: operands dx0 / dx1 elements apart
    X0 += blockIdx.y * dx0;
    X1 += blockIdx.y * dx1;
    p1 += (int64_t)blockIdx.y * 5 * (gA + gB);
    const bool first = blockIdx.x < gA;
    const T *X = first ? X0 : X1;
    const int64_t blk = first ? blockIdx.x : blockIdx.x - gA;
    const int64_t nblk = first ? gA : gB;
    Acc1 a{0u, 0u, 0u, 0u};
    for_each_scalar(X, first ? rows0 : rows1, first ? cols0 : cols1, first ? ld0 : ld1,
                    blk * kS2Threads + threadIdx.x, nblk * kS2Threads,
                    [&](float x) { acc1_scalar(a, x); });
    const uint32_t bmax = block_max(a.bmax, shm);
    const uint64_t zeros = block_sum(a.zeros, shs);
    const uint64_t nonfin = block_sum(a.nonfinite, shs);
    const uint64_t under1 = block_sum(a.under1, shs);
    if (threadIdx.x == 0) {
        int64_t *o = p1 + (int64_t)blockIdx.x * 5;
        o[0] = bmax;
        o[1] = 0;
        o[2] = (int64_t)zeros;
        o[3] = (int64_t)nonfin;
        o[4] = (int64_t)under1;
    }
}

struct Sum1 {
    int64_t bmax, nnz, zeros, nonfinite, under1;
};

// Block-cooperative reduction of pass-1 partials [b0, b1); every thread
// returns the same result.
__device__ Sum1 reduce_p1(const int64_t *p1, int b0, int b1, int64_t total, uint32_t *shm,
                          uint64_t *shs) {
    uint32_t bmax = 0;
    uint64_t zeros = 0, nonfin = 0, under1 = 0;
    for (int b = b0 + (int)threadIdx.x; b < b1; b += (int)blockDim.x) {
        const int64_t *o = p1 + (int64_t)b * 5;
        bmax = max(bmax, (uint32_t)o[0]);
        zeros += (uint64_t)o[2];
        nonfin += (uint64_t)o[3];
        under1 += (uint64_t)o[4];
    }
    Sum1 s;
    s.bmax = block_max(bmax, shm);
    s.zeros = (int64_t)block_sum(zeros, shs);
    s.nonfinite = (int64_t)block_sum(nonfin, shs);
    s.under1 = (int64_t)block_sum(under1, shs);
    s.nnz = total - s.zeros - s.nonfinite;
    if (s.nnz == 0) s.bmax = -1;
    return s;
}

// Does the rule need Stage 2 (the shifted-window count)?  Same function in
// pass 2 and in the final selection, so both take the same decision.
__device__ bool needs_stage2(const Sum1 &a, const Sum1 &b, double tol, int forced) {
    if (forced == QCS_MODE_FP16X_SCALED) return false;
    if (a.nonfinite > 0 || b.nonfinite > 0 || a.bmax >= 254 || b.bmax >= 254) return false;
    auto ok1 = [&](const Sum1 &s) {
        return s.bmax < 0 || (s.bmax - 127 <= 14 && (double)s.under1 <= tol * (double)s.nnz);
    };
    return !(ok1(a) && ok1(b));
}

template <class T>
__global__ void __launch_bounds__(kS2Threads) stats_pass2_kernel(
    const T *__restrict__ X0, int64_t rows0, int64_t cols0, int64_t ld0, int gA,
    const T *__restrict__ X1, int64_t rows1, int64_t cols1, int64_t ld1, int gB,
    const int64_t *__restrict__ p1, double tol, int forced, int64_t *__restrict__ p2,
    int64_t dx0, int64_t dx1) {
    __shared__ uint64_t shs[kS2Threads / 32];
    __shared__ uint32_t shm[kS2Threads / 32];
    X0 += blockIdx.y * dx0;
    X1 += blockIdx.y * dx1;
    p1 += (int64_t)blockIdx.y * 5 * (gA + gB);
    p2 += (int64_t)blockIdx.y * (gA + gB);
    const Sum1 a = reduce_p1(p1, 0, gA, scalars_per<T>() * rows0 * cols0, shm, shs);
    const Sum1 b = reduce_p1(p1, gA, gA + gB, scalars_per<T>() * rows1 * cols1, shm, shs);
    if (!needs_stage2(a, b, tol, forced)) return;  // uniform across the block
    const int64_t bmax = (blockIdx.x < gA) ? a.bmax : b.bmax;
    const uint32_t thr = (uint32_t)(bmax - 28 > 1 ? bmax - 28 : 1);  // biased exponents below are outside
    const bool first = blockIdx.x < gA;
    const T *X = first ? X0 : X1;
    const int64_t blk = first ? blockIdx.x : blockIdx.x - gA;
    const int64_t nblk = first ? gA : gB;
    uint32_t under2 = 0;
    for_each_scalar(X, first ? rows0 : rows1, first ? cols0 : cols1, first ? ld0 : ld1,
                    blk * kS2Threads + threadIdx.x, nblk * kS2Threads, [&](float x) {
                        const uint32_t mag = __float_as_uint(x) & 0x7FFFFFFFu;
                        under2 += (mag != 0u && (mag >> 23) < thr);
                    });
    const uint64_t tot = block_sum(under2, shs);
    if (threadIdx.x == 0) p2[blockIdx.x] = (int64_t)tot;
}

__global__ void select2_kernel(const int64_t *__restrict__ p1, const int64_t *__restrict__ p2,
                               int gA, int gB, int64_t nA, int64_t nB, double tol, int forced,
                               qcs_gemm_desc_t *desc, unsigned long long *counts, double work,
                               int64_t *summary) {
    __shared__ uint64_t shs[kS2Threads / 32];
    __shared__ uint32_t shm[kS2Threads / 32];
    // instance blockIdx.x of a batch: its partials and its descriptor
    p1 += (int64_t)blockIdx.x * 5 * (gA + gB);
    p2 += (int64_t)blockIdx.x * (gA + gB);
    desc += blockIdx.x;
    const Sum1 a = reduce_p1(p1, 0, gA, nA, shm, shs);
    const Sum1 b = reduce_p1(p1, gA, gA + gB, nB, shm, shs);
    uint64_t u2a = 0, u2b = 0;
    const bool need2 = needs_stage2(a, b, tol, forced);
    if (need2) {
        for (int i = (int)threadIdx.x; i < gA + gB; i += (int)blockDim.x) {
            if (i < gA)
                u2a += (uint64_t)p2[i];
            else
                u2b += (uint64_t)p2[i];
        }
    }
    u2a = block_sum(u2a, shs);
    u2b = block_sum(u2b, shs);
    if (threadIdx.x != 0) return;
    Summary sa, sb;
    sa.nnz = a.nnz;
    sa.nonfinite = a.nonfinite;
    sa.under1 = a.under1;
    sa.bmax = (int)a.bmax;
    sb.nnz = b.nnz;
    sb.nonfinite = b.nonfinite;
    sb.under1 = b.under1;
    sb.bmax = (int)b.bmax;
    sa.under2 = (int64_t)u2a;
    sb.under2 = (int64_t)u2b;
    select_rule(sa, sb, tol, forced, desc);
    if (summary) {
        // per operand: biased e_max (-1: none), nonzero, Inf/NaN, below 2^-14,
        // below the shifted window (-1: Stage 2 not taken)
        const Sum1 *ss[2] = {&a, &b};
        const int64_t u2[2] = {(int64_t)u2a, (int64_t)u2b};
        for (int o = 0; o < 2; ++o) {
            summary[5 * o + 0] = ss[o]->bmax;
            summary[5 * o + 1] = ss[o]->nnz;
            summary[5 * o + 2] = ss[o]->nonfinite;
            summary[5 * o + 3] = ss[o]->under1;
            summary[5 * o + 4] = need2 ? u2[o] : -1;
        }
    }
    if (counts) {
        // counts[0..5]: GEMMs per selected mode; then 6 doubles of their 8 m n k
        atomicAdd(&counts[desc->mode], 1ULL);
        atomicAdd(reinterpret_cast<double *>(counts + QCS_NUM_MODES) + desc->mode, work);
    }
}

static bool g_stats_configured = false;

cudaError_t launch_stats2(const float2 *X0, int64_t rows0, int64_t cols0, int64_t ld0, int gA,
                          const float2 *X1, int64_t rows1, int64_t cols1, int64_t ld1, int gB,
                          int64_t *partials, cudaStream_t s) {
    if (!g_stats_configured) {
        cudaError_t e = cudaFuncSetAttribute(stats2_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kStatsSmem);
        if (e != cudaSuccess) return e;
        g_stats_configured = true;
    }
    stats2_kernel<<<gA + gB, kStatsThreads, kStatsSmem, s>>>(X0, rows0, cols0, ld0, gA, X1, rows1,
                                                            cols1, ld1, gB, partials);
    return cudaGetLastError();
}

cudaError_t launch_select(const int64_t *partials, int gA, int gB, int64_t nA, int64_t nB,
                          double tol, int forced_mode, qcs_stats_t *statsA, qcs_stats_t *statsB,
                          qcs_gemm_desc_t *desc, cudaStream_t s) {
    select_kernel<<<1, 256, 0, s>>>(partials, gA, gB, nA, nB, tol, forced_mode, statsA, statsB,
                                    desc);
    return cudaGetLastError();
}

template <class T>
static cudaError_t stats_select_2stage(const T *X0, int64_t rows0, int64_t cols0, int64_t ld0,
                                       int gA, const T *X1, int64_t rows1, int64_t cols1,
                                       int64_t ld1, int gB, double tol, int forced, int64_t *p1,
                                       int64_t *p2, qcs_gemm_desc_t *desc,
                                       unsigned long long *counts, double work, cudaStream_t s,
                                       int64_t *summary, int G = 1, int64_t dx0 = 0,
                                       int64_t dx1 = 0) {
    if (G < 1 || G > 65535 || (G > 1 && summary)) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)(gA + gB), (unsigned)G);
    stats_pass1_kernel<T><<<grid, kS2Threads, 0, s>>>(X0, rows0, cols0, ld0, gA, X1, rows1,
                                                      cols1, ld1, gB, p1, dx0, dx1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    stats_pass2_kernel<T><<<grid, kS2Threads, 0, s>>>(X0, rows0, cols0, ld0, gA, X1, rows1,
                                                      cols1, ld1, gB, p1, tol, forced,
                                                      p2, dx0, dx1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    select2_kernel<<<G, kS2Threads, 0, s>>>(p1, p2, gA, gB, scalars_per<T>() * rows0 * cols0,
                                            scalars_per<T>() * rows1 * cols1, tol, forced, desc,
                                            counts, work, summary);
    return cudaGetLastError();
}

cudaError_t launch_stats_select_2stage_batch(const float2 *X0, int64_t rows0, int64_t cols0,
                                             int64_t ld0, int gA, int64_t dx0, const float2 *X1,
                                             int64_t rows1, int64_t cols1, int64_t ld1, int gB,
                                             int64_t dx1, int G, double tol, int forced,
                                             int64_t *p1, int64_t *p2, qcs_gemm_desc_t *desc,
                                             unsigned long long *counts, double work,
                                             cudaStream_t s) {
    return stats_select_2stage(X0, rows0, cols0, ld0, gA, X1, rows1, cols1, ld1, gB, tol, forced,
                               p1, p2, desc, counts, work, s, (int64_t *)nullptr, G, dx0, dx1);
}

cudaError_t launch_stats_select_2stage(const float2 *X0, int64_t rows0, int64_t cols0, int64_t ld0,
                                       int gA, const float2 *X1, int64_t rows1, int64_t cols1,
                                       int64_t ld1, int gB, double tol, int forced, int64_t *p1,
                                       int64_t *p2, qcs_gemm_desc_t *desc,
                                       unsigned long long *counts, double work, cudaStream_t s,
                                       int64_t *summary) {
    return stats_select_2stage(X0, rows0, cols0, ld0, gA, X1, rows1, cols1, ld1, gB, tol, forced,
                               p1, p2, desc, counts, work, s, summary);
}

cudaError_t launch_stats_select_2stage_real(const float *X0, int64_t rows0, int64_t cols0,
                                            int64_t ld0, int gA, const float *X1, int64_t rows1,
                                            int64_t cols1, int64_t ld1, int gB, double tol,
                                            int forced, int64_t *p1, int64_t *p2,
                                            qcs_gemm_desc_t *desc, unsigned long long *counts,
                                            double work, cudaStream_t s) {
    return stats_select_2stage(X0, rows0, cols0, ld0, gA, X1, rows1, cols1, ld1, gB, tol, forced,
                               p1, p2, desc, counts, work, s, (int64_t *)nullptr);
}

cudaError_t launch_select_from_stats(const qcs_stats_t *a, const qcs_stats_t *b, double tol,
                                     qcs_gemm_desc_t *desc, cudaStream_t s) {
    select_from_stats_kernel<<<1, 256, 0, s>>>(a, b, tol, desc);
    return cudaGetLastError();
}

cudaError_t launch_set_desc(qcs_gemm_desc_t *desc, int mode, cudaStream_t s, int count) {
    if (count < 1) return cudaSuccess;
    set_desc_kernel<<<(count + 255) / 256, 256, 0, s>>>(desc, mode, count);
    return cudaGetLastError();
}

cudaError_t launch_stats_finalize(const int64_t *partials, int g, int64_t n, qcs_stats_t *out,
                                  cudaStream_t s) {
    stats_finalize_kernel<<<1, 256, 0, s>>>(partials, g, n, out);
    return cudaGetLastError();
}

// ===========================================================================
// Split (Eq. 1) into tensor-core planes
// ===========================================================================

namespace {

constexpr int kSplitR = 32, kSplitC = 64;

// Eq. 1 for one scaled value xs: hi = toLow(xs), lo = toLow((xs - hi) 2^11),
// as bit patterns of the mode's low-precision type.
__device__ __forceinline__ void split_value(int mode, float xs, uint32_t &hi, uint32_t &lo) {
    if (mode == QCS_MODE_TF32X) {
        const uint32_t h = tf32_rn(xs);
        hi = h;
        lo = tf32_rn((xs - __uint_as_float(h)) * 2048.0f);
    } else if (mode == QCS_MODE_BF16X3) {
        const __nv_bfloat16 h = __float2bfloat16_rn(xs);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn((xs - __bfloat162float(h)) * 2048.0f));
    } else {
        const __half h = __float2half_rn(xs);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn((xs - __half2float(h)) * 2048.0f));
    }
}

// Multiplication by 2^s as one or two exact power-of-two factors: x * m1 * m2
// is the correctly rounded x 2^s, the value ldexpf(x, s) returns, at the cost
// of one or two multiplications.  s = 14 - e_max lies in [-113, 163]: one
// factor up to 2^127, two (each exact: the operand only grows) above.
struct Pow2Scale {
    float m1 = 1.f, m2 = 1.f;
};
__device__ __forceinline__ Pow2Scale pow2_scale(int s) {
    Pow2Scale p;
    const int s1 = s > 127 ? 127 : (s < -126 ? -126 : s);
    p.m1 = __int_as_float((127 + s1) << 23);
    const int s2 = s - s1;  // 0 unless s > 127 (s < -126 does not occur)
    p.m2 = __int_as_float((127 + (s2 > 127 ? 127 : s2)) << 23);
    return p;
}
__device__ __forceinline__ float apply_scale(float x, Pow2Scale p) { return (x * p.m1) * p.m2; }

// The scale exponent of a row of op(A) or a column of op(B) from its largest
// biased binary32 exponent E (-1: no nonzero finite scalar): the line is
// multiplied by 2^(14 - e_max), e_max = E - 127, so that its largest
// magnitude lands in [2^14, 2^15) as for a whole matrix in Section 4.1.
__device__ __forceinline__ int line_scale(int E) { return E < 0 ? 0 : 141 - E; }

// planes6: write op(B) as the five planes of the GEMM path (-hi.im, hi.re,
// hi.im, lo.re, lo.im) instead of hi.re, hi.im, lo.re, lo.im.
__global__ void __launch_bounds__(256, 8) split_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int which, const float2 *__restrict__ X, int64_t sr,
    int64_t sc, int conj, int64_t R, int64_t K, int64_t R_pad, int64_t K_pad, void *planes,
    int64_t pitch, int64_t plane_stride, int planes6, int64_t plane_off, void *planes32,
    int skip_tf32, int64_t x_bstride, int64_t off_bstride, const int *__restrict__ line_emax) {
    desc += blockIdx.z;  // instance z of a batch (SplitBatch)
    X += blockIdx.z * x_bstride;
    plane_off += blockIdx.z * off_bstride;
    const int mode = desc->mode;
    if (mode == QCS_MODE_FP32 || mode == QCS_MODE_AUTO || (skip_tf32 && mode == QCS_MODE_TF32X))
        return;
    // per-row (op(A)) / per-column (op(B)) scales: only when the descriptor
    // says so (reserved == kDescLineScales, written by rowcol_select_kernel)
    const bool lines = line_emax != nullptr && desc->reserved == kDescLineScales;
    const int s = (mode == QCS_MODE_FP16X_SCALED) ? (which == 0 ? desc->sA : desc->sB) : 0;
    const Pow2Scale ps2 = pow2_scale(s);

    __shared__ float2 tile[kSplitR][kSplitC + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * kSplitR;
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kSplitC;
    if (sc == 1) {
#pragma unroll
        for (int i = 0; i < kSplitR / 8; ++i) {
            const int rr = warp + 8 * i;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cc = lane + 32 * h;
                float2 v = make_float2(0.f, 0.f);
                if (r0 + rr < R && c0 + cc < K) v = X[(r0 + rr) * sr + (c0 + cc)];
                tile[rr][cc] = v;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < kSplitC / 8; ++i) {
            const int cc = warp + 8 * i;
            const int rr = lane;
            float2 v = make_float2(0.f, 0.f);
            if (r0 + rr < R && c0 + cc < K) v = X[(r0 + rr) * sr + (c0 + cc) * sc];
            tile[rr][cc] = v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSplitR / 8; ++i) {
        const int rr = warp + 8 * i;
        const int64_t r = r0 + rr;
        const int cc = 2 * lane;
        const int64_t c = c0 + cc;
        if (r >= R_pad || c >= K_pad) continue;
        float x[4];
        x[0] = tile[rr][cc].x;
        x[1] = conj ? -tile[rr][cc].y : tile[rr][cc].y;
        x[2] = tile[rr][cc + 1].x;
        x[3] = conj ? -tile[rr][cc + 1].y : tile[rr][cc + 1].y;
        int sr_ = s;
        Pow2Scale pr_ = ps2;
        if (lines) {
            sr_ = (r < R) ? line_scale(line_emax[r]) : 0;
            pr_ = pow2_scale(sr_);
        }
        const bool two = (c + 1 < K_pad);
        if (mode == QCS_MODE_FP16X || mode == QCS_MODE_FP16X_SCALED) {
            // Eq. 1 on the pairs (column c, column c + 1) of the real and of
            // the imaginary parts with packed conversions: per value the same
            // round-to-nearest steps as split_value, half the instructions
            float2 re = make_float2(x[0], x[2]), im = make_float2(x[1], x[3]);
            if (sr_ != 0) {
                re = make_float2(apply_scale(re.x, pr_), apply_scale(re.y, pr_));
                im = make_float2(apply_scale(im.x, pr_), apply_scale(im.y, pr_));
            }
            const __half2 hr = __float22half2_rn(re), hm = __float22half2_rn(im);
            const float2 fr = __half22float2(hr), fm = __half22float2(hm);
            const __half2 lr = __float22half2_rn(
                make_float2((re.x - fr.x) * 2048.0f, (re.y - fr.y) * 2048.0f));
            const __half2 lm = __float22half2_rn(
                make_float2((im.x - fm.x) * 2048.0f, (im.y - fm.y) * 2048.0f));
            auto bits = [](__half2 v) { return *reinterpret_cast<const uint32_t *>(&v); };
            uint32_t w[5];
            int nw = 0;
            if (planes6) w[nw++] = bits(hm) ^ 0x80008000u;  // -hi.im
            w[nw++] = bits(hr);
            w[nw++] = bits(hm);
            w[nw++] = bits(lr);
            w[nw++] = bits(lm);
            uint16_t *p = static_cast<uint16_t *>(planes) + plane_off + r * pitch + c;
            const bool vec = two && ((reinterpret_cast<uintptr_t>(p) & 3u) == 0);
#pragma unroll
            for (int pl = 0; pl < 5; ++pl) {
                if (pl < nw) {
                    if (vec) {
                        *reinterpret_cast<uint32_t *>(p) = w[pl];
                    } else {
                        p[0] = (uint16_t)(w[pl] & 0xFFFFu);
                        if (two) p[1] = (uint16_t)(w[pl] >> 16);
                    }
                }
                p += plane_stride;
            }
            continue;
        }
        // hi/lo of re and im for columns c and c+1
        uint32_t hib[4], lob[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_value(mode, (sr_ != 0) ? apply_scale(x[e], pr_) : x[e], hib[e], lob[e]);
        // x[0]/x[2] real, x[1]/x[3] imaginary parts of columns c, c+1; the
        // planes in the order written, two consecutive values each
        uint32_t v0[5], v1[5];
        int nv;
        if (!planes6) {
            v0[0] = hib[0], v1[0] = hib[2];
            v0[1] = hib[1], v1[1] = hib[3];
            v0[2] = lob[0], v1[2] = lob[2];
            v0[3] = lob[1], v1[3] = lob[3];
            nv = 4;
        } else {
            const uint32_t sg = (mode == QCS_MODE_TF32X) ? 0x80000000u : 0x8000u;
            v0[0] = hib[1] ^ sg, v1[0] = hib[3] ^ sg;
            v0[1] = hib[0], v1[1] = hib[2];
            v0[2] = hib[1], v1[2] = hib[3];
            v0[3] = lob[0], v1[3] = lob[2];
            v0[4] = lob[1], v1[4] = lob[3];
            nv = 5;
        }
        // plane_stride is even (K_pad is a multiple of 32), so every plane has
        // the alignment of the first
        if (mode == QCS_MODE_TF32X) {
            uint32_t *p = static_cast<uint32_t *>(planes32 ? planes32 : planes) + plane_off +
                          r * pitch + c;
            const bool vec = two && ((reinterpret_cast<uintptr_t>(p) & 7u) == 0);
#pragma unroll
            for (int pl = 0; pl < 5; ++pl) {
                if (pl < nv) {
                    if (vec) {
                        *reinterpret_cast<uint2 *>(p) = make_uint2(v0[pl], v1[pl]);
                    } else {
                        p[0] = v0[pl];
                        if (two) p[1] = v1[pl];
                    }
                }
                p += plane_stride;
            }
        } else {
            uint16_t *p = static_cast<uint16_t *>(planes) + plane_off + r * pitch + c;
            const bool vec = two && ((reinterpret_cast<uintptr_t>(p) & 3u) == 0);
#pragma unroll
            for (int pl = 0; pl < 5; ++pl) {
                if (pl < nv) {
                    if (vec) {
                        *reinterpret_cast<uint32_t *>(p) = v0[pl] | (v1[pl] << 16);
                    } else {
                        p[0] = (uint16_t)v0[pl];
                        if (two) p[1] = (uint16_t)v1[pl];
                    }
                }
                p += plane_stride;
            }
        }
    }
}

}  // namespace

cudaError_t launch_split(const qcs_gemm_desc_t *desc, int which, const float2 *X, int64_t sr,
                         int64_t sc, int conj, int64_t R, int64_t K, int64_t R_pad, int64_t K_pad,
                         void *planes, int64_t pitch, int64_t plane_stride, cudaStream_t s,
                         int planes6, int64_t plane_off, void *planes32, int skip_tf32,
                         const SplitBatch &sb, const int *line_emax) {
    if (R_pad <= 0 || K_pad <= 0 || sb.count < 1) return cudaSuccess;
    if (line_emax && sb.count != 1) return cudaErrorInvalidValue;
    dim3 grid((unsigned)((K_pad + kSplitC - 1) / kSplitC), (unsigned)((R_pad + kSplitR - 1) / kSplitR),
              (unsigned)sb.count);
    if (grid.y > 65535u || sb.count > 65535) return cudaErrorInvalidValue;
    split_kernel<<<grid, 256, 0, s>>>(desc, which, X, sr, sc, conj, R, K, R_pad, K_pad, planes,
                                      pitch, plane_stride, planes6, plane_off, planes32, skip_tf32,
                                      sb.in_stride, sb.off_stride, line_emax);
    return cudaGetLastError();
}

// ===========================================================================
// Per-row / per-column power-of-two scaling (a variant beyond the paper: the
// per-matrix scaling of Section 4.1 applied to each row of op(A) and each
// column of op(B)).
// ===========================================================================

namespace {

constexpr int kLineTile = 32;  // 32 x 32 tiles of the stored matrix, 256 threads

// biased binary32 exponent of a nonzero finite x (0: subnormal), -1 otherwise
__device__ __forceinline__ int biased_exp_nz(float x) {
    const uint32_t b = __float_as_uint(x) & 0x7FFFFFFFu;
    if (b == 0u) return -1;
    const int e = (int)(b >> 23);
    return e == 255 ? -1 : e;
}

__global__ void __launch_bounds__(256) line_emax_kernel(const float2 *__restrict__ X, int64_t rows,
                                                        int64_t cols, int64_t ld, int per_row,
                                                        int *__restrict__ emax) {
    __shared__ int red[8][kLineTile + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * kLineTile + lane;
    const int64_t ctiles = (cols + kLineTile - 1) / kLineTile;
    // a block walks several column tiles of its 32 rows; a row's maximum is
    // kept in registers across them and reduced once at the end
    int mine = -1;
    for (int64_t ct = blockIdx.y; ct < ctiles; ct += gridDim.y) {
        const int64_t c0 = ct * kLineTile;
        float2 v[kLineTile / 8];
#pragma unroll
        for (int i = 0; i < kLineTile / 8; ++i) {
            const int64_t c = c0 + warp + 8 * i;
            v[i] = (r < rows && c < cols) ? X[r + c * ld] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < kLineTile / 8; ++i) {
            const int64_t c = c0 + warp + 8 * i;
            int e = max(biased_exp_nz(v[i].x), biased_exp_nz(v[i].y));
            if (per_row) {
                mine = max(mine, e);
            } else {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
                if (lane == 0 && c < cols && e >= 0) atomicMax(emax + c, e);
            }
        }
    }
    if (per_row) {
        red[warp][lane] = mine;
        __syncthreads();
        if (warp == 0) {
            int m = red[0][lane];
#pragma unroll
            for (int w = 1; w < 8; ++w) m = max(m, red[w][lane]);
            if (r < rows && m >= 0) atomicMax(emax + r, m);
        }
    }
}

__global__ void __launch_bounds__(256) line_under_kernel(const float2 *__restrict__ X, int64_t rows,
                                                         int64_t cols, int64_t ld, int per_row,
                                                         const int *__restrict__ emax,
                                                         unsigned long long *__restrict__ counts) {
    __shared__ unsigned long long su[8], sn[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t r = (int64_t)blockIdx.x * kLineTile + lane;
    const int64_t ctiles = (cols + kLineTile - 1) / kLineTile;
    unsigned long long under = 0, nnz = 0;
    const int er = (per_row && r < rows) ? emax[r] : -1;
    for (int64_t ct = blockIdx.y; ct < ctiles; ct += gridDim.y) {
        const int64_t c0 = ct * kLineTile;
        float2 v[kLineTile / 8];
        int E[kLineTile / 8];
#pragma unroll
        for (int i = 0; i < kLineTile / 8; ++i) {
            const int64_t c = c0 + warp + 8 * i;
            const bool in = r < rows && c < cols;
            v[i] = in ? X[r + c * ld] : make_float2(0.f, 0.f);  // zeros count nowhere
            E[i] = per_row ? er : (c < cols ? emax[c] : -1);
        }
#pragma unroll
        for (int i = 0; i < kLineTile / 8; ++i) {
            const float parts[2] = {v[i].x, v[i].y};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int b = biased_exp_nz(parts[h]);
                if (b < 0) continue;
                ++nnz;
                if (b == 0 || b < E[i] - 28) ++under;
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        under += __shfl_xor_sync(0xffffffffu, under, o);
        nnz += __shfl_xor_sync(0xffffffffu, nnz, o);
    }
    if (lane == 0) {
        su[warp] = under;
        sn[warp] = nnz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long tu = 0, tn = 0;
        for (int w = 0; w < 8; ++w) {
            tu += su[w];
            tn += sn[w];
        }
        if (tu) atomicAdd(counts, tu);
        if (tn) atomicAdd(counts + 1, tn);
    }
}

__global__ void rowcol_select_kernel(const qcs_gemm_desc_t *__restrict__ desc0,
                                     const unsigned long long *__restrict__ counts, double tol,
                                     qcs_gemm_desc_t *descK, qcs_gemm_desc_t *descOut) {
    qcs_gemm_desc_t d = *desc0;
    qcs_gemm_desc_t out = d;
    d.reserved = 0;
    // only where Section 4.1 gives up on FP16 (TF32X): every line scaled to
    // its own maximum, each operand's count below the shifted windows
    // tolerated as the whole-matrix count is
    if (d.mode == QCS_MODE_TF32X && (double)counts[0] <= tol * (double)counts[1] &&
        (double)counts[2] <= tol * (double)counts[3]) {
        d.mode = QCS_MODE_FP16X_SCALED;
        d.sA = d.sB = 0;
        d.reserved = kDescLineScales;
        out.mode = QCS_MODE_FP16X_ROWCOL;
        out.sA = out.sB = 0;
        out.reserved = 0;
    }
    *descK = d;
    *descOut = out;
}

__global__ void __launch_bounds__(256) rowcol_combine_kernel(
    const qcs_gemm_desc_t *__restrict__ descK, const int *__restrict__ emaxA,
    const int *__restrict__ emaxB, const float2 *__restrict__ P, int64_t m, int64_t n,
    float2 alpha, float2 beta, float2 *__restrict__ C, int64_t ldc) {
    const bool lines = descK->reserved == kDescLineScales;
    const bool use_beta = (beta.x != 0.0f) || (beta.y != 0.0f);
    const int64_t mn = m * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < mn;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = t / m, i = t - j * m;
        float pr = P[t].x, pi = P[t].y;
        if (lines) {
            // 2^-(sA_i + sB_j) in one correctly rounded step
            const int sh = -(line_scale(emaxA[i]) + line_scale(emaxB[j]));
            pr = ldexpf(pr, sh);
            pi = ldexpf(pi, sh);
        }
        float2 o;
        o.x = alpha.x * pr - alpha.y * pi;
        o.y = alpha.x * pi + alpha.y * pr;
        float2 *dst = C + i + j * ldc;
        if (use_beta) {
            const float2 c = *dst;
            o.x += beta.x * c.x - beta.y * c.y;
            o.y += beta.x * c.y + beta.y * c.x;
        }
        *dst = o;
    }
}

// 32-row block columns, each block walking up to kLineTilesPerBlock column
// tiles (fewer blocks, more bytes in flight per thread)
constexpr int kLineTilesPerBlock = 16;
dim3 line_grid(int64_t rows, int64_t cols) {
    const int64_t gx = (rows + kLineTile - 1) / kLineTile;
    const int64_t ct = (cols + kLineTile - 1) / kLineTile;
    const int64_t gy = (ct + kLineTilesPerBlock - 1) / kLineTilesPerBlock;
    return dim3((unsigned)gx, (unsigned)std::min<int64_t>(gy, 65535));
}

}  // namespace

cudaError_t launch_line_emax(const float2 *X, int64_t rows, int64_t cols, int64_t ld, int per_row,
                             int *emax, cudaStream_t s) {
    const int64_t lines = per_row ? rows : cols;
    if (lines > 0) {
        cudaError_t e = cudaMemsetAsync(emax, 0xFF, sizeof(int) * (size_t)lines, s);
        if (e != cudaSuccess) return e;
    }
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if ((rows + kLineTile - 1) / kLineTile > INT32_MAX) return cudaErrorInvalidValue;
    line_emax_kernel<<<line_grid(rows, cols), 256, 0, s>>>(X, rows, cols, ld, per_row, emax);
    return cudaGetLastError();
}

cudaError_t launch_line_under(const float2 *X, int64_t rows, int64_t cols, int64_t ld,
                              int per_row, const int *emax, unsigned long long *counts,
                              cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return cudaSuccess;
    if ((rows + kLineTile - 1) / kLineTile > INT32_MAX) return cudaErrorInvalidValue;
    line_under_kernel<<<line_grid(rows, cols), 256, 0, s>>>(X, rows, cols, ld, per_row, emax,
                                                            counts);
    return cudaGetLastError();
}

cudaError_t launch_rowcol_select(const qcs_gemm_desc_t *desc0, const unsigned long long *counts,
                                 double tol, qcs_gemm_desc_t *descK, qcs_gemm_desc_t *descOut,
                                 cudaStream_t s) {
    rowcol_select_kernel<<<1, 1, 0, s>>>(desc0, counts, tol, descK, descOut);
    return cudaGetLastError();
}

cudaError_t launch_rowcol_combine(const qcs_gemm_desc_t *descK, const int *emaxA,
                                  const int *emaxB, const float2 *P, int64_t m, int64_t n,
                                  float2 alpha, float2 beta, float2 *C, int64_t ldc, int num_sms,
                                  cudaStream_t s) {
    if (m <= 0 || n <= 0) return cudaSuccess;
    const int64_t need = (m * n + 255) / 256, cap = (int64_t)num_sms * 16;
    rowcol_combine_kernel<<<(unsigned)std::min(need, cap), 256, 0, s>>>(descK, emaxA, emaxB, P, m,
                                                                       n, alpha, beta, C, ldc);
    return cudaGetLastError();
}


namespace {

// Eq. 1 for a real operand: op(X) (R x K, element (r, c) at X[r sr + c sc])
// into two planes, hi and lo, of R_pad x K_pad (row pitch ``pitch``, planes
// ``plane_stride`` elements apart), zero beyond R x K.  Elements are FP16,
// BF16 (2 bytes) or TF32 (4 bytes), the kind the descriptor selected.
__global__ void __launch_bounds__(256) split_real_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int which, const float *__restrict__ X, int64_t sr,
    int64_t sc, int64_t R, int64_t K, int64_t R_pad, int64_t K_pad, void *planes, int64_t pitch,
    int64_t plane_stride) {
    const int mode = desc->mode;
    if (mode == QCS_MODE_FP32 || mode == QCS_MODE_AUTO) return;
    const int s = (mode == QCS_MODE_FP16X_SCALED) ? (which == 0 ? desc->sA : desc->sB) : 0;
    const Pow2Scale ps2 = pow2_scale(s);

    __shared__ float tile[kSplitR][kSplitC + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * kSplitR;
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kSplitC;
    if (sc == 1) {
#pragma unroll
        for (int i = 0; i < kSplitR / 8; ++i) {
            const int rr = warp + 8 * i;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cc = lane + 32 * h;
                float v = 0.f;
                if (r0 + rr < R && c0 + cc < K) v = X[(r0 + rr) * sr + (c0 + cc)];
                tile[rr][cc] = v;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < kSplitC / 8; ++i) {
            const int cc = warp + 8 * i;
            const int rr = lane;
            float v = 0.f;
            if (r0 + rr < R && c0 + cc < K) v = X[(r0 + rr) * sr + (c0 + cc) * sc];
            tile[rr][cc] = v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kSplitR / 8; ++i) {
        const int rr = warp + 8 * i;
        const int64_t r = r0 + rr;
        const int cc = 2 * lane;
        const int64_t c = c0 + cc;
        if (r >= R_pad || c >= K_pad) continue;
        uint32_t hib[2], lob[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const float x = tile[rr][cc + e];
            split_value(mode, (s != 0) ? apply_scale(x, ps2) : x, hib[e], lob[e]);
        }
        const bool two = (c + 1 < K_pad);
        if (mode == QCS_MODE_TF32X) {
            uint32_t *p = static_cast<uint32_t *>(planes) + r * pitch + c;
            const bool vec = two && ((reinterpret_cast<uintptr_t>(p) & 7u) == 0);
            if (vec) {
                *reinterpret_cast<uint2 *>(p) = make_uint2(hib[0], hib[1]);
                *reinterpret_cast<uint2 *>(p + plane_stride) = make_uint2(lob[0], lob[1]);
            } else {
                p[0] = hib[0];
                p[plane_stride] = lob[0];
                if (two) {
                    p[1] = hib[1];
                    p[plane_stride + 1] = lob[1];
                }
            }
        } else {
            uint16_t *p = static_cast<uint16_t *>(planes) + r * pitch + c;
            const bool vec = two && ((reinterpret_cast<uintptr_t>(p) & 3u) == 0);
            if (vec) {
                *reinterpret_cast<uint32_t *>(p) = hib[0] | (hib[1] << 16);
                *reinterpret_cast<uint32_t *>(p + plane_stride) = lob[0] | (lob[1] << 16);
            } else {
                p[0] = (uint16_t)hib[0];
                p[plane_stride] = (uint16_t)lob[0];
                if (two) {
                    p[1] = (uint16_t)hib[1];
                    p[plane_stride + 1] = (uint16_t)lob[1];
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_split_real(const qcs_gemm_desc_t *desc, int which, const float *X, int64_t sr,
                              int64_t sc, int64_t R, int64_t K, int64_t R_pad, int64_t K_pad,
                              void *planes, int64_t pitch, int64_t plane_stride, cudaStream_t s) {
    if (R_pad <= 0 || K_pad <= 0) return cudaSuccess;
    dim3 grid((unsigned)((K_pad + kSplitC - 1) / kSplitC), (unsigned)((R_pad + kSplitR - 1) / kSplitR));
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    split_real_kernel<<<grid, 256, 0, s>>>(desc, which, X, sr, sc, R, K, R_pad, K_pad, planes,
                                           pitch, plane_stride);
    return cudaGetLastError();
}

namespace {

// Descriptors of the three real GEMMs of a Gauss product from the selected
// one (desc[0]): T1 = Ar Br and T2 = Ai Bi keep it; T3 = (Ar + Ai)(Br + Bi)
// takes one binade less of scaling for the FP16 kind, whose operand sums can
// reach twice the largest part (FP16X becomes FP16X_SCALED by 2^-1).
__global__ void derive_3m_desc_kernel(qcs_gemm_desc_t *desc) {
    qcs_gemm_desc_t d = desc[0];
    desc[1] = d;
    if (d.mode == QCS_MODE_FP16X || d.mode == QCS_MODE_FP16X_SCALED) {
        if (d.mode == QCS_MODE_FP16X) d.sA = d.sB = 0;
        d.mode = QCS_MODE_FP16X_SCALED;
        d.sA -= 1;
        d.sB -= 1;
    }
    desc[2] = d;
}

// C = alpha (T1 - T2 + i (T3 - T1 - T2)) + beta C from the three real
// products (consecutive m x n blocks of T, ld m); runs unless FP32 was
// selected.
__global__ void __launch_bounds__(256) combine_3m_kernel(const qcs_gemm_desc_t *__restrict__ desc,
                                                         int64_t m, int64_t n,
                                                         const float *__restrict__ T, float2 alpha,
                                                         float2 beta, float2 *__restrict__ C,
                                                         int64_t ldc) {
    if (desc->mode == QCS_MODE_FP32) return;
    const int64_t mn = m * n;
    const bool use_beta = (beta.x != 0.0f) || (beta.y != 0.0f);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mn;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float t1 = __ldcs(T + i), t2 = __ldcs(T + mn + i), t3 = __ldcs(T + 2 * mn + i);
        const float pr = t1 - t2;
        const float pi = (t3 - t1) - t2;
        const int64_t col = i / m;
        float2 *dst = C + col * ldc + (i - col * m);
        float2 o;
        o.x = alpha.x * pr - alpha.y * pi;
        o.y = alpha.x * pi + alpha.y * pr;
        if (use_beta) {
            const float2 c = *dst;
            o.x += beta.x * c.x - beta.y * c.y;
            o.y += beta.x * c.y + beta.y * c.x;
        }
        *dst = o;
    }
}

}  // namespace

namespace {

// The three real operands of a Gauss product in one pass over the complex
// op(X) (R x K, element (r, c) at X[r sr + c sc], conj: negate imaginary
// parts): part 0 the real parts, 1 the imaginary parts, 2 their binary32
// sum, each split by Eq. 1 into hi and lo planes at element offset
// p part_off (planes ``plane_stride`` apart).  Parts 0 and 1 take desc[0]'s
// scale, part 2 desc[2]'s; all three the kind of desc[0].  X is read once.
__global__ void __launch_bounds__(256) split_gauss_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int which, const float2 *__restrict__ X, int64_t sr,
    int64_t sc, int conj, int64_t R, int64_t K, int64_t R_pad, int64_t K_pad, void *planes,
    int64_t pitch, int64_t plane_stride, int64_t part_off) {
    const int mode = desc[0].mode;
    if (mode == QCS_MODE_FP32 || mode == QCS_MODE_AUTO) return;
    const int s12 = (mode == QCS_MODE_FP16X_SCALED) ? (which == 0 ? desc[0].sA : desc[0].sB) : 0;
    const int mode3 = desc[2].mode;
    const int s3 = (mode3 == QCS_MODE_FP16X_SCALED) ? (which == 0 ? desc[2].sA : desc[2].sB) : 0;
    const Pow2Scale ps12 = pow2_scale(s12), ps3 = pow2_scale(s3);

    __shared__ float2 tile[kSplitR][kSplitC + 1];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t r0 = static_cast<int64_t>(blockIdx.y) * kSplitR;
    const int64_t c0 = static_cast<int64_t>(blockIdx.x) * kSplitC;
    if (sc == 1) {
#pragma unroll
        for (int i = 0; i < kSplitR / 8; ++i) {
            const int rr = warp + 8 * i;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int cc = lane + 32 * h;
                float2 v = make_float2(0.f, 0.f);
                if (r0 + rr < R && c0 + cc < K) v = X[(r0 + rr) * sr + (c0 + cc)];
                tile[rr][cc] = v;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < kSplitC / 8; ++i) {
            const int cc = warp + 8 * i;
            const int rr = lane;
            float2 v = make_float2(0.f, 0.f);
            if (r0 + rr < R && c0 + cc < K) v = X[(r0 + rr) * sr + (c0 + cc) * sc];
            tile[rr][cc] = v;
        }
    }
    __syncthreads();
    const float isign = conj ? -1.0f : 1.0f;
#pragma unroll
    for (int i = 0; i < kSplitR / 8; ++i) {
        const int rr = warp + 8 * i;
        const int64_t r = r0 + rr;
        const int cc = 2 * lane;
        const int64_t c = c0 + cc;
        if (r >= R_pad || c >= K_pad) continue;
        const bool two = (c + 1 < K_pad);
#pragma unroll
        for (int part = 0; part < 3; ++part) {
            uint32_t hib[2], lob[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float2 v = tile[rr][cc + e];
                const float x = part == 0 ? v.x : (part == 1 ? isign * v.y : v.x + isign * v.y);
                const int s = part == 2 ? s3 : s12;
                split_value(part == 2 ? mode3 : mode,
                            (s != 0) ? apply_scale(x, part == 2 ? ps3 : ps12) : x, hib[e], lob[e]);
            }
            const int64_t off = part * part_off + r * pitch + c;
            if (mode == QCS_MODE_TF32X) {
                uint32_t *p = static_cast<uint32_t *>(planes) + off;
                const bool vec = two && ((reinterpret_cast<uintptr_t>(p) & 7u) == 0);
                if (vec) {
                    *reinterpret_cast<uint2 *>(p) = make_uint2(hib[0], hib[1]);
                    *reinterpret_cast<uint2 *>(p + plane_stride) = make_uint2(lob[0], lob[1]);
                } else {
                    p[0] = hib[0];
                    p[plane_stride] = lob[0];
                    if (two) {
                        p[1] = hib[1];
                        p[plane_stride + 1] = lob[1];
                    }
                }
            } else {
                uint16_t *p = static_cast<uint16_t *>(planes) + off;
                const bool vec = two && ((reinterpret_cast<uintptr_t>(p) & 3u) == 0);
                if (vec) {
                    *reinterpret_cast<uint32_t *>(p) = hib[0] | (hib[1] << 16);
                    *reinterpret_cast<uint32_t *>(p + plane_stride) = lob[0] | (lob[1] << 16);
                } else {
                    p[0] = (uint16_t)hib[0];
                    p[plane_stride] = (uint16_t)lob[0];
                    if (two) {
                        p[1] = (uint16_t)hib[1];
                        p[plane_stride + 1] = (uint16_t)lob[1];
                    }
                }
            }
        }
    }
}

}  // namespace

cudaError_t launch_split_gauss(const qcs_gemm_desc_t *desc, int which, const float2 *X, int64_t sr,
                               int64_t sc, int conj, int64_t R, int64_t K, int64_t R_pad,
                               int64_t K_pad, void *planes, int64_t pitch, int64_t plane_stride,
                               int64_t part_off, cudaStream_t s) {
    if (R_pad <= 0 || K_pad <= 0) return cudaSuccess;
    dim3 grid((unsigned)((K_pad + kSplitC - 1) / kSplitC), (unsigned)((R_pad + kSplitR - 1) / kSplitR));
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    split_gauss_kernel<<<grid, 256, 0, s>>>(desc, which, X, sr, sc, conj, R, K, R_pad, K_pad,
                                            planes, pitch, plane_stride, part_off);
    return cudaGetLastError();
}

cudaError_t launch_derive_3m_desc(qcs_gemm_desc_t *desc, cudaStream_t s) {
    derive_3m_desc_kernel<<<1, 1, 0, s>>>(desc);
    return cudaGetLastError();
}

cudaError_t launch_combine_3m(const qcs_gemm_desc_t *desc, int64_t m, int64_t n, const float *T,
                              float2 alpha, float2 beta, float2 *C, int64_t ldc, int num_sms,
                              cudaStream_t s) {
    if (m == 0 || n == 0) return cudaSuccess;
    const int64_t need = (m * n + 255) / 256, cap = (int64_t)num_sms * 8;
    combine_3m_kernel<<<(unsigned)(need < cap ? need : cap), 256, 0, s>>>(desc, m, n, T, alpha, beta,
                                                                         C, ldc);
    return cudaGetLastError();
}

// ===========================================================================
// Permute / gather, FP64 accumulation
// ===========================================================================

static int grid_for(int64_t total) {
    const int64_t blocks = (total + 255) / 256;
    return (int)(blocks < 65536 ? (blocks > 0 ? blocks : 1) : 65536);
}

namespace {

// Strided copy over a common index space of ``rank`` dims (first fastest):
// out[sum x_d os_d] (+)= in[sum x_d is_d].  A gather has dense output strides,
// a scatter dense input strides.  When some dims form a contiguous run in the
// output (group X, the run starting at stride 1) and others a contiguous run
// in the input (group Y), a 32 x 32 tile of (x, y) goes through shared
// memory: it is read with lanes along y (coalesced input) and written with
// lanes along x (coalesced output).  The remaining dims index the tiles.
struct CopyParams {
    int rank;
    int nx, ny, nr;       // sizes of the X, Y and rest groups
    int pow2;             // every dim is a power of two: decompose with shifts
    int64_t px, py;       // products of the X and Y dims
    int64_t tiles_x, tiles_y;
    int64_t rest;         // product of the rest dims
    int8_t lg[QCS_MAX_RANK];  // log2 of each dim (when pow2)
    int64_t dims[QCS_MAX_RANK];
    int64_t is[QCS_MAX_RANK];
    int64_t os[QCS_MAX_RANK];
    int8_t gx[QCS_MAX_RANK], gy[QCS_MAX_RANK], gr[QCS_MAX_RANK];  // dim ids per group
    // Batch (blockIdx.y = g): the input of copy g starts boff[g * boff_stride]
    // elements in (or g * bin when boff is NULL), its output g * bout.
    const int64_t *boff;
    int64_t boff_stride, bin, bout;
    const int64_t *oboff;  // not NULL: copy g writes oboff[g * oboff_stride] further too
    int64_t oboff_stride;
    const qcs_gemm_desc_t *gate;  // not NULL: copy only if the GEMM selected plain FP32
};

// The split form of the tiled copy: each element is stored as its Eq. 1
// planes (hi.re, hi.im, lo.re, lo.im), element ``out offset`` of each plane.
struct SplitOut {
    const qcs_gemm_desc_t *desc;
    int which;  // 0: op(A), scale sA; 1: op(B), scale sB
    void *planes;
    int64_t plane_stride;
    int planes6;  // the five-plane op(B) layout of the GEMM path
    int64_t off;  // element offset of this operand's rows in every plane
    void *planes32;  // not NULL: the planes of a TF32 selection (else ``planes``)
    int64_t off_bstride;  // batch (blockIdx.y = g): desc + g, rows g off_bstride further
};

// The SplitOut of instance blockIdx.y of a batched split.
__device__ __forceinline__ SplitOut batch_split_out(const SplitOut &so) {
    SplitOut r = so;
    r.desc = so.desc + blockIdx.y;
    r.off = so.off + blockIdx.y * so.off_bstride;
    return r;
}

__device__ __forceinline__ int64_t batch_in(const CopyParams &P) {
    const int64_t g = blockIdx.y;
    return P.boff ? P.boff[g * P.boff_stride] : g * P.bin;
}

__device__ __forceinline__ int64_t batch_out(const CopyParams &P) {
    const int64_t g = blockIdx.y;
    return g * P.bout + (P.oboff ? P.oboff[g * P.oboff_stride] : 0);
}

__device__ __forceinline__ void decompose(const CopyParams &P, const int8_t *g, int ng, int64_t v,
                                          int64_t &io, int64_t &oo) {
    io = 0;
    oo = 0;
    if (P.pow2) {
        for (int t = 0; t < ng; ++t) {
            const int d = g[t];
            const int64_t c = v & ((int64_t(1) << P.lg[d]) - 1);
            io += c * P.is[d];
            oo += c * P.os[d];
            v >>= P.lg[d];
        }
        return;
    }
    for (int t = 0; t < ng; ++t) {
        const int d = g[t];
        const int64_t q = v / P.dims[d];
        const int64_t c = v - q * P.dims[d];
        io += c * P.is[d];
        oo += c * P.os[d];
        v = q;
    }
}

constexpr int kTilesPerBlock = 8;

// Up to kTilesPerBlock tiles (consecutive rest indices) per block, software
// pipelined over two shared-memory buffers: the loads of tile t + 1 are in
// flight while tile t is written out, so a warp keeps global reads and
// writes outstanding at once.  Buffer t & 1 is rewritten two tiles later,
// after a barrier that every thread reaches only once it has finished
// reading that buffer.
template <bool SPLIT>
__global__ void __launch_bounds__(256, SPLIT ? 4 : 5) copy_tiled_kernel(CopyParams P,
                                                            const float2 *__restrict__ in,
                                                            float2 *__restrict__ out,
                                                            int accumulate, SplitOut so_batch) {
    int mode = 0, scale = 0;
    Pow2Scale pscale;
    const SplitOut so = SPLIT ? batch_split_out(so_batch) : so_batch;
    if (SPLIT) {
        mode = so.desc->mode;
        if (mode == QCS_MODE_FP32 || mode == QCS_MODE_AUTO) return;
        if (mode == QCS_MODE_FP16X_SCALED) scale = so.which == 0 ? so.desc->sA : so.desc->sB;
        pscale = pow2_scale(scale);
    } else if (P.gate && P.gate->mode != QCS_MODE_FP32) {
        return;
    }
    __shared__ float2 tile[2][32][33];
    __shared__ int64_t sxi[32], sxo[32], syi[32], syo[32], sr[kTilesPerBlock][2];
    in += batch_in(P);
    out += batch_out(P);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    int64_t b = blockIdx.x;
    const int64_t bx = b % P.tiles_x;
    b /= P.tiles_x;
    const int64_t by = b % P.tiles_y;
    const int64_t rb = (b / P.tiles_y) * kTilesPerBlock;  // first rest index of this block
    const int64_t x0 = bx * 32, y0 = by * 32;
    // offsets of the tile's rows and columns (shared by all its rest indices)
    // and of each rest index, computed once
    if (threadIdx.x < 32) {
        const int64_t x = x0 + threadIdx.x;
        int64_t io = 0, oo = 0;
        if (x < P.px) decompose(P, P.gx, P.nx, x, io, oo);
        sxi[threadIdx.x] = io;
        sxo[threadIdx.x] = oo;
    } else if (threadIdx.x < 64) {
        const int64_t y = y0 + threadIdx.x - 32;
        int64_t io = 0, oo = 0;
        if (y < P.py) decompose(P, P.gy, P.ny, y, io, oo);
        syi[threadIdx.x - 32] = io;
        syo[threadIdx.x - 32] = oo;
    } else if (threadIdx.x < 64 + kTilesPerBlock) {
        const int t = threadIdx.x - 64;
        int64_t io = 0, oo = 0;
        if (rb + t < P.rest) decompose(P, P.gr, P.nr, rb + t, io, oo);
        sr[t][0] = io;
        sr[t][1] = oo;
    }
    __syncthreads();
    const bool yok = (y0 + tx) < P.py;
    const bool xok = (x0 + tx) < P.px;
    const int nt = (int)min((int64_t)kTilesPerBlock, P.rest - rb);
    // this thread's four read and four write offsets within a tile, the same
    // for every rest index: kept in registers
    int64_t rin[4], rout[4];
    bool okin[4], okout[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int l = ty + 8 * r;
        rin[r] = sxi[l] + syi[tx];
        okin[r] = yok && x0 + l < P.px;
        rout[r] = sxo[tx] + syo[l];
        okout[r] = xok && y0 + l < P.py;
    }
    // read: lanes along y (contiguous input)
    float2 v[4];
    auto load = [&](int t) {
        const int64_t ri = sr[t][0];
#pragma unroll
        for (int r = 0; r < 4; ++r)
            if (okin[r]) v[r] = in[ri + rin[r]];
    };
    load(0);
    for (int t = 0; t < nt; ++t) {
        const int buf = t & 1;
#pragma unroll
        for (int r = 0; r < 4; ++r) tile[buf][ty + 8 * r][tx] = v[r];
        __syncthreads();
        if (t + 1 < nt) load(t + 1);
        // write: lanes along x (contiguous output)
        const int64_t ro = sr[t][1];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int yl = ty + 8 * r;
            if (okout[r]) {
                float2 w = tile[buf][tx][yl];
                const int64_t o = ro + rout[r];
                if (SPLIT) {
                    uint32_t h0, l0, h1, l1;
                    split_value(mode, scale ? apply_scale(w.x, pscale) : w.x, h0, l0);
                    split_value(mode, scale ? apply_scale(w.y, pscale) : w.y, h1, l1);
                    const int64_t ps = so.plane_stride;
                    const uint32_t sg = (mode == QCS_MODE_TF32X) ? 0x80000000u : 0x8000u;
                    uint32_t v[5];
                    int nv;
                    if (so.planes6) {
                        v[0] = h1 ^ sg;
                        v[1] = h0;
                        v[2] = h1;
                        v[3] = l0;
                        v[4] = l1;
                        nv = 5;
                    } else {
                        v[0] = h0;
                        v[1] = h1;
                        v[2] = l0;
                        v[3] = l1;
                        nv = 4;
                    }
                    // unrolled over the five possible planes, so that v stays in
                    // registers
                    if (mode == QCS_MODE_TF32X) {
                        uint32_t *p =
                            static_cast<uint32_t *>(so.planes32 ? so.planes32 : so.planes) + so.off + o;
#pragma unroll
                        for (int pl = 0; pl < 5; ++pl)
                            if (pl < nv) p[pl * ps] = v[pl];
                    } else {
                        uint16_t *p = static_cast<uint16_t *>(so.planes) + so.off + o;
#pragma unroll
                        for (int pl = 0; pl < 5; ++pl)
                            if (pl < nv) p[pl * ps] = (uint16_t)v[pl];
                    }
                    continue;
                }
                float2 *dst = out + o;
                if (accumulate) {
                    const float2 u = *dst;
                    w.x += u.x;
                    w.y += u.y;
                }
                *dst = w;
            }
        }
    }
}

// The split through a gather map with quads: the same tiles as
// copy_tiled_kernel<true>, and each thread writes one run of four
// consecutive output elements per tile (reading them from a column of the
// shared tile, 33 elements per row so that the reads spread over banks), so
// that every plane gets one 8-byte (16-bit kinds) or 16-byte (TF32) store
// per four elements.  Needs the output-contiguous run X to be a multiple of
// 4 elements long and every other output stride, the operand's plane offset
// and the plane stride to be multiples of 4 (split_quads_ok).  The kind of
// the low-precision type is read from the descriptor once per block.
constexpr int kQuadStages = 4;  // tiles in the cp.async ring: three in flight while one is written

template <int KIND, bool P5>
__device__ __forceinline__ void split_quads_body(const CopyParams &P, const float2 *__restrict__ in,
                                                 const SplitOut &so, const Pow2Scale &pscale,
                                                 float2 (*tile)[32][33], const int64_t *sxi,
                                                 const int64_t *sxo, const int64_t *syi,
                                                 const int64_t *syo, const int64_t (*sr)[2],
                                                 int64_t x0, int64_t y0, int nt) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // read: lanes along y
    const int xq = threadIdx.x & 7, yq = threadIdx.x >> 3;   // write: a quad of x per thread
    int64_t rin[4];
    bool okin[4];
    const bool yok = (y0 + tx) < P.py;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int l = ty + 8 * r;
        rin[r] = sxi[l] + syi[tx];
        okin[r] = yok && x0 + l < P.px;
    }
    const bool okout = (x0 + 4 * xq < P.px) && (y0 + yq < P.py);
    const int64_t rout = sxo[4 * xq] + syo[yq];
    const int64_t ps = so.plane_stride;
    // tile t -> ring slot t % kQuadStages as tile[slot][x][y]: a warp's copies
    // land in one contiguous 256-byte row (lanes along y); elements outside
    // the tensor are zero-filled
    auto load = [&](int t) {
        const int64_t ri = sr[t][0];
        const int buf = t % kQuadStages;
#pragma unroll
        for (int r = 0; r < 4; ++r)
            cp_async8(&tile[buf][ty + 8 * r][tx], okin[r] ? in + ri + rin[r] : in, okin[r] ? 8u : 0u);
    };
#pragma unroll
    for (int t = 0; t < kQuadStages - 1; ++t) {
        if (t < nt) load(t);
        cp_async_commit();
    }
    for (int t = 0; t < nt; ++t) {
        const int buf = t % kQuadStages;
        cp_async_wait<kQuadStages - 2>();  // this thread's copies of tile t have landed
        __syncthreads();  // everyone's have; and slot (t - 1) % kQuadStages is no longer read
        if (t + kQuadStages - 1 < nt) load(t + kQuadStages - 1);
        cp_async_commit();
        if (okout) {
            uint32_t h[2][4], lo[2][4];  // [re | im][element of the quad]
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 w = tile[buf][4 * xq + e][yq];
                split_value(KIND == 1 ? QCS_MODE_TF32X : (KIND == 2 ? QCS_MODE_BF16X3 : QCS_MODE_FP16X),
                            apply_scale(w.x, pscale), h[0][e], lo[0][e]);
                split_value(KIND == 1 ? QCS_MODE_TF32X : (KIND == 2 ? QCS_MODE_BF16X3 : QCS_MODE_FP16X),
                            apply_scale(w.y, pscale), h[1][e], lo[1][e]);
            }
            const int64_t o = so.off + sr[t][1] + rout;
            // plane order: P5 -hi.im, hi.re, hi.im, lo.re, lo.im; else hi.re, hi.im, lo.re, lo.im
            constexpr int NP = P5 ? 5 : 4;
            if (KIND == 1) {
                uint4 *p0 = reinterpret_cast<uint4 *>(static_cast<uint32_t *>(
                                so.planes32 ? so.planes32 : so.planes) + o);
                const int64_t step = ps / 4;  // plane stride in uint4
                uint4 q[NP];
                int k = 0;
                if (P5)
                    q[k++] = make_uint4(h[1][0] ^ 0x80000000u, h[1][1] ^ 0x80000000u,
                                        h[1][2] ^ 0x80000000u, h[1][3] ^ 0x80000000u);
                q[k++] = make_uint4(h[0][0], h[0][1], h[0][2], h[0][3]);
                q[k++] = make_uint4(h[1][0], h[1][1], h[1][2], h[1][3]);
                q[k++] = make_uint4(lo[0][0], lo[0][1], lo[0][2], lo[0][3]);
                q[k++] = make_uint4(lo[1][0], lo[1][1], lo[1][2], lo[1][3]);
#pragma unroll
                for (int pl = 0; pl < NP; ++pl) p0[pl * step] = q[pl];
            } else {
                uint2 *p0 = reinterpret_cast<uint2 *>(static_cast<uint16_t *>(so.planes) + o);
                const int64_t step = ps / 4;  // plane stride in uint2 (four 16-bit values)
                auto pack = [](const uint32_t (&x)[4], uint32_t flip) {
                    return make_uint2(((x[0] ^ flip) & 0xFFFFu) | ((x[1] ^ flip) << 16),
                                      ((x[2] ^ flip) & 0xFFFFu) | ((x[3] ^ flip) << 16));
                };
                uint2 q[NP];
                int k = 0;
                if (P5) q[k++] = pack(h[1], 0x8000u);
                q[k++] = pack(h[0], 0u);
                q[k++] = pack(h[1], 0u);
                q[k++] = pack(lo[0], 0u);
                q[k++] = pack(lo[1], 0u);
#pragma unroll
                for (int pl = 0; pl < NP; ++pl) p0[pl * step] = q[pl];
            }
        }
    }
    cp_async_wait<0>();
}

constexpr int kQuadMaxTiles = 64;  // tiles (rest indices) per block, at most

template <bool P5>
__global__ void __launch_bounds__(256, 4) split_quads_kernel(CopyParams P,
                                                             const float2 *__restrict__ in,
                                                             SplitOut so_batch, int tpb) {
    const SplitOut so = batch_split_out(so_batch);
    const int mode = so.desc->mode;
    if (mode == QCS_MODE_FP32 || mode == QCS_MODE_AUTO) return;
    const int scale =
        (mode == QCS_MODE_FP16X_SCALED) ? (so.which == 0 ? so.desc->sA : so.desc->sB) : 0;
    const Pow2Scale pscale = pow2_scale(scale);
    __shared__ __align__(16) float2 tile[kQuadStages][32][33];
    __shared__ int64_t sxi[32], sxo[32], syi[32], syo[32], sr[kQuadMaxTiles][2];
    in += batch_in(P);
    int64_t b = blockIdx.x;
    const int64_t bx = b % P.tiles_x;
    b /= P.tiles_x;
    const int64_t by = b % P.tiles_y;
    const int64_t rb = (b / P.tiles_y) * tpb;  // first rest index of this block
    const int64_t x0 = bx * 32, y0 = by * 32;
    if (threadIdx.x < 32) {
        const int64_t x = x0 + threadIdx.x;
        int64_t io = 0, oo = 0;
        if (x < P.px) decompose(P, P.gx, P.nx, x, io, oo);
        sxi[threadIdx.x] = io;
        sxo[threadIdx.x] = oo;
    } else if (threadIdx.x < 64) {
        const int64_t y = y0 + threadIdx.x - 32;
        int64_t io = 0, oo = 0;
        if (y < P.py) decompose(P, P.gy, P.ny, y, io, oo);
        syi[threadIdx.x - 32] = io;
        syo[threadIdx.x - 32] = oo;
    } else if (threadIdx.x < 64 + kQuadMaxTiles) {
        const int t = threadIdx.x - 64;
        int64_t io = 0, oo = 0;
        if (t < tpb && rb + t < P.rest) decompose(P, P.gr, P.nr, rb + t, io, oo);
        sr[t][0] = io;
        sr[t][1] = oo;
    }
    __syncthreads();
    const int nt = (int)min((int64_t)tpb, P.rest - rb);
    if (mode == QCS_MODE_TF32X)
        split_quads_body<1, P5>(P, in, so, pscale, tile, sxi, sxo, syi, syo, sr, x0, y0, nt);
    else if (mode == QCS_MODE_BF16X3)
        split_quads_body<2, P5>(P, in, so, pscale, tile, sxi, sxo, syi, syo, sr, x0, y0, nt);
    else
        split_quads_body<0, P5>(P, in, so, pscale, tile, sxi, sxo, syi, syo, sr, x0, y0, nt);
}

// Shared contiguous prefix (dims 0..nv-1 contiguous from stride 1 in both
// input and output, product pv): one block per ``per_block`` outer indices,
// threads copy the contiguous runs.
__global__ void __launch_bounds__(256) copy_vector_kernel(CopyParams P, int nv, int64_t pv,
                                                          int64_t outer, const float2 *__restrict__ in,
                                                          float2 *__restrict__ out, int accumulate) {
    if (P.gate && P.gate->mode != QCS_MODE_FP32) return;
    __shared__ int64_t so[2];
    in += batch_in(P);
    out += batch_out(P);
    for (int64_t q = blockIdx.x; q < outer; q += gridDim.x) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int64_t rem = q, io = 0, oo = 0;
            for (int d = nv; d < P.rank; ++d) {
                const int64_t t = rem / P.dims[d];
                const int64_t c = rem - t * P.dims[d];
                io += c * P.is[d];
                oo += c * P.os[d];
                rem = t;
            }
            so[0] = io;
            so[1] = oo;
        }
        __syncthreads();
        const float2 *src = in + so[0];
        float2 *dst = out + so[1];
        for (int64_t v = threadIdx.x; v < pv; v += blockDim.x) {
            float2 x = src[v];
            if (accumulate) {
                const float2 w = dst[v];
                x.x += w.x;
                x.y += w.y;
            }
            dst[v] = x;
        }
    }
}

// Element-wise fallback (neither a tile nor a contiguous run applies).
__global__ void copy_simple_kernel(CopyParams P, int64_t total, const float2 *__restrict__ in,
                                   float2 *__restrict__ out, int accumulate) {
    if (P.gate && P.gate->mode != QCS_MODE_FP32) return;
    in += batch_in(P);
    out += batch_out(P);
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total;
         o += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = o, io = 0, oo = 0;
        for (int d = 0; d < P.rank; ++d) {
            const int64_t q = rem / P.dims[d];
            const int64_t c = rem - q * P.dims[d];
            io += c * P.is[d];
            oo += c * P.os[d];
            rem = q;
        }
        float2 v = in[io];
        if (accumulate) {
            const float2 w = out[oo];
            v.x += w.x;
            v.y += w.y;
        }
        out[oo] = v;
    }
}

// X: the dims forming the output's contiguous run from stride 1 (up to 32
// elements).  Y: the dims outside X met while walking the input's
// contiguous run from stride 1 (dims of X may lie on that run too; their
// elements are read by neighbouring tile rows) until Y holds 32 elements.
void choose_groups(CopyParams &P) {
    bool inx[QCS_MAX_RANK] = {false};
    P.nx = 0;
    P.px = 1;
    {
        bool used[QCS_MAX_RANK] = {false};
        while (P.px < 32) {
            int f = -1;
            for (int d = 0; d < P.rank; ++d)
                if (!used[d] && P.os[d] == P.px && P.dims[d] > 1) f = d;
            if (f < 0) break;
            used[f] = inx[f] = true;
            P.gx[P.nx++] = (int8_t)f;
            P.px *= P.dims[f];
        }
    }
    P.ny = 0;
    P.py = 1;
    {
        bool used[QCS_MAX_RANK] = {false};
        int64_t run = 1;
        while (P.py < 32) {
            int f = -1;
            for (int d = 0; d < P.rank; ++d)
                if (!used[d] && P.is[d] == run && P.dims[d] > 1) f = d;
            if (f < 0) break;
            used[f] = true;
            run *= P.dims[f];
            if (!inx[f]) {
                P.gy[P.ny++] = (int8_t)f;
                P.py *= P.dims[f];
            }
        }
    }
}

// Dims, strides and the power-of-two shortcut of a copy.
void set_dims(CopyParams &P, int rank, const int64_t *dims, const int64_t *is, const int64_t *os) {
    P.rank = rank;
    P.pow2 = 1;
    for (int d = 0; d < rank; ++d) {
        P.dims[d] = dims[d];
        P.is[d] = is[d];
        P.os[d] = os[d];
        if (dims[d] & (dims[d] - 1)) P.pow2 = 0;
        int lg = 0;
        while ((int64_t(1) << lg) < dims[d]) ++lg;
        P.lg[d] = (int8_t)lg;
    }
}

// With the X and Y groups chosen: the rest group and the tile counts.
// Returns the number of blocks of the tiled kernel.
int64_t finish_tiled(CopyParams &P) {
    P.nr = 0;
    int64_t rest = 1;
    for (int d = 0; d < P.rank; ++d) {
        bool in_group = false;
        for (int a = 0; a < P.nx; ++a) in_group |= (P.gx[a] == d);
        for (int c = 0; c < P.ny; ++c) in_group |= (P.gy[c] == d);
        if (!in_group) {
            P.gr[P.nr++] = (int8_t)d;
            rest *= P.dims[d];
        }
    }
    P.tiles_x = (P.px + 31) / 32;
    P.tiles_y = (P.py + 31) / 32;
    P.rest = rest;
    return P.tiles_x * P.tiles_y * ((rest + kTilesPerBlock - 1) / kTilesPerBlock);
}

bool tiles_well(const CopyParams &P) { return P.nx > 0 && P.ny > 0 && P.px >= 4 && P.py >= 4; }

cudaError_t launch_copy(int rank, const int64_t *dims, const int64_t *is, const int64_t *os,
                        const float2 *in, float2 *out, int accumulate, cudaStream_t s,
                        const CopyBatch &cb = CopyBatch{}) {
    if (cb.count < 1 || cb.count > 65535) return cudaErrorInvalidValue;
    CopyParams P{};
    set_dims(P, rank, dims, is, os);
    P.boff = cb.off;
    P.boff_stride = cb.off_stride;
    P.bin = cb.in_stride;
    P.bout = cb.out_stride;
    P.oboff = cb.out_off;
    P.oboff_stride = cb.out_off_stride;
    P.gate = cb.gate;
    const unsigned G = (unsigned)cb.count;
    int64_t total = 1;
    for (int d = 0; d < rank; ++d) total *= dims[d];
    if (total == 0) return cudaSuccess;
    // dims contiguous from stride 1 on both sides (same dims, same order)
    int nv = 0;
    int64_t pv = 1;
    while (nv < rank && P.is[nv] == pv && P.os[nv] == pv) pv *= P.dims[nv++];
    choose_groups(P);
    const bool tiled_ok = tiles_well(P);
    if (pv >= 32 || (!tiled_ok && pv >= 4)) {
        const int64_t outer = total / pv;
        const int64_t blocks = outer < 65536 ? outer : 65536;
        copy_vector_kernel<<<dim3((unsigned)blocks, G), pv >= 256 ? 256 : (pv >= 128 ? 128 : 64), 0,
                             s>>>(P, nv, pv, outer, in, out, accumulate);
        return cudaGetLastError();
    }
    if (!tiled_ok) {
        copy_simple_kernel<<<dim3(grid_for(total), G), 256, 0, s>>>(P, total, in, out, accumulate);
        return cudaGetLastError();
    }
    const int64_t blocks = finish_tiled(P);
    if (blocks > INT32_MAX) return cudaErrorInvalidValue;
    copy_tiled_kernel<false><<<dim3((unsigned)blocks, G), 256, 0, s>>>(P, in, out, accumulate,
                                                                      SplitOut{});
    return cudaGetLastError();
}

// The split of a gathered operand as one tiled copy (see launch_split_gather).
bool split_gather_params(int which, int rank, const int64_t *dims, const int64_t *strides,
                         int64_t rows, int64_t pitch, CopyParams &P) {
    int64_t d2[QCS_MAX_RANK], is[QCS_MAX_RANK], os[QCS_MAX_RANK];
    int r2 = 0;
    // a dim of the gather view contributes x * cum to the view's linear index
    // t = (fast index) + rows * (slow index); its plane offset is fixed by
    // which part it lies in
    auto push = [&](int64_t dim, int64_t stride, int64_t cum) {
        if (r2 >= QCS_MAX_RANK) return false;
        const bool fast = cum < rows;
        const int64_t unit = fast ? cum : cum / rows;
        // op(A): plane row = fast index, column = slow; op(B): the other way round
        const bool to_row = (which == 0) == fast;
        d2[r2] = dim;
        is[r2] = stride;
        os[r2] = to_row ? unit * pitch : unit;
        ++r2;
        return true;
    };
    int64_t cum = 1;
    for (int d = 0; d < rank; ++d) {
        const int64_t dd = dims[d];
        if (cum < rows && cum * dd > rows) {  // straddles the boundary: two dims
            if (rows % cum != 0) return false;
            const int64_t d1 = rows / cum;
            if (dd % d1 != 0) return false;
            if (!push(d1, strides[d], cum) || !push(dd / d1, strides[d] * d1, cum * d1)) return false;
        } else if (!push(dd, strides[d], cum)) {
            return false;
        }
        cum *= dd;
    }
    P = CopyParams{};
    set_dims(P, r2, d2, is, os);
    choose_groups(P);
    return tiles_well(P);
}

}  // namespace

bool split_gather_supported(int which, int rank, const int64_t *dims, const int64_t *strides,
                            int64_t rows, int64_t pitch) {
    CopyParams P;
    return split_gather_params(which, rank, dims, strides, rows, pitch, P);
}

cudaError_t launch_split_gather(const qcs_gemm_desc_t *desc, int which, int rank,
                                const int64_t *dims, const int64_t *strides, const float2 *src,
                                int64_t rows, void *planes, int64_t pitch, int64_t plane_stride,
                                cudaStream_t s, int planes6, int64_t plane_off, void *planes32,
                                const SplitBatch &sb) {
    CopyParams P;
    if (!split_gather_params(which, rank, dims, strides, rows, pitch, P))
        return cudaErrorNotSupported;
    const int64_t blocks = finish_tiled(P);
    if (blocks == 0 || sb.count < 1) return cudaSuccess;
    if (blocks > INT32_MAX || sb.count > 65535) return cudaErrorInvalidValue;
    P.bin = sb.in_stride;  // instance blockIdx.y reads from src + y in_stride
    SplitOut so{desc, which, planes, plane_stride, planes6, plane_off, planes32, sb.off_stride};
    // quads: every output run of four elements lies inside the X run and
    // starts at a multiple of 4 in every plane
    bool quads = P.px % 4 == 0 && plane_off % 4 == 0 && plane_stride % 4 == 0;
    for (int d = 0; d < P.rank && quads; ++d) {
        bool in_x = false;
        for (int a = 0; a < P.nx; ++a) in_x |= (P.gx[a] == d);
        if (!in_x && P.os[d] % 4 != 0) quads = false;
    }
    if (quads) {
        // tiles per block: as many as make the grid a whole number of waves
        // (4 blocks of 256 threads per SM), at most kQuadMaxTiles
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return cudaGetLastError();
        const int64_t xy = P.tiles_x * P.tiles_y * sb.count, wave = 4 * (int64_t)sms;
        const int64_t min_blocks = xy * ((P.rest + kQuadMaxTiles - 1) / kQuadMaxTiles);
        const int64_t want = ((min_blocks + wave - 1) / wave) * wave;
        const int64_t chunks = std::max<int64_t>(1, want / xy);
        const int tpb = (int)std::min<int64_t>(kQuadMaxTiles, (P.rest + chunks - 1) / chunks);
        const int64_t qblocks = P.tiles_x * P.tiles_y * ((P.rest + tpb - 1) / tpb);
        if (qblocks > INT32_MAX) return cudaErrorInvalidValue;
        const dim3 grid((unsigned)qblocks, (unsigned)sb.count);
        if (planes6)
            split_quads_kernel<true><<<grid, 256, 0, s>>>(P, src, so, tpb);
        else
            split_quads_kernel<false><<<grid, 256, 0, s>>>(P, src, so, tpb);
    } else {
        copy_tiled_kernel<true><<<dim3((unsigned)blocks, (unsigned)sb.count), 256, 0, s>>>(
            P, src, nullptr, 0, so);
    }
    return cudaGetLastError();
}

namespace {

// dst[j] += (double) src[index ? index[j] : j], j < count (FP64 sums over
// slices, Section 5.3).
__global__ void accumulate_gather_c128_kernel(const float2 *__restrict__ src,
                                              const int64_t *__restrict__ index,
                                              double2 *__restrict__ dst, int64_t count) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = src[index ? index[j] : j];
        double2 d = dst[j];
        d.x += (double)v.x;
        d.y += (double)v.y;
        dst[j] = d;
    }
}

// grad_root[index ? index[j] : j] += (float) g[j]; atomics because an index
// may repeat (the same bitstring asked for twice).
__global__ void seed_grad_kernel(const double2 *__restrict__ g, const int64_t *__restrict__ index,
                                 float2 *__restrict__ grad_root, int64_t count) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = g[j];
        float2 *t = grad_root + (index ? index[j] : j);
        atomicAdd(&t->x, (float)v.x);
        atomicAdd(&t->y, (float)v.y);
    }
}

__global__ void accumulate_c128_kernel(const float2 *__restrict__ src, double2 *__restrict__ dst,
                                       int64_t count, int overwrite) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = src[i];
        double2 d = overwrite ? make_double2(0.0, 0.0) : dst[i];
        d.x += (double)v.x;
        d.y += (double)v.y;
        dst[i] = d;
    }
}

}  // namespace

cudaError_t launch_permute(int rank, const int64_t *dims, const int64_t *strides, int64_t offset,
                           const float2 *in, float2 *out, int64_t *stats_partials, int gstats,
                           cudaStream_t s, const CopyBatch &cb) {
    (void)stats_partials;
    (void)gstats;
    int64_t dense[QCS_MAX_RANK];
    int64_t acc = 1;
    for (int d = 0; d < rank; ++d) {
        dense[d] = acc;
        acc *= dims[d];
    }
    return launch_copy(rank, dims, strides, dense, in + offset, out, 0, s, cb);
}

cudaError_t launch_scatter(int rank, const int64_t *dims, const int64_t *strides, int64_t offset,
                           const float2 *src, float2 *dst, int accumulate, cudaStream_t s,
                           const CopyBatch &cb) {
    int64_t dense[QCS_MAX_RANK];
    int64_t acc = 1;
    for (int d = 0; d < rank; ++d) {
        dense[d] = acc;
        acc *= dims[d];
    }
    return launch_copy(rank, dims, dense, strides, src, dst + offset, accumulate, s, cb);
}

cudaError_t launch_accumulate_gather_c128(const float2 *src, const int64_t *index, double *dst,
                                          int64_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    accumulate_gather_c128_kernel<<<grid_for(count), 256, 0, s>>>(
        src, index, reinterpret_cast<double2 *>(dst), count);
    return cudaGetLastError();
}

cudaError_t launch_seed_grad(const double *g, const int64_t *index, float2 *grad_root,
                             int64_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    seed_grad_kernel<<<grid_for(count), 256, 0, s>>>(reinterpret_cast<const double2 *>(g), index,
                                                    grad_root, count);
    return cudaGetLastError();
}

cudaError_t launch_accumulate_c128(const float2 *src, double *dst, int64_t count, int overwrite,
                                   cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    const int64_t blocks = (count + 255) / 256;
    accumulate_c128_kernel<<<(unsigned)(blocks < 65536 ? blocks : 65536), 256, 0, s>>>(
        src, reinterpret_cast<double2 *>(dst), count, overwrite);
    return cudaGetLastError();
}

// ===========================================================================
// Small plain-FP32 contraction steps of one tree level, all in one launch
// ===========================================================================

namespace {

constexpr int kTreeSmallWarps = 4;

// One warp per (step, instance): the warp gathers op(A) and op(B) through
// the step's offset tables into its slice of shared memory, then each lane
// forms output elements e = lane, lane + 32, ... (i = e mod m, j = e div m)
// as the same FP32 FMA chain over l = 0 .. k-1 as the per-element FP32
// kernels (re: + ar br - ai bi, im: + ar bi + ai br), scaled by alpha the
// same way, and writes C contiguously.
__global__ void __launch_bounds__(32 * kTreeSmallWarps) tree_small_kernel(
    const TreeSmallStep *__restrict__ steps, int n_steps, int G, int inst0, int g0,
    const int64_t *__restrict__ off, int nl, const int32_t *__restrict__ tab, int smem_elems,
    float2 alpha) {
    extern __shared__ float2 tree_small_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * kTreeSmallWarps + warp;
    if (p >= (int64_t)n_steps * G) return;  // the whole warp; no block barrier follows
    const int r = (int)(p % G);
    const TreeSmallStep &st = steps[p / G];
    const int m = st.m, n = st.n, k = st.k;
    const int64_t inst = (int64_t)inst0 + r, g = (int64_t)g0 + r;
    const float2 *A = st.a + (st.a_leaf >= 0 ? off[inst * nl + st.a_leaf] : g * st.a_istride);
    const float2 *B = st.b + (st.b_leaf >= 0 ? off[inst * nl + st.b_leaf] : g * st.b_istride);
    float2 *C = st.c + g * st.c_istride;
    float2 *As = tree_small_smem + (size_t)warp * smem_elems;
    float2 *Bs = As + m * k;
    const int32_t *ta = tab + st.a_tab, *tb = tab + st.b_tab;
    for (int e = lane; e < m * k; e += 32) As[e] = A[ta[e]];
    for (int e = lane; e < k * n; e += 32) Bs[e] = B[tb[e]];
    __syncwarp();
    for (int e = lane; e < m * n; e += 32) {
        const int i = e % m, j = e / m;
        float sr = 0.f, si = 0.f;
        for (int l = 0; l < k; ++l) {
            const float2 a = As[i + l * m], b = Bs[l + j * k];
            sr = fmaf(a.x, b.x, sr);
            sr = fmaf(-a.y, b.y, sr);
            si = fmaf(a.x, b.y, si);
            si = fmaf(a.y, b.x, si);
        }
        float2 o;
        o.x = alpha.x * sr - alpha.y * si;
        o.y = alpha.x * si + alpha.y * sr;
        C[e] = o;
    }
}

// One warp per step of the level: gc, op(A) and op(B) into shared memory,
// then grad_A (m x k) and grad_B (k x n) element by element as FP32 FMA
// chains in the order of the per-element kernels with op C on the
// conjugated operand (the conjugation applied on load), and the writes
// through the offset tables.
__global__ void __launch_bounds__(32 * kTreeSmallWarps) tree_small_bwd_kernel(
    const TreeSmallBwd *__restrict__ steps, int n_steps, int G, int inst0,
    const int64_t *__restrict__ off, int nl, const int32_t *__restrict__ tab, int smem_elems) {
    extern __shared__ float2 tree_small_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t p = (int64_t)blockIdx.x * kTreeSmallWarps + warp;
    if (p >= (int64_t)n_steps * G) return;  // the whole warp; no block barrier follows
    const int r = (int)(p % G);
    const TreeSmallBwd &st = steps[p / G];
    const int m = st.m, n = st.n, k = st.k;
    const int64_t inst = (int64_t)inst0 + r;
    // element offsets of this instance's operands and their gradients
    const int64_t oa = st.a_leaf >= 0 ? off[inst * nl + st.a_leaf] : r * st.a_istride;
    const int64_t ob = st.b_leaf >= 0 ? off[inst * nl + st.b_leaf] : r * st.b_istride;
    const int64_t oga = (st.a_leaf >= 0 ? off[inst * nl + st.a_leaf] : 0) + r * st.ga_istride;
    const int64_t ogb = (st.b_leaf >= 0 ? off[inst * nl + st.b_leaf] : 0) + r * st.gb_istride;
    const float2 *gc = st.gc + r * st.gc_istride;
    float2 *Gs = tree_small_smem + (size_t)warp * smem_elems;
    float2 *As = Gs + m * n;
    float2 *Bs = As + m * k;
    const int32_t *ta = tab + st.a_tab, *tb = tab + st.b_tab;
    for (int e = lane; e < m * n; e += 32) Gs[e] = gc[e];
    for (int e = lane; e < m * k; e += 32) As[e] = st.a[oa + ta[e]];
    for (int e = lane; e < k * n; e += 32) Bs[e] = st.b[ob + tb[e]];
    __syncwarp();
    // grad_A[i, l] = sum_j gc[i, j] conj(B[l, j])
    for (int e = lane; e < m * k; e += 32) {
        const int i = e % m, l = e / m;
        float sr = 0.f, si = 0.f;
        for (int j = 0; j < n; ++j) {
            const float2 a = Gs[i + j * m];
            float2 b = Bs[l + j * k];
            b.y = -b.y;
            sr = fmaf(a.x, b.x, sr);
            sr = fmaf(-a.y, b.y, sr);
            si = fmaf(a.x, b.y, si);
            si = fmaf(a.y, b.x, si);
        }
        float2 *dst = st.ga + oga + ta[e];
        if (st.a_leaf >= 0) {
            const float2 u = *dst;
            sr += u.x;
            si += u.y;
        }
        *dst = make_float2(sr, si);
    }
    // grad_B[l, j] = sum_i conj(A[i, l]) gc[i, j]
    for (int e = lane; e < k * n; e += 32) {
        const int l = e % k, j = e / k;
        float sr = 0.f, si = 0.f;
        for (int i = 0; i < m; ++i) {
            float2 a = As[i + l * m];
            a.y = -a.y;
            const float2 b = Gs[i + j * m];
            sr = fmaf(a.x, b.x, sr);
            sr = fmaf(-a.y, b.y, sr);
            si = fmaf(a.x, b.y, si);
            si = fmaf(a.y, b.x, si);
        }
        float2 *dst = st.gb + ogb + tb[e];
        if (st.b_leaf >= 0) {
            const float2 u = *dst;
            sr += u.x;
            si += u.y;
        }
        *dst = make_float2(sr, si);
    }
}

}  // namespace

cudaError_t launch_tree_small(const TreeSmallStep *steps, int n_steps, int G, int inst0, int g0,
                              const int64_t *off, int nl, const int32_t *tab, int smem_elems,
                              cudaStream_t s) {
    if (n_steps <= 0 || G <= 0) return cudaSuccess;
    if (smem_elems < 1 || smem_elems > 2 * kTreeSmallOperand) return cudaErrorInvalidValue;
    static bool configured = false;  // the attribute is per function, set once
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(
            tree_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)(sizeof(float2) * 2 * kTreeSmallOperand * kTreeSmallWarps));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int64_t warps = (int64_t)n_steps * G;
    const int64_t blocks = (warps + kTreeSmallWarps - 1) / kTreeSmallWarps;
    if (blocks > INT32_MAX) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float2) * (size_t)smem_elems * kTreeSmallWarps;
    tree_small_kernel<<<(unsigned)blocks, 32 * kTreeSmallWarps, smem, s>>>(
        steps, n_steps, G, inst0, g0, off, nl, tab, smem_elems, make_float2(1.f, 0.f));
    return cudaGetLastError();
}

cudaError_t launch_tree_small_bwd(const TreeSmallBwd *steps, int n_steps, int G, int inst0,
                                  const int64_t *off, int nl, const int32_t *tab, int smem_elems,
                                  cudaStream_t s) {
    if (n_steps <= 0 || G <= 0) return cudaSuccess;
    if (smem_elems < 1 || smem_elems > kTreeSmallBwdElems) return cudaErrorInvalidValue;
    static bool configured = false;  // the attribute is per function, set once
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(
            tree_small_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)(sizeof(float2) * kTreeSmallBwdElems * kTreeSmallWarps));
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int64_t blocks = ((int64_t)n_steps * G + kTreeSmallWarps - 1) / kTreeSmallWarps;
    if (blocks > INT32_MAX) return cudaErrorInvalidValue;
    const size_t smem = sizeof(float2) * (size_t)smem_elems * kTreeSmallWarps;
    tree_small_bwd_kernel<<<(unsigned)blocks, 32 * kTreeSmallWarps, smem, s>>>(
        steps, n_steps, G, inst0, off, nl, tab, smem_elems);
    return cudaGetLastError();
}

namespace {

__global__ void leaf_grad_reduce_kernel(const LeafGradRef *__restrict__ leaves,
                                        const float2 *__restrict__ scratch, int64_t stride, int G) {
    const LeafGradRef &L = leaves[blockIdx.y];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L.size;
         e += (int64_t)gridDim.x * blockDim.x) {
        float2 acc = L.grad[e];
        for (int g = 0; g < G; ++g) {
            const float2 v = scratch[g * stride + L.scratch_off + e];
            acc.x += v.x;
            acc.y += v.y;
        }
        L.grad[e] = acc;
    }
}

}  // namespace

cudaError_t launch_leaf_grad_reduce(const LeafGradRef *leaves, int nl, int64_t max_size,
                                    const float2 *scratch, int64_t stride, int G, cudaStream_t s) {
    if (nl <= 0 || max_size <= 0) return cudaSuccess;
    if (nl > 65535) return cudaErrorInvalidValue;
    const int64_t bx = std::min<int64_t>((max_size + 255) / 256, 1024);
    leaf_grad_reduce_kernel<<<dim3((unsigned)bx, (unsigned)nl), 256, 0, s>>>(leaves, scratch,
                                                                           stride, G);
    return cudaGetLastError();
}

// ===========================================================================
// FP64 fidelity and error sums (qcs_fidelity_stats)
// ===========================================================================

namespace {

constexpr int kFidThreads = 256;

// The six quantities of one block in shared memory, summed (max for [5])
// over the block in a fixed tree.
__device__ void fid_block_reduce(double (&v)[6], double (*sh)[kFidThreads]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) sh[q][threadIdx.x] = v[q];
    __syncthreads();
    for (int w = kFidThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
#pragma unroll
            for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
            sh[5][threadIdx.x] = fmax(sh[5][threadIdx.x], sh[5][threadIdx.x + w]);
        }
        __syncthreads();
    }
}

// Block b sums the elements j = b, b + G, ... in one thread each, thread t
// of the block taking every kFidThreads-th of them, then the block's tree.
__global__ void __launch_bounds__(kFidThreads) fidelity_partials_kernel(
    const void *__restrict__ a, int a_c64, const double2 *__restrict__ ref, int64_t n,
    double *__restrict__ partials) {
    __shared__ double sh[6][kFidThreads];
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int64_t j = blockIdx.x * (int64_t)kFidThreads + threadIdx.x; j < n;
         j += (int64_t)gridDim.x * kFidThreads) {
        double2 x;
        if (a_c64) {
            const float2 f = reinterpret_cast<const float2 *>(a)[j];
            x = make_double2((double)f.x, (double)f.y);
        } else {
            x = reinterpret_cast<const double2 *>(a)[j];
        }
        v[0] = fma(x.x, x.x, fma(x.y, x.y, v[0]));
        if (ref) {
            const double2 r = ref[j];
            v[1] = fma(r.x, r.x, fma(r.y, r.y, v[1]));
            v[2] = fma(r.x, x.x, fma(r.y, x.y, v[2]));   // Re conj(r) x
            v[3] = fma(r.x, x.y, fma(-r.y, x.x, v[3]));  // Im conj(r) x
            const double dx = x.x - r.x, dy = x.y - r.y;
            const double d2 = fma(dx, dx, dy * dy);
            v[4] += d2;
            v[5] = fmax(v[5], sqrt(d2));
        }
    }
    fid_block_reduce(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < 6; ++q) partials[(int64_t)blockIdx.x * 6 + q] = sh[q][0];
}

__global__ void __launch_bounds__(kFidThreads) fidelity_final_kernel(
    const double *__restrict__ partials, int blocks, double *__restrict__ out) {
    __shared__ double sh[6][kFidThreads];
    double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < blocks; b += kFidThreads) {
#pragma unroll
        for (int q = 0; q < 5; ++q) v[q] += partials[(int64_t)b * 6 + q];
        v[5] = fmax(v[5], partials[(int64_t)b * 6 + 5]);
    }
    fid_block_reduce(v, sh);
    if (threadIdx.x < 6) out[threadIdx.x] = sh[threadIdx.x][0];
}

}  // namespace

cudaError_t launch_fidelity_stats(const void *a, int a_c64, const double *ref, int64_t n,
                                  double *partials, int blocks, double *out, cudaStream_t s) {
    if (blocks < 1 || blocks > kFidBlocksMax) return cudaErrorInvalidValue;
    fidelity_partials_kernel<<<blocks, kFidThreads, 0, s>>>(
        a, a_c64, reinterpret_cast<const double2 *>(ref), n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    fidelity_final_kernel<<<1, kFidThreads, 0, s>>>(partials, blocks, out);
    return cudaGetLastError();
}

// ===========================================================================
// Plain FP32 CGEMM on the CUDA cores
// ===========================================================================

namespace {

// C = alpha op(A) op(B) + beta C on the CUDA cores, four FP32 FMAs per
// complex multiply-add.  A block of 256 threads computes a 128 x 64 complex
// tile of C: warp w owns the 32 x 32 sub-tile at rows 32 (w % 4), columns
// 32 (w / 4); lane (ty, tx) = (lane / 8, lane % 8) owns rows 4 ty .. 4 ty + 3
// and 16 + 4 ty .. 16 + 4 ty + 3 of it, columns 2 tx, 2 tx + 1, 16 + 2 tx,
// 16 + 2 tx + 1 (8 x 4 complex accumulators).  Per k the lane reads its A
// and B values as six 16-byte shared loads, each one shared-memory wavefront
// (the A loads are broadcast over tx, the B loads contiguous over tx).
// Operand tiles of 16 k move from global to shared memory with 8-byte
// cp.async copies (zero-filled outside the matrix) in a three-stage ring, so
// the copies of k-tile t + 2 overlap the products of tile t.  op T and op C
// change the copy addressing; the conjugation of op C is folded into the
// signs of the FMAs (template flags CA, CB).
constexpr int kSBM = 128, kSBN = 64, kSBK = 16, kSStages = 3;
constexpr int kSRowA = kSBM + 2, kSRowB = kSBN + 2;  // padded rows (16-byte multiples)
constexpr size_t kSimtSmemA = sizeof(float2) * kSStages * kSBK * kSRowA;
constexpr size_t kSimtSmemBytes = kSimtSmemA + sizeof(float2) * kSStages * kSBK * kSRowB;

__device__ __forceinline__ float2 ld_op(const float2 *X, int op, int64_t r, int64_t c, int64_t ld) {
    float2 v = (op == QCS_OP_N) ? X[r + c * ld] : X[c + r * ld];
    if (op == QCS_OP_C) v.y = -v.y;
    return v;
}

template <int OPA, int OPB>
__global__ void __launch_bounds__(256, 2) cgemm_simt_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int m, int n, int k, float2 alpha,
    const float2 *__restrict__ A, int64_t lda, const float2 *__restrict__ B, int64_t ldb,
    float2 beta, float2 *__restrict__ C, int64_t ldc, GemmBatch bt) {
    constexpr bool transA = OPA != QCS_OP_N, transB = OPB != QCS_OP_N;
    constexpr bool CA = OPA == QCS_OP_C, CB = OPB == QCS_OP_C;
    if (desc && desc->mode != QCS_MODE_FP32) return;
    A += blockIdx.z * bt.sA;
    B += blockIdx.z * bt.sB;
    C += blockIdx.z * bt.sC;
    extern __shared__ __align__(16) unsigned char simt_smem[];
    float2 (*As)[kSBK][kSRowA] = reinterpret_cast<float2 (*)[kSBK][kSRowA]>(simt_smem);
    float2 (*Bs)[kSBK][kSRowB] = reinterpret_cast<float2 (*)[kSBK][kSRowB]>(simt_smem + kSimtSmemA);
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int ty = lane >> 3, tx = lane & 7;
    const int wm = (warp & 3) * 32, wn = (warp >> 2) * 32;
    const int64_t bm = static_cast<int64_t>(blockIdx.y) * kSBM;
    const int64_t bn = static_cast<int64_t>(blockIdx.x) * kSBN;

    // Copy assignment (fixed per thread): op(A) tile element (i, l) and op(B)
    // tile element (l, j).  op N of A: i = tid % 128, l = tid / 128 + 2 q;
    // op T/C: l = tid % 16, i = tid / 16 + 16 q (q < 8).  op N of B:
    // l = tid % 16, j = tid / 16 + 16 q; op T/C: j = tid % 64,
    // l = tid / 64 + 4 q (q < 4).  Consecutive threads read consecutive
    // addresses.  Copy q of k-tile kt reads base + kt kstep + q qstep; the
    // rows / columns outside the matrix are fixed per thread (bit q of the
    // mask), and k is checked only in the last k-tile.
    const int aI = transA ? (tid >> 4) : (tid & (kSBM - 1));
    const int aL = transA ? (tid & (kSBK - 1)) : (tid >> 7);
    const int bL = transB ? (tid >> 6) : (tid & (kSBK - 1));
    const int bJ = transB ? (tid & (kSBN - 1)) : (tid >> 4);
    const int64_t a_kstep = transA ? kSBK : kSBK * lda;
    const int64_t a_qstep = transA ? 16 * lda : 2 * lda;
    const int64_t b_kstep = transB ? kSBK * ldb : kSBK;
    const int64_t b_qstep = transB ? 4 * ldb : 16 * ldb;
    const float2 *a_base = A + (transA ? aL + (bm + aI) * lda : bm + aI + aL * lda);
    const float2 *b_base = B + (transB ? bn + bJ + bL * ldb : bL + (bn + bJ) * ldb);
    uint32_t a_mask = 0, b_mask = 0;  // bit q: copy q's row (column) lies inside the matrix
#pragma unroll
    for (int q = 0; q < 8; ++q)
        a_mask |= uint32_t(bm + aI + (transA ? 16 * q : 0) < m) << q;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        b_mask |= uint32_t(bn + bJ + (transB ? 0 : 16 * q) < n) << q;

    // a tile whose rows and columns all lie inside C copies without checks
    // except in the last k-tile
    const bool interior = bm + kSBM <= m && bn + kSBN <= n;

    // k-tile kt of both operands into ring slot st (8 + 4 copies per thread)
    auto load_tile = [&](int st, int kt) {
        const int64_t k0 = static_cast<int64_t>(kt) * kSBK;
        const bool tail = k0 + kSBK > k;
        const float2 *pa = a_base + kt * a_kstep;
        const float2 *pb = b_base + kt * b_kstep;
        if (interior && !tail) {
#pragma unroll
            for (int q = 0; q < 8; ++q)
                cp_async8(&As[st][transA ? aL : aL + 2 * q][transA ? aI + 16 * q : aI],
                          pa + q * a_qstep, 8u);
#pragma unroll
            for (int q = 0; q < 4; ++q)
                cp_async8(&Bs[st][transB ? bL + 4 * q : bL][transB ? bJ : bJ + 16 * q],
                          pb + q * b_qstep, 8u);
            return;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int l = transA ? aL : aL + 2 * q;
            const int i = transA ? aI + 16 * q : aI;
            bool ok = (a_mask >> q) & 1u;
            if (tail) ok = ok && k0 + l < k;
            cp_async8(&As[st][l][i], ok ? pa + q * a_qstep : A, ok ? 8u : 0u);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int l = transB ? bL + 4 * q : bL;
            const int j = transB ? bJ : bJ + 16 * q;
            bool ok = (b_mask >> q) & 1u;
            if (tail) ok = ok && k0 + l < k;
            cp_async8(&Bs[st][l][j], ok ? pb + q * b_qstep : B, ok ? 8u : 0u);
        }
    };

    float2 acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);

    const int ktiles = (k + kSBK - 1) / kSBK;
    if (ktiles > 0) load_tile(0, 0);
    cp_async_commit();
    if (ktiles > 1) load_tile(1, 1);
    cp_async_commit();
    for (int kt = 0; kt < ktiles; ++kt) {
        cp_async_wait<1>();  // every group but the newest has landed: tile kt
        __syncthreads();     // ... for all threads; and slot (kt + 2) % 3 is free
        if (kt + 2 < ktiles) load_tile((kt + 2) % kSStages, kt + 2);
        cp_async_commit();
        const int st = kt % kSStages;
#pragma unroll
        for (int l = 0; l < kSBK; ++l) {
            float2 a[8], b[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const float4 v = *reinterpret_cast<const float4 *>(
                    &As[st][l][wm + (h >> 1) * 16 + ty * 4 + (h & 1) * 2]);
                a[2 * h] = make_float2(v.x, v.y);
                a[2 * h + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 v = *reinterpret_cast<const float4 *>(&Bs[st][l][wn + h * 16 + tx * 2]);
                b[2 * h] = make_float2(v.x, v.y);
                b[2 * h + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // op(A) = (ar, sA ai), op(B) = (br, sB bi):
                    // re += ar br - sA sB ai bi, im += sB ar bi + sA ai br
                    acc[i][j].x = fmaf(a[i].x, b[j].x, acc[i][j].x);
                    acc[i][j].x = fmaf((CA == CB) ? -a[i].y : a[i].y, b[j].y, acc[i][j].x);
                    acc[i][j].y = fmaf(CB ? -a[i].x : a[i].x, b[j].y, acc[i][j].y);
                    acc[i][j].y = fmaf(CA ? -a[i].y : a[i].y, b[j].x, acc[i][j].y);
                }
        }
    }
    cp_async_wait<0>();

    const bool use_beta = (beta.x != 0.f) || (beta.y != 0.f);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t gj = bn + wn + (j >> 1) * 16 + tx * 2 + (j & 1);
        if (gj >= n) continue;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int64_t gi = bm + wm + (i >> 2) * 16 + ty * 4 + (i & 3);
            if (gi >= m) continue;
            float2 o;
            o.x = alpha.x * acc[i][j].x - alpha.y * acc[i][j].y;
            o.y = alpha.x * acc[i][j].y + alpha.y * acc[i][j].x;
            float2 *dst = C + gi + gj * ldc;
            if (use_beta) {
                const float2 c = *dst;
                o.x += beta.x * c.x - beta.y * c.y;
                o.y += beta.x * c.y + beta.y * c.x;
            }
            *dst = o;
        }
    }
}

template <int OPA, int OPB>
cudaError_t launch_simt_tiles(dim3 grid, cudaStream_t s, const qcs_gemm_desc_t *desc, int m,
                              int n, int k, float2 alpha, const float2 *A, int64_t lda,
                              const float2 *B, int64_t ldb, float2 beta, float2 *C, int64_t ldc,
                              const GemmBatch &bt) {
    static bool configured = false;  // the attribute is per function, set once
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(cgemm_simt_kernel<OPA, OPB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSimtSmemBytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    cgemm_simt_kernel<OPA, OPB><<<grid, 256, kSimtSmemBytes, s>>>(desc, m, n, k, alpha, A, lda, B,
                                                                  ldb, beta, C, ldc, bt);
    return cudaGetLastError();
}

template <int OPA>
cudaError_t launch_simt_tiles_b(int opB, dim3 grid, cudaStream_t s, const qcs_gemm_desc_t *desc,
                                int m, int n, int k, float2 alpha, const float2 *A, int64_t lda,
                                const float2 *B, int64_t ldb, float2 beta, float2 *C, int64_t ldc,
                                const GemmBatch &bt) {
    if (opB == QCS_OP_N)
        return launch_simt_tiles<OPA, QCS_OP_N>(grid, s, desc, m, n, k, alpha, A, lda, B, ldb,
                                                beta, C, ldc, bt);
    if (opB == QCS_OP_T)
        return launch_simt_tiles<OPA, QCS_OP_T>(grid, s, desc, m, n, k, alpha, A, lda, B, ldb,
                                                beta, C, ldc, bt);
    return launch_simt_tiles<OPA, QCS_OP_C>(grid, s, desc, m, n, k, alpha, A, lda, B, ldb, beta,
                                            C, ldc, bt);
}

// Small k with one small output side: the (2, 2^N, 2) and (2^N, 2, 2)
// shapes of Section 5.1.2.
//   rows: n <= 16, k <= KMAX: a thread per output row i keeps op(A)[i, :] in
//         KMAX registers and writes its n outputs (consecutive threads write
//         consecutive elements of each column of C).
//   cols: m <= 16, k <= 16: a thread per output element, i = lane bits below
//         log2(M2) (M2 = m rounded up to a power of two), j from the rest, so
//         that a warp writes C contiguously when ldc == m; op(B)[:, j] is read
//         by the M2 threads of column j (L1 broadcast).
template <int KMAX>
__global__ void __launch_bounds__(256) cgemm_skinny_rows_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int opA, int opB, int64_t m, int64_t n, int k,
    float2 alpha, const float2 *__restrict__ A, int64_t lda, const float2 *__restrict__ B,
    int64_t ldb, float2 beta, float2 *__restrict__ C, int64_t ldc, GemmBatch bt) {
    if (desc && desc->mode != QCS_MODE_FP32) return;
    A += blockIdx.y * bt.sA;
    B += blockIdx.y * bt.sB;
    C += blockIdx.y * bt.sC;
    const bool use_beta = (beta.x != 0.f) || (beta.y != 0.f);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 a[KMAX];
#pragma unroll
        for (int l = 0; l < KMAX; ++l) a[l] = (l < k) ? ld_op(A, opA, i, l, lda) : make_float2(0.f, 0.f);
        for (int64_t j = 0; j < n; ++j) {
            float sr = 0.f, si = 0.f;
#pragma unroll
            for (int l = 0; l < KMAX; ++l) {
                if (l < k) {
                    const float2 b = ld_op(B, opB, l, j, ldb);
                    sr = fmaf(a[l].x, b.x, sr);
                    sr = fmaf(-a[l].y, b.y, sr);
                    si = fmaf(a[l].x, b.y, si);
                    si = fmaf(a[l].y, b.x, si);
                }
            }
            float2 o;
            o.x = alpha.x * sr - alpha.y * si;
            o.y = alpha.x * si + alpha.y * sr;
            float2 *dst = C + i + j * ldc;
            if (use_beta) {
                const float2 c = *dst;
                o.x += beta.x * c.x - beta.y * c.y;
                o.y += beta.x * c.y + beta.y * c.x;
            }
            *dst = o;
        }
    }
}

// (2, n, 2) with op(B) = B stored 2 x n contiguous and C 2 x n contiguous
// (the (2, 2^N, 2) shape of Section 5.1.2): a thread per column, one 16-byte
// load of B's column and one 16-byte store of C's, four columns in flight.
__global__ void __launch_bounds__(256) cgemm_2x2_cols_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int opA, const float2 *__restrict__ A, int64_t lda,
    const float4 *__restrict__ B, float4 *__restrict__ C, int64_t n, float2 alpha, float2 beta,
    GemmBatch bt) {
    if (desc && desc->mode != QCS_MODE_FP32) return;
    A += blockIdx.y * bt.sA;
    B += blockIdx.y * (bt.sB >> 1);
    C += blockIdx.y * (bt.sC >> 1);
    const float2 a00 = ld_op(A, opA, 0, 0, lda), a01 = ld_op(A, opA, 0, 1, lda);
    const float2 a10 = ld_op(A, opA, 1, 0, lda), a11 = ld_op(A, opA, 1, 1, lda);
    const bool use_beta = (beta.x != 0.f) || (beta.y != 0.f);
    constexpr int U = 4;
    const int64_t S = (int64_t)gridDim.x * blockDim.x;
    auto cmul_add = [](float2 a, float2 b, float2 c, float2 d) {  // a b + c d
        float2 r;
        r.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, fmaf(c.x, d.x, -c.y * d.y)));
        r.y = fmaf(a.x, b.y, fmaf(a.y, b.x, fmaf(c.x, d.y, c.y * d.x)));
        return r;
    };
    for (int64_t j0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j0 < n; j0 += U * S) {
        float4 b[U], cold[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + u * S;
            if (j < n) {
                b[u] = __ldcs(B + j);
                if (use_beta) cold[u] = C[j];
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t j = j0 + u * S;
            if (j >= n) continue;
            const float2 b0 = make_float2(b[u].x, b[u].y), b1 = make_float2(b[u].z, b[u].w);
            const float2 s0 = cmul_add(a00, b0, a01, b1), s1 = cmul_add(a10, b0, a11, b1);
            float4 o;
            o.x = alpha.x * s0.x - alpha.y * s0.y;
            o.y = alpha.x * s0.y + alpha.y * s0.x;
            o.z = alpha.x * s1.x - alpha.y * s1.y;
            o.w = alpha.x * s1.y + alpha.y * s1.x;
            if (use_beta) {
                o.x += beta.x * cold[u].x - beta.y * cold[u].y;
                o.y += beta.x * cold[u].y + beta.y * cold[u].x;
                o.z += beta.x * cold[u].z - beta.y * cold[u].w;
                o.w += beta.x * cold[u].w + beta.y * cold[u].z;
            }
            __stcs(C + j, o);
        }
    }
}

// (m, 2, 2) with op(A) = A stored m x 2 and C m x 2, both with an even
// leading dimension and 16-byte aligned (the (2^N, 2, 2) shape of Section
// 5.1.2): a thread per pair of rows, one 16-byte load per column of A and
// one 16-byte store per column of C, four pairs in flight.  The arithmetic
// per output element is that of cgemm_skinny_rows_kernel (same FMA chain).
// An odd last row is done by the first thread of the grid.
__global__ void __launch_bounds__(256) cgemm_nx2x2_rows_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int opB, const float4 *__restrict__ A, int64_t lda2,
    const float2 *__restrict__ B, int64_t ldb, float4 *__restrict__ C, int64_t ldc2, int64_t m,
    float2 alpha, float2 beta, GemmBatch bt) {
    if (desc && desc->mode != QCS_MODE_FP32) return;
    A += blockIdx.y * (bt.sA >> 1);
    B += blockIdx.y * bt.sB;
    C += blockIdx.y * (bt.sC >> 1);
    float2 b[2][2];
#pragma unroll
    for (int l = 0; l < 2; ++l)
#pragma unroll
        for (int j = 0; j < 2; ++j) b[l][j] = ld_op(B, opB, l, j, ldb);
    const bool use_beta = (beta.x != 0.f) || (beta.y != 0.f);
    auto dot2 = [&](float2 a0, float2 a1, int j) {
        float sr = 0.f, si = 0.f;
        sr = fmaf(a0.x, b[0][j].x, sr);
        sr = fmaf(-a0.y, b[0][j].y, sr);
        si = fmaf(a0.x, b[0][j].y, si);
        si = fmaf(a0.y, b[0][j].x, si);
        sr = fmaf(a1.x, b[1][j].x, sr);
        sr = fmaf(-a1.y, b[1][j].y, sr);
        si = fmaf(a1.x, b[1][j].y, si);
        si = fmaf(a1.y, b[1][j].x, si);
        return make_float2(alpha.x * sr - alpha.y * si, alpha.x * si + alpha.y * sr);
    };
    auto add_beta = [&](float2 o, float2 c) {
        o.x += beta.x * c.x - beta.y * c.y;
        o.y += beta.x * c.y + beta.y * c.x;
        return o;
    };
    const int64_t pairs = m >> 1;
    constexpr int U = 4;
    const int64_t S = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p0 < pairs; p0 += U * S) {
        float4 a0[U], a1[U], c0[U], c1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t p = p0 + u * S;
            if (p < pairs) {
                a0[u] = __ldcs(A + p);
                a1[u] = __ldcs(A + lda2 + p);
                if (use_beta) {
                    c0[u] = C[p];
                    c1[u] = C[ldc2 + p];
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t p = p0 + u * S;
            if (p >= pairs) continue;
            // rows 2p (x, y of each float4) and 2p + 1 (z, w)
            const float2 r0a0 = make_float2(a0[u].x, a0[u].y), r0a1 = make_float2(a1[u].x, a1[u].y);
            const float2 r1a0 = make_float2(a0[u].z, a0[u].w), r1a1 = make_float2(a1[u].z, a1[u].w);
            float2 o00 = dot2(r0a0, r0a1, 0), o10 = dot2(r1a0, r1a1, 0);
            float2 o01 = dot2(r0a0, r0a1, 1), o11 = dot2(r1a0, r1a1, 1);
            if (use_beta) {
                o00 = add_beta(o00, make_float2(c0[u].x, c0[u].y));
                o10 = add_beta(o10, make_float2(c0[u].z, c0[u].w));
                o01 = add_beta(o01, make_float2(c1[u].x, c1[u].y));
                o11 = add_beta(o11, make_float2(c1[u].z, c1[u].w));
            }
            __stcs(C + p, make_float4(o00.x, o00.y, o10.x, o10.y));
            __stcs(C + ldc2 + p, make_float4(o01.x, o01.y, o11.x, o11.y));
        }
    }
    if ((m & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        const float2 *Af = reinterpret_cast<const float2 *>(A);
        float2 *Cf = reinterpret_cast<float2 *>(C);
        const int64_t i = m - 1;
        const float2 ra0 = Af[i], ra1 = Af[2 * lda2 + i];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            float2 o = dot2(ra0, ra1, j);
            float2 *dst = Cf + i + j * (2 * ldc2);
            if (use_beta) o = add_beta(o, *dst);
            *dst = o;
        }
    }
}

__global__ void __launch_bounds__(256) cgemm_skinny_cols_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int opA, int opB, int64_t m, int64_t n, int k,
    int lg_m2, float2 alpha, const float2 *__restrict__ A, int64_t lda, const float2 *__restrict__ B,
    int64_t ldb, float2 beta, float2 *__restrict__ C, int64_t ldc, GemmBatch bt) {
    if (desc && desc->mode != QCS_MODE_FP32) return;
    A += blockIdx.y * bt.sA;
    B += blockIdx.y * bt.sB;
    C += blockIdx.y * bt.sC;
    const bool use_beta = (beta.x != 0.f) || (beta.y != 0.f);
    const int64_t total = n << lg_m2;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = t & ((int64_t(1) << lg_m2) - 1), j = t >> lg_m2;
        if (i >= m) continue;
        float sr = 0.f, si = 0.f;
        for (int l = 0; l < k; ++l) {
            const float2 a = ld_op(A, opA, i, l, lda);
            const float2 b = ld_op(B, opB, l, j, ldb);
            sr = fmaf(a.x, b.x, sr);
            sr = fmaf(-a.y, b.y, sr);
            si = fmaf(a.x, b.y, si);
            si = fmaf(a.y, b.x, si);
        }
        float2 o;
        o.x = alpha.x * sr - alpha.y * si;
        o.y = alpha.x * si + alpha.y * sr;
        float2 *dst = C + i + j * ldc;
        if (use_beta) {
            const float2 c = *dst;
            o.x += beta.x * c.x - beta.y * c.y;
            o.y += beta.x * c.y + beta.y * c.x;
        }
        *dst = o;
    }
}

// One thread per output element on a 2-D grid (x: rows, consecutive threads
// write consecutive elements of a column-major C; y: columns), k loop in the
// thread: small k with both output sides large, or small outputs with
// moderate k.
__global__ void __launch_bounds__(256) cgemm_perelem_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int opA, int opB, int64_t m, int64_t n, int64_t k,
    float2 alpha, const float2 *__restrict__ A, int64_t lda, const float2 *__restrict__ B,
    int64_t ldb, float2 beta, float2 *__restrict__ C, int64_t ldc, GemmBatch bt) {
    if (desc && desc->mode != QCS_MODE_FP32) return;
    A += blockIdx.z * bt.sA;
    B += blockIdx.z * bt.sB;
    C += blockIdx.z * bt.sC;
    const bool use_beta = (beta.x != 0.f) || (beta.y != 0.f);
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        float sr = 0.f, si = 0.f;
        for (int64_t l = 0; l < k; ++l) {
            const float2 a = ld_op(A, opA, i, l, lda);
            const float2 b = ld_op(B, opB, l, j, ldb);
            sr = fmaf(a.x, b.x, sr);
            sr = fmaf(-a.y, b.y, sr);
            si = fmaf(a.x, b.y, si);
            si = fmaf(a.y, b.x, si);
        }
        float2 o;
        o.x = alpha.x * sr - alpha.y * si;
        o.y = alpha.x * si + alpha.y * sr;
        float2 *dst = C + i + j * ldc;
        if (use_beta) {
            const float2 c = *dst;
            o.x += beta.x * c.x - beta.y * c.y;
            o.y += beta.x * c.y + beta.y * c.x;
        }
        *dst = o;
    }
}

// Small k (<= KMAX <= 16) with both output sides large -- the contraction
// of a tensor with a gate or a few-index tensor: a block owns R rows
// (R = 256 / lanes, the rows of op(A) kept in registers) and a chunk of
// kSmallKCols columns, whose op(B) values it stages in shared memory; each
// thread then produces the outputs of its row for every lanes-th column of
// the chunk.  C is written column by column, R consecutive rows at a time.
constexpr int kSmallKCols = 64;

template <int KMAX>
__global__ void __launch_bounds__(256) cgemm_smallk_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int opA, int opB, int64_t m, int64_t n, int k,
    int rows, float2 alpha, const float2 *__restrict__ A, int64_t lda,
    const float2 *__restrict__ B, int64_t ldb, float2 beta, float2 *__restrict__ C, int64_t ldc,
    GemmBatch bt) {
    if (desc && desc->mode != QCS_MODE_FP32) return;
    A += blockIdx.z * bt.sA;
    B += blockIdx.z * bt.sB;
    C += blockIdx.z * bt.sC;
    __shared__ float2 sb[kSmallKCols][KMAX + 1];
    const int64_t j0 = (int64_t)blockIdx.y * kSmallKCols;
    const int jn = (int)min((int64_t)kSmallKCols, n - j0);
    for (int t = threadIdx.x; t < kSmallKCols * KMAX; t += blockDim.x) {
        const int jj = t / KMAX, l = t - jj * KMAX;
        float2 v = make_float2(0.f, 0.f);
        if (l < k && jj < jn) v = ld_op(B, opB, l, j0 + jj, ldb);
        sb[jj][l] = v;
    }
    const int r = threadIdx.x % rows, lane_c = threadIdx.x / rows, lanes = blockDim.x / rows;
    const int64_t i = (int64_t)blockIdx.x * rows + r;
    float2 a[KMAX];
#pragma unroll
    for (int l = 0; l < KMAX; ++l)
        a[l] = (i < m && l < k) ? ld_op(A, opA, i, l, lda) : make_float2(0.f, 0.f);
    __syncthreads();
    if (i >= m) return;
    const bool use_beta = (beta.x != 0.f) || (beta.y != 0.f);
    for (int jj = lane_c; jj < jn; jj += lanes) {
        float sr = 0.f, si = 0.f;
#pragma unroll
        for (int l = 0; l < KMAX; ++l) {
            const float2 b = sb[jj][l];
            sr = fmaf(a[l].x, b.x, sr);
            sr = fmaf(-a[l].y, b.y, sr);
            si = fmaf(a[l].x, b.y, si);
            si = fmaf(a[l].y, b.x, si);
        }
        float2 o;
        o.x = alpha.x * sr - alpha.y * si;
        o.y = alpha.x * si + alpha.y * sr;
        float2 *dst = C + i + (j0 + jj) * ldc;
        if (use_beta) {
            const float2 c = *dst;
            o.x += beta.x * c.x - beta.y * c.y;
            o.y += beta.x * c.y + beta.y * c.x;
        }
        *dst = o;
    }
}

// Split-K for small m*n with long k (the end of a contraction tree reduces
// large tensors to a few numbers): warp w handles output o = w mod (m n) over
// the w-th k chunk; lanes stride along k, a warp shuffle reduces, and the
// partial goes to part[chunk * m n + o].  cgemm_splitk_reduce then adds the
// chunks in order (deterministic) and applies alpha/beta.
__global__ void __launch_bounds__(256) cgemm_splitk_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int opA, int opB, int64_t m, int64_t n, int64_t k,
    int64_t chunk, int64_t chunks, const float2 *__restrict__ A, int64_t lda,
    const float2 *__restrict__ B, int64_t ldb, float2 *__restrict__ part, GemmBatch bt) {
    if (desc && desc->mode != QCS_MODE_FP32) return;
    const int64_t mn = m * n;
    A += blockIdx.y * bt.sA;
    B += blockIdx.y * bt.sB;
    part += blockIdx.y * chunks * mn;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= mn * chunks) return;
    const int64_t o = w % mn, c = w / mn;
    const int64_t i = o % m, j = o / m;
    const int64_t l0 = c * chunk, l1 = min(k, l0 + chunk);
    float sr = 0.f, si = 0.f;
    for (int64_t l = l0 + lane; l < l1; l += 32) {
        const float2 a = ld_op(A, opA, i, l, lda);
        const float2 b = ld_op(B, opB, l, j, ldb);
        sr = fmaf(a.x, b.x, sr);
        sr = fmaf(-a.y, b.y, sr);
        si = fmaf(a.x, b.y, si);
        si = fmaf(a.y, b.x, si);
    }
    for (int off = 16; off > 0; off >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, off);
        si += __shfl_xor_sync(0xffffffffu, si, off);
    }
    if (lane == 0) part[c * mn + o] = make_float2(sr, si);
}

// One block per output: thread t adds chunks t, t + 256, ... in order, then a
// fixed shared-memory tree adds the 256 sums, so the result does not depend
// on scheduling.
__global__ void __launch_bounds__(256) cgemm_splitk_reduce(
    const qcs_gemm_desc_t *__restrict__ desc, int64_t m, int64_t n, int64_t chunks,
    const float2 *__restrict__ part, float2 alpha, float2 beta, float2 *__restrict__ C,
    int64_t ldc, GemmBatch bt) {
    if (desc && desc->mode != QCS_MODE_FP32) return;
    __shared__ float2 red[256];
    const int64_t mn = m * n;
    C += blockIdx.y * bt.sC;
    part += blockIdx.y * chunks * mn;
    const int64_t o = blockIdx.x;
    float sr = 0.f, si = 0.f;
    for (int64_t c = threadIdx.x; c < chunks; c += 256) {
        const float2 v = part[c * mn + o];
        sr += v.x;
        si += v.y;
    }
    red[threadIdx.x] = make_float2(sr, si);
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const float2 a = red[threadIdx.x], b = red[threadIdx.x + w];
            red[threadIdx.x] = make_float2(a.x + b.x, a.y + b.y);
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    sr = red[0].x;
    si = red[0].y;
    const int64_t i = o % m, j = o / m;
    float2 r;
    r.x = alpha.x * sr - alpha.y * si;
    r.y = alpha.x * si + alpha.y * sr;
    float2 *dst = C + i + j * ldc;
    if ((beta.x != 0.f) || (beta.y != 0.f)) {
        const float2 cv = *dst;
        r.x += beta.x * cv.x - beta.y * cv.y;
        r.y += beta.x * cv.y + beta.y * cv.x;
    }
    *dst = r;
}

}  // namespace

cudaError_t launch_cgemm_simt(const qcs_gemm_desc_t *desc, int opA, int opB, int64_t m,
                              int64_t n, int64_t k, float2 alpha, const float2 *A, int64_t lda,
                              const float2 *B, int64_t ldb, float2 beta, float2 *C, int64_t ldc,
                              float2 *splitk, cudaStream_t s, const GemmBatch &bt) {
    if (m == 0 || n == 0) return cudaSuccess;
    if (bt.count < 1 || bt.count > 65535) return cudaErrorInvalidValue;
    const unsigned G = (unsigned)bt.count;
    const int64_t mn = m * n;
    if (splitk && mn <= kSplitKMaxOutputs && k >= 1024) {
        // enough warps to fill the GPU, at least 256 k values per warp; the
        // buffer holds kSplitKMaxPartials partials per batch entry, so the
        // chunking (and the result) does not depend on the batch
        int64_t chunks = kSplitKMaxPartials / mn;
        chunks = std::min<int64_t>(chunks, (k + 255) / 256);
        chunks = std::max<int64_t>(chunks, 1);
        const int64_t chunk = (k + chunks - 1) / chunks;
        chunks = (k + chunk - 1) / chunk;
        const int64_t warps = mn * chunks;
        const int64_t blocks = (warps * 32 + 255) / 256;
        cgemm_splitk_kernel<<<dim3((unsigned)blocks, G), 256, 0, s>>>(
            desc, opA, opB, m, n, k, chunk, chunks, A, lda, B, ldb, splitk, bt);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        cgemm_splitk_reduce<<<dim3((unsigned)mn, G), 256, 0, s>>>(desc, m, n, chunks, splitk, alpha,
                                                                  beta, C, ldc, bt);
        return cudaGetLastError();
    }
    if (k <= 16 && (m <= 16 || n <= 16)) {
        if (m >= n && n == 2 && k == 2 && opA == QCS_OP_N && lda % 2 == 0 && ldc % 2 == 0 &&
            ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(C)) & 15u) == 0 &&
            (bt.sA % 2) == 0 && (bt.sC % 2) == 0) {
            const int64_t blocks = (m / 2 + 4 * 256 - 1) / (4 * 256);
            const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, 65535)), G);
            cgemm_nx2x2_rows_kernel<<<grid, 256, 0, s>>>(
                desc, opB, reinterpret_cast<const float4 *>(A), lda / 2, B, ldb,
                reinterpret_cast<float4 *>(C), ldc / 2, m, alpha, beta, bt);
        } else if (m >= n) {  // then n <= 16: a thread per row
            const int64_t blocks = (m + 255) / 256;
            const dim3 grid((unsigned)(blocks < 65536 ? blocks : 65536), G);
            const int kk = (int)k;
            if (kk <= 2)
                cgemm_skinny_rows_kernel<2><<<grid, 256, 0, s>>>(desc, opA, opB, m, n, kk, alpha, A,
                                                                lda, B, ldb, beta, C, ldc, bt);
            else if (kk <= 4)
                cgemm_skinny_rows_kernel<4><<<grid, 256, 0, s>>>(desc, opA, opB, m, n, kk, alpha, A,
                                                                lda, B, ldb, beta, C, ldc, bt);
            else if (kk <= 8)
                cgemm_skinny_rows_kernel<8><<<grid, 256, 0, s>>>(desc, opA, opB, m, n, kk, alpha, A,
                                                                lda, B, ldb, beta, C, ldc, bt);
            else
                cgemm_skinny_rows_kernel<16><<<grid, 256, 0, s>>>(desc, opA, opB, m, n, kk, alpha, A,
                                                                 lda, B, ldb, beta, C, ldc, bt);
        } else if (m == 2 && k == 2 && opB == QCS_OP_N && ldb == 2 && ldc == 2 &&
                   ((reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15u) == 0 &&
                   (bt.sB % 2) == 0 && (bt.sC % 2) == 0) {
            const int64_t blocks = (n + 4 * 256 - 1) / (4 * 256);
            const dim3 grid((unsigned)(blocks < 65536 ? blocks : 65536), G);
            cgemm_2x2_cols_kernel<<<grid, 256, 0, s>>>(
                desc, opA, A, lda, reinterpret_cast<const float4 *>(B), reinterpret_cast<float4 *>(C),
                n, alpha, beta, bt);
        } else {  // m <= 16: a thread per element, rows in the low bits
            int lg = 0;
            while ((int64_t(1) << lg) < m) ++lg;
            const int64_t total = n << lg;
            const int64_t blocks = (total + 255) / 256;
            const dim3 grid((unsigned)(blocks < 65536 ? blocks : 65536), G);
            cgemm_skinny_cols_kernel<<<grid, 256, 0, s>>>(desc, opA, opB, m, n, (int)k, lg, alpha, A,
                                                          lda, B, ldb, beta, C, ldc, bt);
        }
        return cudaGetLastError();
    }
    // 16 < k <= 32 with m too small for the 128-row SIMT tile (half of it or
    // more would stay empty): the small-k kernel below with 32 registers of k
    if (k > 16 && k <= 32 && m <= 64 && mn > 4096) {
        const int rows = m <= 32 ? 32 : 64;
        const int64_t gy = (n + kSmallKCols - 1) / kSmallKCols;
        if (gy <= 65535) {
            dim3 grid(1u, (unsigned)gy, G);
            cgemm_smallk_kernel<32><<<grid, 256, 0, s>>>(desc, opA, opB, m, n, (int)k, rows, alpha,
                                                         A, lda, B, ldb, beta, C, ldc, bt);
            return cudaGetLastError();
        }
    }
    if (k <= 16 && mn > 4096 && m <= INT32_MAX) {
        // rows per block: all of m up to 256, at least a warp
        const int rows = m >= 256 ? 256 : (m <= 32 ? 32 : (m <= 64 ? 64 : (m <= 128 ? 128 : 256)));
        const int64_t gy = (n + kSmallKCols - 1) / kSmallKCols;
        const int64_t gx = (m + rows - 1) / rows;
        if (gy <= 65535 && gx <= INT32_MAX) {
            dim3 grid((unsigned)gx, (unsigned)gy, G);
            if (k <= 4)
                cgemm_smallk_kernel<4><<<grid, 256, 0, s>>>(desc, opA, opB, m, n, (int)k, rows, alpha,
                                                            A, lda, B, ldb, beta, C, ldc, bt);
            else if (k <= 8)
                cgemm_smallk_kernel<8><<<grid, 256, 0, s>>>(desc, opA, opB, m, n, (int)k, rows, alpha,
                                                            A, lda, B, ldb, beta, C, ldc, bt);
            else
                cgemm_smallk_kernel<16><<<grid, 256, 0, s>>>(desc, opA, opB, m, n, (int)k, rows,
                                                             alpha, A, lda, B, ldb, beta, C, ldc, bt);
            return cudaGetLastError();
        }
    }
    const bool perelem = (k <= 16) || (mn <= 4096);
    if (perelem || m > INT32_MAX || n > INT32_MAX || k > INT32_MAX) {
        const int64_t bx = (m + 255) / 256;
        if (bx > INT32_MAX) return cudaErrorInvalidValue;
        dim3 grid((unsigned)bx, (unsigned)(n < 65535 ? n : 65535), G);
        cgemm_perelem_kernel<<<grid, 256, 0, s>>>(desc, opA, opB, m, n, k, alpha, A, lda, B, ldb,
                                                  beta, C, ldc, bt);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((n + kSBN - 1) / kSBN), (unsigned)((m + kSBM - 1) / kSBM), G);
    if (grid.y > 65535u) return cudaErrorInvalidValue;
    auto launch = opA == QCS_OP_N   ? launch_simt_tiles_b<QCS_OP_N>
                  : opA == QCS_OP_T ? launch_simt_tiles_b<QCS_OP_T>
                                    : launch_simt_tiles_b<QCS_OP_C>;
    return launch(opB, grid, s, desc, (int)m, (int)n, (int)k, alpha, A, lda, B, ldb, beta, C, ldc,
                  bt);
}

// ===========================================================================
// Plain FP32 real GEMM (the FP32 mode of qcs_sgemm and its AUTO candidate)
// ===========================================================================

namespace {

constexpr int kRT = 128;    // output rows and columns of a tile
constexpr int kRK = 16;     // k per shared-memory stage
constexpr int kRStages = 3;
constexpr int kRPad = 132;  // row length of a shared tile (16-byte rows; transposed copies spread over banks)
constexpr size_t kRSmemBytes = sizeof(float) * 2 * kRStages * kRK * kRPad;

// 16-byte asynchronous copy to shared memory (both addresses 16-byte aligned)
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)),
                 "l"(reinterpret_cast<uint64_t>(src))
                 : "memory");
}

// C = alpha op(A) op(B) + beta C on the CUDA cores: 128 x 128 tiles, 256
// threads with 8 x 8 outputs each (rows 4t..4t+3 and 64+4t..64+4t+3 of the
// tile, likewise columns).  Operand tiles of 16 k move to shared memory with
// 4-byte cp.async copies (zero-filled outside the matrix) in a three-stage
// ring, unchecked for tiles inside the matrix except in the last k-tile;
// TA / TB: op(A) / op(B) is op T (op C acts as op T on real matrices).
// Runs only when the descriptor selected FP32 (always when desc is NULL).
// Tiles in y are walked in a grid-stride loop.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256, 2) sgemm_simt_kernel(
    const qcs_gemm_desc_t *__restrict__ desc, int64_t m, int64_t n, int64_t k, float alpha,
    const float *__restrict__ A, int64_t lda, const float *__restrict__ B, int64_t ldb, float beta,
    float *__restrict__ C, int64_t ldc) {
    if (desc && desc->mode != QCS_MODE_FP32) return;
    extern __shared__ __align__(16) unsigned char sgemm_smem[];
    float (*As)[kRK][kRPad] = reinterpret_cast<float (*)[kRK][kRPad]>(sgemm_smem);
    float (*Bs)[kRK][kRPad] =
        reinterpret_cast<float (*)[kRK][kRPad]>(sgemm_smem + sizeof(float) * kRStages * kRK * kRPad);
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    // copy assignment: op N of A: i = tid % 128, l = tid / 128 + 2 q; op T:
    // l = tid % 16, i = tid / 16 + 16 q (q < 8); op N of B: l = tid % 16,
    // j = tid / 16 + 16 q; op T: j = tid % 128, l = tid / 128 + 2 q
    const int aI = TA ? (tid >> 4) : (tid & (kRT - 1));
    const int aL = TA ? (tid & (kRK - 1)) : (tid >> 7);
    const int bJ = TB ? (tid & (kRT - 1)) : (tid >> 4);
    const int bL = TB ? (tid >> 7) : (tid & (kRK - 1));
    const int64_t a_kstep = TA ? kRK : kRK * lda, a_qstep = TA ? 16 * lda : 2 * lda;
    const int64_t b_kstep = TB ? kRK * ldb : kRK, b_qstep = TB ? 2 * ldb : 16 * ldb;
    const int64_t i0 = static_cast<int64_t>(blockIdx.x) * kRT;
    const int64_t tiles_n = (n + kRT - 1) / kRT;
    const int ktiles = (int)((k + kRK - 1) / kRK);
    for (int64_t tj = blockIdx.y; tj < tiles_n; tj += gridDim.y) {
        const int64_t j0 = tj * kRT;
        const float *a_base = A + (TA ? aL + (i0 + aI) * lda : i0 + aI + aL * lda);
        const float *b_base = B + (TB ? j0 + bJ + bL * ldb : bL + (j0 + bJ) * ldb);
        uint32_t a_mask = 0, b_mask = 0;  // bit q: copy q's row (column) lies inside the matrix
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            a_mask |= uint32_t(i0 + aI + (TA ? 16 * q : 0) < m) << q;
            b_mask |= uint32_t(j0 + bJ + (TB ? 0 : 16 * q) < n) << q;
        }
        const bool interior = i0 + kRT <= m && j0 + kRT <= n;
        // operands contiguous along the shared tile's rows (op(A) N, op(B) T)
        // with 16-byte aligned columns move in 16-byte copies inside the matrix
        const bool a16 = !TA && interior && lda % 4 == 0 &&
                         (reinterpret_cast<uintptr_t>(A) & 15u) == 0;
        const bool b16 = TB && interior && ldb % 4 == 0 &&
                         (reinterpret_cast<uintptr_t>(B) & 15u) == 0;
        auto load_tile = [&](int st, int kt) {
            const int64_t k0 = static_cast<int64_t>(kt) * kRK;
            const bool tail = k0 + kRK > k;
            if (a16 && !tail) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int c = tid + 256 * q, i = 4 * (c & 31), l = c >> 5;
                    cp_async16(&As[st][l][i], A + (i0 + i) + (k0 + l) * lda);
                }
            } else {
                const float *pa = a_base + kt * a_kstep;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int l = TA ? aL : aL + 2 * q;
                    const int i = TA ? aI + 16 * q : aI;
                    bool ok = true;
                    if (!interior || tail) ok = ((a_mask >> q) & 1u) && k0 + l < k;
                    cp_async4(&As[st][l][i], ok ? pa + q * a_qstep : A, ok ? 4u : 0u);
                }
            }
            if (b16 && !tail) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int c = tid + 256 * q, j = 4 * (c & 31), l = c >> 5;
                    cp_async16(&Bs[st][l][j], B + (j0 + j) + (k0 + l) * ldb);
                }
            } else {
                const float *pb = b_base + kt * b_kstep;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int l = TB ? bL + 2 * q : bL;
                    const int j = TB ? bJ : bJ + 16 * q;
                    bool ok = true;
                    if (!interior || tail) ok = ((b_mask >> q) & 1u) && k0 + l < k;
                    cp_async4(&Bs[st][l][j], ok ? pb + q * b_qstep : B, ok ? 4u : 0u);
                }
            }
        };
        float acc[8][8];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
        __syncthreads();  // the previous tile's readers are done with the ring
        if (ktiles > 0) load_tile(0, 0);
        cp_async_commit();
        if (ktiles > 1) load_tile(1, 1);
        cp_async_commit();
        for (int kt = 0; kt < ktiles; ++kt) {
            cp_async_wait<1>();  // every group but the newest has landed: k-tile kt
            __syncthreads();     // ... for all threads; and slot (kt + 2) % 3 is free
            if (kt + 2 < ktiles) load_tile((kt + 2) % kRStages, kt + 2);
            cp_async_commit();
            const int st = kt % kRStages;
#pragma unroll
            for (int kk = 0; kk < kRK; ++kk) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&As[st][kk][tx * 4]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&As[st][kk][64 + tx * 4]);
                const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[st][kk][ty * 4]);
                const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[st][kk][64 + ty * 4]);
                const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
            }
        }
        cp_async_wait<0>();
        const bool vec = ((reinterpret_cast<uintptr_t>(C) & 15u) == 0) && (ldc % 4 == 0);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int64_t col = j0 + (c < 4 ? ty * 4 + c : 64 + ty * 4 + (c - 4));
            if (col >= n) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t row = i0 + h * 64 + tx * 4;
                float *dst = C + col * ldc + row;
                float v[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) v[r] = alpha * acc[h * 4 + r][c];
                if (vec && row + 3 < m) {
                    if (beta != 0.0f) {
                        const float4 o = *reinterpret_cast<const float4 *>(dst);
                        v[0] = fmaf(beta, o.x, v[0]);
                        v[1] = fmaf(beta, o.y, v[1]);
                        v[2] = fmaf(beta, o.z, v[2]);
                        v[3] = fmaf(beta, o.w, v[3]);
                    }
                    *reinterpret_cast<float4 *>(dst) = make_float4(v[0], v[1], v[2], v[3]);
                } else {
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        if (row + r < m) {
                            float o = v[r];
                            if (beta != 0.0f) o = fmaf(beta, dst[r], o);
                            dst[r] = o;
                        }
                    }
                }
            }
        }
    }
}

template <bool TA, bool TB>
cudaError_t launch_sgemm_tiles(dim3 grid, cudaStream_t s, const qcs_gemm_desc_t *desc, int64_t m,
                               int64_t n, int64_t k, float alpha, const float *A, int64_t lda,
                               const float *B, int64_t ldb, float beta, float *C, int64_t ldc) {
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(sgemm_simt_kernel<TA, TB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kRSmemBytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    sgemm_simt_kernel<TA, TB><<<grid, 256, kRSmemBytes, s>>>(desc, m, n, k, alpha, A, lda, B, ldb,
                                                             beta, C, ldc);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sgemm_simt(const qcs_gemm_desc_t *desc, int opA, int opB, int64_t m,
                              int64_t n, int64_t k, float alpha, const float *A, int64_t lda,
                              const float *B, int64_t ldb, float beta, float *C, int64_t ldc,
                              cudaStream_t s) {
    if (m == 0 || n == 0) return cudaSuccess;
    const int64_t gx = (m + kRT - 1) / kRT, gy = (n + kRT - 1) / kRT;
    if (gx > INT32_MAX) return cudaErrorInvalidValue;
    dim3 grid((unsigned)gx, (unsigned)(gy < 65535 ? gy : 65535));
    const bool ta = opA != QCS_OP_N, tb = opB != QCS_OP_N;
    auto launch = ta ? (tb ? launch_sgemm_tiles<true, true> : launch_sgemm_tiles<true, false>)
                     : (tb ? launch_sgemm_tiles<false, true> : launch_sgemm_tiles<false, false>);
    return launch(grid, s, desc, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
}

}  // namespace qcs
