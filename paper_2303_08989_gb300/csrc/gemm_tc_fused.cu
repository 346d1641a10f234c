// TF32X CGEMM with the Eq. 1 split fused into the shared-memory staging
// (Section 2.1, Eq. 1; Section 3), for sm_103a.
//
// The two-pass TF32X path splits op(A) and op(B) into hi / lo TF32 planes in
// HBM (split_kernel: 8 bytes read, 16 / 20 bytes written per complex
// element) and the tensor-core kernel reads the planes back through TMA.
// Here the planes never leave the SM: the TMA producer loads the caller's
// complex64 tiles as they are stored, and the eight epilogue warps, which
// only drain an accumulator every DRAIN stages, spend the rest of the K loop
// converting each raw stage into the same four (op(A)) and five (op(B))
// 64-byte-swizzled TF32 planes that a TMA load of the split planes would
// have produced.  The MMA issuer and the accumulator drains are those of
// cgemm_tc_kernel's TF32 instantiation, stage for stage, so the result is
// bit-identical to the two-pass path.  TF32 has FP32's exponent range, so
// no scaling is involved (the descriptor's sA = sB = 0).
//
// Roles (one CTA per SM, persistent over 128 x 128 complex tiles):
//   warp 0     TMA producer: per stage one box of 128 rows x 16 complex of
//              op(A) and of op(B) into a two-slot raw ring (16 KB each).
//              Boxes whose rows are K-contiguous (op T / op C of A, op N of
//              B) use the 128-byte swizzle, the others (M- or N-contiguous)
//              none; out-of-range elements arrive as zeros.
//   warp 1     MMA issuer: as cgemm_tc_kernel<TF32> on a two-slot ring of
//              converted stages (72 KB each).
//   warps 2-9  converters and epilogue: per stage, 32 warp-rows of four
//              consecutive k (A and B) each -> hi = tf32(x), lo =
//              tf32((x - hi) 2^11) into the planes; before each stage, the
//              acc0 drains that are due (forced once the MMA would otherwise
//              wait for them; earlier when acc0 is already complete); at the
//              end of a tile the last drain with acc1 and the alpha / beta
//              epilogue.
// Shared memory: 2 x 72 KB converted + 4 x 16 KB raw = 208 KB.
//
// Limits (checked by the caller): one GEMM per launch, one K range, lda and
// ldb even and A, B 16-byte aligned (TMA strides and base), DRAIN = 4.
#include <cuda_fp16.h>

#include "internal.h"
#include "ptx.cuh"

namespace qcs {

namespace {

constexpr int kFDrain = 4;
constexpr int kFRaw = 2, kFConv = 2;
constexpr int kFK = 16;                         // complex k per stage (two TF32 MMA K steps)
constexpr int kFRawBytes = kBM * kFK * 8;       // 16 KB: 128 rows x 16 complex
constexpr int kFConvBytes = kAStageBytes + kBStageBytes;  // 72 KB
constexpr int kFEpiCols = kBN / 2;
constexpr int kEpiWarpsFused = 8;

struct FusedSmem {
    uint8_t conv[kFConv][kFConvBytes];
    uint8_t rawA[kFRaw][kFRawBytes];
    uint8_t rawB[kFRaw][kFRawBytes];
    uint64_t raw_full[kFRaw], raw_empty[kFRaw];
    uint64_t conv_full[kFConv], conv_empty[kFConv];
    uint64_t acc0_full, acc0_empty, drain;
    uint32_t tmem_base;
    int abort;
};

__device__ __forceinline__ void ftile_coords(int t, int tiles_m, int tiles_n, int group_m, int &tm,
                                             int &tn) {
    const int per_group = group_m * tiles_n;
    const int g = t / per_group;
    const int first_m = g * group_m;
    const int gsize = min(tiles_m - first_m, group_m);
    const int r = t - g * per_group;
    tm = first_m + r % gsize;
    tn = r / gsize;
}

__device__ __forceinline__ void fraise_abort(FusedSmem &S, int *d_err, int code) {
    *reinterpret_cast<volatile int *>(&S.abort) = 1;
    atomicCAS(d_err, 0, code);
}

// Four consecutive k (complex) of row r of a raw tile.  kfast: rows are 128
// K-contiguous bytes with the 128-byte swizzle (16-byte chunk c of row r at
// c ^ (r % 8)); otherwise the tile is [k][128 rows] of 8-byte elements.
template <bool KFAST>
__device__ __forceinline__ void load_quad(const uint8_t *raw, int r, int c4, float2 (&v)[4]) {
    if (KFAST) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int chunk = (2 * c4 + h) ^ (r & 7);
            const float4 t = *reinterpret_cast<const float4 *>(raw + r * 128 + chunk * 16);
            v[2 * h] = make_float2(t.x, t.y);
            v[2 * h + 1] = make_float2(t.z, t.w);
        }
    } else {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            v[e] = *reinterpret_cast<const float2 *>(raw + (4 * c4 + e) * (kBM * 8) + r * 8);
    }
}

// Eq. 1 on four complex values, into the planes of row r, 16-byte chunk c4
// (the 64-byte swizzle: chunk c4 of row r at c4 ^ ((r / 2) % 4)).  op(A):
// hi.re, hi.im, lo.re, lo.im; op(B): -hi.im, hi.re, hi.im, lo.re, lo.im.
template <bool B_OPERAND>
__device__ __forceinline__ void split_quad(const float2 (&v)[4], bool conj, uint8_t *planes, int r,
                                           int c4) {
    uint32_t hr[4], hi[4], lr[4], li[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const float re = v[e].x, im = conj ? -v[e].y : v[e].y;
        hr[e] = tf32_rn(re);
        lr[e] = tf32_rn((re - __uint_as_float(hr[e])) * 2048.0f);
        hi[e] = tf32_rn(im);
        li[e] = tf32_rn((im - __uint_as_float(hi[e])) * 2048.0f);
    }
    uint8_t *p = planes + r * 64 + ((c4 ^ ((r >> 1) & 3)) << 4);
    int pl = 0;
    if (B_OPERAND)
        *reinterpret_cast<uint4 *>(p + (pl++) * kTileBytes) =
            make_uint4(hi[0] ^ 0x80000000u, hi[1] ^ 0x80000000u, hi[2] ^ 0x80000000u,
                       hi[3] ^ 0x80000000u);
    *reinterpret_cast<uint4 *>(p + (pl++) * kTileBytes) = make_uint4(hr[0], hr[1], hr[2], hr[3]);
    *reinterpret_cast<uint4 *>(p + (pl++) * kTileBytes) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4 *>(p + (pl++) * kTileBytes) = make_uint4(lr[0], lr[1], lr[2], lr[3]);
    *reinterpret_cast<uint4 *>(p + pl * kTileBytes) = make_uint4(li[0], li[1], li[2], li[3]);
}

// TA: op(A) is op T / op C (raw A rows K-contiguous); TB: op(B) is op T /
// op C (raw B rows N-contiguous, i.e. not K-contiguous).
template <bool TA, bool TB>
__global__ void __launch_bounds__(kTcThreads, 1)
    cgemm_tc_fused_kernel(const __grid_constant__ CUtensorMap mapA,
                          const __grid_constant__ CUtensorMap mapB,
                          const qcs_gemm_desc_t *__restrict__ desc, int m, int n, int k_pad,
                          int conjA, int conjB, float2 alpha, float2 beta, float2 *__restrict__ C,
                          int64_t ldc, int *d_err, int group_m, const TcWork w) {
    if (desc->mode != QCS_MODE_TF32X) return;
    extern __shared__ uint8_t smem_raw[];
    FusedSmem &S = *reinterpret_cast<FusedSmem *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    volatile int *abort_flag = &S.abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kFRaw; ++s) {
            mbar_init(&S.raw_full[s], 1);
            mbar_init(&S.raw_empty[s], kEpiWarpsFused);
        }
        for (int s = 0; s < kFConv; ++s) {
            mbar_init(&S.conv_full[s], kEpiWarpsFused);
            mbar_init(&S.conv_empty[s], 1);
        }
        mbar_init(&S.acc0_full, 1);
        mbar_init(&S.acc0_empty, kEpiWarpsFused);
        mbar_init(&S.drain, 1);
        S.abort = 0;
        fence_barrier_init();
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
    }
    if (warp == 1) {
        tmem_alloc(&S.tmem_base, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;

    const int tiles_m = (m + kBM - 1) / kBM;
    const int tiles_n = (n + kBN - 1) / kBN;
    const int num_tiles = tiles_m * tiles_n;
    const int nkb = k_pad / kFK;

    if (warp == 0) {
        // ---------------- TMA producer (raw complex64 tiles) ----------------
        if (lane == 0) {
            int rs = 0;
            uint32_t rph = 0;
            int issued = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < num_tiles && ok && !w.stall; t += gridDim.x) {
                int tm, tn;
                ftile_coords(t, tiles_m, tiles_n, group_m, tm, tn);
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&S.raw_empty[rs], rph ^ 1u, globaltimer_ns() + w.wait_ns,
                                   abort_flag)) {
                        if (!*abort_flag) fraise_abort(S, d_err, kErrTimeoutProducer);
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&S.raw_full[rs], 2 * kFRawBytes);
                    const int k0 = kb * kFK;
                    if (TA)
                        tma_load_2d(S.rawA[rs], &mapA, &S.raw_full[rs], k0, tm * kBM);
                    else
                        tma_load_2d(S.rawA[rs], &mapA, &S.raw_full[rs], tm * kBM, k0);
                    if (TB)
                        tma_load_2d(S.rawB[rs], &mapB, &S.raw_full[rs], tn * kBN, k0);
                    else
                        tma_load_2d(S.rawB[rs], &mapB, &S.raw_full[rs], k0, tn * kBN);
                    ++issued;
                    if (++rs == kFRaw) {
                        rs = 0;
                        rph ^= 1u;
                    }
                }
            }
            if (!ok) {
                // bounded wait for the copies already in flight
                int st = rs;
                uint32_t ph = rph;
                for (int i = 0; i < kFRaw && i < issued; ++i) {
                    st = (st + kFRaw - 1) % kFRaw;
                    if (st == kFRaw - 1) ph ^= 1u;
                    volatile int never = 0;
                    (void)mbar_wait(&S.raw_full[st], ph, globaltimer_ns() + 100000000ull, &never);
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer (as cgemm_tc_kernel, TF32) ----------------
        if (lane == 0) {
            constexpr uint32_t id = idesc_make(2u, kBM, 2 * kBN, 0);
            constexpr uint32_t idh = idesc_make(2u, kBM, kBN, 0);
            constexpr uint32_t idhn = idesc_make(2u, kBM, kBN, 1);
            const uint32_t a0 = tmem, a1 = tmem + 256;
            const uint32_t a1r = a1, a1i = a1 + 128;
            int cs = 0;
            uint32_t cph = 0, e_phase = 0;
            bool pending = false;
            bool ok = true;
            auto wait_drained = [&]() -> bool {
                if (!pending) return true;
                if (!mbar_wait(&S.acc0_empty, e_phase, globaltimer_ns() + w.wait_ns, abort_flag))
                    return false;
                e_phase ^= 1u;
                pending = false;
                tc_fence_after();
                return true;
            };
            for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
                for (int kb = 0; kb < nkb; ++kb) {
                    if (!mbar_wait(&S.conv_full[cs], cph, globaltimer_ns() + w.wait_ns,
                                   abort_flag)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (kb == 0 && !wait_drained()) {
                        ok = false;
                        break;
                    }
                    const uint64_t dA = sdesc_kmajor_sw64(smem_u32(S.conv[cs]));
                    const uint64_t dB = dA + (kAStageBytes >> 4);
#define A_(ks, p) (dA + (uint64_t)(((p) * kTileBytes + (ks) * 32) >> 4))
#define B_(ks, p) (dB + (uint64_t)(((p) * kTileBytes + (ks) * 32) >> 4))
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint32_t first = (kb == 0 && ks == 0) ? 0u : 1u;
                        mma_tf32(a1, A_(ks, 2), B_(ks, 1), id, first);   // Ar_lo [Br_hi; Bi_hi]
                        mma_tf32(a1, A_(ks, 3), B_(ks, 0), id, 1u);      // Ai_lo [-Bi_hi; Br_hi]
                        mma_tf32(a1r, A_(ks, 0), B_(ks, 3), idh, 1u);    //  Ar_hi Br_lo
                        mma_tf32(a1i, A_(ks, 0), B_(ks, 4), idh, 1u);    //  Ar_hi Bi_lo
                        mma_tf32(a1r, A_(ks, 1), B_(ks, 4), idhn, 1u);   // -Ai_hi Bi_lo
                        mma_tf32(a1i, A_(ks, 1), B_(ks, 3), idh, 1u);    //  Ai_hi Br_lo
                    }
                    const bool group_start = (kb % kFDrain) == 0;
                    const bool group_end = (kb % kFDrain) == kFDrain - 1 || kb == nkb - 1;
                    if (group_start && !wait_drained()) {
                        ok = false;
                        break;
                    }
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint32_t first = (ks == 0 && group_start) ? 0u : 1u;
                        mma_tf32(a0, A_(ks, 0), B_(ks, 1), id, first);   // Ar_hi [Br_hi; Bi_hi]
                        mma_tf32(a0, A_(ks, 1), B_(ks, 0), id, 1u);      // Ai_hi [-Bi_hi; Br_hi]
                    }
#undef A_
#undef B_
                    tc_commit(&S.conv_empty[cs]);
                    if (group_end) {
                        tc_commit(&S.acc0_full);
                        pending = true;
                    }
                    if (++cs == kFConv) {
                        cs = 0;
                        cph ^= 1u;
                    }
                }
            }
            if (!ok && !*abort_flag) fraise_abort(S, d_err, kErrTimeoutMma);
            tc_commit(&S.drain);
            volatile int never = 0;
            (void)mbar_wait(&S.drain, 0, globaltimer_ns() + w.wait_ns, &never);
        }
    } else {
        // ---------------- converters + epilogue (warps 2..9) ----------------
        const int ew = warp - 2;                    // 0..7
        const int q = warp & 3;                     // tensor-memory lane quadrant
        const int half = (warp - 2) >> 2;
        const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16) + half * kFEpiCols;
        const bool use_beta = (beta.x != 0.0f) || (beta.y != 0.0f);
        const int ngroups = (nkb + kFDrain - 1) / kFDrain;
        uint32_t f_phase = 0;
        int rs = 0, cs = 0;
        uint32_t rph = 0, cph = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < num_tiles && ok; t += gridDim.x) {
            int tm, tn;
            ftile_coords(t, tiles_m, tiles_n, group_m, tm, tn);
            float racc[kFEpiCols], iacc[kFEpiCols];
#pragma unroll
            for (int j = 0; j < kFEpiCols; ++j) racc[j] = iacc[j] = 0.0f;
            // drain group g: acc0 (and acc1 with the last group) into the registers
            auto drain = [&](int g) -> bool {
                int got = 0;
                if (lane == 0)
                    got = mbar_wait(&S.acc0_full, f_phase, globaltimer_ns() + w.wait_ns,
                                    abort_flag)
                              ? 1
                              : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    if (lane == 0 && !*abort_flag) fraise_abort(S, d_err, kErrTimeoutEpilogue);
                    return false;
                }
                f_phase ^= 1u;
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < kFEpiCols; c += 16) {
                    uint32_t vr[16], vi[16];
                    tmem_ld16(trow + 0 + c, vr);
                    tmem_ld16(trow + 128 + c, vi);
                    tmem_ld_wait(vr);
                    tmem_ld_wait(vi);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        racc[c + j] += __uint_as_float(vr[j]);
                        iacc[c + j] += __uint_as_float(vi[j]);
                    }
                }
                if (g == ngroups - 1) {
#pragma unroll
                    for (int c = 0; c < kFEpiCols; c += 16) {
                        uint32_t vr[16], vi[16];
                        tmem_ld16(trow + 256 + c, vr);
                        tmem_ld16(trow + 384 + c, vi);
                        tmem_ld_wait(vr);
                        tmem_ld_wait(vi);
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            racc[c + j] = fmaf(__uint_as_float(vr[j]), 0x1p-11f, racc[c + j]);
                            iacc[c + j] = fmaf(__uint_as_float(vi[j]), 0x1p-11f, iacc[c + j]);
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&S.acc0_empty);
                return true;
            };
            auto group_last = [&](int g) { return min((g + 1) * kFDrain, nkb) - 1; };
            int g_next = 0;
            for (int kb = 0; kb < nkb && ok; ++kb) {
                // Drains before converting stage kb.  Converting kb needs the
                // MMAs of kb - 2 done, and those wait for every group that
                // ends at or before kb - 3: such a drain is forced.  A group
                // that ended earlier still is drained if acc0 is complete.
                while (g_next < ngroups && group_last(g_next) <= kb - 1) {
                    if (group_last(g_next) > kb - 3) {
                        int ready = lane == 0 ? (mbar_test(&S.acc0_full, f_phase) ? 1 : 0) : 0;
                        if (!__shfl_sync(0xffffffffu, ready, 0)) break;
                    }
                    if (!drain(g_next)) {
                        ok = false;
                        break;
                    }
                    ++g_next;
                }
                if (!ok) break;
                int got = 0;
                if (lane == 0)
                    got = (mbar_wait(&S.raw_full[rs], rph, globaltimer_ns() + w.wait_ns,
                                     abort_flag) &&
                           mbar_wait(&S.conv_empty[cs], cph ^ 1u, globaltimer_ns() + w.wait_ns,
                                     abort_flag))
                              ? 1
                              : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    if (lane == 0 && !*abort_flag) fraise_abort(S, d_err, kErrTimeoutEpilogue);
                    ok = false;
                    break;
                }
                // 32 warp-rounds per stage (op(A) then op(B): 4 row blocks x 4
                // chunks each), four per warp
#pragma unroll
                for (int rq = 0; rq < 4; ++rq) {
                    const int g = ew + 8 * rq;  // 0..31: warp-uniform
                    const int c4 = g & 3;
                    const int r = ((g >> 2) & 3) * 32 + lane;
                    float2 v[4];
                    if (g < 16) {
                        load_quad<TA>(S.rawA[rs], r, c4, v);
                        split_quad<false>(v, conjA != 0, S.conv[cs], r, c4);
                    } else {
                        load_quad<!TB>(S.rawB[rs], r, c4, v);
                        split_quad<true>(v, conjB != 0, S.conv[cs] + kAStageBytes, r, c4);
                    }
                }
                fence_proxy_async_shared();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&S.conv_full[cs]);
                    mbar_arrive(&S.raw_empty[rs]);
                }
                if (++rs == kFRaw) {
                    rs = 0;
                    rph ^= 1u;
                }
                if (++cs == kFConv) {
                    cs = 0;
                    cph ^= 1u;
                }
            }
            while (ok && g_next < ngroups) {
                if (!drain(g_next)) ok = false;
                ++g_next;
            }
            if (!ok) break;
            const int row = tm * kBM + q * 32 + lane;
            const int col0 = tn * kBN + half * kFEpiCols;
            if (row < m) {
                const float unA = ldexpf(1.0f, -desc->sA), unB = ldexpf(1.0f, -desc->sB);
                float2 *crow = C + row;
#pragma unroll
                for (int j = 0; j < kFEpiCols; ++j) {
                    const int col = col0 + j;
                    if (col < n) {
                        const float pr = (racc[j] * unA) * unB;
                        const float pi = (iacc[j] * unA) * unB;
                        float2 o;
                        o.x = alpha.x * pr - alpha.y * pi;
                        o.y = alpha.x * pi + alpha.y * pr;
                        float2 *dst = crow + static_cast<int64_t>(col) * ldc;
                        if (use_beta) {
                            const float2 c = *dst;
                            o.x += beta.x * c.x - beta.y * c.y;
                            o.y += beta.x * c.y + beta.y * c.x;
                        }
                        *dst = o;
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        __syncwarp();
        tmem_dealloc(tmem, kTmemCols);
    }
}

// Tensor map of a raw complex64 operand: 8-byte elements, dims {inner, outer}
// with row stride ld, box {box_inner, box_outer}.
CUresult encode_raw(EncodeTiledFn encode, CUtensorMap *map, const float2 *X, int64_t inner,
                    int64_t outer, int64_t ld, int box_inner, int box_outer, bool swizzle128) {
    cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t gstride[1] = {(cuuint64_t)(ld * 8)};
    cuuint32_t box[2] = {(cuuint32_t)box_inner, (cuuint32_t)box_outer};
    cuuint32_t estride[2] = {1, 1};
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<float2 *>(X), gdim, gstride,
                  box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

template <bool TA, bool TB>
cudaError_t launch_fused(const CUtensorMap &ma, const CUtensorMap &mb, const qcs_gemm_desc_t *desc,
                         int64_t m, int64_t n, int64_t k_pad, int conjA, int conjB, float2 alpha,
                         float2 beta, float2 *C, int64_t ldc, int *d_err, int num_sms,
                         int group_m, const TcWork &w, cudaStream_t s) {
    const size_t smem = sizeof(FusedSmem) + 1024;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(cgemm_tc_fused_kernel<TA, TB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int64_t tiles = ((m + kBM - 1) / kBM) * ((n + kBN - 1) / kBN);
    const int grid = static_cast<int>(tiles < num_sms ? tiles : num_sms);
    cgemm_tc_fused_kernel<TA, TB><<<grid, kTcThreads, smem, s>>>(
        ma, mb, desc, (int)m, (int)n, (int)k_pad, conjA, conjB, alpha, beta, C, ldc, d_err,
        group_m < 1 ? 1 : group_m, w);
    return cudaGetLastError();
}

}  // namespace

bool tc_fused_supported(int opA, int opB, int64_t m, int64_t n, int64_t k, const float2 *A,
                        int64_t lda, const float2 *B, int64_t ldb) {
    (void)opA;
    (void)opB;
    if (m < 1 || n < 1 || k < 1 || m > INT32_MAX || n > INT32_MAX || k > INT32_MAX - 32)
        return false;
    if ((lda & 1) || (ldb & 1)) return false;  // row strides must be multiples of 16 bytes
    return ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) == 0;
}

cudaError_t launch_cgemm_tc_fused(EncodeTiledFn encode, const qcs_gemm_desc_t *desc, int opA,
                                  int opB, int64_t m, int64_t n, int64_t k, float2 alpha,
                                  const float2 *A, int64_t lda, const float2 *B, int64_t ldb,
                                  float2 beta, float2 *C, int64_t ldc, int *d_err, int num_sms,
                                  int group_m, const TcWork &w, cudaStream_t s) {
    if (!tc_fused_supported(opA, opB, m, n, k, A, lda, B, ldb) || w.G != 1 || w.S != 1)
        return cudaErrorNotSupported;
    const bool ta = opA != QCS_OP_N, tb = opB != QCS_OP_N;
    CUtensorMap ma, mb;
    // op N of A: A is m x k (m contiguous); op T / C: A is k x m (k contiguous)
    CUresult r = ta ? encode_raw(encode, &ma, A, k, m, lda, kFK, kBM, true)
                    : encode_raw(encode, &ma, A, m, k, lda, kBM, kFK, false);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    // op N of B: B is k x n (k contiguous); op T / C: B is n x k (n contiguous)
    r = tb ? encode_raw(encode, &mb, B, n, k, ldb, kBN, kFK, false)
           : encode_raw(encode, &mb, B, k, n, ldb, kFK, kBN, true);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int64_t k_pad = (k + 31) / 32 * 32;  // the two-pass path's stage count
    const int ca = opA == QCS_OP_C, cb = opB == QCS_OP_C;
    if (ta)
        return tb ? launch_fused<true, true>(ma, mb, desc, m, n, k_pad, ca, cb, alpha, beta, C, ldc,
                                             d_err, num_sms, group_m, w, s)
                  : launch_fused<true, false>(ma, mb, desc, m, n, k_pad, ca, cb, alpha, beta, C,
                                              ldc, d_err, num_sms, group_m, w, s);
    return tb ? launch_fused<false, true>(ma, mb, desc, m, n, k_pad, ca, cb, alpha, beta, C, ldc,
                                          d_err, num_sms, group_m, w, s)
              : launch_fused<false, false>(ma, mb, desc, m, n, k_pad, ca, cb, alpha, beta, C, ldc,
                                           d_err, num_sms, group_m, w, s);
}

}  // namespace qcs
