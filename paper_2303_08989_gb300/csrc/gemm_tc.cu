// Error-corrected complex GEMM on the fifth-generation tensor cores
// (tcgen05, sm_103a).
//
// Method (Section 2.1, Eq. 1; Section 3): every FP32 operand x is split into
// hi = toLow(x 2^s) and lo = toLow((x 2^s - hi) 2^11) by the split kernel.
// A complex product is four real products (Re = ArBr - AiBi,
// Im = ArBi + AiBr); each real product is emulated by three tensor-core
// products, hi*hi into accumulator 0 and lo*hi + hi*lo into accumulator 1:
//   C = 2^-(sA+sB) (acc0 + 2^-11 acc1).
//
// Complex products as N = 256 MMAs.  op(A) has four planes (hi.re, hi.im,
// lo.re, lo.im); op(B) has five, -Bi_hi, Br_hi, Bi_hi, Br_lo, Bi_lo, so that
// two consecutive hi planes are one 256-row operand.  With an accumulator
// laid out as [re | im] (256 columns),
//   Ar x [Br; Bi]  adds [Ar Br | Ar Bi],   Ai x [-Bi; Br]  adds [-Ai Bi | Ai Br],
// so the hi*hi and lo*hi products of a complex product are two MMAs each
// that read 12 KB of shared memory for 128 x 256 x 16 instead of two 8 KB
// reads per 128 x 128 x 16; the hi*lo products stay N = 128 MMAs (the
// -Ai Bi term through the negate-A bit), which keeps a stage at 72 KB so that
// three stages fit.  Per K step the tensor core reads 80 KB of shared memory
// instead of 96 KB: those reads paced the all-N = 128 form.
//
// Rounding.  Section 2.1 adds the hi*hi products outside the tensor core with
// round-to-nearest because the A100 tensor core truncates inside its
// accumulation.  The sm_103a tensor core truncates too (measured: 1 + 0.75 ulp
// accumulates to 1, within one MMA and across MMAs, for FP16 and TF32
// inputs), which makes the error of a TMEM-resident hi*hi sum grow linearly
// with k.  So accumulator 0 is drained every DRAIN pipeline stages (two MMA
// K steps each): that group's hi*hi sum is computed fresh in tensor memory
// and added with round-to-nearest FP32 adds into registers of the epilogue
// warps.  The correction products (accumulator 1, weight 2^-11) stay in
// tensor memory for the whole K loop: their truncation error enters the
// result scaled by 2^-11.
//
// Kernel structure (one CTA per SM, persistent over 128 x 128 complex tiles):
//   warp 0     TMA producer: per stage, one 3-D box of the four A planes and
//              one of the five B planes (128 rows x 64 bytes each, 64-byte
//              swizzle) into a 3-stage shared-memory ring.
//   warp 1     MMA issuer (one thread).  Per stage (two K steps): the 12
//              correction MMAs into acc1 first; then, once the epilogue has
//              drained the previous group's acc0, the 4 hi*hi MMAs (into a
//              fresh acc0 at a group's first stage).  The drain thus overlaps
//              the correction MMAs.
//              Tensor memory: 512 columns = acc0 [re | im], acc1 [re | im].
//   warps 2-9  epilogue, two warps per tensor-memory lane quadrant (each owns
//              64 columns of its 32 rows): per drain group, tcgen05.ld of acc0
//              and round-to-nearest adds into 128 registers; at the end of a
//              tile, + 2^-11 acc1, the alpha/beta epilogue and coalesced stores
//              (32 consecutive complex values of one column per store).
// The descriptor the selector wrote decides at run time whether this
// instantiation runs at all (the "launch all candidates, the unselected one
// exits" scheme of Section 4.2).
//
// Work units.  One launch covers G equal-shape GEMMs (a group of
// contraction instances: instance g has its own planes, descriptor and
// output) and splits each GEMM's K loop into S equal ranges; a unit is
// (instance, K range, output tile) and the persistent CTAs walk the units in
// that order, tiles fastest.  Units of an instance whose descriptor selected
// another kind are skipped.  With S > 1 a unit writes its scaled partial
// 2^-(sA+sB) (acc0 + 2^-11 acc1) to a partial buffer and tc_splitk_reduce
// forms C = alpha sum_s P_s + beta C, summing the ranges in a fixed order,
// so the result does not depend on scheduling.  Splitting K fills the SMs
// when a GEMM has few output tiles for its K (1024^3: 64 tiles on 152 SMs).
//
// Real GEMMs (REAL = true; the SGEMM of Section 2.1 itself).  op(A) has two
// planes (hi, lo), op(B) two planes (hi, lo) of 256 rows, and a tile is
// 128 x 256 real outputs: per K step one N = 256 MMA of hi*hi into acc0 and
// two of lo*hi and hi*lo into acc1, the same tensor-memory layout (the
// "re" and "im" halves of an accumulator are output columns 0-127 and
// 128-255 of the tile) and the same drain.  A stage is 48 KB, so four fit.
//
// Clusters (MC = true, complex kernel, qcs_set_tc_multicast): two CTAs along
// M work on tile rows 2p and 2p + 1 of the same tile column in lockstep and
// share its B box: rank 0 loads planes 0-2 of it, rank 1 planes 3-4, each
// with one TMA multicast into the shared memory of both.  A stage is freed
// once the MMAs of both CTAs have read it (each commit arrives on both CTAs'
// "empty" barriers), so the B traffic from L2 per CTA halves.
//
// CTA pairs (CL = kClPair, qcs_set_tc_pairs): the two CTAs of a cluster run
// one M = 256 tile (tile rows 2p and 2p + 1) with tcgen05 MMAs of
// cta_group::2, issued by one thread of the even CTA.  Each CTA keeps its own
// 128 rows of A and HALF of every B operand: a pair MMA takes the first N/2
// rows of its K-major B from the even CTA and the rest from the odd one, at
// the same shared-memory offset, so each tensor core reads half the B bytes
// per MMA it did alone (complex: 56 KB of shared-memory reads per K step
// instead of 80).  Per complex stage the even CTA holds B planes 0, 1
// (-Bi_hi, Br_hi) and the odd one planes 1, 2 (Br_hi, Bi_hi), so that the
// same slot is [-Bi; Br] or [Br; Bi] across the pair; and each holds its 64
// of the 128 rows of the lo planes 3, 4 for the N = 128 MMAs.  A stage is
// 32 + 24 KB and four fit.  Real pairs: each CTA holds 128 of the 256 B rows
// of both planes (32 KB stages, six of them).  Each CTA loads its own
// operands (TMA, its own "full" barriers); the odd CTA's MMA warp forwards
// each completed stage to the even CTA's "full" barrier (a remote arrive),
// the even CTA's commits arrive on both CTAs' "empty" and "acc0_full"
// barriers, and the odd CTA's epilogue warps arrive remotely on the even
// CTA's "acc0_empty".  Every tensor-core result of a tile is the same MMA
// sequence as in one CTA.
#include <cuda_fp16.h>

#include "internal.h"
#include "ptx.cuh"

namespace qcs {

namespace {

constexpr int kEpiWarps = 8;
constexpr int kEpiCols = kBN / 2;  // columns per epilogue warp

// Cluster forms of a launch: one CTA per tile, two CTAs sharing each B box
// by TMA multicast, or a CTA pair running M = 256 tiles.
constexpr int kClNone = 0, kClMulticast = 1, kClPair = 2;

// Stage geometry of the complex (REAL = false) and real kernels.
template <bool REAL, int CL = kClNone>
struct TcGeom {
    static constexpr bool pair = CL == kClPair;
    static constexpr int stages = pair ? (REAL ? 6 : 4) : (REAL ? 4 : kStages);
    static constexpr int a_bytes = REAL ? 2 * kTileBytes : kAStageBytes;  // 16 | 32 KB
    // B bytes per CTA and stage: alone 32 | 40 KB; pairs 16 | 24 KB
    static constexpr int b_bytes =
        pair ? (REAL ? 2 * kTileBytes : 3 * kTileBytes) : (REAL ? 4 * kTileBytes : kBStageBytes);
    static constexpr int stage_bytes = a_bytes + b_bytes;  // 48 | 72 KB; pairs 32 | 56 KB
    static constexpr int tile_n = REAL ? 2 * kBN : kBN;  // output columns of a tile
    // Byte offset, in the B part of a stage, of the operand the MMAs call B
    // plane p (complex: 0 -Bi_hi, 1 Br_hi, 3 Br_lo, 4 Bi_lo, the 256-row
    // operands at 0 and 1; real: 0 hi, 2 lo).  Pairs: this CTA's half of it.
    __host__ __device__ static constexpr int b_off(int p) {
        return !pair ? p * kTileBytes
               : REAL ? (p / 2) * kTileBytes
                      : (p <= 1 ? p * kTileBytes : 2 * kTileBytes + (p - 3) * (kTileBytes / 2));
    }
};

template <bool REAL, int CL = kClNone>
struct TcSmem {
    uint8_t stage[TcGeom<REAL, CL>::stages][TcGeom<REAL, CL>::stage_bytes];
    uint64_t full[TcGeom<REAL, CL>::stages];
    uint64_t empty[TcGeom<REAL, CL>::stages];
    uint64_t acc0_full;
    uint64_t acc0_empty;
    uint64_t drain;
    uint32_t tmem_base;
    int abort;
};

// Tile t of the raster: groups of group_m tile rows, column after column
// inside a group, so that the tiles in flight share A and B panels in L2.
__device__ __forceinline__ void tile_coords(int t, int tiles_m, int tiles_n, int group_m, int &tm,
                                            int &tn) {
    const int per_group = group_m * tiles_n;
    const int g = t / per_group;
    const int first_m = g * group_m;
    const int gsize = min(tiles_m - first_m, group_m);
    const int r = t - g * per_group;
    tm = first_m + r % gsize;
    tn = r / gsize;
}

template <class Smem>
__device__ __forceinline__ void raise_abort(Smem &S, int *d_err, int code) {
    *reinterpret_cast<volatile int *>(&S.abort) = 1;
    atomicCAS(d_err, 0, code);
}

__device__ __forceinline__ bool kind_runs(int kind, int mode) {
    if (kind == 0) return mode == QCS_MODE_FP16X || mode == QCS_MODE_FP16X_SCALED;
    if (kind == 1) return mode == QCS_MODE_TF32X;
    return mode == QCS_MODE_BF16X3;
}

template <int KIND, bool PAIR = false>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t acc) {
    if constexpr (PAIR) {
        if (KIND == 1)
            mma_tf32_pair(d, a, b, idesc, acc);
        else
            mma_f16_pair(d, a, b, idesc, acc);
    } else {
        if (KIND == 1)
            mma_tf32(d, a, b, idesc, acc);
        else
            mma_f16(d, a, b, idesc, acc);
    }
}

// Unit u of a launch: instance g, K range r (of S), tile t (of tiles).
struct Unit {
    int g, r, t;
};
__device__ __forceinline__ Unit unit_of(int u, int tiles, int S) {
    Unit x;
    x.t = u % tiles;
    const int q = u / tiles;
    x.r = q % S;
    x.g = q / S;
    return x;
}

template <int KIND, int DRAIN, bool REAL, int CL>
__global__ void __launch_bounds__(kTcThreads, 1)
    cgemm_tc_kernel(const __grid_constant__ CUtensorMap mapA,
                    const __grid_constant__ CUtensorMap mapB,
                    const __grid_constant__ CUtensorMap mapB2,
                    const qcs_gemm_desc_t *__restrict__ desc, int m, int n, int k_pad,
                    float2 alpha, float2 beta, float2 *__restrict__ C, int64_t ldc, int *d_err,
                    int group_m, const TcWork w) {
    constexpr bool MC = CL == kClMulticast;
    constexpr bool PAIR = CL == kClPair;
    constexpr bool CLU = CL != kClNone;  // clusters of two CTAs
    static_assert(!(MC && REAL), "multicast clusters are built for the complex kernel");
    // a single GEMM that did not select this kind exits before touching anything
    // (both CTAs of a cluster read the same descriptor)
    if (w.G == 1 && !kind_runs(KIND, desc->mode)) return;

    using Geo = TcGeom<REAL, CL>;
    constexpr int NST = Geo::stages;
    extern __shared__ uint8_t smem_raw[];
    TcSmem<REAL, CL> &S = *reinterpret_cast<TcSmem<REAL, CL> *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    volatile int *abort_flag = &S.abort;
    // PAIR: the even CTA (rank 0) issues the MMAs of the pair
    const bool leader = !PAIR || cluster_ctarank() == 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            // PAIR: the leader's stage is full once its own bytes landed and
            // the peer forwarded its own stage's completion
            mbar_init(&S.full[s], (PAIR && leader) ? 2 : 1);
            mbar_init(&S.empty[s], MC ? 2 : 1);  // MC: the MMAs of both CTAs of the cluster
        }
        mbar_init(&S.acc0_full, 1);
        mbar_init(&S.acc0_empty, PAIR ? 2 * kEpiWarps : kEpiWarps);  // PAIR: both epilogues
        mbar_init(&S.drain, 1);
        S.abort = 0;
        fence_barrier_init();
        tma_prefetch_desc(&mapA);
        tma_prefetch_desc(&mapB);
        if (CLU) tma_prefetch_desc(&mapB2);
    }
    if (warp == 1) {
        if constexpr (PAIR) {
            tmem_alloc_pair(&S.tmem_base, kTmemCols);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(&S.tmem_base, kTmemCols);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem_base;
    // clusters: the peer's barriers are initialised before anything reaches them
    if constexpr (CLU) cluster_sync();

    const int tiles_m = (m + kBM - 1) / kBM;
    const int tiles_n = (n + Geo::tile_n - 1) / Geo::tile_n;
    // clusters: units over pairs of tile rows (the host makes tiles_m even),
    // one per cluster at a time; a cluster's rank-r CTA takes row 2 p + r
    const int num_tiles = (CLU ? tiles_m / 2 : tiles_m) * tiles_n;
    const int num_units = w.G * w.S * num_tiles;
    auto first_unit = [] { return CLU ? (int)(blockIdx.x >> 1) : (int)blockIdx.x; };
    auto unit_step = [] { return CLU ? (int)(gridDim.x >> 1) : (int)gridDim.x; };
    auto coords = [&](int t, int &tm, int &tn) {
        if constexpr (CLU) {
            tile_coords(t, tiles_m / 2, tiles_n, group_m / 2 > 0 ? group_m / 2 : 1, tm, tn);
            tm = 2 * tm + (int)cluster_ctarank();
        } else {
            tile_coords(t, tiles_m, tiles_n, group_m, tm, tn);
        }
    };
    constexpr int kElemBytes = (KIND == 1) ? 4 : 2;
    constexpr int kKPerStage = kRowBytes / kElemBytes;  // two MMA K steps: 32 (16-bit) or 16 (TF32)
    const int num_kb = k_pad / kKPerStage;
    // stages [kb_begin(r), kb_begin(r + 1)) of K range r; S <= num_kb, so none is empty
    auto kb_begin = [&](int r) { return static_cast<int>((int64_t)r * num_kb / w.S); };

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int issued = 0;
            bool ok = true;
            for (int u = first_unit(); u < num_units && ok && !w.stall; u += unit_step()) {
                const Unit x = unit_of(u, num_tiles, w.S);
                if (w.G > 1 && !kind_runs(KIND, desc[x.g].mode)) continue;
                int tm, tn;
                coords(x.t, tm, tn);
                const int rowA = static_cast<int>(x.g * w.a_rows) + tm * kBM;
                const int rowB = static_cast<int>(x.g * w.b_rows) + tn * Geo::tile_n;
                const int kb1 = kb_begin(x.r + 1);
                for (int kb = kb_begin(x.r); kb < kb1; ++kb) {
                    if (!mbar_wait(&S.empty[stage], phase ^ 1u, globaltimer_ns() + w.wait_ns,
                                   abort_flag)) {
                        if (!*abort_flag) raise_abort(S, d_err, kErrTimeoutProducer);
                        ok = false;
                        break;
                    }
                    mbar_arrive_expect_tx(&S.full[stage], Geo::stage_bytes);
                    tma_load_3d(S.stage[stage], &mapA, &S.full[stage], kb * kKPerStage, rowA, 0);
                    if constexpr (PAIR) {
                        // this CTA's half of the B operands (box of mapB: 128 rows x 2
                        // planes; of mapB2: 64 rows x 2 planes)
                        const int rk = (int)cluster_ctarank();
                        uint8_t *bst = S.stage[stage] + Geo::a_bytes;
                        if constexpr (REAL) {
                            tma_load_3d(bst, &mapB, &S.full[stage], kb * kKPerStage,
                                        rowB + rk * kBM, 0);
                        } else {
                            tma_load_3d(bst, &mapB, &S.full[stage], kb * kKPerStage, rowB, rk);
                            tma_load_3d(bst + Geo::b_off(3), &mapB2, &S.full[stage],
                                        kb * kKPerStage, rowB + rk * (kBN / 2), 3);
                        }
                    } else if constexpr (MC) {
                        // this CTA's share of the B box, to both CTAs of the cluster
                        if (cluster_ctarank() == 0)
                            tma_load_3d_mc(S.stage[stage] + Geo::a_bytes, &mapB, &S.full[stage],
                                           kb * kKPerStage, rowB, 0, (uint16_t)0x3);
                        else
                            tma_load_3d_mc(S.stage[stage] + Geo::a_bytes + 3 * kTileBytes, &mapB2,
                                           &S.full[stage], kb * kKPerStage, rowB, 3, (uint16_t)0x3);
                    } else {
                        tma_load_3d(S.stage[stage] + Geo::a_bytes, &mapB, &S.full[stage],
                                    kb * kKPerStage, rowB, 0);
                    }
                    ++issued;
                    if (++stage == NST) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) {
                // Give the copies already in flight a bounded chance to land
                // before this CTA's shared memory goes away.
                int st = stage;
                uint32_t ph = phase;
                for (int i = 0; i < NST && i < issued; ++i) {
                    st = (st + NST - 1) % NST;
                    if (st == NST - 1) ph ^= 1u;
                    volatile int never = 0;
                    (void)mbar_wait(&S.full[st], ph, globaltimer_ns() + 100000000ull, &never);
                }
            }
        }
    } else if (warp == 1 && !leader) {
        // ---------------- PAIR, odd CTA: forward its stages to the leader ----------------
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int u = first_unit(); u < num_units && ok; u += unit_step()) {
                const Unit x = unit_of(u, num_tiles, w.S);
                if (w.G > 1 && !kind_runs(KIND, desc[x.g].mode)) continue;
                const int kb1 = kb_begin(x.r + 1);
                for (int kb = kb_begin(x.r); kb < kb1; ++kb) {
                    if (!mbar_wait(&S.full[stage], phase, globaltimer_ns() + w.wait_ns,
                                   abort_flag)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_cluster(&S.full[stage], 0);
                    if (++stage == NST) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok && !*abort_flag) raise_abort(S, d_err, kErrTimeoutMma);
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            constexpr uint32_t fmt = (KIND == 0) ? 0u : (KIND == 1 ? 2u : 1u);
            constexpr uint32_t MM = PAIR ? 2 * kBM : kBM;                // M 128 (PAIR: 256)
            constexpr uint32_t id = idesc_make(fmt, MM, 2 * kBN, 0);     // N 256
            constexpr uint32_t idh = idesc_make(fmt, MM, kBN, 0);        // N 128
            constexpr uint32_t idhn = idesc_make(fmt, MM, kBN, 1);       // ... negated A
            const uint32_t a0 = tmem, a1 = tmem + 256;  // [re | im] each
            const uint32_t a1r = a1, a1i = a1 + 128;
            int stage = 0;
            uint32_t phase = 0, e_phase = 0;
            bool pending = false;  // an acc0 drain the epilogue has not yet confirmed
            bool ok = true;
            // PAIR: the peer's threads arrive on these barriers too
            auto wait_bar = [&](uint64_t *bar, uint32_t par) -> bool {
                if constexpr (PAIR)
                    return mbar_wait_cluster(bar, par, globaltimer_ns() + w.wait_ns, abort_flag);
                else
                    return mbar_wait(bar, par, globaltimer_ns() + w.wait_ns, abort_flag);
            };
            auto commit = [&](uint64_t *bar) {
                if constexpr (PAIR)
                    tc_commit_pair_mc(bar, (uint16_t)0x3);  // on both CTAs' barrier
                else if constexpr (MC)
                    tc_commit_mc(bar, (uint16_t)0x3);
                else
                    tc_commit(bar);
            };
            auto wait_drained = [&]() -> bool {
                if (!pending) return true;
                if (!wait_bar(&S.acc0_empty, e_phase)) return false;
                e_phase ^= 1u;
                pending = false;
                tc_fence_after();
                return true;
            };
            for (int u = first_unit(); u < num_units && ok; u += unit_step()) {
                const Unit x = unit_of(u, num_tiles, w.S);
                if (w.G > 1 && !kind_runs(KIND, desc[x.g].mode)) continue;
                const int kb0 = kb_begin(x.r), kb1 = kb_begin(x.r + 1);
                for (int kb = kb0; kb < kb1; ++kb) {
                    if (!wait_bar(&S.full[stage], phase)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // acc1 is read by the epilogue at the end of the previous
                    // unit: wait for that before overwriting it.
                    if (kb == kb0 && !wait_drained()) {
                        ok = false;
                        break;
                    }
                    // Descriptors differ only in the start-address field (bits 0..13,
                    // address >> 4), which never carries out for shared memory.
                    // A planes: 0 Ar_hi, 1 Ai_hi, 2 Ar_lo, 3 Ai_lo.  B planes:
                    // 0 -Bi_hi, 1 Br_hi, 2 Bi_hi, 3 Br_lo, 4 Bi_lo; the 256-row
                    // operand at plane p covers planes p and p + 1 (PAIR: slot p
                    // of both CTAs).  K step ks starts 32 bytes into each 64-byte row.
                    // Real kernel: A planes 0 hi, 1 lo; B planes of 256 rows, hi at
                    // tile offset 0, lo at 2 (PAIR: 128 rows each).
                    const uint64_t dA = sdesc_kmajor_sw64(smem_u32(S.stage[stage]));
                    const uint64_t dB = dA + (Geo::a_bytes >> 4);
#define A_(ks, p) (dA + (uint64_t)(((p) * kTileBytes + (ks) * 32) >> 4))
#define B_(ks, p) (dB + (uint64_t)((Geo::b_off(p) + (ks) * 32) >> 4))
                    // correction products: acc1 += lo*hi + hi*lo
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint32_t first = (kb == kb0 && ks == 0) ? 0u : 1u;
                        if constexpr (REAL) {
                            mma<KIND, PAIR>(a1, A_(ks, 1), B_(ks, 0), id, first);   // A_lo B_hi
                            mma<KIND, PAIR>(a1, A_(ks, 0), B_(ks, 2), id, 1u);      // A_hi B_lo
                        } else {
                            mma<KIND, PAIR>(a1, A_(ks, 2), B_(ks, 1), id, first);   // Ar_lo [Br_hi; Bi_hi]
                            mma<KIND, PAIR>(a1, A_(ks, 3), B_(ks, 0), id, 1u);      // Ai_lo [-Bi_hi; Br_hi]
                            mma<KIND, PAIR>(a1r, A_(ks, 0), B_(ks, 3), idh, 1u);    //  Ar_hi Br_lo
                            mma<KIND, PAIR>(a1i, A_(ks, 0), B_(ks, 4), idh, 1u);    //  Ar_hi Bi_lo
                            mma<KIND, PAIR>(a1r, A_(ks, 1), B_(ks, 4), idhn, 1u);   // -Ai_hi Bi_lo
                            mma<KIND, PAIR>(a1i, A_(ks, 1), B_(ks, 3), idh, 1u);    //  Ai_hi Br_lo
                        }
                    }
                    // hi*hi products: a fresh acc0 every DRAIN stages, once the
                    // previous one was drained
                    const bool group_start = ((kb - kb0) % DRAIN) == 0;
                    const bool group_end = ((kb - kb0) % DRAIN) == DRAIN - 1 || kb == kb1 - 1;
                    if (group_start && !wait_drained()) {
                        ok = false;
                        break;
                    }
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        const uint32_t first = (ks == 0 && group_start) ? 0u : 1u;
                        if constexpr (REAL) {
                            mma<KIND, PAIR>(a0, A_(ks, 0), B_(ks, 0), id, first);   // A_hi B_hi
                        } else {
                            mma<KIND, PAIR>(a0, A_(ks, 0), B_(ks, 1), id, first);   // Ar_hi [Br_hi; Bi_hi]
                            mma<KIND, PAIR>(a0, A_(ks, 1), B_(ks, 0), id, 1u);      // Ai_hi [-Bi_hi; Br_hi]
                        }
                    }
#undef A_
#undef B_
                    // frees the smem stage when these MMAs finish (clusters: in both CTAs)
                    commit(&S.empty[stage]);
                    if (group_end) {
                        // acc0 (and, on a tile's last stage, acc1) ready (MC: this
                        // CTA's only; PAIR: in both CTAs)
                        if constexpr (PAIR)
                            commit(&S.acc0_full);
                        else
                            tc_commit(&S.acc0_full);
                        pending = true;
                    }
                    if (++stage == NST) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok && !*abort_flag) raise_abort(S, d_err, kErrTimeoutMma);
            // Wait (bounded) until every MMA this thread issued has finished,
            // so tensor memory is idle before it is released.
            if constexpr (PAIR)
                tc_commit_pair(&S.drain);
            else
                tc_commit(&S.drain);
            volatile int never = 0;
            (void)mbar_wait(&S.drain, 0, globaltimer_ns() + w.wait_ns, &never);
        }
    } else {
        // ---------------- epilogue (warps 2..9) ----------------
        const int q = warp & 3;                         // lane quadrant this warp may access
        const int half = (warp - 2) >> 2;               // which 64 of the 128 columns
        const uint32_t trow = tmem + (static_cast<uint32_t>(q * 32) << 16) + half * kEpiCols;
        const bool use_beta = (beta.x != 0.0f) || (beta.y != 0.0f);
        uint32_t f_phase = 0;
        bool ok = true;
        for (int u = first_unit(); u < num_units && ok; u += unit_step()) {
            const Unit x = unit_of(u, num_tiles, w.S);
            const qcs_gemm_desc_t dg = desc[x.g];
            if (w.G > 1 && !kind_runs(KIND, dg.mode)) continue;
            const float unA = ldexpf(1.0f, -dg.sA);
            const float unB = ldexpf(1.0f, -dg.sB);
            const int nkb = kb_begin(x.r + 1) - kb_begin(x.r);
            int tm, tn;
            coords(x.t, tm, tn);
            float racc[kEpiCols], iacc[kEpiCols];
#pragma unroll
            for (int j = 0; j < kEpiCols; ++j) racc[j] = iacc[j] = 0.0f;
            for (int kb = DRAIN - 1; kb < nkb + DRAIN - 1; kb += DRAIN) {
                const bool last = kb >= nkb - 1;  // the group holding the unit's last stage
                int got = 0;
                if (lane == 0)
                    got = mbar_wait(&S.acc0_full, f_phase, globaltimer_ns() + w.wait_ns,
                                    abort_flag)
                              ? 1
                              : 0;
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    if (lane == 0 && !*abort_flag) raise_abort(S, d_err, kErrTimeoutEpilogue);
                    ok = false;
                    break;
                }
                f_phase ^= 1u;
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < kEpiCols; c += 16) {
                    uint32_t vr[16], vi[16];
                    tmem_ld16(trow + 0 + c, vr);
                    tmem_ld16(trow + 128 + c, vi);
                    tmem_ld_wait(vr);
                    tmem_ld_wait(vi);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        racc[c + j] += __uint_as_float(vr[j]);  // round-to-nearest FP32 adds
                        iacc[c + j] += __uint_as_float(vi[j]);
                    }
                }
                if (last) {
#pragma unroll
                    for (int c = 0; c < kEpiCols; c += 16) {
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
                if (lane == 0) {
                    if (leader)
                        mbar_arrive(&S.acc0_empty);
                    else
                        mbar_arrive_cluster(&S.acc0_empty, 0);  // PAIR: the leader's barrier
                }
            }
            if (!ok) break;
            const int row = tm * kBM + q * 32 + lane;
            if constexpr (REAL) {
                // the two accumulator halves are output columns c0 and c0 + 128
                if (row < m) {
                    const int c0 = tn * Geo::tile_n + half * kEpiCols;
                    float *out;
                    int64_t ld;
                    if (w.S > 1) {
                        out = reinterpret_cast<float *>(w.P) +
                              ((int64_t)x.r * w.G + x.g) * (int64_t)m * n + row;
                        ld = m;
                    } else {
                        out = reinterpret_cast<float *>(C) + x.g * w.c_stride + row;
                        ld = ldc;
                    }
                    const bool epi = w.S == 1;
#pragma unroll
                    for (int hv = 0; hv < 2; ++hv) {
#pragma unroll
                        for (int j = 0; j < kEpiCols; ++j) {
                            const int col = c0 + hv * kBN + j;
                            if (col < n) {
                                float v = ((hv ? iacc[j] : racc[j]) * unA) * unB;
                                float *dst = out + static_cast<int64_t>(col) * ld;
                                if (epi) {
                                    v *= alpha.x;
                                    if (use_beta) v = fmaf(beta.x, *dst, v);
                                }
                                *dst = v;
                            }
                        }
                    }
                }
                continue;
            }
            const int col0 = tn * kBN + half * kEpiCols;
            if (w.S > 1) {
                // a K range's partial, scaled back, into its [r][g] block (ld m)
                if (row < m) {
                    float2 *prow = w.P + ((int64_t)x.r * w.G + x.g) * (int64_t)m * n + row;
#pragma unroll
                    for (int j = 0; j < kEpiCols; ++j) {
                        const int col = col0 + j;
                        if (col < n)
                            prow[(int64_t)col * m] =
                                make_float2((racc[j] * unA) * unB, (iacc[j] * unA) * unB);
                    }
                }
                continue;
            }
            if (row < m) {
                float2 *crow = C + x.g * w.c_stride + row;
#pragma unroll
                for (int j = 0; j < kEpiCols; ++j) {
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
    // clusters: neither CTA leaves while the other may still write into its
    // shared memory or tensor memory, or arrive on its barriers
    if constexpr (CLU) cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        __syncwarp();
        if constexpr (PAIR)
            tmem_dealloc_pair(tmem, kTmemCols);
        else
            tmem_dealloc(tmem, kTmemCols);
    }
}

// C_g = alpha sum_r P[r][g] + beta C_g for every instance g whose GEMM ran on
// the tensor cores (its descriptor did not select FP32); the K ranges are
// added in order r = 0, 1, ... with round-to-nearest FP32 adds.
__global__ void __launch_bounds__(256)
    tc_splitk_reduce_kernel(const qcs_gemm_desc_t *__restrict__ desc, int G, int S, int64_t m,
                            int64_t n, const float2 *__restrict__ P, float2 alpha, float2 beta,
                            float2 *__restrict__ C, int64_t ldc, int64_t c_stride) {
    const int g = blockIdx.y;
    if (desc[g].mode == QCS_MODE_FP32) return;
    const int64_t mn = m * n;
    const bool use_beta = (beta.x != 0.0f) || (beta.y != 0.0f);
    float2 *Cg = C + g * c_stride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mn;
         i += (int64_t)gridDim.x * blockDim.x) {
        float2 acc = P[(int64_t)g * mn + i];
        for (int r = 1; r < S; ++r) {
            const float2 v = P[((int64_t)r * G + g) * mn + i];
            acc.x += v.x;
            acc.y += v.y;
        }
        const int64_t col = i / m;
        float2 *dst = Cg + col * ldc + (i - col * m);
        float2 o;
        o.x = alpha.x * acc.x - alpha.y * acc.y;
        o.y = alpha.x * acc.y + alpha.y * acc.x;
        if (use_beta) {
            const float2 c = *dst;
            o.x += beta.x * c.x - beta.y * c.y;
            o.y += beta.x * c.y + beta.y * c.x;
        }
        *dst = o;
    }
}

// The real counterpart: C_g = alpha sum_r P[r][g] + beta C_g over m x n
// floats.
__global__ void __launch_bounds__(256)
    tc_splitk_reduce_real_kernel(const qcs_gemm_desc_t *__restrict__ desc, int G, int S,
                                 int64_t m, int64_t n, const float *__restrict__ P, float alpha,
                                 float beta, float *__restrict__ C, int64_t ldc, int64_t c_stride) {
    const int g = blockIdx.y;
    if (desc[g].mode == QCS_MODE_FP32) return;
    const int64_t mn = m * n;
    float *Cg = C + g * c_stride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < mn;
         i += (int64_t)gridDim.x * blockDim.x) {
        float acc = P[(int64_t)g * mn + i];
        for (int r = 1; r < S; ++r) acc += P[((int64_t)r * G + g) * mn + i];
        const int64_t col = i / m;
        float *dst = Cg + col * ldc + (i - col * m);
        float o = alpha * acc;
        if (beta != 0.0f) o = fmaf(beta, *dst, o);
        *dst = o;
    }
}

// A launch in clusters of two CTAs (CL = kClMulticast or kClPair): one
// cluster per pair of tile rows at a time, as many clusters as fit at once.
template <int KIND, int DRAIN, bool REAL, int CL>
cudaError_t launch_clusters(const CUtensorMap &mapA, const CUtensorMap &mapB,
                            const CUtensorMap &mapB2, const qcs_gemm_desc_t *desc, int64_t m,
                            int64_t n, int64_t k_pad, float2 alpha, float2 beta, float2 *C,
                            int64_t ldc, int *d_err, int num_sms, int gm, int64_t units,
                            const TcWork &w, cudaStream_t s) {
    auto kern = cgemm_tc_kernel<KIND, DRAIN, REAL, CL>;
    const size_t smem = sizeof(TcSmem<REAL, CL>) + 1024;
    static int max_clusters = 0;  // clusters of two that fit at once, measured once
    if (max_clusters == 0) {
        cudaError_t e =
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t q = {};
        cudaLaunchAttribute qa[1];
        qa[0].id = cudaLaunchAttributeClusterDimension;
        qa[0].val.clusterDim.x = 2;
        qa[0].val.clusterDim.y = 1;
        qa[0].val.clusterDim.z = 1;
        q.gridDim = dim3((unsigned)(num_sms & ~1));
        q.blockDim = dim3(kTcThreads);
        q.dynamicSmemBytes = smem;
        q.attrs = qa;
        q.numAttrs = 1;
        e = cudaOccupancyMaxActiveClusters(&max_clusters, kern, &q);
        if (e != cudaSuccess || max_clusters < 1) {
            max_clusters = 0;
            cudaGetLastError();
            return cudaErrorNotSupported;
        }
    }
    const int64_t pair_units = units / 2;
    const int clusters = (int)std::min<int64_t>(pair_units, max_clusters);
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)(2 * clusters));
    cfg.blockDim = dim3(kTcThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, mapA, mapB, mapB2, desc, (int)m, (int)n, (int)k_pad,
                              alpha, beta, C, ldc, d_err, gm, w);
}

// With an even number of tile rows: pairB not NULL runs CTA pairs (complex:
// pairB[0] boxes of 128 rows x 2 planes, pairB[1] 64 rows x 2 planes; real:
// pairB[0] 128 rows x 2 planes; the default drain only), else mcB not NULL
// (complex kernel) clusters of two CTAs sharing each B box, mcB[0] covering
// B planes 0-2 and mcB[1] planes 3-4 of every box.  Otherwise one CTA per
// tile with mapB (all planes of a box).
template <int KIND, int DRAIN, bool REAL>
cudaError_t launch_kind(const qcs_gemm_desc_t *desc, const CUtensorMap *mapA,
                        const CUtensorMap *mapB, const CUtensorMap *mcB,
                        const CUtensorMap *pairB, int64_t m, int64_t n, int64_t k_pad,
                        float2 alpha, float2 beta, float2 *C, int64_t ldc, int *d_err,
                        int num_sms, int group_m, const TcWork &w, cudaStream_t s) {
    const size_t smem = sizeof(TcSmem<REAL>) + 1024;
    constexpr int tn = TcGeom<REAL>::tile_n;
    const int64_t tiles_m = (m + kBM - 1) / kBM;
    const int64_t units = tiles_m * ((n + tn - 1) / tn) * w.G * w.S;
    if (units == 0 || k_pad == 0) return cudaSuccess;
    const int gm = group_m < 1 ? 1 : group_m;
    if constexpr (DRAIN == 4) {
        if (pairB && tiles_m % 2 == 0)
            return launch_clusters<KIND, DRAIN, REAL, kClPair>(
                *mapA, pairB[0], REAL ? pairB[0] : pairB[1], desc, m, n, k_pad, alpha, beta, C,
                ldc, d_err, num_sms, gm, units, w, s);
    }
    if constexpr (!REAL) {
        if (mcB && tiles_m % 2 == 0)
            return launch_clusters<KIND, DRAIN, REAL, kClMulticast>(
                *mapA, mcB[0], mcB[1], desc, m, n, k_pad, alpha, beta, C, ldc, d_err, num_sms,
                gm, units, w, s);
    }
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(cgemm_tc_kernel<KIND, DRAIN, REAL, kClNone>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    const int grid = static_cast<int>(units < num_sms ? units : num_sms);
    cgemm_tc_kernel<KIND, DRAIN, REAL, kClNone><<<grid, kTcThreads, smem, s>>>(
        *mapA, *mapB, *mapB, desc, (int)m, (int)n, (int)k_pad, alpha, beta, C, ldc, d_err, gm, w);
    return cudaGetLastError();
}

// ``drain``: pipeline stages per group, each two MMA K steps (32 k for the
// 16-bit kinds, 16 for TF32).
template <int KIND, bool REAL>
cudaError_t launch_drain(int drain, const qcs_gemm_desc_t *desc, const CUtensorMap *mapA,
                         const CUtensorMap *mapB, const CUtensorMap *mcB,
                         const CUtensorMap *pairB, int64_t m, int64_t n,
                         int64_t k_pad, float2 alpha, float2 beta, float2 *C, int64_t ldc,
                         int *d_err, int num_sms, int group_m, const TcWork &w, cudaStream_t s) {
    if (drain >= 4)
        return launch_kind<KIND, 4, REAL>(desc, mapA, mapB, mcB, pairB, m, n, k_pad, alpha, beta, C,
                                          ldc, d_err, num_sms, group_m, w, s);
    if (drain == 2)
        return launch_kind<KIND, 2, REAL>(desc, mapA, mapB, mcB, pairB, m, n, k_pad, alpha, beta, C,
                                          ldc, d_err, num_sms, group_m, w, s);
    return launch_kind<KIND, 1, REAL>(desc, mapA, mapB, mcB, pairB, m, n, k_pad, alpha, beta, C, ldc,
                                      d_err, num_sms, group_m, w, s);
}

template <bool REAL>
cudaError_t launch_any(int kind, int drain, const qcs_gemm_desc_t *desc, const CUtensorMap *mapA,
                       const CUtensorMap *mapB, const CUtensorMap *mcB,
                       const CUtensorMap *pairB, int64_t m, int64_t n,
                       int64_t k_pad, float2 alpha, float2 beta, float2 *C, int64_t ldc,
                       int *d_err, int num_sms, int group_m, cudaStream_t s, const TcWork &w) {
    if (w.G < 1 || w.S < 1 || (w.S > 1 && !w.P)) return cudaErrorInvalidValue;
    switch (kind) {
        case 0:
            return launch_drain<0, REAL>(drain, desc, mapA, mapB, mcB, pairB, m, n, k_pad, alpha, beta,
                                         C, ldc, d_err, num_sms, group_m, w, s);
        case 1:
            return launch_drain<1, REAL>(drain, desc, mapA, mapB, mcB, pairB, m, n, k_pad, alpha, beta,
                                         C, ldc, d_err, num_sms, group_m, w, s);
        default:
            return launch_drain<2, REAL>(drain, desc, mapA, mapB, mcB, pairB, m, n, k_pad, alpha, beta,
                                         C, ldc, d_err, num_sms, group_m, w, s);
    }
}

}  // namespace

cudaError_t launch_cgemm_tc(int kind, int drain, const qcs_gemm_desc_t *desc,
                            const CUtensorMap *mapA, const CUtensorMap *mapB, int64_t m,
                            int64_t n, int64_t k_pad, float2 alpha, float2 beta, float2 *C,
                            int64_t ldc, int *d_err, int num_sms, int group_m, cudaStream_t s,
                            const TcWork &w, const CUtensorMap *mcB,
                            const CUtensorMap *pairB) {
    return launch_any<false>(kind, drain, desc, mapA, mapB, mcB, pairB, m, n, k_pad, alpha, beta, C,
                             ldc, d_err, num_sms, group_m, s, w);
}

cudaError_t launch_sgemm_tc(int kind, int drain, const qcs_gemm_desc_t *desc,
                            const CUtensorMap *mapA, const CUtensorMap *mapB, int64_t m,
                            int64_t n, int64_t k_pad, float alpha, float beta, float *C,
                            int64_t ldc, int *d_err, int num_sms, int group_m, cudaStream_t s,
                            const TcWork &w, const CUtensorMap *pairB) {
    return launch_any<true>(kind, drain, desc, mapA, mapB, nullptr, pairB, m, n, k_pad,
                            make_float2(alpha, 0.f),
                            make_float2(beta, 0.f), reinterpret_cast<float2 *>(C), ldc, d_err,
                            num_sms, group_m, s, w);
}

cudaError_t launch_tc_reduce(const qcs_gemm_desc_t *desc, int64_t m, int64_t n, float2 alpha,
                             float2 beta, float2 *C, int64_t ldc, int num_sms, const TcWork &w,
                             cudaStream_t s) {
    if (w.S <= 1 || m == 0 || n == 0) return cudaSuccess;
    const int64_t blocks_needed = (m * n + 255) / 256;
    const int64_t cap = (int64_t)num_sms * 8;
    dim3 grid(static_cast<unsigned>(blocks_needed < cap ? blocks_needed : cap),
              static_cast<unsigned>(w.G));
    tc_splitk_reduce_kernel<<<grid, 256, 0, s>>>(desc, w.G, w.S, m, n, w.P, alpha, beta, C, ldc,
                                                 w.c_stride);
    return cudaGetLastError();
}

cudaError_t launch_tc_reduce_real(const qcs_gemm_desc_t *desc, int64_t m, int64_t n, float alpha,
                                  float beta, float *C, int64_t ldc, int num_sms, const TcWork &w,
                                  cudaStream_t s) {
    if (w.S <= 1 || m == 0 || n == 0) return cudaSuccess;
    const int64_t blocks_needed = (m * n + 255) / 256;
    const int64_t cap = (int64_t)num_sms * 8;
    dim3 grid(static_cast<unsigned>(blocks_needed < cap ? blocks_needed : cap),
              static_cast<unsigned>(w.G));
    tc_splitk_reduce_real_kernel<<<grid, 256, 0, s>>>(desc, w.G, w.S, m, n,
                                                      reinterpret_cast<const float *>(w.P), alpha,
                                                      beta, C, ldc, w.c_stride);
    return cudaGetLastError();
}

// Stages of the K loop per unit are ~1.2 us on one SM for a complex tile
// (measured: 16384^3 FP16X, 16384 tiles x 512 stages over 152 SMs in 67 ms)
// and take half the MMAs for a real one; the partials cost (2 S + 1) m n
// bytes-per-output of HBM traffic per GEMM at ~6 TB/s plus a launch.  The
// count minimises waves x stages per unit + that cost.
int tc_split_count(int64_t m, int64_t n, int64_t k, int64_t G, int num_sms, int forced,
                   bool real) {
    const int64_t nkb = (k + 31) / 32;  // 16-bit stages (TF32 has twice as many)
    if (nkb <= 1) return 1;
    if (forced > 0) return static_cast<int>(forced < nkb ? forced : nkb);
    const int64_t tile_n = real ? 2 * kBN : kBN;
    const int64_t tiles = ((m + kBM - 1) / kBM) * ((n + tile_n - 1) / tile_n) * G;
    if (tiles == 0 || num_sms <= 0) return 1;
    const double stage_us = real ? 0.65 : 1.2;
    const double out_bytes = real ? 4.0 : 8.0;
    double best = -1.0;
    int best_s = 1;
    for (int S = 1; S <= kMaxSplits && S <= nkb; ++S) {
        const int64_t units = tiles * S;
        const int64_t waves = (units + num_sms - 1) / num_sms;
        double t = (double)waves * (double)((nkb + S - 1) / S) * stage_us;
        if (S > 1) t += (2.0 * S + 1.0) * (double)(m * n * G) * out_bytes / 6.0e6 + 4.0;
        if (best < 0 || t < best * 0.97) {  // a split must win by 3% to be taken
            best = t;
            best_s = S;
        }
    }
    return best_s;
}

}  // namespace qcs
