// qhd_umma_gemm.cu -- the dense DFT products of the tensor-core transform on the
// 5th-generation tensor cores (tcgen05.mma, accumulators in tensor memory, TMA
// operand loads).
//
// C[rows][N] = alpha * sum_g scale_g * (A_g . B_g^T) + beta * C, with A FP16
// row-major (K contiguous) and B FP16 stored as B^T, row-major [N][K] (K
// contiguous): both operands K-major.  The K range is a list of segments, each
// pairing a K range of A with one of B (so one A segment can meet several B
// segments without being stored twice) and carrying a power-of-two scale.
//
// Accumulation.  The tensor cores add into an FP32 accumulator that is not
// rounded to nearest: over a long K loop the sum drifts towards zero (measured
// about -1e-9 K relative), which over thousands of transforms decides the
// error of a floating hi/lo split.  So K is cut into groups: each group
// accumulates in its own tensor-memory partial (fresh at the group's first
// MMA), and the epilogue warps add the finished partial, times the group's
// scale, into FP32 registers with round-to-nearest FMAs.  A segment either
// makes every MMA (K = 16) a group of its own -- with operands whose 16-term
// sums are exact in FP32 (integer slices below 2^24), every partial is exact
// and the whole product is rounded to nearest -- or opens a group that
// following segments continue (exact integer sums over the whole group).
//
// One CTA computes a 128 x 128 tile: warp 0 issues the TMA loads into a ring of
// STAGES shared-memory stages, warp 1 allocates the tensor memory and one of
// its threads issues the MMAs, warps 2..9 drain the partials (two warps per
// 32-lane quarter of the accumulator, each half of the columns) and write C.
// Every wait is bounded in time; a wait that gives up sets an error word that
// the host reads (QHD_ERR_TIMEOUT), and the CTA winds down, waits for its
// MMAs and frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "qhd.h"
#include "qhd_tcdft.h"
#include "qhd_umma.cuh"

namespace qhd {

namespace {

constexpr int UG_BM = 128, UG_BK = 64;
constexpr int UG_THREADS = 320;
constexpr int UG_EPI_WARPS = 8;
constexpr uint32_t UG_TMEM_COLS = 512;

// Two tile widths.  128 columns: the epilogue threads hold 64 FP32 accumulators
// each across groups (each SM sub-partition holds at most 16K registers, so 3
// warps of a sub-partition get <= 170 each), which the per-MMA groups need.
// 256 columns (long tensor-memory accumulations only): 128 columns per
// epilogue thread do not fit in registers, so each finished group is added to
// C in global memory (read-modify-write, FP32 round-to-nearest, the same
// arithmetic as the register path); one MMA instruction does twice the work and
// the operands cost 3/4 of the bytes per flop.
template <int BN> struct UgCfg {
    static constexpr int NBUF = (int)UG_TMEM_COLS / BN;     // partial buffers in tensor memory
    static constexpr int STAGES = BN == 256 ? 4 : 6;        // shared-memory ring
    static constexpr int A_BYTES = UG_BM * UG_BK * 2;       // 16 KB
    static constexpr int B_BYTES = BN * UG_BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr int COLS = BN / 2;                     // columns per epilogue thread
    static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + 1024;  // alignment + tiles + barriers
    static_assert(BN == 128 || BN == 256, "tile width");
    static_assert(A_BYTES % 1024 == 0 && B_BYTES % 1024 == 0, "1024-byte aligned tiles");
};

// Visits the accumulation groups of the K list in order with their scales,
// deciding the boundaries per segment in registers (the MMA thread's walk):
// every MMA of a per-MMA segment is a group (scaled, for the block-scaled mode,
// by this row's exponent of the MMA's 16 K values, 1 past the last row), and a
// run of UG_OPEN + UG_CONTINUE segments is one group with the opening
// segment's scale.  f(scale) handles one group; false stops the walk.
template <typename F>
__device__ __forceinline__ bool for_each_group(const UgArgs &a, const int8_t *erp, F &&f) {
    float open_scale = 1.f;
    for (int sg = 0; sg < a.nseg; ++sg) {
        const int mode = a.seg[sg].mode, kbs = a.seg[sg].kblocks;
        const float scale = a.seg[sg].scale;
        if (mode == UG_EACH_MMA || mode == UG_EACH_MMA_FLOAT || mode == UG_EACH_MMA_BEXP) {
            const bool bexp = mode == UG_EACH_MMA_BEXP;
            const int e0 = a.seg[sg].e0;
            for (int kb = 0; kb < kbs; ++kb) {
                // the four MMAs' exponents of this K block in one load (0 past the last row)
                const uint32_t e4 = bexp && erp ? __ldg(reinterpret_cast<const uint32_t *>(erp + e0 + kb * 4)) : 0u;
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float sc = scale;
                    if (bexp) sc *= __int_as_float(((int)(int8_t)(e4 >> (8 * i)) + 127) << 23);
                    if (!f(sc)) return false;
                }
            }
        } else {
            if (mode == UG_OPEN) open_scale = scale;
            const bool closes = sg + 1 >= a.nseg || a.seg[sg + 1].mode != UG_CONTINUE;
            if (closes && !f(open_scale)) return false;
        }
    }
    return true;
}

template <int BN>
__global__ void __launch_bounds__(UG_THREADS, 1)
    k_umma_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const __grid_constant__ UgArgs a) {
    using Cfg = UgCfg<BN>;
    constexpr int STAGES = Cfg::STAGES, NBUF = Cfg::NBUF;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *tiles = base;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + (size_t)STAGES * Cfg::STAGE_BYTES);
    uint64_t *full = bars, *empty = bars + STAGES, *pfull = bars + 2 * STAGES, *pempty = pfull + NBUF;
    uint64_t *done = pempty + NBUF;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int m_tile = blockIdx.x / a.n_tiles, n_tile = blockIdx.x % a.n_tiles;
    const int m0 = m_tile * UG_BM, n0 = n_tile * BN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            umma::mbar_init(&full[s], 1);
            umma::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NBUF; ++b) {
            umma::mbar_init(&pfull[b], 1);
            umma::mbar_init(&pempty[b], UG_EPI_WARPS);
        }
        umma::mbar_init(done, 1);
        umma::mbar_fence_init();
    }
    if (warp == 1) umma::tmem_alloc(tslot, UG_TMEM_COLS);
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        // ------------------------------------------------------ TMA producer
        if (lane == 0) {
            umma::tma_prefetch_desc(&tmA);
            umma::tma_prefetch_desc(&tmB);
            int kb = 0;
            bool ok = true;
            for (int sg = 0; sg < a.nseg && ok; ++sg) {
                const UgSeg &s = a.seg[sg];
                for (int j = 0; j < s.kblocks && ok; ++j, ++kb) {
                    const int st = kb % STAGES;
                    if (kb >= STAGES) ok = umma::mbar_wait(&empty[st], ((kb / STAGES) - 1) & 1, a.err, a.limit_ns);
                    if (!ok) break;
                    uint8_t *ta = tiles + (size_t)st * Cfg::STAGE_BYTES;
                    umma::mbar_expect_tx(&full[st], Cfg::STAGE_BYTES);
                    umma::tma_load_2d(ta, &tmA, &full[st], s.a_k0 + j * UG_BK, m0);
                    umma::tma_load_2d(ta + Cfg::A_BYTES, &tmB, &full[st], s.b_k0 + j * UG_BK, n0);
                }
            }
            if (!ok) {
                // loads may still be landing: wait (briefly bounded) for the last ones issued
                for (int k = kb - 1; k >= 0 && k >= kb - STAGES; --k)
                    umma::mbar_wait(&full[k % STAGES], (k / STAGES) & 1, a.err + 1, 50000000ull);
            }
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issue
        if (lane == 0) {
            constexpr uint32_t IDESC = umma::idesc_f16_f32(UG_BM, BN);
            // The group structure is decided per segment in registers: the issue
            // rate of this one thread bounds the tensor pipe, so the per-MMA path
            // carries no parameter-space lookups.
            int kb = 0, buf = 0, grp = 0;
            bool ok = a.nseg > 0;
            auto open_group = [&]() -> bool {
                if (grp < NBUF) return true;
                if (!umma::mbar_wait(&pempty[buf], ((grp / NBUF) - 1) & 1, a.err, a.limit_ns)) return false;
                umma::tc_fence_after();
                return true;
            };
            auto close_group = [&]() {
                umma::mma_commit(&pfull[buf]);
                buf = (buf + 1) % NBUF;
                ++grp;
            };
            for (int sg = 0; sg < a.nseg && ok; ++sg) {
                const int mode = a.seg[sg].mode, kbs = a.seg[sg].kblocks;
                const bool each = mode == UG_EACH_MMA || mode == UG_EACH_MMA_FLOAT || mode == UG_EACH_MMA_BEXP;
                const bool opens = mode == UG_OPEN;
                const bool closes = sg + 1 >= a.nseg || a.seg[sg + 1].mode != UG_CONTINUE;
                for (int j = 0; j < kbs; ++j, ++kb) {
                    const int st = kb % STAGES;
                    ok = umma::mbar_wait(&full[st], (kb / STAGES) & 1, a.err, a.limit_ns);
                    if (!ok) break;
                    umma::tc_fence_after();
                    const uint32_t sa = umma::smem_u32(tiles + (size_t)st * Cfg::STAGE_BYTES);
                    const uint64_t da = umma::sdesc_k128(sa), db = umma::sdesc_k128(sa + Cfg::A_BYTES);
                    // 16 FP16 along K = 32 bytes: start address advances by 2 (16-byte units)
                    if (each) {
                        for (int i = 0; i < 4 && ok; ++i) {
                            ok = open_group();
                            if (!ok) break;
                            umma::mma_f16(tmem + (uint32_t)(buf * BN), da + 2u * i, db + 2u * i, IDESC, 0u);
                            close_group();
                        }
                        if (!ok) break;
                    } else {
                        const bool first = opens && j == 0;
                        if (first) {
                            ok = open_group();
                            if (!ok) break;
                        }
                        const uint32_t d = tmem + (uint32_t)(buf * BN);
                        umma::mma_f16(d, da, db, IDESC, first ? 0u : 1u);
#pragma unroll
                        for (int i = 1; i < 4; ++i) umma::mma_f16(d, da + 2u * i, db + 2u * i, IDESC, 1u);
                        if (closes && j == kbs - 1) close_group();
                    }
                    umma::mma_commit(&empty[st]);
                }
            }
            // every MMA issued has completed before the tensor memory is freed
            umma::mma_commit(done);
            umma::mbar_wait(done, 0, a.err + 1, 1000000000ull);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int ew = warp - 2;
        const int q = warp & 3;                  // accumulator lanes 32 q .. 32 q + 31 (hardware quarter)
        const int h = ew >> 2;                   // column half
        constexpr int COLS = Cfg::COLS;
        if constexpr (BN == 256) {
            int grp = 0;
            const int64_t row = (int64_t)m0 + q * 32 + lane;
            float *crow = row < a.rows ? a.C + row * a.ldc + n0 + h * COLS : nullptr;
            auto group = [&](float scale) -> bool {
                const float sc = scale * a.alpha;
                const int buf = grp % NBUF;
                int okw = 1;
                if (lane == 0) okw = umma::mbar_wait(&pfull[buf], (grp / NBUF) & 1, a.err, a.limit_ns) ? 1 : 0;
                if (__shfl_sync(0xffffffffu, okw, 0) == 0) return false;
                umma::tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + h * COLS);
#pragma unroll 1
                for (int ch = 0; ch < COLS / 32; ++ch) {
                    uint32_t r[32];
                    umma::tmem_ld32(taddr + (uint32_t)(ch * 32), r);
                    umma::tmem_ld_wait();
                    if (crow) {
                        float4 *cp = reinterpret_cast<float4 *>(crow + ch * 32);
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            float4 base = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (grp > 0) {
                                base = cp[k];
                            } else if (a.beta != 0.f) {
                                const float4 old = cp[k];
                                base = make_float4(old.x * a.beta, old.y * a.beta, old.z * a.beta, old.w * a.beta);
                            }
                            cp[k] = make_float4(fmaf(__uint_as_float(r[4 * k]), sc, base.x),
                                                fmaf(__uint_as_float(r[4 * k + 1]), sc, base.y),
                                                fmaf(__uint_as_float(r[4 * k + 2]), sc, base.z),
                                                fmaf(__uint_as_float(r[4 * k + 3]), sc, base.w));
                        }
                    }
                }
                umma::tc_fence_before();
                __syncwarp();
                if (lane == 0) umma::mbar_arrive(&pempty[buf]);
                ++grp;
                return true;
            };
            if (a.nseg > 0) for_each_group(a, nullptr, group);
        } else {
        float2 acc[COLS / 2];
#pragma unroll
        for (int k = 0; k < COLS / 2; ++k) acc[k] = make_float2(0.f, 0.f);
        int grp = 0;
        const int64_t erow = (int64_t)m0 + q * 32 + lane;
        const int8_t *erp = (a.expo && erow < a.rows) ? a.expo + erow * a.expo_ld : nullptr;
        auto group = [&](float sc) -> bool {
            const int buf = grp % NBUF;
            // lane 0 waits and the warp follows, so the warp-wide tensor-memory
            // loads below run with every lane or none
            int okw = 1;
            if (lane == 0) okw = umma::mbar_wait(&pfull[buf], (grp / NBUF) & 1, a.err, a.limit_ns) ? 1 : 0;
            if (__shfl_sync(0xffffffffu, okw, 0) == 0) return false;
            umma::tc_fence_after();
            const float2 s2 = make_float2(sc, sc);
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + h * COLS);
            // all of this thread's columns in flight at once, one wait
            uint32_t r[COLS];
            static_assert(COLS == 64, "one 64-column load per thread");
            umma::tmem_ld64(taddr, r);
            umma::tmem_ld_wait();
#pragma unroll
            for (int k = 0; k < COLS / 2; ++k)
                acc[k] = umma::fma2(make_float2(__uint_as_float(r[2 * k]), __uint_as_float(r[2 * k + 1])), s2, acc[k]);
            umma::tc_fence_before();
            __syncwarp();
            if (lane == 0) umma::mbar_arrive(&pempty[buf]);
            ++grp;
            return true;
        };
        const bool ok = a.nseg > 0 && for_each_group(a, erp, group);
        const int64_t row = (int64_t)m0 + q * 32 + lane;
        if (ok && row < a.rows) {
            float *crow = a.C + row * a.ldc + n0 + h * COLS;
            // expected truncation of the per-MMA partials: result * (1 + kappa), formed
            // as alpha acc + (alpha kappa) acc with one rounding
            const float ak = a.alpha * a.kappa;
            const float2 al = make_float2(a.alpha, a.alpha), be = make_float2(a.beta, a.beta);
#pragma unroll
            for (int k = 0; k < COLS / 4; ++k) {
                float2 lo = acc[2 * k], hi = acc[2 * k + 1];
                lo = make_float2(fmaf(lo.x, ak, lo.x * a.alpha), fmaf(lo.y, ak, lo.y * a.alpha));
                hi = make_float2(fmaf(hi.x, ak, hi.x * a.alpha), fmaf(hi.y, ak, hi.y * a.alpha));
                if (a.beta != 0.f) {
                    const float4 old = *reinterpret_cast<const float4 *>(crow + 4 * k);
                    lo = make_float2(fmaf(old.x, a.beta, lo.x), fmaf(old.y, a.beta, lo.y));
                    hi = make_float2(fmaf(old.z, a.beta, hi.x), fmaf(old.w, a.beta, hi.y));
                }
                (void)be;
                *reinterpret_cast<float4 *>(crow + 4 * k) = make_float4(lo.x, lo.y, hi.x, hi.y);
            }
        }
        }
    }
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    if (warp == 1) umma::tmem_dealloc(tmem, UG_TMEM_COLS);
}

char g_launch_diag[512] = "";

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 2-D FP16 map of a row-major [rows][cols] array, box {64, box_rows}, 128-byte swizzle.
bool make_map(CUtensorMap *m, const void *ptr, int64_t rows, int64_t cols, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)UG_BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_bn(const __half *A, int64_t lda, const __half *B, int64_t ldb, int64_t n_cols, const UgArgs &a,
                      cudaStream_t s) {
    using Cfg = UgCfg<BN>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_umma_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa{};
        e = cudaFuncGetAttributes(&fa, k_umma_gemm<BN>);
        if (e != cudaSuccess) return e;
        if (fa.maxThreadsPerBlock < UG_THREADS) {
            snprintf(g_launch_diag, sizeof g_launch_diag, "GEMM kernel fits %d threads, needs %d (%d registers)",
                     fa.maxThreadsPerBlock, UG_THREADS, fa.numRegs);
            return cudaErrorLaunchOutOfResources;
        }
        attr = true;
    }
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, a.rows, lda, UG_BM) || !make_map(&mb, B, n_cols, ldb, BN))
        return cudaErrorInvalidValue;
    k_umma_gemm<BN><<<(unsigned)(a.m_tiles * a.n_tiles), UG_THREADS, Cfg::SMEM, s>>>(ma, mb, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFuncAttributes fa{};
        cudaFuncGetAttributes(&fa, k_umma_gemm<BN>);
        int dev = 0, optin = 0, regs = 0, smsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        cudaDeviceGetAttribute(&regs, cudaDevAttrMaxRegistersPerBlock, dev);
        cudaDeviceGetAttribute(&smsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        snprintf(g_launch_diag, sizeof g_launch_diag,
                 "regs/thread %d, max threads %d, static smem %zu, max dyn smem %d, local %zu, requested dyn smem "
                 "%zu x %d threads; device: smem/block opt-in %d, smem/SM %d, regs/block %d",
                 fa.numRegs, fa.maxThreadsPerBlock, fa.sharedSizeBytes, fa.maxDynamicSharedSizeBytes,
                 fa.localSizeBytes, Cfg::SMEM, UG_THREADS, optin, smsm, regs);
    }
    return e;
}

}  // namespace

bool umma_gemm_shape_ok(int64_t rows, int64_t n_cols, int64_t lda, int64_t ldb, int bn) {
    return (bn == 128 || bn == 256) && rows > 0 && n_cols > 0 && n_cols % bn == 0 && lda % UG_BK == 0 &&
           ldb % UG_BK == 0 && (rows + UG_BM - 1) / UG_BM <= (int64_t(1) << 20);
}

cudaError_t umma_gemm(const __half *A, int64_t lda, const __half *B, int64_t ldb, float *C, int64_t ldc, int64_t rows,
                      int64_t n_cols, const UgSeg *segs, int nseg, float alpha, float beta, int bn, unsigned *err,
                      cudaStream_t s, const int8_t *expo, int64_t expo_ld) {
    if (!umma_gemm_shape_ok(rows, n_cols, lda, ldb, bn) || nseg < 1 || nseg > UG_MAX_SEG) return cudaErrorInvalidValue;
    // 256-column tiles when every group is a long tensor-memory accumulation
    bool long_groups = true;
    for (int i = 0; i < nseg; ++i) long_groups = long_groups && (segs[i].mode == UG_OPEN || segs[i].mode == UG_CONTINUE);
    const int tile = (bn == 256 && long_groups && n_cols % 256 == 0) ? 256 : 128;
    UgArgs a{};
    a.C = C;
    a.ldc = ldc;
    a.rows = rows;
    a.m_tiles = (int)((rows + UG_BM - 1) / UG_BM);
    a.n_tiles = (int)(n_cols / tile);
    a.nseg = nseg;
    for (int i = 0; i < nseg; ++i) {
        const UgSeg &g = segs[i];
        // every K block must lie inside its operand's row
        if (g.kblocks < 1 || g.a_k0 < 0 || g.b_k0 < 0 || g.a_k0 % UG_BK || g.b_k0 % UG_BK ||
            g.a_k0 + (int64_t)g.kblocks * UG_BK > lda || g.b_k0 + (int64_t)g.kblocks * UG_BK > ldb)
            return cudaErrorInvalidValue;
        if (g.mode == UG_CONTINUE && i == 0) return cudaErrorInvalidValue;
        // the epilogue reads a K block's four exponents as one aligned 32-bit word
        if (g.mode == UG_EACH_MMA_BEXP && (!expo || ((uintptr_t)expo & 3) || expo_ld % 4 || g.e0 < 0 || g.e0 % 4 ||
                                           g.e0 + 4 * (int64_t)g.kblocks > expo_ld))
            return cudaErrorInvalidValue;
        a.seg[i] = g;
    }
    a.alpha = alpha;
    a.beta = beta;
    a.expo = expo;
    a.expo_ld = expo_ld;
    // Each MMA returns its exact 16-term sum truncated towards zero to FP32
    // (measured: per-MMA partials are biased by -3.9e-8 relative).  A value of
    // mantissa m in [1, 2) loses on average half an ulp, 2^-24 / m of itself;
    // over the mantissas of the partials (log-uniform) the expected loss is the
    // fraction kappa = 2^-24 / (2 ln 2) of each partial, so the sum of
    // partials is the exact product times (1 - kappa) in expectation.  Only the
    // every-MMA groups of floating operands follow this model (exact integer
    // partials lose nothing, and a long accumulation truncates the running sum,
    // whose expectation has no such form).
    bool every = true;
    for (int i = 0; i < nseg; ++i) every = every && segs[i].mode == UG_EACH_MMA_FLOAT;
    a.kappa = every ? (float)(5.9604644775390625e-08 / (2.0 * 0.6931471805599453)) : 0.f;
    a.err = err;
    a.limit_ns = 2000000000ull;  // 2 s of global time per wait
    return tile == 256 ? launch_bn<256>(A, lda, B, ldb, n_cols, a, s) : launch_bn<128>(A, lda, B, ldb, n_cols, a, s);
}

}  // namespace qhd

static thread_local char g_gemm_err[768] = "";

extern "C" const char *qhd_tc_gemm_last_error(void) { return g_gemm_err; }

extern "C" qhd_status qhd_tc_gemm_f16(const void *A_dev, const void *B_dev, float *C_dev, int64_t ldc, int64_t rows,
                                      int64_t n_cols, int64_t k, int group_every_mma, float alpha, float beta,
                                      unsigned *err_dev, void *stream) {
    using namespace qhd;
    if (!A_dev || !B_dev || !C_dev || !err_dev || ((uintptr_t)A_dev & 15) || ((uintptr_t)B_dev & 15) ||
        ((uintptr_t)C_dev & 15) || ((uintptr_t)err_dev & 3))
        return QHD_ERR_INVALID_ARG;
    if (k < 64 || k > (int64_t(1) << 20) || ldc < n_cols || ldc % 4 || n_cols % 128 ||
        !umma_gemm_shape_ok(rows, n_cols, k, k, 128) || group_every_mma < 0 || group_every_mma > 2)
        return QHD_ERR_INVALID_ARG;
    const int mode = group_every_mma == 0 ? (int)UG_OPEN : group_every_mma == 1 ? (int)UG_EACH_MMA : (int)UG_EACH_MMA_FLOAT;
    UgSeg seg{0, 0, (int)(k / 64), 1.f, mode};
    cudaError_t e = umma_gemm(reinterpret_cast<const __half *>(A_dev), k, reinterpret_cast<const __half *>(B_dev), k,
                              C_dev, ldc, rows, n_cols, &seg, 1, alpha, beta, n_cols % 256 == 0 ? 256 : 128, err_dev,
                              (cudaStream_t)stream);
    snprintf(g_gemm_err, sizeof g_gemm_err, "%s%s%s", e == cudaSuccess ? "" : cudaGetErrorString(e),
             e == cudaSuccess ? "" : " | ", e == cudaSuccess ? "" : g_launch_diag);
    return e == cudaSuccess ? QHD_OK : (e == cudaErrorInvalidValue ? QHD_ERR_INVALID_ARG : QHD_ERR_CUDA);
}
