// qhd_tcdft.h -- split-precision tensor-core DFT form of the 2-D step (internal).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace qhd {

struct TcState;

// ----------------------------------------------- tcgen05 GEMM (qhd_umma_gemm.cu)
// K segments of C = alpha * sum_g scale_g (A_g . B_g^T) + beta * C: a_k0 / b_k0
// are the K offsets (elements, multiples of 64) of the segment in A's and B's
// rows, kblocks its length in blocks of 64.  mode: UG_EACH_MMA makes every
// K = 16 MMA a group of its own (its partial added in FP32 with round to
// nearest); UG_OPEN starts a group that accumulates in tensor memory and
// following UG_CONTINUE segments extend (one FP32 rounding per group).
// UG_EACH_MMA_FLOAT: every MMA its own group, for operands whose 16-term sums
// are not exact in FP32: the result is scaled by (1 + kappa) to undo the
// expected truncation of each partial (see qhd_umma_gemm.cu).
// UG_EACH_MMA_BEXP: every MMA its own group, A holding integers scaled per row
// and per block of 16 K values: the group's scale is scale * 2^E[row][e0 + j]
// for the segment's j-th MMA (E from UgArgs::expo).
enum { UG_EACH_MMA = 0, UG_OPEN = 1, UG_CONTINUE = 2, UG_EACH_MMA_FLOAT = 3, UG_EACH_MMA_BEXP = 4 };
constexpr int UG_MAX_SEG = 16;
struct UgSeg {
    int a_k0, b_k0, kblocks;
    float scale;
    int mode;
    int e0;              // UG_EACH_MMA_BEXP: exponent column of the segment's first MMA
};
struct UgArgs {
    float *C;
    int64_t ldc;
    int64_t rows;        // rows of A and C (the last tile may be partial)
    int m_tiles, n_tiles;
    int nseg;
    UgSeg seg[UG_MAX_SEG];
    float alpha, beta;
    float kappa;         // expected relative truncation of per-MMA partials, undone in the epilogue
    const int8_t *expo;  // UG_EACH_MMA_BEXP: per-row exponents [rows][expo_ld]
    int64_t expo_ld;
    unsigned *err;       // 2 words: [0] a bounded wait gave up, [1] scratch of the wind-down waits
    uint64_t limit_ns;   // global-time limit of each wait
};
// n_cols % 128 == 0, lda and ldb multiples of 64; bn = 128; any rows >= 1 (the
// loads of a partial last row tile read zeros past the end, its stores stop there).
bool umma_gemm_shape_ok(int64_t rows, int64_t n_cols, int64_t lda, int64_t ldb, int bn);
// A: FP16 [rows][lda], B: FP16 [n_cols][ldb] (B^T, K contiguous), C: FP32 [rows][ldc].
cudaError_t umma_gemm(const __half *A, int64_t lda, const __half *B, int64_t ldb, float *C, int64_t ldc, int64_t rows,
                      int64_t n_cols, const UgSeg *segs, int nseg, float alpha, float beta, int bn, unsigned *err,
                      cudaStream_t s, const int8_t *expo = nullptr, int64_t expo_ld = 0);

// Arguments of one split kernel: the state lives in the FP32 product buffer
// of the state object between transforms; psi only at the start and end.
struct TcPhaseArgs {
    float2 *psi;              // interleaved complex64 state (first split / finish)
    const uint32_t *fq;       // fixed-point potential, B x n x n
    const uint64_t *pot;      // per-instance phase coefficient of this split
    const float4 *ptab;       // potential phase table (hi/lo)
    uint32_t dither;          // global-phase dither of the step (0 at the finish)
    const float4 *kt;         // kinetic factors of the step, hi/lo per axis
    int64_t kt_batch;         // 1: shared by all instances, else one per instance
    int ksum;                 // entries per instance of kt (n + n)
};

bool tc_supported(int n0, int n1, int64_t batch);
// products: 3 or 5 (block-scaled FP16 hi/lo integer slices), 10 (fixed-point slices, n <= 512)
bool tc_products_ok(int n, int products);
size_t tc_workspace_bytes(int n, int64_t batch, int products);
// Returns nullptr with *why set when the workspace is short or a CUDA call fails.
TcState *tc_create(int n, int64_t batch, int products, void *ws, size_t ws_bytes, cudaStream_t s,
                   const char **why);
void tc_destroy(TcState *t);
int tc_products(const TcState *t);

// The four transforms of one Strang step, each a split and the GEMM(s) of one
// axis transform.  from_psi: the first potential split of an evolve call
// reads psi.  *launches counts the kernels issued.
cudaError_t tc_split_potential(TcState *t, const TcPhaseArgs &a, bool from_psi, cudaStream_t s, int64_t *launches);
cudaError_t tc_split_transpose(TcState *t, cudaStream_t s, int64_t *launches);
cudaError_t tc_split_kinetic(TcState *t, const TcPhaseArgs &a, cudaStream_t s, int64_t *launches);
cudaError_t tc_gemm(TcState *t, bool inverse, cudaStream_t s, int64_t *launches);
// Block-scaled forms: re-round the last DFT-matrix slice of both directions with
// the step's dither (an offset in [0, 1) taken from its top 24 bits).
cudaError_t tc_dither_w(TcState *t, uint32_t dither, cudaStream_t s, int64_t *launches);
// 1 when a bounded wait of a tensor-core GEMM gave up (reads a device word;
// synchronises the stream); -1 when the read itself failed.
int tc_timed_out(TcState *t, cudaStream_t s);
// The product buffer (position space, natural layout) -> psi, with the final
// potential phase a.pot when phase is set.
cudaError_t tc_finish(TcState *t, const TcPhaseArgs &a, bool phase, cudaStream_t s, int64_t *launches);

}  // namespace qhd
