// qhd_tcdft.h -- split-precision tensor-core DFT form of the 2-D step (internal).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace qhd {

struct TcState;

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
// products: 3 or 5 (floating FP16 hi/lo operands), 10 (fixed-point slices, n <= 512)
bool tc_products_ok(int n, int products);
size_t tc_workspace_bytes(int n, int64_t batch, int products);
// Returns nullptr with *why set when the workspace is short, a CUDA call or
// cuBLAS set-up fails.
TcState *tc_create(int n, int64_t batch, int products, void *ws, size_t ws_bytes, cudaStream_t s,
                   const char **why);
void tc_destroy(TcState *t);
int tc_products(const TcState *t);

// The four transforms of one Strang step, each a split and the GEMM(s) of one
// axis transform.  from_psi: the first potential split of an evolve call
// reads psi.  *launches / *calls count the kernels / cuBLAS calls issued.
cudaError_t tc_split_potential(TcState *t, const TcPhaseArgs &a, bool from_psi, cudaStream_t s, int64_t *launches);
cudaError_t tc_split_transpose(TcState *t, cudaStream_t s, int64_t *launches);
cudaError_t tc_split_kinetic(TcState *t, const TcPhaseArgs &a, cudaStream_t s, int64_t *launches);
cudaError_t tc_gemm(TcState *t, bool inverse, int64_t *calls);
// The product buffer (position space, natural layout) -> psi, with the final
// potential phase a.pot when phase is set.
cudaError_t tc_finish(TcState *t, const TcPhaseArgs &a, bool phase, cudaStream_t s, int64_t *launches);

}  // namespace qhd
