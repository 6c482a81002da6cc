// qhd_plane.cu -- kernels built on the cluster-resident plane engine.
//
// k_plane_pass: one fused pass over the last two axes of a 3-D grid (for
//   every (instance, i0) plane): inverse transform of the previous step along
//   axes 2 and 1, potential phase, forward transform along axes 1 and 2.  With
//   the axis-0 pass (forward, kinetic phase, inverse) a 3-D Strang step then
//   reads and writes psi twice instead of four times.
// k_plane_whole: a whole 2-D instance resident in one cluster for every step
//   of a chunk: per step the cross-cluster exchange with the potential phase,
//   then the local transforms with the kinetic phase in between.  psi touches
//   global memory only at the chunk's start and end.
#include "qhd_kernels.h"
#include "qhd_plane.cuh"

namespace qhd {

// Resident CTAs per SM the pass is compiled for: as many as the tile's shared
// memory allows, at most 3 (the pass is issue-bound; more warps hide latency).
template <int N1, int N2, int C> constexpr int plane_min_blocks() {
    constexpr size_t smem = PlaneCfg<N1, N2, C>::SMEM;
    constexpr int by_smem = (int)((227 * 1024) / smem);
    return by_smem >= 3 ? 3 : by_smem < 1 ? 1 : by_smem;
}

template <int N1, int N2, int C>
__global__ void __launch_bounds__(PLANE_THREADS, plane_min_blocks<N1, N2, C>()) k_plane_pass(PlaneArgs a) {
    using P = PlaneCfg<N1, N2, C>;
    extern __shared__ __align__(16) float4 smem4[];
    float4 *ptab = smem4;
    float2 *tile = reinterpret_cast<float2 *>(smem4 + PHASE_TAB);
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int64_t plane = blockIdx.x / C;
    uint32_t tiles[C];
#pragma unroll
    for (int q = 0; q < C; ++q) tiles[q] = cluster_addr(tile, (uint32_t)q);
    float2 *g = a.psi + plane * (int64_t)N1 * N2 + (int64_t)rank * P::R * N2;
    const bool inv = a.mode & MODE_INV, fwd = a.mode & MODE_FWD;

    plane_copy<N1, N2, C, true>(tile, g);
    const uint32_t *fqr = a.fq + plane * (int64_t)N1 * N2;
    {
        // the potential rows this CTA's exchange positions read (R / C rows in
        // each of the C row blocks) go to L2 now, during the tile load and the
        // inverse transforms, so the exchange's potential loads hit L2
        // (measured: 163.2 -> 160.5 us per 256^3 pass)
        constexpr uint32_t FQB = (uint32_t)((P::R / C) * N2 * sizeof(uint32_t));
        if (FQB % 16 == 0 && (int)threadIdx.x < C) {
            const uint32_t *src = fqr + (int64_t)(P::R * threadIdx.x + rank * (P::R / C)) * N2;
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(FQB) : "memory");
        }
    }
    load_phase_tab(ptab, a.ptab);
    const uint64_t coef = a.pot[plane / a.planes_per_inst];
    plane_copy_wait();
    if (inv) {
        plane_rows<N1, N2, C, 1>(tile, a.tw_row, nullptr, nullptr, rank);
        __syncthreads();
        plane_columns<N1, N2, C, true>(tile);
    }
    cluster.sync();
    plane_exchange<N1, N2, C, (C >= 8 ? 1 : 2)>(tiles, rank, inv, true, fwd, a.twx, fqr, coef, a.dither, ptab);
    cluster.sync();
    if (fwd) {
        plane_columns<N1, N2, C, false>(tile);
        __syncthreads();
        plane_rows<N1, N2, C, 0>(tile, a.tw_row, nullptr, nullptr, rank);
        __syncthreads();
    }
    plane_copy<N1, N2, C, false>(tile, g);
}

// MINB: CTAs per SM the kernel is compiled for (2 for batches; 1 for the wide
// split, which runs only when every CTA has an SM of its own).
template <int N1, int N2, int C, int MINB>
__global__ void __launch_bounds__(PLANE_THREADS, MINB) k_plane_whole(PlaneArgs a) {
    extern __shared__ __align__(16) float4 smem4[];
    float4 *ptab = smem4;
    float2 *tile = reinterpret_cast<float2 *>(smem4 + PHASE_TAB);
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    uint32_t tiles[C];
#pragma unroll
    for (int q = 0; q < C; ++q) tiles[q] = cluster_addr(tile, (uint32_t)q);
    plane_whole_run<N1, N2, C, 1>(a, blockIdx.x / C, rank, tiles, ptab, tile, true, cluster);
}

// ---------------------------------------------------------------- launchers
template <typename K>
static cudaError_t launch_cluster(K kernel, int64_t clusters, int c, size_t smem, const PlaneArgs &a,
                                  cudaStream_t s, bool &attr_done) {
    if (!attr_done) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_done = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * c), 1, 1);
    cfg.blockDim = dim3(PLANE_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, a);
}

// The shared-memory attribute is a per-device property of the kernel; it is set
// on the first launch of each instantiation (one device per process here).
template <int N1, int N2, int C>
static cudaError_t plane_pass_impl(const PlaneArgs &a, cudaStream_t s) {
    static bool attr_done = false;
    return launch_cluster(k_plane_pass<N1, N2, C>, a.planes, C, PlaneCfg<N1, N2, C>::SMEM, a, s, attr_done);
}

template <int N1, int N2, int C, int MINB = 2>
static cudaError_t plane_whole_impl(const PlaneArgs &a, cudaStream_t s) {
    static bool attr_done = false;
    return launch_cluster(k_plane_whole<N1, N2, C, MINB>, a.batch, C, PlaneCfg<N1, N2, C>::SMEM, a, s, attr_done);
}

// Cluster size per distributed-axis length: R = 32 rows per CTA (16 for 32).
__host__ __device__ constexpr int plane_c(int n1) { return n1 >= 256 ? 8 : n1 >= 128 ? 4 : n1 >= 64 ? 2 : n1 >= 32 ? 2 : 0; }

bool plane_supported(int n1, int n2) {
    return (n1 == 32 || n1 == 64 || n1 == 128 || n1 == 256) && (n2 == 32 || n2 == 64 || n2 == 128 || n2 == 256);
}

int plane_cluster(int n1) { return plane_c(n1); }

#define QHD_PLANE_DISPATCH(fn)                                                        \
    switch (n1 * 1000 + n2) {                                                         \
    case 32032: return fn<32, 32, plane_c(32)>(a, s);                                 \
    case 32064: return fn<32, 64, plane_c(32)>(a, s);                                 \
    case 32128: return fn<32, 128, plane_c(32)>(a, s);                                \
    case 32256: return fn<32, 256, plane_c(32)>(a, s);                                \
    case 64032: return fn<64, 32, plane_c(64)>(a, s);                                 \
    case 64064: return fn<64, 64, plane_c(64)>(a, s);                                 \
    case 64128: return fn<64, 128, plane_c(64)>(a, s);                                \
    case 64256: return fn<64, 256, plane_c(64)>(a, s);                                \
    case 128032: return fn<128, 32, plane_c(128)>(a, s);                              \
    case 128064: return fn<128, 64, plane_c(128)>(a, s);                              \
    case 128128: return fn<128, 128, plane_c(128)>(a, s);                             \
    case 128256: return fn<128, 256, plane_c(128)>(a, s);                             \
    case 256032: return fn<256, 32, plane_c(256)>(a, s);                              \
    case 256064: return fn<256, 64, plane_c(256)>(a, s);                              \
    case 256128: return fn<256, 128, plane_c(256)>(a, s);                             \
    case 256256: return fn<256, 256, plane_c(256)>(a, s);                             \
    default: return cudaErrorInvalidValue;                                            \
    }

cudaError_t launch_plane_pass(int n1, int n2, const PlaneArgs &a, cudaStream_t s) {
    QHD_PLANE_DISPATCH(plane_pass_impl)
}

cudaError_t launch_plane_whole(int n1, int n2, const PlaneArgs &a, cudaStream_t s) {
    QHD_PLANE_DISPATCH(plane_whole_impl)
}

// The whole-run kernel with twice the CTAs per instance (half the rows each) for
// distributed axes of 64 and 128: a batch too small to fill the GPU then runs on
// twice the SMs.
__host__ __device__ constexpr int plane_c_wide(int n1) { return n1 == 128 ? 8 : n1 == 64 ? 4 : 0; }

int plane_cluster_wide(int n1) { return plane_c_wide(n1); }

cudaError_t launch_plane_whole_wide(int n1, int n2, const PlaneArgs &a, cudaStream_t s) {
    switch (n1 * 1000 + n2) {
    case 64032: return plane_whole_impl<64, 32, plane_c_wide(64), 1>(a, s);
    case 64064: return plane_whole_impl<64, 64, plane_c_wide(64), 1>(a, s);
    case 64128: return plane_whole_impl<64, 128, plane_c_wide(64), 1>(a, s);
    case 64256: return plane_whole_impl<64, 256, plane_c_wide(64), 1>(a, s);
    case 128032: return plane_whole_impl<128, 32, plane_c_wide(128), 1>(a, s);
    case 128064: return plane_whole_impl<128, 64, plane_c_wide(128), 1>(a, s);
    case 128128: return plane_whole_impl<128, 128, plane_c_wide(128), 1>(a, s);
    case 128256: return plane_whole_impl<128, 256, plane_c_wide(128), 1>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace qhd
