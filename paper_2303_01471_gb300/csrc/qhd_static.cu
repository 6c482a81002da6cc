// qhd_static.cu -- observables of caller-provided states without any device
// allocation: the reduction scratch is a fixed array in this file.
//
// Who needs this: callers that cannot call cudaMalloc at the point where they
// want observables -- for example a host application whose device memory is
// entirely reserved by another allocator (so a new allocation would fail or
// fragment that pool), or a latency-critical caller that must not pay for
// cudaMalloc, which can synchronise the device.  Such a caller passes the
// state, the FP64 objective and an output buffer it already owns, and this
// entry point uses nothing else.
#include <cmath>
#include <cstring>
#include <mutex>

#include "qhd.h"
#include "qhd_device.cuh"
#include "qhd_kernels.h"

using namespace qhd;

namespace {

constexpr int S_MAX_BATCH = 32;
constexpr int S_MAX_AXIS = 1024;
constexpr int S_MAX_BLOCKS = 1024;

// Layout of the fixed scratch: per-instance data, mesh coordinates, results,
// per-block partial sums.  Every call overwrites each part before reading it.
constexpr size_t S_INST_OFF = 0;
constexpr size_t S_COORD_OFF = S_INST_OFF + sizeof(InstDev) * S_MAX_BATCH;
constexpr size_t S_RES_OFF = S_COORD_OFF + sizeof(double) * 3 * S_MAX_AXIS;
constexpr size_t S_PART_OFF = S_RES_OFF + sizeof(double) * 3 * S_MAX_BATCH;
constexpr size_t S_TOTAL = S_PART_OFF + sizeof(double) * 3 * S_MAX_BLOCKS * S_MAX_BATCH;

static_assert(S_INST_OFF % 16 == 0 && S_COORD_OFF % 16 == 0 && S_RES_OFF % 16 == 0 && S_PART_OFF % 16 == 0,
              "scratch parts must stay aligned");

// QHD_STATIC_SCRATCH_BYTES (include/qhd.h) is the public upper bound.
static_assert(S_TOTAL <= QHD_STATIC_SCRATCH_BYTES, "scratch exceeds the documented maximum");

}  // namespace

// The scratch itself.  Every device that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_obs_scratch[QHD_STATIC_SCRATCH_BYTES];

namespace {

struct SetupParams {
    int ndim;
    int n[3];
    double lo[3], hi[3];
    int batch;
    double xs[S_MAX_BATCH][3];
};

// Writes the per-instance minimiser coordinates and the mesh coordinates
// x = lo + (j (hi - lo)) / N into the scratch (same operation order as the
// context path's host-side table).
__global__ void k_static_setup(SetupParams p, unsigned char *scratch) {
    InstDev *inst = (InstDev *)(scratch + S_INST_OFF);
    double *coord = (double *)(scratch + S_COORD_OFF);
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    if (tid < p.batch) {
        InstDev d;
        d.fmin = 0.0;
        d.shift = 0;
        d.pad_ = 0;
        for (int k = 0; k < 3; ++k) d.xs[k] = p.xs[tid][k];
        inst[tid] = d;
    }
    int off = 0;
    for (int ax = 0; ax < p.ndim; ++ax) {
        if (tid < p.n[ax])
            coord[off + tid] =
                __dadd_rn(p.lo[ax], __ddiv_rn(__dmul_rn((double)tid, __dsub_rn(p.hi[ax], p.lo[ax])), (double)p.n[ax]));
        off += p.n[ax];
    }
}

std::mutex g_mu;
void *g_dev_ptr[128] = {};

// Device address of g_obs_scratch for the current device, looked up once per
// device with that device current.
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_obs_scratch);
        if (e != cudaSuccess) return e;
        g_dev_ptr[dev] = ptr;
    }
    *out = g_dev_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" qhd_status qhd_observables_static(int ndim, const int64_t *n, const double *lo, const double *hi,
                                             int64_t batch, const void *psi_dev, const double *f_dev,
                                             const double *x_star, double radius, double *out_dev,
                                             float *prob_dev, void *stream) {
    if (ndim < 1 || ndim > 3 || !n || !lo || !hi || !psi_dev || !f_dev || !x_star || !out_dev)
        return QHD_ERR_INVALID_ARG;
    if (batch < 1 || batch > S_MAX_BATCH) return QHD_ERR_INVALID_ARG;
    if (!std::isfinite(radius) || !(radius > 0)) return QHD_ERR_INVALID_ARG;
    int64_t g = 1;
    for (int d = 0; d < ndim; ++d) {
        if (!supported_n(n[d]) || n[d] > S_MAX_AXIS) return QHD_ERR_INVALID_ARG;
        if (!std::isfinite(lo[d]) || !std::isfinite(hi[d]) || !(lo[d] < hi[d])) return QHD_ERR_INVALID_ARG;
        g *= n[d];
    }
    int nblk = (int)((g + 255) / 256);
    if (nblk > S_MAX_BLOCKS) nblk = S_MAX_BLOCKS;

    void *base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return QHD_ERR_CUDA;
    unsigned char *scratch = (unsigned char *)base;
    cudaStream_t s = (cudaStream_t)stream;

    SetupParams sp{};
    sp.ndim = ndim;
    sp.batch = (int)batch;
    for (int d = 0; d < ndim; ++d) {
        sp.n[d] = (int)n[d];
        sp.lo[d] = lo[d];
        sp.hi[d] = hi[d];
    }
    for (int64_t b = 0; b < batch; ++b)
        for (int k = 0; k < 3; ++k) sp.xs[b][k] = k < ndim ? x_star[3 * b + k] : 0.0;
    k_static_setup<<<(S_MAX_AXIS + 255) / 256, 256, 0, s>>>(sp, scratch);
    if (cudaGetLastError() != cudaSuccess) return QHD_ERR_CUDA;

    ObsArgs a{};
    a.psi = (const float2 *)psi_dev;
    a.f64 = f_dev;
    a.inst = (const InstDev *)(scratch + S_INST_OFF);
    a.coord = (const double *)(scratch + S_COORD_OFF);
    a.prob = prob_dev;
    a.partial = (double *)(scratch + S_PART_OFF);
    a.result = (double *)(scratch + S_RES_OFF);
    a.g = g;
    a.ndim = ndim;
    int off = 0;
    for (int d = 0; d < 3; ++d) {
        a.n[d] = d < ndim ? (int)n[d] : 1;
        a.log_n[d] = d < ndim ? (int)std::log2((double)n[d]) : 0;
        a.coff[d] = d < ndim ? off : 0;
        if (d < ndim) off += (int)n[d];
    }
    a.radius = radius;
    a.nblk = nblk;
    if (launch_observables(a, batch, s) != cudaSuccess) return QHD_ERR_CUDA;
    if (cudaMemcpyAsync(out_dev, scratch + S_RES_OFF, sizeof(double) * 3 * (size_t)batch,
                        cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return QHD_ERR_CUDA;
    return QHD_OK;
}
