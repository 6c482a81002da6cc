// qhd_probe.cu -- arithmetic throughput probe used to state roofline peaks.
//
// The box-mesh passes are bound by 32 x 32 -> 64-bit integer multiply-adds,
// the Fourier-mesh passes by FP32 FMAs; the observables reduce in FP64 and the
// phases use the special-function unit.  None of these rates is a published
// figure for this part, so they are measured: every thread runs eight
// independent dependency chains of one operation, enough warps to fill every
// SM, timed with CUDA events.
#include <cuda_runtime.h>

#include "qhd_probe.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_ITERS = 8192;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_ffma(float *out, float a, float b, int keep) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fmaf(x[k], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (keep) out[0] = s;  // keep = 0: never stores, but the compiler cannot know
}

// acc += (low 32 bits of acc) * a: one 32 x 32 -> 64-bit multiply-add per step
// whose operand depends on the previous step, so no closed form exists.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_imad_wide(long long *out, int a, int keep) {
    long long x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (long long)(threadIdx.x * 8 + k + 1);
    for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] += (long long)(int)x[k] * a;
    }
    long long s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s ^= x[k];
    if (keep) out[0] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_dfma(double *out, double a, double b, int keep) {
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (double)(threadIdx.x + k) * 1e-3;
    for (int it = 0; it < PROBE_ITERS / 8; ++it) {  // FP64 is slow: fewer steps
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (keep) out[0] = s;
}

// The special-function unit: one hardware sine approximation per step.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_sfu(float *out, float a, int keep) {
    float x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = __sinf(x[k] + a);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (keep) out[0] = s;
}

}  // namespace

extern "C" int qhd_probe_alu_rates(double *out) {
    constexpr int OK = 0, ERR_INVALID_ARG = 1, ERR_CUDA = 4;
    if (!out) return ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return ERR_CUDA;
    const int blocks = sms * 16;
    const size_t n = (size_t)blocks * PROBE_THREADS;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int st = OK;
    float ms[4] = {0.f, 0.f, 0.f, 0.f};
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) st = ERR_CUDA;
    for (int kind = 0; kind < 4 && st == OK; ++kind) {
        for (int rep = 0; rep < 2 && st == OK; ++rep) {  // the first run warms up
            cudaEventRecord(e0);
            if (kind == 0) k_probe_ffma<<<blocks, PROBE_THREADS>>>(nullptr, 0.999f, 1e-4f, 0);
            else if (kind == 1) k_probe_imad_wide<<<blocks, PROBE_THREADS>>>(nullptr, 3, 0);
            else if (kind == 2) k_probe_dfma<<<blocks, PROBE_THREADS>>>(nullptr, 0.999, 1e-4, 0);
            else k_probe_sfu<<<blocks, PROBE_THREADS>>>(nullptr, 0.5f, 0);
            cudaEventRecord(e1);
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms[kind], e0, e1) != cudaSuccess)
                st = ERR_CUDA;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st != OK) return st;
    const double ops = (double)n * PROBE_ITERS * 8;
    out[0] = ops / (ms[0] * 1e-3);        // FP32 FMAs per second
    out[1] = ops / (ms[1] * 1e-3);        // 32x32->64 integer multiply-adds per second
    out[2] = ops / 8 / (ms[2] * 1e-3);    // FP64 FMAs per second
    out[3] = ops / (ms[3] * 1e-3);        // hardware sine approximations per second
    return OK;
}
