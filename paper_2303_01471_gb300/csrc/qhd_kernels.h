// qhd_kernels.h -- launch interface between the host library and the kernels.
// Host-only declarations; the kernels themselves live in qhd_kernels.cu.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qhd {

// Pass modes.
enum : int { MODE_FWD = 1, MODE_INV = 2, MODE_KIN = 4 };

// Damping schedule as the device evaluates it (one per instance).
struct SchedDev {
    int32_t kind;  // 0 Nesterov, 1 table, 2 power family
    int32_t ns;    // table samples
    double c_phi, eps, c_chi;
    const double *t, *phi, *chi;  // workspace copies of the samples
    double power;  // power family: p
};

// Per-instance potential data written by set_potential.
struct InstDev {
    double fmin;     // offset of the fixed-point potential
    int32_t shift;   // fq = rint((f - fmin) * 2^shift)
    int32_t pad_;
    double xs[3];    // grid minimiser coordinates
};

// Per-block partial of the min/max/argmin reduction over f.
struct MinMaxPart {
    double fmin, fmax;
    int64_t argmin;
    int64_t nonfinite;
};

struct RowArgs {
    float2 *psi;
    const uint32_t *fq;
    const uint64_t *pot;   // potential coefficient of this pass, one per instance
    const float4 *tw2;
    int64_t rows;          // batch * rows per instance
    int64_t rows_per_inst;
    int mode;              // MODE_INV: inverse FFT before the phase; MODE_FWD: forward after
    uint32_t dither;       // global phase of this pass in 2^-32 turns (step_dither)
    const float4 *ptab;    // potential phase table (PHASE_TAB hi/lo entries)
};

struct AxisArgs {
    float2 *psi;
    const float4 *tw2;
    const float4 *kt;      // kinetic tables of this step: [batch][ksum] (MODE_KIN only)
    int64_t inner;         // product of the axis lengths after this axis (line stride)
    int64_t planes;        // product of batch and the axis lengths before this axis
    int ksum;              // sum of the axis lengths
    int koff1, koff2;      // table offsets of axes 1 and 2
    int log_n2;            // log2 n[2] (3-D only)
    int ndim;
    int mode;
    int64_t kt_batch;      // 1: every instance shares the kinetic table; else batch
    int perm1_r, perm1_c;  // 3-D after a plane pass: stored axis-1 row s holds
                           // frequency s / perm1_r + perm1_c * (s % perm1_r); 0 = natural
};

// Plane engine (qhd_plane.cu): N1 distributed over a cluster, N2 per row.
struct PlaneArgs {
    float2 *psi;
    const uint32_t *fq;
    const uint64_t *pot;     // pass: coefficients of this pass [batch]; whole: chunk [cnt+1][batch]
    const float4 *kt;        // whole: chunk kinetic tables [cnt][batch][ksum]
    const float4 *tw_row;    // stage-2 twiddles of the row length
    const float4 *twx;       // exchange twiddles twx[q*R + n2] = exp(-2 pi i n2 q / N1), (hi, lo)
    int64_t planes;          // pass: batch * n0 planes
    int64_t planes_per_inst; // pass: n0
    int64_t batch;
    int mode;                // pass: MODE_INV (previous step's inverse first), MODE_FWD
    uint32_t dither;         // pass: global phase of this step
    int cnt;                 // whole: steps in the chunk
    int final_phase;         // whole: apply pot[cnt] at the end
    int ksum;
    uint64_t dither_base;    // whole: global index of the chunk's first step
    const float4 *ptab;      // potential phase table
    int64_t kt_batch;        // whole: 1 = shared kinetic table, else batch
};

struct OneDArgs {
    float2 *psi;
    const uint32_t *fq;
    const uint64_t *pot;   // chunk potential coefficients [cnt+1][batch]
    const float4 *kt;      // chunk kinetic tables [cnt][batch][n]
    const float4 *tw2;
    int64_t batch;
    int cnt;
    int final_phase;       // apply pot[cnt] after the last step
    uint64_t dither_base;  // global step index of the chunk's first step
    const float4 *ptab;    // potential phase table
    int64_t kt_batch;      // 1: shared kinetic table; else batch
};

struct PrepArgs {
    const SchedDev *sched;
    const InstDev *inst;
    uint64_t *pot;         // [cnt+1][batch]
    float4 *kt;            // [cnt][kt_batch][ksum], (hi.re, hi.im, lo.re, lo.im)
    int64_t kt_batch;      // 1 when every instance has the same kinetic schedule
    double t_start, dt;
    int64_t j0, cnt, nsteps, batch;
    int ndim;
    int n[3];
    double len[3];
    int koff[3];
    int ksum;
    double inv_g;          // 1/G (exact power of two)
    int split;             // 0 Strang (midpoint, merged halves), 1 first-order Lie-Trotter
    int kinetic;           // 0 spectral |k|^2, 1 central second difference (4/h^2) sin^2(pi m/N)
};

struct ObsArgs {
    const float2 *psi;
    const double *f64;
    const InstDev *inst;
    const double *coord;   // mesh coordinates per axis, concatenated
    float *prob;           // optional
    double *partial;       // [batch][nblk][3]
    double *result;        // [batch][3]
    int64_t g;
    int ndim;
    int n[3];
    int log_n[3];
    int coff[3];
    double radius;
    int nblk;
};

// Launchers; each returns the launch error (cudaSuccess on success).
cudaError_t launch_row(int n, const RowArgs &a, cudaStream_t s);
cudaError_t launch_axis(int n, const AxisArgs &a, cudaStream_t s);
cudaError_t launch_oned(int n, const OneDArgs &a, cudaStream_t s);
cudaError_t launch_prep(const PrepArgs &a, cudaStream_t s);
cudaError_t launch_uniform(float2 *psi, int64_t count, float value, cudaStream_t s);
cudaError_t launch_minmax(const double *f, int64_t g, int64_t batch, MinMaxPart *part, int nblk,
                          cudaStream_t s);
cudaError_t launch_quantize(const double *f, uint32_t *fq, const InstDev *inst, int64_t g,
                            int64_t batch, cudaStream_t s);
cudaError_t launch_observables(const ObsArgs &a, int64_t batch, cudaStream_t s);
cudaError_t launch_plane_pass(int n1, int n2, const PlaneArgs &a, cudaStream_t s);
cudaError_t launch_plane_whole(int n1, int n2, const PlaneArgs &a, cudaStream_t s);
bool plane_supported(int n1, int n2);
int plane_cluster(int n1);
// Whole-run kernel with twice the CTAs per instance (distributed axis 64 or 128; 0: none).
int plane_cluster_wide(int n1);
cudaError_t launch_plane_whole_wide(int n1, int n2, const PlaneArgs &a, cudaStream_t s);

// Plans shared with the host (twiddle tables are built on the host).
void plan_of(int n, int *r1, int *r2);
bool supported_n(int64_t n);

}  // namespace qhd
