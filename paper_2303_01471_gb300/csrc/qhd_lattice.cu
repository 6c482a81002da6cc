// qhd_lattice.cu -- QHD on the finite-difference box mesh (the Sim-QHD solver).
//
// The semi-discrete QHD equation of the paper's finite-difference
// discretisation, Eq. (finite-qhd-discrete), and of its relaxed form,
// Eq. (relaxed-qhd-discrete):
//     i d/dt phi = [ a(t) sum_k K_k + b(t) F ] phi,      K = -(r^2 / 2) A,
// on the mesh {0, 1/r, ..., 1}^d (n = r + 1 points per axis), A the chain
// adjacency of Eq. (discretize-pde) or the relaxed A' of Eq. (relaxed_adjacency).
// One Strang step with the coefficients at the step midpoint is
//     phi <- P(dt b/2) [prod_k U_k] P(dt b/2) phi,      U = exp(-i dt a K),
// where U_k is U acting along axis k: the axis terms commute, so the kinetic
// factor is the same dense n x n unitary along every axis.  Consecutive half
// potential phases merge as on the Fourier mesh (theta_j = dt (b_{j-1}+b_j)/2).
//
// A step is one pass per group of consecutive axes.  A pass holds tiles of psi
// in shared memory, each tile a set of columns that contain whole lines of the
// group's axes, and applies U along each axis of the group in place.  The
// group of the last axes is contiguous in memory (its columns are consecutive
// blocks of P points); the others are strided (their columns are consecutive
// inner indices, read as W-wide row segments).  The first pass applies the
// merged potential phase on load; the last pass of an evolve call applies the
// final half phase on store.  U is computed per step in FP64 from the host's
// eigendecomposition of A (U = V diag(exp(i dt a r^2/2 lambda)) V^T).  The
// state is fixed point (see below), which keeps the norm to a few 1e-7 at most
// over 10^3 steps where FP32 storage drifts by several 1e-6 on concentrated
// states.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qhd.h"
#include "qhd_device.cuh"
#include "qhd_kernels.h"
#include "qhd_sched.cuh"
#include "qhd_trace.h"

using namespace qhd;

namespace {

constexpr int LAT_MAX_D = 6;
constexpr int LAT_MAX_R = 16;
constexpr int LAT_MAX_N = LAT_MAX_R + 1;
constexpr int GROUP_MAX = 1024;          // points of one column (the group's axes)
constexpr int TILE_MAX = 4608;           // points of one tile (36 KB): with 64 registers, 4 CTAs per SM
constexpr int PASS_THREADS_MAX = 256;
constexpr int64_t LAT_MAX_CHUNK = 1024;
constexpr size_t U_BUDGET = size_t(64) << 20;  // bytes of propagators per chunk
constexpr int OBS_BLOCKS_MAX = 1024;
constexpr int MINMAX_BLOCKS_MAX = 512;

// ------------------------------------------------------------------ kernels
// The working state is fixed point: each amplitude component is an int32 in
// units of 2^-29 (|psi| <= 1 by unitarity, so |component| <= 2^29, and the
// sums re + im of the three-product complex multiply stay below 2^31).  A line
// transform forms every output as an exact int64 sum of int32 x int32 products
// and rounds it once; the potential phase is an exact int64 complex product
// rounded once.  Every stored value therefore carries one
// rounding of at most 2^-30 absolute, independent of how concentrated the state
// is, where FP32 storage carries 2^-24 relative on the few dominant amplitudes
// of a concentrated state.
constexpr int FX_SHIFT = 30;                 // scale of U and of the phase factors: Q1.30
constexpr double FX_ONE = 1073741824.0;      // 2^30
constexpr double FX_STATE = 536870912.0;     // 2^29: the state is Q2.29 (one bit of headroom for
                                             // the sums of the three-product complex multiply)

__device__ __forceinline__ int fx_round(long long v) {
    return (int)((v + (1ll << (FX_SHIFT - 1))) >> FX_SHIFT);
}

// Potential phase table: T[k] = exp(-2 pi i k / PHASE_TAB) as Q1.30 (rounded
// from FP64) and as FP32 (for the small correction term).
struct LatPhase {
    int2 fx;
    float2 f;
};

// z * exp(-2 pi i u / 2^32) in fixed point.  u = 2^24 k + r as in the FP32
// path: exp(-2 pi i u / 2^32) = T[k] (1 + eps), eps = exp(-i delta) - 1 with
// delta = 2 pi r / 2^32, |delta| <= pi / 256, from its Taylor series.  T[k] eps
// is below 0.0123 in modulus, so its FP32 value times 2^30 is below 2^24 and
// converts with an error of about one unit; the factor is accurate to ~2^-30.
__device__ __forceinline__ int2 fx_phase(int2 z, uint32_t u, const LatPhase *tab) {
    const uint32_t k = ((u + (1u << 23)) >> 24) & (PHASE_TAB - 1);
    const int32_t r = (int32_t)(u - (k << 24));
    const float d = (float)r * 1.4629180792671596e-09f;  // 2 pi / 2^32
    const float d2 = d * d;
    const float cm1 = d2 * fmaf(d2, 1.0f / 24.0f, -0.5f);  // cos d - 1
    const float sn = d * fmaf(d2, -1.0f / 6.0f, 1.0f);     // sin d
    const LatPhase t = tab[k];
    const float er = fmaf(t.f.x, cm1, t.f.y * sn), ei = fmaf(t.f.y, cm1, -t.f.x * sn);
    const long long wr = t.fx.x + __float2int_rn(er * (float)FX_ONE);
    const long long wi = t.fx.y + __float2int_rn(ei * (float)FX_ONE);
    return make_int2(fx_round(z.x * wr - z.y * wi), fx_round(z.x * wi + z.y * wr));
}

struct LatPass {
    int2 *psi;                 // state, units of 2^-29
    const uint32_t *fq;
    const uint64_t *pot_pre;   // [batch] phase coefficient applied on load, or null
    const uint64_t *pot_post;  // [batch] applied on store, or null
    uint32_t dither_pre, dither_post;
    const int4 *U;             // this step's propagator blocks [u_batch][M*M + H*H]: (re, im, re + im, 0), Q1.30
    int64_t u_batch;
    const LatPhase *ptab;
    int P, q, W, pitch, lines_per_col;
    int64_t col_count, col_stride, g_stride, row_stride, rows_per_inst, tiles_per_row;
    uint64_t mg_P, mg_W, mg_lpc;   // reciprocals for division by P, W, lines_per_col
    uint64_t mg_s[12];             // ... and by the group strides N^ax
};

// floor(l / d) for l < 2^16 and 1 <= d <= 2^13 from mg = floor(2^32 / d) + 1
// (exact in that range: l * (mg - 2^32/d) / 2^32 < 2^-16 < 1/d).
__host__ __device__ __forceinline__ uint64_t lat_magic(uint32_t d) { return (uint64_t(1) << 32) / d + 1; }
__device__ __forceinline__ int lat_div(int l, uint64_t mg) { return (int)(((uint64_t)(uint32_t)l * mg) >> 32); }

// Shared-memory index of group point g: even line lengths get one pad slot per
// line so that threads walking lines of stride 1 hit distinct banks.
template <int N>
__device__ __forceinline__ int lat_idx(int g) {
    return (N & 1) ? g : g + g / N;
}

// Both per-axis operators commute with the reversal j -> n-1-j, and so does U.
// With s_m = x_m + x_{n-1-m}, a_m = x_m - x_{n-1-m} (m < H = n/2; s_H = x_H for
// odd n), y = U x is
//     y_i = S_i + A_i,  y_{n-1-i} = S_i - A_i  (i < H),   y_H = S_H  (odd n),
//     S = Ps s,  A = Pa a,   Ps_{im} = (U_{im} + U_{i,n-1-m}) / 2  (Ps_{iH} = U_{iH}),
//     Pa_{im} = (U_{im} - U_{i,n-1-m}) / 2,
// an M x M and an H x H block (M = n - H) instead of n x n: 41 products for
// n = 9 rather than 81.  s and a are exact integer sums; each output is one
// exact int64 sum rounded once.
template <int N>
__global__ void __launch_bounds__(PASS_THREADS_MAX, N <= 9 ? 4 : 2) k_lat_pass(LatPass a) {
    constexpr int H = N / 2, M = N - H;
    extern __shared__ __align__(16) LatPhase lsm[];
    LatPhase *ptab = lsm;
    int4 *Ps = reinterpret_cast<int4 *>(lsm + PHASE_TAB);
    int4 *Pa = Ps + M * M;
    int2 *tile = reinterpret_cast<int2 *>(Pa + H * H);
    const int64_t row = blockIdx.x / a.tiles_per_row;
    const int64_t c0 = (blockIdx.x - row * a.tiles_per_row) * a.W;
    const int64_t inst = row / a.rows_per_inst;
    if (a.pot_pre || a.pot_post)
        for (int i = threadIdx.x; i < PHASE_TAB; i += blockDim.x) ptab[i] = a.ptab[i];
    const int4 *Ug = a.U + (a.u_batch == 1 ? 0 : inst) * (M * M + H * H);
    for (int i = threadIdx.x; i < M * M + H * H; i += blockDim.x) Ps[i] = __ldg(&Ug[i]);
    __syncthreads();
    const int P = a.P, W = a.W, pitch = a.pitch;
    const int64_t left = a.col_count - c0;
    const int ncol = left < W ? (int)left : W;
    const int64_t base = row * a.row_stride + c0 * a.col_stride;
    const bool contig = a.g_stride == 1;
    const int tot = P * W;
    {
        // four loads in flight per thread before their results are used
        constexpr int UNR = 4;
        const uint64_t c = a.pot_pre ? a.pot_pre[inst] : 0;
        for (int l0 = threadIdx.x; l0 < tot; l0 += UNR * blockDim.x) {
            int2 v[UNR];
            uint32_t q[UNR];
            int si[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const int l = l0 + u * blockDim.x;
                int g, col;
                if (contig) {
                    col = lat_div(l, a.mg_P);
                    g = l - col * P;
                } else {
                    g = lat_div(l, a.mg_W);
                    col = l - g * W;
                }
                si[u] = -1;
                q[u] = 0;
                if (l < tot && col < ncol) {
                    const int64_t off = base + col * a.col_stride + (int64_t)g * a.g_stride;
                    v[u] = a.psi[off];
                    if (a.pot_pre) q[u] = __ldg(&a.fq[off]);
                    si[u] = col * pitch + lat_idx<N>(g);
                }
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                if (si[u] < 0) continue;
                int2 w = v[u];
                if (a.pot_pre) w = fx_phase(w, turns_mul(c, q[u]) + a.dither_pre, ptab);
                tile[si[u]] = w;
            }
        }
    }
    __syncthreads();
    const int lpc = a.lines_per_col;
    const int lines = lpc * W;
    int s = 1;  // stride of the current axis inside the group (last axis first)
    for (int ax = 0; ax < a.q; ++ax, s *= N) {
        const uint64_t mg_s = a.mg_s[ax];
        for (int l = threadIdx.x; l < lines; l += blockDim.x) {
            const int col = lat_div(l, a.mg_lpc);
            const int h = l - col * lpc;
            if (col >= ncol) continue;
            const int hs = lat_div(h, mg_s);
            const int g0 = hs * (s * N) + (h - hs * s);
            int2 *cb = tile + col * pitch;
            int2 x[N];
#pragma unroll
            for (int m = 0; m < N; ++m) x[m] = cb[lat_idx<N>(g0 + m * s)];
            // (s, a) and their re + im sums; |s|^2 + |a|^2 <= 4 |x|^2 keeps every sum
            // below 2^31 at the 2^-29 scale
            int3 sv[M], av[H];
#pragma unroll
            for (int m = 0; m < H; ++m) {
                const int sx = x[m].x + x[N - 1 - m].x, sy = x[m].y + x[N - 1 - m].y;
                const int ax = x[m].x - x[N - 1 - m].x, ay = x[m].y - x[N - 1 - m].y;
                sv[m] = make_int3(sx, sy, sx + sy);
                av[m] = make_int3(ax, ay, ax + ay);
            }
            if (N & 1) sv[M - 1] = make_int3(x[H].x, x[H].y, x[H].x + x[H].y);
            int2 y[N];
#pragma unroll
            for (int i = 0; i < M; ++i) {
                // three products per complex term (Gauss): with k1 = ur vr, k2 = ui vi,
                // k3 = (ur + ui)(vr + vi):  re = k1 - k2,  im = k3 - k1 - k2
                long long s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const int4 u = Ps[i * M + m];
                    s1 += (long long)u.x * sv[m].x;
                    s2 += (long long)u.y * sv[m].y;
                    s3 += (long long)u.z * sv[m].z;
                }
                const long long sr = s1 - s2, si = s3 - s1 - s2;
                if (i < H) {
                    long long a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
                    for (int m = 0; m < H; ++m) {
                        const int4 u = Pa[i * H + m];
                        a1 += (long long)u.x * av[m].x;
                        a2 += (long long)u.y * av[m].y;
                        a3 += (long long)u.z * av[m].z;
                    }
                    const long long ar = a1 - a2, ai = a3 - a1 - a2;
                    y[i] = make_int2(fx_round(sr + ar), fx_round(si + ai));
                    y[N - 1 - i] = make_int2(fx_round(sr - ar), fx_round(si - ai));
                } else {
                    y[i] = make_int2(fx_round(sr), fx_round(si));
                }
            }
#pragma unroll
            for (int m = 0; m < N; ++m) cb[lat_idx<N>(g0 + m * s)] = y[m];
        }
        __syncthreads();
    }
    {
        const uint64_t c = a.pot_post ? a.pot_post[inst] : 0;
        for (int l = threadIdx.x; l < tot; l += blockDim.x) {
            int g, col;
            if (contig) {
                col = lat_div(l, a.mg_P);
                g = l - col * P;
            } else {
                g = lat_div(l, a.mg_W);
                col = l - g * W;
            }
            if (col >= ncol) continue;
            const int64_t off = base + col * a.col_stride + (int64_t)g * a.g_stride;
            int2 v = tile[col * pitch + lat_idx<N>(g)];
            if (a.pot_post) v = fx_phase(v, turns_mul(c, __ldg(&a.fq[off])) + a.dither_post, ptab);
            a.psi[off] = v;
        }
    }
}

struct LatPrep {
    const SchedDev *sched;
    const InstDev *inst;
    uint64_t *pot;       // [cnt+1][batch]
    int4 *U;             // [cnt][u_batch][M*M + H*H]
    const double *V;     // eigenvectors of A, V[i*n + k] = component i of vector k
    const double *lam;   // eigenvalues of A
    double kin_scale;    // r^2 / 2
    double t_start, dt;
    int64_t j0, cnt, nsteps, batch, u_batch;
    uint64_t step_base;  // global index of the chunk's first step (rounding dither)
    int n;
};

// Unbiased rounding of U to Q1.30: floor(U 2^30 + v) with v uniform in [0,1)
// from a counter hash of (step, entry), so that the rounding error of a matrix
// that changes little from step to step does not repeat coherently.
__device__ __forceinline__ int fx_dither_round(double v, uint64_t key) {
    const uint32_t h = step_dither(key);
    return (int)floor(v * FX_ONE + (double)h * 2.3283064365386963e-10);
}

__global__ void k_lat_prep(LatPrep a) {
    const int64_t jl = blockIdx.x;  // local step 0..cnt (cnt: the final half phase)
    const int64_t b = blockIdx.y;
    const int64_t j = a.j0 + jl;
    __shared__ double s_c[LAT_MAX_N], s_s[LAT_MAX_N];
    __shared__ double s_a;
    if (threadIdx.x == 0) {
        const SchedDev &sd = a.sched[b];
        const double PI = 3.141592653589793238462643383279502884;
        double a_m = 0, b_m = 0, a_p = 0, b_p = 0;
        if (j >= 1) {
            const double tm = __dadd_rn(a.t_start, __dmul_rn((double)(j - 1) + 0.5, a.dt));
            sched_eval_dev(sd, tm, &a_m, &b_m);
        }
        if (j < a.nsteps) {
            const double tp = __dadd_rn(a.t_start, __dmul_rn((double)j + 0.5, a.dt));
            sched_eval_dev(sd, tp, &a_p, &b_p);
        }
        const double theta = __dmul_rn(a.dt, __dadd_rn(j >= 1 ? b_m : 0.0, j < a.nsteps ? b_p : 0.0)) * 0.5;
        // turns per unit of the fixed-point potential: theta / (2 pi) * 2^-shift
        a.pot[jl * a.batch + b] = frac_to_u64(ldexp(theta / (2.0 * PI), -a.inst[b].shift));
        s_a = a_p;
    }
    __syncthreads();
    if (jl >= a.cnt || b >= a.u_batch) return;
    const int n = a.n;
    if (threadIdx.x < n) {
        // eigenphase of U: exp(-i dt a K) = V diag(exp(+i dt a (r^2/2) lambda)) V^T
        const double ph = __dmul_rn(__dmul_rn(__dmul_rn(a.dt, s_a), a.kin_scale), a.lam[threadIdx.x]);
        sincos(ph, &s_s[threadIdx.x], &s_c[threadIdx.x]);
    }
    __syncthreads();
    __shared__ double s_ur[LAT_MAX_N * LAT_MAX_N], s_ui[LAT_MAX_N * LAT_MAX_N];
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, m = e - (e / n) * n;
        double re = 0.0, im = 0.0;
        for (int k = 0; k < n; ++k) {
            const double w = __dmul_rn(a.V[i * n + k], a.V[m * n + k]);
            re = __dadd_rn(re, __dmul_rn(w, s_c[k]));
            im = __dadd_rn(im, __dmul_rn(w, s_s[k]));
        }
        s_ur[e] = re;
        s_ui[e] = im;
    }
    __syncthreads();
    // reversal-symmetric blocks Ps (M x M) and Pa (H x H) of U, see k_lat_pass
    const int H = n / 2, M = n - H;
    int4 *out = a.U + (jl * a.u_batch + b) * (int64_t)(M * M + H * H);
    const uint64_t key0 = ((a.step_base + (uint64_t)jl) * 0x100000001B3ull) ^ ((uint64_t)b * 0x9E3779B97F4A7C15ull);
    for (int e = threadIdx.x; e < M * M + H * H; e += blockDim.x) {
        double re, im;
        if (e < M * M) {
            const int i = e / M, m = e - (e / M) * M;
            if (m == H) {  // odd n: the middle column
                re = s_ur[i * n + H];
                im = s_ui[i * n + H];
            } else {
                re = 0.5 * (s_ur[i * n + m] + s_ur[i * n + n - 1 - m]);
                im = 0.5 * (s_ui[i * n + m] + s_ui[i * n + n - 1 - m]);
            }
        } else {
            const int e2 = e - M * M, i = e2 / H, m = e2 - (e2 / H) * H;
            re = 0.5 * (s_ur[i * n + m] - s_ur[i * n + n - 1 - m]);
            im = 0.5 * (s_ui[i * n + m] - s_ui[i * n + n - 1 - m]);
        }
        const int ur = fx_dither_round(re, key0 + 2 * e), ui = fx_dither_round(im, key0 + 2 * e + 1);
        out[e] = make_int4(ur, ui, ur + ui, 0);
    }
}

// |psi|^2 of a fixed-point amplitude (units of 2^-29) in FP64.
__device__ __forceinline__ double fx_prob(int2 z) {
    const double x = (double)z.x / FX_STATE, y = (double)z.y / FX_STATE;
    return __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
}

__global__ void k_lat_ground(int2 *psi, const double *v, int n, int d, int64_t g, int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t rem = (uint32_t)(i % g);  // G < 2^31
        double amp = 1.0;
        for (int k = d - 1; k >= 0; --k) {
            const uint32_t q = rem / (uint32_t)n;
            amp *= v[rem - q * n];
            rem = q;
        }
        psi[i] = make_int2(__double2int_rn(amp * FX_STATE), 0);
    }
}

__global__ void k_lat_fill(int2 *psi, int value, int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x)
        psi[i] = make_int2(value, 0);
}

// complex64 <-> the 2^-29 fixed-point state.  Loading flags components of
// modulus >= 2 (or not finite) and leaves them zero; qhd_lattice_set_state
// then checks every instance's norm.
__global__ void k_lat_from_c64(int2 *psi, const float2 *in, int64_t total, int *bad) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 z = in[i];
        const bool ok = fabsf(z.x) < 2.0f && fabsf(z.y) < 2.0f;  // false for NaN too
        if (!ok) atomicOr(bad, 1);
        psi[i] = ok ? make_int2(__double2int_rn((double)z.x * FX_STATE), __double2int_rn((double)z.y * FX_STATE))
                    : make_int2(0, 0);
    }
}

__global__ void k_lat_to_c64(float2 *out, const int2 *psi, int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int2 z = psi[i];
        out[i] = make_float2((float)((double)z.x / FX_STATE), (float)((double)z.y / FX_STATE));
    }
}

__global__ void k_lat_qp(double *f, const double *Q, const double *bv, const double *coord, int n, int d,
                         int64_t g, int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t inst = i / g;
        uint32_t rem = (uint32_t)(i - inst * g);
        double x[LAT_MAX_D];
        for (int k = d - 1; k >= 0; --k) {
            const uint32_t q = rem / (uint32_t)n;
            x[k] = coord[rem - q * n];
            rem = q;
        }
        const double *Qi = Q + inst * d * d;
        const double *bi = bv + inst * d;
        double quad = 0.0, lin = 0.0;
        for (int p = 0; p < d; ++p) {
            double row = 0.0;
            for (int q = 0; q < d; ++q) row += Qi[p * d + q] * x[q];
            quad += x[p] * row;
            lin += bi[p] * x[p];
        }
        f[i] = 0.5 * quad + lin;
    }
}

struct LatObs {
    const int2 *psi;
    const double *f64;
    const double *fmin;   // [batch]
    const double *xs;     // [batch][LAT_MAX_D] mesh minimiser
    const double *coord;  // mesh coordinates j / r, j = 0..r
    float *prob;
    double *partial;      // [batch][nblk][4]
    int64_t g;
    int d, n;
    double r, radius2, gap;
    int nblk;
};

__device__ double lat_block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o /= 2) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x / 32, l = threadIdx.x % 32;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x / 32); ++i) s += sh[i];
    return s;
}

__global__ void k_lat_obs_partial(LatObs a) {
    const int64_t b = blockIdx.y;
    const int2 *psi = a.psi + b * a.g;
    const double *f = a.f64 + b * a.g;
    const double fmin = a.fmin[b];
    const double *xs = a.xs + b * LAT_MAX_D;
    double sn = 0.0, sf = 0.0, sp = 0.0, sg = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.g;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int2 z = psi[i];
        const double p = fx_prob(z);
        if (a.prob) a.prob[b * a.g + i] = (float)p;
        sn += p;
        sf += p * f[i];
        // squared Euclidean distance to x*, summed over the axes in ascending order
        int dig[LAT_MAX_D];
        uint32_t rem = (uint32_t)i;
        for (int k = a.d - 1; k >= 0; --k) {
            const uint32_t q = rem / (uint32_t)a.n;
            dig[k] = (int)(rem - q * a.n);
            rem = q;
        }
        double r2 = 0.0;
        for (int k = 0; k < a.d; ++k) {
            const double dx = __dsub_rn(a.coord[dig[k]], xs[k]);
            r2 = __dadd_rn(r2, __dmul_rn(dx, dx));
        }
        if (r2 < a.radius2) sp += p;
        if (__dsub_rn(f[i], fmin) <= a.gap) sg += p;
    }
    __shared__ double sh[32];
    const double v0 = lat_block_sum(sn, sh);
    const double v1 = lat_block_sum(sf, sh);
    const double v2 = lat_block_sum(sp, sh);
    const double v3 = lat_block_sum(sg, sh);
    if (threadIdx.x == 0) {
        double *o = a.partial + (b * a.nblk + blockIdx.x) * 4;
        o[0] = v0;
        o[1] = v1;
        o[2] = v2;
        o[3] = v3;
    }
}

__global__ void k_lat_obs_final(const double *partial, double *result, int nblk) {
    const int64_t b = blockIdx.x;
    __shared__ double sh[4][256];
    for (int k = 0; k < 4; ++k) {
        double s = 0.0;
        for (int i = threadIdx.x; i < nblk; i += blockDim.x) s += partial[(b * nblk + i) * 4 + k];
        sh[k][threadIdx.x] = s;
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w /= 2) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) result[b * 4 + k] = sh[k][0];
}

// Marginal of axis k at mesh index j: the sum of |psi|^2 over the points whose
// k-th index is j (one block per (k, j) and instance, fixed summation order).
__global__ void k_lat_marginal(const int2 *psi, double *out, int64_t g, int d, int n) {
    const int kj = blockIdx.x, k = kj / n, j = kj - (kj / n) * n;
    const int64_t b = blockIdx.y;
    int64_t inner = 1;
    for (int a = d - 1; a > k; --a) inner *= n;
    const int64_t cnt = g / n;
    const int2 *pb = psi + b * g;
    double s = 0.0;
    for (int64_t idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
        const int64_t hi = idx / inner, lo = idx - hi * inner;
        s += fx_prob(pb[(hi * n + j) * inner + lo]);
    }
    __shared__ double sh[32];
    s = lat_block_sum(s, sh);
    if (threadIdx.x == 0) out[(b * d + k) * n + j] = s;
}

template <int N>
cudaError_t launch_pass_n(const LatPass &a, int64_t blocks, int threads, size_t smem, cudaStream_t s) {
    k_lat_pass<N><<<(unsigned)blocks, threads, smem, s>>>(a);
    return cudaGetLastError();
}

template <int N>
cudaError_t set_pass_smem(size_t bytes) {
    return cudaFuncSetAttribute(k_lat_pass<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

cudaError_t launch_pass(int n, const LatPass &a, int64_t blocks, int threads, size_t smem, cudaStream_t s) {
    switch (n) {
#define QHD_LAT_CASE(K) \
    case K: return launch_pass_n<K>(a, blocks, threads, smem, s);
        QHD_LAT_CASE(2) QHD_LAT_CASE(3) QHD_LAT_CASE(4) QHD_LAT_CASE(5) QHD_LAT_CASE(6) QHD_LAT_CASE(7)
        QHD_LAT_CASE(8) QHD_LAT_CASE(9) QHD_LAT_CASE(10) QHD_LAT_CASE(11) QHD_LAT_CASE(12) QHD_LAT_CASE(13)
        QHD_LAT_CASE(14) QHD_LAT_CASE(15) QHD_LAT_CASE(16) QHD_LAT_CASE(17)
#undef QHD_LAT_CASE
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t pass_smem_attr(int n, size_t bytes) {
    switch (n) {
#define QHD_LAT_CASE(K) \
    case K: return set_pass_smem<K>(bytes);
        QHD_LAT_CASE(2) QHD_LAT_CASE(3) QHD_LAT_CASE(4) QHD_LAT_CASE(5) QHD_LAT_CASE(6) QHD_LAT_CASE(7)
        QHD_LAT_CASE(8) QHD_LAT_CASE(9) QHD_LAT_CASE(10) QHD_LAT_CASE(11) QHD_LAT_CASE(12) QHD_LAT_CASE(13)
        QHD_LAT_CASE(14) QHD_LAT_CASE(15) QHD_LAT_CASE(16) QHD_LAT_CASE(17)
#undef QHD_LAT_CASE
        default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------- host
size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

int64_t ipow(int64_t b, int e) {
    int64_t r = 1;
    for (int i = 0; i < e; ++i) r *= b;
    return r;
}

bool sizes_ok(int ndim, int r, int64_t batch) {
    // batch indexes the second grid dimension of the per-instance kernels (<= 65535)
    if (ndim < 1 || ndim > LAT_MAX_D || r < 1 || r > LAT_MAX_R || batch < 1 || batch > 65535) return false;
    const int64_t g = ipow(r + 1, ndim);
    return batch <= (int64_t(1) << 31) / g;
}

struct PassPlan {
    int a0, a1, P, q, W, pitch, threads;
    int64_t col_count, col_stride, g_stride, row_stride, rows, rows_per_inst, tiles_per_row, blocks;
    size_t smem;
};

// Group the axes from the last one: as many consecutive axes as fit GROUP_MAX
// points per column; columns per tile up to TILE_MAX points.
std::vector<PassPlan> plan_passes(int d, int n, int64_t batch) {
    std::vector<PassPlan> out;
    const int64_t G = ipow(n, d);
    int a1 = d;
    while (a1 > 0) {
        int a0 = a1 - 1;
        int64_t P = n;
        while (a0 > 0 && P * n <= GROUP_MAX) {
            --a0;
            P *= n;
        }
        PassPlan p{};
        p.a0 = a0;
        p.a1 = a1;
        p.P = (int)P;
        p.q = a1 - a0;
        const int64_t inner = ipow(n, d - a1), outer = ipow(n, a0);
        if (inner == 1) {
            p.rows = batch;
            p.rows_per_inst = 1;
            p.col_count = outer;
            p.col_stride = P;
            p.g_stride = 1;
            p.row_stride = G;
        } else {
            p.rows = batch * outer;
            p.rows_per_inst = outer;
            p.col_count = inner;
            p.col_stride = 1;
            p.g_stride = inner;
            p.row_stride = P * inner;
        }
        int64_t W = TILE_MAX / P;
        if (W > p.col_count) W = p.col_count;
        if (inner > 1 && W > 8) W -= W % 8;  // whole 64-byte row segments
        if (W < 1) W = 1;
        p.W = (int)W;
        const int padded = (n & 1) ? p.P : p.P + p.P / n;
        p.pitch = padded | 1;
        const int64_t lines = (P / n) * W;
        const int64_t rounds = (lines + PASS_THREADS_MAX - 1) / PASS_THREADS_MAX;
        int64_t th = (lines + rounds - 1) / rounds;
        th = (th + 31) / 32 * 32;
        p.threads = (int)th;
        p.tiles_per_row = (p.col_count + W - 1) / W;
        p.blocks = p.rows * p.tiles_per_row;
        const int hh = n / 2, mm = n - hh;
        p.smem = sizeof(LatPhase) * PHASE_TAB + sizeof(int4) * (size_t)(mm * mm + hh * hh) +
                 sizeof(int2) * (size_t)(p.W * p.pitch);
        out.push_back(p);
        a1 = a0;
    }
    return out;
}

// Cyclic Jacobi eigendecomposition of a small real symmetric matrix (FP64):
// A = V diag(lam) V^T, V[i*n + k] the i-th component of eigenvector k.
void jacobi_eig(int n, std::vector<double> A, std::vector<double> &V, std::vector<double> &lam) {
    V.assign((size_t)(n * n), 0.0);
    for (int i = 0; i < n; ++i) V[(size_t)(i * n + i)] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                const double v = A[(size_t)(i * n + j)] * A[(size_t)(i * n + j)];
                tot += v;
                if (i != j) off += v;
            }
        if (off <= 1e-32 * tot || off == 0.0) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[(size_t)(p * n + q)];
                if (apq == 0.0) continue;
                const double app = A[(size_t)(p * n + p)], aqq = A[(size_t)(q * n + q)];
                // rotation that zeroes A[p][q]: tan(theta) = t, the smaller root of
                // t^2 + 2 tau t - 1 = 0 with tau = (aqq - app) / (2 apq)
                const double tau = (aqq - app) / (2.0 * apq);
                const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
                for (int k = 0; k < n; ++k) {
                    const double akp = A[(size_t)(k * n + p)], akq = A[(size_t)(k * n + q)];
                    A[(size_t)(k * n + p)] = c * akp - s * akq;
                    A[(size_t)(k * n + q)] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[(size_t)(p * n + k)], aqk = A[(size_t)(q * n + k)];
                    A[(size_t)(p * n + k)] = c * apk - s * aqk;
                    A[(size_t)(q * n + k)] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[(size_t)(k * n + p)], vkq = V[(size_t)(k * n + q)];
                    V[(size_t)(k * n + p)] = c * vkp - s * vkq;
                    V[(size_t)(k * n + q)] = s * vkp + c * vkq;
                }
            }
    }
    lam.resize((size_t)n);
    for (int i = 0; i < n; ++i) lam[(size_t)i] = A[(size_t)(i * n + i)];
}

struct LatLayout {
    size_t f64, fq, sched, samples, inst, xs, fmin, mm, ptab, flag, V, lam, ground, coord, Q, bq, U, pot, obs_part,
        obs_res, marg, total;
    int64_t chunk, chunk_shared;
    int obs_blocks, mm_blocks;
};

int blocks_for(int64_t g, int cap) {
    int64_t b = (g + 255) / 256;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

LatLayout lat_layout(int d, int r, int64_t batch) {
    LatLayout L{};
    const int n = r + 1;
    const int64_t G = ipow(n, d), BG = G * batch;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L.obs_blocks = blocks_for(G, OBS_BLOCKS_MAX);
    L.mm_blocks = blocks_for(G, MINMAX_BLOCKS_MAX);
    const size_t ubytes = sizeof(int4) * (size_t)((n - n / 2) * (n - n / 2) + (n / 2) * (n / 2));
    int64_t ch = (int64_t)(U_BUDGET / (ubytes * (size_t)batch));
    L.chunk = ch < 1 ? 1 : ch > LAT_MAX_CHUNK ? LAT_MAX_CHUNK : ch;
    ch = (int64_t)(U_BUDGET / ubytes);
    L.chunk_shared = ch > LAT_MAX_CHUNK ? LAT_MAX_CHUNK : ch;
    L.f64 = take(sizeof(double) * (size_t)BG);
    L.fq = take(sizeof(uint32_t) * (size_t)BG);
    L.sched = take(sizeof(SchedDev) * (size_t)batch);
    L.samples = take(sizeof(double) * 3 * SCHED_MAX_SAMPLES * (size_t)batch);
    L.inst = take(sizeof(InstDev) * (size_t)batch);
    L.xs = take(sizeof(double) * LAT_MAX_D * (size_t)batch);
    L.fmin = take(sizeof(double) * (size_t)batch);
    L.mm = take(sizeof(MinMaxPart) * (size_t)(L.mm_blocks * batch));
    L.ptab = take(sizeof(LatPhase) * PHASE_TAB);
    L.flag = take(sizeof(int));
    L.V = take(sizeof(double) * (size_t)(n * n));
    L.lam = take(sizeof(double) * (size_t)n);
    L.ground = take(sizeof(double) * (size_t)n);
    L.coord = take(sizeof(double) * (size_t)n);
    L.Q = take(sizeof(double) * (size_t)(d * d * batch));
    L.bq = take(sizeof(double) * (size_t)(d * batch));
    const int64_t umax = L.chunk * batch > L.chunk_shared ? L.chunk * batch : L.chunk_shared;
    L.U = take(ubytes * (size_t)umax);
    const int64_t cmax = L.chunk > L.chunk_shared ? L.chunk : L.chunk_shared;
    L.pot = take(sizeof(uint64_t) * (size_t)((cmax + 1) * batch));
    L.obs_part = take(sizeof(double) * 4 * (size_t)(L.obs_blocks * batch));
    L.obs_res = take(sizeof(double) * 4 * (size_t)batch);
    L.marg = take(sizeof(double) * (size_t)(d * n * batch));
    L.total = off;
    return L;
}

}  // namespace

struct qhd_lattice {
    int d = 0, r = 0, n = 0, kind = 0;
    int64_t batch = 1, g = 1;
    int2 *psi = nullptr;  // state in units of 2^-29 (the caller's buffer)
    char *work = nullptr;
    size_t work_bytes = 0;
    cudaStream_t stream = nullptr;
    LatLayout L{};
    std::vector<PassPlan> passes;
    // workspace views
    double *f64 = nullptr, *xs = nullptr, *fmin = nullptr, *V = nullptr, *lam = nullptr, *ground = nullptr,
           *coord = nullptr;
    double *Q = nullptr, *bq = nullptr, *obs_part = nullptr, *obs_res = nullptr, *marg = nullptr;
    uint32_t *fq = nullptr;
    SchedDev *sched = nullptr;
    double *samples = nullptr;
    InstDev *inst = nullptr;
    MinMaxPart *mm = nullptr;
    LatPhase *ptab = nullptr;
    int4 *U = nullptr;
    int *flag = nullptr;
    uint64_t *pot = nullptr;
    // host state
    bool have_f = false, have_sched = false, u_shared = false;
    double t = 0.0;
    int64_t steps_done = 0, launches = 0;
    qhd_status sticky = QHD_OK;
    std::string err;
    std::vector<double> fmin_host;
    std::vector<int64_t> argmin_host;
    int timing_every = 0;
    struct Timed {
        int kclass;
        cudaEvent_t start, stop;
    };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> pool;
    ~qhd_lattice() {
        for (auto &x : timed) {
            cudaEventDestroy(x.start);
            cudaEventDestroy(x.stop);
        }
        for (auto e : pool) cudaEventDestroy(e);
    }
};

namespace {

qhd_status lfail(qhd_lattice *c, qhd_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (s == QHD_ERR_CUDA || s == QHD_ERR_TIMEOUT) c->sticky = s;
    }
    return s;
}

#define LAT_CUDA(c, call)                                                                      \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess) return lfail((c), QHD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define LAT_LAUNCH(c, call)          \
    do {                             \
        LAT_CUDA(c, call);           \
        (c)->launches++;             \
    } while (0)

constexpr size_t LAT_MAX_TIMED = 65536;

cudaEvent_t lat_event(qhd_lattice *c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}

// Event pair around one launch when timing is on and this step is sampled.
struct LatTimed {
    qhd_lattice *c;
    int kclass;
    bool on = false;
    cudaEvent_t start = nullptr, stop = nullptr;
    LatTimed(qhd_lattice *c_, int k, bool sample) : c(c_), kclass(k) {
        if (!sample || c->timing_every <= 0 || c->timed.size() >= LAT_MAX_TIMED) return;
        start = lat_event(c);
        stop = lat_event(c);
        if (!start || !stop) return;
        on = cudaEventRecord(start, c->stream) == cudaSuccess;
    }
    ~LatTimed() {
        if (on && cudaEventRecord(stop, c->stream) == cudaSuccess) {
            c->timed.push_back({kclass, start, stop});
            return;
        }
        if (start) c->pool.push_back(start);
        if (stop) c->pool.push_back(stop);
    }
};

qhd_status lcheck(qhd_lattice *c) {
    if (!c) return QHD_ERR_INVALID_ARG;
    return c->sticky;
}

qhd_status lat_potential_common(qhd_lattice *c) {
    const int64_t B = c->batch, G = c->g;
    const int nb = c->L.mm_blocks;
    LAT_LAUNCH(c, launch_minmax(c->f64, G, B, c->mm, nb, c->stream));
    std::vector<MinMaxPart> part((size_t)(nb * B));
    LAT_CUDA(c, cudaMemcpyAsync(part.data(), c->mm, part.size() * sizeof(MinMaxPart), cudaMemcpyDeviceToHost,
                                c->stream));
    LAT_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<InstDev> inst((size_t)B);
    std::vector<double> xs((size_t)(B * LAT_MAX_D), 0.0), fm((size_t)B);
    std::vector<int64_t> am_all((size_t)B);
    for (int64_t b = 0; b < B; ++b) {
        double mn = INFINITY, mx = -INFINITY;
        int64_t am = INT64_MAX, nf = 0;
        for (int i = 0; i < nb; ++i) {
            const MinMaxPart &p = part[(size_t)(b * nb + i)];
            nf += p.nonfinite;
            if (p.fmin < mn || (p.fmin == mn && p.argmin < am)) {
                mn = p.fmin;
                am = p.argmin;
            }
            if (p.fmax > mx) mx = p.fmax;
        }
        // the FP64 copy is already overwritten: a rejected F discards the previous one
        if (nf > 0) {
            c->have_f = false;
            return lfail(c, QHD_ERR_INVALID_ARG, "instance %lld: %lld non-finite f values", (long long)b,
                         (long long)nf);
        }
        const double range = mx - mn;
        if (!(range < 2147483648.0)) {
            c->have_f = false;
            return lfail(c, QHD_ERR_INVALID_ARG, "instance %lld: f range %g >= 2^31", (long long)b, range);
        }
        int shift = 52;
        if (range > 0.0) {
            shift = (int)std::floor(std::log2((4294967296.0 - 4096.0) / range));
            while (shift > 0 && std::ldexp(range, shift) >= 4294967296.0 - 4096.0) --shift;
            if (shift > 52) shift = 52;
        }
        InstDev &ip = inst[(size_t)b];
        ip.fmin = mn;
        ip.shift = shift;
        ip.pad_ = 0;
        ip.xs[0] = ip.xs[1] = ip.xs[2] = 0.0;
        int64_t rem = am;
        for (int k = c->d - 1; k >= 0; --k) {
            xs[(size_t)(b * LAT_MAX_D + k)] = (double)(rem % c->n) / (double)c->r;
            rem /= c->n;
        }
        fm[(size_t)b] = mn;
        am_all[(size_t)b] = am;
    }
    LAT_CUDA(c, cudaMemcpyAsync(c->inst, inst.data(), inst.size() * sizeof(InstDev), cudaMemcpyHostToDevice,
                                c->stream));
    LAT_CUDA(c, cudaMemcpyAsync(c->xs, xs.data(), xs.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    LAT_CUDA(c, cudaMemcpyAsync(c->fmin, fm.data(), fm.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    LAT_LAUNCH(c, launch_quantize(c->f64, c->fq, c->inst, G, B, c->stream));
    LAT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->fmin_host = fm;
    c->argmin_host = am_all;
    c->have_f = true;
    return QHD_OK;
}

int grid_blocks(int64_t total) {
    int64_t b = (total + 255) / 256;
    if (b > 4096) b = 4096;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

extern "C" {

size_t qhd_lattice_workspace_bytes(int ndim, int r, int64_t batch) {
    if (!sizes_ok(ndim, r, batch)) return 0;
    return lat_layout(ndim, r, batch).total;
}

qhd_status qhd_lattice_init(qhd_lattice **out, int ndim, int r, int kind, int64_t batch, void *psi_dev,
                            void *work_dev, size_t work_bytes, void *stream) {
    if (!out) return QHD_ERR_INVALID_ARG;
    *out = nullptr;
    if (!sizes_ok(ndim, r, batch)) return QHD_ERR_INVALID_ARG;
    if (kind != QHD_LATTICE_CHAIN && kind != QHD_LATTICE_RELAXED) return QHD_ERR_INVALID_ARG;
    if (!psi_dev || ((uintptr_t)psi_dev & 7)) return QHD_ERR_INVALID_ARG;
    const LatLayout L = lat_layout(ndim, r, batch);
    if (!work_dev || ((uintptr_t)work_dev & 255) || work_bytes < L.total) return QHD_ERR_WORKSPACE;
    qhd_lattice *c = new qhd_lattice();
    c->d = ndim;
    c->r = r;
    c->n = r + 1;
    c->kind = kind;
    c->batch = batch;
    c->g = ipow(c->n, ndim);
    c->psi = (int2 *)psi_dev;
    c->work = (char *)work_dev;
    c->work_bytes = work_bytes;
    c->stream = (cudaStream_t)stream;
    c->L = L;
    c->passes = plan_passes(ndim, c->n, batch);
    c->f64 = (double *)(c->work + L.f64);
    c->fq = (uint32_t *)(c->work + L.fq);
    c->sched = (SchedDev *)(c->work + L.sched);
    c->samples = (double *)(c->work + L.samples);
    c->inst = (InstDev *)(c->work + L.inst);
    c->xs = (double *)(c->work + L.xs);
    c->fmin = (double *)(c->work + L.fmin);
    c->mm = (MinMaxPart *)(c->work + L.mm);
    c->ptab = (LatPhase *)(c->work + L.ptab);
    c->flag = (int *)(c->work + L.flag);
    c->V = (double *)(c->work + L.V);
    c->lam = (double *)(c->work + L.lam);
    c->ground = (double *)(c->work + L.ground);
    c->coord = (double *)(c->work + L.coord);
    c->Q = (double *)(c->work + L.Q);
    c->bq = (double *)(c->work + L.bq);
    c->U = (int4 *)(c->work + L.U);
    c->pot = (uint64_t *)(c->work + L.pot);
    c->obs_part = (double *)(c->work + L.obs_part);
    c->obs_res = (double *)(c->work + L.obs_res);
    c->marg = (double *)(c->work + L.marg);
    // per-axis operator A, its eigendecomposition and the ground state of -A
    const int n = c->n;
    std::vector<double> A((size_t)(n * n), 0.0);
    for (int j = 0; j < r; ++j) {
        const double w = kind == QHD_LATTICE_CHAIN ? 1.0 : std::sqrt((double)(j + 1) * (double)(r - j) / (double)r);
        A[(size_t)(j * n + j + 1)] = w;
        A[(size_t)((j + 1) * n + j)] = w;
    }
    std::vector<double> V, lam;
    jacobi_eig(n, A, V, lam);
    int top = 0;
    for (int k = 1; k < n; ++k)
        if (lam[(size_t)k] > lam[(size_t)top]) top = k;
    std::vector<double> ground((size_t)n);
    double sum = 0.0;
    for (int i = 0; i < n; ++i) sum += V[(size_t)(i * n + top)];
    for (int i = 0; i < n; ++i) ground[(size_t)i] = (sum < 0 ? -1.0 : 1.0) * V[(size_t)(i * n + top)];
    std::vector<LatPhase> ptab((size_t)PHASE_TAB);
    for (int k = 0; k < PHASE_TAB; ++k) {
        const double ang = -2.0 * 3.141592653589793238462643383279502884 * (double)k / PHASE_TAB;
        const double cr = std::cos(ang), ci = std::sin(ang);
        ptab[(size_t)k].fx = make_int2((int)std::nearbyint(cr * FX_ONE), (int)std::nearbyint(ci * FX_ONE));
        ptab[(size_t)k].f = make_float2((float)cr, (float)ci);
    }
    std::vector<double> coord((size_t)n);
    for (int j = 0; j < n; ++j) coord[(size_t)j] = (double)j / (double)r;
    cudaError_t e = cudaMemcpyAsync(c->V, V.data(), V.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->coord, coord.data(), coord.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->lam, lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->ground, ground.data(), ground.size() * sizeof(double), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->ptab, ptab.data(), ptab.size() * sizeof(LatPhase), cudaMemcpyHostToDevice, c->stream);
    size_t smax = 0;
    for (auto &p : c->passes) smax = p.smem > smax ? p.smem : smax;
    if (e == cudaSuccess && smax > 48 * 1024) e = pass_smem_attr(n, smax);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        delete c;
        return QHD_ERR_CUDA;
    }
    *out = c;
    return QHD_OK;
}

qhd_status qhd_lattice_set_potential(qhd_lattice *c, const double *f_dev) {
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    if (!f_dev) return lfail(c, QHD_ERR_INVALID_ARG, "f_dev is NULL");
    LAT_CUDA(c, cudaMemcpyAsync(c->f64, f_dev, sizeof(double) * (size_t)(c->g * c->batch), cudaMemcpyDeviceToDevice,
                                c->stream));
    return lat_potential_common(c);
}

qhd_status qhd_lattice_set_qp(qhd_lattice *c, const double *Q_host, const double *b_host) {
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    if (!Q_host || !b_host) return lfail(c, QHD_ERR_INVALID_ARG, "Q or b is NULL");
    const int64_t nq = c->batch * c->d * c->d, nb = c->batch * c->d;
    for (int64_t i = 0; i < nq; ++i)
        if (!std::isfinite(Q_host[i])) return lfail(c, QHD_ERR_INVALID_ARG, "non-finite Q");
    for (int64_t i = 0; i < nb; ++i)
        if (!std::isfinite(b_host[i])) return lfail(c, QHD_ERR_INVALID_ARG, "non-finite b");
    LAT_CUDA(c, cudaMemcpyAsync(c->Q, Q_host, sizeof(double) * (size_t)nq, cudaMemcpyHostToDevice, c->stream));
    LAT_CUDA(c, cudaMemcpyAsync(c->bq, b_host, sizeof(double) * (size_t)nb, cudaMemcpyHostToDevice, c->stream));
    const int64_t total = c->g * c->batch;
    LAT_LAUNCH(c, (k_lat_qp<<<grid_blocks(total), 256, 0, c->stream>>>(c->f64, c->Q, c->bq, c->coord, c->n,
                                                                        c->d, c->g, total),
                   cudaGetLastError()));
    return lat_potential_common(c);
}

qhd_status qhd_lattice_set_schedule(qhd_lattice *c, const qhd_schedule *sc) {
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    if (!sc) return lfail(c, QHD_ERR_INVALID_ARG, "schedule is NULL");
    std::vector<SchedDev> dev;
    std::vector<double> samples;
    bool shared = false;
    const std::string why = convert_schedules(sc, c->batch, c->samples, dev, samples, &shared);
    if (!why.empty()) return lfail(c, QHD_ERR_INVALID_ARG, "%s", why.c_str());
    LAT_CUDA(c, cudaMemcpyAsync(c->samples, samples.data(), samples.size() * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream));
    LAT_CUDA(c, cudaMemcpyAsync(c->sched, dev.data(), dev.size() * sizeof(SchedDev), cudaMemcpyHostToDevice,
                                c->stream));
    LAT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->u_shared = shared;
    c->have_sched = true;
    return QHD_OK;
}

qhd_status qhd_lattice_reset_state(qhd_lattice *c, int init) {
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    const int64_t total = c->g * c->batch;
    if (init == QHD_LATTICE_INIT_UNIFORM) {
        const int v = (int)std::nearbyint(FX_STATE / std::sqrt((double)c->g));
        LAT_LAUNCH(c, (k_lat_fill<<<grid_blocks(total), 256, 0, c->stream>>>(c->psi, v, total), cudaGetLastError()));
    } else if (init == QHD_LATTICE_INIT_GROUND) {
        LAT_LAUNCH(c, (k_lat_ground<<<grid_blocks(total), 256, 0, c->stream>>>(c->psi, c->ground, c->n, c->d, c->g,
                                                                                total),
                       cudaGetLastError()));
    } else {
        return lfail(c, QHD_ERR_INVALID_ARG, "unknown initial state %d", init);
    }
    c->t = 0.0;
    c->steps_done = 0;
    return QHD_OK;
}

qhd_status qhd_lattice_evolve(qhd_lattice *c, double T, double dt) {
    qhd::TraceRange trace("qhd_lattice_evolve");
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    if (!std::isfinite(T) || !std::isfinite(dt) || dt == 0.0)
        return lfail(c, QHD_ERR_INVALID_ARG, "T and dt must be finite and dt nonzero");
    const double ratio = T / dt;
    const double nr = std::nearbyint(ratio);
    if (!(nr >= 1.0) || std::fabs(ratio - nr) > 1e-9 * nr || nr > 1e12)
        return lfail(c, QHD_ERR_INVALID_ARG, "T/dt = %.17g is not a positive integer", ratio);
    if (!c->have_f || !c->have_sched)
        return lfail(c, QHD_ERR_STATE, "evolve needs a potential and a schedule first");
    const int64_t nsteps = (int64_t)nr, B = c->batch;
    const int n = c->n;
    const int64_t ub = c->u_shared ? 1 : B;
    const int64_t ch = c->u_shared ? c->L.chunk_shared : c->L.chunk;
    LatPrep pa{};
    pa.sched = c->sched;
    pa.inst = c->inst;
    pa.pot = c->pot;
    pa.U = c->U;
    pa.V = c->V;
    pa.lam = c->lam;
    pa.kin_scale = 0.5 * (double)c->r * (double)c->r;
    pa.t_start = c->t;
    pa.dt = dt;
    pa.nsteps = nsteps;
    pa.batch = B;
    pa.u_batch = ub;
    pa.n = n;
    const int np = (int)c->passes.size();
    for (int64_t j0 = 0; j0 < nsteps; j0 += ch) {
        const int64_t cnt = nsteps - j0 < ch ? nsteps - j0 : ch;
        const bool last_chunk = j0 + cnt == nsteps;
        pa.j0 = j0;
        pa.cnt = cnt;
        pa.step_base = (uint64_t)(c->steps_done + j0);
        {
            LatTimed tm(c, QHD_LKCLASS_PREP, true);
            LAT_LAUNCH(c, (k_lat_prep<<<dim3((unsigned)(cnt + 1), (unsigned)B), 64, 0, c->stream>>>(pa),
                           cudaGetLastError()));
        }
        for (int64_t jl = 0; jl < cnt; ++jl) {
            const int64_t jg = c->steps_done + j0 + jl;  // global step index (dither)
            const bool sample = c->timing_every > 0 && ((j0 + jl) % c->timing_every) == 0;
            for (int p = 0; p < np; ++p) {
                const PassPlan &pl = c->passes[(size_t)p];
                LatPass a{};
                a.psi = c->psi;
                a.fq = c->fq;
                a.pot_pre = p == 0 ? c->pot + jl * B : nullptr;
                a.pot_post = (p == np - 1 && last_chunk && jl == cnt - 1) ? c->pot + cnt * B : nullptr;
                a.dither_pre = step_dither((uint64_t)jg);
                a.dither_post = step_dither((uint64_t)jg + 1);
                a.U = c->U + jl * ub * (int64_t)((n - n / 2) * (n - n / 2) + (n / 2) * (n / 2));
                a.u_batch = ub;
                a.ptab = c->ptab;
                a.P = pl.P;
                a.q = pl.q;
                a.W = pl.W;
                a.pitch = pl.pitch;
                a.lines_per_col = pl.P / n;
                a.col_count = pl.col_count;
                a.col_stride = pl.col_stride;
                a.g_stride = pl.g_stride;
                a.row_stride = pl.row_stride;
                a.rows_per_inst = pl.rows_per_inst;
                a.tiles_per_row = pl.tiles_per_row;
                a.mg_P = lat_magic((uint32_t)pl.P);
                a.mg_W = lat_magic((uint32_t)pl.W);
                a.mg_lpc = lat_magic((uint32_t)(pl.P / n));
                for (int k = 0, sk = 1; k < pl.q; ++k, sk *= n) a.mg_s[k] = lat_magic((uint32_t)sk);
                LatTimed tm(c, p == 0 ? QHD_LKCLASS_PASS0 : QHD_LKCLASS_PASS1, sample);
                LAT_LAUNCH(c, launch_pass(n, a, pl.blocks, pl.threads, pl.smem, c->stream));
            }
        }
    }
    c->t += (double)nsteps * dt;
    c->steps_done += nsteps;
    return QHD_OK;
}

qhd_status qhd_lattice_observables(qhd_lattice *c, qhd_lattice_obs *out, float *prob_dev, double *marginals_host,
                                   double radius, double gap) {
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    if (!out) return lfail(c, QHD_ERR_INVALID_ARG, "out is NULL");
    if (!c->have_f) return lfail(c, QHD_ERR_STATE, "observables need a potential");
    if (!std::isfinite(radius) || radius < 0 || !std::isfinite(gap))
        return lfail(c, QHD_ERR_INVALID_ARG, "bad radius or gap");
    const int64_t B = c->batch;
    LatObs a{};
    a.psi = c->psi;
    a.f64 = c->f64;
    a.fmin = c->fmin;
    a.xs = c->xs;
    a.coord = c->coord;
    a.prob = prob_dev;
    a.partial = c->obs_part;
    a.g = c->g;
    a.d = c->d;
    a.n = c->n;
    a.r = (double)c->r;
    a.radius2 = radius * radius;
    a.gap = gap;
    a.nblk = c->L.obs_blocks;
    LAT_LAUNCH(c, (k_lat_obs_partial<<<dim3((unsigned)a.nblk, (unsigned)B), 256, 0, c->stream>>>(a),
                   cudaGetLastError()));
    LAT_LAUNCH(c, (k_lat_obs_final<<<(unsigned)B, 256, 0, c->stream>>>(c->obs_part, c->obs_res, a.nblk),
                   cudaGetLastError()));
    std::vector<double> res((size_t)(4 * B));
    LAT_CUDA(c, cudaMemcpyAsync(res.data(), c->obs_res, res.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    if (marginals_host) {
        LAT_LAUNCH(c, (k_lat_marginal<<<dim3((unsigned)(c->d * c->n), (unsigned)B), 256, 0, c->stream>>>(
                           c->psi, c->marg, c->g, c->d, c->n),
                       cudaGetLastError()));
        LAT_CUDA(c, cudaMemcpyAsync(marginals_host, c->marg, sizeof(double) * (size_t)(B * c->d * c->n),
                                    cudaMemcpyDeviceToHost, c->stream));
    }
    LAT_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int64_t b = 0; b < B; ++b) {
        qhd_lattice_obs &o = out[b];
        o.t = c->t;
        o.norm = res[(size_t)(4 * b)];
        o.e_f = res[(size_t)(4 * b + 1)];
        o.p_succ = res[(size_t)(4 * b + 2)];
        o.p_gap = res[(size_t)(4 * b + 3)];
        o.f_min = c->fmin_host[(size_t)b];
        o.argmin = c->argmin_host[(size_t)b];
        o.steps_done = c->steps_done;
    }
    return QHD_OK;
}

qhd_status qhd_lattice_evolve_trajectory(qhd_lattice *c, double T, double dt, int64_t every, double radius,
                                         double gap, double *traj_dev) {
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    if (!traj_dev) return lfail(c, QHD_ERR_INVALID_ARG, "traj_dev is NULL");
    if (!std::isfinite(radius) || radius < 0 || !std::isfinite(gap))
        return lfail(c, QHD_ERR_INVALID_ARG, "bad radius or gap");
    if (!std::isfinite(T) || !std::isfinite(dt) || dt == 0.0)
        return lfail(c, QHD_ERR_INVALID_ARG, "T and dt must be finite and dt nonzero");
    const double ratio = T / dt;
    const double nr = std::nearbyint(ratio);
    if (!(nr >= 1.0) || std::fabs(ratio - nr) > 1e-9 * nr || nr > 1e12)
        return lfail(c, QHD_ERR_INVALID_ARG, "T/dt = %.17g is not a positive integer", ratio);
    const int64_t nsteps = (int64_t)nr;
    if (every < 1 || nsteps % every != 0)
        return lfail(c, QHD_ERR_INVALID_ARG, "every = %lld must divide the %lld steps", (long long)every,
                     (long long)nsteps);
    if (!c->have_f || !c->have_sched)
        return lfail(c, QHD_ERR_STATE, "evolve needs a potential and a schedule first");
    LatObs a{};
    a.psi = c->psi;
    a.f64 = c->f64;
    a.fmin = c->fmin;
    a.xs = c->xs;
    a.coord = c->coord;
    a.prob = nullptr;
    a.partial = c->obs_part;
    a.g = c->g;
    a.d = c->d;
    a.n = c->n;
    a.r = (double)c->r;
    a.radius2 = radius * radius;
    a.gap = gap;
    a.nblk = c->L.obs_blocks;
    // Consecutive segments are one Strang run: the closing half phase of a
    // segment and the opening one of the next make the merged phase.
    for (int64_t k = 0; k < nsteps / every; ++k) {
        s = qhd_lattice_evolve(c, (double)every * dt, dt);
        if (s != QHD_OK) return s;
        LAT_LAUNCH(c, (k_lat_obs_partial<<<dim3((unsigned)a.nblk, (unsigned)c->batch), 256, 0, c->stream>>>(a),
                       cudaGetLastError()));
        LAT_LAUNCH(c, (k_lat_obs_final<<<(unsigned)c->batch, 256, 0, c->stream>>>(c->obs_part,
                                                                                  traj_dev + k * c->batch * 4,
                                                                                  a.nblk),
                       cudaGetLastError()));
    }
    return QHD_OK;
}

qhd_status qhd_lattice_get_state(qhd_lattice *c, void *out_dev) {
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    if (!out_dev || ((uintptr_t)out_dev & 7)) return lfail(c, QHD_ERR_INVALID_ARG, "out_dev NULL or misaligned");
    const int64_t total = c->g * c->batch;
    LAT_LAUNCH(c, (k_lat_to_c64<<<grid_blocks(total), 256, 0, c->stream>>>((float2 *)out_dev, c->psi, total),
                   cudaGetLastError()));
    return QHD_OK;
}

qhd_status qhd_lattice_set_state(qhd_lattice *c, const void *in_dev) {
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    if (!in_dev || ((uintptr_t)in_dev & 7)) return lfail(c, QHD_ERR_INVALID_ARG, "in_dev NULL or misaligned");
    const int64_t total = c->g * c->batch;
    LAT_CUDA(c, cudaMemsetAsync(c->flag, 0, sizeof(int), c->stream));
    LAT_LAUNCH(c, (k_lat_from_c64<<<grid_blocks(total), 256, 0, c->stream>>>(c->psi, (const float2 *)in_dev, total,
                                                                            c->flag),
                   cudaGetLastError()));
    // Per-instance norms (the observables reduction; its other sums are not used
    // here).  The integer line products are sized for states of norm <= 1.
    LatObs o{};
    o.psi = c->psi;
    o.f64 = c->f64;
    o.fmin = c->fmin;
    o.xs = c->xs;
    o.coord = c->coord;
    o.prob = nullptr;
    o.partial = c->obs_part;
    o.g = c->g;
    o.d = c->d;
    o.n = c->n;
    o.r = (double)c->r;
    o.radius2 = 0.0;
    o.gap = -1.0;
    o.nblk = c->L.obs_blocks;
    LAT_LAUNCH(c, (k_lat_obs_partial<<<dim3((unsigned)o.nblk, (unsigned)c->batch), 256, 0, c->stream>>>(o),
                   cudaGetLastError()));
    LAT_LAUNCH(c, (k_lat_obs_final<<<(unsigned)c->batch, 256, 0, c->stream>>>(c->obs_part, c->obs_res, o.nblk),
                   cudaGetLastError()));
    std::vector<double> res((size_t)(4 * c->batch));
    int bad = 0;
    LAT_CUDA(c, cudaMemcpyAsync(&bad, c->flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    LAT_CUDA(c, cudaMemcpyAsync(res.data(), c->obs_res, res.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    LAT_CUDA(c, cudaStreamSynchronize(c->stream));
    int64_t worst = -1;
    for (int64_t b = 0; b < c->batch; ++b)
        if (!(res[(size_t)(4 * b)] <= 1.0 + 1e-3)) worst = b;
    if (bad || worst >= 0) {
        LAT_LAUNCH(c, (k_lat_fill<<<grid_blocks(total), 256, 0, c->stream>>>(c->psi, 0, total), cudaGetLastError()));
        if (bad) return lfail(c, QHD_ERR_INVALID_ARG, "state component not finite or of modulus >= 2 (state set to 0)");
        return lfail(c, QHD_ERR_INVALID_ARG, "instance %lld: state norm^2 %g > 1 + 1e-3 (state set to 0)",
                     (long long)worst, res[(size_t)(4 * worst)]);
    }
    return QHD_OK;
}

qhd_status qhd_lattice_timing_enable(qhd_lattice *c, int every) {
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    if (every < 0) return lfail(c, QHD_ERR_INVALID_ARG, "every must be >= 0");
    c->timing_every = every;
    return QHD_OK;
}

qhd_status qhd_lattice_timing_read(qhd_lattice *c, double *ms_out, int64_t *launches_out, int reset) {
    qhd_status s = lcheck(c);
    if (s != QHD_OK) return s;
    double ms[QHD_LKCLASS_COUNT] = {};
    int64_t cnt[QHD_LKCLASS_COUNT] = {};
    for (auto &x : c->timed) {
        LAT_CUDA(c, cudaEventSynchronize(x.stop));
        float v = 0.f;
        LAT_CUDA(c, cudaEventElapsedTime(&v, x.start, x.stop));
        ms[x.kclass] += v;
        cnt[x.kclass] += 1;
    }
    if (ms_out)
        for (int k = 0; k < QHD_LKCLASS_COUNT; ++k) ms_out[k] = ms[k];
    if (launches_out)
        for (int k = 0; k < QHD_LKCLASS_COUNT; ++k) launches_out[k] = cnt[k];
    if (reset) {
        for (auto &x : c->timed) {
            c->pool.push_back(x.start);
            c->pool.push_back(x.stop);
        }
        c->timed.clear();
    }
    return QHD_OK;
}

int64_t qhd_lattice_launch_count(const qhd_lattice *c) { return c ? c->launches : 0; }

const char *qhd_lattice_last_error(const qhd_lattice *c) { return c ? c->err.c_str() : ""; }

qhd_status qhd_lattice_destroy(qhd_lattice *c) {
    if (!c) return QHD_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    delete c;
    return e == cudaSuccess ? QHD_OK : QHD_ERR_CUDA;
}

}  // extern "C"
