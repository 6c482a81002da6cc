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
// eigendecomposition of A (U = V diag(exp(i dt a r^2/2 lambda)) V^T) and
// carried as FP32 hi + lo: the same rounded matrix would otherwise perturb the
// norm coherently in step after step.
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

using namespace qhd;

namespace {

constexpr int LAT_MAX_D = 6;
constexpr int LAT_MAX_R = 16;
constexpr int LAT_MAX_N = LAT_MAX_R + 1;
constexpr int GROUP_MAX = 1024;          // points of one column (the group's axes)
constexpr int TILE_MAX = 6144;           // points of one tile (48 KB of complex64)
constexpr int PASS_THREADS_MAX = 256;
constexpr int64_t LAT_MAX_CHUNK = 1024;
constexpr size_t U_BUDGET = size_t(64) << 20;  // bytes of propagators per chunk
constexpr int OBS_BLOCKS_MAX = 1024;
constexpr int MINMAX_BLOCKS_MAX = 512;

// ------------------------------------------------------------------ kernels
struct LatPass {
    float2 *psi;
    const uint32_t *fq;
    const uint64_t *pot_pre;   // [batch] phase coefficient applied on load, or null
    const uint64_t *pot_post;  // [batch] applied on store, or null
    uint32_t dither_pre, dither_post;
    const float4 *U;           // this step's propagator [u_batch][n*n], U[i][m], (hi.re, hi.im, lo.re, lo.im)
    int64_t u_batch;
    const float4 *ptab;
    int P, q, W, pitch, lines_per_col;
    int64_t col_count, col_stride, g_stride, row_stride, rows_per_inst, tiles_per_row;
};

// Shared-memory index of group point g: even line lengths get one pad slot per
// line so that threads walking lines of stride 1 hit distinct banks.
template <int N>
__device__ __forceinline__ int lat_idx(int g) {
    return (N & 1) ? g : g + g / N;
}

template <int N>
__global__ void __launch_bounds__(PASS_THREADS_MAX) k_lat_pass(LatPass a) {
    extern __shared__ __align__(16) float4 lsm[];
    float4 *ptab = lsm;
    float4 *U = lsm + PHASE_TAB;
    float2 *tile = reinterpret_cast<float2 *>(U + N * N);
    const int64_t row = blockIdx.x / a.tiles_per_row;
    const int64_t c0 = (blockIdx.x - row * a.tiles_per_row) * a.W;
    const int64_t inst = row / a.rows_per_inst;
    if (a.pot_pre || a.pot_post) load_phase_tab(ptab, a.ptab);
    const float4 *Ug = a.U + (a.u_batch == 1 ? 0 : inst) * (N * N);
    for (int i = threadIdx.x; i < N * N; i += blockDim.x) U[i] = __ldg(&Ug[i]);
    __syncthreads();
    const int P = a.P, W = a.W, pitch = a.pitch;
    const int64_t left = a.col_count - c0;
    const int ncol = left < W ? (int)left : W;
    const int64_t base = row * a.row_stride + c0 * a.col_stride;
    const bool contig = a.g_stride == 1;
    const int tot = P * W;
    {
        const uint64_t c = a.pot_pre ? a.pot_pre[inst] : 0;
        for (int l = threadIdx.x; l < tot; l += blockDim.x) {
            int g, col;
            if (contig) {
                col = l / P;
                g = l - col * P;
            } else {
                g = l / W;
                col = l - g * W;
            }
            if (col >= ncol) continue;
            const int64_t off = base + col * a.col_stride + (int64_t)g * a.g_stride;
            float2 v = a.psi[off];
            if (a.pot_pre) v = apply_phase_tab(v, turns_mul(c, __ldg(&a.fq[off])) + a.dither_pre, ptab);
            tile[col * pitch + lat_idx<N>(g)] = v;
        }
    }
    __syncthreads();
    const int lpc = a.lines_per_col;
    const int lines = lpc * W;
    int s = 1;  // stride of the current axis inside the group (last axis first)
    for (int ax = 0; ax < a.q; ++ax, s *= N) {
        for (int l = threadIdx.x; l < lines; l += blockDim.x) {
            const int col = l / lpc;
            const int h = l - col * lpc;
            if (col >= ncol) continue;
            const int hs = h / s;
            const int g0 = hs * (s * N) + (h - hs * s);
            float2 *cb = tile + col * pitch;
            float2 x[N];
#pragma unroll
            for (int m = 0; m < N; ++m) x[m] = cb[lat_idx<N>(g0 + m * s)];
            float2 y[N];
#pragma unroll
            for (int i = 0; i < N; ++i) {
                float hr = 0.f, hi = 0.f, lr = 0.f, li = 0.f;
#pragma unroll
                for (int m = 0; m < N; ++m) {
                    const float4 u = U[i * N + m];
                    hr = fmaf(u.x, x[m].x, hr);
                    hr = fmaf(-u.y, x[m].y, hr);
                    hi = fmaf(u.x, x[m].y, hi);
                    hi = fmaf(u.y, x[m].x, hi);
                    lr = fmaf(u.z, x[m].x, lr);
                    lr = fmaf(-u.w, x[m].y, lr);
                    li = fmaf(u.z, x[m].y, li);
                    li = fmaf(u.w, x[m].x, li);
                }
                y[i] = make_float2(hr + lr, hi + li);
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
                col = l / P;
                g = l - col * P;
            } else {
                g = l / W;
                col = l - g * W;
            }
            if (col >= ncol) continue;
            const int64_t off = base + col * a.col_stride + (int64_t)g * a.g_stride;
            float2 v = tile[col * pitch + lat_idx<N>(g)];
            if (a.pot_post) v = apply_phase_tab(v, turns_mul(c, __ldg(&a.fq[off])) + a.dither_post, ptab);
            a.psi[off] = v;
        }
    }
}

struct LatPrep {
    const SchedDev *sched;
    const InstDev *inst;
    uint64_t *pot;       // [cnt+1][batch]
    float4 *U;           // [cnt][u_batch][n*n]
    const double *V;     // eigenvectors of A, V[i*n + k] = component i of vector k
    const double *lam;   // eigenvalues of A
    double kin_scale;    // r^2 / 2
    double t_start, dt;
    int64_t j0, cnt, nsteps, batch, u_batch;
    int n;
};

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
    float4 *out = a.U + (jl * a.u_batch + b) * (int64_t)(n * n);
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const int i = e / n, m = e - (e / n) * n;
        double re = 0.0, im = 0.0;
        for (int k = 0; k < n; ++k) {
            const double w = __dmul_rn(a.V[i * n + k], a.V[m * n + k]);
            re = __dadd_rn(re, __dmul_rn(w, s_c[k]));
            im = __dadd_rn(im, __dmul_rn(w, s_s[k]));
        }
        const float hr = (float)re, hi = (float)im;
        out[e] = make_float4(hr, hi, (float)(re - (double)hr), (float)(im - (double)hi));
    }
}

// Multi-index digit k (axis k, row-major, n per axis) of flat index i.
__device__ __forceinline__ int lat_digit(int64_t i, int k, int d, int n) {
    for (int a = d - 1; a > k; --a) i /= n;
    return (int)(i % n);
}

__global__ void k_lat_ground(float2 *psi, const double *v, int n, int d, int64_t g, int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t rem = i % g;
        double amp = 1.0;
        for (int k = d - 1; k >= 0; --k) {
            amp *= v[rem % n];
            rem /= n;
        }
        psi[i] = make_float2((float)amp, 0.0f);
    }
}

__global__ void k_lat_qp(double *f, const double *Q, const double *bv, int n, int d, double r, int64_t g,
                         int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t inst = i / g;
        int64_t rem = i - inst * g;
        double x[LAT_MAX_D];
        for (int k = d - 1; k >= 0; --k) {
            x[k] = (double)(rem % n) / r;
            rem /= n;
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
    const float2 *psi;
    const double *f64;
    const double *fmin;   // [batch]
    const double *xs;     // [batch][LAT_MAX_D] mesh minimiser
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
    const float2 *psi = a.psi + b * a.g;
    const double *f = a.f64 + b * a.g;
    const double fmin = a.fmin[b];
    const double *xs = a.xs + b * LAT_MAX_D;
    double sn = 0.0, sf = 0.0, sp = 0.0, sg = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.g;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 z = psi[i];
        const double p = __dadd_rn(__dmul_rn((double)z.x, (double)z.x), __dmul_rn((double)z.y, (double)z.y));
        if (a.prob) a.prob[b * a.g + i] = (float)p;
        sn += p;
        sf += p * f[i];
        // squared Euclidean distance to x*, summed over the axes in ascending order
        double r2 = 0.0;
        for (int k = 0; k < a.d; ++k) {
            const double dx = __dsub_rn(__ddiv_rn((double)lat_digit(i, k, a.d, a.n), a.r), xs[k]);
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
__global__ void k_lat_marginal(const float2 *psi, double *out, int64_t g, int d, int n) {
    const int kj = blockIdx.x, k = kj / n, j = kj - (kj / n) * n;
    const int64_t b = blockIdx.y;
    int64_t inner = 1;
    for (int a = d - 1; a > k; --a) inner *= n;
    const int64_t cnt = g / n;
    const float2 *pb = psi + b * g;
    double s = 0.0;
    for (int64_t idx = threadIdx.x; idx < cnt; idx += blockDim.x) {
        const int64_t hi = idx / inner, lo = idx - hi * inner;
        const float2 z = pb[(hi * n + j) * inner + lo];
        s += __dadd_rn(__dmul_rn((double)z.x, (double)z.x), __dmul_rn((double)z.y, (double)z.y));
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
    if (ndim < 1 || ndim > LAT_MAX_D || r < 1 || r > LAT_MAX_R || batch < 1) return false;
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
        p.smem = sizeof(float4) * (size_t)(PHASE_TAB + n * n) + sizeof(float2) * (size_t)(p.W * p.pitch);
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
    size_t f64, fq, sched, samples, inst, xs, fmin, mm, ptab, V, lam, ground, Q, bq, U, pot, obs_part, obs_res, marg,
        total;
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
    const size_t ubytes = sizeof(float4) * (size_t)(n * n);
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
    L.ptab = take(sizeof(float4) * PHASE_TAB);
    L.V = take(sizeof(double) * (size_t)(n * n));
    L.lam = take(sizeof(double) * (size_t)n);
    L.ground = take(sizeof(double) * (size_t)n);
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
    float2 *psi = nullptr;
    char *work = nullptr;
    size_t work_bytes = 0;
    cudaStream_t stream = nullptr;
    LatLayout L{};
    std::vector<PassPlan> passes;
    // workspace views
    double *f64 = nullptr, *xs = nullptr, *fmin = nullptr, *V = nullptr, *lam = nullptr, *ground = nullptr;
    double *Q = nullptr, *bq = nullptr, *obs_part = nullptr, *obs_res = nullptr, *marg = nullptr;
    uint32_t *fq = nullptr;
    SchedDev *sched = nullptr;
    double *samples = nullptr;
    InstDev *inst = nullptr;
    MinMaxPart *mm = nullptr;
    float4 *ptab = nullptr, *U = nullptr;
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
        if (nf > 0)
            return lfail(c, QHD_ERR_INVALID_ARG, "instance %lld: %lld non-finite f values", (long long)b,
                         (long long)nf);
        const double range = mx - mn;
        if (!(range < 2147483648.0))
            return lfail(c, QHD_ERR_INVALID_ARG, "instance %lld: f range %g >= 2^31", (long long)b, range);
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
    c->psi = (float2 *)psi_dev;
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
    c->ptab = (float4 *)(c->work + L.ptab);
    c->V = (double *)(c->work + L.V);
    c->lam = (double *)(c->work + L.lam);
    c->ground = (double *)(c->work + L.ground);
    c->Q = (double *)(c->work + L.Q);
    c->bq = (double *)(c->work + L.bq);
    c->U = (float4 *)(c->work + L.U);
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
    std::vector<float4> ptab((size_t)PHASE_TAB);
    for (int k = 0; k < PHASE_TAB; ++k) {
        const double ang = -2.0 * 3.141592653589793238462643383279502884 * (double)k / PHASE_TAB;
        const double cr = std::cos(ang), ci = std::sin(ang);
        const float hr = (float)cr, hi = (float)ci;
        ptab[(size_t)k] = make_float4(hr, hi, (float)(cr - (double)hr), (float)(ci - (double)hi));
    }
    cudaError_t e = cudaMemcpyAsync(c->V, V.data(), V.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->lam, lam.data(), lam.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->ground, ground.data(), ground.size() * sizeof(double), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->ptab, ptab.data(), ptab.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream);
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
    LAT_LAUNCH(c, (k_lat_qp<<<grid_blocks(total), 256, 0, c->stream>>>(c->f64, c->Q, c->bq, c->n, c->d,
                                                                        (double)c->r, c->g, total),
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
        LAT_LAUNCH(c, launch_uniform(c->psi, total, (float)(1.0 / std::sqrt((double)c->g)), c->stream));
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
                a.U = c->U + jl * ub * (int64_t)(n * n);
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
