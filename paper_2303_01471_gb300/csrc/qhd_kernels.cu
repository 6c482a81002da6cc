// qhd_kernels.cu -- the hot path of the split-operator QHD step on sm_103a.
//
// One Strang step (Eq. (prod_qhd_fft) in its symmetric form) is
//   psi <- P(dt b/2) F^-1 K(dt a) F P(dt b/2) psi
// with P the potential phase exp(-i theta f(x)) (diagonal in position) and K
// the kinetic phase exp(-i dt a |k|^2/2) (diagonal in Fourier space,
// k = 2 pi m / L).  The half potential phases of consecutive steps commute and
// are merged: theta_j = dt (b_{j-1} + b_j)/2.  The multi-dimensional DFT is
// split by axis, and the per-axis transforms are fused with the phases so that
// each launch reads and writes psi once:
//   2-D:  row pass    F_1 . P . F_1^-1           (contiguous rows)
//         column pass F_0^-1 . K . F_0           (strided columns)
//   3-D:  x pass F_2 . P . F_2^-1,  y pass F_1,  z pass F_0^-1 K F_0,  y pass F_1^-1
//   1-D:  one launch runs every step of a chunk with the line in registers.
// Between passes psi is stored with the fastest axis in Fourier space
// (natural frequency order), the others in position space.
//
// Phase arithmetic is exact in fixed point: the potential uses f quantised to
// 32 bits with a per-instance power-of-two scale, and a 64-bit fraction of a
// turn per unit of f; the kinetic phase uses integer m^2 and a 64-bit fraction
// of a turn per unit of m^2.  The product modulo one turn is exact to 2^-32,
// so the FP32 sine/cosine only ever sees a reduced argument.
#include "qhd_device.cuh"
#include "qhd_kernels.h"
#include "qhd_sched.cuh"
#include "qhd_prep.cuh"

namespace qhd {

struct WarpSync {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

constexpr int ROW_THREADS = 128;

__host__ __device__ constexpr int axis_w(int n) {
    // columns per tile of a strided pass: 32-byte row segments at least,
    // 128 threads per block
    return n >= 1024 ? 4 : n >= 256 ? 8 : n >= 64 ? 16 : 32;
}

// --------------------------------------------------------------- row pass
template <int N>
__global__ void __launch_bounds__(ROW_THREADS) k_row(RowArgs a) {
    using C = LineCfg<N>;
    constexpr int E = C::E, T = C::T;
    constexpr int S = line_stride<N>(true, 0);
    extern __shared__ __align__(16) float4 smem4[];
    float4 *ptab = smem4;
    float2 *smem = reinterpret_cast<float2 *>(smem4 + PHASE_TAB);
    load_phase_tab(ptab, a.ptab);
    __syncthreads();
    const int lpb = blockDim.x / T;
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int64_t row = (int64_t)blockIdx.x * lpb + line;
    const bool valid = row < a.rows;
    const int64_t r = valid ? row : 0;
    float2 *g = a.psi + r * N;
    const uint32_t *fq = a.fq + r * N;
    float2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = g[t + T * e];
    float2 *sm = smem + (C::TWO_STAGE ? line * S : 0);
    if (a.mode & MODE_INV) line_fft<N, true>(x, sm, t, a.tw2, WarpSync{});
    const uint64_t c = a.pot[r / a.rows_per_inst];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        x[e] = apply_phase_tab(x[e], turns_mul(c, __ldg(&fq[t + T * e])) + a.dither, ptab);
    }
    if (a.mode & MODE_FWD) line_fft<N, false>(x, sm, t, a.tw2, WarpSync{});
    if (valid) {
#pragma unroll
        for (int e = 0; e < E; ++e) g[t + T * e] = x[e];
    }
}

// ------------------------------------------------------ strided axis pass
// Lines of length N at stride `inner`; a block owns W adjacent lines (columns)
// of one plane, lanes run along the columns so each global access moves W
// consecutive complex values per row.
// Strided passes over lines up to 256 points are compiled for 4 resident blocks
// per SM (issue-bound, latency hidden by warps); longer lines keep their
// registers (32 points per thread).
template <int N, int W>
__global__ void __launch_bounds__(W * LineCfg<N>::T, N <= 256 ? 4 : 1) k_axis(AxisArgs a) {
    using C = LineCfg<N>;
    constexpr int E = C::E, T = C::T;
    constexpr int S = line_stride<N>(false, W);
    extern __shared__ float2 smem[];
    const int c = threadIdx.x % W, t = threadIdx.x / W;
    const int64_t tiles = a.inner / W;
    const int64_t o = blockIdx.x / tiles;
    const int64_t ci = (blockIdx.x - o * tiles) * W + c;
    float2 *g = a.psi + o * (int64_t)N * a.inner + ci;
    float2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = g[(int64_t)(t + T * e) * a.inner];
    float2 *sm = smem + (C::TWO_STAGE ? c * S : 0);
    // zero-mode split (qhd_device.cuh) in the forward-kinetic-inverse pass, for
    // the tile holding column 0 (frequency 0 of the other axes) of each
    // instance: the T threads of a column span several warps, so their partial
    // sums meet in shared memory behind the exchange buffer and every thread
    // adds them in the same order.
    constexpr int ALL3 = MODE_FWD | MODE_KIN | MODE_INV;
    const bool split0 = (a.mode & ALL3) == ALL3 && blockIdx.x == o * tiles;
    float2 sum = make_float2(0.f, 0.f), mean_part = make_float2(0.f, 0.f);
    if (split0) {
        float2 *red = smem + (C::TWO_STAGE ? W * S : 0);
        float2 s = x[0];
#pragma unroll
        for (int e = 1; e < E; ++e) s = cadd(s, x[e]);
        red[t * W + c] = s;
        __syncthreads();
        sum = red[c];
#pragma unroll
        for (int q = 1; q < T; ++q) sum = cadd(sum, red[q * W + c]);
        sub_line_mean<N, E>(x, sum);
    }
    if (a.mode & MODE_FWD) line_fft<N, false>(x, sm, t, a.tw2, BlockSync{});
    if (a.mode & MODE_KIN) {
        // axis 0 pass: plane index o is the instance.  Each per-axis factor is
        // an FP32 hi/lo pair applied with a compensated product: a table entry
        // is shared by every point with the same frequency index, so a plain
        // FP32 rounding of it would perturb the norm coherently.
        const float4 *kb = a.kt + (a.kt_batch == 1 ? 0 : o) * a.ksum;
        int64_t i1 = a.ndim == 2 ? ci : (ci >> a.log_n2);
        if (a.perm1_r) i1 = i1 / a.perm1_r + (int64_t)a.perm1_c * (i1 % a.perm1_r);
        const float4 k1 = __ldg(&kb[a.koff1 + i1]);
        float4 k2 = make_float4(1.f, 0.f, 0.f, 0.f);
        if (a.ndim == 3) k2 = __ldg(&kb[a.koff2 + (ci & ((1 << a.log_n2) - 1))]);
        auto kin = [&](float2 v, float4 k0) {
            float2 y = cmul_comp(v, make_float2(k0.x, k0.y), make_float2(k0.z, k0.w));
            y = cmul_comp(y, make_float2(k1.x, k1.y), make_float2(k1.z, k1.w));
            if (a.ndim == 3) y = cmul_comp(y, make_float2(k2.x, k2.y), make_float2(k2.z, k2.w));
            return y;
        };
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = kin(x[e], __ldg(&kb[t + T * e]));
        // the mean's part: N mu = sum through the factor of frequency 0
        if (split0) mean_part = kin(sum, __ldg(&kb[0]));
    }
    if (a.mode & MODE_INV) line_fft<N, true>(x, sm, t, a.tw2, BlockSync{});
    if (split0) {
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = cadd(x[e], mean_part);
    }
#pragma unroll
    for (int e = 0; e < E; ++e) g[(int64_t)(t + T * e) * a.inner] = x[e];
}

// --------------------------------------------- 1-D: a whole chunk per launch
template <int N>
__global__ void __launch_bounds__(ROW_THREADS) k_oned(OneDArgs a) {
    using C = LineCfg<N>;
    constexpr int E = C::E, T = C::T;
    constexpr int S = line_stride<N>(true, 0);
    extern __shared__ __align__(16) float4 smem4[];
    float4 *ptab = smem4;
    float2 *smem = reinterpret_cast<float2 *>(smem4 + PHASE_TAB);
    load_phase_tab(ptab, a.ptab);
    __syncthreads();
    const int lpb = blockDim.x / T;
    const int line = threadIdx.x / T, t = threadIdx.x % T;
    const int64_t row = (int64_t)blockIdx.x * lpb + line;
    const bool valid = row < a.batch;
    const int64_t b = valid ? row : 0;
    float2 *g = a.psi + b * N;
    const uint32_t *fq = a.fq + b * N;
    float2 x[E];
    uint32_t fv[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        x[e] = g[t + T * e];
        fv[e] = fq[t + T * e];
    }
    float2 *sm = smem + (C::TWO_STAGE ? line * S : 0);
    for (int j = 0; j < a.cnt; ++j) {
        const uint64_t c = a.pot[(int64_t)j * a.batch + b];
        const uint32_t dz = step_dither(a.dither_base + (uint64_t)j);
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = apply_phase_tab(x[e], turns_mul(c, fv[e]) + dz, ptab);
        // zero-mode split (qhd_device.cuh): the line is the whole instance, so
        // its zero mode is the global one
        const float2 sum = line_sum_lanes<E, T>(x);
        sub_line_mean<N, E>(x, sum);
        line_fft<N, false>(x, sm, t, a.tw2, WarpSync{});
        const float4 *kb = a.kt + ((int64_t)j * a.kt_batch + (a.kt_batch == 1 ? 0 : b)) * N;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float4 k0 = __ldg(&kb[t + T * e]);
            x[e] = cmul_comp(x[e], make_float2(k0.x, k0.y), make_float2(k0.z, k0.w));
        }
        const float4 z0 = __ldg(&kb[0]);
        const float2 mean_part = cmul_comp(sum, make_float2(z0.x, z0.y), make_float2(z0.z, z0.w));
        line_fft<N, true>(x, sm, t, a.tw2, WarpSync{});
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = cadd(x[e], mean_part);
    }
    if (a.final_phase) {
        const uint64_t c = a.pot[(int64_t)a.cnt * a.batch + b];
#pragma unroll
        for (int e = 0; e < E; ++e) x[e] = apply_phase_tab(x[e], turns_mul(c, fv[e]), ptab);
    }
    if (valid) {
#pragma unroll
        for (int e = 0; e < E; ++e) g[t + T * e] = x[e];
    }
}

// ------------------------------------------------------------- prep kernel
// Schedule evaluation at the step midpoints, the merged potential coefficients
// and the per-axis kinetic phase tables of one chunk of steps (qhd_prep.cuh).

__global__ void k_prep(PrepArgs a) {
    const int64_t jl = blockIdx.x;  // local step 0..cnt (cnt is the extra potential entry)
    const int64_t b = blockIdx.y;
    __shared__ uint64_t s_k[3];
    __shared__ double s_fd[3];
    if (threadIdx.x == 0) prep_coefficients(a, jl, b, s_k, s_fd);
    __syncthreads();
    if (jl >= a.cnt || b >= a.kt_batch) return;
    for (int i = threadIdx.x; i < a.ksum; i += blockDim.x) prep_kinetic_entry(a, jl, b, i, s_k, s_fd);
}

// ------------------------------------------------------------ small kernels
__global__ void k_uniform(float2 *psi, int64_t count, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        psi[i] = make_float2(v, 0.0f);
}

__global__ void k_minmax(const double *f, int64_t g, MinMaxPart *part) {
    const int64_t b = blockIdx.y;
    const double *fb = f + b * g;
    double mn = INFINITY, mx = -INFINITY;
    int64_t am = INT64_MAX, nf = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double v = fb[i];
        if (!isfinite(v)) {
            ++nf;
            continue;
        }
        if (v < mn || (v == mn && i < am)) {
            mn = v;
            am = i;
        }
        mx = fmax(mx, v);
    }
    __shared__ double s_mn[256], s_mx[256];
    __shared__ int64_t s_am[256], s_nf[256];
    s_mn[threadIdx.x] = mn;
    s_mx[threadIdx.x] = mx;
    s_am[threadIdx.x] = am;
    s_nf[threadIdx.x] = nf;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w /= 2) {
        if (threadIdx.x < w) {
            const int o = threadIdx.x + w;
            if (s_mn[o] < s_mn[threadIdx.x] || (s_mn[o] == s_mn[threadIdx.x] && s_am[o] < s_am[threadIdx.x])) {
                s_mn[threadIdx.x] = s_mn[o];
                s_am[threadIdx.x] = s_am[o];
            }
            s_mx[threadIdx.x] = fmax(s_mx[threadIdx.x], s_mx[o]);
            s_nf[threadIdx.x] += s_nf[o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        MinMaxPart p;
        p.fmin = s_mn[0];
        p.fmax = s_mx[0];
        p.argmin = s_am[0];
        p.nonfinite = s_nf[0];
        part[b * gridDim.x + blockIdx.x] = p;
    }
}

__global__ void k_quantize(const double *f, uint32_t *fq, const InstDev *inst, int64_t g, int64_t total) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const InstDev &p = inst[i / g];
        double q = rint(ldexp(f[i] - p.fmin, p.shift));
        q = fmin(fmax(q, 0.0), 4294967295.0);
        fq[i] = (uint32_t)q;
    }
}

// Observables: FP64 partial sums per block, then a fixed-order final sum.
__device__ __forceinline__ double block_sum(double v, double *sh) {
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

__global__ void k_obs_partial(ObsArgs a) {
    const int64_t b = blockIdx.y;
    const float2 *psi = a.psi + b * a.g;
    const double *f = a.f64 + b * a.g;
    const InstDev &ip = a.inst[b];
    double sn = 0.0, sf = 0.0, sp = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.g;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float2 z = psi[i];
        const double p = __dadd_rn(__dmul_rn((double)z.x, (double)z.x), __dmul_rn((double)z.y, (double)z.y));
        if (a.prob) a.prob[b * a.g + i] = (float)p;
        sn += p;
        sf += p * f[i];
        // Euclidean distance to x*, evaluated in the same operation order as a
        // plain loop over the axes from the last to the first
        int64_t rem = i;
        double r2 = 0.0;
        for (int d = a.ndim - 1; d >= 0; --d) {
            const int idx = (int)(rem & ((1 << a.log_n[d]) - 1));
            rem >>= a.log_n[d];
            const double dx = __dsub_rn(a.coord[a.coff[d] + idx], ip.xs[d]);
            r2 = __dadd_rn(r2, __dmul_rn(dx, dx));
        }
        if (sqrt(r2) < a.radius) sp += p;
    }
    __shared__ double sh[32];
    const double tn = block_sum(sn, sh);
    const double tf = block_sum(sf, sh);
    const double tp = block_sum(sp, sh);
    if (threadIdx.x == 0) {
        double *o = a.partial + (b * a.nblk + blockIdx.x) * 3;
        o[0] = tn;
        o[1] = tf;
        o[2] = tp;
    }
}

__global__ void k_obs_final(ObsArgs a) {
    const int64_t b = blockIdx.x;
    __shared__ double sh[3][256];
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int i = threadIdx.x; i < a.nblk; i += blockDim.x) s += a.partial[(b * a.nblk + i) * 3 + k];
        sh[k][threadIdx.x] = s;
    }
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w /= 2) {
        if (threadIdx.x < w)
            for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) a.result[b * 3 + k] = sh[k][0];
}

// ---------------------------------------------------------------- launchers
template <int N>
static cudaError_t row_impl(const RowArgs &a, cudaStream_t s) {
    using C = LineCfg<N>;
    constexpr int S = line_stride<N>(true, 0);
    const int lpb = ROW_THREADS / C::T;
    const int64_t blocks = (a.rows + lpb - 1) / lpb;
    const size_t sm = PHASE_TAB * sizeof(float4) + (C::TWO_STAGE ? (size_t)lpb * S * sizeof(float2) : 0);
    k_row<N><<<(unsigned)blocks, ROW_THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

template <int N, int W>
static cudaError_t axis_w_impl(const AxisArgs &a, cudaStream_t s) {
    using C = LineCfg<N>;
    constexpr int S = line_stride<N>(false, W);
    const int64_t blocks = a.planes * (a.inner / W);
    // exchange buffer, then the column partial sums of the zero-mode split
    const size_t xch = (C::TWO_STAGE ? (size_t)W * S * sizeof(float2) : 0) + (size_t)W * C::T * sizeof(float2);
    k_axis<N, W><<<(unsigned)blocks, W * C::T, xch, s>>>(a);
    return cudaGetLastError();
}

template <int N>
static cudaError_t axis_impl(const AxisArgs &a, cudaStream_t s) {
    constexpr int WD = axis_w(N);
    if (a.inner >= WD) return axis_w_impl<N, WD>(a, s);
    if constexpr (WD > 16) if (a.inner >= 16) return axis_w_impl<N, 16>(a, s);
    if constexpr (WD > 8) if (a.inner >= 8) return axis_w_impl<N, 8>(a, s);
    if constexpr (WD > 4) if (a.inner >= 4) return axis_w_impl<N, 4>(a, s);
    if (a.inner >= 2) return axis_w_impl<N, 2>(a, s);
    return axis_w_impl<N, 1>(a, s);
}

template <int N>
static cudaError_t oned_impl(const OneDArgs &a, cudaStream_t s) {
    using C = LineCfg<N>;
    constexpr int S = line_stride<N>(true, 0);
    const int lpb = ROW_THREADS / C::T;
    const int64_t blocks = (a.batch + lpb - 1) / lpb;
    const size_t sm = PHASE_TAB * sizeof(float4) + (C::TWO_STAGE ? (size_t)lpb * S * sizeof(float2) : 0);
    k_oned<N><<<(unsigned)blocks, ROW_THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

#define QHD_DISPATCH_N(n, fn, ...)                        \
    switch (n) {                                          \
    case 2: return fn<2>(__VA_ARGS__);                    \
    case 4: return fn<4>(__VA_ARGS__);                    \
    case 8: return fn<8>(__VA_ARGS__);                    \
    case 16: return fn<16>(__VA_ARGS__);                  \
    case 32: return fn<32>(__VA_ARGS__);                  \
    case 64: return fn<64>(__VA_ARGS__);                  \
    case 128: return fn<128>(__VA_ARGS__);                \
    case 256: return fn<256>(__VA_ARGS__);                \
    case 512: return fn<512>(__VA_ARGS__);                \
    case 1024: return fn<1024>(__VA_ARGS__);              \
    default: return cudaErrorInvalidValue;                \
    }

cudaError_t launch_row(int n, const RowArgs &a, cudaStream_t s) { QHD_DISPATCH_N(n, row_impl, a, s) }
cudaError_t launch_axis(int n, const AxisArgs &a, cudaStream_t s) { QHD_DISPATCH_N(n, axis_impl, a, s) }
cudaError_t launch_oned(int n, const OneDArgs &a, cudaStream_t s) { QHD_DISPATCH_N(n, oned_impl, a, s) }

cudaError_t launch_prep(const PrepArgs &a, cudaStream_t s) {
    dim3 grid((unsigned)(a.cnt + 1), (unsigned)a.batch);
    k_prep<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_uniform(float2 *psi, int64_t count, float value, cudaStream_t s) {
    int64_t blocks = (count + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_uniform<<<(unsigned)blocks, 256, 0, s>>>(psi, count, value);
    return cudaGetLastError();
}

cudaError_t launch_minmax(const double *f, int64_t g, int64_t batch, MinMaxPart *part, int nblk,
                          cudaStream_t s) {
    k_minmax<<<dim3((unsigned)nblk, (unsigned)batch), 256, 0, s>>>(f, g, part);
    return cudaGetLastError();
}

cudaError_t launch_quantize(const double *f, uint32_t *fq, const InstDev *inst, int64_t g,
                            int64_t batch, cudaStream_t s) {
    const int64_t total = g * batch;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_quantize<<<(unsigned)blocks, 256, 0, s>>>(f, fq, inst, g, total);
    return cudaGetLastError();
}

cudaError_t launch_observables(const ObsArgs &a, int64_t batch, cudaStream_t s) {
    k_obs_partial<<<dim3((unsigned)a.nblk, (unsigned)batch), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_obs_final<<<(unsigned)batch, 256, 0, s>>>(a);
    return cudaGetLastError();
}

void plan_of(int n, int *r1, int *r2) {
    switch (n) {
#define QHD_PLAN_CASE(N)      \
    case N:                   \
        *r1 = Plan<N>::R1;    \
        *r2 = Plan<N>::R2;    \
        return;
        QHD_PLAN_CASE(2) QHD_PLAN_CASE(4) QHD_PLAN_CASE(8) QHD_PLAN_CASE(16) QHD_PLAN_CASE(32)
        QHD_PLAN_CASE(64) QHD_PLAN_CASE(128) QHD_PLAN_CASE(256) QHD_PLAN_CASE(512) QHD_PLAN_CASE(1024)
#undef QHD_PLAN_CASE
    default:
        *r1 = 0;
        *r2 = 0;
    }
}

bool supported_n(int64_t n) { return n >= 2 && n <= 1024 && (n & (n - 1)) == 0; }

}  // namespace qhd
