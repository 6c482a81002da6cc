// qhd_spectrum.cu -- the QHD Hamiltonian as an operator, and its lowest
// eigenpairs by Lanczos (the probability spectrum and the energy ratio E1/E0
// of the paper's section on the three phases of QHD).
//
// H(t) = e^{phi_t} (-Lap/2) + e^{chi_t} f on one instance's mesh.  The
// kinetic part goes through the same line transforms as the time stepping:
// forward along every axis, a real factor per frequency (e^{phi} |k|^2 / 2 / G,
// or the finite-difference eigenvalue), inverse along every axis; the
// potential part is a pointwise product with the FP64 f.  Vectors are
// complex64; every inner product accumulates in FP64.
//
// Lanczos: from a seeded random start vector, each step applies H, removes the
// components along all previous basis vectors twice (classical Gram-Schmidt,
// repeated), and normalises.  The projected matrix is tridiagonal with
// alpha_j = <v_j, H v_j> and beta_j = ||w_j||; its lowest eigenvalues come from
// bisection on Sturm counts, its eigenvectors from inverse iteration with a
// pivoted tridiagonal solve, and the Ritz vectors u = V y are formed on the
// device.  Residuals ||H u - theta u|| are computed, not estimated.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "qhd.h"
#include "qhd_device.cuh"
#include "qhd_spectrum.h"

namespace qhd {

namespace {

constexpr int HT = 128;   // threads per block of the line passes
constexpr int RT = 256;   // threads per block of the vector kernels
constexpr int DOT_BLOCKS = 64;

struct SyncAll {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

// One transform along one axis of one instance: lines of N points at stride s.
struct HPass {
    float2 *data;
    int64_t s;       // element stride along the axis
    int64_t lines;   // lines in the instance: G / N
    const float4 *tw2;
};

template <int N>
__global__ void __launch_bounds__(HT) k_hpass(HPass a, int inv) {
    using C = LineCfg<N>;
    constexpr int E = C::E, T = C::T;
    constexpr int LPB = (HT / T) > 0 ? HT / T : 1;
    constexpr int S = C::TWO_STAGE ? C::PADDED : 1;
    __shared__ float2 sm_all[LPB * S];
    const int li = threadIdx.x / T, t = threadIdx.x - li * T;
    const int64_t line = (int64_t)blockIdx.x * LPB + li;
    const bool valid = li < LPB && line < a.lines;
    const int64_t l = valid ? line : 0;
    const int64_t outer = l / a.s, inner = l - outer * a.s;
    float2 *g = a.data + outer * (int64_t)N * a.s + inner;
    float2 x[E];
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = g[(int64_t)(t + T * e) * a.s];
    float2 *sm = sm_all + (li < LPB ? li : 0) * S;
    if (inv) line_fft<N, true>(x, sm, t, a.tw2, SyncAll{});
    else line_fft<N, false>(x, sm, t, a.tw2, SyncAll{});
    if (valid) {
#pragma unroll
        for (int e = 0; e < E; ++e) g[(int64_t)(t + T * e) * a.s] = x[e];
    }
}

// Kinetic factor in Fourier space: data[i] *= coef * sum_d lambda_d(m_d).
struct HMult {
    float2 *data;
    int64_t g;
    int n[3];
    double len[3];
    int kinetic;
    double coef;  // e^{phi} / (2 G)
};

__device__ __forceinline__ double kin_eig(int i, int n, double len, int kinetic) {
    if (n == 1) return 0.0;  // an axis the grid does not have
    const int m = i < n / 2 ? i : i - n;
    if (kinetic == QHD_KINETIC_FD2) {
        const double h = len / (double)n;
        const double s = sinpi((double)m / (double)n);
        return 4.0 * s * s / (h * h);
    }
    const double k = 2.0 * 3.141592653589793238462643383279502884 * (double)m / len;
    return k * k;
}

__global__ void k_hmult(HMult a) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.g; i += (int64_t)gridDim.x * blockDim.x) {
        const int i2 = (int)(i % a.n[2]);
        const int i1 = (int)((i / a.n[2]) % a.n[1]);
        const int i0 = (int)(i / ((int64_t)a.n[1] * a.n[2]));
        const double lam = kin_eig(i0, a.n[0], a.len[0], a.kinetic) + kin_eig(i1, a.n[1], a.len[1], a.kinetic) +
                           kin_eig(i2, a.n[2], a.len[2], a.kinetic);
        const float c = (float)(a.coef * lam);
        const float2 v = a.data[i];
        a.data[i] = make_float2(v.x * c, v.y * c);
    }
}

// out += b f in
__global__ void k_hadd(float2 *out, const float2 *in, const double *f, double b, int64_t g) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
        const float w = (float)(b * f[i]);
        const float2 v = in[i], o = out[i];
        out[i] = make_float2(fmaf(w, v.x, o.x), fmaf(w, v.y, o.y));
    }
}

// part[j * DOT_BLOCKS + blk] = partial sum over the block's chunk of conj(V_j) w
__global__ void k_lz_dots(const float2 *V, int64_t vstride, int nvec, const float2 *w, int64_t g, double2 *part) {
    __shared__ double sr[RT], si[RT];
    const int j = blockIdx.y;
    const float2 *v = V + (int64_t)j * vstride;
    double re = 0, im = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = v[i], b = w[i];
        re += (double)a.x * b.x + (double)a.y * b.y;
        im += (double)a.x * b.y - (double)a.y * b.x;
    }
    sr[threadIdx.x] = re;
    si[threadIdx.x] = im;
    __syncthreads();
    for (int s = RT / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sr[threadIdx.x] += sr[threadIdx.x + s];
            si[threadIdx.x] += si[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)j * gridDim.x + blockIdx.x] = make_double2(sr[0], si[0]);
}

__global__ void k_lz_reduce(const double2 *part, int nvec, int nblk, double2 *c) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nvec) return;
    double re = 0, im = 0;
    for (int b = 0; b < nblk; ++b) {
        re += part[(int64_t)j * nblk + b].x;
        im += part[(int64_t)j * nblk + b].y;
    }
    c[j] = make_double2(re, im);
}

// w -= sum_j c_j V_j
__global__ void k_lz_sub(float2 *w, const float2 *V, int64_t vstride, int nvec, const double2 *c, int64_t g) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
        double re = w[i].x, im = w[i].y;
        for (int j = 0; j < nvec; ++j) {
            const float2 v = V[(int64_t)j * vstride + i];
            const double2 cj = c[j];
            re -= cj.x * v.x - cj.y * v.y;
            im -= cj.x * v.y + cj.y * v.x;
        }
        w[i] = make_float2((float)re, (float)im);
    }
}

// out = sum_j y_j V_j (real coefficients)
__global__ void k_lz_combine(float2 *out, const float2 *V, int64_t vstride, int nvec, const double *y, int64_t g) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
        double re = 0, im = 0;
        for (int j = 0; j < nvec; ++j) {
            const float2 v = V[(int64_t)j * vstride + i];
            re += y[j] * v.x;
            im += y[j] * v.y;
        }
        out[i] = make_float2((float)re, (float)im);
    }
}

__global__ void k_lz_scale(float2 *v, double s, int64_t g) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = v[i];
        v[i] = make_float2((float)(a.x * s), (float)(a.y * s));
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// start vector: independent uniform(-1/2, 1/2) parts from a counter hash
__global__ void k_lz_random(float2 *v, int64_t g, uint64_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t h1 = mix64(seed * 0x9E3779B97F4A7C15ull + 2 * (uint64_t)i + 1);
        const uint64_t h2 = mix64(seed * 0x9E3779B97F4A7C15ull + 2 * (uint64_t)i + 2);
        v[i] = make_float2((float)((double)(h1 >> 11) * 0x1.0p-53 - 0.5), (float)((double)(h2 >> 11) * 0x1.0p-53 - 0.5));
    }
}

int vec_grid(int64_t g) {
    int64_t b = (g + RT - 1) / RT;
    if (b > 152 * 8) b = 152 * 8;
    return b < 1 ? 1 : (int)b;
}

size_t al(size_t v) { return (v + 255) & ~size_t(255); }

template <int N>
cudaError_t hpass_n(const HPass &p, int inv, cudaStream_t s) {
    using C = LineCfg<N>;
    constexpr int T = C::T;
    constexpr int LPB = (HT / T) > 0 ? HT / T : 1;
    const int64_t blocks = (p.lines + LPB - 1) / LPB;
    k_hpass<N><<<(unsigned)blocks, HT, 0, s>>>(p, inv);
    return cudaGetLastError();
}

cudaError_t hpass(int n, const HPass &p, int inv, cudaStream_t s) {
    switch (n) {
    case 2: return hpass_n<2>(p, inv, s);
    case 4: return hpass_n<4>(p, inv, s);
    case 8: return hpass_n<8>(p, inv, s);
    case 16: return hpass_n<16>(p, inv, s);
    case 32: return hpass_n<32>(p, inv, s);
    case 64: return hpass_n<64>(p, inv, s);
    case 128: return hpass_n<128>(p, inv, s);
    case 256: return hpass_n<256>(p, inv, s);
    case 512: return hpass_n<512>(p, inv, s);
    case 1024: return hpass_n<1024>(p, inv, s);
    default: return cudaErrorInvalidValue;
    }
}

// out = H in for instance inst (out != in)
cudaError_t apply_h(const CtxView &v, int64_t inst, double a, double b, const float2 *in, float2 *out) {
    const int64_t g = v.g;
    cudaError_t e = cudaMemcpyAsync(out, in, g * sizeof(float2), cudaMemcpyDeviceToDevice, v.stream);
    if (e != cudaSuccess) return e;
    int64_t stride[3];
    stride[v.ndim - 1] = 1;
    for (int d = v.ndim - 2; d >= 0; --d) stride[d] = stride[d + 1] * v.n[d + 1];
    for (int d = v.ndim - 1; d >= 0; --d) {
        const HPass p{out, stride[d], g / v.n[d], v.tw[d]};
        if ((e = hpass((int)v.n[d], p, 0, v.stream)) != cudaSuccess) return e;
    }
    HMult m{};
    m.data = out;
    m.g = g;
    for (int d = 0; d < 3; ++d) {
        m.n[d] = (int)v.n[d];
        m.len[d] = v.len[d];
    }
    m.kinetic = v.kinetic;
    m.coef = a / (2.0 * (double)g);
    k_hmult<<<vec_grid(g), RT, 0, v.stream>>>(m);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int d = 0; d < v.ndim; ++d) {
        const HPass p{out, stride[d], g / v.n[d], v.tw[d]};
        if ((e = hpass((int)v.n[d], p, 1, v.stream)) != cudaSuccess) return e;
    }
    k_hadd<<<vec_grid(g), RT, 0, v.stream>>>(out, in, v.f64 + inst * g, b, g);
    return cudaGetLastError();
}

// ------------------------------------------------ symmetric tridiagonal (host)
// Number of eigenvalues below x (Sturm count of the LDL^T pivots).
int sturm_count(const std::vector<double> &al_, const std::vector<double> &be, double x) {
    const int n = (int)al_.size();
    int cnt = 0;
    double q = al_[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < n; ++i) {
        if (q == 0.0) q = 1e-300;
        q = al_[i] - x - be[i - 1] * be[i - 1] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// i-th smallest eigenvalue (0-based) by bisection
double tri_eig(const std::vector<double> &al_, const std::vector<double> &be, int i, double lo, double hi) {
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(al_, be, mid) >= i + 1) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Solve (T - s I) x = r by Gaussian elimination with partial pivoting on the
// tridiagonal band (the band grows to two superdiagonals under row swaps).
void tri_solve(const std::vector<double> &al_, const std::vector<double> &be, double s, std::vector<double> &x) {
    const int n = (int)al_.size();
    std::vector<double> dl(n, 0.0), d(n), du(n, 0.0), du2(n, 0.0);
    for (int i = 0; i < n; ++i) d[i] = al_[i] - s;
    for (int i = 0; i + 1 < n; ++i) {
        dl[i] = be[i];
        du[i] = be[i];
    }
    std::vector<int> swapped(n, 0);
    const double tiny = 1e-300;
    for (int i = 0; i + 1 < n; ++i) {
        if (std::fabs(d[i]) >= std::fabs(dl[i])) {
            if (d[i] == 0.0) d[i] = tiny;
            const double f = dl[i] / d[i];
            dl[i] = f;
            d[i + 1] -= f * du[i];
            x[i + 1] -= f * x[i];
            du2[i] = 0.0;
        } else {
            // swap rows i and i + 1
            const double f = d[i] / dl[i];
            d[i] = dl[i];
            const double tmp = d[i + 1];
            d[i + 1] = du[i] - f * tmp;
            du2[i] = i + 2 < n ? du[i + 1] : 0.0;
            if (i + 2 < n) du[i + 1] = -f * du2[i];
            du[i] = tmp;
            std::swap(x[i], x[i + 1]);
            x[i + 1] -= f * x[i];
            dl[i] = f;
            swapped[i] = 1;
        }
    }
    if (d[n - 1] == 0.0) d[n - 1] = tiny;
    // back substitution with the upper band (d, du, du2)
    x[n - 1] /= d[n - 1];
    if (n > 1) x[n - 2] = (x[n - 2] - du[n - 2] * x[n - 1]) / d[n - 2];
    for (int i = n - 3; i >= 0; --i) x[i] = (x[i] - du[i] * x[i + 1] - du2[i] * x[i + 2]) / d[i];
}

}  // namespace

}  // namespace qhd

using namespace qhd;

extern "C" {

size_t qhd_spectrum_workspace_bytes(const qhd_ctx *ctx, int m) {
    const int64_t g = ctx_grid_points(ctx);
    if (g <= 0 || m < 2 || m > 1024) return 0;
    size_t t = 0;
    t += al((size_t)(m + 1) * g * sizeof(float2));  // Lanczos basis
    t += 2 * al((size_t)g * sizeof(float2));        // Ritz vector, H times it
    t += al((size_t)DOT_BLOCKS * (m + 1) * sizeof(double2));
    t += al((size_t)(m + 1) * sizeof(double2));
    t += al((size_t)(m + 1) * sizeof(double));
    return t;
}

qhd_status qhd_apply_hamiltonian(qhd_ctx *ctx, int64_t inst, double t, const void *in_dev, void *out_dev) {
    CtxView v;
    qhd_status st = ctx_view(ctx, &v);
    if (st != QHD_OK) return st;
    if (inst < 0 || inst >= v.batch || !in_dev || !out_dev || in_dev == out_dev || !std::isfinite(t))
        return ctx_fail(ctx, QHD_ERR_INVALID_ARG, "apply_hamiltonian: bad instance, time or buffers");
    double a = 0, b = 0;
    ctx_sched_ab(ctx, inst, t, &a, &b);
    cudaError_t e = apply_h(v, inst, a, b, (const float2 *)in_dev, (float2 *)out_dev);
    if (e != cudaSuccess) return ctx_fail(ctx, QHD_ERR_CUDA, cudaGetErrorString(e));
    return QHD_OK;
}

qhd_status qhd_lowest_eigenpairs(qhd_ctx *ctx, int64_t inst, double t, int m, int k, uint64_t seed, void *work_dev,
                                 size_t work_bytes, double *eigvals, double *residuals, double *overlaps,
                                 void *eigvecs_dev) {
    CtxView v;
    qhd_status st = ctx_view(ctx, &v);
    if (st != QHD_OK) return st;
    const int64_t g = v.g;
    if (inst < 0 || inst >= v.batch || m < 2 || m > 1024 || (int64_t)m > g || k < 1 || k > m || !std::isfinite(t))
        return ctx_fail(ctx, QHD_ERR_INVALID_ARG, "lowest_eigenpairs: bad instance, time, m or k");
    const size_t need = qhd_spectrum_workspace_bytes(ctx, m);
    if (!work_dev || ((uintptr_t)work_dev & 255) || work_bytes < need)
        return ctx_fail(ctx, QHD_ERR_WORKSPACE, "lowest_eigenpairs: workspace too small or misaligned");
    cudaStream_t s = v.stream;
    char *p = (char *)work_dev;
    float2 *V = (float2 *)p;
    p += al((size_t)(m + 1) * g * sizeof(float2));
    float2 *u = (float2 *)p;
    p += al((size_t)g * sizeof(float2));
    float2 *hu = (float2 *)p;
    p += al((size_t)g * sizeof(float2));
    double2 *part = (double2 *)p;
    p += al((size_t)DOT_BLOCKS * (m + 1) * sizeof(double2));
    double2 *cdev = (double2 *)p;
    p += al((size_t)(m + 1) * sizeof(double2));
    double *ydev = (double *)p;

    double a = 0, b = 0;
    ctx_sched_ab(ctx, inst, t, &a, &b);
    const int gb = vec_grid(g);
    std::vector<double2> ch((size_t)m + 1);
    cudaError_t e = cudaSuccess;
    // c[0..nvec) = V^H w on the host as well (synchronises)
    auto dots = [&](const float2 *Vb, int nvec, const float2 *w) -> cudaError_t {
        k_lz_dots<<<dim3(DOT_BLOCKS, (unsigned)nvec), RT, 0, s>>>(Vb, g, nvec, w, g, part);
        k_lz_reduce<<<(nvec + 127) / 128, 128, 0, s>>>(part, nvec, DOT_BLOCKS, cdev);
        cudaError_t r = cudaMemcpyAsync(ch.data(), cdev, nvec * sizeof(double2), cudaMemcpyDeviceToHost, s);
        if (r == cudaSuccess) r = cudaStreamSynchronize(s);
        return r;
    };
#define SPEC_TRY(call)                                                                \
    do {                                                                              \
        e = (call);                                                                   \
        if (e != cudaSuccess) return ctx_fail(ctx, QHD_ERR_CUDA, cudaGetErrorString(e)); \
    } while (0)

    // start vector
    k_lz_random<<<gb, RT, 0, s>>>(V, g, seed);
    SPEC_TRY(cudaGetLastError());
    SPEC_TRY(dots(V, 1, V));
    k_lz_scale<<<gb, RT, 0, s>>>(V, 1.0 / std::sqrt(ch[0].x), g);
    std::vector<double> alpha, beta;
    int meff = 0;
    for (int j = 0; j < m; ++j) {
        float2 *vj = V + (int64_t)j * g, *w = V + (int64_t)(j + 1) * g;
        SPEC_TRY(apply_h(v, inst, a, b, vj, w));
        double aj = 0;
        for (int pass = 0; pass < 2; ++pass) {
            SPEC_TRY(dots(V, j + 1, w));
            aj += ch[j].x;
            k_lz_sub<<<gb, RT, 0, s>>>(w, V, g, j + 1, cdev, g);
            SPEC_TRY(cudaGetLastError());
        }
        alpha.push_back(aj);
        meff = j + 1;
        SPEC_TRY(dots(w, 1, w));
        const double bj = std::sqrt(std::max(ch[0].x, 0.0));
        if (j + 1 == m || !(bj > 1e-12 * std::max(1.0, std::fabs(aj)))) break;
        beta.push_back(bj);
        k_lz_scale<<<gb, RT, 0, s>>>(w, 1.0 / bj, g);
    }
    if (k > meff) return ctx_fail(ctx, QHD_ERR_INVALID_ARG, "lowest_eigenpairs: the Krylov space closed before k vectors");
    beta.resize((size_t)meff - 1);
    // Gershgorin bounds of the tridiagonal matrix
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < meff; ++i) {
        const double r = (i > 0 ? std::fabs(beta[i - 1]) : 0.0) + (i + 1 < meff ? std::fabs(beta[i]) : 0.0);
        lo = std::min(lo, alpha[i] - r);
        hi = std::max(hi, alpha[i] + r);
    }
    const double span = std::max(hi - lo, 1e-300);
    lo -= 1e-9 * span;
    hi += 1e-9 * span;
    std::vector<std::vector<double>> Y;
    for (int i = 0; i < k; ++i) {
        const double th = tri_eig(alpha, beta, i, lo, hi);
        // inverse iteration for the eigenvector of the tridiagonal matrix
        std::vector<double> y((size_t)meff);
        for (int q = 0; q < meff; ++q) y[q] = 1.0 + 0.01 * std::sin(1.0 + q * 0.7 + i);
        for (int it = 0; it < 4; ++it) {
            tri_solve(alpha, beta, th + 1e-13 * span, y);
            for (const auto &yp : Y) {  // keep clusters orthogonal
                double d = 0;
                for (int q = 0; q < meff; ++q) d += yp[q] * y[q];
                for (int q = 0; q < meff; ++q) y[q] -= d * yp[q];
            }
            double nn = 0;
            for (double c : y) nn += c * c;
            nn = std::sqrt(nn);
            for (double &c : y) c /= nn;
        }
        Y.push_back(y);
        // Ritz vector, its residual and its overlap with the state
        SPEC_TRY(cudaMemcpyAsync(ydev, y.data(), meff * sizeof(double), cudaMemcpyHostToDevice, s));
        k_lz_combine<<<gb, RT, 0, s>>>(u, V, g, meff, ydev, g);
        SPEC_TRY(cudaGetLastError());
        SPEC_TRY(dots(u, 1, u));
        k_lz_scale<<<gb, RT, 0, s>>>(u, 1.0 / std::sqrt(ch[0].x), g);
        SPEC_TRY(apply_h(v, inst, a, b, u, hu));
        SPEC_TRY(dots(u, 1, hu));
        const double rq = ch[0].x;  // Rayleigh quotient of the normalised Ritz vector
        if (eigvals) eigvals[i] = rq;
        if (residuals) {
            const double2 c0 = make_double2(rq, 0.0);
            SPEC_TRY(cudaMemcpyAsync(cdev, &c0, sizeof(double2), cudaMemcpyHostToDevice, s));
            k_lz_sub<<<gb, RT, 0, s>>>(hu, u, g, 1, cdev, g);
            SPEC_TRY(cudaGetLastError());
            SPEC_TRY(dots(hu, 1, hu));
            residuals[i] = std::sqrt(std::max(ch[0].x, 0.0));
        }
        if (overlaps) {
            const float2 *psi = v.psi + inst * g;
            SPEC_TRY(dots(psi, 1, psi));
            const double pn = ch[0].x;
            SPEC_TRY(dots(u, 1, psi));
            overlaps[i] = (ch[0].x * ch[0].x + ch[0].y * ch[0].y) / (pn > 0 ? pn : 1.0);
        }
        if (eigvecs_dev)
            SPEC_TRY(cudaMemcpyAsync((float2 *)eigvecs_dev + (int64_t)i * g, u, g * sizeof(float2),
                                     cudaMemcpyDeviceToDevice, s));
    }
    SPEC_TRY(cudaStreamSynchronize(s));
#undef SPEC_TRY
    return QHD_OK;
}

}  // extern "C"
