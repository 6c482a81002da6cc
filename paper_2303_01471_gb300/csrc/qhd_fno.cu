// qhd_fno.cu -- Fourier-neural-operator surrogate of the QHD solver: maps the
// sampled objective f (and the schedule scale sigma) on an n x n mesh to the
// distribution |psi(T)|^2 that the split-operator path computes.
//
// Network (per instance, channel-last activations [point][channel]):
//   features  q = ((f - mean f) / std f, sigma, x, y)                 (4 channels)
//   lift      v0 = Wl q + bl                                          (C channels)
//   layer l   a_l = SC_l(v_l) + Ww_l v_l + bw_l,  v_{l+1} = gelu(a_l) (no gelu after the last layer)
//   SC_l      truncated spectral convolution: V^(kx,ky) = sum_{x,y} v e^{-2 pi i (kx x + ky y)/n} for
//             kx in {0..M-1} U {n-M..n-1}, ky in {0..M-1};  W^ = R_l(kx,ky) V^  (C x C complex);
//             u(x,y) = n^-2 sum_{kx,ky} c_ky Re(W^ e^{+2 pi i (kx x + ky y)/n}),  c_0 = 1, c_ky = 2
//   project   h = gelu(Wp1 v_L + bp1) (H channels),  z = Wp2 h + bp2
//   output    p = softmax over the mesh of z   (a distribution, like |psi|^2)
//   loss      KL(p_true || p) summed over the batch, divided by B;  dL/dz = (p - p_true) / B
// The spectral convolution runs as two separable truncated DFT stages per
// direction (axis 1 over ky, then axis 0 over kx) in shared memory; the mode
// mixing sits between the axis-0 stages.  Every backward kernel is the
// adjoint of a forward one: the adjoint of a truncated DFT stage is the
// opposite-direction stage over the same modes.
//
// Precision: activations are stored as BF16 (or FP32 for gradient checks),
// all arithmetic and every accumulation is FP32, weight gradients are reduced
// through FP64 block partials, weights and Adam moments are FP32.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "qhd.h"

namespace {

constexpr int FT = 256;     // threads per block
constexpr int WG_PTS = 32;  // points per shared-memory tile of the weight-gradient kernel

struct Dims {
    int n, C, M, MX, H, L;
    int64_t B;
    __host__ __device__ int64_t G() const { return (int64_t)n * n; }
    __host__ __device__ int64_t P() const { return B * G(); }
};

template <typename T> __device__ __forceinline__ float ldv(const T *p);
template <> __device__ __forceinline__ float ldv<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float ldv<__nv_bfloat16>(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
template <typename T> __device__ __forceinline__ void stv(T *p, float v);
template <> __device__ __forceinline__ void stv<float>(float *p, float v) { *p = v; }
template <> __device__ __forceinline__ void stv<__nv_bfloat16>(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

__device__ __forceinline__ float gelu(float a) { return 0.5f * a * (1.f + erff(a * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float a) {
    return 0.5f * (1.f + erff(a * 0.70710678118654752f)) + a * 0.39894228040143268f * expf(-0.5f * a * a);
}

// cos / sin of 2 pi k / n for k < n into shared memory
__device__ __forceinline__ void twiddle_table(float *cs, float *sn, int n) {
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        float s, c;
        sincospif(2.f * (float)k / (float)n, &s, &c);
        cs[k] = c;
        sn[k] = s;
    }
}

// frequency of retained axis-0 mode index kx (M low, M high)
__device__ __forceinline__ int kx_freq(int kx, int M, int n) { return kx < M ? kx : n - 2 * M + kx; }

// ------------------------------------------------------------- features, lift
// Per-instance mean and 1/std of f (FP64).
__global__ void k_fno_fstats(const double *f, int64_t G, double2 *stats) {
    const int64_t b = blockIdx.x;
    double s = 0, s2 = 0;
    for (int64_t i = threadIdx.x; i < G; i += blockDim.x) {
        const double v = f[b * G + i];
        s += v;
        s2 += v * v;
    }
    __shared__ double r1[FT], r2[FT];
    r1[threadIdx.x] = s;
    r2[threadIdx.x] = s2;
    __syncthreads();
    for (int w = FT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            r1[threadIdx.x] += r1[threadIdx.x + w];
            r2[threadIdx.x] += r2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = r1[0] / (double)G;
        const double var = r2[0] / (double)G - mean * mean;
        stats[b] = make_double2(mean, var > 0 ? 1.0 / sqrt(var) : 1.0);
    }
}

template <typename T>
__global__ void k_fno_lift(const double *f, const float *sigma, const double2 *stats, const float *W, const float *bias,
                           Dims d, float *feat, T *v0) {
    const int64_t P = d.P(), G = d.G();
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = p / G, g = p - b * G;
        const double2 st = stats[b];
        float q[4];
        q[0] = (float)((f[p] - st.x) * st.y);
        q[1] = sigma[b];
        q[2] = (float)(g / d.n) / (float)d.n;
        q[3] = (float)(g % d.n) / (float)d.n;
        *reinterpret_cast<float4 *>(&feat[p * 4]) = make_float4(q[0], q[1], q[2], q[3]);
        if (sizeof(T) == 2 && d.C == 32) {
            // BF16 at width 32: the point's 64 bytes as four 16-byte stores
            uint32_t w[16];
#pragma unroll
            for (int c = 0; c < 32; c += 2) {
                float a0 = bias[c], a1 = bias[c + 1];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    a0 = fmaf(W[c * 4 + j], q[j], a0);
                    a1 = fmaf(W[(c + 1) * 4 + j], q[j], a1);
                }
                const __nv_bfloat162 h = __floats2bfloat162_rn(a0, a1);
                w[c / 2] = *reinterpret_cast<const uint32_t *>(&h);
            }
            uint4 *dst = reinterpret_cast<uint4 *>(&v0[p * d.C]);
#pragma unroll
            for (int k = 0; k < 4; ++k) dst[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
        } else {
            for (int c = 0; c < d.C; ++c) {
                float a = bias[c];
                for (int j = 0; j < 4; ++j) a = fmaf(W[c * 4 + j], q[j], a);
                stv(&v0[p * d.C + c], a);
            }
        }
    }
}

// ------------------------------------------------ axis-1 truncated DFT stage
// out[b][x][ky][c] = s(ky) sum_y in[b][x][y][c] e^{-2 pi i ky y / n}, s(0) = s0, s(ky>0) = s1.
// One block per (b, x) row.
template <typename T>
__global__ void k_fno_dfty(const T *in, Dims d, float s0, float s1, float2 *out) {
    extern __shared__ float smem[];
    const int n = d.n, C = d.C, M = d.M;
    float *row = smem;  // n * C
    float *cs = row + n * C, *sn = cs + n;
    const int64_t bx = blockIdx.x;  // b * n + x
    const T *src = in + bx * (int64_t)n * C;
    for (int i = threadIdx.x; i < n * C; i += blockDim.x) row[i] = ldv(&src[i]);
    twiddle_table(cs, sn, n);
    __syncthreads();
    for (int o = threadIdx.x; o < M * C; o += blockDim.x) {
        const int ky = o / C, c = o - ky * C;
        float re = 0.f, im = 0.f;
        for (int y = 0; y < n; ++y) {
            const int k = (ky * y) & (n - 1);
            const float v = row[y * C + c];
            re = fmaf(v, cs[k], re);
            im = fmaf(-v, sn[k], im);
        }
        const float s = ky == 0 ? s0 : s1;
        out[bx * (int64_t)M * C + o] = make_float2(re * s, im * s);
    }
}

// ------------------------------------- axis-0 stages with the mode mixing
// One block per (b, ky).  X[x][c] = in[b][x][ky][c];
//   Y1[kx][c] = sum_x X[x][c] e^{-2 pi i f(kx) x / n}                 (stored to mid)
//   forward: Y2[kx][o] = sum_i R[kx][ky][i][o] Y1[kx][i];  adjoint: Y2[kx][i] = sum_o conj(R[..][i][o]) Y1[kx][o]
//   out[b][x][ky][c] = sum_kx Y2[kx][c] e^{+2 pi i f(kx) x / n}
template <bool ADJ>
__global__ void k_fno_specx(const float2 *in, const float2 *R, Dims d, float2 *mid, float2 *out) {
    extern __shared__ float smem[];
    const int n = d.n, C = d.C, M = d.M, MX = d.MX;
    float2 *X = reinterpret_cast<float2 *>(smem);  // n * C
    float2 *Y1 = X + n * C;                        // MX * C
    float2 *Y2 = Y1 + MX * C;                      // MX * C
    float *cs = reinterpret_cast<float *>(Y2 + MX * C), *sn = cs + n;
    const int64_t b = blockIdx.x / M;
    const int ky = blockIdx.x - (int)(b * M);
    for (int i = threadIdx.x; i < n * C; i += blockDim.x) {
        const int x = i / C, c = i - x * C;
        X[i] = in[((b * n + x) * M + ky) * (int64_t)C + c];
    }
    twiddle_table(cs, sn, n);
    __syncthreads();
    for (int o = threadIdx.x; o < MX * C; o += blockDim.x) {
        const int kx = o / C, c = o - kx * C;
        const int fr = kx_freq(kx, M, n);
        float re = 0.f, im = 0.f;
        for (int x = 0; x < n; ++x) {
            const int k = (fr * x) & (n - 1);
            const float2 v = X[x * C + c];
            // v * (cos - i sin)
            re = fmaf(v.x, cs[k], fmaf(v.y, sn[k], re));
            im = fmaf(v.y, cs[k], fmaf(-v.x, sn[k], im));
        }
        Y1[o] = make_float2(re, im);
        mid[((b * MX + kx) * M + ky) * (int64_t)C + c] = make_float2(re, im);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < MX * C; o += blockDim.x) {
        const int kx = o / C, c = o - kx * C;
        const float2 *Rm = R + ((int64_t)(kx * M + ky) * C) * C;  // [i][o]
        float re = 0.f, im = 0.f;
        for (int j = 0; j < C; ++j) {
            const float2 y = Y1[kx * C + j];
            if (!ADJ) {
                const float2 r = Rm[j * C + c];  // R[i=j][o=c]
                re += r.x * y.x - r.y * y.y;
                im += r.x * y.y + r.y * y.x;
            } else {
                const float2 r = Rm[c * C + j];  // conj(R[i=c][o=j])
                re += r.x * y.x + r.y * y.y;
                im += r.x * y.y - r.y * y.x;
            }
        }
        Y2[o] = make_float2(re, im);
    }
    __syncthreads();
    for (int o = threadIdx.x; o < n * C; o += blockDim.x) {
        const int x = o / C, c = o - x * C;
        float re = 0.f, im = 0.f;
        for (int kx = 0; kx < MX; ++kx) {
            const int k = (kx_freq(kx, M, n) * x) & (n - 1);
            const float2 v = Y2[kx * C + c];
            // v * (cos + i sin)
            re = fmaf(v.x, cs[k], fmaf(-v.y, sn[k], re));
            im = fmaf(v.y, cs[k], fmaf(v.x, sn[k], im));
        }
        out[((b * n + x) * M + ky) * (int64_t)C + c] = make_float2(re, im);
    }
}

// ------------------------- inverse axis-1 stage + pointwise part + activation
// One block per (b, x) row: a = n^-2 sum_ky c_ky Re(S[ky] e^{+2 pi i ky y/n}) + Ww v + bw.
template <typename T>
__global__ void k_fno_layer_out(const float2 *S, const T *v, const float *Ww, const float *bw, Dims d, int act,
                                T *a_out, T *v_out) {
    extern __shared__ float smem[];
    const int n = d.n, C = d.C, M = d.M;
    float2 *Ss = reinterpret_cast<float2 *>(smem);       // M * C
    float *row = reinterpret_cast<float *>(Ss + M * C);  // n * C
    float *W = row + n * C;                              // C * C, stored W[c][o]
    float *cs = W + C * C, *sn = cs + n;
    const int64_t bx = blockIdx.x;
    for (int i = threadIdx.x; i < M * C; i += blockDim.x) Ss[i] = S[bx * (int64_t)M * C + i];
    for (int i = threadIdx.x; i < n * C; i += blockDim.x) row[i] = ldv(&v[bx * (int64_t)n * C + i]);
    for (int i = threadIdx.x; i < C * C; i += blockDim.x) W[(i % C) * C + i / C] = Ww[i];
    twiddle_table(cs, sn, n);
    __syncthreads();
    const float inv = 1.f / ((float)n * (float)n);
    for (int o = threadIdx.x; o < n * C; o += blockDim.x) {
        const int y = o / C, co = o - y * C;
        float u = Ss[co].x;
        for (int ky = 1; ky < M; ++ky) {
            const int k = (ky * y) & (n - 1);
            const float2 s = Ss[ky * C + co];
            u = fmaf(2.f * s.x, cs[k], fmaf(-2.f * s.y, sn[k], u));
        }
        float a = fmaf(u, inv, bw[co]);
        for (int c = 0; c < C; ++c) a = fmaf(W[c * C + co], row[y * C + c], a);
        const int64_t idx = bx * (int64_t)n * C + o;
        if (act) {
            stv(&a_out[idx], a);
            stv(&v_out[idx], gelu(a));
        } else {
            stv(&v_out[idx], a);
        }
    }
}

// ------------------------------------------- tensor-core forms (BF16 path)
// With BF16 activations, width C = 32, M <= 16 modes and H a multiple of 8, the
// two dense per-point contractions of the forward pass run on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation): the layer output
// (pointwise 32 x 32 map plus the inverse axis-1 DFT stage, both one product
// per row) and the projection's 32 -> H map.  The FP32 activation path (the
// gradient checks) keeps the SIMT kernels above.
constexpr int TC_C = 32;       // width the tensor-core kernels are written for
constexpr int TC_LD = 20;      // words per 16-word row of a shared B operand (conflict-free fragment loads)

__device__ __forceinline__ uint32_t bf2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// D (16 x 8, FP32) += A (16 x 16, BF16, row) . B (16 x 8, BF16, col)
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

bool tc_layer_ok(const Dims &d) { return d.C == TC_C && d.M <= 16 && d.n % 16 == 0; }
// the axis-0 stages: 2 MX = 4 M retained axis-0 modes in tiles of 16 (M = 8 or 16)
bool tc_specx_ok(const Dims &d) { return tc_layer_ok(d) && d.MX % 16 == 0; }
bool tc_proj_ok(const Dims &d) { return d.C == TC_C && d.H % 16 == 0 && d.H <= 128; }

// A-operand fragments of the DFT products (the same for every row and mode),
// built once per network by k_fno_frags from the same cos/sin table the
// SIMT kernels use; entry (tile, k step, lane) holds the lane's four BF16 pairs
// of mma.m16n8k16's A operand.
struct TcFrags {
    const uint4 *dfty;  // [2][n/16][32]: T[k][y] (k < 16 cos, else -sin) for the axis-1 stage
    const uint4 *lay;   // [n/16][2][32]: T[y][k] for the layer output / layer-input backward
    const uint4 *sx1;   // [MX/16][2n/16][2][32]: axis-0 forward rows (re, im)
    const uint4 *sx2;   // [n/16][2 MX/16][2][32]: axis-0 inverse rows (re, im)
};

__host__ __device__ size_t frag_count(const Dims &d, int which) {
    const int n = d.n, MX = d.MX;
    switch (which) {
    case 0: return 2 * (size_t)(n / 16) * 32;
    case 1: return (size_t)(n / 16) * 2 * 32;
    case 2: return (size_t)(MX / 16) * (2 * n / 16) * 2 * 32;
    default: return (size_t)(n / 16) * (2 * MX / 16) * 2 * 32;
    }
}

__global__ void __launch_bounds__(FT) k_fno_frags(uint4 *dfty, uint4 *lay, uint4 *sx1, uint4 *sx2, Dims d) {
    __shared__ float cs[256], sn[256];
    const int n = d.n, M = d.M, MX = d.MX;
    twiddle_table(cs, sn, n);
    __syncthreads();
    auto twk = [&](int k, int y) {  // k < 16: cos, else -sin of 2 pi (k & 15) y / n
        const int idx = ((k & 15) * y) & (n - 1);
        return k < 16 ? cs[idx] : -sn[idx];
    };
    auto cth = [&](int f, int x) { return cs[(f * x) & (n - 1)]; };
    auto sth = [&](int f, int x) { return sn[(f * x) & (n - 1)]; };
    const size_t c0 = frag_count(d, 0), c1 = frag_count(d, 1);
    const size_t c2 = sx1 ? frag_count(d, 2) : 0, c3 = sx2 ? frag_count(d, 3) : 0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < c0 + c1 + c2 + c3;
         e += (size_t)gridDim.x * blockDim.x) {
        const int lane = (int)(e % 32), r = lane / 4, q = 2 * (lane % 4);
        if (e < c0) {
            const int t = (int)(e / 32), KS = n / 16, mt = t / KS, ks = t % KS;
            const int y = 16 * ks + q, ka = 16 * mt + r, kb = ka + 8;
            dfty[e] = make_uint4(bf2(twk(ka, y), twk(ka, y + 1)), bf2(twk(kb, y), twk(kb, y + 1)),
                                 bf2(twk(ka, y + 8), twk(ka, y + 9)), bf2(twk(kb, y + 8), twk(kb, y + 9)));
        } else if (e < c0 + c1) {
            const size_t e1 = e - c0;
            const int t = (int)(e1 / 32), yt = t / 2, ks = t % 2;
            const int k = 16 * ks + q, ya = 16 * yt + r, yb = ya + 8;
            lay[e1] = make_uint4(bf2(twk(k, ya), twk(k + 1, ya)), bf2(twk(k, yb), twk(k + 1, yb)),
                                 bf2(twk(k + 8, ya), twk(k + 9, ya)), bf2(twk(k + 8, yb), twk(k + 9, yb)));
        } else if (e < c0 + c1 + c2) {
            const size_t e2 = e - c0 - c1;
            const int t = (int)(e2 / 32), kind = t % 2, t2 = t / 2, S1 = 2 * n / 16, st = t2 % S1, kt = t2 / S1;
            const int k0 = 16 * st;
            const bool imx = k0 >= n;
            const int x = (imx ? k0 - n : k0) + q;
            const int fa = kx_freq(16 * kt + r, M, n), fb = kx_freq(16 * kt + r + 8, M, n);
            // real rows: [cos | sin] over (Re X | Im X); imaginary rows: [-sin | cos]
            auto v = [&](int f, int xx) {
                return kind == 0 ? (imx ? sth(f, xx) : cth(f, xx)) : (imx ? cth(f, xx) : -sth(f, xx));
            };
            sx1[e2] = make_uint4(bf2(v(fa, x), v(fa, x + 1)), bf2(v(fb, x), v(fb, x + 1)),
                                 bf2(v(fa, x + 8), v(fa, x + 9)), bf2(v(fb, x + 8), v(fb, x + 9)));
        } else {
            const size_t e3 = e - c0 - c1 - c2;
            const int t = (int)(e3 / 32), kind = t % 2, t2 = t / 2, S2 = 2 * MX / 16, st = t2 % S2, xt = t2 / S2;
            const int k0 = 16 * st;
            const bool imk = k0 >= MX;
            const int kx = (imk ? k0 - MX : k0) + q;
            const int xa = 16 * xt + r, xb = xa + 8;
            // real rows: [cos | -sin] over (Re Y2 | Im Y2); imaginary rows: [sin | cos]
            auto v = [&](int xx, int kk) {
                const int f = kx_freq(kk, M, n);
                return kind == 0 ? (imk ? -sth(f, xx) : cth(f, xx)) : (imk ? cth(f, xx) : sth(f, xx));
            };
            sx2[e3] = make_uint4(bf2(v(xa, kx), v(xa, kx + 1)), bf2(v(xb, kx), v(xb, kx + 1)),
                                 bf2(v(xa, kx + 8), v(xa, kx + 9)), bf2(v(xb, kx + 8), v(xb, kx + 9)));
        }
    }
}

// Layer output of row bx = (b, x) on the tensor cores:
//   a[y][o] = sum_c v[y][c] Ww[o][c] + sum_k T[y][k] U[k][o] + bw[o],
//   T[y][k] = cos(2 pi k y / n) (k < 16), -sin(2 pi (k - 16) y / n) (k >= 16),
//   U[k][o] = c_k Re S[k][o] / n^2, U[16 + k][o] = c_k Im S[k][o] / n^2 (zero for k >= M),
// which is n^-2 sum_ky c_ky Re(S[ky] e^{+2 pi i ky y / n}) as in k_fno_layer_out.
// Each warp takes 16 rows y at a time: K = 32 (channels) + 32 (spectral).
__global__ void __launch_bounds__(FT) k_fno_layer_out_tc(const float2 *S, const __nv_bfloat16 *v, const float *Ww,
                                                         const float *bw, Dims d, int act, __nv_bfloat16 *a_out,
                                                         __nv_bfloat16 *v_out, const uint4 *lay) {
    __shared__ uint32_t Wb[TC_C * TC_LD], Ub[TC_C * TC_LD];  // [o][k pair]
    __shared__ float bs[TC_C];
    const int n = d.n, M = d.M;
    const int64_t bx = blockIdx.x;
    const float inv = 1.f / ((float)n * (float)n);
    for (int i = threadIdx.x; i < TC_C * 16; i += blockDim.x) {
        const int o = i / 16, j = i % 16;
        Wb[o * TC_LD + j] = bf2(Ww[o * TC_C + 2 * j], Ww[o * TC_C + 2 * j + 1]);
        // spectral rows 2j, 2j + 1 of U (k < 16: real parts, k >= 16: imaginary parts)
        float u[2];
        for (int e = 0; e < 2; ++e) {
            const int k = 2 * j + e, ky = k & 15;
            float val = 0.f;
            if (ky < M) {
                const float2 sv = S[(bx * M + ky) * (int64_t)TC_C + o];
                val = (ky == 0 ? 1.f : 2.f) * inv * (k < 16 ? sv.x : sv.y);
            }
            u[e] = val;
        }
        Ub[o * TC_LD + j] = bf2(u[0], u[1]);
    }
    for (int i = threadIdx.x; i < TC_C; i += blockDim.x) bs[i] = bw[i];
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int r = lane / 4, q = 2 * (lane % 4);
    const uint32_t *vrow = reinterpret_cast<const uint32_t *>(v + bx * (int64_t)n * TC_C);
    for (int y0 = 16 * warp; y0 < n; y0 += 16 * (FT / 32)) {
        float acc[4][4] = {};
        // channels: A = v rows y0.., K = 32 in two steps
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int k = 16 * ks + q;
            const uint32_t a0 = vrow[((y0 + r) * TC_C + k) / 2], a1 = vrow[((y0 + r + 8) * TC_C + k) / 2];
            const uint32_t a2 = vrow[((y0 + r) * TC_C + k + 8) / 2], a3 = vrow[((y0 + r + 8) * TC_C + k + 8) / 2];
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int o = 8 * nt + r;
                mma_bf16(acc[nt], a0, a1, a2, a3, Wb[o * TC_LD + k / 2], Wb[o * TC_LD + k / 2 + 4]);
            }
        }
        // spectral: A = T rows y0.., K = 32 (cos | -sin) in two steps
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int k = 16 * ks + q;
            const uint4 A = __ldg(&lay[((y0 / 16) * 2 + ks) * 32 + lane]);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int o = 8 * nt + r;
                mma_bf16(acc[nt], A.x, A.y, A.z, A.w, Ub[o * TC_LD + k / 2], Ub[o * TC_LD + k / 2 + 4]);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int o = 8 * nt + q;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int y = y0 + r + 8 * h;
                const float x0 = acc[nt][2 * h] + bs[o], x1 = acc[nt][2 * h + 1] + bs[o + 1];
                const int64_t idx = (bx * (int64_t)n + y) * TC_C + o;
                if (act) {
                    *reinterpret_cast<uint32_t *>(&a_out[idx]) = bf2(x0, x1);
                    *reinterpret_cast<uint32_t *>(&v_out[idx]) = bf2(gelu(x0), gelu(x1));
                } else {
                    *reinterpret_cast<uint32_t *>(&v_out[idx]) = bf2(x0, x1);
                }
            }
        }
    }
}

// Projection on the tensor cores: per 16 points, h = W1 v + b1 (16 x H, K = 32)
// in registers, then z = sum_k w2[k] gelu(h[k]) + b2 reduced over each row's
// four lanes.
__global__ void __launch_bounds__(FT) k_fno_proj_tc(const __nv_bfloat16 *v, const float *W1, const float *b1,
                                                    const float *W2, const float *b2, Dims d, float *z) {
    __shared__ uint32_t Wb[128 * TC_LD];  // [h][c pair]
    __shared__ float bb[128], ww[128];
    const int H = d.H;
    for (int i = threadIdx.x; i < H * 16; i += blockDim.x) {
        const int h = i / 16, j = i % 16;
        Wb[h * TC_LD + j] = bf2(W1[h * TC_C + 2 * j], W1[h * TC_C + 2 * j + 1]);
    }
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        bb[i] = b1[i];
        ww[i] = W2[i];
    }
    __syncthreads();
    const float bias2 = b2[0];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int r = lane / 4, q = 2 * (lane % 4);
    const int64_t P = d.P();
    const uint32_t *vv = reinterpret_cast<const uint32_t *>(v);
    const int64_t wstride = (int64_t)gridDim.x * (FT / 32) * 16;
    for (int64_t p0 = ((int64_t)blockIdx.x * (FT / 32) + warp) * 16; p0 < P; p0 += wstride) {
        uint32_t a[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int k = 16 * ks + q;
            a[ks][0] = vv[((p0 + r) * TC_C + k) / 2];
            a[ks][1] = vv[((p0 + r + 8) * TC_C + k) / 2];
            a[ks][2] = vv[((p0 + r) * TC_C + k + 8) / 2];
            a[ks][3] = vv[((p0 + r + 8) * TC_C + k + 8) / 2];
        }
        float t0 = 0.f, t1 = 0.f;  // rows r and r + 8
        for (int nt = 0; nt < H / 8; ++nt) {
            float acc[4] = {};
            const int h = 8 * nt + r;
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
                const int k = 16 * ks + q;
                mma_bf16(acc, a[ks][0], a[ks][1], a[ks][2], a[ks][3], Wb[h * TC_LD + k / 2], Wb[h * TC_LD + k / 2 + 4]);
            }
            const int hc = 8 * nt + q;
            t0 = fmaf(ww[hc], gelu(acc[0] + bb[hc]), fmaf(ww[hc + 1], gelu(acc[1] + bb[hc + 1]), t0));
            t1 = fmaf(ww[hc], gelu(acc[2] + bb[hc]), fmaf(ww[hc + 1], gelu(acc[3] + bb[hc + 1]), t1));
        }
        t0 += __shfl_xor_sync(0xffffffffu, t0, 1);
        t0 += __shfl_xor_sync(0xffffffffu, t0, 2);
        t1 += __shfl_xor_sync(0xffffffffu, t1, 1);
        t1 += __shfl_xor_sync(0xffffffffu, t1, 2);
        if ((lane & 3) == 0) {
            z[p0 + r] = t0 + bias2;
            z[p0 + r + 8] = t1 + bias2;
        }
    }
}

// Axis-1 truncated DFT stage of row bx on the tensor cores (BF16 path):
//   D[k][c] = sum_y T[k][y] V[y][c],  T[k][y] = cos(2 pi k y / n) (k < 16), -sin(2 pi (k - 16) y / n) (k >= 16),
// so out[bx][ky][c] = s(ky) (D[ky][c], D[16 + ky][c]) as k_fno_dfty.  V (bf16 activations or FP32
// gradients) is staged transposed in shared memory as BF16 pairs; each warp owns one 16 x 8 tile of D.
template <typename T>
__global__ void __launch_bounds__(FT) k_fno_dfty_tc(const T *in, Dims d, float s0, float s1, float2 *out,
                                                    const uint4 *fr) {
    __shared__ uint32_t Vt[TC_C * (128 + 4)];  // [c][y pair], n <= 256
    __shared__ float Ds[32 * 33];
    const int n = d.n, M = d.M, LDV = n / 2 + 4;
    const int64_t bx = blockIdx.x;
    const T *src = in + bx * (int64_t)n * TC_C;
    for (int i = threadIdx.x; i < TC_C * (n / 2); i += blockDim.x) {
        const int c = i % TC_C, j = i / TC_C;
        Vt[c * LDV + j] = bf2(ldv(&src[(2 * j) * TC_C + c]), ldv(&src[(2 * j + 1) * TC_C + c]));
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int r = lane / 4, q = 2 * (lane % 4);
    const int mt = warp / 4, nt = warp % 4;  // 2 x 4 tiles of 16 x 8
    float acc[4] = {};
    const int ka = 16 * mt + r, kb = ka + 8, c = 8 * nt + r;
    const uint4 *frm = fr + (size_t)mt * (n / 16) * 32 + lane;
    for (int y0 = 0; y0 < n; y0 += 16) {
        const int y = y0 + q;
        const uint4 A = __ldg(&frm[(y0 / 16) * 32]);
        mma_bf16(acc, A.x, A.y, A.z, A.w, Vt[c * LDV + y / 2], Vt[c * LDV + y / 2 + 4]);
    }
    const int co = 8 * nt + q;
    Ds[ka * 33 + co] = acc[0];
    Ds[ka * 33 + co + 1] = acc[1];
    Ds[kb * 33 + co] = acc[2];
    Ds[kb * 33 + co + 1] = acc[3];
    __syncthreads();
    for (int o = threadIdx.x; o < M * TC_C; o += blockDim.x) {
        const int ky = o / TC_C, cc = o % TC_C;
        const float sc = ky == 0 ? s0 : s1;
        out[bx * (int64_t)M * TC_C + o] = make_float2(Ds[ky * 33 + cc] * sc, Ds[(16 + ky) * 33 + cc] * sc);
    }
}

// Backward of the layer input on the tensor cores (BF16 path), as k_fno_layer_in_bwd:
//   dv[y][c] = sum_o Ww[o][c] da[y][o] + sum_k T[y][k] U[k][c],  U = [Re dT ; Im dT] (zero past M).
__global__ void __launch_bounds__(FT) k_fno_layer_in_bwd_tc(const float2 *dT, const float *da, const float *Ww, Dims d,
                                                            float *dv, const uint4 *lay) {
    __shared__ uint32_t Wt[TC_C * TC_LD], Ub[TC_C * TC_LD];  // [c][k pair]
    const int n = d.n, M = d.M;
    const int64_t bx = blockIdx.x;
    for (int i = threadIdx.x; i < TC_C * 16; i += blockDim.x) {
        const int c = i / 16, j = i % 16;
        Wt[c * TC_LD + j] = bf2(Ww[(2 * j) * TC_C + c], Ww[(2 * j + 1) * TC_C + c]);
        float u[2];
        for (int e = 0; e < 2; ++e) {
            const int k = 2 * j + e, ky = k & 15;
            float val = 0.f;
            if (ky < M) {
                const float2 t = dT[(bx * M + ky) * (int64_t)TC_C + c];
                val = k < 16 ? t.x : t.y;
            }
            u[e] = val;
        }
        Ub[c * TC_LD + j] = bf2(u[0], u[1]);
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int r = lane / 4, q = 2 * (lane % 4);
    const float *drow = da + bx * (int64_t)n * TC_C;
    for (int y0 = 16 * warp; y0 < n; y0 += 16 * (FT / 32)) {
        float acc[4][4] = {};
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int k = 16 * ks + q;
            auto pr = [&](int y, int kk) {
                const float2 t = *reinterpret_cast<const float2 *>(&drow[y * TC_C + kk]);
                return bf2(t.x, t.y);
            };
            const uint32_t a0 = pr(y0 + r, k), a1 = pr(y0 + r + 8, k), a2 = pr(y0 + r, k + 8), a3 = pr(y0 + r + 8, k + 8);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = 8 * nt + r;
                mma_bf16(acc[nt], a0, a1, a2, a3, Wt[c * TC_LD + k / 2], Wt[c * TC_LD + k / 2 + 4]);
            }
        }
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int k = 16 * ks + q;
            const uint4 A = __ldg(&lay[((y0 / 16) * 2 + ks) * 32 + lane]);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = 8 * nt + r;
                mma_bf16(acc[nt], A.x, A.y, A.z, A.w, Ub[c * TC_LD + k / 2], Ub[c * TC_LD + k / 2 + 4]);
            }
        }
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int c = 8 * nt + q;
            float *out = dv + bx * (int64_t)n * TC_C;
            *reinterpret_cast<float2 *>(&out[(y0 + r) * TC_C + c]) = make_float2(acc[nt][0], acc[nt][1]);
            *reinterpret_cast<float2 *>(&out[(y0 + r + 8) * TC_C + c]) = make_float2(acc[nt][2], acc[nt][3]);
        }
    }
}

// Projection backward on the tensor cores (BF16 path), as k_fno_proj_bwd: per 16
// points, h = W1 v + b1 (MMA), q = dz w2 gelu'(h) (stored to dh for the W1
// gradient), dv = W1^T q (a second MMA whose A operand is q in registers), and
// block partial sums of dz gelu(h) (W2 gradient) and dz (b2 gradient).
__global__ void __launch_bounds__(FT) k_fno_proj_bwd_tc(const __nv_bfloat16 *v, const float *dz, const float *W1,
                                                        const float *b1, const float *W2, Dims d, float *dh, float *dv,
                                                        double *part) {
    constexpr int LDT = 64 + 4;                   // words per row of W1^T pairs (H <= 128)
    __shared__ uint32_t Wb[128 * TC_LD];          // [h][c pair]
    __shared__ uint32_t Wt[TC_C * LDT];           // [c][h pair]
    __shared__ float bb[128], ww[128], acc_s[129];
    const int H = d.H;
    for (int i = threadIdx.x; i < H * 16; i += blockDim.x) {
        const int h = i / 16, j = i % 16;
        Wb[h * TC_LD + j] = bf2(W1[h * TC_C + 2 * j], W1[h * TC_C + 2 * j + 1]);
    }
    for (int i = threadIdx.x; i < TC_C * (H / 2); i += blockDim.x) {
        const int c = i % TC_C, j = i / TC_C;
        Wt[c * LDT + j] = bf2(W1[(2 * j) * TC_C + c], W1[(2 * j + 1) * TC_C + c]);
    }
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        bb[i] = b1[i];
        ww[i] = W2[i];
    }
    for (int i = threadIdx.x; i <= H; i += blockDim.x) acc_s[i] = 0.f;
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int r = lane / 4, q = 2 * (lane % 4);
    const int64_t P = d.P();
    const uint32_t *vv = reinterpret_cast<const uint32_t *>(v);
    const int64_t wstride = (int64_t)gridDim.x * (FT / 32) * 16;
    for (int64_t p0 = ((int64_t)blockIdx.x * (FT / 32) + warp) * 16; p0 < P; p0 += wstride) {
        uint32_t a[2][4];
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
            const int k = 16 * ks + q;
            a[ks][0] = vv[((p0 + r) * TC_C + k) / 2];
            a[ks][1] = vv[((p0 + r + 8) * TC_C + k) / 2];
            a[ks][2] = vv[((p0 + r) * TC_C + k + 8) / 2];
            a[ks][3] = vv[((p0 + r + 8) * TC_C + k + 8) / 2];
        }
        const float e0 = dz[p0 + r], e1 = dz[p0 + r + 8];
        float dva[4][4] = {};
        for (int nt2 = 0; nt2 < H / 16; ++nt2) {
            uint32_t qa[4];
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                float acc[4] = {};
                const int hr = 16 * nt2 + 8 * half + r;
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const int k = 16 * ks + q;
                    mma_bf16(acc, a[ks][0], a[ks][1], a[ks][2], a[ks][3], Wb[hr * TC_LD + k / 2],
                             Wb[hr * TC_LD + k / 2 + 4]);
                }
                const int hc = 16 * nt2 + 8 * half + q;
                const float h0 = acc[0] + bb[hc], h1 = acc[1] + bb[hc + 1];
                const float h2 = acc[2] + bb[hc], h3 = acc[3] + bb[hc + 1];
                // W2 gradient: sum over the warp's 16 points of dz gelu(h)
                float g0 = fmaf(e0, gelu(h0), e1 * gelu(h2)), g1 = fmaf(e0, gelu(h1), e1 * gelu(h3));
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {
                    g0 += __shfl_xor_sync(0xffffffffu, g0, o);
                    g1 += __shfl_xor_sync(0xffffffffu, g1, o);
                }
                if (lane < 4) {
                    atomicAdd(&acc_s[hc], g0);
                    atomicAdd(&acc_s[hc + 1], g1);
                }
                const float q0 = e0 * ww[hc] * gelu_d(h0), q1 = e0 * ww[hc + 1] * gelu_d(h1);
                const float q2 = e1 * ww[hc] * gelu_d(h2), q3 = e1 * ww[hc + 1] * gelu_d(h3);
                *reinterpret_cast<float2 *>(&dh[(p0 + r) * H + hc]) = make_float2(q0, q1);
                *reinterpret_cast<float2 *>(&dh[(p0 + r + 8) * H + hc]) = make_float2(q2, q3);
                qa[2 * half] = bf2(q0, q1);      // rows r: k = hc, hc + 1 of this 16-wide step
                qa[2 * half + 1] = bf2(q2, q3);  // rows r + 8
            }
            // dv[p][c] += sum_h q[p][h] W1[h][c] over this step's 16 h
            const int kh = 16 * nt2 + q;
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int c = 8 * nt + r;
                mma_bf16(dva[nt], qa[0], qa[1], qa[2], qa[3], Wt[c * LDT + kh / 2], Wt[c * LDT + kh / 2 + 4]);
            }
        }
        float t = e0 + e1;
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) atomicAdd(&acc_s[H], t);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int c = 8 * nt + q;
            *reinterpret_cast<float2 *>(&dv[(p0 + r) * TC_C + c]) = make_float2(dva[nt][0], dva[nt][1]);
            *reinterpret_cast<float2 *>(&dv[(p0 + r + 8) * TC_C + c]) = make_float2(dva[nt][2], dva[nt][3]);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= H; i += blockDim.x) part[(int64_t)blockIdx.x * (H + 1) + i] = acc_s[i];
}

// Axis-0 stages with the mode mixing on the tensor cores (BF16 path), as
// k_fno_specx: one block per (b, ky).  With theta = 2 pi f(kx) x / n,
//   Y1[kx][c] = sum_x X[x][c] e^{-i theta}:  [Re; Im] Y1 = [[cos, sin], [-sin, cos]] . [Re X; Im X]
//   (a 2 MX x 2n by 2n x C product, K over (x, re|im)),
//   the per-mode mixing in FP32 as k_fno_specx,
//   out[x][c] = sum_kx Y2[kx][c] e^{+i theta}:  [Re; Im] out = [[cos, -sin], [sin, cos]] . [Re Y2; Im Y2]
//   (2n x 2 MX by 2 MX x C, K over (kx, re|im)).
// X and Y2 enter the products as BF16, transposed into shared memory; each
// warp computes the real and the imaginary tile of the same rows, so it writes
// complex outputs directly.
template <bool ADJ>
__global__ void __launch_bounds__(FT) k_fno_specx_tc(const float2 *in, const float2 *R, Dims d, float2 *mid,
                                                     float2 *out, const uint4 *sx1, const uint4 *sx2) {
    extern __shared__ __align__(16) uint32_t sm32[];
    const int n = d.n, M = d.M, MX = d.MX;
    const int LDX = n + 4;                         // words per row of Xt: n/2 (re) pairs, n/2 (im) pairs, padding
    uint32_t *Xt = sm32;                           // [c][k pair], k over (re x | im x), 2n values
    float2 *Y1 = reinterpret_cast<float2 *>(Xt + TC_C * LDX);  // [kx][c]
    float2 *Y2 = Y1 + MX * TC_C;                   // [kx][c]
    uint32_t *Yt = reinterpret_cast<uint32_t *>(Y2 + MX * TC_C);  // [c][k pair], k over (re kx | im kx), 2 MX values
    constexpr int LDY = 32 + 4;
    const int64_t b = blockIdx.x / M;
    const int ky = blockIdx.x - (int)(b * M);
    for (int i = threadIdx.x; i < TC_C * (n / 2); i += blockDim.x) {
        const int c = i % TC_C, j = i / TC_C;  // x pair (2j, 2j + 1)
        const float2 v0 = in[((b * n + 2 * j) * M + ky) * (int64_t)TC_C + c];
        const float2 v1 = in[((b * n + 2 * j + 1) * M + ky) * (int64_t)TC_C + c];
        Xt[c * LDX + j] = bf2(v0.x, v1.x);
        Xt[c * LDX + n / 2 + j] = bf2(v0.y, v1.y);
    }
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int r = lane / 4, q = 2 * (lane % 4);
    const int S1 = 2 * n / 16, S2 = 2 * MX / 16;
    // ---- Y1: warp -> (kx tile kt, column tile nt); real and imaginary rows together
    for (int t = warp; t < (MX / 16) * 4; t += FT / 32) {
        const int kt = t / 4, nt = t % 4;
        const int ka = 16 * kt + r, kb = ka + 8;
        float re[4] = {}, im[4] = {};
        const int c = 8 * nt + r;
        for (int k0 = 0; k0 < 2 * n; k0 += 16) {
            // real rows: cos . Re X + sin . Im X;  imaginary rows: -sin . Re X + cos . Im X
            const uint4 *fa = &sx1[(((size_t)kt * S1 + k0 / 16) * 2) * 32 + lane];
            const uint4 A = __ldg(fa), B = __ldg(fa + 32);
            const uint32_t ar[4] = {A.x, A.y, A.z, A.w}, ai[4] = {B.x, B.y, B.z, B.w};
            const int kw = (k0 + q) / 2;
            const uint32_t b0 = Xt[c * LDX + kw], b1 = Xt[c * LDX + kw + 4];
            mma_bf16(re, ar[0], ar[1], ar[2], ar[3], b0, b1);
            mma_bf16(im, ai[0], ai[1], ai[2], ai[3], b0, b1);
        }
        const int co = 8 * nt + q;
        const float2 ya0 = make_float2(re[0], im[0]), ya1 = make_float2(re[1], im[1]);
        const float2 yb0 = make_float2(re[2], im[2]), yb1 = make_float2(re[3], im[3]);
        Y1[ka * TC_C + co] = ya0;
        Y1[ka * TC_C + co + 1] = ya1;
        Y1[kb * TC_C + co] = yb0;
        Y1[kb * TC_C + co + 1] = yb1;
        mid[((b * MX + ka) * M + ky) * (int64_t)TC_C + co] = ya0;
        mid[((b * MX + ka) * M + ky) * (int64_t)TC_C + co + 1] = ya1;
        mid[((b * MX + kb) * M + ky) * (int64_t)TC_C + co] = yb0;
        mid[((b * MX + kb) * M + ky) * (int64_t)TC_C + co + 1] = yb1;
    }
    __syncthreads();
    // ---- mode mixing (FP32), then Y2 as BF16 pairs over (re kx | im kx)
    for (int o = threadIdx.x; o < MX * TC_C; o += blockDim.x) {
        const int kx = o / TC_C, c = o - kx * TC_C;
        const float2 *Rm = R + ((int64_t)(kx * M + ky) * TC_C) * TC_C;  // [i][o]
        float re = 0.f, im = 0.f;
        for (int j = 0; j < TC_C; ++j) {
            const float2 y = Y1[kx * TC_C + j];
            if (!ADJ) {
                const float2 rr = Rm[j * TC_C + c];
                re += rr.x * y.x - rr.y * y.y;
                im += rr.x * y.y + rr.y * y.x;
            } else {
                const float2 rr = Rm[c * TC_C + j];
                re += rr.x * y.x + rr.y * y.y;
                im += rr.x * y.y - rr.y * y.x;
            }
        }
        Y2[o] = make_float2(re, im);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < TC_C * (MX / 2); i += blockDim.x) {
        const int c = i % TC_C, j = i / TC_C;  // kx pair (2j, 2j + 1)
        const float2 v0 = Y2[(2 * j) * TC_C + c], v1 = Y2[(2 * j + 1) * TC_C + c];
        Yt[c * LDY + j] = bf2(v0.x, v1.x);
        Yt[c * LDY + MX / 2 + j] = bf2(v0.y, v1.y);
    }
    __syncthreads();
    // ---- out: warp -> (x tile, column tile); real and imaginary rows together
    for (int t = warp; t < (n / 16) * 4; t += FT / 32) {
        const int xt = t / 4, nt = t % 4;
        const int xa = 16 * xt + r, xb = xa + 8;
        float re[4] = {}, im[4] = {};
        const int c = 8 * nt + r;
        for (int k0 = 0; k0 < 2 * MX; k0 += 16) {
            // real rows: cos . Re Y2 - sin . Im Y2;  imaginary rows: sin . Re Y2 + cos . Im Y2
            const uint4 *fa = &sx2[(((size_t)xt * S2 + k0 / 16) * 2) * 32 + lane];
            const uint4 A = __ldg(fa), B = __ldg(fa + 32);
            const uint32_t ar[4] = {A.x, A.y, A.z, A.w}, ai[4] = {B.x, B.y, B.z, B.w};
            const int kw = (k0 + q) / 2;
            const uint32_t b0 = Yt[c * LDY + kw], b1 = Yt[c * LDY + kw + 4];
            mma_bf16(re, ar[0], ar[1], ar[2], ar[3], b0, b1);
            mma_bf16(im, ai[0], ai[1], ai[2], ai[3], b0, b1);
        }
        const int co = 8 * nt + q;
        out[((b * n + xa) * M + ky) * (int64_t)TC_C + co] = make_float2(re[0], im[0]);
        out[((b * n + xa) * M + ky) * (int64_t)TC_C + co + 1] = make_float2(re[1], im[1]);
        out[((b * n + xb) * M + ky) * (int64_t)TC_C + co] = make_float2(re[2], im[2]);
        out[((b * n + xb) * M + ky) * (int64_t)TC_C + co + 1] = make_float2(re[3], im[3]);
    }
}

size_t smem_specx_tc(const Dims &d) {
    return (size_t)TC_C * (d.n + 4) * 4 + 2 * (size_t)d.MX * TC_C * 8 + (size_t)TC_C * 36 * 4;
}

// Weight-gradient partials on the tensor cores (BF16 path, Cc = 32 columns of
// BF16 activations Y, O a multiple of 16 up to 128 rows of FP32 gradients X):
//   part[blk][o * 32 + c] = sum_p X[p][o] Y[p][c],  part[blk][O * 32 + o] = sum_p X[p][o]
// over the block's range of points, as k_fno_wgrad.  Each warp takes 16 points
// at a time: A = X^T (O x 16, X rounded to BF16), B = Y (16 x 32); the warps'
// FP32 tiles and the FP32 column sums of X meet in shared memory.
__global__ void __launch_bounds__(FT) k_fno_wgrad_tc(const float *X, const __nv_bfloat16 *Y, int64_t P, int O,
                                                     double *part) {
    __shared__ float Dsum[128 * TC_C], bsum[128];
    for (int i = threadIdx.x; i < O * TC_C; i += blockDim.x) Dsum[i] = 0.f;
    for (int i = threadIdx.x; i < O; i += blockDim.x) bsum[i] = 0.f;
    __syncthreads();
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const int r = lane / 4, q = 2 * (lane % 4);
    const int64_t per_blk = ((P + gridDim.x - 1) / gridDim.x + 15) / 16 * 16;
    const int64_t p0 = (int64_t)blockIdx.x * per_blk;
    const int64_t p1 = p0 + per_blk < P ? p0 + per_blk : P;
    const int MT = O / 16;
    float acc[8][4][4];
    float bacc[8][2];
#pragma unroll
    for (int mt = 0; mt < 8; ++mt) {
        bacc[mt][0] = bacc[mt][1] = 0.f;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
    }
    const unsigned short *Yh = reinterpret_cast<const unsigned short *>(Y);
    for (int64_t t = p0 + 16 * warp; t < p1; t += 16 * (FT / 32)) {
        // B fragments: rows (points) t + q, t + q + 1 (and + 8), column c = 8 nt + r
        uint32_t b[4][2];
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int c = 8 * nt + r;
            const uint32_t y0 = Yh[(t + q) * TC_C + c], y1 = Yh[(t + q + 1) * TC_C + c];
            const uint32_t y8 = Yh[(t + q + 8) * TC_C + c], y9 = Yh[(t + q + 9) * TC_C + c];
            b[nt][0] = y0 | (y1 << 16);
            b[nt][1] = y8 | (y9 << 16);
        }
#pragma unroll
        for (int mt = 0; mt < 8; ++mt) {
            if (mt >= MT) break;
            const int oa = 16 * mt + r, ob = oa + 8;
            const float xa0 = X[(t + q) * O + oa], xa1 = X[(t + q + 1) * O + oa];
            const float xb0 = X[(t + q) * O + ob], xb1 = X[(t + q + 1) * O + ob];
            const float xa8 = X[(t + q + 8) * O + oa], xa9 = X[(t + q + 9) * O + oa];
            const float xb8 = X[(t + q + 8) * O + ob], xb9 = X[(t + q + 9) * O + ob];
            bacc[mt][0] += (xa0 + xa1) + (xa8 + xa9);
            bacc[mt][1] += (xb0 + xb1) + (xb8 + xb9);
            const uint32_t a0 = bf2(xa0, xa1), a1 = bf2(xb0, xb1), a2 = bf2(xa8, xa9), a3 = bf2(xb8, xb9);
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a0, a1, a2, a3, b[nt][0], b[nt][1]);
        }
    }
#pragma unroll
    for (int mt = 0; mt < 8; ++mt) {
        if (mt >= MT) break;
        const int oa = 16 * mt + r, ob = oa + 8;
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
            const int c = 8 * nt + q;
            atomicAdd(&Dsum[oa * TC_C + c], acc[mt][nt][0]);
            atomicAdd(&Dsum[oa * TC_C + c + 1], acc[mt][nt][1]);
            atomicAdd(&Dsum[ob * TC_C + c], acc[mt][nt][2]);
            atomicAdd(&Dsum[ob * TC_C + c + 1], acc[mt][nt][3]);
        }
        float s0 = bacc[mt][0], s1 = bacc[mt][1];
        s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
        s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
        s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
        if ((lane & 3) == 0) {
            atomicAdd(&bsum[oa], s0);
            atomicAdd(&bsum[ob], s1);
        }
    }
    __syncthreads();
    double *dst = part + (int64_t)blockIdx.x * (O * TC_C + O);
    for (int i = threadIdx.x; i < O * TC_C; i += blockDim.x) dst[i] = Dsum[i];
    for (int i = threadIdx.x; i < O; i += blockDim.x) dst[O * TC_C + i] = bsum[i];
}

bool tc_wgrad_ok(const Dims &d, int O) { return d.C == TC_C && O % 16 == 0 && O <= 128; }

// ------------------------------------------------------------- projection
template <typename T>
__global__ void k_fno_proj(const T *v, const float *W1, const float *b1, const float *W2, const float *b2, Dims d,
                           float *z) {
    extern __shared__ float smem[];
    const int C = d.C, H = d.H;
    float *w1 = smem, *bb1 = w1 + H * C, *w2 = bb1 + H;
    for (int i = threadIdx.x; i < H * C; i += blockDim.x) w1[i] = W1[i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        bb1[i] = b1[i];
        w2[i] = W2[i];
    }
    __syncthreads();
    const int64_t P = d.P();
    float x[32];
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 32; ++c) x[c] = c < C ? ldv(&v[p * C + c]) : 0.f;
        float acc = b2[0];
        for (int k = 0; k < H; ++k) {
            float h = bb1[k];
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (c < C) h = fmaf(w1[k * C + c], x[c], h);
            acc = fmaf(w2[k], gelu(h), acc);
        }
        z[p] = acc;
    }
}

// block-wide reductions over FT threads
__device__ float block_max(float v, float *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = FT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    const float r = red[0];
    __syncthreads();
    return r;
}
__device__ double block_sum(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = FT / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

// softmax over the mesh per instance; lse = log sum exp z
__global__ void k_fno_softmax(const float *z, int64_t G, float *p, float *lse) {
    __shared__ float rf[FT];
    __shared__ double rd[FT];
    const int64_t b = blockIdx.x;
    float m = -INFINITY;
    for (int64_t i = threadIdx.x; i < G; i += blockDim.x) m = fmaxf(m, z[b * G + i]);
    m = block_max(m, rf);
    double s = 0;
    for (int64_t i = threadIdx.x; i < G; i += blockDim.x) s += (double)expf(z[b * G + i] - m);
    s = block_sum(s, rd);
    const float l = m + (float)log(s);
    for (int64_t i = threadIdx.x; i < G; i += blockDim.x) p[b * G + i] = expf(z[b * G + i] - l);
    if (threadIdx.x == 0) lse[b] = l;
}

// KL(p_true || p) per instance and dz = (p - p_true) / B
__global__ void k_fno_loss(const float *z, const float *lse, const float *p, const float *pt, int64_t G, float invB,
                           float *dz, double *loss) {
    __shared__ double rd[FT];
    const int64_t b = blockIdx.x;
    double s = 0;
    for (int64_t i = threadIdx.x; i < G; i += blockDim.x) {
        const int64_t k = b * G + i;
        const float q = pt[k];
        if (q > 0.f) s += (double)q * ((double)logf(q) - (double)(z[k] - lse[b]));
        dz[k] = (p[k] - q) * invB;
    }
    s = block_sum(s, rd);
    if (threadIdx.x == 0) loss[b] = s;
}

// projection backward, one thread per point: dh = dz Wp2 gelu'(h_pre), dv = Wp1^T dh;
// per-block partial sums of dz * gelu(h_pre) (grad of Wp2) and dz (grad of bp2)
template <typename T>
__global__ void k_fno_proj_bwd(const T *v, const float *dz, const float *W1, const float *b1, const float *W2, Dims d,
                               float *dh, float *dv, double *part) {
    extern __shared__ float smem[];
    const int C = d.C, H = d.H;
    float *w1 = smem, *bb1 = w1 + H * C, *w2 = bb1 + H;
    float *acc = w2 + H;  // H + 1 block sums
    for (int i = threadIdx.x; i < H * C; i += blockDim.x) w1[i] = W1[i];
    for (int i = threadIdx.x; i < H; i += blockDim.x) {
        bb1[i] = b1[i];
        w2[i] = W2[i];
    }
    for (int i = threadIdx.x; i <= H; i += blockDim.x) acc[i] = 0.f;
    __syncthreads();
    const int64_t P = d.P();
    float x[32], g[32];
    // the loop trip count is uniform over the block, so whole warps reduce together
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < P; base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = base + threadIdx.x;
        const bool ok = p < P;
#pragma unroll
        for (int c = 0; c < 32; ++c) {
            x[c] = ok && c < C ? ldv(&v[p * C + c]) : 0.f;
            g[c] = 0.f;
        }
        const float e = ok ? dz[p] : 0.f;
        for (int k = 0; k < H; ++k) {
            float h = bb1[k];
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (c < C) h = fmaf(w1[k * C + c], x[c], h);
            float t = e * gelu(h);
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if ((threadIdx.x & 31) == 0) atomicAdd(&acc[k], t);
            const float q = e * w2[k] * gelu_d(h);
            if (ok) dh[p * H + k] = q;
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (c < C) g[c] = fmaf(w1[k * C + c], q, g[c]);
        }
        float t = e;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&acc[H], t);
        if (ok)
#pragma unroll
            for (int c = 0; c < 32; ++c)
                if (c < C) dv[p * C + c] = g[c];
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= H; i += blockDim.x) part[(int64_t)blockIdx.x * (H + 1) + i] = acc[i];
}

// da = dv * gelu'(a) (or dv for the last layer)
template <typename T>
__global__ void k_fno_act_bwd(const float *dv, const T *a, int64_t count, int act, float *da) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        da[i] = act ? dv[i] * gelu_d(ldv(&a[i])) : dv[i];
}

// Weight-gradient partials: per block, over its range of points,
//   part[blk][o * Cc + c] = sum_p X[p][o] Y[p][c],  part[blk][O * Cc + o] = sum_p X[p][o].
// X: [P][O] FP32, Y: [P][Cc] (T).  O <= 128, Cc <= 32, O * Cc <= FT * 16.
template <typename T>
__global__ void k_fno_wgrad(const float *X, const T *Y, int64_t P, int O, int Cc, double *part) {
    __shared__ float xs[WG_PTS * 128], ys[WG_PTS * 32];
    constexpr int PER = 16;
    float acc[PER], bacc = 0.f;
    for (int k = 0; k < PER; ++k) acc[k] = 0.f;
    const int nout = O * Cc;
    const int64_t per_blk = (P + gridDim.x - 1) / gridDim.x;
    const int64_t p0 = (int64_t)blockIdx.x * per_blk;
    const int64_t p1 = p0 + per_blk < P ? p0 + per_blk : P;
    for (int64_t t0 = p0; t0 < p1; t0 += WG_PTS) {
        const int np = (int)(p1 - t0 < WG_PTS ? p1 - t0 : WG_PTS);
        __syncthreads();
        for (int i = threadIdx.x; i < np * O; i += blockDim.x) xs[i] = X[t0 * O + i];
        for (int i = threadIdx.x; i < np * Cc; i += blockDim.x) ys[i] = ldv(&Y[t0 * Cc + i]);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int q = threadIdx.x + k * FT;
            if (q < nout) {
                const int o = q / Cc, c = q - o * Cc;
                float s = acc[k];
                for (int j = 0; j < np; ++j) s = fmaf(xs[j * O + o], ys[j * Cc + c], s);
                acc[k] = s;
            }
        }
        if ((int)threadIdx.x < O)
            for (int j = 0; j < np; ++j) bacc += xs[j * O + threadIdx.x];
    }
    double *dst = part + (int64_t)blockIdx.x * (nout + O);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        const int q = threadIdx.x + k * FT;
        if (q < nout) dst[q] = acc[k];
    }
    if ((int)threadIdx.x < O) dst[nout + threadIdx.x] = bacc;
}

// out[k] = sum over blocks of part[blk][k]
__global__ void k_fno_reduce(const double *part, int nblk, int K, float *out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
        double s = 0;
        for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * K + k];
        out[k] = (float)s;
    }
}

// gradient of the spectral weights: dR[kx][ky][i][o] = sum_b dW_b[kx][ky][o] conj(V_b[kx][ky][i])
__global__ void k_fno_dR(const float2 *dW, const float2 *V, Dims d, float2 *dR) {
    extern __shared__ float smem[];
    const int C = d.C, MM = d.MX * d.M;
    float2 *vs = reinterpret_cast<float2 *>(smem), *ws = vs + C;
    const int mode = blockIdx.x;  // kx * M + ky
    float2 acc[4] = {};
    for (int64_t b = 0; b < d.B; ++b) {
        __syncthreads();
        for (int i = threadIdx.x; i < C; i += blockDim.x) {
            vs[i] = V[(b * MM + mode) * (int64_t)C + i];
            ws[i] = dW[(b * MM + mode) * (int64_t)C + i];
        }
        __syncthreads();
        for (int k = 0; k < 4; ++k) {
            const int q = threadIdx.x + k * FT;
            if (q < C * C) {
                const int i = q / C, o = q - i * C;
                const float2 w = ws[o], v = vs[i];
                acc[k].x += w.x * v.x + w.y * v.y;
                acc[k].y += w.y * v.x - w.x * v.y;
            }
        }
    }
    for (int k = 0; k < 4; ++k) {
        const int q = threadIdx.x + k * FT;
        if (q < C * C) dR[(int64_t)mode * C * C + q] = acc[k];
    }
}

// inverse of the axis-1 stage for the backward pass, plus the pointwise part:
// dv[y][c] = sum_o Ww[o][c] da[y][o] + sum_ky Re(dT[ky][c] e^{+2 pi i ky y / n})
__global__ void k_fno_layer_in_bwd(const float2 *dT, const float *da, const float *Ww, Dims d, float *dv) {
    extern __shared__ float smem[];
    const int n = d.n, C = d.C, M = d.M;
    float2 *Ts = reinterpret_cast<float2 *>(smem);
    float *row = reinterpret_cast<float *>(Ts + M * C);
    float *W = row + n * C;
    float *cs = W + C * C, *sn = cs + n;
    const int64_t bx = blockIdx.x;
    for (int i = threadIdx.x; i < M * C; i += blockDim.x) Ts[i] = dT[bx * (int64_t)M * C + i];
    for (int i = threadIdx.x; i < n * C; i += blockDim.x) row[i] = da[bx * (int64_t)n * C + i];
    for (int i = threadIdx.x; i < C * C; i += blockDim.x) W[i] = Ww[i];
    twiddle_table(cs, sn, n);
    __syncthreads();
    for (int o = threadIdx.x; o < n * C; o += blockDim.x) {
        const int y = o / C, c = o - y * C;
        float g = 0.f;
        for (int ky = 0; ky < M; ++ky) {
            const int k = (ky * y) & (n - 1);
            const float2 t = Ts[ky * C + c];
            g = fmaf(t.x, cs[k], fmaf(-t.y, sn[k], g));
        }
        for (int j = 0; j < C; ++j) g = fmaf(W[j * C + c], row[y * C + j], g);
        dv[bx * (int64_t)n * C + o] = g;
    }
}

__global__ void k_fno_adam(float *w, const float *g, float *m, float *v, int64_t count, float lr, float b1, float b2,
                           float eps, float c1, float c2) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

size_t al(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

// ---------------------------------------------------------------- host side
struct qhd_fno {
    Dims d{};
    int64_t batch_max = 0;
    int train = 0, bf16 = 1;
    float *params = nullptr;
    cudaStream_t stream = nullptr;
    int64_t nparam = 0;
    int64_t off_lw = 0, off_lb = 0, off_R[8] = {}, off_W[8] = {}, off_b[8] = {}, off_p1 = 0, off_p1b = 0, off_p2 = 0,
            off_p2b = 0;
    // workspace views
    double2 *stats = nullptr;
    float *feat = nullptr;
    void *v[9] = {}, *a[8] = {};
    float2 *tspec = nullptr, *sspec = nullptr, *vhat[8] = {};
    float *z = nullptr, *p = nullptr, *lse = nullptr;
    float *dz = nullptr, *dh = nullptr, *dv = nullptr, *da = nullptr;
    float2 *dspec = nullptr, *dwhat = nullptr;
    uint4 *fr[4] = {};  // A-operand fragment tables of the tensor-core path (k_fno_frags)
    double *part = nullptr, *loss = nullptr;
    float *m = nullptr, *vv = nullptr;
    int64_t launches = 0;
    std::string err;
};

namespace {

bool cfg_ok(const qhd_fno_config *c) {
    if (!c) return false;
    const int n = c->n;
    // even widths keep every weight block and its bias contiguous in the parameter vector
    return n >= 8 && n <= 256 && (n & (n - 1)) == 0 && c->width >= 2 && c->width <= 32 && c->width % 2 == 0 &&
           c->modes >= 1 && 2 * c->modes <= n && c->modes <= 32 && c->layers >= 1 && c->layers <= 8 &&
           c->hidden >= 2 && c->hidden <= 128 && c->hidden % 2 == 0 && c->hidden * c->width <= FT * 16;
}

Dims dims_of(const qhd_fno_config *c, int64_t B) {
    Dims d;
    d.n = c->n;
    d.C = c->width;
    d.M = c->modes;
    d.MX = 2 * c->modes;
    d.H = c->hidden;
    d.L = c->layers;
    d.B = B;
    return d;
}

int64_t layout_params(const qhd_fno_config *c, qhd_fno *f) {
    const int64_t C = c->width, M = c->modes, H = c->hidden;
    int64_t o = 0;
    auto take = [&](int64_t k) {
        const int64_t r = o;
        o += (k + 1) & ~int64_t(1);  // keep complex blocks 8-byte aligned
        return r;
    };
    const int64_t lw = take(4 * C), lb = take(C);
    int64_t R[8], W[8], bb[8];
    for (int l = 0; l < c->layers; ++l) {
        R[l] = take(2 * M * M * C * C * 2);
        W[l] = take(C * C);
        bb[l] = take(C);
    }
    const int64_t p1 = take(H * C), p1b = take(H), p2 = take(H), p2b = take(1);
    if (f) {
        f->off_lw = lw;
        f->off_lb = lb;
        for (int l = 0; l < c->layers; ++l) {
            f->off_R[l] = R[l];
            f->off_W[l] = W[l];
            f->off_b[l] = bb[l];
        }
        f->off_p1 = p1;
        f->off_p1b = p1b;
        f->off_p2 = p2;
        f->off_p2b = p2b;
    }
    return o;
}

int part_blocks() { return 512; }

// Carves the workspace (base = f->stats on entry when f is given); returns its size.
size_t workspace(const qhd_fno_config *c, int64_t B, int train, qhd_fno *f) {
    const Dims d = dims_of(c, B);
    const int64_t P = d.P();
    const size_t act = c->act_bf16 ? 2 : 4;
    const size_t spec = (size_t)B * d.n * d.M * d.C * sizeof(float2);
    const size_t vh = (size_t)B * d.MX * d.M * d.C * sizeof(float2);
    const int64_t np = layout_params(c, nullptr);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t r = off;
        off = al(off + bytes);
        return r;
    };
    const size_t o_stats = take(B * sizeof(double2));
    const size_t o_feat = take(P * 4 * sizeof(float));
    size_t o_v[9], o_a[8], o_vh[8];
    for (int l = 0; l <= c->layers; ++l) o_v[l] = take(P * d.C * act);
    for (int l = 0; l + 1 < c->layers; ++l) o_a[l] = take(P * d.C * act);
    const size_t o_t = take(spec), o_s = take(spec);
    for (int l = 0; l < c->layers; ++l) o_vh[l] = take(vh);
    const size_t o_z = take(P * sizeof(float)), o_p = take(P * sizeof(float)), o_lse = take(B * sizeof(float));
    size_t o_fr[4] = {0, 0, 0, 0};
    const bool frl = c->act_bf16 && tc_layer_ok(d), frs = frl && tc_specx_ok(d);
    for (int k = 0; k < 4; ++k)
        if (k < 2 ? frl : frs) o_fr[k] = take(frag_count(d, k) * sizeof(uint4));
    size_t o_dz = 0, o_dh = 0, o_dv = 0, o_da = 0, o_ds = 0, o_dw = 0, o_part = 0, o_loss = 0, o_m = 0, o_vv = 0;
    if (train) {
        o_dz = take(P * sizeof(float));
        o_dh = take(P * d.H * sizeof(float));
        o_dv = take(P * d.C * sizeof(float));
        o_da = take(P * d.C * sizeof(float));
        o_ds = take(spec);
        o_dw = take(vh);
        // longest partial row: projection (H C + H), pointwise layer (C C + C), lift (5 C), H + 1
        int64_t K = (int64_t)d.H * d.C + d.H;
        if ((int64_t)d.C * d.C + d.C > K) K = (int64_t)d.C * d.C + d.C;
        if (5 * (int64_t)d.C > K) K = 5 * (int64_t)d.C;
        if ((int64_t)d.H + 1 > K) K = d.H + 1;
        o_part = take((size_t)part_blocks() * (size_t)K * sizeof(double));
        o_loss = take(B * sizeof(double));
        o_m = take(np * sizeof(float));
        o_vv = take(np * sizeof(float));
    }
    if (f) {
        char *w = (char *)f->stats;
        f->stats = (double2 *)(w + o_stats);
        f->feat = (float *)(w + o_feat);
        for (int l = 0; l <= c->layers; ++l) f->v[l] = w + o_v[l];
        for (int l = 0; l + 1 < c->layers; ++l) f->a[l] = w + o_a[l];
        f->tspec = (float2 *)(w + o_t);
        f->sspec = (float2 *)(w + o_s);
        for (int l = 0; l < c->layers; ++l) f->vhat[l] = (float2 *)(w + o_vh[l]);
        f->z = (float *)(w + o_z);
        f->p = (float *)(w + o_p);
        f->lse = (float *)(w + o_lse);
        for (int k = 0; k < 4; ++k) f->fr[k] = (k < 2 ? frl : frs) ? (uint4 *)(w + o_fr[k]) : nullptr;
        if (train) {
            f->dz = (float *)(w + o_dz);
            f->dh = (float *)(w + o_dh);
            f->dv = (float *)(w + o_dv);
            f->da = (float *)(w + o_da);
            f->dspec = (float2 *)(w + o_ds);
            f->dwhat = (float2 *)(w + o_dw);
            f->part = (double *)(w + o_part);
            f->loss = (double *)(w + o_loss);
            f->m = (float *)(w + o_m);
            f->vv = (float *)(w + o_vv);
        }
    }
    return off;
}

int grid_for(int64_t count) {
    int64_t b = (count + FT - 1) / FT;
    if (b > 152 * 16) b = 152 * 16;
    return b < 1 ? 1 : (int)b;
}

qhd_status ffail(qhd_fno *f, qhd_status s, const char *msg) {
    if (f) f->err = msg;
    return s;
}

#define FNO_CHECK(f)                                                                    \
    do {                                                                                \
        cudaError_t e_ = cudaGetLastError();                                            \
        if (e_ != cudaSuccess) return ffail((f), QHD_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

// blocks of the tensor-core projection: 128 points per block pass, at most 16 blocks per SM
int64_t tc_proj_grid(const Dims &d) {
    const int64_t tiles = (d.P() + 127) / 128;
    return tiles < 152 * 16 ? tiles : 152 * 16;
}

size_t smem_dfty(const Dims &d) { return (size_t)(d.n * d.C + 2 * d.n) * sizeof(float); }
size_t smem_specx(const Dims &d) {
    return (size_t)(d.n * d.C + 2 * d.MX * d.C) * sizeof(float2) + 2 * d.n * sizeof(float);
}
size_t smem_layer(const Dims &d) {
    return (size_t)d.M * d.C * sizeof(float2) + (size_t)(d.n * d.C + d.C * d.C + 2 * d.n) * sizeof(float);
}
size_t smem_proj(const Dims &d) { return (size_t)(d.H * d.C + 3 * d.H + 1) * sizeof(float); }

template <typename T>
void set_smem_limits() {
    const int big = 200 * 1024;
    cudaFuncSetAttribute(k_fno_dfty<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_fno_dfty<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_fno_specx<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_fno_specx<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_fno_specx_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_fno_specx_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_fno_layer_out<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
    cudaFuncSetAttribute(k_fno_layer_in_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, big);
}

// forward pass over `B` instances; activations kept for the backward pass
template <typename T>
qhd_status forward(qhd_fno *f, const double *fx, const float *sigma, int64_t B, float *p_out) {
    Dims d = f->d;
    d.B = B;
    cudaStream_t s = f->stream;
    const float *W = f->params;
    k_fno_fstats<<<(unsigned)B, FT, 0, s>>>(fx, d.G(), f->stats);
    k_fno_lift<T><<<grid_for(d.P()), FT, 0, s>>>(fx, sigma, f->stats, W + f->off_lw, W + f->off_lb, d, f->feat,
                                                 (T *)f->v[0]);
    f->launches += 2;
    for (int l = 0; l < d.L; ++l) {
        const T *vin = (const T *)f->v[l];
        if (f->bf16 && tc_layer_ok(d))
            k_fno_dfty_tc<T><<<(unsigned)(B * d.n), FT, 0, s>>>(vin, d, 1.f, 1.f, f->tspec, f->fr[0]);
        else
            k_fno_dfty<T><<<(unsigned)(B * d.n), FT, smem_dfty(d), s>>>(vin, d, 1.f, 1.f, f->tspec);
        if (f->bf16 && tc_specx_ok(d))
            k_fno_specx_tc<false><<<(unsigned)(B * d.M), FT, smem_specx_tc(d), s>>>(
                f->tspec, reinterpret_cast<const float2 *>(W + f->off_R[l]), d, f->vhat[l], f->sspec, f->fr[2],
                f->fr[3]);
        else
            k_fno_specx<false><<<(unsigned)(B * d.M), FT, smem_specx(d), s>>>(
                f->tspec, reinterpret_cast<const float2 *>(W + f->off_R[l]), d, f->vhat[l], f->sspec);
        const int act = l + 1 < d.L;
        if (f->bf16 && tc_layer_ok(d))
            k_fno_layer_out_tc<<<(unsigned)(B * d.n), FT, 0, s>>>(
                f->sspec, (const __nv_bfloat16 *)vin, W + f->off_W[l], W + f->off_b[l], d, act,
                act ? (__nv_bfloat16 *)f->a[l] : nullptr, (__nv_bfloat16 *)f->v[l + 1], f->fr[1]);
        else
            k_fno_layer_out<T><<<(unsigned)(B * d.n), FT, smem_layer(d), s>>>(
                f->sspec, vin, W + f->off_W[l], W + f->off_b[l], d, act, act ? (T *)f->a[l] : nullptr,
                (T *)f->v[l + 1]);
        f->launches += 3;
    }
    if (f->bf16 && tc_proj_ok(d))
        k_fno_proj_tc<<<(unsigned)tc_proj_grid(d), FT, 0, s>>>((const __nv_bfloat16 *)f->v[d.L], W + f->off_p1,
                                                              W + f->off_p1b, W + f->off_p2, W + f->off_p2b, d, f->z);
    else
        k_fno_proj<T><<<grid_for(d.P()), FT, smem_proj(d), s>>>((const T *)f->v[d.L], W + f->off_p1, W + f->off_p1b,
                                                              W + f->off_p2, W + f->off_p2b, d, f->z);
    k_fno_softmax<<<(unsigned)B, FT, 0, s>>>(f->z, d.G(), p_out ? p_out : f->p, f->lse);
    f->launches += 2;
    FNO_CHECK(f);
    return QHD_OK;
}

template <typename T>
qhd_status backward(qhd_fno *f, const float *p_true, int64_t B, float *grad, double *loss_host) {
    Dims d = f->d;
    d.B = B;
    cudaStream_t s = f->stream;
    const float *W = f->params;
    const int64_t P = d.P();
    const int nb = part_blocks();
    k_fno_loss<<<(unsigned)B, FT, 0, s>>>(f->z, f->lse, f->p, p_true, d.G(), 1.f / (float)B, f->dz, f->loss);
    // projection
    const size_t sp = smem_proj(d) + (size_t)(d.H + 1) * sizeof(float);
    if (f->bf16 && tc_proj_ok(d))
        k_fno_proj_bwd_tc<<<nb, FT, 0, s>>>((const __nv_bfloat16 *)f->v[d.L], f->dz, W + f->off_p1, W + f->off_p1b,
                                             W + f->off_p2, d, f->dh, f->dv, f->part);
    else
        k_fno_proj_bwd<T><<<nb, FT, sp, s>>>((const T *)f->v[d.L], f->dz, W + f->off_p1, W + f->off_p1b, W + f->off_p2,
                                              d, f->dh, f->dv, f->part);
    k_fno_reduce<<<1, FT, 0, s>>>(f->part, nb, d.H + 1, grad + f->off_p2);
    if (f->bf16 && tc_wgrad_ok(d, d.H))
        k_fno_wgrad_tc<<<nb, FT, 0, s>>>(f->dh, (const __nv_bfloat16 *)f->v[d.L], P, d.H, f->part);
    else
        k_fno_wgrad<T><<<nb, FT, 0, s>>>(f->dh, (const T *)f->v[d.L], P, d.H, d.C, f->part);
    k_fno_reduce<<<grid_for((int64_t)d.H * d.C + d.H), FT, 0, s>>>(f->part, nb, d.H * d.C + d.H, grad + f->off_p1);
    f->launches += 5;
    for (int l = d.L - 1; l >= 0; --l) {
        const int act = l + 1 < d.L;
        k_fno_act_bwd<T><<<grid_for(P * d.C), FT, 0, s>>>(f->dv, act ? (const T *)f->a[l] : nullptr, P * d.C, act,
                                                        f->da);
        // pointwise weights and bias: sum over points of da (x) v_l
        if (f->bf16 && tc_wgrad_ok(d, d.C))
            k_fno_wgrad_tc<<<nb, FT, 0, s>>>(f->da, (const __nv_bfloat16 *)f->v[l], P, d.C, f->part);
        else
            k_fno_wgrad<T><<<nb, FT, 0, s>>>(f->da, (const T *)f->v[l], P, d.C, d.C, f->part);
        k_fno_reduce<<<grid_for((int64_t)d.C * d.C + d.C), FT, 0, s>>>(f->part, nb, d.C * d.C + d.C,
                                                                      grad + f->off_W[l]);
        // spectral path: adjoint of the inverse axis-1 stage, then of the axis-0 stages
        const float inv = 1.f / ((float)d.n * (float)d.n);
        if (f->bf16 && tc_layer_ok(d))
            k_fno_dfty_tc<float><<<(unsigned)(B * d.n), FT, 0, s>>>(f->da, d, inv, 2.f * inv, f->dspec, f->fr[0]);
        else
            k_fno_dfty<float><<<(unsigned)(B * d.n), FT, smem_dfty(d), s>>>(f->da, d, inv, 2.f * inv, f->dspec);
        if (f->bf16 && tc_specx_ok(d))
            k_fno_specx_tc<true><<<(unsigned)(B * d.M), FT, smem_specx_tc(d), s>>>(
                f->dspec, reinterpret_cast<const float2 *>(W + f->off_R[l]), d, f->dwhat, f->tspec, f->fr[2],
                f->fr[3]);
        else
            k_fno_specx<true><<<(unsigned)(B * d.M), FT, smem_specx(d), s>>>(
                f->dspec, reinterpret_cast<const float2 *>(W + f->off_R[l]), d, f->dwhat, f->tspec);
        k_fno_dR<<<(unsigned)(d.MX * d.M), FT, 2 * d.C * sizeof(float2), s>>>(
            f->dwhat, f->vhat[l], d, reinterpret_cast<float2 *>(grad + f->off_R[l]));
        if (f->bf16 && tc_layer_ok(d))
            k_fno_layer_in_bwd_tc<<<(unsigned)(B * d.n), FT, 0, s>>>(f->tspec, f->da, W + f->off_W[l], d, f->dv,
                                                                      f->fr[1]);
        else
            k_fno_layer_in_bwd<<<(unsigned)(B * d.n), FT, smem_layer(d), s>>>(f->tspec, f->da, W + f->off_W[l], d,
                                                                               f->dv);
        f->launches += 7;
    }
    // lift: sum over points of dv0 (x) features
    k_fno_wgrad<float><<<nb, FT, 0, s>>>(f->dv, f->feat, P, d.C, 4, f->part);
    k_fno_reduce<<<grid_for(5 * d.C), FT, 0, s>>>(f->part, nb, 4 * d.C + d.C, grad + f->off_lw);
    f->launches += 2;
    FNO_CHECK(f);
    if (loss_host) {
        std::vector<double> l(B);
        if (cudaMemcpyAsync(l.data(), f->loss, B * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return ffail(f, QHD_ERR_CUDA, "loss copy failed");
        double t = 0;
        for (double v : l) t += v;
        *loss_host = t / (double)B;
    }
    return QHD_OK;
}

}  // namespace

extern "C" {

int64_t qhd_fno_param_count(const qhd_fno_config *cfg) { return cfg_ok(cfg) ? layout_params(cfg, nullptr) : 0; }

size_t qhd_fno_workspace_bytes(const qhd_fno_config *cfg, int64_t batch_max, int train) {
    if (!cfg_ok(cfg) || batch_max < 1 || batch_max > 65535) return 0;
    return workspace(cfg, batch_max, train ? 1 : 0, nullptr);
}

qhd_status qhd_fno_create(qhd_fno **out, const qhd_fno_config *cfg, int64_t batch_max, int train, float *params_dev,
                          void *work_dev, size_t work_bytes, void *stream) {
    if (!out || !cfg_ok(cfg) || !params_dev || batch_max < 1 || batch_max > 65535) return QHD_ERR_INVALID_ARG;
    if (((uintptr_t)params_dev & 7) != 0) return QHD_ERR_INVALID_ARG;
    const size_t need = workspace(cfg, batch_max, train ? 1 : 0, nullptr);
    if (!work_dev || ((uintptr_t)work_dev & 255) || work_bytes < need) return QHD_ERR_WORKSPACE;
    qhd_fno *f = new qhd_fno();
    f->d = dims_of(cfg, batch_max);
    f->batch_max = batch_max;
    f->train = train ? 1 : 0;
    f->bf16 = cfg->act_bf16 ? 1 : 0;
    f->params = params_dev;
    f->stream = (cudaStream_t)stream;
    f->nparam = layout_params(cfg, f);
    f->stats = (double2 *)work_dev;
    workspace(cfg, batch_max, f->train, f);
    if (f->bf16) set_smem_limits<__nv_bfloat16>();
    else set_smem_limits<float>();
    if (f->fr[0]) {
        k_fno_frags<<<64, FT, 0, f->stream>>>(f->fr[0], f->fr[1], f->fr[2], f->fr[3], f->d);
        if (cudaGetLastError() != cudaSuccess) {
            delete f;
            return QHD_ERR_CUDA;
        }
    }
    if (f->train) {
        if (cudaMemsetAsync(f->m, 0, f->nparam * sizeof(float), f->stream) != cudaSuccess ||
            cudaMemsetAsync(f->vv, 0, f->nparam * sizeof(float), f->stream) != cudaSuccess) {
            delete f;
            return QHD_ERR_CUDA;
        }
    }
    *out = f;
    return QHD_OK;
}

qhd_status qhd_fno_forward(qhd_fno *f, const double *f_dev, const float *sigma_dev, int64_t batch, float *p_dev) {
    if (!f) return QHD_ERR_INVALID_ARG;
    if (!f_dev || !sigma_dev || !p_dev || batch < 1 || batch > f->batch_max)
        return ffail(f, QHD_ERR_INVALID_ARG, "bad forward arguments");
    return f->bf16 ? forward<__nv_bfloat16>(f, f_dev, sigma_dev, batch, p_dev)
                   : forward<float>(f, f_dev, sigma_dev, batch, p_dev);
}

qhd_status qhd_fno_loss_grad(qhd_fno *f, const double *f_dev, const float *sigma_dev, const float *p_true_dev,
                             int64_t batch, float *grad_dev, double *loss_host) {
    if (!f) return QHD_ERR_INVALID_ARG;
    if (!f->train) return ffail(f, QHD_ERR_STATE, "created without training buffers");
    if (!f_dev || !sigma_dev || !p_true_dev || !grad_dev || batch < 1 || batch > f->batch_max)
        return ffail(f, QHD_ERR_INVALID_ARG, "bad loss_grad arguments");
    qhd_status s = f->bf16 ? forward<__nv_bfloat16>(f, f_dev, sigma_dev, batch, nullptr)
                           : forward<float>(f, f_dev, sigma_dev, batch, nullptr);
    if (s != QHD_OK) return s;
    return f->bf16 ? backward<__nv_bfloat16>(f, p_true_dev, batch, grad_dev, loss_host)
                   : backward<float>(f, p_true_dev, batch, grad_dev, loss_host);
}

qhd_status qhd_fno_adam_step(qhd_fno *f, const float *grad_dev, float lr, float beta1, float beta2, float eps,
                             int64_t t) {
    if (!f) return QHD_ERR_INVALID_ARG;
    if (!f->train) return ffail(f, QHD_ERR_STATE, "created without training buffers");
    if (!grad_dev || t < 1 || !(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
        !(eps > 0.f))
        return ffail(f, QHD_ERR_INVALID_ARG, "bad Adam arguments");
    const float c1 = 1.f / (1.f - powf(beta1, (float)t)), c2 = 1.f / (1.f - powf(beta2, (float)t));
    k_fno_adam<<<grid_for(f->nparam), FT, 0, f->stream>>>(f->params, grad_dev, f->m, f->vv, f->nparam, lr, beta1,
                                                          beta2, eps, c1, c2);
    f->launches += 1;
    FNO_CHECK(f);
    return QHD_OK;
}

int64_t qhd_fno_launch_count(const qhd_fno *f) { return f ? f->launches : 0; }

const char *qhd_fno_last_error(const qhd_fno *f) { return f ? f->err.c_str() : ""; }

qhd_status qhd_fno_destroy(qhd_fno *f) {
    if (!f) return QHD_OK;
    const cudaError_t e = cudaStreamSynchronize(f->stream);
    delete f;
    return e == cudaSuccess ? QHD_OK : QHD_ERR_CUDA;
}

}  // extern "C"
