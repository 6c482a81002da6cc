// qhd_tcdft.cu -- tensor-core DFT form of the 2-D step.
//
// The per-axis transforms of the pseudo-spectral step (Eq. prod_qhd_fft) are
// dense matrix products on the tensor cores.  B instances of n x n points are
// a matrix of B*n rows of n complex values, stored per row as [re | im]; one
// axis transform is the product of that matrix with the real block form of
// the DFT matrix,
//     [xr | xi] . [[Wr, Wi], [-Wi, Wr]] = [Xr | Xi],   W_jk = exp(-+2 pi i jk / n).
// W is symmetric, so the transform along axis 0 is the same right product
// after each instance is transposed; a step is
//     potential phase -> W (axis 1) -> transpose -> W (axis 0) -> kinetic phase
//     -> conj W (axis 0) -> transpose -> conj W (axis 1)
// and ends in natural layout, ready for the next step's potential phase.  The
// state stays in the FP32 product buffer between steps; psi is read at the
// start of an evolve call and written at its end.  The kernels here apply the
// phases, transpose and split the operands; the GEMMs are the project's
// tcgen05 kernel (qhd_umma_gemm.cu): FP16 operands, FP32 accumulation in
// tensor memory, partials added in FP32 with round-to-nearest.
//
// Two operand forms.
//
// Block-scaled hi/lo (3 products, the FP16 hi-lo form).  Each run of 16
// consecutive K values of a row (16 real or 16 imaginary parts) shares an
// exponent e with 2^e > their largest magnitude; a value x is cut into FP16
// integers a = rint(x 2^(10-e)) and c = rint((x 2^(10-e) - a) 2^11), both in
// [-1024, 1024], and W (|W| <= 1) into W_hi = rint(2^10 W) and
// W_lo = rint((2^10 W - W_hi) 2^11).  The products a W_hi, a W_lo and c W_hi
// (c W_lo, of order 2^-22, is dropped) are integers below 2^20, so the exact
// 16-term sum of one MMA stays below 2^24 and FP32 holds it exactly: every
// MMA is an accumulation group of its own, scaled by 2^(e - 20) or
// 2^(e - 31) and added to the FP32 result with round-to-nearest.  No partial
// is ever truncated, so no bias enters (the tensor cores truncate each MMA's
// sum towards zero, and a long accumulation in tensor memory drifts towards
// zero by about 1e-9 K relative: measured).  x keeps 21 bits below the
// largest value of its block and W 21 bits; the block exponents travel in a
// [rows][2n/16] int8 table.  All scales are exact powers of two, the
// transforms are unnormalised, and the kinetic table's 1/n^2 brings each step
// back to psi's scale.
//
// Fixed-point slices (10 products, an error-free splitting in the manner of
// Ozaki et al.).  Each instance is scaled by a power of two 2^(7-e) with
// 2^e > max |z| over the instance, and every real value u (|u| <= 2^7) is
// cut into integer slices u = a0 + 2^-7 a1 + 2^-14 a2 + 2^-21 a3, each
// |a_i| <= 2^7 (this holds the FP32 value to 2^-28 of the instance maximum);
// 2^7 W likewise into integer slices w0..w3 (29 bits).  A GEMM of one slice
// level sums integers that the FP32 accumulator holds exactly whatever its
// rounding (below 2^24 for levels 0 and 1; levels 2 and 3 are ~2^-14 and
// ~2^-21 corrections), so no bias enters:
//   level L: [a0 | .. | aL] . [wL; ..; w0]        (K = 2n (L + 1))
// and each level is one accumulation group of the GEMM whose exact partial is
// added to the FP32 result times 2^-7L.  A per-instance
// power-of-two exponent E (true value = buffer * 2^E) follows the scales and
// is read back at the end.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include <cuda_fp16.h>

#include "qhd_device.cuh"
#include "qhd_tcdft.h"

namespace qhd {

namespace {

constexpr int TC_BFP = 3;              // split of the block-scaled forms (3 and 5 products)
constexpr int TC_THREADS = 256;
constexpr int TC_TR = 64, TC_TC = 32;  // transpose tile: input rows x input columns
constexpr int TC_FIXED = 10;           // products of the fixed-point form
// GEMM tile width (columns of C per CTA) requested: 256 where the 2n columns allow
// it (the GEMM keeps 128 for per-MMA groups)
int tc_bn(int n) { return (2 * n) % 256 == 0 ? 256 : 128; }

struct SplitOut {
    __half *a;     // B*n rows of segments of 2n FP16
    int64_t kp;    // row length in halves
    int n;
    int8_t *e;     // block-scaled form: exponent of each 16 K values, [B*n][2n/16]
    int64_t eld;
};

// Per-instance scale state of the fixed-point form.
struct FixedScale {
    const unsigned *maxin;  // max |z|^2 of the split's input, per instance (float bits)
    unsigned *maxclr;       // the other max buffer, cleared for the next transform
    int *e;                 // per-instance exponent: true value = buffer * 2^E
    int e_add;              // extra exponent of this split (-2 log2 n for the kinetic split)
    int from_psi;           // E restarts at this split
};

// ------------------------------------------------------ block-scaled hi/lo
// Exponent e with 2^e > max |x| over the 16 values held by 8 neighbouring
// lanes (two each); the lanes of one block must be converged.
__device__ __forceinline__ int block_exponent16(float m) {
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
    m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 4));
    int e = -100;  // an all-zero block: any scale holds it
    if (m > 0.f) frexpf(m, &e);
    // blocks below 2^-100 (far under the state's rounding) keep the floor, so
    // 2^(10 - e) and 2^e stay normal floats
    return e < -100 ? -100 : e;
}

// Values x0, x1 of columns col, col+1 of one row (col + 16 k .. col + 16 k + 15
// held by lanes 8g .. 8g+7): segments [a | c] and the block's exponent.  The
// power-of-two scaling and the subtraction are exact; a and c are integers in
// [-1024, 1024], exact in FP16.
__device__ __forceinline__ void put_bfp_pair(const SplitOut &o, int64_t row, int col, float x0, float x1) {
    const int e = block_exponent16(fmaxf(fabsf(x0), fabsf(x1)));
    const float sc = __int_as_float((127 + 10 - e) << 23);  // 2^(10 - e)
    const float u0 = x0 * sc, u1 = x1 * sc;
    const float a0 = rintf(u0), a1 = rintf(u1);
    const float c0 = rintf((u0 - a0) * 2048.f), c1 = rintf((u1 - a1) * 2048.f);
    const int m = 2 * o.n;
    __half2 *dst = reinterpret_cast<__half2 *>(o.a + row * o.kp + col);
    dst[0] = __floats2half2_rn(a0, a1);
    dst[m / 2] = __floats2half2_rn(c0, c1);
    if ((threadIdx.x & 7) == 0) o.e[row * o.eld + col / 16] = (int8_t)e;
}

// Fixed-point slices of two neighbouring values u0, u1 (|u| <= 2^7):
// segments [a0 | a1 | a2 | a3].  Each subtraction and power-of-two product is
// exact in FP32; only the last slice rounds (below 2^-21).
__device__ __forceinline__ void put_fixed_pair(const SplitOut &o, int64_t row, int col, float u0, float u1) {
    const int m = 2 * o.n;
    __half2 *dst = reinterpret_cast<__half2 *>(o.a + row * o.kp + col);
    float r0 = u0, r1 = u1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float p = rintf(r0), q = rintf(r1);
        dst[k * (m / 2)] = __floats2half2_rn(p, q);
        r0 = (r0 - p) * 128.f;
        r1 = (r1 - q) * 128.f;
    }
}

// Exponent e with 2^e > max |z| of an instance (max |z|^2 given as float bits).
__device__ __forceinline__ int tc_exponent(unsigned m2bits) {
    const float m2 = __uint_as_float(m2bits);
    if (!(m2 > 0.f)) return 0;
    int e;
    frexpf(sqrtf(m2), &e);
    return e;
}

template <int P>
__device__ __forceinline__ void put_two(const SplitOut &o, int64_t row, int col, float x0, float x1) {
    if (P == TC_FIXED) put_fixed_pair(o, row, col, x0, x1);
    else put_bfp_pair(o, row, col, x0, x1);
}

// mode 0: potential phase, input psi (interleaved); 1: potential phase, input
// the product buffer; 2: kinetic phase, input the product buffer (rows hold
// frequency k1 of axis 1, columns frequency k0 of axis 0).  One thread per two
// neighbouring columns of one row (a warp covers 64 columns of one row, so the
// block-scaled form's 16-column blocks lie in 8-lane groups).  scale: a
// power of two applied on input.
template <int P, int MODE>
__global__ void __launch_bounds__(TC_THREADS) k_tc_split(SplitOut o, const float *cbuf, TcPhaseArgs a,
                                                         int64_t rows, float scale, FixedScale fs) {
    __shared__ float4 ptab[PHASE_TAB];
    if (MODE != 2) {
        load_phase_tab(ptab, a.ptab);
        __syncthreads();
    }
    const int n = o.n, half = n / 2;
    const int64_t total = rows * half;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / half;
        const int col = 2 * (int)(i - row * half);
        const int64_t b = row / n;
        float sc = scale;
        if (P == TC_FIXED) {
            const int e = tc_exponent(fs.maxin[b]);
            sc = ldexpf(scale, 7 - e);
            if (row == b * n && col == 0) {  // one thread per instance
                fs.e[b] = (fs.from_psi ? 0 : fs.e[b]) + e - 14 + fs.e_add;
                fs.maxclr[b] = 0u;
            }
        }
        float2 z0, z1;
        if (MODE == 0) {
            const float4 v = *reinterpret_cast<const float4 *>(a.psi + row * n + col);
            z0 = make_float2(v.x * sc, v.y * sc);
            z1 = make_float2(v.z * sc, v.w * sc);
        } else {
            const float2 re = *reinterpret_cast<const float2 *>(cbuf + row * 2 * n + col);
            const float2 im = *reinterpret_cast<const float2 *>(cbuf + row * 2 * n + n + col);
            z0 = make_float2(re.x * sc, im.x * sc);
            z1 = make_float2(re.y * sc, im.y * sc);
        }
        if (MODE == 2) {
            // kinetic factor of (k0, k1): axis 0 first, then axis 1
            const float4 *kb = a.kt + (a.kt_batch == 1 ? 0 : b) * a.ksum;
            const int k1 = (int)(row - b * n);
            const float4 f1 = __ldg(&kb[n + k1]);
            const float4 f0a = __ldg(&kb[col]), f0b = __ldg(&kb[col + 1]);
            z0 = cmul_comp(z0, make_float2(f0a.x, f0a.y), make_float2(f0a.z, f0a.w));
            z0 = cmul_comp(z0, make_float2(f1.x, f1.y), make_float2(f1.z, f1.w));
            z1 = cmul_comp(z1, make_float2(f0b.x, f0b.y), make_float2(f0b.z, f0b.w));
            z1 = cmul_comp(z1, make_float2(f1.x, f1.y), make_float2(f1.z, f1.w));
        } else {
            const uint64_t coef = a.pot[b];
            const uint2 f = *reinterpret_cast<const uint2 *>(a.fq + row * n + col);
            z0 = apply_phase_tab(z0, turns_mul(coef, f.x) + a.dither, ptab);
            z1 = apply_phase_tab(z1, turns_mul(coef, f.y) + a.dither, ptab);
        }
        put_two<P>(o, row, col, z0.x, z1.x);
        put_two<P>(o, row, n + col, z0.y, z1.y);
    }
}

// Product buffer rows (b, r), columns c -> split rows (b, c), columns r.
// Tile: TC_TR input rows x TC_TC input columns, block (32, 8).
template <int P>
__global__ void __launch_bounds__(TC_THREADS) k_tc_split_t(SplitOut o, const float *cbuf, FixedScale fs) {
    __shared__ float tr[TC_TR][TC_TC + 1], ti[TC_TR][TC_TC + 1];
    const int n = o.n;
    const int64_t b = blockIdx.z;
    const int r0 = blockIdx.y * TC_TR, c0 = blockIdx.x * TC_TC;
    float sc = 1.f;
    if (P == TC_FIXED) {
        const int e = tc_exponent(fs.maxin[b]);
        sc = ldexpf(1.f, 7 - e);
        if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
            fs.e[b] = fs.e[b] + e - 14;
            fs.maxclr[b] = 0u;
        }
    }
    const float *base = cbuf + b * (int64_t)n * 2 * n;
    for (int k = threadIdx.y; k < TC_TR; k += blockDim.y) {
        const float *rp = base + (int64_t)(r0 + k) * 2 * n + c0 + threadIdx.x;
        tr[k][threadIdx.x] = rp[0] * sc;
        ti[k][threadIdx.x] = rp[n] * sc;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < TC_TC; k += blockDim.y) {
        const int64_t row = b * n + c0 + k;
        const int r = 2 * threadIdx.x;
        put_two<P>(o, row, r0 + r, tr[r][k], tr[r + 1][k]);
        put_two<P>(o, row, n + r0 + r, ti[r][k], ti[r + 1][k]);
    }
}

// Per-instance max |z|^2 of psi (interleaved) or of the product buffer
// (rows of [re | im]); grid (blocks per instance, B).
template <bool INTERLEAVED>
__global__ void __launch_bounds__(TC_THREADS) k_tc_absmax(const float *in, int n, unsigned *maxbits) {
    const int64_t b = blockIdx.y;
    const int64_t g = (int64_t)n * n;
    const float *base = in + b * g * 2;
    const int half = n / 2;
    float m = 0.f;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < g / 2; p += (int64_t)gridDim.x * blockDim.x) {
        if (INTERLEAVED) {
            const float4 v = reinterpret_cast<const float4 *>(base)[p];
            m = fmaxf(m, fmaxf(v.x * v.x + v.y * v.y, v.z * v.z + v.w * v.w));
        } else {
            const int64_t row = p / half;
            const int col = 2 * (int)(p - row * half);
            const float2 re = *reinterpret_cast<const float2 *>(base + row * 2 * n + col);
            const float2 im = *reinterpret_cast<const float2 *>(base + row * 2 * n + n + col);
            m = fmaxf(m, fmaxf(re.x * re.x + im.x * im.x, re.y * re.y + im.y * im.y));
        }
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[TC_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < TC_THREADS / 32; ++w) m = fmaxf(m, wm[w]);
        atomicMax(&maxbits[b], __float_as_uint(m));
    }
}

// Product buffer (natural layout) -> psi, with the final potential phase.
// Block-scaled forms: a fixed scale (1); fixed-point form: 2^E per instance.
__global__ void __launch_bounds__(TC_THREADS) k_tc_finish(const float *cbuf, TcPhaseArgs a, int n, int64_t rows,
                                                         float scale, const int *e, int phase) {
    __shared__ float4 ptab[PHASE_TAB];
    load_phase_tab(ptab, a.ptab);
    __syncthreads();
    const int half = n / 2;
    const int64_t total = rows * half;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / half;
        const int col = 2 * (int)(i - row * half);
        const int64_t b = row / n;
        const float sc = e ? ldexpf(1.f, e[b]) : scale;
        const float2 re = *reinterpret_cast<const float2 *>(cbuf + row * 2 * n + col);
        const float2 im = *reinterpret_cast<const float2 *>(cbuf + row * 2 * n + n + col);
        float2 z0 = make_float2(re.x * sc, im.x * sc), z1 = make_float2(re.y * sc, im.y * sc);
        if (phase) {
            const uint64_t coef = a.pot[b];
            const uint2 f = *reinterpret_cast<const uint2 *>(a.fq + row * n + col);
            z0 = apply_phase_tab(z0, turns_mul(coef, f.x), ptab);
            z1 = apply_phase_tab(z1, turns_mul(coef, f.y), ptab);
        }
        *reinterpret_cast<float4 *>(a.psi + row * n + col) = make_float4(z0.x, z0.y, z1.x, z1.y);
    }
}

size_t tc_align(size_t v) { return (v + 255) & ~size_t(255); }

int log2i(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// K extent (in units of 2n) of the DFT-matrix buffers of one direction, and
// the row length (in units of 2n) of the split operands.
int w_segments(int products) { return products == TC_FIXED ? 4 : products == 5 ? 3 : 2; }
int a_segments(int products) { return products == TC_FIXED ? 4 : 2; }
// Row pitch (halves) of an operand of `segs` segments of m values: 128 bytes more
// than the segments need, so consecutive rows of a TMA box (a power-of-two
// number of bytes apart otherwise) spread over the L2 slices.
int64_t tc_pitch(int segs, size_t m) { return (int64_t)segs * (int64_t)m + 64; }

}  // namespace

struct TcState {
    int n = 0, products = 3, l = 0;
    int64_t batch = 0;
    unsigned *err = nullptr;            // GEMM wait time-out word (2 words)
    __half *w[2] = {nullptr, nullptr};  // forward, inverse DFT matrix, stored transposed [2n][pitch]: K-major
    float *wres[2] = {nullptr, nullptr}; // block-scaled forms: the last W slice before rounding, [2n][2n]
    __half *a = nullptr;                // B*n rows of split operands (padded pitch, tc_pitch)
    float *c = nullptr;                 // B*n x 2n products
    unsigned *maxbits = nullptr;        // fixed form: 2 x B max |z|^2 buffers
    int *e = nullptr;                   // fixed form: B exponents
    int8_t *e8 = nullptr;               // block-scaled form: [B*n][2n/16] block exponents
    int cur = 0;                        // max buffer of the next split
    int grid = 0;
};

bool tc_supported(int n0, int n1, int64_t batch) {
    // transpose grids index instances by blockIdx.z; the GEMM takes B*n rows as int
    return n0 == n1 && n0 >= 64 && n0 <= 1024 && (n0 & (n0 - 1)) == 0 && batch >= 1 && batch <= 65535;
}

bool tc_products_ok(int n, int products) {
    // the fixed-point level-0 and level-1 sums stay below 2^24 for K = 2n <= 1024
    return products == 3 || products == 5 || (products == TC_FIXED && n <= 512);
}

size_t tc_workspace_bytes(int n, int64_t batch, int products) {
    const size_t m = 2 * (size_t)n, rows = (size_t)batch * (size_t)n;
    size_t t = 0;
    t += 2 * tc_align((size_t)tc_pitch(w_segments(products), m) * m * sizeof(__half));
    t += tc_align(rows * (size_t)tc_pitch(a_segments(products), m) * sizeof(__half));
    t += tc_align(rows * m * sizeof(float));
    t += tc_align(2 * (size_t)batch * sizeof(unsigned));
    t += tc_align((size_t)batch * sizeof(int));
    t += tc_align(2 * sizeof(unsigned));  // GEMM wait time-out word
    t += tc_align(rows * (m / 16));       // block exponents of the block-scaled form
    if (products != TC_FIXED) t += 2 * tc_align(m * m * sizeof(float));  // residuals of the dithered slice
    return t;
}

int tc_products(const TcState *t) { return t ? t->products : 0; }

// Real block form [[Wr, Wi], [-Wi, Wr]] of W (d = 0) or conj W (d = 1), entry (row, col).
static double dft_block(int n, int d, size_t row, size_t col) {
    const size_t j = row % n, k = col % n;
    const double ang = 2.0 * 3.141592653589793238462643383279502884 * (double)((j * k) % n) / (double)n;
    const double wr = cos(ang), wi = (d == 0 ? -1.0 : 1.0) * sin(ang);
    const int q = (int)(row / n) * 2 + (int)(col / n);
    return q == 0 || q == 3 ? wr : (q == 1 ? wi : -wi);
}

TcState *tc_create(int n, int64_t batch, int products, void *ws, size_t ws_bytes, cudaStream_t s, const char **why) {
    *why = nullptr;
    if (!tc_products_ok(n, products)) {
        *why = "unsupported number of products for this n";
        return nullptr;
    }
    if (!ws || ((uintptr_t)ws & 255) || ws_bytes < tc_workspace_bytes(n, batch, products)) {
        *why = "tensor-core workspace too small or not 256-byte aligned";
        return nullptr;
    }
    TcState *t = new TcState();
    t->n = n;
    t->batch = batch;
    t->products = products;
    t->l = log2i(n);
    const size_t m = 2 * (size_t)n, rows = (size_t)batch * (size_t)n;
    const size_t wseg = (size_t)w_segments(products);
    char *p = (char *)ws;
    const size_t wp = (size_t)tc_pitch((int)wseg, m);
    t->w[0] = (__half *)p;
    p += tc_align(wp * m * sizeof(__half));
    t->w[1] = (__half *)p;
    p += tc_align(wp * m * sizeof(__half));
    t->a = (__half *)p;
    p += tc_align(rows * (size_t)tc_pitch(a_segments(products), m) * sizeof(__half));
    t->c = (float *)p;
    p += tc_align(rows * m * sizeof(float));
    t->maxbits = (unsigned *)p;
    p += tc_align(2 * (size_t)batch * sizeof(unsigned));
    t->e = (int *)p;
    p += tc_align((size_t)batch * sizeof(int));
    t->err = (unsigned *)p;
    p += tc_align(2 * sizeof(unsigned));
    t->e8 = (int8_t *)p;
    p += tc_align(rows * (m / 16));
    if (products != TC_FIXED) {
        t->wres[0] = (float *)p;
        p += tc_align(m * m * sizeof(float));
        t->wres[1] = (float *)p;
        p += tc_align(m * m * sizeof(float));
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    t->grid = (sms > 0 ? sms : 152) * 8;
    if (cudaMemsetAsync(t->err, 0, 2 * sizeof(unsigned), s) != cudaSuccess) {
        *why = "clearing the GEMM time-out word failed";
        delete t;
        return nullptr;
    }

    // W and conj W from FP64, split on the host
    std::vector<__half> host(wp * m, __float2half(0.f));
    std::vector<float> res(products != TC_FIXED ? m * m : 0);
    for (int d = 0; d < 2; ++d) {
        for (size_t row = 0; row < m; ++row)
            for (size_t col = 0; col < m; ++col) {
                const double v = dft_block(n, d, row, col);
                if (products != TC_FIXED) {
                    // W_hi = rint(2^10 v), W_lo = rint((2^10 v - W_hi) 2^11) and, for 5
                    // products, W_lo2 = rint(next residual 2^11): integers in [-1024, 1024]
                    double r = v * 1024.0;
                    for (int k = 0; k < wseg; ++k) {
                        if (k == (int)wseg - 1) res[col * m + row] = (float)r;
                        const double w = std::nearbyint(r);
                        host[col * wp + k * m + row] = __double2half(w);
                        r = (r - w) * 2048.0;
                    }
                } else {
                    // integer slices of 2^7 v: w0 + 2^-7 w1 + 2^-14 w2 + 2^-21 w3
                    double r = v * 128.0, w[4];
                    for (int k = 0; k < 4; ++k) {
                        w[k] = std::nearbyint(r);
                        r = (r - w[k]) * 128.0;
                    }
                    // segments w0 | w1 | w2 | w3 along K; level L pairs a_i with w_(L-i)
                    for (int k = 0; k < 4; ++k) host[col * wp + k * m + row] = __double2half(w[k]);
                }
            }
        if (cudaMemcpyAsync(t->w[d], host.data(), host.size() * sizeof(__half), cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            (products != TC_FIXED &&
             cudaMemcpyAsync(t->wres[d], res.data(), res.size() * sizeof(float), cudaMemcpyHostToDevice, s) !=
                 cudaSuccess) ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            *why = "copy of the DFT matrices failed";
            delete t;
            return nullptr;
        }
    }
    return t;
}

void tc_destroy(TcState *t) { delete t; }

static SplitOut split_out(TcState *t) {
    SplitOut o;
    o.a = t->a;
    o.kp = tc_pitch(a_segments(t->products), 2 * (size_t)t->n);
    o.n = t->n;
    o.e = t->e8;
    o.eld = 2 * t->n / 16;
    return o;
}

// Fixed form: the max pass over the split's input, and the scale state the
// split reads (the current max buffer) and prepares (the other one).
static cudaError_t fixed_prepare(TcState *t, const float *in, bool interleaved, int e_add, bool from_psi,
                                 cudaStream_t s, FixedScale *fs, int64_t *launches) {
    if (from_psi) {
        cudaError_t e = cudaMemsetAsync(t->maxbits, 0, 2 * (size_t)t->batch * sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        t->cur = 0;
    }
    unsigned *mcur = t->maxbits + (size_t)t->cur * t->batch;
    const int64_t pairs = (int64_t)t->n * t->n / 2;
    int per = (int)((pairs + TC_THREADS - 1) / TC_THREADS);
    const int cap = (int)((t->grid + t->batch - 1) / t->batch) * 2;
    if (per > cap) per = cap;
    if (per < 1) per = 1;
    const dim3 grid((unsigned)per, (unsigned)t->batch);
    if (interleaved) k_tc_absmax<true><<<grid, TC_THREADS, 0, s>>>(in, t->n, mcur);
    else k_tc_absmax<false><<<grid, TC_THREADS, 0, s>>>(in, t->n, mcur);
    ++*launches;
    fs->maxin = mcur;
    fs->maxclr = t->maxbits + (size_t)(t->cur ^ 1) * t->batch;
    fs->e = t->e;
    fs->e_add = e_add;
    fs->from_psi = from_psi ? 1 : 0;
    t->cur ^= 1;
    return cudaGetLastError();
}

cudaError_t tc_split_potential(TcState *t, const TcPhaseArgs &a, bool from_psi, cudaStream_t s, int64_t *launches) {
    const int64_t rows = t->batch * t->n;
    const SplitOut o = split_out(t);
    FixedScale fs{};
    if (t->products == TC_FIXED) {
        cudaError_t e = fixed_prepare(t, from_psi ? reinterpret_cast<const float *>(a.psi) : t->c, from_psi, 0,
                                      from_psi, s, &fs, launches);
        if (e != cudaSuccess) return e;
        if (from_psi) k_tc_split<TC_FIXED, 0><<<t->grid, TC_THREADS, 0, s>>>(o, t->c, a, rows, 1.f, fs);
        else k_tc_split<TC_FIXED, 1><<<t->grid, TC_THREADS, 0, s>>>(o, t->c, a, rows, 1.f, fs);
    } else {
        // unnormalised transforms and the kinetic table's 1/n^2: psi's scale throughout
        if (from_psi) k_tc_split<TC_BFP, 0><<<t->grid, TC_THREADS, 0, s>>>(o, t->c, a, rows, 1.f, fs);
        else k_tc_split<TC_BFP, 1><<<t->grid, TC_THREADS, 0, s>>>(o, t->c, a, rows, 1.f, fs);
    }
    ++*launches;
    return cudaGetLastError();
}

cudaError_t tc_split_kinetic(TcState *t, const TcPhaseArgs &a, cudaStream_t s, int64_t *launches) {
    const int64_t rows = t->batch * t->n;
    const SplitOut o = split_out(t);
    FixedScale fs{};
    if (t->products == TC_FIXED) {
        // the axis-0 kinetic factors carry the inverse transform's 1 / n^2; the
        // fixed form tracks its scale in the exponent, so it is taken out here
        const float scale = ldexpf(1.f, 2 * t->l);
        cudaError_t e = fixed_prepare(t, t->c, false, -2 * t->l, false, s, &fs, launches);
        if (e != cudaSuccess) return e;
        k_tc_split<TC_FIXED, 2><<<t->grid, TC_THREADS, 0, s>>>(o, t->c, a, rows, scale, fs);
    } else {
        k_tc_split<TC_BFP, 2><<<t->grid, TC_THREADS, 0, s>>>(o, t->c, a, rows, 1.f, fs);
    }
    ++*launches;
    return cudaGetLastError();
}

cudaError_t tc_split_transpose(TcState *t, cudaStream_t s, int64_t *launches) {
    const dim3 grid((unsigned)(t->n / TC_TC), (unsigned)(t->n / TC_TR), (unsigned)t->batch), block(32, 8);
    const SplitOut o = split_out(t);
    FixedScale fs{};
    if (t->products == TC_FIXED) {
        cudaError_t e = fixed_prepare(t, t->c, false, 0, false, s, &fs, launches);
        if (e != cudaSuccess) return e;
        k_tc_split_t<TC_FIXED><<<grid, block, 0, s>>>(o, t->c, fs);
    } else {
        k_tc_split_t<TC_BFP><<<grid, block, 0, s>>>(o, t->c, fs);
    }
    ++*launches;
    return cudaGetLastError();
}

// One axis transform: C[rows][2n] = products of the split rows with the block
// DFT matrix.  Block-scaled forms: every K = 16 MMA its own exact group, scaled
// by the row's block exponent.  Fixed form: level L = segments (a_i, w_(L-i)),
// i = 0..L, one exact group scaled by 2^-7L.
cudaError_t tc_gemm(TcState *t, bool inverse, cudaStream_t s, int64_t *launches) {
    const int m = 2 * t->n;
    const int kb = m / 64;
    const __half *w = t->w[inverse ? 1 : 0];
    const int64_t rows = t->batch * t->n;
    UgSeg seg[UG_MAX_SEG];
    int nseg = 0;
    float alpha = 1.f;
    int64_t lda, ldb;
    if (t->products == TC_FIXED) {
        lda = tc_pitch(4, m);
        ldb = tc_pitch(4, m);
        for (int lev = 0; lev < 4; ++lev)
            for (int i = 0; i <= lev; ++i)
                seg[nseg++] = UgSeg{i * m, (lev - i) * m, kb, ldexpf(1.f, -7 * lev), i == 0 ? (int)UG_OPEN : (int)UG_CONTINUE};
    } else {
        // a W_hi (2^-20), a W_lo and c W_hi (2^-31), each times the row's block
        // exponent; 5 products add a W_lo2 and c W_lo (2^-42), smallest last
        lda = tc_pitch(2, m);
        ldb = tc_pitch(w_segments(t->products), m);
        seg[nseg++] = UgSeg{0, 0, kb, ldexpf(1.f, -20), (int)UG_EACH_MMA_BEXP, 0};
        seg[nseg++] = UgSeg{0, m, kb, ldexpf(1.f, -31), (int)UG_EACH_MMA_BEXP, 0};
        seg[nseg++] = UgSeg{m, 0, kb, ldexpf(1.f, -31), (int)UG_EACH_MMA_BEXP, 0};
        if (t->products == 5) {
            seg[nseg++] = UgSeg{0, 2 * m, kb, ldexpf(1.f, -42), (int)UG_EACH_MMA_BEXP, 0};
            seg[nseg++] = UgSeg{m, m, kb, ldexpf(1.f, -42), (int)UG_EACH_MMA_BEXP, 0};
        }
    }
    cudaError_t e = umma_gemm(t->a, lda, w, ldb, t->c, m, rows, m, seg, nseg, alpha, 0.f, tc_bn(t->n), t->err, s,
                              t->e8, m / 16);
    ++*launches;
    return e;
}

// Dithered rounding of the last DFT-matrix slice (block-scaled forms).  The
// DFT matrix has only n distinct entries and enters every transform of every
// step, so a fixed rounding of it is one structured perturbation repeated
// thousands of times: its effect on the norm adds up coherently (a steady loss
// of ~2e-4 over 1000 steps with the 21-bit matrix).  Rounding the last slice
// per step as floor(r + u), with u a fresh pseudo-random offset in [0, 1) for
// the step (the same for every entry), makes the slice exact on average over
// steps: the rounding errors of different steps are independent and add as a
// random walk.  r is the slice before rounding, r in [-1024, 1024], so every
// slice stays an integer in [-1024, 1024] and every MMA partial stays exact.
__global__ void k_tc_w_dither(__half *w0, __half *w1, const float *res0, const float *res1, int64_t m, int64_t wp,
                              int seg, float u0, float u1) {
    const int d = blockIdx.y;
    __half *w = d == 0 ? w0 : w1;
    const float *res = d == 0 ? res0 : res1;
    const float u = d == 0 ? u0 : u1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m * m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t col = i / m, row = i - col * m;
        w[col * wp + seg * m + row] = __float2half_rn(floorf(res[i] + u));
    }
}

cudaError_t tc_dither_w(TcState *t, uint32_t dither, cudaStream_t s, int64_t *launches) {
    if (t->products == TC_FIXED) return cudaSuccess;
    const int64_t m = 2 * (int64_t)t->n;
    const int seg = w_segments(t->products) - 1;
    // offsets of the forward and inverse matrices: 24 bits of the step's
    // dither, the inverse half a unit apart
    const uint32_t q = dither >> 8;
    const float u0 = (float)q * 5.9604644775390625e-08f;                         // 2^-24
    const float u1 = (float)((q + 0x800000u) & 0xFFFFFFu) * 5.9604644775390625e-08f;
    k_tc_w_dither<<<dim3((unsigned)t->grid, 2), TC_THREADS, 0, s>>>(t->w[0], t->w[1], t->wres[0], t->wres[1], m,
                                                                    tc_pitch(w_segments(t->products), (size_t)m), seg,
                                                                    u0, u1);
    ++*launches;
    return cudaGetLastError();
}

int tc_timed_out(TcState *t, cudaStream_t s) {
    unsigned v = 0;
    if (cudaMemcpyAsync(&v, t->err, sizeof v, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return -1;
    return v ? 1 : 0;
}

cudaError_t tc_finish(TcState *t, const TcPhaseArgs &a, bool phase, cudaStream_t s, int64_t *launches) {
    const int64_t rows = t->batch * t->n;
    k_tc_finish<<<t->grid, TC_THREADS, 0, s>>>(t->c, a, t->n, rows, 1.f,
                                               t->products == TC_FIXED ? t->e : nullptr, phase ? 1 : 0);
    ++*launches;
    return cudaGetLastError();
}

}  // namespace qhd
