// qhd_device.cuh -- device building blocks of the split-operator step: complex
// arithmetic, in-register DFTs, the two-stage shared-memory line FFT and the
// fixed-point phase helpers.
//
// The kinetic factor of the pseudo-spectral product formula is diagonal in the
// Fourier basis (Eq. (prod_qhd_fft)), so every step needs a forward and an
// inverse DFT along each axis.  A line of N = R1 * R2 points is transformed by
// T = N / E threads that each hold E points in registers: stage 1 is an
// R1-point DFT done entirely in registers, a padded shared-memory exchange,
// then twiddles and an R2-point DFT in registers (a two-stage Stockham
// factorisation, so input and output are both in natural order).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qhd {

// ------------------------------------------------------------------ complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// cos(2 pi k / 64), k = 0..16, correctly rounded to double.
__host__ __device__ constexpr double cos64_q(int k) {
    constexpr double q[17] = {1.0,
                              0.9951847266721968862448,
                              0.9807852804032304491262,
                              0.9569403357322088649358,
                              0.9238795325112867561282,
                              0.8819212643483550297128,
                              0.8314696123025452370788,
                              0.7730104533627369608109,
                              0.7071067811865475244008,
                              0.6343932841636454982152,
                              0.5555702330196022247428,
                              0.4713967368259976485564,
                              0.3826834323650897717285,
                              0.2902846772544623676362,
                              0.1950903220161282678483,
                              0.0980171403295606019942,
                              0.0};
    return q[k];
}
__host__ __device__ constexpr double cos64(int k) {
    k &= 63;
    return k <= 16 ? cos64_q(k) : k <= 32 ? -cos64_q(32 - k) : k <= 48 ? -cos64_q(k - 32) : cos64_q(64 - k);
}
__host__ __device__ constexpr double sin64(int k) { return cos64(k - 16); }

// v * (hi + lo) for a twiddle carried as an FP32 pair: hi is the rounded
// value, lo the rounding residual.  The residual product is formed first and
// folded into the two FMAs of the leading product, so the twiddle enters with
// ~2^-48 relative precision and only the product itself is rounded.  A plain
// FP32 twiddle would perturb the transform by the same ~2^-24 every step, an
// error that accumulates coherently over thousands of steps.
// Both components add the cross term (v.y hi.y, v.x hi.y) to the residual
// products first and the diagonal term (v hi.x) last.  For a small rotation
// hi.x rounds to exactly 1, and its residual is the second-order shrink
// (cos - 1) v: added first to the exact diagonal term, it would be rounded away
// every time, a systematic norm gain (measured +1e-5 over 10^4 steps, from the
// kinetic factors of the low modes late in a run).
__device__ __forceinline__ float2 cmul_comp(float2 v, float2 hi, float2 lo) {
    const float cre = v.x * lo.x - v.y * lo.y;
    const float cim = v.x * lo.y + v.y * lo.x;
    return make_float2(fmaf(v.x, hi.x, fmaf(-v.y, hi.y, cre)), fmaf(v.y, hi.x, fmaf(v.x, hi.y, cim)));
}
// v * conj(hi + lo)
__device__ __forceinline__ float2 cmulc_comp(float2 v, float2 hi, float2 lo) {
    return cmul_comp(v, make_float2(hi.x, -hi.y), make_float2(lo.x, -lo.y));
}

// v * W_R^k with W_R = exp(-2 pi i / R) (forward) or its conjugate (inverse);
// k is a compile-time constant after unrolling, so the trivial cases fold and
// the hi/lo split of the constant is evaluated by the compiler.
template <int R, bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 v, int k) {
    static_assert(64 % R == 0, "in-register DFT sizes up to 64");
    if (k == 0) return v;
    if (4 * k == R) return mul_mi<INV>(v);
    if (2 * k == R) return make_float2(-v.x, -v.y);
    if (4 * k == 3 * R) return mul_mi<!INV>(v);
    const double cd = cos64(k * (64 / R));
    const double sd = INV ? sin64(k * (64 / R)) : -sin64(k * (64 / R));
    const float ch = (float)cd, sh = (float)sd;
    const float cl = (float)(cd - (double)ch), sl = (float)(sd - (double)sh);
    return cmul_comp(v, make_float2(ch, sh), make_float2(cl, sl));
}

// -------------------------------------------------------- in-register DFT
// In-place R-point DFT of v[0..R) (natural order in and out), unnormalised,
// exp(-2 pi i jk/R) forward, exp(+2 pi i jk/R) inverse.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2 *v) {
    if constexpr (R == 1) {
        return;
    } else if constexpr (R == 2) {
        float2 a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        float2 t2 = cadd(v[1], v[3]), t3 = mul_mi<INV>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    } else if constexpr (R == 8) {
        // radix-2 split: two 4-point DFTs of the even / odd samples
        float2 e[4], o[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            e[i] = v[2 * i];
            o[i] = v[2 * i + 1];
        }
        dft<4, INV>(e);
        dft<4, INV>(o);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float2 w = twiddle_const<8, INV>(o[k], k);
            v[k] = cadd(e[k], w);
            v[k + 4] = csub(e[k], w);
        }
    } else {
        // radix-4 split: four (R/4)-point DFTs of the samples r mod 4
        constexpr int Q = R / 4;
        float2 d[4][Q];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int i = 0; i < Q; ++i) d[r][i] = v[4 * i + r];
#pragma unroll
        for (int r = 0; r < 4; ++r) dft<Q, INV>(d[r]);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            float2 a0 = d[0][k];
            float2 a1 = twiddle_const<R, INV>(d[1][k], k);
            float2 a2 = twiddle_const<R, INV>(d[2][k], 2 * k);
            float2 a3 = twiddle_const<R, INV>(d[3][k], 3 * k);
            float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
            float2 t2 = cadd(a1, a3), t3 = mul_mi<INV>(csub(a1, a3));
            v[k] = cadd(t0, t2);
            v[k + 2 * Q] = csub(t0, t2);
            v[k + Q] = cadd(t1, t3);
            v[k + 3 * Q] = csub(t1, t3);
        }
    }
}

// ------------------------------------------------------------ line plans
// N = R1 * R2 points per line, E points per thread, T = N / E threads per line.
template <int N> struct Plan;
template <> struct Plan<2>    { static constexpr int R1 = 2,  R2 = 1,  E = 2;  };
template <> struct Plan<4>    { static constexpr int R1 = 4,  R2 = 1,  E = 4;  };
template <> struct Plan<8>    { static constexpr int R1 = 8,  R2 = 1,  E = 8;  };
template <> struct Plan<16>   { static constexpr int R1 = 16, R2 = 1,  E = 16; };
template <> struct Plan<32>   { static constexpr int R1 = 4,  R2 = 8,  E = 8;  };
template <> struct Plan<64>   { static constexpr int R1 = 8,  R2 = 8,  E = 8;  };
template <> struct Plan<128>  { static constexpr int R1 = 8,  R2 = 16, E = 16; };
template <> struct Plan<256>  { static constexpr int R1 = 16, R2 = 16, E = 16; };
template <> struct Plan<512>  { static constexpr int R1 = 16, R2 = 32, E = 32; };
template <> struct Plan<1024> { static constexpr int R1 = 32, R2 = 32, E = 32; };

template <int N> struct LineCfg {
    static constexpr int R1 = Plan<N>::R1, R2 = Plan<N>::R2, E = Plan<N>::E;
    static constexpr int T = N / E;
    static constexpr bool TWO_STAGE = R2 > 1;
    static constexpr int LOG_R1 = R1 == 2 ? 1 : R1 == 4 ? 2 : R1 == 8 ? 3 : R1 == 16 ? 4 : 5;
    static constexpr int PADDED = TWO_STAGE ? N + N / R1 : 0;  // padded line length (float2)
    static_assert(E % R1 == 0 && E % R2 == 0 && N == R1 * R2, "bad plan");
};

__host__ __device__ constexpr int pad_index(int i, int log_r1) { return i + (i >> log_r1); }

// Worst shared-memory bank conflict (8-byte words, evaluated per half warp)
// of the two exchange patterns for a line stride S.  lanes: lane l works on
// line (ROWMAJOR ? l / T : l % W) at thread index (ROWMAJOR ? l % T : l / W).
template <int N>
__host__ __device__ constexpr int conflicts(int S, bool rowmajor, int W) {
    using C = LineCfg<N>;
    int worst = 1;
    for (int pass = 0; pass < 2; ++pass) {
        const int R = pass == 0 ? C::R1 : C::R2;
        for (int q = 0; q < C::E / R; ++q)
            for (int m = 0; m < R; ++m)
                for (int h = 0; h < 2; ++h) {
                    int addr[16] = {};
                    for (int l = 0; l < 16; ++l) {
                        int lane = 16 * h + l;
                        int line = rowmajor ? (C::T >= 32 ? 0 : lane / C::T) : lane % W;
                        int t = rowmajor ? (C::T >= 32 ? lane : lane % C::T) : lane / W;
                        if (t >= C::T) t %= C::T;
                        int j = t + C::T * q;
                        int i = pass == 0 ? j * C::R1 + m : j + m * C::R1;
                        addr[l] = line * S + pad_index(i, C::LOG_R1);
                    }
                    int per_bank[16] = {};
                    for (int l = 0; l < 16; ++l) {
                        bool dup = false;
                        for (int l2 = 0; l2 < l; ++l2) dup = dup || addr[l2] == addr[l];
                        if (!dup) ++per_bank[addr[l] & 15];
                    }
                    for (int b = 0; b < 16; ++b) worst = per_bank[b] > worst ? per_bank[b] : worst;
                }
    }
    return worst;
}

// Best line stride (in float2) in [PADDED, PADDED + 16] for the lane layout.
template <int N>
__host__ __device__ constexpr int line_stride(bool rowmajor, int W) {
    using C = LineCfg<N>;
    if (!C::TWO_STAGE) return 0;
    int best = C::PADDED, best_c = 1 << 30;
    for (int S = C::PADDED; S <= C::PADDED + 16; ++S) {
        int c = conflicts<N>(S, rowmajor, W);
        if (c < best_c) {
            best_c = c;
            best = S;
        }
    }
    return best;
}

// ------------------------------------------------------------ line FFT
// x[e] holds line element t + T*e on entry and transform element t + T*e on
// exit.  sm: this line's shared buffer (stride-padded), tw2: stage-2 twiddles
// tw2[m*R1 + j] = exp(-2 pi i j m / N) as (hi.re, hi.im, lo.re, lo.im).  SYNC() orders the exchange among
// the T threads of the line (a warp barrier when a line lives in one warp).
template <int N, bool INV, typename Sync>
__device__ __forceinline__ void line_fft(float2 *x, float2 *sm, int t, const float4 *__restrict__ tw2,
                                         Sync sync) {
    using C = LineCfg<N>;
    if constexpr (!C::TWO_STAGE) {
        dft<N, INV>(x);
    } else {
        constexpr int R1 = C::R1, R2 = C::R2, E = C::E, T = C::T;
#pragma unroll
        for (int q = 0; q < E / R1; ++q) {
            float2 v[R1];
#pragma unroll
            for (int m = 0; m < R1; ++m) v[m] = x[q + m * (E / R1)];
            dft<R1, INV>(v);
            const int j = t + T * q;
#pragma unroll
            for (int m = 0; m < R1; ++m) sm[pad_index(j * R1 + m, C::LOG_R1)] = v[m];
        }
        sync();
#pragma unroll
        for (int q = 0; q < E / R2; ++q) {
            const int j = t + T * q;  // < R1
            float2 v[R2];
#pragma unroll
            for (int m = 0; m < R2; ++m) v[m] = sm[pad_index(j + m * R1, C::LOG_R1)];
#pragma unroll
            for (int m = 1; m < R2; ++m) {
                const float4 w = __ldg(&tw2[m * R1 + j]);
                const float2 hi = make_float2(w.x, w.y), lo = make_float2(w.z, w.w);
                v[m] = INV ? cmulc_comp(v[m], hi, lo) : cmul_comp(v[m], hi, lo);
            }
            dft<R2, INV>(v);
#pragma unroll
            for (int m = 0; m < R2; ++m) x[q + m * (E / R2)] = v[m];
        }
        sync();
    }
}

// ------------------------------------------------------ zero-mode split
// A state close to uniform keeps almost all of its norm in one Fourier value,
// the global zero mode.  Each FP32 rounding of that value inside the
// butterflies moves every point of its line coherently, so the norm takes a
// random walk of ~2^-24 per rounding while the state is near uniform (most of
// the walk of a run on a fine mesh).  The pass that applies the last forward
// transform, the kinetic factor and the inverse transform along one line
// therefore transforms the line through frequency 0 of the other axes as
// x - mu (mu = the line mean) and adds back K0 (N mu), K0 being the (exactly
// known) kinetic factor of the line's zero mode: the same linear map, with the
// large value kept out of the transforms.  Every other line's zero mode holds
// only the small share of the norm at its own frequency, so those lines are
// transformed as they are.  N is a power of two, so mu = sum / N and
// N mu = sum are exact.
//
// Sum of a line's points held E per thread by T consecutive lanes (T a power of
// two dividing 32; mask: those lanes): a local sum, then an xor butterfly over
// the T lanes; both partners add the same two values, so every lane ends with
// the same bits.
template <int E, int T>
__device__ __forceinline__ float2 line_sum_lanes(const float2 *x, unsigned mask = 0xffffffffu) {
    float2 s = x[0];
#pragma unroll
    for (int e = 1; e < E; ++e) s = cadd(s, x[e]);
#pragma unroll
    for (int m = 1; m < T; m <<= 1) {
        s.x += __shfl_xor_sync(mask, s.x, m);
        s.y += __shfl_xor_sync(mask, s.y, m);
    }
    return s;
}

// x[e] -= sum / N for the E points of this thread.
template <int N, int E>
__device__ __forceinline__ void sub_line_mean(float2 *x, float2 sum) {
    const float2 mu = make_float2(sum.x * (1.0f / N), sum.y * (1.0f / N));
#pragma unroll
    for (int e = 0; e < E; ++e) x[e] = csub(x[e], mu);
}

// ------------------------------------------------------- phase helpers
// Fixed-point turns: a phase angle 2 pi u / 2^32 is carried as u (uint32).
// hi32((c * v) mod 2^64) for a 64-bit fraction c (units of 2^-64 turns) and a
// 32-bit integer v: the fractional turns of c*v to 2^-32, exact up to the
// dropped low word (< 1 unit).
__device__ __forceinline__ uint32_t turns_mul(uint64_t c, uint32_t v) {
    const uint32_t lo = (uint32_t)c, hi = (uint32_t)(c >> 32);
    return __umulhi(lo, v) + hi * v;
}

// Potential phase factor exp(-2 pi i u / 2^32) applied to z.
// u = 2^24 k + 2^23 + r with k = floor(u / 2^24) and r in [-2^23, 2^23):
// exp(-2 pi i u/2^32) = T[k] (1 + eps), T[k] = exp(-2 pi i (k + 1/2)/256) an
// FP32 hi/lo pair from FP64, and eps = exp(-i delta) - 1, delta = 2 pi r / 2^32,
// |delta| <= pi/256, from its Taylor series (truncation < 3e-12).  eps is
// small, so it is formed in FP32 to ~1e-9 absolute and |T (1 + eps)| = 1 to
// ~1e-9; the whole factor enters as hi + lo of one compensated product, so
// only the product is rounded.  The table entries sit half a step off the
// axes: an entry with a component exactly +-1 would make that product exact
// and let the rounding of the sum drop eps's second-order shrink, (cos delta
// - 1) z, systematically at small delta, a norm gain of ~1e-9 per step.
// tab: the 256-entry table in shared memory.
constexpr int PHASE_TAB = 256;

__device__ __forceinline__ float2 apply_phase_tab(float2 z, uint32_t u, const float4 *tab) {
    const uint32_t k = u >> 24;
    const int32_t r = (int32_t)(u & 0xFFFFFFu) - (1 << 23);
    const float d = (float)r * 1.4629180792671596e-09f;  // 2 pi / 2^32
    const float d2 = d * d;
    const float cm1 = d2 * fmaf(d2, 1.0f / 24.0f, -0.5f);  // cos d - 1
    const float sn = d * fmaf(d2, -1.0f / 6.0f, 1.0f);     // sin d
    const float4 t = tab[k];
    // lo = T_lo + T_hi * eps, eps = (cm1, -sn)
    const float2 lo = make_float2(fmaf(t.x, cm1, fmaf(t.y, sn, t.z)), fmaf(t.y, cm1, fmaf(-t.x, sn, t.w)));
    return cmul_comp(z, make_float2(t.x, t.y), lo);
}

// Copy the phase table (global, PHASE_TAB float4) into shared memory.
__device__ __forceinline__ void load_phase_tab(float4 *dst, const float4 *__restrict__ src) {
    for (int i = threadIdx.x; i < PHASE_TAB; i += blockDim.x) dst[i] = __ldg(&src[i]);
}

// Per-step dither: a pseudo-random global phase (in turns, 2^-32 units) added
// to the potential phase of every point.  A global phase changes no
// observable, but it changes the FP32 values every later operation rounds, so
// the rounding errors of consecutive steps decorrelate.
__host__ __device__ inline uint32_t step_dither(uint64_t step) {
    uint64_t z = step + 0x9E3779B97F4A7C15ull;  // splitmix64 finaliser
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return (uint32_t)((z ^ (z >> 31)) >> 32);
}

}  // namespace qhd
