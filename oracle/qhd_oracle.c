/*
 * qhd_oracle.c -- plain FP64 CPU oracle for the QHD split-operator simulation.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference for
 * the CUDA path.  Only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark may load it.  It shares no code, header, table or helper
 * with the product library, and the product library never calls it.
 *
 * What it computes (paper: Leng, Hickman, Li, Wu, "Quantum Hamiltonian
 * Descent", arXiv 2303.01471):
 *   - the QHD Hamiltonian H(t) = e^{phi_t}(-1/2 Lap) + e^{chi_t} f(x)
 *     (Sec. "A genuine quantum gradient descent", Eq. (main1); Eq. (qhd_operator));
 *   - on the regular periodic mesh of the box [a,b]^d with N = 2^q points per
 *     axis, x_j in {a, a+dx, ..., b-dx}, state normalised in l2
 *     (Sec. "Implementing QHD using product formulae", Eq. (wave-rep));
 *   - the Nesterov-type damping e^{phi}=2/(s+t^3), e^{chi}=2t^3 of the
 *     paper's simulations (Eq. (nonconvex_QHD_h)), generalised here to
 *     e^{phi}=c_phi/(eps+t^3), e^{chi}=c_chi t^3, plus a piecewise-linear
 *     tabulated (phi, chi), plus the power family of the three-parameter
 *     form (Eq. (qhd_operator_convex)) under the ideal scaling condition
 *     (Eq. (ideal_scaling)) met with equality: alpha = log p - log t,
 *     beta = p log t + log C, gamma = p log t give e^{phi} = e^{alpha-gamma}
 *     = p t^{-(p+1)} and e^{chi} = e^{alpha+beta+gamma} = p C t^{2p-1};
 *     here e^{phi} = c_phi/(eps + |t|^{p+1}), e^{chi} = c_chi |t|^{2p-1}
 *     (p = 2 is the Nesterov kind);
 *   - time stepping by the pseudo-spectral product formula, Eqs. (prod_qhd)
 *     and (prod_qhd_fft), Algorithm 1: the potential factor is diagonal in
 *     position, the kinetic factor is diagonal in Fourier space with the
 *     eigenvalues |k|^2/2, k = 2 pi m / L.  The symmetric (Strang) form
 *     P(dt/2) K(dt) P(dt/2) is used, with both coefficients sampled at the
 *     step midpoint; the half potential factors are NOT merged here;
 *   - observables: |psi|^2, the loss E[f] (Eq. (expect_O)) and the success
 *     probability, the mass within Euclidean distance r of the grid
 *     minimiser (Fig. 2 caption).
 *
 * The FFT is the textbook recursive radix-2 Cooley-Tukey, twiddles from libm
 * cos/sin of FP64 angles.  Phase arguments are formed in FP64 and reduced
 * modulo 2 pi before cos/sin.  Sums use fixed-order pairwise summation so the
 * results do not depend on the thread count.  OpenMP (when available) only
 * splits independent FFT lines and independent pointwise work.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (see build.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846264338327950288

typedef struct {
    double re, im;
} c128;

/* ---------------------------------------------------------------- schedule */

/* Schedule kinds, mirroring the two families the oracle supports. */
enum { ORACLE_SCHED_NESTEROV = 0, ORACLE_SCHED_TABLE = 1, ORACLE_SCHED_POWER = 2 };

typedef struct {
    int kind;
    double c_phi, eps, c_chi;          /* NESTEROV: a=c_phi/(eps+t^3), b=c_chi t^3 */
    const double *ts, *phis, *chis;    /* TABLE: samples of phi(t), chi(t) */
    int64_t ns;
    double power;                      /* POWER: a=c_phi/(eps+|t|^{p+1}), b=c_chi |t|^{2p-1} */
} sched_t;

/* Piecewise-linear interpolation of samples (ts increasing), constant beyond
 * the ends. */
static double interp(const double *ts, const double *vs, int64_t ns, double t)
{
    if (t <= ts[0]) return vs[0];
    if (t >= ts[ns - 1]) return vs[ns - 1];
    int64_t lo = 0, hi = ns - 1;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (ts[mid] <= t) lo = mid; else hi = mid;
    }
    double w = (t - ts[lo]) / (ts[hi] - ts[lo]);
    return vs[lo] + w * (vs[hi] - vs[lo]);
}

/* a(t) = e^{phi_t} (kinetic weight), b(t) = e^{chi_t} (potential weight). */
static void sched_eval(const sched_t *s, double t, double *a, double *b)
{
    if (s->kind == ORACLE_SCHED_NESTEROV) {
        double t3 = t * t * t;
        *a = s->c_phi / (s->eps + t3);
        *b = s->c_chi * t3;
    } else if (s->kind == ORACLE_SCHED_POWER) {
        double at = fabs(t);
        *a = s->c_phi / (s->eps + pow(at, s->power + 1.0));
        *b = s->c_chi * pow(at, 2.0 * s->power - 1.0);
    } else {
        *a = exp(interp(s->ts, s->phis, s->ns, t));
        *b = exp(interp(s->ts, s->chis, s->ns, t));
    }
}

/* --------------------------------------------------------------------- FFT */

/* Recursive radix-2 decimation-in-time DFT of n (power of two) samples read
 * from x with the given stride: out[k] = sum_j x[j] exp(sign*2 pi i j k / n). */
static void fft_rec(const c128 *x, int64_t stride, int64_t n, c128 *out, int sign)
{
    if (n == 1) {
        out[0] = x[0];
        return;
    }
    int64_t h = n / 2;
    fft_rec(x, 2 * stride, h, out, sign);               /* even samples */
    fft_rec(x + stride, 2 * stride, h, out + h, sign);  /* odd samples  */
    for (int64_t k = 0; k < h; ++k) {
        double ang = (double)sign * 2.0 * ORACLE_PI * (double)k / (double)n;
        double wr = cos(ang), wi = sin(ang);
        c128 e = out[k], o = out[k + h];
        double tr = wr * o.re - wi * o.im;
        double ti = wr * o.im + wi * o.re;
        out[k].re = e.re + tr;
        out[k].im = e.im + ti;
        out[k + h].re = e.re - tr;
        out[k + h].im = e.im - ti;
    }
}

/* DFT along one axis of a row-major array with dims n[0..ndim-1]
 * (last axis fastest).  Unnormalised in both directions. */
static void fft_axis(c128 *data, int ndim, const int64_t *n, int axis, int sign)
{
    int64_t len = n[axis];
    int64_t inner = 1, outer = 1;
    for (int d = axis + 1; d < ndim; ++d) inner *= n[d];
    for (int d = 0; d < axis; ++d) outer *= n[d];
    int64_t lines = outer * inner;
#pragma omp parallel
    {
        c128 *tmp = (c128 *)malloc(sizeof(c128) * (size_t)len * 2);
        c128 *res = tmp + len;
#pragma omp for schedule(static)
        for (int64_t l = 0; l < lines; ++l) {
            int64_t o = l / inner, i = l % inner;
            c128 *base = data + o * len * inner + i;
            for (int64_t j = 0; j < len; ++j) tmp[j] = base[j * inner];
            fft_rec(tmp, 1, len, res, sign);
            for (int64_t j = 0; j < len; ++j) base[j * inner] = res[j];
        }
        free(tmp);
    }
}

/* Multi-dimensional DFT over all axes.  sign=-1 forward (unnormalised),
 * sign=+1 inverse including the 1/G factor. */
static void fft_nd(c128 *data, int ndim, const int64_t *n, int sign)
{
    for (int ax = 0; ax < ndim; ++ax) fft_axis(data, ndim, n, ax, sign);
    if (sign > 0) {
        int64_t g = 1;
        for (int d = 0; d < ndim; ++d) g *= n[d];
        double inv = 1.0 / (double)g;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < g; ++i) {
            data[i].re *= inv;
            data[i].im *= inv;
        }
    }
}

/* Exported for the FFT pins: in-place DFT of a (re,im)-interleaved array. */
void oracle_fft(int ndim, const int64_t *n, double *data, int sign)
{
    fft_nd((c128 *)data, ndim, n, sign);
}

/* ------------------------------------------------------------ Strang step */

/* Multiply by exp(-i*ang) with ang reduced modulo 2 pi in FP64 first. */
static void apply_phase(c128 *z, double ang)
{
    double r = fmod(ang, 2.0 * ORACLE_PI);
    double c = cos(r), s = sin(r);
    double re = z->re * c + z->im * s;
    double im = z->im * c - z->re * s;
    z->re = re;
    z->im = im;
}

/* psi <- exp(-i * h * b * f(x)) psi, pointwise in position space. */
static void potential_factor(c128 *psi, const double *f, int64_t g, double h, double b)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < g; ++i) apply_phase(&psi[i], h * b * f[i]);
}

/* psi_hat <- exp(-i * dt * a * |k|^2 / 2) psi_hat, k_d = 2 pi m_d / L_d with the
 * signed frequency number m_d in [-N_d/2, N_d/2).
 * kinetic = 1 replaces -Lap by the central second difference of Eq. (discretize-pde),
 * (2 psi_j - psi_{j+1} - psi_{j-1}) / h_d^2 with h_d = L_d / N_d, on the periodic mesh:
 * its eigenvalue for the Fourier mode m_d is (4 / h_d^2) sin^2(pi m_d / N_d). */
static void kinetic_factor(c128 *psi, int ndim, const int64_t *n, const double *len,
                           double dt, double a, int kinetic)
{
    int64_t g = 1;
    for (int d = 0; d < ndim; ++d) g *= n[d];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < g; ++i) {
        int64_t rem = i;
        double k2 = 0.0;
        for (int d = ndim - 1; d >= 0; --d) {
            int64_t idx = rem % n[d];
            rem /= n[d];
            int64_t m = idx < n[d] / 2 ? idx : idx - n[d];
            if (kinetic == 1) {
                double h = len[d] / (double)n[d];
                double sn = sin(ORACLE_PI * (double)m / (double)n[d]);
                k2 += 4.0 * sn * sn / (h * h);
            } else {
                double k = 2.0 * ORACLE_PI * (double)m / len[d];
                k2 += k * k;
            }
        }
        apply_phase(&psi[i], dt * a * k2 / 2.0);
    }
}

/*
 * Evolve psi (interleaved re,im; G complex values) by nsteps Strang steps of
 * size dt starting at time t0.  Step j uses a, b at t0 + (j + 1/2) dt and is
 * P(dt/2) . IFFT . K(dt) . FFT . P(dt/2).  dt may be negative (time reversal).
 * Returns 0 on success, nonzero on bad arguments.
 */
int oracle_evolve(int ndim, const int64_t *n, const double *lo, const double *hi,
                  const double *f, double *psi_io, double t0, double dt, int64_t nsteps,
                  int sched_kind, double c_phi, double eps, double c_chi,
                  const double *ts, const double *phis, const double *chis, int64_t ns,
                  double power, int kinetic)
{
    if (ndim < 1 || ndim > 3 || nsteps < 0) return 1;
    sched_t s = {sched_kind, c_phi, eps, c_chi, ts, phis, chis, ns, power};
    if (sched_kind == ORACLE_SCHED_TABLE && (ns < 1 || !ts || !phis || !chis)) return 1;
    double len[3];
    int64_t g = 1;
    for (int d = 0; d < ndim; ++d) {
        len[d] = hi[d] - lo[d];
        g *= n[d];
    }
    c128 *psi = (c128 *)psi_io;
    for (int64_t j = 0; j < nsteps; ++j) {
        double t = t0 + ((double)j + 0.5) * dt;
        double a, b;
        sched_eval(&s, t, &a, &b);
        potential_factor(psi, f, g, dt / 2.0, b);
        fft_nd(psi, ndim, n, -1);
        kinetic_factor(psi, ndim, n, len, dt, a, kinetic);
        fft_nd(psi, ndim, n, +1);
        potential_factor(psi, f, g, dt / 2.0, b);
    }
    return 0;
}

/* psi_out = H psi_in with H = a (-Lap/2) + b f (Eq. (qhd_operator)), the kinetic
 * part exact on the mesh's Fourier modes (or the central difference of
 * Eq. (discretize-pde) for kinetic = 1): FFT, multiply by a |k|^2 / 2, inverse
 * FFT (which carries the 1/G), plus the pointwise b f psi_in. */
int oracle_apply_h(int ndim, const int64_t *n, const double *lo, const double *hi,
                   const double *f, const double *psi_in, double *psi_out, double a, double b, int kinetic)
{
    if (ndim < 1 || ndim > 3) return 1;
    double len[3];
    int64_t g = 1;
    for (int d = 0; d < ndim; ++d) {
        len[d] = hi[d] - lo[d];
        g *= n[d];
    }
    const c128 *in = (const c128 *)psi_in;
    c128 *out = (c128 *)psi_out;
    for (int64_t i = 0; i < g; ++i) out[i] = in[i];
    fft_nd(out, ndim, n, -1);
    for (int64_t i = 0; i < g; ++i) {
        int64_t rem = i;
        double k2 = 0.0;
        for (int d = ndim - 1; d >= 0; --d) {
            int64_t idx = rem % n[d];
            rem /= n[d];
            int64_t m = idx < n[d] / 2 ? idx : idx - n[d];
            if (kinetic == 1) {
                double h = len[d] / (double)n[d];
                double sn = sin(ORACLE_PI * (double)m / (double)n[d]);
                k2 += 4.0 * sn * sn / (h * h);
            } else {
                double k = 2.0 * ORACLE_PI * (double)m / len[d];
                k2 += k * k;
            }
        }
        double w = a * k2 / 2.0;  /* the inverse transform carries the 1/G */
        out[i].re *= w;
        out[i].im *= w;
    }
    fft_nd(out, ndim, n, +1);
    for (int64_t i = 0; i < g; ++i) {
        out[i].re += b * f[i] * in[i].re;
        out[i].im += b * f[i] * in[i].im;
    }
    return 0;
}

/* Lie-Trotter variant of the paper as printed (Eq. (prod_qhd)): coefficients
 * at the left end point t_j = t0 + j dt, psi <- IFFT K(dt) FFT P(dt) psi. */
int oracle_evolve_trotter(int ndim, const int64_t *n, const double *lo, const double *hi,
                          const double *f, double *psi_io, double t0, double dt,
                          int64_t nsteps, double c_phi, double eps, double c_chi, int kinetic)
{
    if (ndim < 1 || ndim > 3 || nsteps < 0) return 1;
    sched_t s = {ORACLE_SCHED_NESTEROV, c_phi, eps, c_chi, 0, 0, 0, 0, 0.0};
    double len[3];
    int64_t g = 1;
    for (int d = 0; d < ndim; ++d) {
        len[d] = hi[d] - lo[d];
        g *= n[d];
    }
    c128 *psi = (c128 *)psi_io;
    for (int64_t j = 0; j < nsteps; ++j) {
        double t = t0 + (double)j * dt;
        double a, b;
        sched_eval(&s, t, &a, &b);
        potential_factor(psi, f, g, dt, b);
        fft_nd(psi, ndim, n, -1);
        kinetic_factor(psi, ndim, n, len, dt, a, kinetic);
        fft_nd(psi, ndim, n, +1);
    }
    return 0;
}

/* Exported schedule evaluation (used by pins that integrate closed forms). */
void oracle_schedule(int sched_kind, double c_phi, double eps, double c_chi,
                     const double *ts, const double *phis, const double *chis, int64_t ns,
                     double power, double t, double *a_out, double *b_out)
{
    sched_t s = {sched_kind, c_phi, eps, c_chi, ts, phis, chis, ns, power};
    sched_eval(&s, t, a_out, b_out);
}

/* ------------------------------------------------------------- observables */

/* Fixed-order pairwise sum. */
static double pairwise(const double *v, int64_t n)
{
    if (n <= 16) {
        double s = 0.0;
        for (int64_t i = 0; i < n; ++i) s += v[i];
        return s;
    }
    int64_t h = n / 2;
    return pairwise(v, h) + pairwise(v + h, n - h);
}

/*
 * Observables of one instance.  out[0]=norm=sum p, out[1]=E[f]=sum p f,
 * out[2]=P_succ=sum of p over points with |x - x*|_2 < radius (Euclidean on
 * the box, not periodic), out[3..5]=x* (grid minimiser of f, lowest flat index
 * on ties; unused axes 0).  prob (optional) receives p = |psi|^2.
 */
int oracle_observables(int ndim, const int64_t *n, const double *lo, const double *hi,
                       const double *f, const double *psi_io, double radius,
                       double *out, double *prob)
{
    if (ndim < 1 || ndim > 3) return 1;
    int64_t g = 1;
    for (int d = 0; d < ndim; ++d) g *= n[d];
    const c128 *psi = (const c128 *)psi_io;
    int64_t amin = 0;
    for (int64_t i = 1; i < g; ++i)
        if (f[i] < f[amin]) amin = i;
    double xs[3] = {0.0, 0.0, 0.0};
    {
        int64_t rem = amin;
        for (int d = ndim - 1; d >= 0; --d) {
            int64_t idx = rem % n[d];
            rem /= n[d];
            xs[d] = lo[d] + (double)idx * (hi[d] - lo[d]) / (double)n[d];
        }
    }
    double *p = (double *)malloc(sizeof(double) * (size_t)g);
    double *pf = (double *)malloc(sizeof(double) * (size_t)g);
    double *ps = (double *)malloc(sizeof(double) * (size_t)g);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < g; ++i) {
        double pi_ = psi[i].re * psi[i].re + psi[i].im * psi[i].im;
        p[i] = pi_;
        pf[i] = pi_ * f[i];
        int64_t rem = i;
        double r2 = 0.0;
        for (int d = ndim - 1; d >= 0; --d) {
            int64_t idx = rem % n[d];
            rem /= n[d];
            double x = lo[d] + (double)idx * (hi[d] - lo[d]) / (double)n[d];
            r2 += (x - xs[d]) * (x - xs[d]);
        }
        ps[i] = sqrt(r2) < radius ? pi_ : 0.0;
    }
    out[0] = pairwise(p, g);
    out[1] = pairwise(pf, g);
    out[2] = pairwise(ps, g);
    out[3] = xs[0];
    out[4] = xs[1];
    out[5] = xs[2];
    if (prob) memcpy(prob, p, sizeof(double) * (size_t)g);
    free(p);
    free(pf);
    free(ps);
    return 0;
}

/* Uniform superposition psi = G^{-1/2} (Eq. (prod_qhd): uniform initial state). */
void oracle_uniform(int64_t g, double *psi_io)
{
    double v = 1.0 / sqrt((double)g);
    for (int64_t i = 0; i < g; ++i) {
        psi_io[2 * i] = v;
        psi_io[2 * i + 1] = 0.0;
    }
}

/* Thread control for timing runs. */
void oracle_set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
