// qhd_prep.cuh -- per-step coefficients of the split-operator step, shared by
// the prep kernel and the persistent batched kernel.
//
// Strang form (Eq. (prod_qhd) made symmetric): a_j = e^{phi}, b_j = e^{chi} at
// the step midpoint t0 + (j + 1/2) dt; the two potential half phases of
// consecutive steps are merged, theta_j = dt (b_{j-1} + b_j) / 2 (theta_0 and
// theta_n are single halves).  First-order form (Eq. (prod_qhd) as printed):
// a_j, b_j at t0 + j dt, one phase dt b_j per step and none after the last.
// The kinetic phase of mode m along an axis of length L is dt a_j |k|^2 / 2
// with k = 2 pi m / L (Eq. (prod_qhd_fft)), or, for the finite-difference
// operator, dt a_j (4 / h^2) sin^2(pi m / N) / 2.
#pragma once
#include "qhd_device.cuh"
#include "qhd_kernels.h"
#include "qhd_sched.cuh"

namespace qhd {

// Potential coefficient pot[jl][b] (64-bit fraction of a turn per unit of the
// fixed-point potential) and, for steps jl < cnt, the per-axis multipliers of
// the kinetic phase: k_turns[d] (turns per unit m^2, 64-bit fraction) and
// k_fd[d] (turns per unit sin^2(pi m / N)).
__device__ inline void prep_coefficients(const PrepArgs &a, int64_t jl, int64_t b, uint64_t *k_turns,
                                         double *k_fd, bool write_pot = true) {
    const int64_t j = a.j0 + jl;  // global step index
    const SchedDev &sd = a.sched[b];
    const double PI = 3.141592653589793238462643383279502884;
    double a_m = 0, b_m = 0, a_p = 0, b_p = 0, theta = 0;
    if (a.split == 0) {
        if (j >= 1) {
            const double tm = __dadd_rn(a.t_start, __dmul_rn((double)(j - 1) + 0.5, a.dt));
            sched_eval_dev(sd, tm, &a_m, &b_m);
        }
        if (j < a.nsteps) {
            const double tp = __dadd_rn(a.t_start, __dmul_rn((double)j + 0.5, a.dt));
            sched_eval_dev(sd, tp, &a_p, &b_p);
        }
        theta = __dmul_rn(a.dt, __dadd_rn(j >= 1 ? b_m : 0.0, j < a.nsteps ? b_p : 0.0)) * 0.5;
    } else if (j < a.nsteps) {
        const double tj = __dadd_rn(a.t_start, __dmul_rn((double)j, a.dt));
        sched_eval_dev(sd, tj, &a_p, &b_p);
        theta = __dmul_rn(a.dt, b_p);
    }
    const int shift = a.inst[b].shift;
    // turns per unit of the fixed-point potential: theta / (2 pi) * 2^-shift
    const double y = ldexp(theta / (2.0 * PI), -shift);
    if (write_pot) a.pot[jl * a.batch + b] = frac_to_u64(y);
    for (int d = 0; d < a.ndim; ++d) {
        // turns per unit m^2: dt * a * |2 pi m / L|^2 / 2 / (2 pi) = dt a pi m^2 / L^2
        const double kap = __ddiv_rn(__dmul_rn(__dmul_rn(a.dt, a_p), PI), __dmul_rn(a.len[d], a.len[d]));
        k_turns[d] = frac_to_u64(kap);
        // finite difference: turns per unit sin^2(pi m/N) = dt * a * (4 / h^2) / 2 / (2 pi) = dt a N^2 / (pi L^2)
        const double nn = (double)a.n[d];
        k_fd[d] = __ddiv_rn(__dmul_rn(__dmul_rn(a.dt, a_p), nn * nn), __dmul_rn(PI, __dmul_rn(a.len[d], a.len[d])));
    }
}

// Kinetic table entry i (axis d, mode m) of step jl and table row b:
// exp(-2 pi i turns), times 1/G on axis 0, as an FP32 hi/lo pair.
__device__ inline void prep_kinetic_entry(const PrepArgs &a, int64_t jl, int64_t b, int i, const uint64_t *k_turns,
                                          const double *k_fd) {
    float4 *out = a.kt + (jl * a.kt_batch + b) * a.ksum;
    int d = 0;
    while (d + 1 < a.ndim && i >= a.koff[d + 1]) ++d;
    const int idx = i - a.koff[d];
    const int nd = a.n[d];
    const int m = idx < nd / 2 ? idx : idx - nd;
    uint32_t u;
    if (a.kinetic == 1) {
        const double sp = sinpi((double)m / (double)nd);
        u = (uint32_t)(frac_to_u64(__dmul_rn(k_fd[d], __dmul_rn(sp, sp))) >> 32);
    } else {
        u = turns_mul(k_turns[d], (uint32_t)(m * m));
    }
    double s, c;
    sincospi((double)(int32_t)u * 4.656612873077392578125e-10, &s, &c);
    const double scale = d == 0 ? a.inv_g : 1.0;  // exact power of two
    const double cr = c * scale, ci = -s * scale;
    const float hr = (float)cr, hi = (float)ci;
    out[i] = make_float4(hr, hi, (float)(cr - (double)hr), (float)(ci - (double)hi));
}

}  // namespace qhd
