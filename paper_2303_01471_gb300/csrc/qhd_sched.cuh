// qhd_sched.cuh -- the damping schedule a(t) = e^{phi_t}, b(t) = e^{chi_t} of
// Eq. (qhd_operator) as both simulators evaluate it: device evaluation in FP64
// at the step midpoints, the 64-bit fraction of a turn used by the fixed-point
// phases, and the host-side validation of qhd_schedule arrays.
#pragma once
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "qhd.h"
#include "qhd_kernels.h"

namespace qhd {

constexpr int SCHED_MAX_SAMPLES = 256;  // table samples per instance

__device__ inline double interp_dev(const double *ts, const double *vs, int ns, double t) {
    if (t <= ts[0]) return vs[0];
    if (t >= ts[ns - 1]) return vs[ns - 1];
    int lo = 0, hi = ns - 1;
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (ts[mid] <= t) lo = mid;
        else hi = mid;
    }
    const double w = __ddiv_rn(__dsub_rn(t, ts[lo]), __dsub_rn(ts[hi], ts[lo]));
    return __dadd_rn(vs[lo], __dmul_rn(w, __dsub_rn(vs[hi], vs[lo])));
}

// a = e^{phi}, b = e^{chi} at time t.
__device__ inline void sched_eval_dev(const SchedDev &s, double t, double *a, double *b) {
    if (s.kind == 0) {
        const double t3 = __dmul_rn(__dmul_rn(t, t), t);
        *a = __ddiv_rn(s.c_phi, __dadd_rn(s.eps, t3));
        *b = __dmul_rn(s.c_chi, t3);
    } else if (s.kind == 2) {
        const double at = fabs(t);
        *a = __ddiv_rn(s.c_phi, __dadd_rn(s.eps, pow(at, s.power + 1.0)));
        *b = __dmul_rn(s.c_chi, pow(at, 2.0 * s.power - 1.0));
    } else {
        *a = exp(interp_dev(s.t, s.phi, s.ns, t));
        *b = exp(interp_dev(s.t, s.chi, s.ns, t));
    }
}

// frac(y) as a 64-bit fraction of one turn, rounded to 2^-64.
__device__ inline uint64_t frac_to_u64(double y) {
    const double f = y - floor(y);                  // exact
    const double h = f * 4294967296.0;              // exact
    double hf = floor(h);
    double lf = rint((h - hf) * 4294967296.0);      // exact except the final rounding
    if (lf >= 4294967296.0) {
        lf = 0.0;
        hf += 1.0;
    }
    uint32_t hi = hf >= 4294967296.0 ? 0u : (uint32_t)hf;
    return ((uint64_t)hi << 32) | (uint64_t)(uint32_t)lf;
}

// Validate `batch` schedules and convert them for the device.  Table samples
// are packed into samples_host (3 * SCHED_MAX_SAMPLES doubles per instance:
// t, phi, chi) and the device records point into samples_dev, where the caller
// copies samples_host.  *shared is set when every instance has the same kinetic
// weight e^{phi_t}.  Returns "" on success, else the reason.
inline std::string convert_schedules(const qhd_schedule *s, int64_t batch, double *samples_dev,
                                     std::vector<SchedDev> &dev, std::vector<double> &samples_host, bool *shared) {
    char buf[160];
    dev.assign((size_t)batch, SchedDev{});
    samples_host.assign((size_t)(3 * SCHED_MAX_SAMPLES * batch), 0.0);
    for (int64_t b = 0; b < batch; ++b) {
        const qhd_schedule &q = s[b];
        SchedDev &d = dev[(size_t)b];
        d.kind = q.kind;
        d.ns = 0;
        d.c_phi = q.c_phi;
        d.eps = q.eps;
        d.c_chi = q.c_chi;
        d.t = d.phi = d.chi = nullptr;
        d.power = 0.0;
        if (q.kind == QHD_SCHED_NESTEROV || q.kind == QHD_SCHED_POWER) {
            if (!std::isfinite(q.c_phi) || !(q.c_phi > 0) || !std::isfinite(q.eps) || q.eps < 0 ||
                !std::isfinite(q.c_chi) || q.c_chi < 0) {
                snprintf(buf, sizeof buf, "instance %lld: bad Nesterov / power schedule", (long long)b);
                return buf;
            }
            if (q.kind == QHD_SCHED_POWER) {
                if (!std::isfinite(q.power) || !(q.power >= 0.5 && q.power <= 8.0)) {
                    snprintf(buf, sizeof buf, "instance %lld: power must be in [0.5, 8]", (long long)b);
                    return buf;
                }
                d.power = q.power;
            }
        } else if (q.kind == QHD_SCHED_TABLE) {
            if (!q.t || !q.phi || !q.chi || q.n_samples < 1 || q.n_samples > SCHED_MAX_SAMPLES) {
                snprintf(buf, sizeof buf, "instance %lld: bad table schedule", (long long)b);
                return buf;
            }
            for (int64_t i = 0; i < q.n_samples; ++i) {
                if (!std::isfinite(q.t[i]) || !std::isfinite(q.phi[i]) || !std::isfinite(q.chi[i])) {
                    snprintf(buf, sizeof buf, "instance %lld: non-finite table sample", (long long)b);
                    return buf;
                }
                if (i > 0 && !(q.t[i] > q.t[i - 1])) {
                    snprintf(buf, sizeof buf, "instance %lld: table times not increasing", (long long)b);
                    return buf;
                }
            }
            double *base = samples_dev + (size_t)(3 * SCHED_MAX_SAMPLES * b);
            d.ns = (int32_t)q.n_samples;
            d.t = base;
            d.phi = base + SCHED_MAX_SAMPLES;
            d.chi = base + 2 * SCHED_MAX_SAMPLES;
            double *hb = samples_host.data() + (size_t)(3 * SCHED_MAX_SAMPLES * b);
            for (int64_t i = 0; i < q.n_samples; ++i) {
                hb[i] = q.t[i];
                hb[SCHED_MAX_SAMPLES + i] = q.phi[i];
                hb[2 * SCHED_MAX_SAMPLES + i] = q.chi[i];
            }
        } else {
            snprintf(buf, sizeof buf, "instance %lld: unknown schedule kind %d", (long long)b, q.kind);
            return buf;
        }
    }
    // One kinetic factor serves every instance when the kinetic weights e^{phi}
    // agree (e.g. instances that differ only in the potential scale).
    bool sh = true;
    for (int64_t b = 1; b < batch && sh; ++b) {
        const qhd_schedule &p = s[0], &q = s[b];
        if (p.kind != q.kind) sh = false;
        else if (p.kind == QHD_SCHED_NESTEROV) sh = p.c_phi == q.c_phi && p.eps == q.eps;
        else if (p.kind == QHD_SCHED_POWER) sh = p.c_phi == q.c_phi && p.eps == q.eps && p.power == q.power;
        else {
            sh = p.n_samples == q.n_samples;
            for (int64_t i = 0; sh && i < p.n_samples; ++i) sh = p.t[i] == q.t[i] && p.phi[i] == q.phi[i];
        }
    }
    *shared = sh;
    return "";
}

}  // namespace qhd
