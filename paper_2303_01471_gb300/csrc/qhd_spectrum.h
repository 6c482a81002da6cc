// qhd_spectrum.h -- what the spectrum code (qhd_spectrum.cu) reads from a
// context (internal; the context itself is defined in qhd_host.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qhd.h"

namespace qhd {

struct CtxView {
    int ndim;
    int64_t n[3];        // axis lengths, 1 beyond ndim
    double len[3];       // box edge lengths hi - lo
    int64_t batch, g;    // instances, points per instance
    float2 *psi;         // the context's state, batch * g
    const double *f64;   // FP64 objective, batch * g
    const float4 *tw[3]; // stage-2 twiddles of the line transforms per axis
    int kinetic;         // QHD_KINETIC_*
    cudaStream_t stream;
};

// Fills v; QHD_ERR_STATE without a potential and a schedule.
qhd_status ctx_view(qhd_ctx *c, CtxView *v);
// a = e^{phi_t}, b = e^{chi_t} of instance `inst` at time t (FP64, host).
void ctx_sched_ab(const qhd_ctx *c, int64_t inst, double t, double *a, double *b);
// Records an error on the context (sticky for QHD_ERR_CUDA) and returns s.
qhd_status ctx_fail(qhd_ctx *c, qhd_status s, const char *msg);

}  // namespace qhd

namespace qhd {
// Points per instance of a context (0 for NULL).
int64_t ctx_grid_points(const qhd_ctx *c);
}  // namespace qhd
