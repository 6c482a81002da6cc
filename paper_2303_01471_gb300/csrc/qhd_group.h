// qhd_group.h -- what the batched persistent launch (qhd_group.cu) reads from
// a context (internal; the context itself is defined in qhd_host.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qhd.h"
#include "qhd_kernels.h"

namespace qhd {

struct GroupCtxView {
    int ndim;
    int64_t n[3];
    double len[3];
    int64_t batch, g;
    int ksum, koff[3];
    float2 *psi;
    const uint32_t *fq;
    uint64_t *pot;           // [chunk + 1][batch]
    float4 *kt;              // [chunk][kt_batch][ksum]
    const float4 *tw_row;    // stage-2 twiddles of axis 1
    const float4 *ptab;
    const SchedDev *sched;
    const InstDev *inst;
    int64_t chunk;           // steps per chunk of tables
    int64_t kt_batch;        // 1 when every instance shares the kinetic schedule
    int split, kinetic;
    double t;
    int64_t steps_done;
    cudaStream_t stream;
    bool whole_run;          // 2-D grid held in one cluster per instance (FFT transform)
    int plane_c;             // CTAs per instance of the context's own whole-run launch (0: none)
};

// Fills v; QHD_ERR_STATE without a potential and a schedule.
qhd_status ctx_group_view(qhd_ctx *c, GroupCtxView *v);
// Advances the context's clock after a batched launch evolved it by nsteps of dt.
void ctx_advance(qhd_ctx *c, int64_t nsteps, double dt);

}  // namespace qhd
