// qhd_host.cu -- host side of the C ABI declared in include/qhd.h.
//
// Owns argument validation, the workspace layout, the per-context state and
// the order of kernel launches of one evolve call.  Device memory and the
// stream belong to the caller; nothing here allocates device memory.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qhd.h"
#include "qhd_device.cuh"
#include "qhd_group.h"
#include "qhd_kernels.h"
#include "qhd_trace.h"
#include "qhd_sched.cuh"
#include "qhd_spectrum.h"
#include "qhd_tcdft.h"

using namespace qhd;

namespace {

constexpr int MAX_TABLE_SAMPLES = SCHED_MAX_SAMPLES;
constexpr size_t KT_BUDGET = size_t(64) << 20;  // bytes of kinetic tables per chunk
constexpr int64_t MAX_CHUNK = 1024;
constexpr int OBS_BLOCKS_MAX = 1024;
constexpr int MINMAX_BLOCKS_MAX = 512;

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
    size_t f64, fq, kt, pot, sched, samples, inst, tw, twx, ptab, coord, obs_part, obs_res, mm, total;
    int64_t chunk;         // steps per chunk with one kinetic table per instance
    int64_t chunk_shared;  // steps per chunk when all instances share the kinetic table
    int obs_blocks, mm_blocks;
};

int64_t grid_points(int ndim, const int64_t *n) {
    int64_t g = 1;
    for (int d = 0; d < ndim; ++d) g *= n[d];
    return g;
}

bool shape_ok(int ndim, const int64_t *n, int64_t batch) {
    if (ndim < 1 || ndim > 3 || !n || batch < 1) return false;
    for (int d = 0; d < ndim; ++d)
        if (!supported_n(n[d])) return false;
    const int64_t g = grid_points(ndim, n);
    if (g > (int64_t(1) << 30)) return false;
    // batch indexes the second grid dimension of the per-instance kernels (<= 65535)
    if (batch > 65535 || g * batch > (int64_t(1) << 34)) return false;
    return true;
}

int block_count(int64_t g, int cap) {
    int64_t b = (g + 255) / 256;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

Layout make_layout(int ndim, const int64_t *n, int64_t batch) {
    Layout L{};
    const int64_t g = grid_points(ndim, n);
    int64_t ksum = 0;
    for (int d = 0; d < ndim; ++d) ksum += n[d];
    // kinetic tables: at most KT_BUDGET bytes, enough for MAX_CHUNK steps of one
    // table per instance when that fits
    const size_t per_step_all = (size_t)batch * (size_t)ksum * sizeof(float4);
    size_t kt_bytes = (size_t)MAX_CHUNK * per_step_all;
    if (kt_bytes > KT_BUDGET) kt_bytes = KT_BUDGET;
    if (kt_bytes < per_step_all) kt_bytes = per_step_all;
    int64_t ch = (int64_t)(kt_bytes / per_step_all);
    L.chunk = ch > MAX_CHUNK ? MAX_CHUNK : ch;
    int64_t chs = (int64_t)(kt_bytes / ((size_t)ksum * sizeof(float4)));
    L.chunk_shared = chs > MAX_CHUNK ? MAX_CHUNK : chs;
    L.obs_blocks = block_count(g, OBS_BLOCKS_MAX);
    L.mm_blocks = block_count(g, MINMAX_BLOCKS_MAX);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    };
    L.f64 = take(sizeof(double) * (size_t)(g * batch));
    L.fq = take(sizeof(uint32_t) * (size_t)(g * batch));
    L.kt = take(kt_bytes);
    L.pot = take(sizeof(uint64_t) * (size_t)((MAX_CHUNK + 1) * batch));
    L.sched = take(sizeof(SchedDev) * (size_t)batch);
    L.samples = take(sizeof(double) * 3 * MAX_TABLE_SAMPLES * (size_t)batch);
    L.inst = take(sizeof(InstDev) * (size_t)batch);
    L.tw = take(sizeof(float4) * (size_t)(ksum));
    L.twx = take(sizeof(float4) * (size_t)(ksum));
    L.ptab = take(sizeof(float4) * (size_t)PHASE_TAB);
    L.coord = take(sizeof(double) * (size_t)ksum);
    L.obs_part = take(sizeof(double) * 3 * (size_t)L.obs_blocks * (size_t)batch);
    L.obs_res = take(sizeof(double) * 3 * (size_t)batch);
    L.mm = take(sizeof(MinMaxPart) * (size_t)L.mm_blocks * (size_t)batch);
    L.total = off;
    return L;
}

}  // namespace

struct qhd_ctx {
    int ndim = 0;
    int64_t n[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    int64_t batch = 1, g = 1;
    int ksum = 0, koff[3] = {0, 0, 0};
    float2 *psi = nullptr;
    char *work = nullptr;
    size_t work_bytes = 0;
    cudaStream_t stream = nullptr;
    Layout L{};
    // workspace views
    double *f64 = nullptr;
    uint32_t *fq = nullptr;
    float4 *kt = nullptr;
    uint64_t *pot = nullptr;
    SchedDev *sched = nullptr;
    double *samples = nullptr;
    InstDev *inst = nullptr;
    float4 *tw[3] = {nullptr, nullptr, nullptr};
    float4 *twx = nullptr;  // exchange twiddles of the cluster-distributed axis
    float4 *ptab = nullptr; // potential phase table exp(-2 pi i (k + 1/2) / PHASE_TAB), hi/lo
    int plane_mode = 0;     // 0 generic passes, 2 whole-run 2-D clusters, 3 3-D plane pass
    int plane_c = 0;        // CTAs per instance (2-D) or per plane (3-D) of the cluster engine
    double *coord = nullptr;
    double *obs_part = nullptr, *obs_res = nullptr;
    MinMaxPart *mm = nullptr;
    // host state
    bool have_f = false, have_sched = false;
    bool kt_shared = false;  // every instance has the same kinetic schedule
    int split = QHD_SPLIT_STRANG;
    int kinetic = QHD_KINETIC_SPECTRAL;
    double t = 0.0;
    int64_t steps_done = 0;
    int64_t launches = 0;
    qhd_status sticky = QHD_OK;
    std::string err;
    // failure injection (qhd_inject_failure): the inject_after-th checked CUDA
    // call from now on is not issued and reports inject_kind instead
    qhd_status inject_kind = QHD_OK;
    int64_t inject_after = 0;
    std::vector<InstDev> inst_host;
    // host copy of the schedules (spectrum: a(t), b(t) on the host)
    struct HostSched {
        int kind = 0;
        double c_phi = 0, eps = 0, c_chi = 0, power = 0;
        std::vector<double> t, phi, chi;
    };
    std::vector<HostSched> sched_host;
    std::vector<double> coord_host;
    // device-time accounting (qhd_timing_*)
    // tensor-core transform (qhd_set_transform)
    TcState *tc = nullptr;
    int64_t lib_calls = 0;
    int timing_every = 0;
    struct TimedLaunch {
        int kclass;
        cudaEvent_t start, stop;
    };
    std::vector<TimedLaunch> timed;
    std::vector<cudaEvent_t> event_pool;
    ~qhd_ctx() {
        for (auto &r : timed) {
            cudaEventDestroy(r.start);
            cudaEventDestroy(r.stop);
        }
        for (auto e : event_pool) cudaEventDestroy(e);
        tc_destroy(tc);
    }
};

namespace {

qhd_status fail(qhd_ctx *c, qhd_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (s == QHD_ERR_CUDA || s == QHD_ERR_TIMEOUT) c->sticky = s;
    }
    return s;
}

qhd_status cuda_fail(qhd_ctx *c, cudaError_t e, const char *where) {
    return fail(c, QHD_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

// True when an injected failure is due at this checked call; the call is then
// skipped and the context fails as the injection asked.
bool injected(qhd_ctx *c) {
    if (c->inject_kind == QHD_OK || --c->inject_after > 0) return false;
    const qhd_status k = c->inject_kind;
    c->inject_kind = QHD_OK;
    fail(c, k, "injected failure (%s)", k == QHD_ERR_TIMEOUT ? "device time-out" : "CUDA call");
    return true;
}

#define QHD_CUDA(c, call)                                        \
    do {                                                         \
        if (injected(c)) return (c)->sticky;                     \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
    } while (0)

#define QHD_LAUNCH(c, call)                                      \
    do {                                                         \
        if (injected(c)) return (c)->sticky;                     \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return cuda_fail((c), e_, #call); \
        (c)->launches++;                                         \
    } while (0)

constexpr size_t MAX_TIMED = 65536;

cudaEvent_t take_event(qhd_ctx *c) {
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Record an event pair around one launch when timing is on for this step.
struct TimedScope {
    qhd_ctx *c;
    int kclass;
    bool on;
    cudaEvent_t start = nullptr, stop = nullptr;
    TimedScope(qhd_ctx *c_, int k, bool sample) : c(c_), kclass(k), on(false) {
        if (!sample || c->timing_every <= 0 || c->timed.size() >= MAX_TIMED) return;
        start = take_event(c);
        stop = take_event(c);
        if (!start || !stop) return;
        on = cudaEventRecord(start, c->stream) == cudaSuccess;
    }
    ~TimedScope() {
        if (on && cudaEventRecord(stop, c->stream) == cudaSuccess) {
            c->timed.push_back({kclass, start, stop});
            return;
        }
        if (start) c->event_pool.push_back(start);
        if (stop) c->event_pool.push_back(stop);
    }
};

qhd_status check_ctx(qhd_ctx *c) {
    if (!c) return QHD_ERR_INVALID_ARG;
    if (c->sticky != QHD_OK) return c->sticky;
    return QHD_OK;
}

}  // namespace

extern "C" {

const char *qhd_status_string(qhd_status s) {
    switch (s) {
    case QHD_OK: return "ok";
    case QHD_ERR_INVALID_ARG: return "invalid argument";
    case QHD_ERR_UNSUPPORTED: return "unsupported";
    case QHD_ERR_STATE: return "bad call order";
    case QHD_ERR_CUDA: return "CUDA error";
    case QHD_ERR_TIMEOUT: return "device time-out";
    case QHD_ERR_WORKSPACE: return "workspace too small or misaligned";
    }
    return "unknown status";
}

const char *qhd_last_error(const qhd_ctx *c) { return c ? c->err.c_str() : ""; }

int64_t qhd_launch_count(const qhd_ctx *c) { return c ? c->launches : 0; }

int qhd_cluster_ctas(const qhd_ctx *c) {
    return c && (c->plane_mode == 2 || c->plane_mode == 3) ? c->plane_c : 0;
}

size_t qhd_workspace_bytes(int ndim, const int64_t *n, int64_t batch) {
    if (!shape_ok(ndim, n, batch)) return 0;
    return make_layout(ndim, n, batch).total;
}

qhd_status qhd_init_grid(qhd_ctx **out, int ndim, const int64_t *n, const double *lo, const double *hi,
                         int64_t batch, void *psi_dev, void *work_dev, size_t work_bytes, void *stream) {
    if (!out || !n || !lo || !hi) return QHD_ERR_INVALID_ARG;
    if (!shape_ok(ndim, n, batch)) return QHD_ERR_INVALID_ARG;
    for (int d = 0; d < ndim; ++d)
        if (!std::isfinite(lo[d]) || !std::isfinite(hi[d]) || !(lo[d] < hi[d])) return QHD_ERR_INVALID_ARG;
    // 16-byte aligned: the passes move psi in 16-byte (two-point) copies
    if (!psi_dev || ((uintptr_t)psi_dev & 15)) return QHD_ERR_INVALID_ARG;
    Layout L = make_layout(ndim, n, batch);
    if (!work_dev || ((uintptr_t)work_dev & 255) || work_bytes < L.total) return QHD_ERR_WORKSPACE;

    qhd_ctx *c = new qhd_ctx();
    c->ndim = ndim;
    c->batch = batch;
    for (int d = 0; d < ndim; ++d) {
        c->n[d] = n[d];
        c->lo[d] = lo[d];
        c->hi[d] = hi[d];
    }
    c->g = grid_points(ndim, n);
    c->ksum = 0;
    for (int d = 0; d < ndim; ++d) {
        c->koff[d] = c->ksum;
        c->ksum += (int)n[d];
    }
    c->psi = (float2 *)psi_dev;
    c->work = (char *)work_dev;
    c->work_bytes = work_bytes;
    c->stream = (cudaStream_t)stream;
    c->L = L;
    c->f64 = (double *)(c->work + L.f64);
    c->fq = (uint32_t *)(c->work + L.fq);
    c->kt = (float4 *)(c->work + L.kt);
    c->pot = (uint64_t *)(c->work + L.pot);
    c->sched = (SchedDev *)(c->work + L.sched);
    c->samples = (double *)(c->work + L.samples);
    c->inst = (InstDev *)(c->work + L.inst);
    c->coord = (double *)(c->work + L.coord);
    c->obs_part = (double *)(c->work + L.obs_part);
    c->obs_res = (double *)(c->work + L.obs_res);
    c->mm = (MinMaxPart *)(c->work + L.mm);

    // stage-2 twiddles per axis, tw2[m*R1 + j] = exp(-2 pi i j m / N) from FP64,
    // stored as the FP32 value and its FP32 rounding residual
    std::vector<float4> tw((size_t)c->ksum, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int d = 0; d < ndim; ++d) {
        int r1 = 0, r2 = 0;
        plan_of((int)n[d], &r1, &r2);
        c->tw[d] = (float4 *)(c->work + L.tw) + c->koff[d];
        if (r2 <= 1) continue;
        for (int m = 0; m < r2; ++m)
            for (int j = 0; j < r1; ++j) {
                const int64_t jm = ((int64_t)j * m) % n[d];
                const double ang = 2.0 * 3.141592653589793238462643383279502884 * (double)jm / (double)n[d];
                const double cr = cos(ang), ci = -sin(ang);
                const float hr = (float)cr, hi = (float)ci;
                tw[(size_t)c->koff[d] + (size_t)(m * r1 + j)] =
                    make_float4(hr, hi, (float)(cr - (double)hr), (float)(ci - (double)hi));
            }
    }
    // cluster plane engine: 2-D grids with both axes in 32..256 stay resident in
    // one cluster per instance; 3-D grids whose last two axes fit use plane passes
    c->twx = (float4 *)(c->work + L.twx);
    int dist_axis = -1;
    if (ndim == 2 && plane_supported((int)n[0], (int)n[1])) {
        c->plane_mode = 2;
        dist_axis = 0;
        c->plane_c = plane_cluster((int)n[0]);
        // a batch that leaves most SMs idle runs each instance on twice the CTAs
        int dev = 0, sms = 0;
        const int wide = plane_cluster_wide((int)n[0]);
        if (wide && cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            batch * (int64_t)wide <= (int64_t)sms)
            c->plane_c = wide;
    }
    else if (ndim == 3 && plane_supported((int)n[1], (int)n[2])) {
        c->plane_mode = 3;
        dist_axis = 1;
        c->plane_c = plane_cluster((int)n[1]);
    }
    std::vector<float4> twx((size_t)c->ksum, make_float4(0.f, 0.f, 0.f, 0.f));
    if (dist_axis >= 0) {
        const int n1 = (int)n[dist_axis], cc = c->plane_c, rr = n1 / cc;
        for (int q = 0; q < cc; ++q)
            for (int j = 0; j < rr; ++j) {
                const double ang = 2.0 * 3.141592653589793238462643383279502884 * (double)(((int64_t)j * q) % n1) /
                                   (double)n1;
                const double cr = cos(ang), ci = -sin(ang);
                const float hr = (float)cr, hi = (float)ci;
                twx[(size_t)(q * rr + j)] = make_float4(hr, hi, (float)(cr - (double)hr), (float)(ci - (double)hi));
            }
    }
    // potential phase table
    c->ptab = (float4 *)(c->work + L.ptab);
    std::vector<float4> ptab((size_t)PHASE_TAB);
    for (int k = 0; k < PHASE_TAB; ++k) {
        const double ang = 2.0 * 3.141592653589793238462643383279502884 * ((double)k + 0.5) / (double)PHASE_TAB;
        const double cr = cos(ang), ci = -sin(ang);
        const float hr = (float)cr, hi = (float)ci;
        ptab[(size_t)k] = make_float4(hr, hi, (float)(cr - (double)hr), (float)(ci - (double)hi));
    }
    // mesh coordinates x = lo + (j (hi - lo)) / N
    c->coord_host.resize((size_t)c->ksum);
    for (int d = 0; d < ndim; ++d)
        for (int64_t j = 0; j < n[d]; ++j)
            c->coord_host[(size_t)(c->koff[d] + j)] = lo[d] + (double)j * (hi[d] - lo[d]) / (double)n[d];

    cudaError_t e = cudaMemcpyAsync(c->work + L.tw, tw.data(), tw.size() * sizeof(float4),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->twx, twx.data(), twx.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->ptab, ptab.data(), ptab.size() * sizeof(float4), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->coord, c->coord_host.data(), c->coord_host.size() * sizeof(double),
                            cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        delete c;
        return QHD_ERR_CUDA;
    }
    c->inst_host.assign((size_t)batch, InstDev{});
    *out = c;
    return QHD_OK;
}

static qhd_status set_potential_common(qhd_ctx *c) {
    const int64_t B = c->batch, G = c->g;
    const int nb = c->L.mm_blocks;
    QHD_LAUNCH(c, launch_minmax(c->f64, G, B, c->mm, nb, c->stream));
    std::vector<MinMaxPart> part((size_t)(nb * B));
    QHD_CUDA(c, cudaMemcpyAsync(part.data(), c->mm, part.size() * sizeof(MinMaxPart), cudaMemcpyDeviceToHost,
                                c->stream));
    QHD_CUDA(c, cudaStreamSynchronize(c->stream));
    std::vector<InstDev> inst((size_t)B);
    for (int64_t b = 0; b < B; ++b) {
        double mn = INFINITY, mx = -INFINITY;
        int64_t am = INT64_MAX, nf = 0;
        for (int i = 0; i < nb; ++i) {
            const MinMaxPart &p = part[(size_t)(b * nb + i)];
            nf += p.nonfinite;
            if (p.fmin < mn || (p.fmin == mn && p.argmin < am)) {
                mn = p.fmin;
                am = p.argmin;
            }
            if (p.fmax > mx) mx = p.fmax;
        }
        // the FP64 copy is already overwritten: a rejected f discards the previous one
        if (nf > 0) {
            c->have_f = false;
            return fail(c, QHD_ERR_INVALID_ARG, "instance %lld: %lld non-finite f values", (long long)b,
                        (long long)nf);
        }
        const double range = mx - mn;
        if (!(range < 2147483648.0)) {
            c->have_f = false;
            return fail(c, QHD_ERR_INVALID_ARG, "instance %lld: f range %g >= 2^31", (long long)b, range);
        }
        // largest power-of-two scale keeping (f - fmin) * 2^shift below 2^32 - 4096
        int shift = 52;
        if (range > 0.0) {
            shift = (int)std::floor(std::log2((4294967296.0 - 4096.0) / range));
            while (shift > 0 && std::ldexp(range, shift) >= 4294967296.0 - 4096.0) --shift;
            if (shift > 52) shift = 52;
        }
        InstDev &ip = inst[(size_t)b];
        ip.fmin = mn;
        ip.shift = shift;
        ip.pad_ = 0;
        int64_t rem = am;
        for (int d = 2; d >= 0; --d) ip.xs[d] = 0.0;
        for (int d = c->ndim - 1; d >= 0; --d) {
            const int64_t idx = rem % c->n[d];
            rem /= c->n[d];
            ip.xs[d] = c->coord_host[(size_t)(c->koff[d] + idx)];
        }
    }
    QHD_CUDA(c, cudaMemcpyAsync(c->inst, inst.data(), inst.size() * sizeof(InstDev), cudaMemcpyHostToDevice,
                                c->stream));
    QHD_LAUNCH(c, launch_quantize(c->f64, c->fq, c->inst, G, B, c->stream));
    QHD_CUDA(c, cudaStreamSynchronize(c->stream));
    c->inst_host = inst;
    c->have_f = true;
    return QHD_OK;
}

qhd_status qhd_set_potential(qhd_ctx *c, const double *f_host) {
    TraceRange trace("qhd_set_potential");
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (!f_host) return fail(c, QHD_ERR_INVALID_ARG, "f_host is NULL");
    QHD_CUDA(c, cudaMemcpyAsync(c->f64, f_host, sizeof(double) * (size_t)(c->g * c->batch), cudaMemcpyHostToDevice,
                                c->stream));
    return set_potential_common(c);
}

qhd_status qhd_set_potential_device(qhd_ctx *c, const double *f_dev) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (!f_dev) return fail(c, QHD_ERR_INVALID_ARG, "f_dev is NULL");
    QHD_CUDA(c, cudaMemcpyAsync(c->f64, f_dev, sizeof(double) * (size_t)(c->g * c->batch), cudaMemcpyDeviceToDevice,
                                c->stream));
    return set_potential_common(c);
}

qhd_status qhd_set_schedule(qhd_ctx *c, const qhd_schedule *s) {
    qhd_status st = check_ctx(c);
    if (st != QHD_OK) return st;
    if (!s) return fail(c, QHD_ERR_INVALID_ARG, "schedule is NULL");
    const int64_t B = c->batch;
    std::vector<SchedDev> dev;
    std::vector<double> samples;
    bool shared = false;
    const std::string why = convert_schedules(s, B, c->samples, dev, samples, &shared);
    if (!why.empty()) return fail(c, QHD_ERR_INVALID_ARG, "%s", why.c_str());
    QHD_CUDA(c, cudaMemcpyAsync(c->samples, samples.data(), samples.size() * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream));
    QHD_CUDA(c, cudaMemcpyAsync(c->sched, dev.data(), dev.size() * sizeof(SchedDev), cudaMemcpyHostToDevice,
                                c->stream));
    // the host vectors die on return: wait for the copies
    QHD_CUDA(c, cudaStreamSynchronize(c->stream));
    c->kt_shared = shared;
    c->sched_host.assign((size_t)B, qhd_ctx::HostSched{});
    for (int64_t b = 0; b < B; ++b) {
        const qhd_schedule &q = s[b];
        qhd_ctx::HostSched &h = c->sched_host[(size_t)b];
        h.kind = q.kind;
        h.c_phi = q.c_phi;
        h.eps = q.eps;
        h.c_chi = q.c_chi;
        h.power = q.kind == QHD_SCHED_POWER ? q.power : 0.0;
        if (q.kind == QHD_SCHED_TABLE) {
            h.t.assign(q.t, q.t + q.n_samples);
            h.phi.assign(q.phi, q.phi + q.n_samples);
            h.chi.assign(q.chi, q.chi + q.n_samples);
        }
    }
    c->have_sched = true;
    return QHD_OK;
}

qhd_status qhd_reset_state(qhd_ctx *c) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    const float v = (float)(1.0 / std::sqrt((double)c->g));
    QHD_LAUNCH(c, launch_uniform(c->psi, c->g * c->batch, v, c->stream));
    c->t = 0.0;
    c->steps_done = 0;
    return QHD_OK;
}

qhd_status qhd_set_time(qhd_ctx *c, double t) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (!std::isfinite(t)) return fail(c, QHD_ERR_INVALID_ARG, "time not finite");
    c->t = t;
    return QHD_OK;
}

qhd_status qhd_get_time(const qhd_ctx *c, double *t_out, int64_t *steps_out) {
    if (!c) return QHD_ERR_INVALID_ARG;
    if (t_out) *t_out = c->t;
    if (steps_out) *steps_out = c->steps_done;
    return QHD_OK;
}

namespace {

// One chunk of steps with the tensor-core transform: per step a potential
// split, W along axis 1, a transposing split, W along axis 0, the kinetic
// split, conj W along axis 0, a transposing split, conj W along axis 1.  The
// state stays in the transform's product buffer between steps and chunks.
qhd_status evolve_tc_chunk(qhd_ctx *c, int64_t j0, int64_t cnt, bool last_chunk, int64_t ktb) {
    const int64_t B = c->batch;
    TcPhaseArgs ta{};
    ta.psi = c->psi;
    ta.fq = c->fq;
    ta.ptab = c->ptab;
    ta.ksum = c->ksum;
    ta.kt_batch = ktb;
    auto gemm = [&](bool inv, bool sample) -> qhd_status {
        TimedScope ts(c, QHD_KCLASS_TC_GEMM, sample);
        if (injected(c)) return c->sticky;
        cudaError_t e = tc_gemm(c->tc, inv, c->stream, &c->launches);
        if (e != cudaSuccess) return fail(c, QHD_ERR_CUDA, "tensor-core GEMM failed: %s", cudaGetErrorString(e));
        return QHD_OK;
    };
    for (int64_t jl = 0; jl < cnt; ++jl) {
        const int64_t j = j0 + jl;
        const bool sample = c->timing_every > 0 && j % c->timing_every == 0;
        ta.pot = c->pot + jl * B;
        ta.dither = step_dither((uint64_t)(c->steps_done + j));
        ta.kt = c->kt + jl * ktb * c->ksum;
        qhd_status s;
        {
            TimedScope ts(c, QHD_KCLASS_TC_SPLIT, sample);
            QHD_CUDA(c, tc_dither_w(c->tc, ta.dither, c->stream, &c->launches));
            QHD_CUDA(c, tc_split_potential(c->tc, ta, j == 0, c->stream, &c->launches));
        }
        if ((s = gemm(false, sample)) != QHD_OK) return s;
        {
            TimedScope ts(c, QHD_KCLASS_TC_SPLIT, sample);
            QHD_CUDA(c, tc_split_transpose(c->tc, c->stream, &c->launches));
        }
        if ((s = gemm(false, sample)) != QHD_OK) return s;
        {
            TimedScope ts(c, QHD_KCLASS_TC_SPLIT, sample);
            QHD_CUDA(c, tc_split_kinetic(c->tc, ta, c->stream, &c->launches));
        }
        if ((s = gemm(true, sample)) != QHD_OK) return s;
        {
            TimedScope ts(c, QHD_KCLASS_TC_SPLIT, sample);
            QHD_CUDA(c, tc_split_transpose(c->tc, c->stream, &c->launches));
        }
        if ((s = gemm(true, sample)) != QHD_OK) return s;
    }
    if (last_chunk) {
        ta.pot = c->pot + cnt * B;
        ta.dither = 0;
        QHD_CUDA(c, tc_finish(c->tc, ta, true, c->stream, &c->launches));
    }
    return QHD_OK;
}

}  // namespace

qhd_status qhd_evolve(qhd_ctx *c, double T, double dt) {
    TraceRange trace("qhd_evolve");
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (!std::isfinite(T) || !std::isfinite(dt) || dt == 0.0)
        return fail(c, QHD_ERR_INVALID_ARG, "T and dt must be finite and dt nonzero");
    const double ratio = T / dt;
    const double nr = std::nearbyint(ratio);
    if (!(nr >= 1.0) || std::fabs(ratio - nr) > 1e-9 * nr || nr > 1e12)
        return fail(c, QHD_ERR_INVALID_ARG, "T/dt = %.17g is not a positive integer", ratio);
    if (!c->have_f || !c->have_sched)
        return fail(c, QHD_ERR_STATE, "evolve needs set_potential and set_schedule first");
    const int64_t nsteps = (int64_t)nr;
    const int ndim = c->ndim;
    const int64_t B = c->batch;

    PrepArgs pa{};
    pa.sched = c->sched;
    pa.inst = c->inst;
    pa.pot = c->pot;
    pa.kt = c->kt;
    pa.t_start = c->t;
    pa.dt = dt;
    pa.nsteps = nsteps;
    pa.batch = B;
    pa.ndim = ndim;
    for (int d = 0; d < 3; ++d) {
        pa.n[d] = d < ndim ? (int)c->n[d] : 1;
        pa.len[d] = d < ndim ? c->hi[d] - c->lo[d] : 1.0;
        pa.koff[d] = d < ndim ? c->koff[d] : c->ksum;
    }
    pa.ksum = c->ksum;
    pa.inv_g = 1.0 / (double)c->g;
    pa.split = c->split == QHD_SPLIT_LIE_TROTTER ? 1 : 0;
    pa.kinetic = c->kinetic == QHD_KINETIC_FD2 ? 1 : 0;

    const int64_t ch = c->kt_shared ? c->L.chunk_shared : c->L.chunk;
    const int64_t ktb = c->kt_shared ? 1 : B;
    pa.kt_batch = ktb;
    for (int64_t j0 = 0; j0 < nsteps; j0 += ch) {
        const int64_t cnt = nsteps - j0 < ch ? nsteps - j0 : ch;
        const bool last_chunk = j0 + cnt == nsteps;
        TraceRange trace_chunk("qhd_evolve chunk");
        pa.j0 = j0;
        pa.cnt = cnt;
        {
            TimedScope ts(c, QHD_KCLASS_PREP, true);
            QHD_LAUNCH(c, launch_prep(pa, c->stream));
        }
        if (ndim == 1) {
            OneDArgs o{};
            o.psi = c->psi;
            o.fq = c->fq;
            o.pot = c->pot;
            o.kt = c->kt;
            o.tw2 = c->tw[0];
            o.batch = B;
            o.cnt = (int)cnt;
            o.final_phase = last_chunk ? 1 : 0;
            o.dither_base = (uint64_t)(c->steps_done + j0);
            o.ptab = c->ptab;
            o.kt_batch = ktb;
            TimedScope ts(c, QHD_KCLASS_ONED, true);
            QHD_LAUNCH(c, launch_oned((int)c->n[0], o, c->stream));
            continue;
        }
        if (c->tc) {
            s = evolve_tc_chunk(c, j0, cnt, last_chunk, ktb);
            if (s != QHD_OK) return s;
            continue;
        }
        if (c->plane_mode == 2) {
            PlaneArgs w{};
            w.psi = c->psi;
            w.fq = c->fq;
            w.pot = c->pot;
            w.kt = c->kt;
            w.tw_row = c->tw[1];
            w.twx = c->twx;
            w.batch = B;
            w.cnt = (int)cnt;
            w.final_phase = last_chunk ? 1 : 0;
            w.ksum = c->ksum;
            w.dither_base = (uint64_t)(c->steps_done + j0);
            w.ptab = c->ptab;
            w.kt_batch = ktb;
            TimedScope ts(c, QHD_KCLASS_WHOLE, true);
            if (c->plane_c == plane_cluster((int)c->n[0]))
                QHD_LAUNCH(c, launch_plane_whole((int)c->n[0], (int)c->n[1], w, c->stream));
            else
                QHD_LAUNCH(c, launch_plane_whole_wide((int)c->n[0], (int)c->n[1], w, c->stream));
            continue;
        }
        const int last_ax = ndim - 1;
        RowArgs r{};
        r.psi = c->psi;
        r.fq = c->fq;
        r.tw2 = c->tw[last_ax];
        r.rows = B * (c->g / c->n[last_ax]);
        r.rows_per_inst = c->g / c->n[last_ax];
        r.ptab = c->ptab;
        AxisArgs ax0{};
        ax0.psi = c->psi;
        ax0.tw2 = c->tw[0];
        ax0.inner = c->g / c->n[0];
        ax0.planes = B;
        ax0.ksum = c->ksum;
        ax0.koff1 = c->koff[1];
        ax0.koff2 = ndim == 3 ? c->koff[2] : 0;
        ax0.log_n2 = ndim == 3 ? (int)std::log2((double)c->n[2]) : 0;
        ax0.ndim = ndim;
        ax0.kt_batch = ktb;
        ax0.mode = MODE_FWD | MODE_KIN | MODE_INV;
        PlaneArgs pl{};
        if (c->plane_mode == 3) {
            pl.psi = c->psi;
            pl.fq = c->fq;
            pl.tw_row = c->tw[2];
            pl.twx = c->twx;
            pl.planes = B * c->n[0];
            pl.planes_per_inst = c->n[0];
            pl.batch = B;
            pl.ptab = c->ptab;
            const int cc = plane_cluster((int)c->n[1]);
            ax0.perm1_r = (int)c->n[1] / cc;
            ax0.perm1_c = cc;
        }
        AxisArgs ax1{};
        if (ndim == 3) {
            ax1.psi = c->psi;
            ax1.tw2 = c->tw[1];
            ax1.inner = c->n[2];
            ax1.planes = B * c->n[0];
            ax1.ndim = ndim;
        }
        for (int64_t jl = 0; jl < cnt; ++jl) {
            const int64_t j = j0 + jl;
            const bool sample = c->timing_every > 0 && j % c->timing_every == 0;
            // row pass before step j: inverse transform of the previous step
            // (if any), merged potential phase theta_j, forward transform
            if (c->plane_mode == 3) {
                // plane pass over axes 1, 2 (inverse of the previous step, potential
                // phase, forward), then the axis-0 pass with the kinetic phase
                pl.pot = c->pot + jl * B;
                pl.mode = (j == 0 ? 0 : MODE_INV) | MODE_FWD;
                pl.dither = step_dither((uint64_t)(c->steps_done + j));
                {
                    TimedScope ts(c, QHD_KCLASS_PLANE, sample);
                    QHD_LAUNCH(c, launch_plane_pass((int)c->n[1], (int)c->n[2], pl, c->stream));
                }
                ax0.kt = c->kt + jl * ktb * c->ksum;
                TimedScope ts(c, QHD_KCLASS_AXIS0, sample);
                QHD_LAUNCH(c, launch_axis((int)c->n[0], ax0, c->stream));
                continue;
            }
            r.pot = c->pot + jl * B;
            r.mode = (j == 0 ? 0 : MODE_INV) | MODE_FWD;
            r.dither = step_dither((uint64_t)(c->steps_done + j));
            {
                TimedScope ts(c, QHD_KCLASS_ROW, sample);
                QHD_LAUNCH(c, launch_row((int)c->n[last_ax], r, c->stream));
            }
            if (ndim == 3) {
                ax1.mode = MODE_FWD;
                TimedScope ts(c, QHD_KCLASS_AXIS1_FWD, sample);
                QHD_LAUNCH(c, launch_axis((int)c->n[1], ax1, c->stream));
            }
            ax0.kt = c->kt + jl * ktb * c->ksum;
            {
                TimedScope ts(c, QHD_KCLASS_AXIS0, sample);
                QHD_LAUNCH(c, launch_axis((int)c->n[0], ax0, c->stream));
            }
            if (ndim == 3) {
                ax1.mode = MODE_INV;
                TimedScope ts(c, QHD_KCLASS_AXIS1_INV, sample);
                QHD_LAUNCH(c, launch_axis((int)c->n[1], ax1, c->stream));
            }
        }
        if (last_chunk) {
            if (c->plane_mode == 3) {
                pl.pot = c->pot + cnt * B;
                pl.mode = MODE_INV;
                pl.dither = 0;
                QHD_LAUNCH(c, launch_plane_pass((int)c->n[1], (int)c->n[2], pl, c->stream));
            } else {
                r.pot = c->pot + cnt * B;
                r.mode = MODE_INV;
                r.dither = 0;
                QHD_LAUNCH(c, launch_row((int)c->n[last_ax], r, c->stream));
            }
        }
    }
    c->t = c->t + (double)nsteps * dt;
    c->steps_done += nsteps;
    return QHD_OK;
}

qhd_status qhd_observables(qhd_ctx *c, qhd_obs *out, float *prob_dev, double radius) {
    TraceRange trace("qhd_observables");
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (!out) return fail(c, QHD_ERR_INVALID_ARG, "out is NULL");
    if (!std::isfinite(radius) || !(radius > 0)) return fail(c, QHD_ERR_INVALID_ARG, "radius must be > 0");
    if (!c->have_f) return fail(c, QHD_ERR_STATE, "observables need set_potential first");
    if (c->tc) {
        // a tensor-core GEMM whose bounded wait gave up leaves the state invalid
        const int to = tc_timed_out(c->tc, c->stream);
        if (to < 0) return fail(c, QHD_ERR_CUDA, "reading the tensor-core GEMM status failed");
        if (to > 0) return fail(c, QHD_ERR_TIMEOUT, "a tensor-core GEMM gave up waiting for its operands");
    }
    ObsArgs a{};
    a.psi = c->psi;
    a.f64 = c->f64;
    a.inst = c->inst;
    a.coord = c->coord;
    a.prob = prob_dev;
    a.partial = c->obs_part;
    a.result = c->obs_res;
    a.g = c->g;
    a.ndim = c->ndim;
    for (int d = 0; d < 3; ++d) {
        a.n[d] = d < c->ndim ? (int)c->n[d] : 1;
        a.log_n[d] = d < c->ndim ? (int)std::log2((double)c->n[d]) : 0;
        a.coff[d] = d < c->ndim ? c->koff[d] : 0;
    }
    a.radius = radius;
    a.nblk = c->L.obs_blocks;
    cudaError_t e = launch_observables(a, c->batch, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "observables");
    c->launches += 2;
    std::vector<double> res((size_t)(3 * c->batch));
    QHD_CUDA(c, cudaMemcpyAsync(res.data(), c->obs_res, res.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    QHD_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int64_t b = 0; b < c->batch; ++b) {
        qhd_obs &o = out[b];
        o.t = c->t;
        o.norm = res[(size_t)(3 * b)];
        o.e_f = res[(size_t)(3 * b + 1)];
        o.p_succ = res[(size_t)(3 * b + 2)];
        for (int d = 0; d < 3; ++d) o.x_star[d] = c->inst_host[(size_t)b].xs[d];
        o.steps_done = c->steps_done;
    }
    return QHD_OK;
}

qhd_status qhd_evolve_trajectory(qhd_ctx *c, double T, double dt, int64_t every, double radius,
                                 double *traj_dev) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (!traj_dev) return fail(c, QHD_ERR_INVALID_ARG, "traj_dev is NULL");
    if (!std::isfinite(radius) || !(radius > 0)) return fail(c, QHD_ERR_INVALID_ARG, "radius must be > 0");
    if (!std::isfinite(T) || !std::isfinite(dt) || dt == 0.0)
        return fail(c, QHD_ERR_INVALID_ARG, "T and dt must be finite and dt nonzero");
    const double ratio = T / dt;
    const double nr = std::nearbyint(ratio);
    if (!(nr >= 1.0) || std::fabs(ratio - nr) > 1e-9 * nr || nr > 1e12)
        return fail(c, QHD_ERR_INVALID_ARG, "T/dt = %.17g is not a positive integer", ratio);
    const int64_t nsteps = (int64_t)nr;
    if (every < 1 || nsteps % every != 0)
        return fail(c, QHD_ERR_INVALID_ARG, "every = %lld must divide the %lld steps", (long long)every,
                    (long long)nsteps);
    if (!c->have_f || !c->have_sched)
        return fail(c, QHD_ERR_STATE, "evolve needs set_potential and set_schedule first");
    const int64_t npts = nsteps / every;
    ObsArgs a{};
    a.psi = c->psi;
    a.f64 = c->f64;
    a.inst = c->inst;
    a.coord = c->coord;
    a.prob = nullptr;
    a.partial = c->obs_part;
    a.g = c->g;
    a.ndim = c->ndim;
    for (int d = 0; d < 3; ++d) {
        a.n[d] = d < c->ndim ? (int)c->n[d] : 1;
        a.log_n[d] = d < c->ndim ? (int)std::log2((double)c->n[d]) : 0;
        a.coff[d] = d < c->ndim ? c->koff[d] : 0;
    }
    a.radius = radius;
    a.nblk = c->L.obs_blocks;
    for (int64_t k = 0; k < npts; ++k) {
        s = qhd_evolve(c, (double)every * dt, dt);
        if (s != QHD_OK) return s;
        a.result = traj_dev + k * c->batch * 3;
        cudaError_t e = launch_observables(a, c->batch, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "trajectory observables");
        c->launches += 2;
    }
    return QHD_OK;
}

qhd_status qhd_set_splitting(qhd_ctx *c, int kind) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (kind != QHD_SPLIT_STRANG && kind != QHD_SPLIT_LIE_TROTTER)
        return fail(c, QHD_ERR_INVALID_ARG, "unknown splitting %d", kind);
    c->split = kind;
    return QHD_OK;
}

size_t qhd_tc_workspace_bytes(int ndim, const int64_t *n, int64_t batch, int products) {
    if (!shape_ok(ndim, n, batch) || ndim != 2 || !tc_supported((int)n[0], (int)n[1], batch)) return 0;
    if (!tc_products_ok((int)n[0], products)) return 0;
    return tc_workspace_bytes((int)n[0], batch, products);
}

qhd_status qhd_set_transform(qhd_ctx *c, int transform, int products, void *tc_work_dev, size_t tc_work_bytes) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (transform == QHD_TRANSFORM_FFT) {
        if (c->tc) {
            QHD_CUDA(c, cudaStreamSynchronize(c->stream));
            tc_destroy(c->tc);
            c->tc = nullptr;
        }
        return QHD_OK;
    }
    if (transform != QHD_TRANSFORM_TC_DFT) return fail(c, QHD_ERR_INVALID_ARG, "unknown transform %d", transform);
    if (products != 3 && products != 5 && products != 10)
        return fail(c, QHD_ERR_INVALID_ARG, "products must be 3, 5 or 10");
    if (c->ndim != 2 || !tc_supported((int)c->n[0], (int)c->n[1], c->batch) ||
        !tc_products_ok((int)c->n[0], products))
        return fail(c, QHD_ERR_UNSUPPORTED,
                    "tensor-core transform needs a square 2-D grid, n a power of two in 64..1024 (64..512 for "
                    "10 products), batch <= 65535");
    if (!tc_work_dev || ((uintptr_t)tc_work_dev & 255) ||
        tc_work_bytes < tc_workspace_bytes((int)c->n[0], c->batch, products))
        return fail(c, QHD_ERR_WORKSPACE, "tensor-core workspace too small or not 256-byte aligned");
    QHD_CUDA(c, cudaStreamSynchronize(c->stream));
    tc_destroy(c->tc);
    c->tc = nullptr;
    const char *why = nullptr;
    c->tc = tc_create((int)c->n[0], c->batch, products, tc_work_dev, tc_work_bytes, c->stream, &why);
    if (!c->tc) return fail(c, QHD_ERR_CUDA, "%s", why ? why : "tensor-core transform set-up failed");
    return QHD_OK;
}

int64_t qhd_library_call_count(const qhd_ctx *c) { return c ? c->lib_calls : 0; }

qhd_status qhd_set_kinetic(qhd_ctx *c, int kind) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (kind != QHD_KINETIC_SPECTRAL && kind != QHD_KINETIC_FD2)
        return fail(c, QHD_ERR_INVALID_ARG, "unknown kinetic operator %d", kind);
    c->kinetic = kind;
    return QHD_OK;
}

qhd_status qhd_timing_enable(qhd_ctx *c, int every) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (every < 0) return fail(c, QHD_ERR_INVALID_ARG, "every must be >= 0");
    c->timing_every = every;
    return QHD_OK;
}

qhd_status qhd_timing_read(qhd_ctx *c, double *ms_out, int64_t *launches_out, int reset) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    double ms[QHD_KCLASS_COUNT] = {};
    int64_t cnt[QHD_KCLASS_COUNT] = {};
    for (auto &r : c->timed) {
        QHD_CUDA(c, cudaEventSynchronize(r.stop));
        float v = 0.f;
        QHD_CUDA(c, cudaEventElapsedTime(&v, r.start, r.stop));
        ms[r.kclass] += v;
        cnt[r.kclass] += 1;
    }
    if (ms_out)
        for (int k = 0; k < QHD_KCLASS_COUNT; ++k) ms_out[k] = ms[k];
    if (launches_out)
        for (int k = 0; k < QHD_KCLASS_COUNT; ++k) launches_out[k] = cnt[k];
    if (reset) {
        for (auto &r : c->timed) {
            c->event_pool.push_back(r.start);
            c->event_pool.push_back(r.stop);
        }
        c->timed.clear();
    }
    return QHD_OK;
}

qhd_status qhd_inject_failure(qhd_ctx *c, int kind, int64_t after) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (kind != QHD_ERR_CUDA && kind != QHD_ERR_TIMEOUT && kind != QHD_OK)
        return fail(c, QHD_ERR_INVALID_ARG, "injected status must be QHD_ERR_CUDA, QHD_ERR_TIMEOUT or QHD_OK");
    if (kind != QHD_OK && after < 1) return fail(c, QHD_ERR_INVALID_ARG, "after must be >= 1");
    c->inject_kind = (qhd_status)kind;
    c->inject_after = after;
    return QHD_OK;
}

qhd_status qhd_destroy(qhd_ctx *c) {
    if (!c) return QHD_OK;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    delete c;
    return e == cudaSuccess ? QHD_OK : QHD_ERR_CUDA;
}

}  // extern "C"

// ------------------------------------------------- views for qhd_spectrum.cu
namespace qhd {

qhd_status ctx_view(qhd_ctx *c, CtxView *v) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (!c->have_f || !c->have_sched) return fail(c, QHD_ERR_STATE, "needs set_potential and set_schedule first");
    v->ndim = c->ndim;
    for (int d = 0; d < 3; ++d) {
        v->n[d] = d < c->ndim ? c->n[d] : 1;
        v->len[d] = d < c->ndim ? c->hi[d] - c->lo[d] : 1.0;
        v->tw[d] = d < c->ndim ? c->tw[d] : nullptr;
    }
    v->batch = c->batch;
    v->g = c->g;
    v->psi = c->psi;
    v->f64 = c->f64;
    v->kinetic = c->kinetic;
    v->stream = c->stream;
    return QHD_OK;
}

qhd_status ctx_group_view(qhd_ctx *c, GroupCtxView *v) {
    qhd_status s = check_ctx(c);
    if (s != QHD_OK) return s;
    if (!c->have_f || !c->have_sched) return fail(c, QHD_ERR_STATE, "needs set_potential and set_schedule first");
    v->ndim = c->ndim;
    for (int d = 0; d < 3; ++d) {
        v->n[d] = d < c->ndim ? c->n[d] : 1;
        v->len[d] = d < c->ndim ? c->hi[d] - c->lo[d] : 1.0;
        v->koff[d] = d < c->ndim ? c->koff[d] : c->ksum;
    }
    v->batch = c->batch;
    v->g = c->g;
    v->ksum = c->ksum;
    v->psi = c->psi;
    v->fq = c->fq;
    v->pot = c->pot;
    v->kt = c->kt;
    v->tw_row = c->ndim >= 2 ? c->tw[1] : nullptr;
    v->ptab = c->ptab;
    v->sched = c->sched;
    v->inst = c->inst;
    v->chunk = c->kt_shared ? c->L.chunk_shared : c->L.chunk;
    v->kt_batch = c->kt_shared ? 1 : c->batch;
    v->split = c->split == QHD_SPLIT_LIE_TROTTER ? 1 : 0;
    v->kinetic = c->kinetic == QHD_KINETIC_FD2 ? 1 : 0;
    v->t = c->t;
    v->steps_done = c->steps_done;
    v->stream = c->stream;
    v->whole_run = c->plane_mode == 2 && c->tc == nullptr;
    v->plane_c = c->plane_mode == 2 ? c->plane_c : 0;
    return QHD_OK;
}

void ctx_advance(qhd_ctx *c, int64_t nsteps, double dt) {
    c->t = c->t + (double)nsteps * dt;
    c->steps_done += nsteps;
}

static double host_interp(const std::vector<double> &ts, const std::vector<double> &vs, double t) {
    const size_t n = ts.size();
    if (t <= ts[0]) return vs[0];
    if (t >= ts[n - 1]) return vs[n - 1];
    size_t lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const size_t mid = (lo + hi) / 2;
        if (ts[mid] <= t) lo = mid;
        else hi = mid;
    }
    const double w = (t - ts[lo]) / (ts[hi] - ts[lo]);
    return vs[lo] + w * (vs[hi] - vs[lo]);
}

void ctx_sched_ab(const qhd_ctx *c, int64_t inst, double t, double *a, double *b) {
    const qhd_ctx::HostSched &h = c->sched_host[(size_t)inst];
    if (h.kind == QHD_SCHED_NESTEROV) {
        const double t3 = t * t * t;
        *a = h.c_phi / (h.eps + t3);
        *b = h.c_chi * t3;
    } else if (h.kind == QHD_SCHED_POWER) {
        const double at = std::fabs(t);
        *a = h.c_phi / (h.eps + std::pow(at, h.power + 1.0));
        *b = h.c_chi * std::pow(at, 2.0 * h.power - 1.0);
    } else {
        *a = std::exp(host_interp(h.t, h.phi, t));
        *b = std::exp(host_interp(h.t, h.chi, t));
    }
}

qhd_status ctx_fail(qhd_ctx *c, qhd_status s, const char *msg) { return fail(c, s, "%s", msg); }

int64_t ctx_grid_points(const qhd_ctx *c) { return c ? c->g : 0; }

}  // namespace qhd
