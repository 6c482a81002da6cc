// qhd_group.cu -- one persistent launch over every instance of several 2-D
// contexts (ragged batches of different mesh sizes), replayed as a CUDA graph.
//
// The launch is a grid of thread-block clusters of GROUP_CL CTAs that pull work
// items from a device queue (an atomic counter) until it is empty:
//   * prep items build the step tables of one context (merged potential
//     coefficients and per-axis kinetic factors of GROUP_PREP_STEPS steps,
//     the same arithmetic as the stand-alone prep kernel, qhd_prep.cuh);
//   * instance items run every Strang step of the chunk for CL / sub instances
//     of one context, each held in the shared memory of `sub` CTAs of the
//     cluster (the whole-run engine of qhd_plane.cuh).
// All prep items precede all instance items in the queue, and a cluster claims
// an item only when it has finished the previous one, so when an instance item
// waits for its context's tables, every prep item it needs has been claimed by
// a running cluster that does not wait: the wait always ends, whether or not
// the whole grid is resident.  It is bounded anyway (GROUP_WAIT_LIMIT polls);
// a wait that gives up sets an error word that qhd_group_status reports as
// QHD_ERR_TIMEOUT, and later waits of the launch return at once.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "qhd.h"
#include "qhd_group.h"
#include "qhd_spectrum.h"
#include "qhd_trace.h"
#include "qhd_kernels.h"
#include "qhd_plane.cuh"
#include "qhd_prep.cuh"

namespace qhd {

constexpr int GROUP_CL = 8;                      // CTAs per cluster of the launch
constexpr int GROUP_MAX_CTX = 8;
constexpr int GROUP_MAX_CHUNKS = 16;             // chunks of steps per evolve call
constexpr int GROUP_PREP_STEPS = 16;             // step rows per prep item
constexpr unsigned GROUP_WAIT_LIMIT = 1u << 20;  // polls of ~256 ns: a few hundred ms

struct GroupClass {
    PrepArgs prep;               // this chunk's schedule tables of the context
    PlaneArgs plane;             // whole-run arguments (pot, kt, twx, ...)
    int n, sub;                  // square edge; CTAs per instance
    int64_t prep_first, prep_count;
    int64_t inst_first, inst_count;  // items of GROUP_CL / sub instances each
    unsigned prep_expected;      // arrivals that complete the tables: prep_count * GROUP_CL
};

struct GroupArgs {
    const GroupClass *cls;       // [n_cls], device memory
    int n_cls;
    int64_t n_items;
    unsigned *queue;             // next item (zeroed before the launch)
    unsigned *prep_done;         // [n_cls] arrivals (zeroed before the launch)
    unsigned *error;             // 1 once a wait gave up (sticky across launches)
    unsigned extra_wait;         // added to every expected count (failure-injection test; 0 otherwise)
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Step tables of prep item k of context c: rows [k S, k S + S) of the chunk's
// cnt + 1 potential rows and cnt kinetic rows, spread over the cluster.
__device__ __noinline__ void group_prep(const GroupArgs &a, const GroupClass &g, int c, int64_t k, int crank) {
    const PrepArgs &pa = g.prep;
    const int64_t j_lo = k * GROUP_PREP_STEPS;
    const int64_t j_hi = min(j_lo + (int64_t)GROUP_PREP_STEPS, pa.cnt + 1);
    const int64_t tid = (int64_t)crank * PLANE_THREADS + threadIdx.x;
    const int64_t nth = (int64_t)GROUP_CL * PLANE_THREADS;
    uint64_t kt_turns[3];
    double kt_fd[3];
    for (int64_t i = tid; i < (j_hi - j_lo) * pa.batch; i += nth)
        prep_coefficients(pa, j_lo + i / pa.batch, i % pa.batch, kt_turns, kt_fd, true);
    // kinetic rows (jl, b) of steps jl < cnt: CTA crank takes rows crank, crank + CL, ...
    __shared__ uint64_t s_k[3];
    __shared__ double s_fd[3];
    const int64_t k_hi = min(j_hi, pa.cnt);
    const int64_t rows = k_hi > j_lo ? (k_hi - j_lo) * pa.kt_batch : 0;
    for (int64_t r = crank; r < rows; r += GROUP_CL) {
        const int64_t jl = j_lo + r / pa.kt_batch, b = r % pa.kt_batch;
        if (threadIdx.x == 0) prep_coefficients(pa, jl, b, s_k, s_fd, false);
        __syncthreads();
        for (int i = threadIdx.x; i < pa.ksum; i += PLANE_THREADS) prep_kinetic_entry(pa, jl, b, i, s_k, s_fd);
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(a.prep_done + c, 1u);
}

template <int N, int C>
__device__ __forceinline__ void group_run(const PlaneArgs &pa, int64_t b, bool live, int grp, int r, float2 *tile,
                                          float4 *ptab, cg::cluster_group &cluster) {
    uint32_t tiles[C];
#pragma unroll
    for (int q = 0; q < C; ++q) tiles[q] = cluster_addr(tile, (uint32_t)(grp * C + q));
    plane_whole_run<N, N, C, 1>(pa, b, r, tiles, ptab, tile, live, cluster);
}

// Instance item k of context c: wait for its tables, then every step of the
// chunk for instances k * (CL / sub) + grp, grp = 0 .. CL / sub - 1.
__device__ __forceinline__ void group_instance(const GroupArgs &a, const GroupClass &g, int c, int64_t k, int crank,
                               cg::cluster_group &cluster, float2 *tile, float4 *ptab) {
    if (threadIdx.x == 0) {
        const unsigned need = g.prep_expected + a.extra_wait;
        unsigned it = 0;
        while (ld_acquire_u32(a.prep_done + c) < need) {
            if (ld_acquire_u32(a.error) != 0u) break;  // an earlier wait of this launch gave up
            if (++it >= GROUP_WAIT_LIMIT) {
                atomicExch(a.error, 1u);
                break;
            }
            __nanosleep(256);
        }
    }
    // the item's arguments live in shared memory, like kernel parameters in the
    // constant bank: the whole-run engine reads them there instead of holding
    // them in registers
    __shared__ PlaneArgs s_pa;
    if (threadIdx.x == 0) s_pa = g.plane;
    __syncthreads();
    const int sub = g.sub, per = GROUP_CL / sub;
    const int grp = crank / sub, r = crank % sub;
    const int64_t b = k * per + grp;
    const bool live = b < s_pa.batch;
    const int64_t bb = live ? b : s_pa.batch - 1;  // idle CTAs read a valid instance's tables
    switch (g.n * 16 + sub) {
    case 64 * 16 + 2: group_run<64, 2>(s_pa, bb, live, grp, r, tile, ptab, cluster); break;
    case 64 * 16 + 4: group_run<64, 4>(s_pa, bb, live, grp, r, tile, ptab, cluster); break;
    case 64 * 16 + 8: group_run<64, 8>(s_pa, bb, live, grp, r, tile, ptab, cluster); break;
    case 128 * 16 + 4: group_run<128, 4>(s_pa, bb, live, grp, r, tile, ptab, cluster); break;
    case 128 * 16 + 8: group_run<128, 8>(s_pa, bb, live, grp, r, tile, ptab, cluster); break;
    case 256 * 16 + 8: group_run<256, 8>(s_pa, bb, live, grp, r, tile, ptab, cluster); break;
    default: break;  // rejected on the host
    }
    __syncthreads();  // s_pa is rewritten by the next item
}

template <int MINB>
__global__ void __launch_bounds__(PLANE_THREADS, MINB) k_group(GroupArgs a) {
    extern __shared__ __align__(16) float4 smem4[];
    float4 *ptab = smem4;
    float2 *tile = reinterpret_cast<float2 *>(smem4 + PHASE_TAB);
    __shared__ unsigned s_item;
    cg::cluster_group cluster = cg::this_cluster();
    const int crank = (int)cluster.block_rank();
    const uint32_t item_src = cluster_addr(&s_item, 0);
    for (;;) {
        if (crank == 0 && threadIdx.x == 0) s_item = atomicAdd(a.queue, 1u);
        cluster.sync();
        unsigned item;
        asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(item) : "r"(item_src) : "memory");
        cluster.sync();  // every CTA holds its copy before rank 0 claims the next item
        if ((int64_t)item >= a.n_items) break;
        int c = 0;
        bool prep = false;
        int64_t k = 0;
        for (; c < a.n_cls; ++c) {
            const GroupClass &g = a.cls[c];
            if ((int64_t)item >= g.prep_first && (int64_t)item < g.prep_first + g.prep_count) {
                prep = true;
                k = (int64_t)item - g.prep_first;
                break;
            }
            if ((int64_t)item >= g.inst_first && (int64_t)item < g.inst_first + g.inst_count) {
                k = (int64_t)item - g.inst_first;
                break;
            }
        }
        if (c == a.n_cls) continue;  // cannot happen: the items tile [0, n_items)
        if (prep) group_prep(a, a.cls[c], c, k, crank);
        else group_instance(a, a.cls[c], c, k, crank, cluster, tile, ptab);
    }
}

// Shared memory of one CTA for a (edge, CTAs per instance) class.
static size_t class_smem(int n, int sub) {
    switch (n * 16 + sub) {
    case 64 * 16 + 2: return PlaneCfg<64, 64, 2>::SMEM;
    case 64 * 16 + 4: return PlaneCfg<64, 64, 4>::SMEM;
    case 64 * 16 + 8: return PlaneCfg<64, 64, 8>::SMEM;
    case 128 * 16 + 4: return PlaneCfg<128, 128, 4>::SMEM;
    case 128 * 16 + 8: return PlaneCfg<128, 128, 8>::SMEM;
    case 256 * 16 + 8: return PlaneCfg<256, 256, 8>::SMEM;
    default: return 0;
    }
}

static void *group_kernel(int min_blocks) {
    return min_blocks == 1 ? (void *)k_group<1> : (void *)k_group<2>;
}

static cudaLaunchConfig_t group_launch_config(int clusters, size_t smem, cudaStream_t s, cudaLaunchAttribute *attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(clusters * GROUP_CL), 1, 1);
    cfg.blockDim = dim3(PLANE_THREADS, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = GROUP_CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

}  // namespace qhd

using namespace qhd;

struct qhd_group {
    std::vector<qhd_ctx *> ctxs;
    std::vector<int> sub;            // CTAs per instance per context
    std::vector<int> edge;           // mesh edge per context
    int min_blocks = 2;
    int clusters = 0;
    size_t smem = 0;
    cudaStream_t stream = nullptr;   // the contexts' (caller's) stream
    cudaStream_t own = nullptr;      // private stream the graph is captured and replayed on
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    char *work = nullptr;
    GroupClass *d_cls = nullptr;     // [GROUP_MAX_CHUNKS][n_ctx]
    unsigned *d_count = nullptr;     // [GROUP_MAX_CHUNKS][1 + n_ctx] queue and arrivals
    unsigned *d_error = nullptr;
    float4 *d_twx = nullptr;         // [n_ctx][256] exchange twiddles for the chosen sub
    std::vector<GroupClass> h_cls;
    unsigned extra_wait = 0;
    cudaGraphExec_t exec = nullptr;
    std::string key;
    int64_t launches = 0, captures = 0;
    qhd_status sticky = QHD_OK;
    std::string err;
    ~qhd_group() {
        if (exec) cudaGraphExecDestroy(exec);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (own) cudaStreamDestroy(own);
    }
};

namespace {

constexpr size_t GROUP_TWX = 256;

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct GroupLayout {
    size_t cls, count, error, twx, total;
};

GroupLayout group_layout(int n_ctx) {
    GroupLayout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L.cls = take(sizeof(GroupClass) * (size_t)GROUP_MAX_CHUNKS * (size_t)n_ctx);
    L.count = take(sizeof(unsigned) * (size_t)GROUP_MAX_CHUNKS * (size_t)(1 + n_ctx));
    L.error = take(sizeof(unsigned));
    L.twx = take(sizeof(float4) * GROUP_TWX * (size_t)n_ctx);
    L.total = off;
    return L;
}

qhd_status gfail(qhd_group *g, qhd_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (g) {
        g->err = buf;
        if (s == QHD_ERR_CUDA || s == QHD_ERR_TIMEOUT) g->sticky = s;
    }
    return s;
}

#define QHD_GCUDA(g, call)                                                                      \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return gfail((g), QHD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

bool edge_ok(int64_t n) { return n == 64 || n == 128 || n == 256; }

int default_sub(int64_t n) { return n == 256 ? 8 : n == 128 ? 4 : 2; }

bool sub_ok(int64_t n, int sub) { return class_smem((int)n, sub) != 0; }

}  // namespace

extern "C" {

size_t qhd_group_workspace_bytes(int n_ctx) {
    if (n_ctx < 1 || n_ctx > GROUP_MAX_CTX) return 0;
    return group_layout(n_ctx).total;
}

qhd_status qhd_group_create(qhd_group **out, qhd_ctx *const *ctxs, int n_ctx, const qhd_group_config *cfg,
                            void *work_dev, size_t work_bytes) {
    if (!out || !ctxs || n_ctx < 1 || n_ctx > GROUP_MAX_CTX) return QHD_ERR_INVALID_ARG;
    const GroupLayout L = group_layout(n_ctx);
    if (!work_dev || ((uintptr_t)work_dev & 255) || work_bytes < L.total) return QHD_ERR_WORKSPACE;
    qhd_group_config c{};
    if (cfg) c = *cfg;
    if (c.min_blocks == 0) c.min_blocks = 2;
    if (c.min_blocks != 1 && c.min_blocks != 2) return QHD_ERR_INVALID_ARG;
    if (c.clusters < 0) return QHD_ERR_INVALID_ARG;
    qhd_group *g = new qhd_group();
    g->min_blocks = c.min_blocks;
    cudaStream_t stream = nullptr;
    for (int i = 0; i < n_ctx; ++i) {
        GroupCtxView v{};
        if (!ctxs[i] || ctx_group_view(ctxs[i], &v) != QHD_OK) {
            delete g;
            return QHD_ERR_STATE;
        }
        for (int j = 0; j < i; ++j)
            if (ctxs[j] == ctxs[i]) {
                delete g;
                return QHD_ERR_INVALID_ARG;
            }
        if (v.ndim != 2 || v.n[0] != v.n[1] || !edge_ok(v.n[0]) || !v.whole_run) {
            delete g;
            return QHD_ERR_UNSUPPORTED;
        }
        if (i == 0) stream = v.stream;
        else if (v.stream != stream) {
            delete g;
            return QHD_ERR_INVALID_ARG;
        }
        const int idx = v.n[0] == 64 ? 0 : v.n[0] == 128 ? 1 : 2;
        // default: the context's own split, so the group runs its arithmetic
        const int sub = c.sub_cluster[idx] ? c.sub_cluster[idx] : (v.plane_c ? v.plane_c : default_sub(v.n[0]));
        if (!sub_ok(v.n[0], sub)) {
            delete g;
            return QHD_ERR_INVALID_ARG;
        }
        g->ctxs.push_back(ctxs[i]);
        g->sub.push_back(sub);
        g->edge.push_back((int)v.n[0]);
        g->smem = std::max(g->smem, class_smem((int)v.n[0], sub));
    }
    g->stream = stream;
    g->work = (char *)work_dev;
    g->d_cls = (GroupClass *)(g->work + L.cls);
    g->d_count = (unsigned *)(g->work + L.count);
    g->d_error = (unsigned *)(g->work + L.error);
    g->d_twx = (float4 *)(g->work + L.twx);
    // exchange twiddles of the distributed axis for the chosen split N = sub * R:
    // twx[q * R + j] = exp(-2 pi i j q / N), FP32 hi/lo from FP64
    std::vector<float4> twx(GROUP_TWX * (size_t)n_ctx, make_float4(0.f, 0.f, 0.f, 0.f));
    for (int i = 0; i < n_ctx; ++i) {
        const int64_t n = g->edge[(size_t)i];
        const int sub = g->sub[(size_t)i], rr = (int)n / sub;
        for (int q = 0; q < sub; ++q)
            for (int j = 0; j < rr; ++j) {
                const double ang = 2.0 * 3.141592653589793238462643383279502884 *
                                   (double)(((int64_t)j * q) % n) / (double)n;
                const double cr = cos(ang), ci = -sin(ang);
                const float hr = (float)cr, hi = (float)ci;
                twx[(size_t)i * GROUP_TWX + (size_t)(q * rr + j)] =
                    make_float4(hr, hi, (float)(cr - (double)hr), (float)(ci - (double)hi));
            }
    }
    void *kern = group_kernel(g->min_blocks);
    // a stream of the group's own: the caller's stream may be one that cannot be
    // captured (the legacy default stream); events keep the two in order
    cudaError_t e = cudaStreamCreateWithFlags(&g->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_out, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g->smem);
    if (e == cudaSuccess) {
        if (c.clusters > 0) {
            g->clusters = c.clusters;
        } else {
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t lc = group_launch_config(1, g->smem, stream, attr);
            int nc = 0;
            e = cudaOccupancyMaxActiveClusters(&nc, kern, &lc);
            g->clusters = nc > 0 ? nc : 1;
        }
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->d_twx, twx.data(), twx.size() * sizeof(float4), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_error, 0, sizeof(unsigned), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        delete g;
        return QHD_ERR_CUDA;
    }
    *out = g;
    return QHD_OK;
}

qhd_status qhd_group_evolve(qhd_group *g, double T, double dt) {
    qhd::TraceRange trace("qhd_group_evolve");
    if (!g) return QHD_ERR_INVALID_ARG;
    if (g->sticky != QHD_OK) return g->sticky;
    if (!std::isfinite(T) || !std::isfinite(dt) || dt == 0.0)
        return gfail(g, QHD_ERR_INVALID_ARG, "T and dt must be finite and dt nonzero");
    const double ratio = T / dt, nr = std::nearbyint(ratio);
    if (!(nr >= 1.0) || std::fabs(ratio - nr) > 1e-9 * nr || nr > 1e12)
        return gfail(g, QHD_ERR_INVALID_ARG, "T/dt = %.17g is not a positive integer", ratio);
    const int64_t nsteps = (int64_t)nr;
    const int n_ctx = (int)g->ctxs.size();
    std::vector<GroupCtxView> views((size_t)n_ctx);
    int64_t chunk = int64_t(1) << 40;
    for (int i = 0; i < n_ctx; ++i) {
        qhd_status s = ctx_group_view(g->ctxs[(size_t)i], &views[(size_t)i]);
        if (s != QHD_OK) return gfail(g, s, "context %d: %s", i, qhd_last_error(g->ctxs[(size_t)i]));
        if (!views[(size_t)i].whole_run || views[(size_t)i].stream != g->stream)
            return gfail(g, QHD_ERR_STATE, "context %d changed transform or stream since qhd_group_create", i);
        chunk = std::min(chunk, views[(size_t)i].chunk);
    }
    const int64_t n_chunks = (nsteps + chunk - 1) / chunk;
    if (n_chunks > GROUP_MAX_CHUNKS)
        return gfail(g, QHD_ERR_UNSUPPORTED, "%lld steps need %lld table chunks (at most %d per call)",
                     (long long)nsteps, (long long)n_chunks, GROUP_MAX_CHUNKS);
    // the launch sequence depends on the steps, the contexts' clocks and tables
    char kb[160];
    std::string key;
    snprintf(kb, sizeof kb, "%.17g/%.17g/%u/", T, dt, g->extra_wait);
    key += kb;
    for (auto &v : views) {
        snprintf(kb, sizeof kb, "%.17g,%lld,%lld,%d,%d;", v.t, (long long)v.steps_done, (long long)v.kt_batch,
                 v.split, v.kinetic);
        key += kb;
    }
    if (key != g->key || !g->exec) {
        g->key.clear();
        g->h_cls.assign((size_t)(n_chunks * n_ctx), GroupClass{});
        std::vector<int64_t> n_items((size_t)n_chunks);
        for (int64_t q = 0; q < n_chunks; ++q) {
            const int64_t j0 = q * chunk, cnt = std::min(chunk, nsteps - j0);
            int64_t item = 0;
            for (int i = 0; i < n_ctx; ++i) {  // prep items first
                GroupClass &gc = g->h_cls[(size_t)(q * n_ctx + i)];
                gc.prep_first = item;
                gc.prep_count = (cnt + 1 + GROUP_PREP_STEPS - 1) / GROUP_PREP_STEPS;
                gc.prep_expected = (unsigned)(gc.prep_count * GROUP_CL);
                item += gc.prep_count;
            }
            for (int i = 0; i < n_ctx; ++i) {
                const GroupCtxView &v = views[(size_t)i];
                GroupClass &gc = g->h_cls[(size_t)(q * n_ctx + i)];
                const int sub = g->sub[(size_t)i], per = GROUP_CL / sub;
                gc.n = (int)v.n[0];
                gc.sub = sub;
                gc.inst_first = item;
                gc.inst_count = (v.batch + per - 1) / per;
                item += gc.inst_count;
                PrepArgs &pa = gc.prep;
                pa.sched = v.sched;
                pa.inst = v.inst;
                pa.pot = v.pot;
                pa.kt = v.kt;
                pa.kt_batch = v.kt_batch;
                pa.t_start = v.t;
                pa.dt = dt;
                pa.j0 = j0;
                pa.cnt = cnt;
                pa.nsteps = nsteps;
                pa.batch = v.batch;
                pa.ndim = 2;
                for (int d = 0; d < 3; ++d) {
                    pa.n[d] = (int)v.n[d];
                    pa.len[d] = v.len[d];
                    pa.koff[d] = v.koff[d];
                }
                pa.ksum = v.ksum;
                pa.inv_g = 1.0 / (double)v.g;
                pa.split = v.split;
                pa.kinetic = v.kinetic;
                PlaneArgs &pl = gc.plane;
                pl.psi = v.psi;
                pl.fq = v.fq;
                pl.pot = v.pot;
                pl.kt = v.kt;
                pl.tw_row = v.tw_row;
                pl.twx = g->d_twx + (size_t)i * GROUP_TWX;
                pl.batch = v.batch;
                pl.cnt = (int)cnt;
                pl.final_phase = j0 + cnt == nsteps ? 1 : 0;
                pl.ksum = v.ksum;
                pl.dither_base = (uint64_t)(v.steps_done + j0);
                pl.ptab = v.ptab;
                pl.kt_batch = v.kt_batch;
            }
            n_items[(size_t)q] = item;
        }
        // the previous replay may still read the descriptors: upload in stream order
        QHD_GCUDA(g, cudaEventRecord(g->ev_in, g->stream));
        QHD_GCUDA(g, cudaStreamWaitEvent(g->own, g->ev_in, 0));
        QHD_GCUDA(g, cudaMemcpyAsync(g->d_cls, g->h_cls.data(), g->h_cls.size() * sizeof(GroupClass),
                                     cudaMemcpyHostToDevice, g->own));
        QHD_GCUDA(g, cudaStreamSynchronize(g->own));
        // capture: per chunk, zero the queue and arrival counters, then the launch
        cudaGraph_t graph = nullptr;
        QHD_GCUDA(g, cudaStreamBeginCapture(g->own, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        void *kern = group_kernel(g->min_blocks);
        for (int64_t q = 0; q < n_chunks && e == cudaSuccess; ++q) {
            unsigned *cnt = g->d_count + q * (1 + n_ctx);
            e = cudaMemsetAsync(cnt, 0, sizeof(unsigned) * (size_t)(1 + n_ctx), g->own);
            if (e != cudaSuccess) break;
            GroupArgs ga{};
            ga.cls = g->d_cls + q * n_ctx;
            ga.n_cls = n_ctx;
            ga.n_items = n_items[(size_t)q];
            ga.queue = cnt;
            ga.prep_done = cnt + 1;
            ga.error = g->d_error;
            ga.extra_wait = g->extra_wait;
            cudaLaunchAttribute attr[1];
            cudaLaunchConfig_t lc = group_launch_config(g->clusters, g->smem, g->own, attr);
            void *args[] = {&ga};
            e = cudaLaunchKernelExC(&lc, kern, args);
        }
        cudaError_t e2 = cudaStreamEndCapture(g->own, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) {
            if (g->exec) {
                cudaGraphExecUpdateResultInfo info;
                if (cudaGraphExecUpdate(g->exec, graph, &info) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphExecDestroy(g->exec);
                    g->exec = nullptr;
                }
            }
            if (!g->exec) e = cudaGraphInstantiate(&g->exec, graph, 0);
        }
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) return gfail(g, QHD_ERR_CUDA, "batched launch capture: %s", cudaGetErrorString(e));
        g->key = key;
        g->captures++;
    }
    QHD_GCUDA(g, cudaEventRecord(g->ev_in, g->stream));
    QHD_GCUDA(g, cudaStreamWaitEvent(g->own, g->ev_in, 0));
    QHD_GCUDA(g, cudaGraphLaunch(g->exec, g->own));
    QHD_GCUDA(g, cudaEventRecord(g->ev_out, g->own));
    QHD_GCUDA(g, cudaStreamWaitEvent(g->stream, g->ev_out, 0));
    g->launches += n_chunks;
    for (auto *c : g->ctxs) ctx_advance(c, nsteps, dt);
    return QHD_OK;
}

qhd_status qhd_group_status(qhd_group *g) {
    if (!g) return QHD_ERR_INVALID_ARG;
    if (g->sticky != QHD_OK) return g->sticky;
    unsigned err = 0;
    QHD_GCUDA(g, cudaMemcpyAsync(&err, g->d_error, sizeof err, cudaMemcpyDeviceToHost, g->stream));
    QHD_GCUDA(g, cudaStreamSynchronize(g->stream));
    if (err) {
        for (auto *c : g->ctxs) ctx_fail(c, QHD_ERR_TIMEOUT, "a batched launch gave up waiting for its step tables");
        return gfail(g, QHD_ERR_TIMEOUT, "a wait for the step tables gave up; the states are not valid");
    }
    return QHD_OK;
}

qhd_status qhd_group_inject_wait_timeout(qhd_group *g, int on) {
    if (!g) return QHD_ERR_INVALID_ARG;
    if (g->sticky != QHD_OK) return g->sticky;
    g->extra_wait = on ? 1u : 0u;
    return QHD_OK;
}

qhd_status qhd_group_info(const qhd_group *g, int64_t *out) {
    if (!g || !out) return QHD_ERR_INVALID_ARG;
    out[0] = g->clusters;
    out[1] = g->min_blocks;
    out[2] = (int64_t)g->smem;
    out[3] = g->launches;
    out[4] = g->captures;
    for (size_t i = 0; i < 3; ++i) out[5 + i] = 0;
    for (size_t i = 0; i < g->ctxs.size(); ++i) {
        const int idx = g->edge[i] == 64 ? 0 : g->edge[i] == 128 ? 1 : 2;
        out[5 + idx] = g->sub[i];
    }
    return QHD_OK;
}

const char *qhd_group_last_error(const qhd_group *g) { return g ? g->err.c_str() : ""; }

qhd_status qhd_group_destroy(qhd_group *g) {
    if (!g) return QHD_OK;
    cudaError_t e = cudaStreamSynchronize(g->own);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    delete g;
    return e == cudaSuccess ? QHD_OK : QHD_ERR_CUDA;
}

}  // extern "C"
