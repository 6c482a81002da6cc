// qhd_plane.cuh -- cluster-resident plane engine.
//
// A plane of N1 x N2 points (the last two axes of a 3-D grid for one index of
// axis 0, or a whole 2-D instance) is held in the shared memory of a cluster of
// C CTAs: CTA r owns R = N1 / C consecutive rows.  The row transforms (axis of
// length N2) run locally with the line engine; the transform along the
// distributed axis is a four-step factorisation N1 = C * R:
//
//   forward  y[k1][n2] = W_N1^{n2 k1} sum_{n1} x[R n1 + n2] W_C^{n1 k1}   (across the cluster)
//            X[k1 + C k2] = sum_{n2} y[k1][n2] W_R^{n2 k2}                 (local, CTA k1, row k2)
//   inverse  the same two steps in reverse order with conjugate factors.
//
// So in Fourier space CTA r's local row k2 holds frequency r + C k2 along the
// distributed axis.  The cross-cluster step reads the C values at one local
// position (n2, c) from every CTA through distributed shared memory, and one
// thread owns each position cluster-wide, so the inverse step, the potential
// phase (diagonal in position space) and the forward step are fused with no
// barrier between them: two cluster barriers per Strang step.
#pragma once
#include <cooperative_groups.h>
#include <type_traits>

#include "qhd_device.cuh"

namespace qhd {

namespace cg = cooperative_groups;

constexpr int PLANE_THREADS = 256;

template <int N1, int N2, int C> struct PlaneCfg {
    static constexpr int R = N1 / C;                      // rows per CTA
    using RowC = LineCfg<N2>;
    static constexpr int S = line_stride<N2>(true, 0);     // row stride in float2 (>= padded row)
    static constexpr int T2 = RowC::T, E2 = RowC::E;
    static constexpr int ROWS_PER_ITER = PLANE_THREADS / T2;
    static constexpr int PAIRS = (R / C) * N2;            // exchange positions owned per CTA
    static constexpr size_t SMEM = PHASE_TAB * sizeof(float4) + (size_t)R * S * sizeof(float2);
    static_assert(RowC::TWO_STAGE, "rows of at least 32 points");
    static_assert(N1 % C == 0 && R % C == 0, "R rows per CTA, R/C exchange rows per CTA");
    static_assert(N2 <= PLANE_THREADS, "one thread per column in the column phase");
    static_assert(R <= 32, "local column transform held in registers");
    static_assert((R * T2) % 32 == 0, "whole warps in the row phase");
    static_assert(S % 2 == 0, "16-byte aligned rows");
};

// Global <-> shared copy of this CTA's R rows (contiguous in global memory).
// Global -> shared uses 16-byte asynchronous copies so that the whole tile is
// in flight at once; the caller waits with plane_copy_wait().
template <int N1, int N2, int C, bool TO_SHARED>
__device__ __forceinline__ void plane_copy(float2 *tile, float2 *g) {
    using P = PlaneCfg<N1, N2, C>;
    constexpr int Q = P::R * N2 / 2;  // float4 chunks
#pragma unroll 4
    for (int i = threadIdx.x; i < Q; i += PLANE_THREADS) {
        const int row = (2 * i) / N2, col = (2 * i) % N2;
        float2 *s = tile + row * P::S + col;
        float2 *d = g + (int64_t)row * N2 + col;
        if (TO_SHARED) {
            const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(d) : "memory");
        } else {
            *reinterpret_cast<float4 *>(d) = *reinterpret_cast<const float4 *>(s);
        }
    }
    if (TO_SHARED) asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void plane_copy_wait() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
}

// Local transform along the distributed axis: each column of the CTA's R rows.
template <int N1, int N2, int C, bool INV>
__device__ __forceinline__ void plane_columns(float2 *tile) {
    using P = PlaneCfg<N1, N2, C>;
    const int c = threadIdx.x;
    if (c < N2) {
        float2 v[P::R];
#pragma unroll
        for (int r = 0; r < P::R; ++r) v[r] = tile[r * P::S + c];
        dft<P::R, INV>(v);
#pragma unroll
        for (int r = 0; r < P::R; ++r) tile[r * P::S + c] = v[r];
    }
}

// Row transforms along N2.  KIN: forward, kinetic phase, inverse (2-D whole
// run); otherwise one direction.  The row's own storage is the exchange buffer
// of the line engine (its content is in registers at that point).
struct WarpSyncP {
    __device__ __forceinline__ void operator()() const { __syncwarp(); }
};

template <int N1, int N2, int C, int DIR>  // DIR: 0 forward, 1 inverse, 2 forward-kinetic-inverse
__device__ __forceinline__ void plane_rows(float2 *tile, const float4 *__restrict__ tw_row, const float4 *kt0,
                                           const float4 *kt1, int rank) {
    using P = PlaneCfg<N1, N2, C>;
    constexpr int T2 = P::T2, E2 = P::E2;
    const int t = threadIdx.x % T2;
    // zero-mode split (qhd_device.cuh): the row transform is the last forward
    // transform before the kinetic factor, and local row 0 of rank 0 (frequency
    // 0 along the distributed axis) holds the global zero mode.  Its T2 threads
    // (lanes 0..T2-1 of warp 0, the ones that transform it below) take the mean
    // out of the shared-memory row before the row loop and add the mean's part
    // back after it, so the loop itself is the same for every row.
    const bool zrow = DIR == 2 && rank == 0 && (int)threadIdx.x < T2;
    float2 mean_part = make_float2(0.f, 0.f);
    if (zrow) {
        float2 v[E2];
#pragma unroll
        for (int e = 0; e < E2; ++e) v[e] = tile[t + T2 * e];
        const float2 sum = line_sum_lanes<E2, T2>(v, T2 >= 32 ? 0xffffffffu : (1u << T2) - 1u);
        sub_line_mean<N2, E2>(v, sum);
#pragma unroll
        for (int e = 0; e < E2; ++e) tile[t + T2 * e] = v[e];
        const float4 k0 = kt0[0], k1 = kt1[0];
        const float2 y = cmul_comp(sum, make_float2(k0.x, k0.y), make_float2(k0.z, k0.w));
        mean_part = cmul_comp(y, make_float2(k1.x, k1.y), make_float2(k1.z, k1.w));
    }
#pragma unroll 1
    for (int base = 0; base < P::R; base += P::ROWS_PER_ITER) {
        const int row = base + threadIdx.x / T2;
        if (row < P::R) {
            float2 *rp = tile + row * P::S;
            float2 x[E2];
#pragma unroll
            for (int e = 0; e < E2; ++e) x[e] = rp[t + T2 * e];
            __syncwarp();
            if (DIR == 1) {
                line_fft<N2, true>(x, rp, t, tw_row, WarpSyncP{});
            } else {
                line_fft<N2, false>(x, rp, t, tw_row, WarpSyncP{});
                if (DIR == 2) {
                    // this local row holds frequency rank + C * row along the distributed axis
                    // plain (coherent) loads: the batched persistent kernel writes
                    // these tables earlier in the same launch
                    const float4 k0 = kt0[rank + C * row];
#pragma unroll
                    for (int e = 0; e < E2; ++e) {
                        const float4 k1 = kt1[t + T2 * e];
                        float2 y = cmul_comp(x[e], make_float2(k0.x, k0.y), make_float2(k0.z, k0.w));
                        x[e] = cmul_comp(y, make_float2(k1.x, k1.y), make_float2(k1.z, k1.w));
                    }
                    line_fft<N2, true>(x, rp, t, tw_row, WarpSyncP{});
                }
            }
#pragma unroll
            for (int e = 0; e < E2; ++e) rp[t + T2 * e] = x[e];
        }
    }
    if (zrow) {
#pragma unroll
        for (int e = 0; e < E2; ++e) tile[t + T2 * e] = cadd(tile[t + T2 * e], mean_part);
    }
}

// Number of exchange positions (n2, c) each thread owns.
template <int N1, int N2, int C> __host__ __device__ constexpr int plane_ppt() {
    return (PlaneCfg<N1, N2, C>::PAIRS + PLANE_THREADS - 1) / PLANE_THREADS;
}

// Distributed shared memory through explicit cluster addresses: mapa gives the
// address of the same shared location in CTA `rank`; ld/st.shared::cluster
// access it without the generic-address path.
__device__ __forceinline__ uint32_t cluster_addr(const void *local, uint32_t rank) {
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"((uint32_t)__cvta_generic_to_shared(local)), "r"(rank));
    return r;
}
__device__ __forceinline__ float2 ld_cluster(uint32_t addr) {
    float2 v;
    asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(addr) : "memory");
    return v;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, float2 v) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// One exchange position (n2, c): the C values are in v, the fixed-point
// potential of the C rows in fv.
template <int N1, int N2, int C>
__device__ __forceinline__ void plane_exchange_math(float2 *v, const uint32_t *fv, int n2, bool inv, bool phase,
                                                    bool fwd, const float4 *__restrict__ twx, uint64_t coef,
                                                    uint32_t dither, const float4 *ptab) {
    constexpr int R = PlaneCfg<N1, N2, C>::R;
    if (inv) {
#pragma unroll
        for (int q = 1; q < C; ++q) {
            const float4 w = __ldg(&twx[q * R + n2]);
            v[q] = cmulc_comp(v[q], make_float2(w.x, w.y), make_float2(w.z, w.w));
        }
        dft<C, true>(v);
    }
    if (phase) {
#pragma unroll
        for (int q = 0; q < C; ++q)
            v[q] = apply_phase_tab(v[q], turns_mul(coef, fv[q]) + dither, ptab);
    }
    if (fwd) {
        dft<C, false>(v);
#pragma unroll
        for (int q = 1; q < C; ++q) {
            const float4 w = __ldg(&twx[q * R + n2]);
            v[q] = cmul_comp(v[q], make_float2(w.x, w.y), make_float2(w.z, w.w));
        }
    }
}

// The cross-cluster step over the positions this CTA owns, INF positions at a
// time so that their INF * C remote loads (and potential loads) are in flight
// before the arithmetic (INF is chosen per kernel by register budget).  base[q] = cluster address of CTA q's tile; fq: this
// plane's fixed-point potential.
template <int N1, int N2, int C, int INF>
__device__ __forceinline__ void plane_exchange(const uint32_t *base, int rank, bool inv, bool phase, bool fwd,
                                               const float4 *__restrict__ twx, const uint32_t *__restrict__ fq,
                                               uint64_t coef, uint32_t dither, const float4 *ptab) {
    using P = PlaneCfg<N1, N2, C>;
    constexpr int R = P::R;
    constexpr int PPT = plane_ppt<N1, N2, C>();
#pragma unroll
    for (int k0 = 0; k0 < PPT; k0 += INF) {
        float2 v[INF][C];
        uint32_t fv[INF][C];
        int n2[INF], c[INF];
        bool live[INF];
#pragma unroll
        for (int h = 0; h < INF; ++h) {
            const int k = k0 + h;
            const int p = threadIdx.x + k * PLANE_THREADS;
            live[h] = k < PPT && p < P::PAIRS;
            n2[h] = rank * (R / C) + (live[h] ? p : 0) / N2;
            c[h] = (live[h] ? p : 0) % N2;
            if (live[h]) {
                const uint32_t off = (uint32_t)((n2[h] * P::S + c[h]) * sizeof(float2));
#pragma unroll
                for (int q = 0; q < C; ++q) v[h][q] = ld_cluster(base[q] + off);
                if (phase) {
#pragma unroll
                    for (int q = 0; q < C; ++q) fv[h][q] = __ldg(&fq[(R * q + n2[h]) * N2 + c[h]]);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < INF; ++h) {
            if (!live[h]) continue;
            plane_exchange_math<N1, N2, C>(v[h], fv[h], n2[h], inv, phase, fwd, twx, coef, dither, ptab);
            const uint32_t off = (uint32_t)((n2[h] * P::S + c[h]) * sizeof(float2));
#pragma unroll
            for (int q = 0; q < C; ++q) st_cluster(base[q] + off, v[h][q]);
        }
    }
}

// Every step of a chunk for one 2-D instance b held by the C CTAs whose
// cluster addresses are tiles[0..C) (rank = this CTA's index among them): per
// step the cross-cluster exchange with the potential phase, then the local
// transforms with the kinetic phase in between.  psi touches global memory only
// at the chunk's start and end.  live = false runs the same steps (and cluster
// barriers) on whatever the tile holds and touches no global memory but the
// tables and the potential of instance b (which must be a valid index), so
// idle CTAs of a shared cluster keep the barrier count of their partners.
template <int N1, int N2, int C, int INF>
__device__ __forceinline__ void plane_whole_run(const PlaneArgs &a, int64_t b, int rank, const uint32_t *tiles,
                                                float4 *ptab, float2 *tile, bool live, cg::cluster_group &cluster) {
    using P = PlaneCfg<N1, N2, C>;
    float2 *g = a.psi + b * (int64_t)N1 * N2 + (int64_t)rank * P::R * N2;
    const uint32_t *fqr = a.fq + b * (int64_t)N1 * N2;
    if (live) plane_copy<N1, N2, C, true>(tile, g);
    load_phase_tab(ptab, a.ptab);
    plane_copy_wait();
    cluster.sync();
#pragma unroll 1
    for (int j = 0; j < a.cnt; ++j) {
        const uint64_t coef = a.pot[(int64_t)j * a.batch + b];
        plane_exchange<N1, N2, C, INF>(tiles, rank, j > 0, true, true, a.twx, fqr, coef,
                                       step_dither(a.dither_base + (uint64_t)j), ptab);
        cluster.sync();
        plane_columns<N1, N2, C, false>(tile);
        __syncthreads();
        const float4 *kb = a.kt + ((int64_t)j * a.kt_batch + (a.kt_batch == 1 ? 0 : b)) * a.ksum;
        plane_rows<N1, N2, C, 2>(tile, a.tw_row, kb, kb + N1, rank);
        __syncthreads();
        plane_columns<N1, N2, C, true>(tile);
        cluster.sync();
    }
    const uint64_t coef = a.pot[(int64_t)a.cnt * a.batch + b];
    plane_exchange<N1, N2, C, INF>(tiles, rank, a.cnt > 0, a.final_phase != 0, false, a.twx, fqr, coef, 0u, ptab);
    cluster.sync();
    if (live) plane_copy<N1, N2, C, false>(tile, g);
}

}  // namespace qhd
