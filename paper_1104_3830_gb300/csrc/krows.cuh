// krows.cuh -- one instance of the batched form on one block of 256 threads, on the
// per-step matrix K (Sec. 4.1.2 iteration in log coordinates, Sec. 4.2 stop rule, the
// deformed warm start of Sec. 4.1 between p steps).  Used by the batched launch
// (sa_batch_scale's K rows path) and by the server's device-resident request queue.
//
// K rows path: the larger instances (n <= 128 CH) one per block of 256 threads, on the
// per-step matrix K of the step path in a global-memory slot of the block (n x ceil(n/4)*4
// FP32, read from L2 in the sweeps).  Warp w owns rows w, w + 8, ... and evaluates and
// reads them itself; lane l owns the 16-byte column chunks l, l + 32, ... of every row, with
// their column factors c_j and column partial sums in registers.  A row sum is then one
// warp reduction (no block barrier per row), and a sweep has one block barrier: the
// warps' column partials meet in shared memory (two buffers by sweep parity), and every
// warp finalises the columns of its lanes from them, so all warps hold the same new c and
// the same residual without a second barrier.  Error independent of p, as on the step
// path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "log2pair.cuh"
#include "sa_internal.h"

namespace sa {

constexpr int kKrowsThreads = 256;

// Shared state of one block (static shared memory, 44.6 KB at CH = 4).
template <int CH>
struct KrowsSmem {
    static constexpr int NW = kKrowsThreads / 32;
    static constexpr int NMAX = 128 * CH;
    float4 l2tab[256];              // log2 table of the float-pair logarithm
    float colpart[2][NW][NMAX];     // the warps' column partials, by sweep parity
    float Cr[NMAX], srow[NMAX];     // row references and row sums
    double Vd[NMAX];                // column potentials, log2 units
    int badk[NW], bad[2][NW];
};

// The block's log2 table; a __syncthreads() must follow before the first instance.
template <int CH>
__device__ __forceinline__ void krows_init(KrowsSmem<CH>& sm) {
    for (int j = threadIdx.x; j < 256; j += kKrowsThreads) sm.l2tab[j] = log2_tab_entry(j);
}

// Scales the instance w (n x n, n <= 128 CH, row pitch ld elements) through the schedule
// P[0..n_p) with the stop rule max_j |S_j - 1| <= tol and at most max_sweeps sweeps per p,
// using K (n x ceil(n/4)*4 floats of global memory, this block's own).  All threads of
// the block call it.  On return the row and column potentials (natural units) are in Uo,
// Vo (not written when the instance lost all mass in a row or column), thread 0 has
// written the sweeps done and the status (0 converged, 1 a step hit max_sweeps,
// -6 non-finite), and the block has passed a barrier.
template <typename WT, int CH>
__device__ __forceinline__ void krows_instance(KrowsSmem<CH>& sm, const WT* wb, int n, int64_t ld,
                                               const double* P, int n_p, double tol, int max_sweeps,
                                               float* K, double* Uo, double* Vo, int32_t* sweeps_out,
                                               int32_t* status_out) {
    constexpr int NT = kKrowsThreads, NW = NT / 32;
    constexpr int M = 4 * CH;           // columns per lane
    constexpr int NMAX = 128 * CH;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    float4* s_l2tab = sm.l2tab;
    auto& colpart = sm.colpart;
    float* Cr = sm.Cr;
    float* srow = sm.srow;
    double* Vd = sm.Vd;
    int* s_badk = sm.badk;
    auto& s_bad = sm.bad;
    // V's FP32 head and tail during the evaluation of K, in the (then idle) partial sums
    float* vhi = &colpart[0][0][0];
    float* vlo = vhi + NMAX;
    const int NC = (n + 3) / 4;
    const int ldk = NC * 4;
    for (int j = tid; j < NMAX; j += NT) Vd[j] = 0.0;
    float c[M];
    int sweeps_all = 0;
    bool bad = false, capped = false;
    __syncthreads();
    for (int k = 0; k < n_p && !bad; ++k) {
        const double p = P[k];
        const double f = k > 0 ? p / P[k - 1] : 1.0;
        for (int j = tid; j < NMAX; j += NT) {
            const double v = Vd[j] * f;
            Vd[j] = v;
            const float h = (float)v;
            vhi[j] = h;
            vlo[j] = (float)(v - (double)h);
        }
        __syncthreads();
        // ---- one evaluation of K for this p: warp w evaluates its own rows ----
        const float ph = (float)p;
        const float pl = (float)(p - (double)ph);
        int badw = 0;
        for (int i = wid; i < n; i += NW) {
            const WT* wr = wb + (int64_t)i * ld;
            int wv[M];
            float m = -INFINITY;
#pragma unroll
            for (int kk = 0; kk < CH; ++kk) {
                const int c4 = lane + 32 * kk;
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = 4 * c4 + e;
                    wv[4 * kk + e] = j < n ? (int)wr[j] : 0;
                    if (wv[4 * kk + e] > 0) m = fmaxf(m, fmaf(ph, lg2_approx((float)wv[4 * kk + e]), -vhi[j]));
                }
            }
            m = warp_max(m);
            if (!(m > -INFINITY)) { badw = 1; m = 0.0f; }
            if (lane == 0) Cr[i] = m;
            float* kr = K + (size_t)i * ldk;
#pragma unroll
            for (int kk = 0; kk < CH; ++kk) {
                const int c4 = lane + 32 * kk;
                if (c4 >= NC) continue;
                float kv[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = 4 * c4 + e;
                    const int w = wv[4 * kk + e];
                    float x = 0.0f;
                    if (w > 0) {
                        const float2 lw = wlog2(s_l2tab, w);
                        const float t = ph * lw.x;
                        const float te = fmaf(ph, lw.x, -t);
                        float e1, e2;
                        const float u1 = two_sum(t, -vhi[j], &e1);
                        const float u2 = two_sum(u1, -m, &e2);
                        const float rest = ((te + e1) + e2) + (fmaf(ph, lw.y, pl * lw.x) - vlo[j]);
                        x = ex2_approx(u2 + rest);
                    }
                    kv[e] = x;
                }
                *(float4*)(kr + 4 * c4) = make_float4(kv[0], kv[1], kv[2], kv[3]);
            }
        }
        if (lane == 0) s_badk[wid] = badw;
#pragma unroll
        for (int kk = 0; kk < CH; ++kk)
#pragma unroll
            for (int e = 0; e < 4; ++e) c[4 * kk + e] = 4 * (lane + 32 * kk) + e < n ? 1.0f : 0.0f;
        __syncthreads();
#pragma unroll
        for (int x = 0; x < NW; ++x) bad = bad || s_badk[x] != 0;
        // ---- sweeps ----
        int sweeps = 0;
        bool done = bad;
        while (!done) {
            const int par = sweeps & 1;
            float S[M];
#pragma unroll
            for (int x = 0; x < M; ++x) S[x] = 0.0f;
            int badr = 0;
            // the warp's next row is loaded while the current one is reduced (its rows follow
            // one another, each waiting for the previous row's sum)
            float4 nx[CH];
            auto load_row = [&](int i) {
                const float* kr = K + (size_t)i * ldk;
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    const int c4 = lane + 32 * kk;
                    nx[kk] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (c4 < NC && i < n) nx[kk] = __ldcg((const float4*)(kr + 4 * c4));
                }
            };
            load_row(wid);
            for (int i = wid; i < n; i += NW) {
                float kv[M];
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    kv[4 * kk] = nx[kk].x;
                    kv[4 * kk + 1] = nx[kk].y;
                    kv[4 * kk + 2] = nx[kk].z;
                    kv[4 * kk + 3] = nx[kk].w;
                }
                load_row(i + NW);
                float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
                for (int kk = 0; kk < CH; ++kk) {
                    a0 = fmaf(kv[4 * kk], c[4 * kk], a0);
                    a1 = fmaf(kv[4 * kk + 1], c[4 * kk + 1], a1);
                    a0 = fmaf(kv[4 * kk + 2], c[4 * kk + 2], a0);
                    a1 = fmaf(kv[4 * kk + 3], c[4 * kk + 3], a1);
                }
                const float sv = warp_sum(a0 + a1);
                if (!(sv >= 0x1p-120f && sv <= 0x1p120f)) badr = 1;
                if (lane == 0) srow[i] = sv;
                const float inv = rcp_approx(sv);
#pragma unroll
                for (int x = 0; x < M; ++x) S[x] = fmaf(kv[x], inv, S[x]);
            }
#pragma unroll
            for (int kk = 0; kk < CH; ++kk) {
                const int c4 = lane + 32 * kk;
                *(float4*)&colpart[par][wid][4 * c4] =
                    make_float4(S[4 * kk], S[4 * kk + 1], S[4 * kk + 2], S[4 * kk + 3]);
            }
            if (lane == 0) s_bad[par][wid] = badr;
            __syncthreads();
            // every warp finalises the columns of its lanes from all warps' partials
            float resid = 0.0f;
            int badc = 0;
#pragma unroll
            for (int kk = 0; kk < CH; ++kk) {
                const int c4 = lane + 32 * kk;
                float4 t = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
                for (int x = 0; x < NW; ++x) {
                    const float4 q = *(const float4*)&colpart[par][x][4 * c4];
                    t.x += q.x;
                    t.y += q.y;
                    t.z += q.z;
                    t.w += q.w;
                }
                const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (4 * c4 + e >= n) continue;
                    const float Sj = c[4 * kk + e] * tv[e];
                    if (!(Sj > 0.0f) || !(Sj < INFINITY)) badc = 1;
                    resid = fmaxf(resid, fabsf(Sj - 1.0f));
                    c[4 * kk + e] = __fdividef(c[4 * kk + e], Sj);
                }
            }
            resid = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(resid)));
            bool anybad = __any_sync(0xffffffffu, badc != 0);
#pragma unroll
            for (int x = 0; x < NW; ++x) anybad = anybad || s_bad[par][x] != 0;
            ++sweeps;
            bad = anybad;
            done = bad || (resid <= (float)tol) || (sweeps >= max_sweeps);
            if (done && !bad && !(resid <= (float)tol)) capped = true;
        }
        sweeps_all += sweeps;
        if (bad) break;
        // potentials reached at this p: V_j <- V_j - log2 c_j (warp 0 for every column)
        if (wid == 0) {
#pragma unroll
            for (int kk = 0; kk < CH; ++kk)
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = 4 * (lane + 32 * kk) + e;
                    if (j < n) Vd[j] -= log2((double)c[4 * kk + e]);
                }
        }
        __syncthreads();
    }
    if (!bad) {
        for (int i = tid; i < n; i += NT) Uo[i] = ((double)Cr[i] + log2((double)srow[i])) * kLn2;
        for (int j = tid; j < n; j += NT) Vo[j] = Vd[j] * kLn2;
    }
    if (tid == 0) {
        *sweeps_out = sweeps_all;
        *status_out = bad ? -6 : (capped ? 1 : 0);
    }
    __syncthreads();   // shared state is rewritten by the next instance
}

}  // namespace sa
