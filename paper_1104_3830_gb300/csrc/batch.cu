// batch.cu -- many independent small instances (n <= 512) scaled in one persistent
// launch: each thread block pulls instances from a queue (largest first) and runs the
// whole p schedule of an instance on chip (Sec. 4.1.2 iteration, Sec. 4.2 stop rule).
//
// Layout inside a block: warp w owns rows w, w + NW, ...; lane l owns the 16-byte column
// chunks l, l + 32, ... of every row.  A row sum is one warp reduction (no block barrier
// per row); column partial sums stay in the lane's registers for the whole sweep and are
// combined across warps once per sweep through shared memory.  The per-element formula
// and the FP32/FP64 split are those of the single-instance fused kernel:
//   t_ij = 2^(p (L_ij - Lr_i) - Vh_j) * c_j,  L = log2 w,  U_i = p Lr_i + log2 s_i,
//   V_j += log2 S_j (FP64),  residual = max_j |S_j - 1| (FP64).
// If the instance's log2 table (n^2 FP32) fits in shared memory it is computed once per
// instance and the sweeps read it (one SFU exp2 per element); otherwise the sweeps read
// the weights from global memory (L2-resident after the first sweep) and take log2 too.
// Two blocks run on each SM (128 registers a thread, 110 KB of shared memory a block, so
// the table fits up to n = 142): a sweep of a small instance is mostly the latency of its
// block-wide reductions, which the other block's instance hides.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "krows.cuh"
#include "log2pair.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kBatchMaxN = 512;

struct BatchArgs {
    const void* const* w;
    const int32_t* n;
    const int64_t* ld;
    const int64_t* off;
    const int32_t* order;   // instance indices, largest n first
    int k;
    int i16;
    const double* P;
    int n_p;
    double tol;
    int max_sweeps;
    double* U;              // natural units on output
    double* V;
    int32_t* sweeps;        // per instance
    int32_t* status;        // per instance: 0 ok, 1 not converged, -6 nonfinite
    unsigned* queue;        // work counter
    size_t smem_table;      // bytes available for the log2 table
    float* kscr;            // K rows path: a global slot of K per block
    size_t kscr_floats;     // floats of one block's slot
};

template <typename WT, int NT, int KC>
__global__ void __launch_bounds__(NT, 2) batch_kernel(BatchArgs A) {
    constexpr int NW = NT / 32;
    constexpr int VEC = 16 / sizeof(WT);
    constexpr int M = KC * VEC;   // columns per lane
    extern __shared__ __align__(16) unsigned char smem[];
    double* Vd = (double*)smem;                              // [512]
    float* Vh = (float*)(Vd + kBatchMaxN);                   // [512]
    float* Vc = Vh + kBatchMaxN;                             // [512]
    float* Lr = Vc + kBatchMaxN;                             // [512]
    float* srow = Lr + kBatchMaxN;                           // [512]
    float* colpart = srow + kBatchMaxN;                      // [NW][512]
    double* red = (double*)(colpart + NW * kBatchMaxN);      // [NW]
    float* Ltab = (float*)(red + NW);                        // [n * npad] when it fits
    __shared__ int s_inst, s_bad, s_stat;

    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (;;) {
        if (tid == 0) {
            const unsigned q = atomicAdd(A.queue, 1u);
            s_inst = q < (unsigned)A.k ? A.order[q] : -1;
            s_bad = 0;
            s_stat = 0;
        }
        __syncthreads();
        const int inst = s_inst;
        if (inst < 0) break;
        const int n = A.n[inst];
        const int64_t ld = A.ld[inst];
        const int NC = (n + VEC - 1) / VEC;
        const int npad = NC * VEC;
        const bool use_tab = (size_t)n * npad * 4 <= A.smem_table;
        const unsigned char* wb = (const unsigned char*)A.w[inst];
        const size_t pitch = (size_t)ld * sizeof(WT);
        double* Uo = A.U + A.off[inst];
        double* Vo = A.V + A.off[inst];
        if (use_tab) {
            for (int e = tid; e < n * npad; e += NT) {
                const int i = e / npad, j = e % npad;
                float L = -INFINITY;
                if (j < n) L = lg2_approx((float)((const WT*)(wb + (size_t)i * pitch))[j]);
                Ltab[e] = L;
            }
        }
        for (int j = tid; j < n; j += NT) { Vd[j] = 0.0; Vh[j] = 0.0f; Vc[j] = 1.0f; }
        for (int i = tid; i < n; i += NT) { Lr[i] = 0.0f; srow[i] = 1.0f; }
        __syncthreads();
        int sweeps_all = 0;
        bool capped = false;
        for (int k = 0; k < A.n_p; ++k) {
            const double p = A.P[k];
            const float pf = (float)p;
            if (k > 0) {
                const double pp = A.P[k - 1];
                const double f = p / pp;
                for (int i = tid; i < n; i += NT) {
                    const double u = pp * (double)Lr[i] + log2((double)srow[i]);   // U at p[k-1]
                    Lr[i] = (float)(u / pp);
                    srow[i] = (float)exp2(u - pp * (double)Lr[i]);
                }
                for (int j = tid; j < n; j += NT) {
                    const double v = Vd[j] * f;
                    Vd[j] = v;
                    Vh[j] = (float)v;
                    Vc[j] = ex2_approx((float)(v - (double)(float)v));
                }
                __syncthreads();
            }
            int sweeps = 0;
            bool done = false;
            while (!done) {
                float S[M], vh[M], vc[M];
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    S[m] = 0.0f;
                    const int j = (lane + 32 * (m / VEC)) * VEC + m % VEC;
                    vh[m] = j < n ? Vh[j] : 0.0f;
                    vc[m] = j < n ? Vc[j] : 0.0f;
                }
                for (int i = wid; i < n; i += NW) {
                    const float lr = Lr[i];
                    float L[M];
#pragma unroll
                    for (int kk = 0; kk < KC; ++kk) {
                        const int c = lane + 32 * kk;
#pragma unroll
                        for (int e = 0; e < VEC; ++e) L[kk * VEC + e] = -INFINITY;
                        if (c < NC) {
                            if (use_tab) {
                                const float4* src = (const float4*)(Ltab + (size_t)i * npad + c * VEC);
#pragma unroll
                                for (int h = 0; h < VEC / 4; ++h) {
                                    const float4 a = src[h];
                                    L[kk * VEC + 4 * h] = a.x;
                                    L[kk * VEC + 4 * h + 1] = a.y;
                                    L[kk * VEC + 4 * h + 2] = a.z;
                                    L[kk * VEC + 4 * h + 3] = a.w;
                                }
                            } else {
                                const uint4 q = *(const uint4*)(wb + (size_t)i * pitch + (size_t)c * 16);
                                const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
                                if (VEC == 8) {
#pragma unroll
                                    for (int h = 0; h < 4; ++h) {
                                        L[kk * VEC + 2 * h] = lg2_approx(lo16_to_float(wd[h]));
                                        L[kk * VEC + 2 * h + 1] = lg2_approx(hi16_to_float(wd[h]));
                                    }
                                } else {
#pragma unroll
                                    for (int h = 0; h < 4; ++h) L[kk * VEC + h] = lg2_approx((float)(int)wd[h]);
                                }
                            }
                        }
                    }
                    float t[M];
                    float sp = 0.0f;
#pragma unroll
                    for (int m = 0; m < M; ++m) {
                        const int j = (lane + 32 * (m / VEC)) * VEC + m % VEC;
                        const float tv = j < n ? ex2_approx(fmaf(pf, L[m] - lr, -vh[m])) * vc[m] : 0.0f;
                        t[m] = tv;
                        sp += tv;
                    }
                    const float s = warp_sum(sp);
                    if (s >= 0x1p-100f && s <= 0x1p100f) {
                        const float inv = 1.0f / s;
#pragma unroll
                        for (int m = 0; m < M; ++m) S[m] = fmaf(t[m], inv, S[m]);
                        if (lane == 0) srow[i] = s;
                    } else {
                        // stale shift: exact max shift for this row (warp-local)
                        float mx = -INFINITY;
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            const int j = (lane + 32 * (m / VEC)) * VEC + m % VEC;
                            const float ev = (j < n && vc[m] > 0.0f) ? fmaf(pf, L[m] - lr, -vh[m]) + log2f(vc[m]) : -INFINITY;
                            t[m] = ev;
                            mx = fmaxf(mx, ev);
                        }
                        mx = warp_max(mx);
                        float s2 = 0.0f;
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            t[m] = mx > -INFINITY ? ex2_approx(t[m] - mx) : 0.0f;
                            s2 += t[m];
                        }
                        s2 = warp_sum(s2);
                        if (!(mx > -INFINITY) || !(s2 > 0.0f)) { s_bad = 1; s2 = 1.0f; }
                        const float inv = 1.0f / s2;
#pragma unroll
                        for (int m = 0; m < M; ++m) S[m] = fmaf(t[m], inv, S[m]);
                        if (lane == 0) {
                            const double un = p * (double)lr + (double)mx + log2((double)s2);
                            const float lrn = (float)(un / p);
                            Lr[i] = lrn;
                            srow[i] = (float)exp2(un - p * (double)lrn);
                        }
                    }
                }
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const int j = (lane + 32 * (m / VEC)) * VEC + m % VEC;
                    if (j < n) colpart[wid * kBatchMaxN + j] = S[m];
                }
                __syncthreads();
                double rmax = 0.0;
                for (int j = tid; j < n; j += NT) {
                    double Sj = 0.0;
                    for (int x = 0; x < NW; ++x) Sj += (double)colpart[x * kBatchMaxN + j];
                    if (!(Sj > 0.0) || !isfinite(Sj)) { s_bad = 1; Sj = 1.0; }
                    const double d = Sj - 1.0;
                    rmax = fmax(rmax, fabs(d));
                    const double lg = fabs(d) < 1e-3
                                          ? d * (1.0 + d * (-0.5 + d * (1.0 / 3.0 + d * (-0.25 + d * 0.2)))) * kLog2e
                                          : log2(Sj);
                    const double v = Vd[j] + lg;
                    Vd[j] = v;
                    float h = Vh[j];
                    if (fabs((double)h - v) > 16.0) { h = (float)v; Vh[j] = h; }
                    Vc[j] = ex2_approx((float)((double)h - v));
                }
                rmax = warp_max(rmax);
                if (lane == 0) red[wid] = rmax;
                __syncthreads();
                double r = 0.0;
                for (int x = 0; x < NW; ++x) r = fmax(r, red[x]);
                ++sweeps;
                const bool bad = s_bad != 0;
                done = bad || (r <= A.tol) || (sweeps >= A.max_sweeps);
                if (done && !bad && !(r <= A.tol)) capped = true;
                __syncthreads();
            }
            sweeps_all += sweeps;
            if (s_bad) break;
        }
        const double pl = A.P[A.n_p - 1];
        for (int i = tid; i < n; i += NT) Uo[i] = (pl * (double)Lr[i] + log2((double)srow[i])) * kLn2;
        for (int j = tid; j < n; j += NT) Vo[j] = Vd[j] * kLn2;
        if (tid == 0) {
            A.sweeps[inst] = sweeps_all;
            A.status[inst] = s_bad ? -6 : (capped ? 1 : 0);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// Group path: a group of G warps (G = 1, 2, 4) scales one small instance (n <= NMAX <= 128)
// on its own, with no block barrier in its sweeps.  The instances of these sizes run the
// most sweeps of a batch (on uniform weights at p = 128 most n <= 32 instances end at the
// sweep cap), so the latency of one sweep, not arithmetic, sets their time; a few warps
// each and many groups per SM keep that latency small and hidden.
//
// Per p step the group evaluates the step matrix of the per-step path once,
//     K_ij = 2^(p log2 w_ij - C_i - V_j)       (C_i ~ max_j (p log2 w_ij - V_j)),
// with the same float-pair exponent (log2 w to about 2^-40, exact two-products and
// two-sums, one SFU exp2), into its shared-memory slot; the sweeps then only multiply
// and add (Sec. 4.1.2 iteration on the diagonally equivalent K, error independent of p):
//     s_i = sum_j K_ij c_j,   S_j = c_j sum_i K_ij / s_i,   c_j <- c_j / S_j,
// residual max_j |S_j - 1| (Sec. 4.2), and at the end of the step U_i = C_i + log2 s_i,
// V_j <- V_j - log2 c_j in FP64.  Thread t of the group owns rows and columns t, t + 32G,
// ...; the row pass reads K by rows (slot rows padded to an odd stride: conflict-free), the
// column pass by columns, the vectors c and 1/s are broadcast from the slot, and the loops
// run over NMAX (compile time, fully unrolled) so that each pass issues its loads at once.
// Sums use four independent FP32 accumulators of at most NMAX/4 terms each.  The group's
// warps meet at a named barrier (one per group of the block) twice a sweep; a group of one
// warp only synchronises the warp.
// ---------------------------------------------------------------------------------------
constexpr int kGroupMaxN = 128;

// floats of one group's slot for instances with n <= nmax: K (n4 x (n4 + 1)), then c, 1/s,
// C (nmax each), V as float pairs (2 nmax) and the warps' residuals (8)
__host__ __device__ inline unsigned group_slot_floats(int nmax) {
    const unsigned n4 = (unsigned)((nmax + 3) & ~3);
    return ((n4 * (n4 + 1) + 3u) & ~3u) + 5u * n4 + 8u;
}

template <int G>
__device__ __forceinline__ void group_sync(int group) {
    if (G == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(32 * G) : "memory");
    }
}

// group barrier that also returns whether `pred` holds in every thread of the group (the
// barrier's own reduction: no shared-memory round of partial results)
template <int G>
__device__ __forceinline__ bool group_sync_and(int group, bool pred) {
    if (G == 1) return __all_sync(0xffffffffu, pred);
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, %3, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)pred), "r"(group + 1), "r"(32 * G)
        : "memory");
    return r != 0;
}

template <typename WT, int G, int NMAX>
__global__ void __launch_bounds__(256) batch_group_kernel(BatchArgs A) {
    constexpr int NT = 32 * G;                  // threads of a group
    constexpr int RPT = (NMAX + NT - 1) / NT;   // rows (and columns) per thread
    constexpr int N4 = (NMAX + 3) & ~3;
    constexpr int CPL = (N4 + 31) / 32;         // columns per lane in the evaluation of K
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float4 s_l2tab[256];
    const int tid = threadIdx.x;
    for (int j = tid; j < 256; j += blockDim.x) s_l2tab[j] = log2_tab_entry(j);
    __syncthreads();   // the only block barrier: the groups are independent from here on
    const int group = tid / NT, tg = tid % NT, lane = tid & 31, wig = tg >> 5;
    float* K = (float*)smem + (size_t)group * group_slot_floats(NMAX);
    float* cs = K + ((N4 * (N4 + 1) + 3) & ~3);
    float* rs = cs + N4;
    float* Cs = rs + N4;
    float2* vp = (float2*)(Cs + N4);
    float* wres = (float*)(vp + N4);
    __shared__ int s_q[8];
    for (;;) {
        if (tg == 0) s_q[group] = (int)atomicAdd(A.queue, 1u);
        group_sync<G>(group);
        const int q = s_q[group];
        group_sync<G>(group);   // s_q is rewritten by the next instance
        if (q >= A.k) break;
        const int inst = A.order[q];
        const int n = A.n[inst];
        const int n4 = (n + 3) & ~3;
        const int stride = n4 + 1;   // odd: the threads' rows fall in distinct banks
        const WT* wb = (const WT*)A.w[inst];
        const int64_t ld = A.ld[inst];
        double V[RPT];               // log2 units, columns tg + r NT
        float c[RPT], sr[RPT];       // column factors; last row sums of rows tg + r NT
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            V[r] = 0.0;
            c[r] = 0.0f;
            sr[r] = 1.0f;
        }
        int sweeps_all = 0;
        bool bad = false, capped = false;
        for (int k = 0; k < A.n_p && !bad; ++k) {
            const double p = A.P[k];
            if (k > 0) {
                const double f = p / A.P[k - 1];
#pragma unroll
                for (int r = 0; r < RPT; ++r) V[r] *= f;
            }
            // ---- one evaluation of K for this p ----
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int j = tg + r * NT;
                if (j < N4) {
                    const float h = (float)V[r];
                    vp[j] = make_float2(h, (float)(V[r] - (double)h));
                }
            }
            group_sync<G>(group);
            const float ph = (float)p;
            const float pl = (float)(p - (double)ph);
            int badk = 0;
            for (int i = wig; i < n; i += G) {   // a row per warp, lanes over its columns
                const WT* wr = wb + (int64_t)i * ld;
                int wv[CPL];
                float m = -INFINITY;
#pragma unroll
                for (int h = 0; h < CPL; ++h) {
                    const int j = lane + 32 * h;
                    wv[h] = j < n ? (int)wr[j] : 0;
                    // reference C ~ max_j (p log2 w - V_j), an FP32 estimate (only a scale:
                    // C enters the row potential exactly)
                    if (wv[h] > 0) m = fmaxf(m, fmaf(ph, lg2_approx((float)wv[h]), -vp[j].x));
                }
                m = warp_max(m);
                if (!(m > -INFINITY)) { badk = 1; m = 0.0f; }
                if (lane == 0) Cs[i] = m;
                float* kr = K + (size_t)i * stride;
#pragma unroll
                for (int h = 0; h < CPL; ++h) {
                    const int j = lane + 32 * h;
                    float x = 0.0f;
                    if (wv[h] > 0) {
                        // p log2 w - V_j - m with 48-bit operands: the large parts cancel
                        // exactly (two-product, two-sums), the small ones are added after
                        const float2 lw = wlog2(s_l2tab, wv[h]);
                        const float2 vj = vp[j];
                        const float t = ph * lw.x;
                        const float te = fmaf(ph, lw.x, -t);
                        float e1, e2;
                        const float u1 = two_sum(t, -vj.x, &e1);
                        const float u2 = two_sum(u1, -m, &e2);
                        const float rest = ((te + e1) + e2) + (fmaf(ph, lw.y, pl * lw.x) - vj.y);
                        x = ex2_approx(u2 + rest);
                    }
                    if (j < n4) kr[j] = x;
                }
            }
            for (int i = n + wig; i < n4; i += G)   // zero rows up to the multiple of four
#pragma unroll
                for (int h = 0; h < CPL; ++h)
                    if (lane + 32 * h < n4) K[(size_t)i * stride + lane + 32 * h] = 0.0f;
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int j = tg + r * NT;
                c[r] = j < n ? 1.0f : 0.0f;
                if (j < N4) {
                    cs[j] = c[r];
                    rs[j] = 0.0f;
                }
            }
            if (lane == 0) wres[wig] = (float)badk;
            group_sync<G>(group);
#pragma unroll
            for (int x = 0; x < G; ++x) bad = bad || wres[x] != 0.0f;
            float Cr[RPT];
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int i = tg + r * NT;
                Cr[r] = i < n ? Cs[i] : 0.0f;
            }
            group_sync<G>(group);   // wres is rewritten by the sweeps
            // ---- sweeps ----
            int sweeps = 0;
            bool done = bad;
            while (!done) {
                // row pass: s_i = sum_j K_ij c_j for the thread's rows
                int badr = 0;
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int i = tg + r * NT;
                    if (i < n) {
                        const float* kr = K + (size_t)i * stride;
                        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
                        for (int j = 0; j < N4; j += 4) {
                            if (j < n4) {
                                const float4 c4 = *(const float4*)(cs + j);
                                a0 = fmaf(kr[j], c4.x, a0);
                                a1 = fmaf(kr[j + 1], c4.y, a1);
                                a2 = fmaf(kr[j + 2], c4.z, a2);
                                a3 = fmaf(kr[j + 3], c4.w, a3);
                            }
                        }
                        const float sv = (a0 + a1) + (a2 + a3);
                        if (!(sv >= 0x1p-120f && sv <= 0x1p120f)) badr = 1;
                        sr[r] = sv;
                        rs[i] = rcp_approx(sv);
                    }
                }
                group_sync<G>(group);
                // column pass: S_j = c_j sum_i K_ij / s_i for the thread's columns
                float resid = 0.0f;
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int j = tg + r * NT;
                    if (j < n) {
                        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
                        for (int i = 0; i < N4; i += 4) {
                            if (i < n4) {
                                const float4 r4 = *(const float4*)(rs + i);
                                const float* kc = K + (size_t)i * stride + j;
                                a0 = fmaf(kc[0], r4.x, a0);
                                a1 = fmaf(kc[stride], r4.y, a1);
                                a2 = fmaf(kc[2 * stride], r4.z, a2);
                                a3 = fmaf(kc[3 * stride], r4.w, a3);
                            }
                        }
                        const float S = c[r] * ((a0 + a1) + (a2 + a3));
                        if (!(S > 0.0f) || !(S < INFINITY)) badr = 1;
                        resid = fmaxf(resid, fabsf(S - 1.0f));
                        c[r] = c[r] / S;
                        cs[j] = c[r];
                    }
                }
                // the group's residual (and failure flag, as a NaN) from every warp
                resid = warp_max(badr ? INFINITY : resid);
                if (G > 1 && lane == 0) wres[wig] = resid;
                group_sync<G>(group);
                if (G > 1) {
                    resid = 0.0f;
#pragma unroll
                    for (int x = 0; x < G; ++x) resid = fmaxf(resid, wres[x]);
                }
                ++sweeps;
                bad = !(resid < INFINITY);
                done = bad || (resid <= (float)A.tol) || (sweeps >= A.max_sweeps);
                if (done && !bad && !(resid <= (float)A.tol)) capped = true;
                if (G > 1) group_sync<G>(group);   // wres is rewritten by the next sweep
            }
            sweeps_all += sweeps;
            if (bad) break;
            // potentials reached at this p: V_j <- V_j - log2 c_j; U from C and s at the end
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const int j = tg + r * NT;
                if (j < n) V[r] -= log2((double)c[r]);
            }
            if (k + 1 == A.n_p) {
                double* Uo = A.U + A.off[inst];
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int i = tg + r * NT;
                    if (i < n) Uo[i] = ((double)Cr[r] + log2((double)sr[r])) * kLn2;
                }
            }
        }
        double* Vo = A.V + A.off[inst];
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
            const int j = tg + r * NT;
            if (j < n) Vo[j] = V[r] * kLn2;
        }
        if (tg == 0) {
            A.sweeps[inst] = sweeps_all;
            A.status[inst] = bad ? -6 : (capped ? 1 : 0);
        }
        group_sync<G>(group);   // the slot is rewritten by the next instance
    }
}

// ---------------------------------------------------------------------------------------
// Register path: the group path with K held in registers during the sweeps.  A group of G
// warps (T = 32 G threads) takes n <= NMAX; each row q (and column q) of the padded NMAX x
// NMAX matrix belongs to P = T / NMAX adjacent lanes, lane part p holding the L = NMAX / P
// entries K_q,[pL, pL+L) of the row and K_[pL, pL+L),q of the column in registers (2 L <= 64
// floats).  A sweep then reads no K: the row pass multiplies the row part by the c of its
// columns (broadcast from shared memory) and adds the P parts with lane shuffles; the
// column pass does the same with 1/s; one group barrier after each pass publishes 1/s and
// c.  K is evaluated once per p step exactly as in the group path (same float-pair
// exponent), staged in shared memory and loaded into the registers.
// ---------------------------------------------------------------------------------------
template <int NMAX, int P>
__host__ __device__ inline unsigned regs_slot_floats() {
    constexpr unsigned L = NMAX / P;
    // staging K (NMAX x (NMAX + 1)), c and 1/s (P segments of L + 4), V pairs, C, flags
    return ((NMAX * (NMAX + 1) + 3u) & ~3u) + 2u * P * (L + 4) + 2u * NMAX + NMAX + 64u;
}

template <typename WT, int G, int NMAX>
__global__ void __launch_bounds__(512) batch_regs_kernel(BatchArgs A) {
    constexpr int NT = 32 * G;
    constexpr int P = NT / NMAX;   // lanes per row (and per column)
    constexpr int L = NMAX / P;    // entries of a row part
    constexpr int SEG = L + 4;     // padded segment of c and 1/s (parts in distinct banks)
    constexpr int CPL = NMAX / 32; // columns per lane in the evaluation of K
    static_assert(P >= 1 && P * NMAX == NT && L <= 32 && (P & (P - 1)) == 0 && P <= 32, "shape");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float4 s_l2tab[256];
    const int tid = threadIdx.x;
    for (int j = tid; j < 256; j += blockDim.x) s_l2tab[j] = log2_tab_entry(j);
    __syncthreads();   // the only block barrier: the groups are independent from here on
    const int group = tid / NT, tg = tid % NT, lane = tid & 31, wig = tg >> 5;
    const int q = tg / P, part = tg % P;   // row and column q, part `part`
    float* Kst = (float*)smem + (size_t)group * regs_slot_floats<NMAX, P>();
    float* cs = Kst + ((NMAX * (NMAX + 1) + 3) & ~3);
    float* rs = cs + P * SEG;
    float2* vp = (float2*)(rs + P * SEG);
    float* Cs = (float*)(vp + NMAX);
    float* wres = Cs + NMAX;                  // [G] per-warp flags of the evaluation of K
    int* s_q = (int*)(wres + 2 * G);
    int* s_bad = s_q + 1;                     // a row or column sum left the FP32 range
    constexpr int STR = NMAX + 1;
    const unsigned FULL = 0xffffffffu;
    for (;;) {
        if (tg == 0) *s_q = (int)atomicAdd(A.queue, 1u);
        group_sync<G>(group);
        const int qi = *s_q;
        group_sync<G>(group);   // s_q is rewritten by the next instance
        if (qi >= A.k) break;
        const int inst = A.order[qi];
        const int n = A.n[inst];
        const WT* wb = (const WT*)A.w[inst];
        const int64_t ld = A.ld[inst];
        double Vq = 0.0;           // column q's potential, log2 units (the same in every part)
        float cq = 0.0f, sq = 1.0f, Cq = 0.0f;
        float kr[L], kc[L];
        int sweeps_all = 0;
        bool bad = false, capped = false;
        for (int k = 0; k < A.n_p && !bad; ++k) {
            const double p = A.P[k];
            if (k > 0) Vq *= p / A.P[k - 1];
            // ---- one evaluation of K for this p, staged in shared memory ----
            if (part == 0) {
                const float h = (float)Vq;
                vp[q] = make_float2(h, (float)(Vq - (double)h));
            }
            group_sync<G>(group);
            const float ph = (float)p;
            const float pl = (float)(p - (double)ph);
            int badk = 0;
            for (int i = wig; i < NMAX; i += G) {   // a row per warp, lanes over its columns
                float* kr_s = Kst + (size_t)i * STR;
                if (i >= n) {
#pragma unroll
                    for (int h = 0; h < CPL; ++h) kr_s[lane + 32 * h] = 0.0f;
                    continue;
                }
                const WT* wr = wb + (int64_t)i * ld;
                int wv[CPL];
                float m = -INFINITY;
#pragma unroll
                for (int h = 0; h < CPL; ++h) {
                    const int j = lane + 32 * h;
                    wv[h] = j < n ? (int)wr[j] : 0;
                    if (wv[h] > 0) m = fmaxf(m, fmaf(ph, lg2_approx((float)wv[h]), -vp[j].x));
                }
                m = warp_max(m);
                if (!(m > -INFINITY)) { badk = 1; m = 0.0f; }
                if (lane == 0) Cs[i] = m;
#pragma unroll
                for (int h = 0; h < CPL; ++h) {
                    const int j = lane + 32 * h;
                    float x = 0.0f;
                    if (wv[h] > 0) {
                        const float2 lw = wlog2(s_l2tab, wv[h]);
                        const float2 vj = vp[j];
                        const float t = ph * lw.x;
                        const float te = fmaf(ph, lw.x, -t);
                        float e1, e2;
                        const float u1 = two_sum(t, -vj.x, &e1);
                        const float u2 = two_sum(u1, -m, &e2);
                        const float rest = ((te + e1) + e2) + (fmaf(ph, lw.y, pl * lw.x) - vj.y);
                        x = ex2_approx(u2 + rest);
                    }
                    kr_s[j] = x;
                }
            }
            if (lane == 0) wres[wig] = (float)badk;
            group_sync<G>(group);
#pragma unroll
            for (int x = 0; x < G; ++x) bad = bad || wres[x] != 0.0f;
#pragma unroll
            for (int l = 0; l < L; ++l) {
                kr[l] = Kst[(size_t)q * STR + part * L + l];
                kc[l] = Kst[(size_t)(part * L + l) * STR + q];
            }
            Cq = q < n ? Cs[q] : 0.0f;
            cq = q < n ? 1.0f : 0.0f;
            if (part == 0) {
                cs[(q / L) * SEG + q % L] = cq;
                rs[(q / L) * SEG + q % L] = 0.0f;   // rows beyond n keep 1/s = 0
            }
            if (tg == 0) *s_bad = 0;
            group_sync<G>(group);   // c published; wres and the staging area are reused
            // ---- sweeps ----
            int sweeps = 0;
            bool done = bad;
            while (!done) {
                // row pass: s_q = sum over the parts of K_q,part . c_part
                const float* cseg = cs + part * SEG;
                float a[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                for (int l = 0; l < L; l += 4) {
                    const float4 c4 = *(const float4*)(cseg + l);
                    a[(l / 4) & 7] = fmaf(kr[l], c4.x, a[(l / 4) & 7]);
                    a[(l / 4 + 2) & 7] = fmaf(kr[l + 1], c4.y, a[(l / 4 + 2) & 7]);
                    a[(l / 4 + 4) & 7] = fmaf(kr[l + 2], c4.z, a[(l / 4 + 4) & 7]);
                    a[(l / 4 + 6) & 7] = fmaf(kr[l + 3], c4.w, a[(l / 4 + 6) & 7]);
                }
                float sv = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
#pragma unroll
                for (int o = 1; o < P; o <<= 1) sv += __shfl_xor_sync(FULL, sv, o);
                int badr = 0;
                if (q < n) {
                    if (!(sv >= 0x1p-120f && sv <= 0x1p120f)) badr = 1;
                    sq = sv;
                    if (part == 0) rs[(q / L) * SEG + q % L] = rcp_approx(sv);
                }
                group_sync<G>(group);
                // column pass: S_q = c_q sum over the parts of K_part,q . (1/s)_part
                const float* rseg = rs + part * SEG;
#pragma unroll
                for (int x = 0; x < 8; ++x) a[x] = 0.0f;
#pragma unroll
                for (int l = 0; l < L; l += 4) {
                    const float4 r4 = *(const float4*)(rseg + l);
                    a[(l / 4) & 7] = fmaf(kc[l], r4.x, a[(l / 4) & 7]);
                    a[(l / 4 + 2) & 7] = fmaf(kc[l + 1], r4.y, a[(l / 4 + 2) & 7]);
                    a[(l / 4 + 4) & 7] = fmaf(kc[l + 2], r4.z, a[(l / 4 + 4) & 7]);
                    a[(l / 4 + 6) & 7] = fmaf(kc[l + 3], r4.w, a[(l / 4 + 6) & 7]);
                }
                float cv = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
#pragma unroll
                for (int o = 1; o < P; o <<= 1) cv += __shfl_xor_sync(FULL, cv, o);
                float resid = 0.0f;
                if (q < n) {
                    const float S = cq * cv;
                    if (!(S > 0.0f) || !(S < INFINITY)) badr = 1;
                    resid = fabsf(S - 1.0f);
                    cq = __fdividef(cq, S);
                    if (part == 0) cs[(q / L) * SEG + q % L] = cq;
                }
                // the group converged when every thread's residual is within tol (the
                // barrier's AND); a non-finite sum anywhere is flagged in shared memory
                // before the barrier and read after it
                if (badr) *s_bad = 1;
                const bool conv = group_sync_and<G>(group, !badr && resid <= (float)A.tol);
                ++sweeps;
                bad = G == 1 ? __any_sync(FULL, badr != 0) : *(volatile int*)s_bad != 0;
                done = bad || conv || (sweeps >= A.max_sweeps);
                if (done && !bad && !conv) capped = true;
            }
            sweeps_all += sweeps;
            if (bad) break;
            if (q < n) Vq -= log2((double)cq);
            if (k + 1 == A.n_p && part == 0 && q < n)
                A.U[A.off[inst] + q] = ((double)Cq + log2((double)sq)) * kLn2;
        }
        if (part == 0 && q < n) A.V[A.off[inst] + q] = Vq * kLn2;
        if (tg == 0) {
            A.sweeps[inst] = sweeps_all;
            A.status[inst] = bad ? -6 : (capped ? 1 : 0);
        }
        group_sync<G>(group);   // the slot is rewritten by the next instance
    }
}

// ---------------------------------------------------------------------------------------
// K rows path: the larger instances (n <= 128 CH) one per block of 256 threads (krows.cuh),
// each block on a global-memory slot of K of its own.
// ---------------------------------------------------------------------------------------
template <typename WT, int CH>
__global__ void __launch_bounds__(256, 2) batch_krows_kernel(BatchArgs A) {
    __shared__ KrowsSmem<CH> sm;
    __shared__ int s_inst;
    krows_init(sm);
    float* K = A.kscr + (size_t)blockIdx.x * A.kscr_floats;
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned q = atomicAdd(A.queue, 1u);
            s_inst = q < (unsigned)A.k ? A.order[q] : -1;
        }
        __syncthreads();
        const int inst = s_inst;
        if (inst < 0) break;
        krows_instance<WT, CH>(sm, (const WT*)A.w[inst], A.n[inst], A.ld[inst], A.P, A.n_p, A.tol, A.max_sweeps, K,
                               A.U + A.off[inst], A.V + A.off[inst], A.sweeps + inst, A.status + inst);
    }
}

}  // namespace
}  // namespace sa

using namespace sa;

namespace {
// group path: `per_block` groups of G warps per block, one slot of K each, as many blocks as
// fit on each SM, at most one group per instance
template <typename WT, int G, int NMAX>
sa_status launch_group(sa_ctx* ctx, cudaStream_t bs, const BatchArgs& args, int per_block) {
    auto kern = batch_group_kernel<WT, G, NMAX>;
    const size_t smem = (size_t)per_block * group_slot_floats(NMAX) * sizeof(float);
    cudaFuncAttributes fa;
    SA_CUDA(cudaFuncGetAttributes(&fa, kern));
    if (smem + fa.sharedSizeBytes > ctx->smem_optin) {
        set_error("batch group path: %d slots for n <= %d need %zu bytes of shared memory (%zu available)", per_block,
                  NMAX, smem + fa.sharedSizeBytes, ctx->smem_optin);
        return SA_E_UNSUPPORTED;
    }
    SA_CUDA(allow_dynamic_smem(kern, ctx->smem_optin));
    int per_sm = 0;
    SA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * G * per_block, smem));
    if (per_sm < 1) {
        set_error("batch group path: %d groups of %d warps (%zu bytes) do not fit on an SM", per_block, G, smem);
        return SA_E_UNSUPPORTED;
    }
    const int blocks = std::max(1, std::min((args.k + per_block - 1) / per_block, ctx->num_sms * per_sm));
    kern<<<blocks, 32 * G * per_block, smem, bs>>>(args);
    count_launch();
    SA_CUDA(cudaGetLastError());
    return SA_OK;
}

template <typename WT, int G>
sa_status launch_group_n(sa_ctx* ctx, cudaStream_t bs, const BatchArgs& args, int nmax, int per_block) {
    if (nmax <= 32) return launch_group<WT, G, 32>(ctx, bs, args, per_block);
    if (nmax <= 64) return launch_group<WT, G, 64>(ctx, bs, args, per_block);
    return launch_group<WT, G, 128>(ctx, bs, args, per_block);
}

// register path: `per_block` groups of G warps per block
template <typename WT, int G, int NMAX>
sa_status launch_regs(sa_ctx* ctx, cudaStream_t bs, const BatchArgs& args, int per_block) {
    constexpr int P = 32 * G / NMAX;
    auto kern = batch_regs_kernel<WT, G, NMAX>;
    const size_t smem = (size_t)per_block * regs_slot_floats<NMAX, P>() * sizeof(float);
    const int threads = 32 * G * per_block;
    cudaFuncAttributes fa;
    SA_CUDA(cudaFuncGetAttributes(&fa, kern));
    if (threads > fa.maxThreadsPerBlock || smem + fa.sharedSizeBytes > ctx->smem_optin) {
        set_error("batch register path: %d groups of %d warps for n <= %d do not fit a block (%d threads, %zu bytes)",
                  per_block, G, NMAX, threads, smem + fa.sharedSizeBytes);
        return SA_E_UNSUPPORTED;
    }
    SA_CUDA(allow_dynamic_smem(kern, ctx->smem_optin));
    int per_sm = 0;
    SA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
    if (per_sm < 1) {
        set_error("batch register path: %d groups of %d warps do not fit on an SM", per_block, G);
        return SA_E_UNSUPPORTED;
    }
    const int blocks = std::max(1, std::min((args.k + per_block - 1) / per_block, ctx->num_sms * per_sm));
    kern<<<blocks, threads, smem, bs>>>(args);
    count_launch();
    SA_CUDA(cudaGetLastError());
    return SA_OK;
}

// the register path's shapes: (warps per instance, largest n) with 2 L <= 64 registers of K
template <typename WT>
sa_status launch_regs_t(sa_ctx* ctx, cudaStream_t bs, const BatchArgs& args, int nmax, int warps, int per_block) {
    if (nmax <= 32 && warps == 1) return launch_regs<WT, 1, 32>(ctx, bs, args, per_block);
    if (nmax <= 32 && warps == 2) return launch_regs<WT, 2, 32>(ctx, bs, args, per_block);
    if (nmax <= 32 && warps == 4) return launch_regs<WT, 4, 32>(ctx, bs, args, per_block);
    if (nmax <= 64 && warps == 4) return launch_regs<WT, 4, 64>(ctx, bs, args, per_block);
    if (nmax <= 64 && warps == 8) return launch_regs<WT, 8, 64>(ctx, bs, args, per_block);
    if (nmax <= 128 && warps == 16) return launch_regs<WT, 16, 128>(ctx, bs, args, per_block);
    set_error("batch register path: no shape of %d warps for n = %d (1, 2 or 4 warps up to 32, 4 or 8 up to 64, "
              "16 up to 128)", warps, nmax);
    return SA_E_UNSUPPORTED;
}

sa_status launch_regs_path(sa_ctx* ctx, cudaStream_t bs, const BatchArgs& args, int nmax, int warps, int per_block,
                           sa_wtype wtype) {
    return wtype == SA_I16 ? launch_regs_t<int16_t>(ctx, bs, args, nmax, warps, per_block)
                           : launch_regs_t<int32_t>(ctx, bs, args, nmax, warps, per_block);
}

sa_status launch_group_path(sa_ctx* ctx, cudaStream_t bs, const BatchArgs& args, int nmax, int warps, int per_block,
                            sa_wtype wtype) {
    if (wtype == SA_I16) {
        if (warps == 1) return launch_group_n<int16_t, 1>(ctx, bs, args, nmax, per_block);
        if (warps == 2) return launch_group_n<int16_t, 2>(ctx, bs, args, nmax, per_block);
        return launch_group_n<int16_t, 4>(ctx, bs, args, nmax, per_block);
    }
    if (warps == 1) return launch_group_n<int32_t, 1>(ctx, bs, args, nmax, per_block);
    if (warps == 2) return launch_group_n<int32_t, 2>(ctx, bs, args, nmax, per_block);
    return launch_group_n<int32_t, 4>(ctx, bs, args, nmax, per_block);
}

// K rows path: one block of 256 threads per instance, two blocks per SM, a global slot of
// K per block (args.kscr, args.kscr_floats); `blocks` is the grid the slots were sized for
sa_status launch_krows_path(sa_ctx* ctx, cudaStream_t bs, const BatchArgs& args, int nmax, int blocks,
                            sa_wtype wtype) {
    auto go = [&](auto kern) -> sa_status {
        kern<<<blocks, 256, 0, bs>>>(args);
        count_launch();
        SA_CUDA(cudaGetLastError());
        return SA_OK;
    };
    if (wtype == SA_I16) {
        if (nmax <= 128) return go(batch_krows_kernel<int16_t, 1>);
        if (nmax <= 256) return go(batch_krows_kernel<int16_t, 2>);
        return go(batch_krows_kernel<int16_t, 4>);
    }
    if (nmax <= 128) return go(batch_krows_kernel<int32_t, 1>);
    if (nmax <= 256) return go(batch_krows_kernel<int32_t, 2>);
    return go(batch_krows_kernel<int32_t, 4>);
}

// block path: one block of 256 threads per instance, two blocks per SM
sa_status launch_block_path(sa_ctx* ctx, cudaStream_t bs, BatchArgs args, int maxn, sa_wtype wtype) {
    const int vec = 16 / wbytes(wtype);
    const int kc = ((maxn + vec - 1) / vec + 31) / 32;   // chunks per lane
    constexpr int NT = 256;
    constexpr int NW = NT / 32;
    const size_t fixed = kBatchMaxN * 8 + 4 * kBatchMaxN * 4 + (size_t)NW * kBatchMaxN * 4 + NW * 8 + 64;
    size_t smem = std::min<size_t>(ctx->smem_optin, 110 * 1024);   // two blocks per SM
    args.smem_table = smem > fixed ? smem - fixed : 0;
    auto go = [&](auto kern) -> sa_status {
        SA_CUDA(allow_dynamic_smem(kern, ctx->smem_optin));
        int per_sm = 0;
        SA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
        const int grid = std::max(1, std::min(args.k, ctx->num_sms * std::max(per_sm, 1)));
        kern<<<grid, NT, smem, bs>>>(args);
        count_launch();
        SA_CUDA(cudaGetLastError());
        return SA_OK;
    };
    if (wtype == SA_I16) return kc <= 1 ? go(batch_kernel<int16_t, NT, 1>) : go(batch_kernel<int16_t, NT, 2>);
    if (kc <= 1) return go(batch_kernel<int32_t, NT, 1>);
    if (kc <= 2) return go(batch_kernel<int32_t, NT, 2>);
    return go(batch_kernel<int32_t, NT, 4>);
}

// per-instance sweeps and statuses to the host; the call's status from the worst instance
sa_status finish_batch(cudaStream_t st, int k, const int32_t* d_sw, const int32_t* d_st, int32_t* sweeps,
                       int32_t* status) {
    std::vector<int32_t> hsw(k), hst(k);
    SA_CUDA(cudaMemcpyAsync(hsw.data(), d_sw, 4 * k, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(hst.data(), d_st, 4 * k, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaStreamSynchronize(st));
    if (sweeps) memcpy(sweeps, hsw.data(), 4 * k);
    if (status) memcpy(status, hst.data(), 4 * k);
    int worst = 0;
    for (int q = 0; q < k; ++q) {
        if (hst[q] < 0) worst = -6;
        else if (hst[q] > 0 && worst == 0) worst = 1;
    }
    if (worst < 0) { set_error("a batch instance lost all mass in a row or column"); return SA_E_NONFINITE; }
    if (worst > 0) { set_error("a batch instance hit max_sweeps_per_p"); return SA_E_NOT_CONVERGED; }
    return SA_OK;
}
}  // namespace

extern "C" sa_status sa_batch_scale(sa_ctx* ctx, int32_t k, const void* const* d_w, const int32_t* d_n,
                                    const int64_t* d_ld, const int64_t* d_off, sa_wtype wtype,
                                    const sa_scale_opts* o, double* d_u, double* d_v, int32_t* sweeps,
                                    int32_t* status) {
    if (!ctx || k <= 0 || !d_w || !d_n || !d_ld || !d_off || !o || !d_u || !d_v) {
        set_error("bad batch arguments");
        return SA_E_INVALID;
    }
    if (!o->p || o->n_p <= 0 || !(o->tol > 0) || o->max_sweeps_per_p <= 0) {
        set_error("bad batch schedule");
        return SA_E_INVALID;
    }
    for (int q = 0; q < o->n_p; ++q)
        if (!(o->p[q] > 0) || (q > 0 && !(o->p[q] > o->p[q - 1]))) {
            set_error("p schedule must be positive and increasing");
            return SA_E_INVALID;
        }
    cudaSetDevice(ctx->device);
    NvtxRange range("sa_batch_scale k=%d", k);
    cudaStream_t st = ctx->stream;
    std::vector<int32_t> hn(k);
    std::vector<int64_t> hld(k);
    SA_CUDA(cudaMemcpyAsync(hn.data(), d_n, 4 * k, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(hld.data(), d_ld, 8 * k, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaStreamSynchronize(st));
    const int sz = wbytes(wtype);
    for (int q = 0; q < k; ++q) {
        if (hn[q] <= 0 || hn[q] > kBatchMaxN) {
            set_error("batch instance %d has n=%d (supported 1..%d)", q, hn[q], kBatchMaxN);
            return SA_E_UNSUPPORTED;
        }
        if (((size_t)hld[q] * sz) % 16 != 0 || hld[q] < (int64_t)align_up((size_t)hn[q] * sz, 16) / sz) {
            set_error("batch instance %d: ld*sizeof(w) must be a multiple of 16 covering n", q);
            return SA_E_INVALID;
        }
    }
    // instances by bucket of the plan: group buckets smallest first (the smallest run the
    // most sweeps), block buckets largest first
    const sa_batch_plan& plan = ctx->batch_plan;
    std::vector<std::vector<int32_t>> members(plan.count);
    for (int q = 0; q < k; ++q) {
        int b = 0;
        while (b + 1 < plan.count && hn[q] > plan.n_hi[b]) ++b;
        members[b].push_back(q);
    }
    std::vector<int32_t> order;
    std::vector<int> first(plan.count), cnt(plan.count);
    for (int b = 0; b < plan.count; ++b) {
        auto& m = members[b];
        if (plan.path[b] == SA_BATCH_GROUP || plan.path[b] == SA_BATCH_REGS)
            std::stable_sort(m.begin(), m.end(), [&](int a, int c) { return hn[a] < hn[c]; });
        else
            std::stable_sort(m.begin(), m.end(), [&](int a, int c) { return hn[a] > hn[c]; });
        first[b] = (int)order.size();
        cnt[b] = (int)m.size();
        order.insert(order.end(), m.begin(), m.end());
    }
    // K rows buckets: a global slot of K (n x ceil(n/4)*4 floats of the bucket's largest n)
    // per block, at most two blocks per SM and one per instance
    std::vector<int> kblocks(plan.count, 0);
    std::vector<size_t> kslot(plan.count, 0);
    size_t need = align_up((size_t)k * 4, 256) * 3 + align_up((size_t)o->n_p * 8, 256) + 1024 +
                  SA_BATCH_MAX_BUCKETS * 256;
    for (int b = 0; b < plan.count; ++b) {
        if (plan.path[b] != SA_BATCH_KROWS || cnt[b] == 0) continue;
        const int nmax = hn[members[b].front()];
        kblocks[b] = std::min(cnt[b], 2 * ctx->num_sms);
        kslot[b] = (size_t)nmax * align_up((size_t)nmax, 4);
        need += align_up((size_t)kblocks[b] * kslot[b] * sizeof(float), 256);
    }
    sa_status rc = ctx->ws.reserve(need);
    if (rc) return rc;
    Carve cv(ctx->ws.ptr);
    int32_t* d_order = cv.take<int32_t>(k);
    int32_t* d_sw = cv.take<int32_t>(k);
    int32_t* d_st = cv.take<int32_t>(k);
    double* d_P = cv.take<double>(o->n_p);
    unsigned* d_q = cv.take<unsigned>(SA_BATCH_MAX_BUCKETS);
    std::vector<float*> kscr(plan.count, nullptr);
    for (int b = 0; b < plan.count; ++b)
        if (kblocks[b] > 0) kscr[b] = cv.take<float>((size_t)kblocks[b] * kslot[b]);
    SA_CUDA(cudaMemcpyAsync(d_order, order.data(), 4 * k, cudaMemcpyHostToDevice, st));
    SA_CUDA(cudaMemcpyAsync(d_P, o->p, 8 * o->n_p, cudaMemcpyHostToDevice, st));
    SA_CUDA(cudaMemsetAsync(d_q, 0, 4 * SA_BATCH_MAX_BUCKETS, st));
    // fork: each non-empty bucket launches on a stream of its own after the set-up above,
    // so the buckets' kernels run side by side; the context stream waits for all of them
    if (!ctx->batch_events[SA_BATCH_MAX_BUCKETS])
        SA_CUDA(cudaEventCreateWithFlags(&ctx->batch_events[SA_BATCH_MAX_BUCKETS], cudaEventDisableTiming));
    SA_CUDA(cudaEventRecord(ctx->batch_events[SA_BATCH_MAX_BUCKETS], st));
    for (int b = 0; b < plan.count; ++b) {
        if (cnt[b] == 0) continue;
        if (!ctx->batch_streams[b]) SA_CUDA(cudaStreamCreateWithFlags(&ctx->batch_streams[b], cudaStreamNonBlocking));
        if (!ctx->batch_events[b]) SA_CUDA(cudaEventCreateWithFlags(&ctx->batch_events[b], cudaEventDisableTiming));
        cudaStream_t bs = ctx->batch_streams[b];
        SA_CUDA(cudaStreamWaitEvent(bs, ctx->batch_events[SA_BATCH_MAX_BUCKETS], 0));
        const auto& m = members[b];
        const bool desc = plan.path[b] == SA_BATCH_BLOCK || plan.path[b] == SA_BATCH_KROWS;
        const int nmax = desc ? hn[m.front()] : hn[m.back()];
        BatchArgs args{d_w, d_n, d_ld, d_off, d_order + first[b], cnt[b], wtype == SA_I16, d_P, o->n_p, o->tol,
                       o->max_sweeps_per_p, d_u, d_v, d_sw, d_st, d_q + b, 0, nullptr, 0};
        if (plan.path[b] == SA_BATCH_GROUP)
            rc = launch_group_path(ctx, bs, args, nmax, plan.warps[b], plan.per_block[b], wtype);
        else if (plan.path[b] == SA_BATCH_REGS)
            rc = launch_regs_path(ctx, bs, args, nmax, plan.warps[b], plan.per_block[b], wtype);
        else if (plan.path[b] == SA_BATCH_KROWS) {
            args.kscr = kscr[b];
            args.kscr_floats = kslot[b];
            rc = launch_krows_path(ctx, bs, args, nmax, kblocks[b], wtype);
        } else rc = launch_block_path(ctx, bs, args, nmax, wtype);
        // joined even after a failed launch: the buckets already running finish first
        SA_CUDA(cudaEventRecord(ctx->batch_events[b], bs));
        SA_CUDA(cudaStreamWaitEvent(st, ctx->batch_events[b], 0));
        if (rc) {
            cudaStreamSynchronize(st);
            return rc;
        }
    }
    return finish_batch(st, k, d_sw, d_st, sweeps, status);
}
