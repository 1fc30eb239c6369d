// newton.cu -- diagonal scaling of A^(p) by Newton iteration (Sec. 5.3, the variant after
// Knight and Ruiz), the SA_KERNEL_NEWTON path of sa_scale.
//
// At every p of the schedule:
//  1. K_ij = 2^(p log2 w_ij - C_i - V_j) with C_i ~ max_j (p log2 w_ij - V_j) (any C_i keeps
//     X; this one keeps K <= ~1): the exponent in float-pair arithmetic (exact two-product
//     and two-sums, log2 w to about 2^-40), then one FP32 exp2, written once as an n x ldk
//     FP32 matrix.  X(p) is invariant under diagonal scaling (Sec. 2.1), so
//     scaling K or A^(p) gives the same X(p), and K has no range limit in p (A^(p) itself
//     needs p (b_max - b_min) within the exponent range, Sec. 4.1.1).  V is the previous
//     step's column potential (warm start).
//  2. Newton on f(x) = D(x) S x - 1 with S = [[0, K], [K^T, 0]] and x = (rho, kappa): the
//     Newton equation A_k x_{k+1} = S x_k + D(x_k)^{-1} 1 of Sec. 5.3, multiplied by
//     D(x_k) and written in y = x_{k+1} / x_k, is the symmetric system
//         (D(x_k) S D(x_k) + D(v)) y = v + 1,   v = D(x_k) S x_k,
//     solved inexactly by conjugate gradients from y = 1 (whose residual is 1 - v).  The
//     CG runs in the Chronopoulos-Gear arrangement: one operator application per
//     iteration, to the residual, with A p carried by a recurrence.  Each application of
//     D(x) S D(x) reads K once and yields both K (kappa o z_c) and K^T (rho o z_r).
//     The iteration starts from the max-normalised point: rho = 1 (rows of K have
//     maximum 1) and kappa_j = 1 / max_i K_ij.  A CG step that leaves min y < 0.1 ends
//     the inner solve and the Newton step is shortened to min y = 0.1.
//
// The whole Newton-CG iteration of a p step is one persistent cooperative kernel.  A step
// of it is: the matvec (one read of K), grid barrier, the finalisation of each block's
// slice of the 2n entries (column sums over the stripes, row sums over the tiles; v or w;
// one set of block partials), grid barrier, then every block reduces all partials in the
// same order and so takes the same decisions; a CG step then updates the block's slice
// (second set of partials, third barrier).  Every barrier wait is bounded (2 s) and ends
// the kernel with an error code.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "log2pair.cuh"
#include "sa_internal.h"

namespace sa {

namespace {

constexpr int kNtThreads = 256;
constexpr int kNtWarps = kNtThreads / 32;
constexpr double kNtDelta = 0.1;     // smallest y kept by a Newton step
constexpr double kNtEtaMax = 0.1;    // forcing term of the inner solve: eta = sqrt(res),
constexpr double kNtEtaMin = 1e-3;   //   clamped to [kNtEtaMin, kNtEtaMax]
constexpr int kNtCgCap = 50;         // CG iterations per Newton step (stagnation guard)
constexpr int kNtStallWindow = 20;   // Newton steps without halving the residual end the p step
constexpr int kNtStages = 6;         // slots of the matvec's bulk-copy ring (row tiles in flight)
constexpr int kNtMaxSmem = 200 * 1024;

enum : int { kNtRes = 0, kNtCg = 1, kNtDone = 2 };
enum : int { kNtRunning = 0, kNtConverged = 1, kNtCapped = 2, kNtNonfinite = 3, kNtStalled = 4 };

// Scalar state of the iteration; every block holds an identical copy in shared memory.
struct NtState {
    int mode;        // kNtRes: the next matvec is of 1 (residual); kNtCg: of r; kNtDone
    int cstage;      // 1: this step applies a CG update
    int first;       // first CG iteration of the Newton step (beta = 0)
    int apply;       // pending x <- x o (1 + tau (y - 1)), applied by the next residual step
    int breakdown;   // CG curvature not positive: end the inner solve
    int status;
    int matvecs;     // operator applications in this p step
    int cg_it;
    int newton_it;
    int stall;       // Newton steps since the residual last fell below half of res_ref
    double tau, res, gamma, gamma0, gamma_prev, alpha, alpha_prev, beta, thr;
    double res_ref;
};

// Result of one p step, written by block 0.
struct NtOut {
    int status;
    int matvecs;
    int newton_it;
    int pad;
    double res;
};

struct NtArgs {
    const float* K;
    int n;
    int ldk;        // row pitch of K and of the column partials (floats, multiple of 4)
    int T;          // column tiles
    int W4;         // float4 chunks per column tile (<= threads x CH)
    int R;          // row stripes
    int rows_per;
    // vectors of 2n entries (rows | columns) in FP64, each updated only by the block that
    // owns the entry (a few dozen per block); the matvec reads FP32 copies of x, y and r,
    // as GB300 runs FP64 arithmetic at a small fraction of the FP32 rate
    double* x;      // rho | kappa
    double* v;      // D(x) S x
    double* y;
    double* r;
    double* pd;
    double* s;
    double* w;
    float* xf;      // FP32 copies of x, y, r
    float* yf;
    float* rf;
    double* prt;    // T x n row partials
    float* pc;      // R x ldk column partials
    double* bred;   // finalisation block partials (4 per block)
    double* cred;   // update block partials (4 per block)
    unsigned* bar;  // grid barrier (count, generation)
    int* err;       // kErr* code of a failed wait or step
};

// Global float4 chunk (columns 4q .. 4q+3) of local chunk ql of column tile t; chunks past
// the tile map beyond the matrix (4q >= n), which every use masks.
__device__ __forceinline__ int nt_chunk(const NtArgs& A, int t, int ql) {
    return ql < A.W4 ? t * A.W4 + ql : (A.n + 3) / 4;
}

// the 256-entry table of log2pair.cuh, built once per call
__global__ void nt_tab_kernel(float4* t) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < 256) t[j] = log2_tab_entry(j);
}

// V_j as a float pair (hi, lo), and the same for p
__global__ void nt_vsplit_kernel(const double* __restrict__ V, float2* __restrict__ vp, int n) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        const float h = (float)V[j];
        vp[j] = make_float2(h, (float)(V[j] - (double)h));
    }
}

// C_i = max_j (p log2 w_ij - V_j) over w_ij > 0 to about 1e-4 (SFU log2; C_i only sets the
// scale of row i of K); one warp per row
template <typename WT>
__global__ void nt_rowmax_kernel(const WT* __restrict__ w, int n, int64_t ld, float ph,
                                 const float2* __restrict__ vp, float* __restrict__ Cf,
                                 double* __restrict__ C) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    const WT* wr = w + (int64_t)row * ld;
    float m = -INFINITY;
    for (int j = lane; j < n; j += 32) {
        const int wv = (int)wr[j];
        if (wv > 0) m = fmaxf(m, fmaf(ph, __log2f((float)wv), -vp[j].x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
        Cf[row] = m;
        C[row] = (double)m;
    }
}

// four weights of a chunk (columns 4q .. 4q+3, all < ld)
__device__ __forceinline__ void load4(const int16_t* p, int v[4]) {
    const short4 q = *(const short4*)p;
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
__device__ __forceinline__ void load4(const int32_t* p, int v[4]) {
    const int4 q = *(const int4*)p;
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}

// K_ij = 2^d with d = p log2 w_ij - V_j - C_i evaluated in float pairs: the leading parts
// cancel exactly (two-product, two-sums) and the small ones are added after, so d is exact
// to about 2^-24 |d|, and one SFU exp2 (2^-22) follows; pad columns and zero weights give
// 0.  Also the column maxima of K over each row stripe (pc), from which the starting kappa
// is taken.
template <typename WT, int CH>
__global__ void __launch_bounds__(kNtThreads) nt_kwrite_kernel(const WT* __restrict__ w, int64_t ld,
                                                               float ph, float pl,
                                                               const float2* __restrict__ vp,
                                                               const float* __restrict__ Cf,
                                                               const float4* __restrict__ gtab,
                                                               NtArgs A) {
    __shared__ float4 s_tab[256];
    const int tid = threadIdx.x;
    s_tab[tid] = gtab[tid];
    __syncthreads();
    const int t = blockIdx.x % A.T, s = blockIdx.x / A.T;
    const int r0 = s * A.rows_per, r1 = min(A.n, r0 + A.rows_per);
    const int n = A.n;
    float2 vj[4 * CH];
    float cm[4 * CH];
    int q[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        q[k] = nt_chunk(A, t, tid + kNtThreads * k);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = 4 * q[k] + e;
            vj[4 * k + e] = j < n ? vp[j] : make_float2(0.0f, 0.0f);
            cm[4 * k + e] = 0.0f;
        }
    }
    for (int i = r0; i < r1; ++i) {
        const float ci = Cf[i];
        const WT* wr = w + (int64_t)i * ld;
        float* kr = (float*)A.K + (int64_t)i * A.ldk;
#pragma unroll
        for (int k = 0; k < CH; ++k) {
            if (4 * q[k] >= n) continue;
            int wv[4];
            load4(wr + 4 * q[k], wv);
            float kv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 4 * q[k] + e;
                kv[e] = 0.0f;
                if (j < n && wv[e] > 0) {
                    const float2 lw = wlog2(s_tab, wv[e]);
                    const float2 v2 = vj[4 * k + e];
                    const float tp = ph * lw.x;
                    const float te = fmaf(ph, lw.x, -tp);
                    float e1, e2;
                    const float s1 = two_sum(tp, -v2.x, &e1);
                    const float s2 = two_sum(s1, -ci, &e2);
                    const float rest = ((te + e1) + e2) + (fmaf(ph, lw.y, pl * lw.x) - v2.y);
                    kv[e] = ex2_approx(s2 + rest);   // SFU exp2, relative error about 2^-22
                }
                cm[4 * k + e] = fmaxf(cm[4 * k + e], kv[e]);
            }
            *(float4*)(kr + 4 * q[k]) = make_float4(kv[0], kv[1], kv[2], kv[3]);
        }
    }
#pragma unroll
    for (int k = 0; k < CH; ++k)
        if (4 * q[k] < n)
            *(float4*)(A.pc + (int64_t)s * A.ldk + 4 * q[k]) =
                make_float4(cm[4 * k], cm[4 * k + 1], cm[4 * k + 2], cm[4 * k + 3]);
}

// Sum (compensated, Kahan) or max over the R stripe partials of column j, the stripes split
// over the 8 warps of the block; each lane issues its loads in batches of 24 independent
// loads.
template <bool MAX>
__device__ __forceinline__ double nt_stripes(const float* __restrict__ pc, int R, int ldk, int j, int wid) {
    constexpr int kB = 24;
    float acc = 0.0f, comp = 0.0f;   // 0 is also the identity of the max: the partials are >= 0
    for (int base = wid; base < R; base += kNtWarps * kB) {
        float a[kB];
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            const int s = base + u * kNtWarps;
            a[u] = s < R ? __ldcg(pc + (int64_t)s * ldk + j) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kB; ++u) {
            if (MAX) {
                acc = fmaxf(acc, a[u]);
            } else {
                const float yk = a[u] - comp;
                const float tk = acc + yk;
                comp = (tk - acc) - yk;
                acc = tk;
            }
        }
    }
    return MAX ? (double)acc : (double)acc - (double)comp;   // the compensated sum in FP64
}

// starting point of a p step: rho = 1, kappa_j = 1 / max_i K_ij.
// Grid: ceil(n/32) column blocks of 32 columns x 8 warps, then the row blocks.
__global__ void __launch_bounds__(kNtThreads) nt_init_kernel(NtArgs A) {
    __shared__ float sred[kNtWarps][33];
    const int n = A.n, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nbc = (n + 31) / 32;
    if ((int)blockIdx.x < nbc) {
        const int j = blockIdx.x * 32 + lane;
        sred[wid][lane] = j < n ? (float)nt_stripes<true>(A.pc, A.R, A.ldk, j, wid) : 0.0f;
        __syncthreads();
        if (wid == 0 && j < n) {
            float m = 0.0f;
            for (int x = 0; x < kNtWarps; ++x) m = fmaxf(m, sred[x][lane]);
            const double k = 1.0 / (double)m;   // +inf for an empty column: caught by the first residual
            A.x[n + j] = k;
            A.xf[n + j] = (float)k;
            A.y[n + j] = 1.0;
            A.yf[n + j] = 1.0f;
        }
    } else {
        const int i = (blockIdx.x - nbc) * kNtThreads + tid;
        if (i < n) {
            A.x[i] = 1.0;
            A.xf[i] = 1.0f;
            A.y[i] = 1.0;
            A.yf[i] = 1.0f;
        }
    }
}

// Block reduction of three FP32 values at once: v0 by max (MAX0) or sum, v1 by sum, v2 by
// min; the warp results are combined in FP64 by thread 0, where the results are valid.
template <bool MAX0>
__device__ __forceinline__ void nt_block_reduce3(float v0, float v1, float v2, float (*sh)[kNtWarps],
                                                 double* o0, double* o1, double* o2) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float u0 = __shfl_xor_sync(0xffffffffu, v0, o);
        v0 = MAX0 ? fmaxf(v0, u0) : v0 + u0;
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 = fminf(v2, __shfl_xor_sync(0xffffffffu, v2, o));
    }
    __syncthreads();   // sh may still be read by thread 0 of the previous reduction
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = v0;
        sh[1][threadIdx.x >> 5] = v1;
        sh[2][threadIdx.x >> 5] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r0 = sh[0][0], r1 = sh[1][0], r2 = sh[2][0];
        for (int k = 1; k < kNtWarps; ++k) {
            r0 = MAX0 ? fmax(r0, (double)sh[0][k]) : r0 + sh[0][k];
            r1 += sh[1][k];
            r2 = fmin(r2, (double)sh[2][k]);
        }
        *o0 = r0;
        *o1 = r1;
        *o2 = r2;
    }
}

// Reduction of the G block partials (4 doubles each, the first three used) by warp 0 in a
// fixed order, so that every block obtains identical values; valid in lane 0 of warp 0.
template <bool MAX0>
__device__ __forceinline__ void nt_grid_reduce3(const double* part, int G, double* g0, double* g1, double* g2) {
    double a0 = 0.0, a1 = 0.0, a2 = INFINITY;   // 0 is also the identity of the max of |v - 1|
    for (int x = threadIdx.x; x < G; x += 32) {
        const double x0 = __ldcg(part + 4 * x);
        a0 = MAX0 ? fmax(a0, x0) : a0 + x0;
        a1 += __ldcg(part + 4 * x + 1);
        a2 = fmin(a2, __ldcg(part + 4 * x + 2));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double u0 = __shfl_xor_sync(0xffffffffu, a0, o);
        a0 = MAX0 ? fmax(a0, u0) : a0 + u0;
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 = fmin(a2, __shfl_xor_sync(0xffffffffu, a2, o));
    }
    *g0 = a0;
    *g1 = a1;
    *g2 = a2;
}

// Decisions after the finalisation (g0: max |v - 1| or sum w r; g1: sum (1 - v)^2;
// g2: min v, or a negative flag for a zero or non-finite value)
__device__ __forceinline__ void nt_after_fin(NtState& S, bool res_mode, double g0, double g1, double g2,
                                             double tol, int cap) {
    S.matvecs += 1;
    S.cstage = 0;
    if (!(g2 > 0.0)) {
        S.status = kNtNonfinite;
        S.mode = kNtDone;
    } else if (res_mode) {
        S.res = g0;
        S.apply = 0;
        // stall guard: the FP32 operator limits how far Newton gets on nearly decomposable
        // X(p) (Sec. 3.1); without progress the step ends instead of cycling to the cap
        if (S.matvecs == 1 || g0 <= 0.5 * S.res_ref) {
            S.res_ref = g0;
            S.stall = 0;
        } else {
            S.stall += 1;
        }
        if (g0 <= tol) {
            S.status = kNtConverged;
            S.mode = kNtDone;
        } else if (S.matvecs >= cap) {
            S.status = kNtCapped;
            S.mode = kNtDone;
        } else if (S.stall >= kNtStallWindow) {
            S.status = kNtStalled;
            S.mode = kNtDone;
        } else {
            const double eta = fmin(kNtEtaMax, fmax(kNtEtaMin, sqrt(g0)));
            S.gamma = S.gamma0 = g1;
            S.thr = eta * eta * g1;
            S.first = 1;
            S.cg_it = 0;
            S.breakdown = 0;
            S.mode = kNtCg;
        }
    } else {
        // Chronopoulos-Gear: alpha = gamma / (delta - beta gamma / alpha_prev), delta = r.Mr
        if (S.first) {
            S.beta = 0.0;
            S.alpha = S.gamma / g0;
        } else {
            S.beta = S.gamma / S.gamma_prev;
            S.alpha = S.gamma / (g0 - S.beta * S.gamma / S.alpha_prev);
        }
        if (!(S.alpha > 0.0 && S.alpha < INFINITY)) {
            S.alpha = 0.0;
            S.breakdown = 1;
        }
        S.cstage = 1;
    }
}

// Decisions after a CG update (g0 = ||r||^2, g1 = min y): end of the inner solve when the
// residual reached eta ||r_0||, at the CG cap, on breakdown, at the matvec cap, or when y
// left [delta, inf) (the Newton step is then shortened to min y = delta)
__device__ __forceinline__ void nt_after_upd(NtState& S, double g0, double g1, int cap) {
    S.gamma_prev = S.gamma;
    S.gamma = g0;
    S.alpha_prev = S.alpha;
    S.first = 0;
    S.cg_it += 1;
    if (!(g0 < INFINITY) || !(g1 > -INFINITY && g1 < INFINITY)) {
        S.status = kNtNonfinite;
        S.mode = kNtDone;
    } else if (g0 <= S.thr || S.cg_it >= kNtCgCap || g1 < kNtDelta || S.breakdown || S.matvecs >= cap) {
        S.apply = 1;
        S.tau = g1 < kNtDelta ? (1.0 - kNtDelta) / (1.0 - g1) : 1.0;
        S.mode = kNtRes;
        S.newton_it += 1;
    }
}

// Dynamic shared memory of the solve kernel: the cp.async stages, the per-warp row dots of
// the stripe, the stripe's row factors and the totals of the owned entries.
__host__ __device__ inline size_t nt_smem_bytes(int ch, int rows_per, int own) {
    return (size_t)kNtStages * ch * kNtThreads * 16 + (size_t)rows_per * kNtWarps * 4 + (size_t)rows_per * 4 +
           8 + (size_t)2 * own * 8;
}

// One p step of the Newton-CG iteration on K.  Block (s, t) = (blockIdx / T, blockIdx % T)
// streams rows [s rows_per, ...) x the columns of tile t in the matvec; for the
// finalisation and the CG update it owns columns [b cs, (b+1) cs) and the rows with the
// same indices.
template <int CH>
__global__ void __launch_bounds__(kNtThreads, 2) nt_solve_kernel(NtArgs A, double tol, int cap,
                                                                 NtOut* out) {
    __shared__ double sred[kNtWarps][33];
    __shared__ float sh[3][kNtWarps];
    __shared__ NtState S;
    __shared__ __align__(8) uint64_t full[kNtStages];   // a slot's row tile has landed
    __shared__ unsigned rel_cnt[kNtStages];               // warp releases of a slot
    __shared__ unsigned iss_cnt[kNtStages];               // copies issued into a slot
    __shared__ int s_fail;
    extern __shared__ __align__(16) unsigned char nt_dyn[];
    if (*(volatile int*)A.err != 0) return;   // an earlier step of this call failed
    const int n = A.n, G = gridDim.x, b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int t = b % A.T, s = b / A.T;
    const int r0 = s * A.rows_per, r1 = min(n, r0 + A.rows_per), nrows = r1 - r0;
    const int cs = (n + G - 1) / G;
    const int c0 = min(n, b * cs), c1 = min(n, c0 + cs);   // owned columns and rows
    const int own = c1 - c0;
    float4* stage = (float4*)nt_dyn;                                   // [slots][CH x threads]
    float* rowdot = (float*)(stage + kNtStages * CH * kNtThreads);     // [rows_per][warps]
    float* zr_s = rowdot + A.rows_per * kNtWarps;                      // [rows_per]
    double* tot_s = (double*)(((uintptr_t)(zr_s + A.rows_per) + 7) & ~(uintptr_t)7);   // [2 cs]
    if (tid == 0) {
        NtState z{};
        z.mode = kNtRes;
        z.status = kNtRunning;
        z.tau = 1.0;
        S = z;
        s_fail = 0;
        for (int k = 0; k < kNtStages; ++k) {
            mbar_init(&full[k], 1);
            rel_cnt[k] = iss_cnt[k] = 0u;
        }
        mbar_fence_init();
    }
    __syncthreads();
    int q[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) q[k] = nt_chunk(A, t, tid + kNtThreads * k);
    // The block's row tiles stream through a ring of kNtStages slots filled by 1-D bulk
    // copies: ring index v is row v % nrows of the stripe, in slot v % kNtStages.  K does
    // not change within the launch, so the ring runs on across matvec phases: the warp
    // whose release completes a slot's count refills it with index v + kNtStages, and the
    // next phase's first rows are in flight during this phase's barriers.
    const int nq = (n + 3) / 4;
    const unsigned tile_bytes = (unsigned)(min(nq, (t + 1) * A.W4) - t * A.W4) * 16u;
    const float* ktile = A.K + (int64_t)r0 * A.ldk + 4 * (int64_t)t * A.W4;
    auto issue = [&](uint32_t v) {   // one thread
        const uint32_t slot = v % (uint32_t)kNtStages;
        iss_cnt[slot] += 1u;
        mbar_arrive_expect_tx(&full[slot], tile_bytes);
        bulk_g2s(stage + (size_t)slot * CH * kNtThreads, ktile + (int64_t)(v % (uint32_t)nrows) * A.ldk, tile_bytes,
                 &full[slot]);
    };
    auto release = [&](uint32_t v) {   // lane 0 after __syncwarp
        const uint32_t slot = v % (uint32_t)kNtStages;
        unsigned old;
        asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(&rel_cnt[slot])), "r"(1u) : "memory");
        if ((old + 1u) % (unsigned)kNtWarps == 0u) {
            fence_proxy_async_smem();
            issue(v + (uint32_t)kNtStages);
        }
    };
    auto wait_copies = [&]() {   // tid 0: the last copy issued into every slot has landed
        for (int k = 0; k < kNtStages; ++k) {
            const unsigned c = iss_cnt[k];
            if (c > 0u && !mbar_wait(&full[k], (c - 1u) & 1u, A.err, kWaitTimeoutNs)) break;
        }
    };
    if (tid == 0)
        for (uint32_t v = 0; v < (uint32_t)kNtStages; ++v) issue(v);
    uint32_t vbase = 0;   // ring index of the phase's first row
    for (;;) {
        const bool res_mode = S.mode == kNtRes;
        const bool apply = S.apply != 0;
        const float tau = (float)S.tau;
        // ---- A: D(x) S D(x) z for z = 1 or r, one read of the block's tile of K ----
        {
            float z[4 * CH], acc[4 * CH];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = 4 * q[k] + e;
                    float zv = 0.0f;
                    if (j < n) {
                        float xe = A.xf[n + j];
                        if (apply) xe *= fmaf(tau, A.yf[n + j] - 1.0f, 1.0f);
                        zv = res_mode ? xe : xe * A.rf[n + j];
                    }
                    z[4 * k + e] = zv;
                    acc[4 * k + e] = 0.0f;
                }
            }
            for (int i = tid; i < nrows; i += kNtThreads) {
                float xe = A.xf[r0 + i];
                if (apply) xe *= fmaf(tau, A.yf[r0 + i] - 1.0f, 1.0f);
                zr_s[i] = res_mode ? xe : xe * A.rf[r0 + i];
            }
            __syncthreads();
            for (int row = 0; row < nrows; ++row) {
                // after a failed wait the warp stops (warp-uniform: lanes meet at __syncwarp)
                if (__any_sync(0xffffffffu, *(volatile int*)&s_fail != 0)) break;
                const uint32_t v = vbase + (uint32_t)row;
                const uint32_t slot = v % (uint32_t)kNtStages;
                if (!mbar_wait(&full[slot], (v / (uint32_t)kNtStages) & 1u, A.err, kWaitTimeoutNs)) s_fail = 1;
                const float4* src = stage + (size_t)slot * CH * kNtThreads + tid;
                const float zr = zr_s[row];
                float d = 0.0f;
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                    if (4 * q[k] < n) {
                        const float4 kv = src[k * kNtThreads];
                        d = fmaf(kv.x, z[4 * k], d);
                        d = fmaf(kv.y, z[4 * k + 1], d);
                        d = fmaf(kv.z, z[4 * k + 2], d);
                        d = fmaf(kv.w, z[4 * k + 3], d);
                        acc[4 * k] = fmaf(kv.x, zr, acc[4 * k]);
                        acc[4 * k + 1] = fmaf(kv.y, zr, acc[4 * k + 1]);
                        acc[4 * k + 2] = fmaf(kv.z, zr, acc[4 * k + 2]);
                        acc[4 * k + 3] = fmaf(kv.w, zr, acc[4 * k + 3]);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
                __syncwarp();
                if (lane == 0) {
                    rowdot[row * kNtWarps + wid] = d;
                    if (*(volatile int*)&s_fail == 0) release(v);   // no refill over a copy that never landed
                }
            }
            vbase += (uint32_t)nrows;
            __syncthreads();
            for (int i = tid; i < nrows; i += kNtThreads) {
                double sm = 0.0;
#pragma unroll
                for (int x = 0; x < kNtWarps; ++x) sm += (double)rowdot[i * kNtWarps + x];
                A.prt[(int64_t)t * n + r0 + i] = sm;
            }
#pragma unroll
            for (int k = 0; k < CH; ++k)
                if (4 * q[k] < n)
                    *(float4*)(A.pc + (int64_t)s * A.ldk + 4 * q[k]) =
                        make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
        }
        if (s_fail) atomicCAS(A.err, 0, kErrTimeout);   // a ring wait gave up: every block stops
        if (!group_barrier(A.bar, G, A.err, kWaitTimeoutNs)) break;
        // ---- B: finalise the owned entries: m = D(x) S D(x) z; v, r, y or w ----
        {
            for (int cb = c0; cb < c1; cb += 32) {
                const int j = cb + lane;
                sred[wid][lane] = j < c1 ? nt_stripes<false>(A.pc, A.R, A.ldk, j, wid) : 0.0;
                __syncthreads();
                if (wid == 0 && j < c1) {
                    double tot = 0.0;
                    for (int x = 0; x < kNtWarps; ++x) tot += sred[x][lane];
                    tot_s[j - c0] = tot;
                }
                __syncthreads();
            }
            for (int i = c0 + tid; i < c1; i += kNtThreads) {
                double tot = 0.0;
                for (int tt = 0; tt < A.T; ++tt) tot += A.prt[(int64_t)tt * n + i];
                tot_s[own + (i - c0)] = tot;
            }
            __syncthreads();
            // residual step: a0 = max |v - 1|, a1 = sum (1 - v)^2, a2 = min v (or -1 for a
            // zero or non-finite sum); CG step: a0 = sum w r, a2 = -1 for a non-finite w
            // the owned entries in FP64 (a few dozen per block)
            float a0 = 0.0f, a1 = 0.0f, a2 = INFINITY;
            const double taud = S.tau;
            for (int x = tid; x < 2 * own; x += kNtThreads) {
                const int e = x < own ? n + c0 + x : c0 + (x - own);
                double xe = A.x[e];
                if (apply) {
                    xe *= 1.0 + taud * (A.y[e] - 1.0);
                    A.x[e] = xe;
                    A.xf[e] = (float)xe;
                }
                const double m = xe * tot_s[x];
                if (res_mode) {
                    const double re = 1.0 - m;
                    A.v[e] = m;
                    A.r[e] = re;
                    A.rf[e] = (float)re;
                    A.y[e] = 1.0;
                    A.yf[e] = 1.0f;
                    a0 = fmaxf(a0, (float)fabs(re));
                    a1 += (float)(re * re);
                    a2 = fminf(a2, (m > 0.0 && m < INFINITY) ? (float)m : -1.0f);
                } else {
                    const double re = A.r[e];
                    const double we = m + A.v[e] * re;
                    A.w[e] = we;
                    a0 += (float)(we * re);
                    a2 = fminf(a2, (we > -INFINITY && we < INFINITY) ? 1.0f : -1.0f);
                }
            }
            double b0, b1, b2;
            if (res_mode) nt_block_reduce3<true>(a0, a1, a2, sh, &b0, &b1, &b2);
            else nt_block_reduce3<false>(a0, a1, a2, sh, &b0, &b1, &b2);
            if (tid == 0) {
                A.bred[4 * b] = b0;
                A.bred[4 * b + 1] = b1;
                A.bred[4 * b + 2] = b2;
            }
        }
        if (!group_barrier(A.bar, G, A.err, kWaitTimeoutNs)) break;
        // ---- C: every block reduces all partials in the same order: same decisions ----
        if (wid == 0) {
            double g0, g1, g2;
            if (res_mode) nt_grid_reduce3<true>(A.bred, G, &g0, &g1, &g2);
            else nt_grid_reduce3<false>(A.bred, G, &g0, &g1, &g2);
            if (lane == 0) nt_after_fin(S, res_mode, g0, g1, g2, tol, cap);
        }
        __syncthreads();
        if (S.mode == kNtDone) break;
        if (!S.cstage) continue;
        // ---- CG update of the owned entries: p, s (= M p), y, r ----
        {
            const bool first = S.first != 0;
            const double alpha = S.alpha, beta = S.beta;
            float rr = 0.0f, ymin = INFINITY;
            for (int x = tid; x < 2 * own; x += kNtThreads) {
                const int e = x < own ? n + c0 + x : c0 + (x - own);
                const double re = A.r[e], we = A.w[e];
                const double pe = first ? re : re + beta * A.pd[e];
                const double se = first ? we : we + beta * A.s[e];
                const double ye = A.y[e] + alpha * pe;
                const double rn = re - alpha * se;
                A.pd[e] = pe;
                A.s[e] = se;
                A.y[e] = ye;
                A.yf[e] = (float)ye;
                A.r[e] = rn;
                A.rf[e] = (float)rn;
                rr += (float)(rn * rn);
                ymin = fminf(ymin, (float)ye);
            }
            double b0, b1, b2;
            nt_block_reduce3<false>(rr, 0.0f, ymin, sh, &b0, &b1, &b2);
            if (tid == 0) {
                A.cred[4 * b] = b0;
                A.cred[4 * b + 1] = 0.0;
                A.cred[4 * b + 2] = b2;
            }
        }
        if (!group_barrier(A.bar, G, A.err, kWaitTimeoutNs)) break;
        if (wid == 0) {
            double g0, g1, g2;
            nt_grid_reduce3<false>(A.cred, G, &g0, &g1, &g2);
            if (lane == 0) nt_after_upd(S, g0, g2, cap);
        }
        __syncthreads();
        if (S.mode == kNtDone) break;
    }
    // the ring's refills in flight (issued for a phase that does not come) land before exit
    __syncthreads();
    if (tid == 0) wait_copies();
    __syncthreads();
    if (b == 0 && tid == 0) {
        NtOut o{};
        o.status = S.status;
        o.matvecs = S.matvecs;
        o.newton_it = S.newton_it;
        o.res = S.res;
        *out = o;
    }
}

// potentials of X = D(rho) K D(kappa) in log2 units: U = C - log2 rho, V -= log2 kappa
__global__ void nt_potentials_kernel(const double* __restrict__ x, const double* __restrict__ C,
                                     double* __restrict__ U, double* __restrict__ V, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        U[i] = C[i] - log2(x[i]);
        V[i] = V[i] - log2(x[n + i]);
    }
}

struct NtPlan {
    int ch, T, W4, R, rows_per, grid;
    size_t smem;
};

template <int CH>
int nt_occupancy(size_t smem) {
    static const cudaError_t attr = cudaFuncSetAttribute(nt_solve_kernel<CH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         kNtMaxSmem);
    if (attr != cudaSuccess) return 0;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, nt_solve_kernel<CH>, kNtThreads, smem);
    return occ;
}

// Column tiles of at most 1024 CH columns (CH float4 chunks per thread), equal in width;
// as many row stripes as fill the co-resident grid.
NtPlan nt_plan(const sa_ctx* ctx, int n) {
    NtPlan P{};
    P.ch = n <= 1024 ? 1 : n <= 2048 ? 2 : 4;
    const int nq = (n + 3) / 4;                                  // float4 chunks of a row
    P.T = (nq + kNtThreads * P.ch - 1) / (kNtThreads * P.ch);
    P.W4 = (nq + P.T - 1) / P.T;                                 // balanced tiles
    auto occupancy = [&](size_t smem) {
        const int occ = P.ch == 1 ? nt_occupancy<1>(smem) : P.ch == 2 ? nt_occupancy<2>(smem) : nt_occupancy<4>(smem);
        return std::max(0, std::min(occ, 2));
    };
    // two blocks per SM when their shared memory fits, else one; the grid must be
    // co-resident for the cooperative launch
    for (int per_sm = 2; per_sm >= 1; --per_sm) {
        int G = ctx->num_sms * per_sm;
        if (ctx->max_grid > 0) G = std::min(G, ctx->max_grid);
        const int R = std::max(1, std::min(n, G / P.T));
        P.rows_per = (n + R - 1) / R;
        P.R = (n + P.rows_per - 1) / P.rows_per;
        P.grid = P.R * P.T;
        const int cs = (n + P.grid - 1) / P.grid;
        P.smem = nt_smem_bytes(P.ch, P.rows_per, cs);
        if (P.smem <= (size_t)kNtMaxSmem && P.grid <= ctx->num_sms * occupancy(P.smem)) return P;
    }
    P.grid = 0;
    return P;
}

sa_status launch_solve(const NtPlan& P, NtArgs A, double tol, int cap, NtOut* out, cudaStream_t st) {
    void* params[] = {(void*)&A, (void*)&tol, (void*)&cap, (void*)&out};
    const void* kern = P.ch == 1 ? (const void*)nt_solve_kernel<1>
                     : P.ch == 2 ? (const void*)nt_solve_kernel<2> : (const void*)nt_solve_kernel<4>;
    SA_CUDA(cudaLaunchCooperativeKernel(kern, dim3(P.grid), dim3(kNtThreads), params, P.smem, st));
    count_launch();
    return SA_OK;
}

}  // namespace

bool newton_supported(const sa_ctx* ctx, const sa_matrix* a) {
    const int sz = wbytes(a->wtype);
    if (((uintptr_t)a->w & 15) != 0) return false;
    if (((size_t)a->ld * sz) % 16 != 0) return false;
    if (a->n < 1 || a->n > (1 << 16)) return false;
    return nt_plan(ctx, a->n).grid > 0;
}

sa_status scale_newton(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U, double* V,
                       sa_scale_info* info) {
    const int n = a->n;
    cudaStream_t st = ctx->stream;
    const NtPlan P = nt_plan(ctx, n);
    if (P.grid <= 0) {
        set_error("newton scaling: no co-resident grid for n = %d", n);
        return SA_E_UNSUPPORTED;
    }
    const int ldk = (int)align_up((size_t)n, 4);
    const size_t bytes = align_up((size_t)n * ldk * 4, 256)       // K
                       + align_up((size_t)n * 8, 256)              // C
                       + 7 * align_up((size_t)2 * n * 8, 256)      // x v y r p s w
                       + 3 * align_up((size_t)2 * n * 4, 256)      // FP32 copies of x y r
                       + align_up((size_t)P.T * n * 8, 256)        // row partials
                       + align_up((size_t)P.R * ldk * 4, 256)      // column partials
                       + 2 * align_up((size_t)P.grid * 32, 256)    // block partials
                       + align_up((size_t)o->n_p * sizeof(NtOut), 256)
                       + align_up((size_t)256 * 16, 256)           // log2 table
                       + align_up((size_t)n * 8, 256)              // V pairs
                       + align_up((size_t)n * 4, 256)              // C (FP32)
                       + 3 * 256;                                  // barrier, error flag
    sa_status rc = ctx->ws.reserve(bytes);
    if (rc) return rc;
    Carve cv(ctx->ws.ptr);
    NtArgs A{};
    A.K = cv.take<float>((size_t)n * ldk);
    double* C = cv.take<double>(n);
    A.x = cv.take<double>(2 * (size_t)n);
    A.v = cv.take<double>(2 * (size_t)n);
    A.y = cv.take<double>(2 * (size_t)n);
    A.r = cv.take<double>(2 * (size_t)n);
    A.pd = cv.take<double>(2 * (size_t)n);
    A.s = cv.take<double>(2 * (size_t)n);
    A.w = cv.take<double>(2 * (size_t)n);
    A.xf = cv.take<float>(2 * (size_t)n);
    A.yf = cv.take<float>(2 * (size_t)n);
    A.rf = cv.take<float>(2 * (size_t)n);
    A.prt = cv.take<double>((size_t)P.T * n);
    A.pc = cv.take<float>((size_t)P.R * ldk);
    A.bred = cv.take<double>((size_t)P.grid * 4);
    A.cred = cv.take<double>((size_t)P.grid * 4);
    NtOut* d_out = cv.take<NtOut>(o->n_p);
    float4* tab = cv.take<float4>(256);
    float2* vp = cv.take<float2>(n);
    float* Cf = cv.take<float>(n);
    A.bar = cv.take<unsigned>(2);
    A.err = cv.take<int>(1);
    A.n = n;
    A.ldk = ldk;
    A.T = P.T;
    A.W4 = P.W4;
    A.R = P.R;
    A.rows_per = P.rows_per;

    const int k0 = o->resume_from > 0 ? o->resume_from : 0;
    if (k0 == 0) {
        SA_CUDA(cudaMemsetAsync(U, 0, n * sizeof(double), st));
        SA_CUDA(cudaMemsetAsync(V, 0, n * sizeof(double), st));
    }
    SA_CUDA(cudaMemsetAsync(A.err, 0, sizeof(int), st));
    SA_CUDA(cudaMemsetAsync(d_out, 0, o->n_p * sizeof(NtOut), st));
    nt_tab_kernel<<<1, 256, 0, st>>>(tab);
    count_launch();
    cudaEvent_t ev0, ev1;
    SA_CUDA(cudaEventCreate(&ev0));
    SA_CUDA(cudaEventCreate(&ev1));
    SA_CUDA(cudaEventRecord(ev0, st));
    for (int k = k0; k < o->n_p; ++k) {
        const double p = o->p[k];
        if (k > 0 && !o->warm_keep_v) launch_scale_vec(V, n, p / o->p[k - 1], st);
        const float ph = (float)p, pl = (float)(p - (double)ph);
        nt_vsplit_kernel<<<(n + 255) / 256, 256, 0, st>>>(V, vp, n);
        if (a->wtype == SA_I16) {
            const int16_t* w = (const int16_t*)a->w;
            nt_rowmax_kernel<int16_t><<<(n + 7) / 8, 256, 0, st>>>(w, n, a->ld, ph, vp, Cf, C);
            if (P.ch == 1) nt_kwrite_kernel<int16_t, 1><<<P.grid, kNtThreads, 0, st>>>(w, a->ld, ph, pl, vp, Cf, tab, A);
            else if (P.ch == 2) nt_kwrite_kernel<int16_t, 2><<<P.grid, kNtThreads, 0, st>>>(w, a->ld, ph, pl, vp, Cf, tab, A);
            else nt_kwrite_kernel<int16_t, 4><<<P.grid, kNtThreads, 0, st>>>(w, a->ld, ph, pl, vp, Cf, tab, A);
        } else {
            const int32_t* w = (const int32_t*)a->w;
            nt_rowmax_kernel<int32_t><<<(n + 7) / 8, 256, 0, st>>>(w, n, a->ld, ph, vp, Cf, C);
            if (P.ch == 1) nt_kwrite_kernel<int32_t, 1><<<P.grid, kNtThreads, 0, st>>>(w, a->ld, ph, pl, vp, Cf, tab, A);
            else if (P.ch == 2) nt_kwrite_kernel<int32_t, 2><<<P.grid, kNtThreads, 0, st>>>(w, a->ld, ph, pl, vp, Cf, tab, A);
            else nt_kwrite_kernel<int32_t, 4><<<P.grid, kNtThreads, 0, st>>>(w, a->ld, ph, pl, vp, Cf, tab, A);
        }
        nt_init_kernel<<<(n + 31) / 32 + (n + kNtThreads - 1) / kNtThreads, kNtThreads, 0, st>>>(A);
        count_launch(4);
        SA_CUDA(cudaMemsetAsync(A.bar, 0, 2 * sizeof(unsigned), st));
        rc = launch_solve(P, A, o->tol, o->max_sweeps_per_p, d_out + k, st);
        if (rc) { cudaEventDestroy(ev0); cudaEventDestroy(ev1); return rc; }
        nt_potentials_kernel<<<(n + 255) / 256, 256, 0, st>>>(A.x, C, U, V, n);
        count_launch();
    }
    SA_CUDA(cudaEventRecord(ev1, st));
    rc = ctx->pinned.reserve(64 + (size_t)o->n_p * sizeof(NtOut));
    if (rc) { cudaEventDestroy(ev0); cudaEventDestroy(ev1); return rc; }
    int* h_err = (int*)ctx->pinned.ptr;
    NtOut* h_out = (NtOut*)((char*)ctx->pinned.ptr + 64);
    SA_CUDA(cudaMemcpyAsync(h_err, A.err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(h_out, d_out, o->n_p * sizeof(NtOut), cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaStreamSynchronize(st));
    float kms = 0.0f;
    SA_CUDA(cudaEventElapsedTime(&kms, ev0, ev1));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    int64_t total = 0;
    int conv = 1, nonfinite = 0;
    double last_res = 0.0;
    for (int k = k0; k < o->n_p; ++k) {
        total += h_out[k].matvecs;
        last_res = h_out[k].res;
        if (h_out[k].status != kNtConverged) conv = 0;
        if (h_out[k].status == kNtNonfinite) nonfinite = 1;
    }
    if (info) {
        info->sweeps_total = total;
        info->residual = last_res;
        info->p_final = o->p[o->n_p - 1];
        info->converged = conv;
        info->steps_done = o->n_p - k0;
        info->fallback_rows = 0;
        info->kernel_used = SA_KERNEL_NEWTON;
        info->kernel_ms = kms;
        info->sparse_epochs = 0;
        info->reanchors = 0;
    }
    if (*h_err == kErrTimeout) {
        set_error("newton scaling: a bounded grid-barrier wait timed out (grid of %d blocks)", P.grid);
        return SA_E_TIMEOUT;
    }
    if (nonfinite) {
        set_error("newton scaling: a row or column sum was zero or not finite (matrix without support?)");
        return SA_E_NONFINITE;
    }
    return conv ? SA_OK : SA_E_NOT_CONVERGED;
}

}  // namespace sa
