// newton.cu -- diagonal scaling of A^(p) by Newton iteration (Sec. 5.3, the variant after
// Knight and Ruiz), the SA_KERNEL_NEWTON path of sa_scale.
//
// At every p of the schedule:
//  1. K_ij = 2^(p log2 w_ij - C_i - V_j) with C_i = max_j (p log2 w_ij - V_j): the exponent
//     in FP64 (exact log2 table for int16 weights), one FP32 rounding, written once as an
//     n x ldk FP32 matrix.  X(p) is invariant under diagonal scaling (Sec. 2.1), so
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
// Control runs on the device.  A step is three launches: the matvec (one read of K),
// the finalisation (column sums, v or w, one reduction) and the vector update (second
// reduction).  The last block of the finalisation and of the update takes the scalar
// decisions in a control block that the next launch reads; once the step converges every
// launch returns at once.  The host queues batches of steps and polls the control block
// between batches; no kernel waits on another block.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "common.cuh"
#include "sa_internal.h"

namespace sa {

namespace {

constexpr int kNtThreads = 256;
constexpr int kNtWarps = kNtThreads / 32;
constexpr int kNtBatch = 8;          // steps queued between polls of the control block
constexpr double kNtDelta = 0.1;     // smallest y kept by a Newton step
constexpr double kNtEtaMax = 0.1;    // forcing term of the inner solve: eta = sqrt(res),
constexpr double kNtEtaMin = 1e-3;   //   clamped to [kNtEtaMin, kNtEtaMax]
constexpr int kNtCgCap = 200;        // CG iterations per Newton step

enum : int { kNtRes = 0, kNtCg = 1, kNtDone = 2 };
enum : int { kNtRunning = 0, kNtConverged = 1, kNtCapped = 2, kNtNonfinite = 3 };

struct NtCtl {
    int mode;        // kNtRes: next matvec is of 1 (residual); kNtCg: of r; kNtDone
    int cstage;      // 1: the update kernel applies a CG step
    int first;       // first CG iteration of the Newton step (beta = 0)
    int apply;       // pending x <- x o (1 + tau (y - 1)), applied by the next matvec step
    int breakdown;   // CG curvature not positive: end the inner solve
    int status;
    int matvecs;     // operator applications in this p step
    int cap;
    int cg_it;
    int newton_it;
    unsigned cnt_b, cnt_c;   // last-block counters of the finalise / update kernels
    double tol, tau, res, gamma, gamma0, gamma_prev, alpha, alpha_prev, beta, thr;
};

struct NtArgs {
    const float* K;
    int n;
    int ldk;        // row pitch of K and of the column partials (floats, multiple of 4)
    int T;          // column tiles
    int W4;         // float4 chunks per column tile
    int R;          // row stripes
    int rows_per;
    double* x;      // 2n: rho | kappa
    double* v;      // 2n
    double* y;
    double* r;
    double* pd;
    double* s;
    double* w;
    double* prt;    // T x n row partials
    float* pc;      // R x ldk column partials
    double* bred;   // finalisation block partials (4 per block)
    double* cred;   // update block partials (4 per block)
    NtCtl* ctl;
};

__device__ __forceinline__ double wlog2_f64(int w, const double* __restrict__ ltab) {
    return w < 32768 ? __ldg(ltab + w) : log2((double)w);
}

template <typename WT>
__device__ __forceinline__ int load_weight(const WT* p) {
    return (int)*p;
}

// log2 of 1..32767 in FP64 (entry 0 unused)
__global__ void nt_ltab_kernel(double* t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 32768) t[i] = i > 0 ? log2((double)i) : -INFINITY;
}

// C_i = max_j (p log2 w_ij - V_j) over w_ij > 0; one warp per row
template <typename WT>
__global__ void nt_rowmax_kernel(const WT* __restrict__ w, int n, int64_t ld, double p,
                                 const double* __restrict__ V, const double* __restrict__ ltab,
                                 double* __restrict__ C) {
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n) return;
    const WT* wr = w + (int64_t)row * ld;
    double m = -INFINITY;
    for (int j = lane; j < n; j += 32) {
        const int wv = load_weight(wr + j);
        if (wv > 0) m = fmax(m, __fma_rn(p, wlog2_f64(wv, ltab), -__ldg(V + j)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) C[row] = m;
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

// K_ij = 2^(d), d = (p log2 w_ij - V_j) - C_i <= 0 in FP64, as 2^hi (1 + lo ln 2) with
// hi + lo = d; pad columns and zero weights give 0.  Also the column maxima of K over each
// row stripe (pc), from which the starting kappa is taken.
template <typename WT, int CH>
__global__ void __launch_bounds__(kNtThreads) nt_kwrite_kernel(const WT* __restrict__ w, int64_t ld,
                                                               double p, const double* __restrict__ V,
                                                               const double* __restrict__ C,
                                                               const double* __restrict__ ltab,
                                                               NtArgs A) {
    const int tid = threadIdx.x;
    const int t = blockIdx.x % A.T, s = blockIdx.x / A.T;
    const int r0 = s * A.rows_per, r1 = min(A.n, r0 + A.rows_per);
    const int n = A.n;
    double vj[4 * CH];
    float cm[4 * CH];
    int q[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        q[k] = t * A.W4 + tid + kNtThreads * k;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = 4 * q[k] + e;
            vj[4 * k + e] = j < n ? V[j] : 0.0;
            cm[4 * k + e] = 0.0f;
        }
    }
    for (int i = r0; i < r1; ++i) {
        const double ci = C[i];
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
                    const double d = __fma_rn(p, wlog2_f64(wv[e], ltab), -vj[4 * k + e]) - ci;
                    const float hi = __double2float_rn(d);
                    const float lo = __double2float_rn(d - (double)hi);
                    const float k0 = exp2f(hi);
                    kv[e] = fmaf(k0, lo * 0.693147182f, k0);
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

// starting point and control block of a p step
__global__ void nt_init_kernel(NtArgs A, double tol, int cap) {
    const int n = A.n;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * n; e += gridDim.x * blockDim.x) {
        double xe = 1.0;
        if (e >= n) {
            const int j = e - n;
            float m = 0.0f;
            for (int s = 0; s < A.R; ++s) m = fmaxf(m, A.pc[(int64_t)s * A.ldk + j]);
            xe = 1.0 / (double)m;   // +inf for an empty column: caught by the first residual
        }
        A.x[e] = xe;
        A.y[e] = 1.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        NtCtl c{};
        c.mode = kNtRes;
        c.status = kNtRunning;
        c.cap = cap;
        c.tol = tol;
        c.tau = 1.0;
        *A.ctl = c;
    }
}

// D(x) S D(x) z for z = 1 (residual) or z = r (CG): one read of K.  Block (s, t) takes the
// rows of stripe s and the columns of tile t; each thread owns CH float4 chunks of columns.
// Row results go to prt[t][i] (FP64, complete over the tile), column results to pc[s][j].
template <int CH>
__global__ void __launch_bounds__(kNtThreads, 2) nt_matvec_kernel(NtArgs A) {
    __shared__ float red[2][kNtWarps][4];
    extern __shared__ float zr_s[];
    const NtCtl* ctl = A.ctl;
    const int mode = ctl->mode;
    if (mode == kNtDone) return;
    const bool res_mode = mode == kNtRes;
    const bool apply = ctl->apply != 0;
    const double tau = ctl->tau;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int t = blockIdx.x % A.T, s = blockIdx.x / A.T;
    const int r0 = s * A.rows_per, r1 = min(A.n, r0 + A.rows_per);
    const int n = A.n;
    float z[4 * CH], acc[4 * CH];
    int q[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        q[k] = t * A.W4 + tid + kNtThreads * k;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int j = 4 * q[k] + e;
            float zv = 0.0f;
            if (j < n) {
                double xe = A.x[n + j];
                if (apply) xe *= 1.0 + tau * (A.y[n + j] - 1.0);
                zv = (float)(res_mode ? xe : xe * A.r[n + j]);
            }
            z[4 * k + e] = zv;
            acc[4 * k + e] = 0.0f;
        }
    }
    for (int i = r0 + tid; i < r1; i += kNtThreads) {
        double xe = A.x[i];
        if (apply) xe *= 1.0 + tau * (A.y[i] - 1.0);
        zr_s[i - r0] = (float)(res_mode ? xe : xe * A.r[i]);
    }
    __syncthreads();
    int buf = 0;
    for (int i = r0; i < r1; i += 4) {
        float4 kv[4][CH];
#pragma unroll
        for (int g = 0; g < 4; ++g)
#pragma unroll
            for (int k = 0; k < CH; ++k)
                kv[g][k] = (i + g < r1 && 4 * q[k] < n)
                               ? *(const float4*)(A.K + (int64_t)(i + g) * A.ldk + 4 * q[k])
                               : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float dot[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const float zr = i + g < r1 ? zr_s[i + g - r0] : 0.0f;
            float d = 0.0f;
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                d = fmaf(kv[g][k].x, z[4 * k], d);
                d = fmaf(kv[g][k].y, z[4 * k + 1], d);
                d = fmaf(kv[g][k].z, z[4 * k + 2], d);
                d = fmaf(kv[g][k].w, z[4 * k + 3], d);
                acc[4 * k] = fmaf(kv[g][k].x, zr, acc[4 * k]);
                acc[4 * k + 1] = fmaf(kv[g][k].y, zr, acc[4 * k + 1]);
                acc[4 * k + 2] = fmaf(kv[g][k].z, zr, acc[4 * k + 2]);
                acc[4 * k + 3] = fmaf(kv[g][k].w, zr, acc[4 * k + 3]);
            }
            dot[g] = d;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int g = 0; g < 4; ++g) dot[g] += __shfl_xor_sync(0xffffffffu, dot[g], o);
        if (lane == 0) {
#pragma unroll
            for (int g = 0; g < 4; ++g) red[buf][wid][g] = dot[g];
        }
        __syncthreads();
        if (tid < 4 && i + tid < r1) {
            double sm = 0.0;
#pragma unroll
            for (int x = 0; x < kNtWarps; ++x) sm += (double)red[buf][x][tid];
            A.prt[(int64_t)t * n + i + tid] = sm;
        }
        buf ^= 1;
    }
#pragma unroll
    for (int k = 0; k < CH; ++k)
        if (4 * q[k] < n)
            *(float4*)(A.pc + (int64_t)s * A.ldk + 4 * q[k]) =
                make_float4(acc[4 * k], acc[4 * k + 1], acc[4 * k + 2], acc[4 * k + 3]);
}

// block sum / min / max of doubles over 256 threads; result valid in thread 0
__device__ __forceinline__ double nt_block_sum(double x, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < kNtWarps; ++k) r += sh[k];
    return r;
}
__device__ __forceinline__ double nt_block_max(double x, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = x;
    __syncthreads();
    double r = -INFINITY;
    if (threadIdx.x == 0)
        for (int k = 0; k < kNtWarps; ++k) r = fmax(r, sh[k]);
    return r;
}
__device__ __forceinline__ double nt_block_min(double x, double* sh) {
    return -nt_block_max(-x, sh);
}

// true in thread 0 of the last block to finish (its partials are then all visible)
__device__ __forceinline__ bool nt_last_block(unsigned* cnt, int* s_last) {
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(cnt, 1u);
        *s_last = prev == gridDim.x - 1;
        if (*s_last) __threadfence();
    }
    __syncthreads();
    return *s_last != 0;
}

// Column sums (over the stripes) and row sums (over the tiles) of the matvec, scaled by x:
// m = D(x) S D(x) z.  Residual step: v = m, r = 1 - v, y = 1.  CG step: w = m + v o r.
// Grid: ceil(n/32) column blocks, then ceil(n/256) row blocks.
__global__ void __launch_bounds__(kNtThreads) nt_fin_kernel(NtArgs A) {
    __shared__ double sred[kNtWarps][33];
    __shared__ double sh[kNtWarps];
    __shared__ int s_last;
    NtCtl* ctl = A.ctl;
    const int mode = ctl->mode;
    if (mode == kNtDone) return;
    const bool res_mode = mode == kNtRes;
    const bool apply = ctl->apply != 0;
    const double tau = ctl->tau;
    const int n = A.n, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nbc = (n + 31) / 32;
    int e = -1;
    double tot = 0.0;
    if ((int)blockIdx.x < nbc) {
        const int j = blockIdx.x * 32 + lane;
        double sm = 0.0;
        if (j < n)
            for (int s = wid; s < A.R; s += kNtWarps) sm += (double)A.pc[(int64_t)s * A.ldk + j];
        sred[wid][lane] = sm;
        __syncthreads();
        if (wid == 0 && j < n) {
            for (int x = 0; x < kNtWarps; ++x) tot += sred[x][lane];
            e = n + j;
        }
    } else {
        const int i = (blockIdx.x - nbc) * kNtThreads + tid;
        if (i < n) {
            for (int t = 0; t < A.T; ++t) tot += A.prt[(int64_t)t * n + i];
            e = i;
        }
    }
    double a0 = 0.0, a1 = 0.0, a2 = INFINITY;   // residual: max|v-1|, sum (1-v)^2, min v
                                                // CG: sum w r
    if (e >= 0) {
        double xe = A.x[e];
        if (apply) {
            xe *= 1.0 + tau * (A.y[e] - 1.0);
            A.x[e] = xe;
        }
        const double m = xe * tot;
        if (res_mode) {
            A.v[e] = m;
            A.r[e] = 1.0 - m;
            A.y[e] = 1.0;
            a0 = fabs(m - 1.0);
            a1 = (1.0 - m) * (1.0 - m);
            a2 = (m > 0.0 && m < INFINITY) ? m : -1.0;   // -1 flags a zero or non-finite sum
        } else {
            const double re = A.r[e];
            const double we = m + A.v[e] * re;
            A.w[e] = we;
            a0 = we * re;
            a2 = (we > -INFINITY && we < INFINITY) ? 1.0 : -1.0;
        }
    }
    const double b0 = res_mode ? nt_block_max(a0, sh) : nt_block_sum(a0, sh);
    const double b1 = nt_block_sum(a1, sh);
    const double b2 = nt_block_min(a2, sh);
    if (tid == 0) {
        A.bred[4 * blockIdx.x] = b0;
        A.bred[4 * blockIdx.x + 1] = b1;
        A.bred[4 * blockIdx.x + 2] = b2;
    }
    if (!nt_last_block(&ctl->cnt_b, &s_last)) return;
    double c0 = res_mode ? -INFINITY : 0.0, c1 = 0.0, c2 = INFINITY;
    for (int b = tid; b < (int)gridDim.x; b += kNtThreads) {
        const double x0 = __ldcg(A.bred + 4 * b), x1 = __ldcg(A.bred + 4 * b + 1), x2 = __ldcg(A.bred + 4 * b + 2);
        c0 = res_mode ? fmax(c0, x0) : c0 + x0;
        c1 += x1;
        c2 = fmin(c2, x2);
    }
    const double g0 = res_mode ? nt_block_max(c0, sh) : nt_block_sum(c0, sh);
    const double g1 = nt_block_sum(c1, sh);
    const double g2 = nt_block_min(c2, sh);
    if (tid != 0) return;
    NtCtl c = *ctl;
    c.cnt_b = 0;
    c.matvecs += 1;
    c.cstage = 0;
    if (!(g2 > 0.0)) {
        c.status = kNtNonfinite;
        c.mode = kNtDone;
    } else if (res_mode) {
        c.res = g0;
        c.apply = 0;
        if (g0 <= c.tol) {
            c.status = kNtConverged;
            c.mode = kNtDone;
        } else if (c.matvecs >= c.cap) {
            c.status = kNtCapped;
            c.mode = kNtDone;
        } else {
            const double eta = fmin(kNtEtaMax, fmax(kNtEtaMin, sqrt(g0)));
            c.gamma = c.gamma0 = g1;
            c.thr = eta * eta * g1;
            c.first = 1;
            c.cg_it = 0;
            c.breakdown = 0;
            c.mode = kNtCg;
        }
    } else {
        const double delta = g0;
        if (c.first) {
            c.beta = 0.0;
            c.alpha = c.gamma / delta;
        } else {
            c.beta = c.gamma / c.gamma_prev;
            c.alpha = c.gamma / (delta - c.beta * c.gamma / c.alpha_prev);
        }
        if (!(c.alpha > 0.0 && c.alpha < INFINITY)) {
            c.alpha = 0.0;
            c.breakdown = 1;
        }
        c.cstage = 1;
    }
    *ctl = c;
}

// p = r + beta p, s = w + beta s, y += alpha p, r -= alpha s; the last block ends the
// inner solve (||r||^2 <= eta^2 ||r_0||^2, CG cap, min y < delta, breakdown, matvec cap)
__global__ void __launch_bounds__(kNtThreads) nt_upd_kernel(NtArgs A) {
    __shared__ double sh[kNtWarps];
    __shared__ int s_last;
    NtCtl* ctl = A.ctl;
    if (ctl->mode == kNtDone || ctl->cstage != 1) return;
    const bool first = ctl->first != 0;
    const double alpha = ctl->alpha, beta = ctl->beta;
    const int n2 = 2 * A.n, tid = threadIdx.x;
    double rr = 0.0, ymin = INFINITY;
    for (int e = blockIdx.x * kNtThreads + tid; e < n2; e += gridDim.x * kNtThreads) {
        const double re = A.r[e], we = A.w[e];
        const double pe = first ? re : re + beta * A.pd[e];
        const double se = first ? we : we + beta * A.s[e];
        const double ye = A.y[e] + alpha * pe;
        const double rn = re - alpha * se;
        A.pd[e] = pe;
        A.s[e] = se;
        A.y[e] = ye;
        A.r[e] = rn;
        rr += rn * rn;
        ymin = fmin(ymin, ye);
    }
    const double b0 = nt_block_sum(rr, sh);
    const double b1 = nt_block_min(ymin, sh);
    if (tid == 0) {
        A.cred[4 * blockIdx.x] = b0;
        A.cred[4 * blockIdx.x + 1] = b1;
    }
    if (!nt_last_block(&ctl->cnt_c, &s_last)) return;
    double c0 = 0.0, c1 = INFINITY;
    for (int b = tid; b < (int)gridDim.x; b += kNtThreads) {
        c0 += __ldcg(A.cred + 4 * b);
        c1 = fmin(c1, __ldcg(A.cred + 4 * b + 1));
    }
    const double g0 = nt_block_sum(c0, sh);
    const double g1 = nt_block_min(c1, sh);
    if (tid != 0) return;
    NtCtl c = *ctl;
    c.cnt_c = 0;
    c.cstage = 0;
    c.gamma_prev = c.gamma;
    c.gamma = g0;
    c.alpha_prev = c.alpha;
    c.first = 0;
    c.cg_it += 1;
    if (!(g0 < INFINITY) || !(g1 > -INFINITY && g1 < INFINITY)) {
        c.status = kNtNonfinite;
        c.mode = kNtDone;
    } else if (g0 <= c.thr || c.cg_it >= kNtCgCap || g1 < kNtDelta || c.breakdown || c.matvecs >= c.cap) {
        c.apply = 1;
        c.tau = g1 < kNtDelta ? (1.0 - kNtDelta) / (1.0 - g1) : 1.0;
        c.mode = kNtRes;
        c.newton_it += 1;
    }
    *ctl = c;
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
    int ch, T, W4, R, rows_per, grid_a, nb_fin, nb_upd;
};

template <int CH>
int nt_occupancy(size_t smem) {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, nt_matvec_kernel<CH>, kNtThreads, smem);
    return occ;
}

NtPlan nt_plan(const sa_ctx* ctx, int n) {
    NtPlan P{};
    P.ch = n <= 1024 ? 1 : n <= 2048 ? 2 : 4;
    P.W4 = kNtThreads * P.ch;
    P.T = (n + 4 * P.W4 - 1) / (4 * P.W4);
    int occ = P.ch == 1 ? nt_occupancy<1>(0) : P.ch == 2 ? nt_occupancy<2>(0) : nt_occupancy<4>(0);
    occ = std::max(1, std::min(occ, 2));
    int G = ctx->num_sms * occ;
    if (ctx->max_grid > 0) G = std::min(G, ctx->max_grid);
    int R = std::max(1, std::min(n, G / P.T));
    P.rows_per = (n + R - 1) / R;
    P.R = (n + P.rows_per - 1) / P.rows_per;
    P.grid_a = P.R * P.T;
    P.nb_fin = (n + 31) / 32 + (n + kNtThreads - 1) / kNtThreads;
    P.nb_upd = std::max(1, std::min((2 * n + kNtThreads - 1) / kNtThreads, 2 * ctx->num_sms));
    return P;
}

sa_status launch_matvec(const NtPlan& P, const NtArgs& A, cudaStream_t st) {
    const size_t smem = (size_t)P.rows_per * sizeof(float);
    if (P.ch == 1) nt_matvec_kernel<1><<<P.grid_a, kNtThreads, smem, st>>>(A);
    else if (P.ch == 2) nt_matvec_kernel<2><<<P.grid_a, kNtThreads, smem, st>>>(A);
    else nt_matvec_kernel<4><<<P.grid_a, kNtThreads, smem, st>>>(A);
    return SA_OK;
}

template <typename WT>
void launch_eval(const NtPlan& P, const sa_matrix* a, double p, const double* V, const double* C,
                 const double* ltab, const NtArgs& A, cudaStream_t st) {
    const WT* w = (const WT*)a->w;
    if (P.ch == 1) nt_kwrite_kernel<WT, 1><<<P.grid_a, kNtThreads, 0, st>>>(w, a->ld, p, V, C, ltab, A);
    else if (P.ch == 2) nt_kwrite_kernel<WT, 2><<<P.grid_a, kNtThreads, 0, st>>>(w, a->ld, p, V, C, ltab, A);
    else nt_kwrite_kernel<WT, 4><<<P.grid_a, kNtThreads, 0, st>>>(w, a->ld, p, V, C, ltab, A);
}

}  // namespace

bool newton_supported(const sa_ctx* ctx, const sa_matrix* a) {
    (void)ctx;
    const int sz = wbytes(a->wtype);
    if (((uintptr_t)a->w & 15) != 0) return false;
    if (((size_t)a->ld * sz) % 16 != 0) return false;
    return a->n >= 1 && a->n <= (1 << 16);
}

sa_status scale_newton(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U, double* V,
                       sa_scale_info* info) {
    const int n = a->n;
    cudaStream_t st = ctx->stream;
    const NtPlan P = nt_plan(ctx, n);
    const int ldk = (int)align_up((size_t)n, 4);
    size_t bytes = 0;
    {
        bytes += align_up((size_t)n * ldk * 4, 256);
        bytes += align_up((size_t)n * 8, 256);            // C
        bytes += 7 * align_up((size_t)2 * n * 8, 256);    // x v y r p s w
        bytes += align_up((size_t)P.T * n * 8, 256);      // prt
        bytes += align_up((size_t)P.R * ldk * 4, 256);    // pc
        bytes += align_up((size_t)P.nb_fin * 32, 256);
        bytes += align_up((size_t)P.nb_upd * 32, 256);
        bytes += align_up(sizeof(NtCtl), 256);
        bytes += align_up((size_t)32768 * 8, 256);
        bytes += 4096;
    }
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
    A.prt = cv.take<double>((size_t)P.T * n);
    A.pc = cv.take<float>((size_t)P.R * ldk);
    A.bred = cv.take<double>((size_t)P.nb_fin * 4);
    A.cred = cv.take<double>((size_t)P.nb_upd * 4);
    A.ctl = cv.take<NtCtl>(1);
    double* ltab = cv.take<double>(32768);
    A.n = n;
    A.ldk = ldk;
    A.T = P.T;
    A.W4 = P.W4;
    A.R = P.R;
    A.rows_per = P.rows_per;

    rc = ctx->pinned.reserve(2 * align_up(sizeof(NtCtl), 64));
    if (rc) return rc;
    NtCtl* h_ctl[2] = {(NtCtl*)ctx->pinned.ptr, (NtCtl*)((char*)ctx->pinned.ptr + align_up(sizeof(NtCtl), 64))};

    const int k0 = o->resume_from > 0 ? o->resume_from : 0;
    if (k0 == 0) {
        SA_CUDA(cudaMemsetAsync(U, 0, n * sizeof(double), st));
        SA_CUDA(cudaMemsetAsync(V, 0, n * sizeof(double), st));
    }
    nt_ltab_kernel<<<32768 / 256, 256, 0, st>>>(ltab);
    count_launch();
    cudaEvent_t ev0, ev1, evb[2];
    SA_CUDA(cudaEventCreate(&ev0));
    SA_CUDA(cudaEventCreate(&ev1));
    SA_CUDA(cudaEventCreateWithFlags(&evb[0], cudaEventDisableTiming));
    SA_CUDA(cudaEventCreateWithFlags(&evb[1], cudaEventDisableTiming));
    auto destroy = [&]() {
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        cudaEventDestroy(evb[0]);
        cudaEventDestroy(evb[1]);
    };
    SA_CUDA(cudaEventRecord(ev0, st));
    int64_t total = 0;
    int conv = 1, nonfinite = 0;
    double last_res = 0.0;
    for (int k = k0; k < o->n_p; ++k) {
        const double p = o->p[k];
        if (k > 0 && !o->warm_keep_v) launch_scale_vec(V, n, p / o->p[k - 1], st);
        if (a->wtype == SA_I16)
            nt_rowmax_kernel<int16_t><<<(n + 7) / 8, 256, 0, st>>>((const int16_t*)a->w, n, a->ld, p, V, ltab, C);
        else
            nt_rowmax_kernel<int32_t><<<(n + 7) / 8, 256, 0, st>>>((const int32_t*)a->w, n, a->ld, p, V, ltab, C);
        if (a->wtype == SA_I16) launch_eval<int16_t>(P, a, p, V, C, ltab, A, st);
        else launch_eval<int32_t>(P, a, p, V, C, ltab, A, st);
        nt_init_kernel<<<std::max(1, std::min((2 * n + 255) / 256, 4 * ctx->num_sms)), 256, 0, st>>>(
            A, o->tol, o->max_sweeps_per_p);
        count_launch(3);
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) { destroy(); return cuda_fail(le, "newton evaluation"); }
        // batches of steps; at most two in flight, polled through pinned copies
        const int max_batches = (o->max_sweeps_per_p + 2) / kNtBatch + 3;
        int issued = 0, polled = 0;
        bool done = false;
        auto issue = [&]() -> sa_status {
            for (int b = 0; b < kNtBatch; ++b) {
                launch_matvec(P, A, st);
                nt_fin_kernel<<<P.nb_fin, kNtThreads, 0, st>>>(A);
                nt_upd_kernel<<<P.nb_upd, kNtThreads, 0, st>>>(A);
            }
            count_launch(3 * kNtBatch);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e, "newton step");
            SA_CUDA(cudaMemcpyAsync(h_ctl[issued & 1], A.ctl, sizeof(NtCtl), cudaMemcpyDeviceToHost, st));
            SA_CUDA(cudaEventRecord(evb[issued & 1], st));
            ++issued;
            return SA_OK;
        };
        while (!done) {
            while (issued - polled < 2 && issued < max_batches) {
                if ((rc = issue())) { destroy(); return rc; }
            }
            if (polled == issued) break;
            cudaError_t e = cudaEventSynchronize(evb[polled & 1]);
            if (e != cudaSuccess) { destroy(); return cuda_fail(e, "newton poll"); }
            done = h_ctl[polled & 1]->mode == kNtDone;
            ++polled;
        }
        SA_CUDA(cudaStreamSynchronize(st));
        const NtCtl& c = *h_ctl[(polled - 1) & 1];
        if (c.mode != kNtDone) {
            destroy();
            set_error("newton scaling: the step at p = %g did not end within its matvec cap", p);
            return SA_E_NOT_CONVERGED;
        }
        total += c.matvecs;
        last_res = c.res;
        if (c.status == kNtNonfinite) {
            nonfinite = 1;
            conv = 0;
            break;
        }
        if (c.status != kNtConverged) conv = 0;
        nt_potentials_kernel<<<(n + 255) / 256, 256, 0, st>>>(A.x, C, U, V, n);
        count_launch();
    }
    SA_CUDA(cudaEventRecord(ev1, st));
    SA_CUDA(cudaStreamSynchronize(st));
    float kms = 0.0f;
    SA_CUDA(cudaEventElapsedTime(&kms, ev0, ev1));
    destroy();
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
    if (nonfinite) {
        set_error("newton scaling: a row or column sum was zero or not finite (matrix without support?)");
        return SA_E_NONFINITE;
    }
    return conv ? SA_OK : SA_E_NOT_CONVERGED;
}

}  // namespace sa
