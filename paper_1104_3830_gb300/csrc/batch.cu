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
#include <numeric>
#include <vector>

#include "common.cuh"
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

}  // namespace
}  // namespace sa

using namespace sa;

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
    std::vector<int32_t> order(k);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hn[a] > hn[b]; });
    const int maxn = hn[order[0]];
    const int vec = 16 / sz;
    const int kc = ((maxn + vec - 1) / vec + 31) / 32;   // chunks per lane
    size_t need = align_up((size_t)k * 4, 256) * 3 + align_up((size_t)o->n_p * 8, 256) + 1024;
    sa_status rc = ctx->ws.reserve(need);
    if (rc) return rc;
    Carve cv(ctx->ws.ptr);
    int32_t* d_order = cv.take<int32_t>(k);
    int32_t* d_sw = cv.take<int32_t>(k);
    int32_t* d_st = cv.take<int32_t>(k);
    double* d_P = cv.take<double>(o->n_p);
    unsigned* d_q = cv.take<unsigned>(1);
    SA_CUDA(cudaMemcpyAsync(d_order, order.data(), 4 * k, cudaMemcpyHostToDevice, st));
    SA_CUDA(cudaMemcpyAsync(d_P, o->p, 8 * o->n_p, cudaMemcpyHostToDevice, st));
    SA_CUDA(cudaMemsetAsync(d_q, 0, 4, st));
    BatchArgs args{d_w, d_n, d_ld, d_off, d_order, k, wtype == SA_I16, d_P, o->n_p, o->tol, o->max_sweeps_per_p,
                   d_u, d_v, d_sw, d_st, d_q, 0};
    constexpr int NT = 256;
    constexpr int NW = NT / 32;
    const size_t fixed = kBatchMaxN * 8 + 4 * kBatchMaxN * 4 + (size_t)NW * kBatchMaxN * 4 + NW * 8 + 64;
    size_t smem = std::min<size_t>(ctx->smem_optin, 110 * 1024);   // two blocks per SM
    args.smem_table = smem > fixed ? smem - fixed : 0;
    int grid = 0;
    auto launch = [&](auto kern) -> sa_status {
        SA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        SA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
        grid = std::max(1, std::min(k, ctx->num_sms * std::max(per_sm, 1)));
        kern<<<grid, NT, smem, st>>>(args);
        count_launch();
        return SA_OK;
    };
    if (wtype == SA_I16) {
        if (kc <= 1) rc = launch(batch_kernel<int16_t, NT, 1>);
        else rc = launch(batch_kernel<int16_t, NT, 2>);
    } else {
        if (kc <= 1) rc = launch(batch_kernel<int32_t, NT, 1>);
        else if (kc <= 2) rc = launch(batch_kernel<int32_t, NT, 2>);
        else rc = launch(batch_kernel<int32_t, NT, 4>);
    }
    if (rc) return rc;
    SA_CUDA(cudaGetLastError());
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
