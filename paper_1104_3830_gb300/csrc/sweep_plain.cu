// sweep_plain.cu -- the unfused Sinkhorn path: one row kernel and one column kernel per
// sweep, launched from a host loop (two reads of A per sweep).
//
// Log-domain iteration of Sec. 4.1.2 (Eqs. dad1-dad3 in log coordinates): in log2 units
//   row update     U_i = LSE2_j (p L_ij - V_j)        (L = log2 w)
//   column update  V_j = LSE2_i (p L_ij - U_i)
// with LSE2_k(e_k) = m + log2 sum_k 2^(e_k - m), m = max_k e_k (the max shift of the paper).
// The stopping residual is max_j |c_j - 1| for the row-stochastic iterate after the row
// update, c_j = 2^(V_new_j - V_old_j) (the eps-bistochastic measure of Sec. 4.2).
//
// Precision (sa_prec): MIXED and FP32 evaluate each exponent in FP32 (SFU log2/exp2);
// MIXED centres it on a per-row FP32 reference Lr_i = U_i/p so that only small numbers
// are added, and keeps U, V in FP64; FP32 also stores U, V as FP32.  FP64 evaluates
// everything in double precision.  This path is the comparison baseline for the fused
// single-read kernel and the fallback for layouts the fused kernel does not take.
#include <cmath>
#include <cstdio>

#include "common.cuh"
#include "sa_internal.h"

namespace sa {

namespace {

template <typename WT>
__device__ __forceinline__ float log2w_f32(WT w) {
    return lg2_approx((float)w);
}
template <typename WT>
__device__ __forceinline__ double log2w_f64(WT w) {
    return log2((double)w);
}

__device__ __forceinline__ void atomic_max_nonneg(float* addr, float v) {
    // non-negative floats order like their bit patterns
    atomicMax((unsigned*)addr, __float_as_uint(v));
}

// One block per row.  Reads V (FP64) or Vf, writes U (new) and the per-row centring
// data the column kernel needs (Lr = float(U/p), D = U - p*Lr).
template <typename WT, typename T, bool CENTER>
__global__ void row_lse_kernel(const WT* __restrict__ w, int n, int64_t ld, double p,
                               const double* __restrict__ Vd, const float* __restrict__ Vf,
                               double* __restrict__ U, float* __restrict__ Lr_out,
                               float* __restrict__ D_out, int* err, int round_f32) {
    const int i = blockIdx.x;
    const WT* row = w + (int64_t)i * ld;
    __shared__ T red[32];
    __shared__ T s_m;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T m = -INFINITY;
    T lr = 0;
    if (CENTER) lr = (T)(float)(U[i] / p);   // reference from the previous sweep
    const T pp = (T)p;
    // pass 1: max
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        T L;
        if constexpr (sizeof(T) == 4) L = log2w_f32(row[j]); else L = log2w_f64(row[j]);
        T vj;
        if constexpr (sizeof(T) == 4) vj = Vf[j]; else vj = Vd[j];
        T e = pp * (L - lr) - vj;
        m = e > m ? e : m;
    }
    if constexpr (sizeof(T) == 4) m = warp_max(m); else m = warp_max((double)m);
    if (lane == 0) red[wid] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        T mm = red[0];
        for (int k = 1; k < nw; ++k) mm = red[k] > mm ? red[k] : mm;
        s_m = mm;
    }
    __syncthreads();
    m = s_m;
    // pass 2: sum of 2^(e - m)
    T s = 0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        T L;
        if constexpr (sizeof(T) == 4) L = log2w_f32(row[j]); else L = log2w_f64(row[j]);
        T vj;
        if constexpr (sizeof(T) == 4) vj = Vf[j]; else vj = Vd[j];
        T e = pp * (L - lr) - vj;
        if constexpr (sizeof(T) == 4) s += ex2_approx(e - m); else s += exp2(e - m);
    }
    if constexpr (sizeof(T) == 4) s = warp_sum(s); else s = warp_sum((double)s);
    __syncthreads();
    if (lane == 0) red[wid] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        T ss = 0;
        for (int k = 0; k < nw; ++k) ss += red[k];
        if (!(m > -INFINITY) || !(ss > 0) || !isfinite((double)ss)) {
            atomicCAS(err, 0, kErrNonfinite);
        }
        double un = p * (double)lr + (double)m + log2((double)ss);
        if (round_f32) un = (double)(float)un;
        U[i] = un;
        float lrn = (float)(un / p);
        Lr_out[i] = lrn;
        D_out[i] = (float)(un - p * (double)lrn);
    }
}

// Column partial LSE over a chunk of rows: one thread per column, online max/sum.
template <typename WT, typename T>
__global__ void col_partial_kernel(const WT* __restrict__ w, int n, int64_t ld, double p,
                                   const double* __restrict__ U, const float* __restrict__ Lr,
                                   const float* __restrict__ D, int rows_per_chunk,
                                   T* __restrict__ pm, T* __restrict__ ps) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int chunk = blockIdx.y;
    if (j >= n) return;
    const int r0 = chunk * rows_per_chunk;
    const int r1 = min(n, r0 + rows_per_chunk);
    const T pp = (T)p;
    T m = -INFINITY, s = 0;
    for (int i = r0; i < r1; ++i) {
        T e;
        if constexpr (sizeof(T) == 4) {
            e = pp * (log2w_f32(w[(int64_t)i * ld + j]) - Lr[i]) - D[i];
        } else {
            e = pp * log2w_f64(w[(int64_t)i * ld + j]) - U[i];
        }
        if (e > m) {
            if constexpr (sizeof(T) == 4) s = s * ex2_approx(m - e) + 1.0f;
            else s = s * exp2(m - e) + 1.0;
            m = e;
        } else {
            if constexpr (sizeof(T) == 4) s += ex2_approx(e - m); else s += exp2(e - m);
        }
    }
    pm[(int64_t)chunk * n + j] = m;
    ps[(int64_t)chunk * n + j] = s;
}

// Combine the chunk partials of each column; V_new = M + log2 S (FP64), residual
// |2^(V_new - V_used) - 1| where V_used is the value the row kernel subtracted.
template <typename T>
__global__ void col_combine_kernel(int n, int nchunks, const T* __restrict__ pm,
                                   const T* __restrict__ ps, double* __restrict__ V,
                                   float* __restrict__ Vf, float* resid, int* err, int round_f32,
                                   int use_vf) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    float r = 0.0f;
    if (j < n) {
        double M = -INFINITY;
        for (int c = 0; c < nchunks; ++c) M = fmax(M, (double)pm[(int64_t)c * n + j]);
        double S = 0.0;
        for (int c = 0; c < nchunks; ++c) {
            double mc = (double)pm[(int64_t)c * n + j];
            if (mc > -INFINITY) S += (double)ps[(int64_t)c * n + j] * exp2(mc - M);
        }
        if (!(M > -INFINITY) || !(S > 0)) atomicCAS(err, 0, kErrNonfinite);
        double vn = M + log2(S);
        double vold = use_vf ? (double)Vf[j] : V[j];
        r = (float)fabs(exp2(vn - vold) - 1.0);
        if (round_f32) vn = (double)(float)vn;
        V[j] = vn;
        Vf[j] = (float)vn;
    }
    r = warp_max(r);
    if ((threadIdx.x & 31) == 0) atomic_max_nonneg(resid, r);
}

__global__ void scale_vec_kernel(double* x, int n, double f) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] *= f;
}
__global__ void to_float_kernel(const double* x, float* y, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (float)x[i];
}

template <typename WT, typename T, bool CENTER>
sa_status run_plain(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U,
                    double* V, sa_scale_info* info) {
    const int n = a->n;
    const int64_t ld = a->ld;
    const WT* w = (const WT*)a->w;
    cudaStream_t st = ctx->stream;
    const int rows_per_chunk = 256;
    const int nchunks = (n + rows_per_chunk - 1) / rows_per_chunk;
    size_t need = 4 * align_up((size_t)n * 4, 256) + 2 * align_up((size_t)nchunks * n * sizeof(T), 256) +
                  4096;
    sa_status rc = ctx->ws.reserve(need);
    if (rc) return rc;
    Carve cv(ctx->ws.ptr);
    float* Vf = cv.take<float>(n);
    float* Lr = cv.take<float>(n);
    float* D = cv.take<float>(n);
    T* pm = cv.take<T>((size_t)nchunks * n);
    T* ps = cv.take<T>((size_t)nchunks * n);
    float* resid = cv.take<float>(1);
    int* err = cv.take<int>(1);
    rc = ctx->pinned.reserve(64);
    if (rc) return rc;
    volatile float* h_res = (volatile float*)ctx->pinned.ptr;
    volatile int* h_err = (volatile int*)((char*)ctx->pinned.ptr + 16);
    SA_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    const int round_f32 = (o->prec == SA_PREC_FP32);
    const int nt = 256;
    const int k0 = o->resume_from > 0 ? o->resume_from : 0;
    if (k0 == 0) {
        SA_CUDA(cudaMemsetAsync(U, 0, n * sizeof(double), st));
        SA_CUDA(cudaMemsetAsync(V, 0, n * sizeof(double), st));
    }
    cudaEvent_t ev0, ev1;
    SA_CUDA(cudaEventCreate(&ev0));
    SA_CUDA(cudaEventCreate(&ev1));
    SA_CUDA(cudaEventRecord(ev0, st));
    int64_t total = 0;
    int conv_all = 1;
    double last_res = INFINITY;
    for (int k = k0; k < o->n_p; ++k) {
        const double p = o->p[k];
        NvtxRange range("p step %d (p=%g)", k, p);
        if (k > 0 && !o->warm_keep_v) {
            double f = p / o->p[k - 1];
            scale_vec_kernel<<<(n + 255) / 256, 256, 0, st>>>(U, n, f);
            count_launch();
            scale_vec_kernel<<<(n + 255) / 256, 256, 0, st>>>(V, n, f);
            count_launch();
        }
        to_float_kernel<<<(n + 255) / 256, 256, 0, st>>>(V, Vf, n);
        count_launch();
        int s = 0;
        bool conv = false;
        while (s < o->max_sweeps_per_p) {
            SA_CUDA(cudaMemsetAsync(resid, 0, sizeof(float), st));
            row_lse_kernel<WT, T, CENTER><<<n, nt, 0, st>>>(w, n, ld, p, V, Vf, U, Lr, D, err, round_f32);
            count_launch();
            dim3 g2((n + 127) / 128, nchunks);
            col_partial_kernel<WT, T><<<g2, 128, 0, st>>>(w, n, ld, p, U, Lr, D, rows_per_chunk, pm, ps);
            count_launch();
            col_combine_kernel<T><<<(n + 255) / 256, 256, 0, st>>>(n, nchunks, pm, ps, V, Vf, resid, err,
                                                                   round_f32, sizeof(T) == 4);
            count_launch();
            ++s;
            SA_CUDA(cudaMemcpyAsync((void*)h_res, resid, sizeof(float), cudaMemcpyDeviceToHost, st));
            SA_CUDA(cudaMemcpyAsync((void*)h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st));
            SA_CUDA(cudaStreamSynchronize(st));
            if (*h_err) break;
            last_res = *h_res;
            if (last_res <= o->tol) { conv = true; break; }
        }
        total += s;
        if (*h_err) {
            set_error("plain sweep: row or column lost all mass at p=%g", p);
            return SA_E_NONFINITE;
        }
        if (!conv) conv_all = 0;
        if (info) { info->steps_done = k - k0 + 1; info->p_final = p; }
    }
    SA_CUDA(cudaEventRecord(ev1, st));
    SA_CUDA(cudaEventSynchronize(ev1));
    float kms = 0.0f;
    cudaEventElapsedTime(&kms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (info) {
        info->kernel_ms = kms;
        info->sweeps_total = total;
        info->residual = last_res;
        info->converged = conv_all;
        info->fallback_rows = 0;
        info->kernel_used = SA_KERNEL_PLAIN;
    }
    return conv_all ? SA_OK : SA_E_NOT_CONVERGED;
}

}  // namespace

void launch_scale_vec(double* x, int n, double f, cudaStream_t s) {
    if (n > 0) scale_vec_kernel<<<(n + 255) / 256, 256, 0, s>>>(x, n, f);
    count_launch();
}

sa_status scale_plain(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U,
                      double* V, sa_scale_info* info) {
    const bool i16 = a->wtype == SA_I16;
    switch (o->prec) {
        case SA_PREC_FP64:
            return i16 ? run_plain<int16_t, double, false>(ctx, a, o, U, V, info)
                       : run_plain<int32_t, double, false>(ctx, a, o, U, V, info);
        case SA_PREC_FP32:
            return i16 ? run_plain<int16_t, float, false>(ctx, a, o, U, V, info)
                       : run_plain<int32_t, float, false>(ctx, a, o, U, V, info);
        default:
            return i16 ? run_plain<int16_t, float, true>(ctx, a, o, U, V, info)
                       : run_plain<int32_t, float, true>(ctx, a, o, U, V, info);
    }
}

}  // namespace sa
