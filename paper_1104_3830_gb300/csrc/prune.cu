// prune.cu -- reduced instance B (Eq. matrixred) as CSR, the certificate of Prop. aoc,
// the LP-duality check of a solution on all of A, FP64 verification of the scaling, and
// int32 -> int16 narrowing.
//
// Keep test: x_ij(p) >= t  <=>  E_ij = p log2 w_ij - U_i - V_j >= log2 t  (log2 units).
// E is first evaluated in FP32 with the same centring as the sweeps; when it lies within
// a margin of the threshold (a bound on the FP32 error, 1e-4 + 4e-6 p) the decision is
// taken again in FP64, so every decision equals the FP64 one (up to the last bit of the
// FP64 logarithm).  Row and column guards (largest entry of every row and column) use the
// FP32 values with the lowest index on ties.
//
// CSR build: count per row -> exclusive scan -> write, one block per row, columns ascend.
// This file is compiled without FMA contraction so that the keep predicate evaluates to
// the same value in the counting and the writing kernels.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "sa_internal.h"

namespace sa {
namespace {

constexpr int kPruneThreads = 256;

struct PruneView {
    const void* w;
    int i16;
    int n;
    int64_t ld;
    double p;
    float pf;
    const double* U;    // log2 units, FP64
    const double* V;
    const float* Lr;    // float(U / p)
    const float* Dr;    // U - p*Lr
    const float* Vf;    // float(V)
    const float* Vd;    // V - Vf
    double log2t;
    float log2tf;
    float margin;
};

__device__ __forceinline__ int load_w(const PruneView& P, int i, int j) {
    return P.i16 ? (int)((const int16_t*)P.w)[(int64_t)i * P.ld + j]
                 : ((const int32_t*)P.w)[(int64_t)i * P.ld + j];
}

// FP32 screened value of E_ij (log2 units)
__device__ __forceinline__ float e32(const PruneView& P, int i, int j, int w) {
    const float L = lg2_approx((float)w);
    return fmaf(P.pf, L - P.Lr[i], -P.Vf[j]) - (P.Dr[i] + P.Vd[j]);
}

__device__ __forceinline__ bool keep_thr(const PruneView& P, int i, int j, int w, float e) {
    if (fabsf(e - P.log2tf) > P.margin) return e >= P.log2tf;
    const double ed = (w > 0 ? P.p * log2((double)w) : -INFINITY) - P.U[i] - P.V[j];
    return ed >= P.log2t;
}

__device__ __forceinline__ int block_sum_int(int v, int* sh) {
    v = __reduce_add_sync(0xffffffffu, v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int tot = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) tot += sh[k];
    __syncthreads();
    return tot;
}

// Per row: number of entries passing the threshold, FP32 argmax of E (lowest index on
// ties), and the certificate term max_j (p ln w_ij - v_j) evaluated in FP64 at it.
__global__ void prune_rows_kernel(PruneView P, int* cnt, int* rarg, double* rterm) {
    const int i = blockIdx.x;
    __shared__ int shc[32];
    __shared__ float shv[32];
    __shared__ int shi[32];
    int c = 0;
    float best = -INFINITY;
    int bj = 0x7fffffff;
    for (int j = threadIdx.x; j < P.n; j += blockDim.x) {
        const int w = load_w(P, i, j);
        const float e = w > 0 ? e32(P, i, j, w) : -INFINITY;
        c += keep_thr(P, i, j, w, e) ? 1 : 0;
        if (e > best) { best = e; bj = j; }
    }
    // (max, lowest index) reduction
    for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ob > best || (ob == best && oj < bj)) { best = ob; bj = oj; }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { shv[wid] = best; shi[wid] = bj; }
    const int tot = block_sum_int(c, shc);
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
            if (shv[k] > best || (shv[k] == best && shi[k] < bj)) { best = shv[k]; bj = shi[k]; }
        if (bj == 0x7fffffff) bj = 0;
        cnt[i] = tot;
        rarg[i] = bj;
        const int w = load_w(P, i, bj);
        rterm[i] = (w > 0 ? P.p * log((double)w) : -INFINITY) - P.V[bj] * kLn2;
    }
}

// Column argmax of E over a chunk of rows (thread per column); (value, row) partials.
__global__ void col_argmax_partial_kernel(PruneView P, int rows_per_chunk, float* pv, int* pi) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.n) return;
    const int r0 = blockIdx.y * rows_per_chunk;
    const int r1 = min(P.n, r0 + rows_per_chunk);
    float best = -INFINITY;
    int bi = r0;
    for (int i = r0; i < r1; ++i) {
        const int w = load_w(P, i, j);
        const float e = w > 0 ? e32(P, i, j, w) : -INFINITY;
        if (e > best) { best = e; bi = i; }
    }
    pv[(int64_t)blockIdx.y * P.n + j] = best;
    pi[(int64_t)blockIdx.y * P.n + j] = bi;
}

__global__ void col_argmax_combine_kernel(int n, int nchunks, const float* pv, const int* pi,
                                          int* carg) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float best = -INFINITY;
    int bi = 0;
    for (int c = 0; c < nchunks; ++c) {
        const float v = pv[(int64_t)c * n + j];
        if (v > best) { best = v; bi = pi[(int64_t)c * n + j]; }   // chunks ascend: lowest row on ties
    }
    carg[j] = bi;
}

// Guard entries not already kept by the threshold add one to their row's count.
__global__ void guard_count_kernel(PruneView P, const int* rarg, const int* carg, int* cnt) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.n) {   // row guard
        const int i = k, j = rarg[i];
        const int w = load_w(P, i, j);
        const float e = w > 0 ? e32(P, i, j, w) : -INFINITY;
        if (!keep_thr(P, i, j, w, e)) atomicAdd(&cnt[i], 1);
    } else if (k < 2 * P.n) {   // column guard
        const int j = k - P.n, i = carg[j];
        if (rarg[i] == j) return;
        const int w = load_w(P, i, j);
        const float e = w > 0 ? e32(P, i, j, w) : -INFINITY;
        if (!keep_thr(P, i, j, w, e)) atomicAdd(&cnt[i], 1);
    }
}

// Exclusive scan of n counts into row_ptr[0..n] (single block, n any size).
__global__ void scan_kernel(const int* cnt, int64_t* row_ptr, int n) {
    __shared__ int64_t sh[1024];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
        const int i = base + threadIdx.x;
        int64_t v = i < n ? cnt[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < (int)blockDim.x; o <<= 1) {
            int64_t add = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < n) row_ptr[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += sh[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) row_ptr[n] = carry;
}

// Write the kept columns of each row in ascending order (ballot ranks).
__global__ void prune_write_kernel(PruneView P, int guard, const int* rarg, const int* carg,
                                   const int64_t* row_ptr, int32_t* col, int32_t* wout) {
    const int i = blockIdx.x;
    __shared__ int wsum[32];
    __shared__ int64_t base_s;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) base_s = row_ptr[i];
    __syncthreads();
    const int ri = rarg[i];
    for (int j0 = 0; j0 < P.n; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        bool k = false;
        int w = 0;
        if (j < P.n) {
            w = load_w(P, i, j);
            const float e = w > 0 ? e32(P, i, j, w) : -INFINITY;
            k = keep_thr(P, i, j, w, e) || (guard && (j == ri || carg[j] == i));
        }
        const unsigned m = __ballot_sync(0xffffffffu, k);
        if (lane == 0) wsum[wid] = __popc(m);
        __syncthreads();
        int off = 0, tot = 0;
        for (int x = 0; x < nw; ++x) {
            if (x < wid) off += wsum[x];
            tot += wsum[x];
        }
        if (k) {
            const int64_t pos = base_s + off + __popc(m & ((1u << lane) - 1u));
            if (pos < row_ptr[i + 1]) {   // counts and writes use the same predicate; never overrun
                col[pos] = j;
                wout[pos] = w;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) base_s += tot;
        __syncthreads();
    }
}

__global__ void prune_prep_kernel(const double* u, const double* v, int n, double p, double* U,
                                  double* V, float* Lr, float* Dr, float* Vf, float* Vd) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double uu = u[k] * kLog2e, vv = v[k] * kLog2e;
    U[k] = uu;
    V[k] = vv;
    const float lr = (float)(uu / p);
    Lr[k] = lr;
    Dr[k] = (float)(uu - p * (double)lr);
    const float vf = (float)vv;
    Vf[k] = vf;
    Vd[k] = (float)(vv - (double)vf);
}

// ---- certificate check on all of A --------------------------------------------------
struct CertView {
    const void* w;
    int i16;
    int n;
    int64_t ld;
    const double* alpha;
    const double* beta;
    const float* af;
    const float* bf;
    double tau;
};

__global__ void certify_kernel(CertView C, unsigned long long* count, int64_t max_add,
                               int32_t* add_i, int32_t* add_j, int32_t* add_w) {
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < C.n; j += blockDim.x) {
        const int w = C.i16 ? (int)((const int16_t*)C.w)[(int64_t)i * C.ld + j]
                            : ((const int32_t*)C.w)[(int64_t)i * C.ld + j];
        if (w <= 0) continue;
        const float g = lg2_approx((float)w) * (float)kLn2 - C.af[i] - C.bf[j];
        // FP32 error of g is below 1e-5 for |alpha|, |beta| < 1e3; re-check in FP64 near tau
        if (g < (float)C.tau - 1e-4f) continue;
        const double gd = log((double)w) - C.alpha[i] - C.beta[j];
        if (gd > C.tau) {
            const unsigned long long k = atomicAdd(count, 1ull);
            if ((int64_t)k < max_add) { add_i[k] = i; add_j[k] = j; add_w[k] = w; }
        }
    }
}

__global__ void to_f32_kernel(const double* x, float* y, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) y[k] = (float)x[k];
}

// ---- FP64 verification of row / column sums -----------------------------------------
__global__ void verify_rows_kernel(const void* w, int i16, int n, int64_t ld, double p,
                                   const double* u, const double* v, double* rows, double* err) {
    const int i = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int wv = i16 ? (int)((const int16_t*)w)[(int64_t)i * ld + j] : ((const int32_t*)w)[(int64_t)i * ld + j];
        if (wv > 0) s += exp(p * log((double)wv) - u[i] - v[j]);
    }
    s = warp_sum(s);
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sh[k];
        if (rows) rows[i] = t;
        err[i] = fabs(t - 1.0);
    }
}

__global__ void verify_cols_kernel(const void* w, int i16, int n, int64_t ld, double p,
                                   const double* u, const double* v, int rows_per_chunk,
                                   double* part) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int r0 = blockIdx.y * rows_per_chunk, r1 = min(n, r0 + rows_per_chunk);
    double s = 0.0;
    for (int i = r0; i < r1; ++i) {
        const int wv = i16 ? (int)((const int16_t*)w)[(int64_t)i * ld + j] : ((const int32_t*)w)[(int64_t)i * ld + j];
        if (wv > 0) s += exp(p * log((double)wv) - u[i] - v[j]);
    }
    part[(int64_t)blockIdx.y * n + j] = s;
}

__global__ void verify_cols_combine(int n, int nchunks, const double* part, double* cols, double* err) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += part[(int64_t)c * n + j];
    if (cols) cols[j] = s;
    err[j] = fabs(s - 1.0);
}

// smallest positive and largest weight of the matrix (zeros are absent entries)
__global__ void minmax_kernel(const void* w, int i16, int n, int64_t ld, unsigned long long* out) {
    unsigned mn = 0xffffffffu, mx = 0u;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)n * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        const int x = i16 ? (int)((const int16_t*)w)[(int64_t)i * ld + j] : ((const int32_t*)w)[(int64_t)i * ld + j];
        if (x > 0) {
            mn = min(mn, (unsigned)x);
            mx = max(mx, (unsigned)x);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out, (unsigned long long)mn);
        atomicMax(out + 1, (unsigned long long)mx);
    }
}

__global__ void max_reduce_kernel(const double* x, int n, double* out) {
    double m = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) m = fmax(m, x[k]);
    m = warp_max(m);
    __shared__ double sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t = fmax(t, sh[k]);
        *out = t;
    }
}

__global__ void narrow_kernel(const int32_t* src, int64_t lds, int16_t* dst, int64_t ldd, int n,
                              unsigned long long* bad) {
    const int i = blockIdx.y;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        int v = src[(int64_t)i * lds + j];
        if (v < 0 || v > 32767) {
            atomicAdd(bad, 1ull);
            v = v < 0 ? 0 : 32767;
        }
        dst[(int64_t)i * ldd + j] = (int16_t)v;
    }
}

}  // namespace

sa_status prune_device(sa_ctx* ctx, const sa_matrix* a, double p, const double* d_u,
                       const double* d_v, double t, int guard, sa_csr* out, double* log_ub) {
    const int n = a->n;
    cudaStream_t st = ctx->stream;
    if (!(t > 0)) t = 1.0 / n;
    const int rows_per_chunk = 512;
    const int nchunks = (n + rows_per_chunk - 1) / rows_per_chunk;
    size_t need = 2 * align_up((size_t)n * 8, 256) + 4 * align_up((size_t)n * 4, 256) +
                  4 * align_up((size_t)n * 4, 256) + align_up((size_t)n * 8, 256) +
                  align_up((size_t)(n + 1) * 8, 256) + 2 * align_up((size_t)nchunks * n * 4, 256) + 4096;
    sa_status rc = ctx->ws.reserve(need);
    if (rc) return rc;
    Carve cv(ctx->ws.ptr);
    double* U = cv.take<double>(n);
    double* V = cv.take<double>(n);
    float* Lr = cv.take<float>(n);
    float* Dr = cv.take<float>(n);
    float* Vf = cv.take<float>(n);
    float* Vd = cv.take<float>(n);
    int* cnt = cv.take<int>(n);
    int* rarg = cv.take<int>(n);
    int* carg = cv.take<int>(n);
    double* rterm = cv.take<double>(n);
    int64_t* row_ptr = cv.take<int64_t>(n + 1);
    float* pv = cv.take<float>((size_t)nchunks * n);
    int* pi = cv.take<int>((size_t)nchunks * n);
    prune_prep_kernel<<<(n + 255) / 256, 256, 0, st>>>(d_u, d_v, n, p, U, V, Lr, Dr, Vf, Vd);
    count_launch();
    PruneView P;
    P.w = a->w;
    P.i16 = a->wtype == SA_I16;
    P.n = n;
    P.ld = a->ld;
    P.p = p;
    P.pf = (float)p;
    P.U = U;
    P.V = V;
    P.Lr = Lr;
    P.Dr = Dr;
    P.Vf = Vf;
    P.Vd = Vd;
    P.log2t = std::log2(t);
    P.log2tf = (float)P.log2t;
    P.margin = (float)(1e-4 + 4e-6 * p);
    prune_rows_kernel<<<n, kPruneThreads, 0, st>>>(P, cnt, rarg, rterm);
    count_launch();
    if (guard) {
        dim3 g((n + 127) / 128, nchunks);
        col_argmax_partial_kernel<<<g, 128, 0, st>>>(P, rows_per_chunk, pv, pi);
        count_launch();
        col_argmax_combine_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, nchunks, pv, pi, carg);
        count_launch();
        guard_count_kernel<<<(2 * n + 255) / 256, 256, 0, st>>>(P, rarg, carg, cnt);
        count_launch();
    }
    scan_kernel<<<1, 1024, 0, st>>>(cnt, row_ptr, n);
    count_launch();
    int64_t nnz = 0;
    SA_CUDA(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaStreamSynchronize(st));
    // output arrays on the device, then to the host CSR
    int32_t* d_col = nullptr;
    int32_t* d_w = nullptr;
    SA_CUDA(cudaMallocAsync((void**)&d_col, std::max<int64_t>(nnz, 1) * 4, st));
    SA_CUDA(cudaMallocAsync((void**)&d_w, std::max<int64_t>(nnz, 1) * 4, st));
    prune_write_kernel<<<n, kPruneThreads, 0, st>>>(P, guard, rarg, carg, row_ptr, d_col, d_w);
    count_launch();
    rc = csr_alloc(out, n, nnz);
    if (rc) { cudaFreeAsync(d_col, st); cudaFreeAsync(d_w, st); return rc; }
    std::vector<double> h_rterm(n), h_v(n);
    SA_CUDA(cudaMemcpyAsync(out->row_ptr, row_ptr, (n + 1) * 8, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(out->col, d_col, nnz * 4, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(out->w, d_w, nnz * 4, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(h_rterm.data(), rterm, n * 8, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(h_v.data(), d_v, n * 8, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaFreeAsync(d_col, st));
    SA_CUDA(cudaFreeAsync(d_w, st));
    SA_CUDA(cudaStreamSynchronize(st));
    SA_CUDA(cudaGetLastError());
    if (log_ub) {
        double acc = 0.0;
        for (int i = 0; i < n; ++i) acc += h_rterm[i];
        for (int j = 0; j < n; ++j) acc += h_v[j];
        *log_ub = acc / p;
    }
    return SA_OK;
}

sa_status certify_device(sa_ctx* ctx, const sa_matrix* a, const double* alpha, const double* beta,
                         double tau, int64_t* n_viol, int64_t max_add, sa_csr* add) {
    const int n = a->n;
    cudaStream_t st = ctx->stream;
    if (max_add < 0) max_add = 0;
    size_t need = 2 * align_up((size_t)n * 8, 256) + 2 * align_up((size_t)n * 4, 256) +
                  3 * align_up((size_t)std::max<int64_t>(max_add, 1) * 4, 256) + 4096;
    sa_status rc = ctx->ws.reserve(need);
    if (rc) return rc;
    Carve cv(ctx->ws.ptr);
    double* al = cv.take<double>(n);
    double* be = cv.take<double>(n);
    float* af = cv.take<float>(n);
    float* bf = cv.take<float>(n);
    unsigned long long* count = cv.take<unsigned long long>(1);
    int32_t* ai = cv.take<int32_t>(std::max<int64_t>(max_add, 1));
    int32_t* aj = cv.take<int32_t>(std::max<int64_t>(max_add, 1));
    int32_t* aw = cv.take<int32_t>(std::max<int64_t>(max_add, 1));
    SA_CUDA(cudaMemcpyAsync(al, alpha, n * 8, cudaMemcpyHostToDevice, st));
    SA_CUDA(cudaMemcpyAsync(be, beta, n * 8, cudaMemcpyHostToDevice, st));
    SA_CUDA(cudaMemsetAsync(count, 0, 8, st));
    to_f32_kernel<<<(n + 255) / 256, 256, 0, st>>>(al, af, n);
    count_launch();
    to_f32_kernel<<<(n + 255) / 256, 256, 0, st>>>(be, bf, n);
    count_launch();
    CertView C{a->w, a->wtype == SA_I16, n, a->ld, al, be, af, bf, tau};
    certify_kernel<<<n, 256, 0, st>>>(C, count, max_add, ai, aj, aw);
    count_launch();
    unsigned long long h_count = 0;
    SA_CUDA(cudaMemcpyAsync(&h_count, count, 8, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaStreamSynchronize(st));
    SA_CUDA(cudaGetLastError());
    *n_viol = (int64_t)h_count;
    if (add) {
        const int64_t k = std::min<int64_t>((int64_t)h_count, max_add);
        std::vector<int32_t> hi(k), hj(k), hw(k);
        if (k > 0) {
            SA_CUDA(cudaMemcpyAsync(hi.data(), ai, k * 4, cudaMemcpyDeviceToHost, st));
            SA_CUDA(cudaMemcpyAsync(hj.data(), aj, k * 4, cudaMemcpyDeviceToHost, st));
            SA_CUDA(cudaMemcpyAsync(hw.data(), aw, k * 4, cudaMemcpyDeviceToHost, st));
            SA_CUDA(cudaStreamSynchronize(st));
        }
        std::vector<int64_t> order(k);
        for (int64_t x = 0; x < k; ++x) order[x] = x;
        std::sort(order.begin(), order.end(), [&](int64_t p1, int64_t p2) {
            return hi[p1] != hi[p2] ? hi[p1] < hi[p2] : hj[p1] < hj[p2];
        });
        rc = csr_alloc(add, n, k);
        if (rc) return rc;
        std::vector<int64_t> cnt(n + 1, 0);
        for (int64_t x = 0; x < k; ++x) cnt[hi[x] + 1]++;
        for (int r = 0; r < n; ++r) cnt[r + 1] += cnt[r];
        for (int r = 0; r <= n; ++r) add->row_ptr[r] = cnt[r];
        for (int64_t x = 0; x < k; ++x) {
            add->col[x] = hj[order[x]];
            add->w[x] = hw[order[x]];
        }
    }
    return SA_OK;
}

sa_status verify_device(sa_ctx* ctx, const sa_matrix* a, double p, const double* d_u,
                        const double* d_v, double* d_rows, double* d_cols, double* max_row_err,
                        double* max_col_err) {
    const int n = a->n;
    cudaStream_t st = ctx->stream;
    const int rows_per_chunk = 256;
    const int nchunks = (n + rows_per_chunk - 1) / rows_per_chunk;
    size_t need = 2 * align_up((size_t)n * 8, 256) + align_up((size_t)nchunks * n * 8, 256) + 4096;
    sa_status rc = ctx->ws.reserve(need);
    if (rc) return rc;
    Carve cv(ctx->ws.ptr);
    double* rerr = cv.take<double>(n);
    double* cerr = cv.take<double>(n);
    double* part = cv.take<double>((size_t)nchunks * n);
    double* mx = cv.take<double>(2);
    const int i16 = a->wtype == SA_I16;
    verify_rows_kernel<<<n, 256, 0, st>>>(a->w, i16, n, a->ld, p, d_u, d_v, d_rows, rerr);
    count_launch();
    dim3 g((n + 127) / 128, nchunks);
    verify_cols_kernel<<<g, 128, 0, st>>>(a->w, i16, n, a->ld, p, d_u, d_v, rows_per_chunk, part);
    count_launch();
    verify_cols_combine<<<(n + 255) / 256, 256, 0, st>>>(n, nchunks, part, d_cols, cerr);
    count_launch();
    max_reduce_kernel<<<1, 1024, 0, st>>>(rerr, n, mx);
    count_launch();
    max_reduce_kernel<<<1, 1024, 0, st>>>(cerr, n, mx + 1);
    count_launch();
    double h[2];
    SA_CUDA(cudaMemcpyAsync(h, mx, 16, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaStreamSynchronize(st));
    SA_CUDA(cudaGetLastError());
    if (max_row_err) *max_row_err = h[0];
    if (max_col_err) *max_col_err = h[1];
    return SA_OK;
}

sa_status weights_minmax(sa_ctx* ctx, const sa_matrix* a, int64_t* wmin, int64_t* wmax) {
    cudaStream_t st = ctx->stream;
    sa_status rc = ctx->ws.reserve(256);
    if (rc) return rc;
    unsigned long long* d = (unsigned long long*)ctx->ws.ptr;
    const unsigned long long init[2] = {~0ull, 0ull};
    SA_CUDA(cudaMemcpyAsync(d, init, sizeof(init), cudaMemcpyHostToDevice, st));
    const int64_t total = (int64_t)a->n * a->n;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)ctx->num_sms * 8);
    minmax_kernel<<<blocks, 256, 0, st>>>(a->w, a->wtype == SA_I16, a->n, a->ld, d);
    count_launch();
    unsigned long long h[2];
    SA_CUDA(cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaStreamSynchronize(st));
    if (h[1] == 0ull) { set_error("matrix has no positive entry"); return SA_E_NO_PERFECT_MATCHING; }
    *wmin = (int64_t)h[0];
    *wmax = (int64_t)h[1];
    return SA_OK;
}

sa_status narrow_device(sa_ctx* ctx, const int32_t* src, int64_t lds, int16_t* dst, int64_t ldd,
                        int n, int64_t* n_bad) {
    cudaStream_t st = ctx->stream;
    sa_status rc = ctx->ws.reserve(256);
    if (rc) return rc;
    unsigned long long* bad = (unsigned long long*)ctx->ws.ptr;
    SA_CUDA(cudaMemsetAsync(bad, 0, 8, st));
    dim3 g((n + 255) / 256 < 8 ? (n + 255) / 256 : 8, n);
    narrow_kernel<<<g, 256, 0, st>>>(src, lds, dst, ldd, n, bad);
    count_launch();
    unsigned long long h = 0;
    SA_CUDA(cudaMemcpyAsync(&h, bad, 8, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaStreamSynchronize(st));
    SA_CUDA(cudaGetLastError());
    if (n_bad) *n_bad = (int64_t)h;
    return SA_OK;
}

}  // namespace sa
