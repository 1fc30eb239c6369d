// auction.cu -- the reduced instance B of Eq. matrixred on the GPU: a forward auction
// (Bertsekas) with eps-scaling, Jacobi-parallel (every unassigned row bids in the same
// round), which brings the column prices within eps of an LP-optimal dual.  The exact
// sparse solver then starts from those prices (sa_solve_reduced_gpu), so the result is the
// exact optimum with its LP duals, as with sa_solve_reduced; the auction only shortens the
// sequential solve of B (Sec. 4.2).
//
// A round is three launches: bids (one warp per unassigned row: best and second-best value
// of log w_ij - price_j over the row; the bid raises the best column's price by their
// difference plus eps, recorded with a 64-bit atomic maximum on the bid's bits, which order
// like the bids since bids are >= 0), winners (equal highest bids resolved by a
// compare-and-swap), updates (per column: the winner takes it, the previous owner is freed,
// the price becomes the winning bid).  The host queues rounds in batches and reads the
// number of free rows between batches; no kernel waits on another.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <limits>
#include <vector>

#include "sa_internal.h"

namespace sa {

namespace {

constexpr int kAuThreads = 256;
constexpr int kAuBatch = 16;          // rounds queued between reads of the free-row count
constexpr double kAuShrink = 8.0;     // eps of the next scaling phase = eps / kAuShrink

// Top-two merge of (v1, j1, v2) triples: ties of the best value keep the smaller column.
__device__ __forceinline__ void au_merge(double& v1, int& j1, double& v2, double ov1, int oj1, double ov2) {
    if (ov1 > v1 || (ov1 == v1 && oj1 >= 0 && (j1 < 0 || oj1 < j1))) {
        v2 = fmax(v1, ov2);
        v1 = ov1;
        j1 = oj1;
    } else {
        v2 = fmax(v2, ov1);
    }
}

// One warp per row: unassigned rows bid for their best column.
__global__ void au_bid_kernel(int n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                              const double* __restrict__ val, const double* __restrict__ price,
                              const int* __restrict__ assigned, double eps, double big,
                              unsigned long long* __restrict__ colbid, double* __restrict__ mybid,
                              int* __restrict__ mycol) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    if (assigned[i] >= 0) {
        if (lane == 0) mycol[i] = -1;
        return;
    }
    double v1 = -INFINITY, v2 = -INFINITY;
    int j1 = -1;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32) {
        const int j = col[e];
        const double x = val[e] - price[j];
        au_merge(v1, j1, v2, x, j, -INFINITY);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov1 = __shfl_xor_sync(0xffffffffu, v1, o);
        const int oj1 = __shfl_xor_sync(0xffffffffu, j1, o);
        const double ov2 = __shfl_xor_sync(0xffffffffu, v2, o);
        au_merge(v1, j1, v2, ov1, oj1, ov2);
    }
    if (lane != 0) return;
    if (j1 < 0 || !(v1 > -INFINITY)) {   // a row without entries: no bid (B has no permutation)
        mycol[i] = -1;
        return;
    }
    if (!(v2 > -INFINITY)) v2 = v1 - big;   // a single column: raise its price by the value range
    const double bid = price[j1] + (v1 - v2) + eps;
    mybid[i] = bid;
    mycol[i] = j1;
    atomicMax(colbid + j1, (unsigned long long)__double_as_longlong(bid));
}

// Bidders whose bid is their column's highest; among equal bids the first CAS wins.
__global__ void au_win_kernel(int n, const double* __restrict__ mybid, const int* __restrict__ mycol,
                              const unsigned long long* __restrict__ colbid, int* __restrict__ colwin) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int j = mycol[i];
    if (j >= 0 && (unsigned long long)__double_as_longlong(mybid[i]) == colbid[j]) atomicCAS(colwin + j, -1, i);
}

// Per column: the winner takes it at its bid; the previous owner becomes free.
__global__ void au_upd_kernel(int n, int* __restrict__ owner, int* __restrict__ assigned, double* __restrict__ price,
                              unsigned long long* __restrict__ colbid, int* __restrict__ colwin, int* __restrict__ nfree) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int w = colwin[j];
    if (w >= 0) {
        const int prev = owner[j];
        if (prev >= 0) assigned[prev] = -1;
        else atomicSub(nfree, 1);
        owner[j] = w;
        assigned[w] = j;
        price[j] = __longlong_as_double((long long)colbid[j]);
        colwin[j] = -1;
    }
    colbid[j] = 0ull;
}

// Start of a scaling phase: every row free, prices kept.
__global__ void au_reset_kernel(int n, int* owner, int* assigned, int* colwin, unsigned long long* colbid, int* nfree) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        owner[j] = -1;
        assigned[j] = -1;
        colwin[j] = -1;
        colbid[j] = 0ull;
    }
    if (j == 0) *nfree = n;
}

}  // namespace

// eps-scaling auction on the device CSR; price (device FP64[n]) holds the starting prices
// (>= 0) and receives the final ones; assigned (device int32[n]) the final assignment
// (complete if *complete).  Rounds are capped at max_rounds in all.
sa_status auction_device(sa_ctx* ctx, int n, const int64_t* d_rp, const int32_t* d_col, const double* d_val,
                         double eps0, double eps_final, int64_t max_rounds, double* d_price, int* d_assigned,
                         int* phases, int64_t* rounds, int* complete) {
    cudaStream_t st = ctx->stream;
    int *owner = nullptr, *colwin = nullptr, *mycol = nullptr, *nfree = nullptr;
    unsigned long long* colbid = nullptr;
    double* mybid = nullptr;
    SA_CUDA(cudaMallocAsync((void**)&owner, sizeof(int) * n, st));
    SA_CUDA(cudaMallocAsync((void**)&colwin, sizeof(int) * n, st));
    SA_CUDA(cudaMallocAsync((void**)&mycol, sizeof(int) * n, st));
    SA_CUDA(cudaMallocAsync((void**)&nfree, sizeof(int), st));
    SA_CUDA(cudaMallocAsync((void**)&colbid, sizeof(unsigned long long) * n, st));
    SA_CUDA(cudaMallocAsync((void**)&mybid, sizeof(double) * n, st));
    sa_status rc = ctx->pinned.reserve(64);
    if (rc) return rc;
    int* h_free = (int*)ctx->pinned.ptr;
    const int gb = (n + 7) / 8, ge = (n + kAuThreads - 1) / kAuThreads;
    // a row with a single column has no second-best value: its bid raises that column's
    // price by this increment (any increment >= eps keeps eps-complementary slackness)
    const double big = std::max(1.0, 8.0 * eps0);
    *phases = 0;
    *rounds = 0;
    *complete = 0;
    for (double eps = eps0;; eps = std::max(eps / kAuShrink, eps_final)) {
        au_reset_kernel<<<ge, kAuThreads, 0, st>>>(n, owner, d_assigned, colwin, colbid, nfree);
        count_launch();
        ++*phases;
        int done = 0;
        while (!done && *rounds < max_rounds) {
            for (int r = 0; r < kAuBatch; ++r) {
                au_bid_kernel<<<gb, kAuThreads, 0, st>>>(n, d_rp, d_col, d_val, d_price, d_assigned, eps, big, colbid,
                                                         mybid, mycol);
                au_win_kernel<<<ge, kAuThreads, 0, st>>>(n, mybid, mycol, colbid, colwin);
                au_upd_kernel<<<ge, kAuThreads, 0, st>>>(n, owner, d_assigned, d_price, colbid, colwin, nfree);
            }
            count_launch(3 * kAuBatch);
            *rounds += kAuBatch;
            SA_CUDA(cudaMemcpyAsync(h_free, nfree, sizeof(int), cudaMemcpyDeviceToHost, st));
            SA_CUDA(cudaStreamSynchronize(st));
            done = *h_free == 0;
        }
        if (!done) break;                    // round cap: incomplete
        if (eps <= eps_final) {
            *complete = 1;
            break;
        }
    }
    cudaFreeAsync(owner, st);
    cudaFreeAsync(colwin, st);
    cudaFreeAsync(mycol, st);
    cudaFreeAsync(nfree, st);
    cudaFreeAsync(colbid, st);
    cudaFreeAsync(mybid, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "auction");
    return SA_OK;
}

}  // namespace sa
