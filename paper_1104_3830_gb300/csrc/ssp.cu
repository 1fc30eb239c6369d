// ssp.cu -- the shortest-augmenting-path phase of the exact solve of B (Sec. 4.2: the
// sequential solve of the reduced instance) with each search on the GPU.
//
// The host solver (solve.cpp) assigns most rows by a greedy pass and augmenting row
// reduction, keeping every assigned row on a least-reduced-cost column for the column
// prices v (minimisation form, cost c = -log w).  Each remaining free row r then needs a
// shortest alternating path to a free column in reduced costs
//     rc(i, k) = c_ik - u_i - v_k >= 0,   u_i = c_{i, rmatch(i)} - v_{rmatch(i)},
// after which the prices move by (dist - D) on the columns closer than the path length D,
// and the path is flipped: the dual update of successive shortest paths, which keeps the
// prices dual feasible and the assignment tight.  Here the distances are found by a
// label-correcting (Bellman-Ford) search over a frontier of columns, one warp per column,
// instead of the host's Dijkstra: distances are FP64, shifted by u_r so that they are all
// >= 0, and a 64-bit atomic minimum on their bits (which order like non-negative doubles)
// resolves concurrent relaxations; relaxations no shorter than the best free column found
// so far are dropped.  A breadth-first pass over tight entries (relaxations that reproduce
// the converged distances exactly) then gives every column on a shortest path a
// predecessor, and the price update and the flip run on the device.  The host queues the
// rounds in batches of eight and reads only the frontier size after each batch and the sink
// after each search; no kernel waits on another.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "sa_internal.h"

namespace sa {

namespace {

constexpr int kSpT = 256;
constexpr int kBatch = 8;   // rounds queued between reads of the next frontier's size
typedef unsigned long long u64;

__device__ __forceinline__ u64 dbits(double x) { return (u64)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(u64 b) { return __longlong_as_double((long long)b); }

struct SpArgs {
    int n;
    const int64_t* rp;
    const int32_t* col;
    const double* cost;      // -log w per entry
    double* v;               // column prices
    int32_t* rmatch;
    int32_t* cmatch;
    double* mcost;           // cost of each row's assigned entry
    u64* dist;               // bits of the distance (>= 0) of each column; +inf unreached
    int32_t* pred;           // row through which each column is reached
    double* pcost;           // cost of the entry (pred, column)
    int32_t* mark;           // frontier round that last queued each column
    int32_t* level;          // hops from the free row in the predecessor tree (-1: none yet)
    int32_t* front[3];       // frontier columns of rounds t, t+1, t+2 (t mod 3)
    int32_t* nfront;         // [3] sizes
    u64* best;               // bits of the shortest distance to a free column so far
    int32_t* sink;
    double* ur;              // potential of the free row (the shift of the distances)
};

// reduced cost of entry e of row i, clamped at +0 (the invariant holds up to rounding;
// a weight of 1 has cost -0.0, and a -0.0 here would order above every distance)
__device__ __forceinline__ double sp_rc(const SpArgs& A, int64_t e, double ui) {
    const double x = A.cost[e] - ui - A.v[A.col[e]];
    return x > 0.0 ? x : 0.0;
}

__global__ void sp_reset_kernel(SpArgs A) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < A.n) {
        A.dist[j] = dbits(INFINITY);
        A.mark[j] = -1;
        A.level[j] = -1;
    }
    if (j == 0) {
        A.nfront[0] = A.nfront[1] = A.nfront[2] = 0;
        *A.best = dbits(INFINITY);
        *A.sink = A.n;
    }
}

// one block: the free row r's potential and its entries as the first frontier
__global__ void sp_seed_kernel(SpArgs A, int r) {
    __shared__ double sh[kSpT / 32];
    const int64_t e0 = A.rp[r], e1 = A.rp[r + 1];
    double m = INFINITY;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kSpT) m = fmin(m, A.cost[e] - A.v[A.col[e]]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    double ur = sh[0];
    for (int k = 1; k < kSpT / 32; ++k) ur = fmin(ur, sh[k]);
    if (threadIdx.x == 0) *A.ur = ur;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += kSpT) {
        const int k = A.col[e];
        const double d = sp_rc(A, e, ur);
        A.dist[k] = dbits(d);          // the columns of one row are distinct
        if (A.cmatch[k] < 0) {
            atomicMin(A.best, dbits(d));
        } else {
            A.mark[k] = 0;
            A.front[0][atomicAdd(&A.nfront[0], 1)] = k;
        }
    }
}

// one warp per frontier column j of round `round`: relax the entries of its assigned row.
// Frontiers and their sizes rotate over three buffers: the round reads buffer round % 3,
// fills (round + 1) % 3 and clears (round + 2) % 3 (read last by the previous round).
__global__ void sp_relax_kernel(SpArgs A, int round) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int cur = round % 3, nxt = (round + 1) % 3;
    if (blockIdx.x == 0 && threadIdx.x == 0) A.nfront[(round + 2) % 3] = 0;
    if (w >= A.nfront[cur]) return;
    const int j = A.front[cur][w];
    const double dj = bitsd(A.dist[j]);
    const double bst = bitsd(*(volatile u64*)A.best);
    if (!(dj < bst)) return;
    const int i = A.cmatch[j];
    const double ui = A.mcost[i] - A.v[j];
    for (int64_t e = A.rp[i] + lane; e < A.rp[i + 1]; e += 32) {
        const int k = A.col[e];
        if (k == j) continue;             // the assigned entry: length 0 back to j
        const double nd = dj + sp_rc(A, e, ui);
        if (nd < bitsd(*(volatile u64*)A.best) && dbits(nd) < A.dist[k]) {
            const u64 old = atomicMin(A.dist + k, dbits(nd));
            if (old > dbits(nd)) {
                if (A.cmatch[k] < 0) atomicMin(A.best, dbits(nd));
                else if (atomicExch(A.mark + k, round + 1) != round + 1)
                    A.front[nxt][atomicAdd(&A.nfront[nxt], 1)] = k;
            }
        }
    }
}

// Predecessors by a breadth-first pass over tight entries (those whose relaxation
// reproduces the converged distance exactly) from the free row through the columns at
// distance <= D: every column on a shortest path to a free column at D is reached, each
// is claimed once, and the
// levels grow along predecessors, so the path to the sink has no cycle (entries of reduced
// cost 0 make equal distances, so a column-by-column choice could close one).
__device__ __forceinline__ void sp_claim(const SpArgs& A, int k, int i, int64_t e, int lvl, double D, int nxt) {
    if (atomicCAS(A.level + k, -1, lvl) != -1) return;
    A.pred[k] = i;
    A.pcost[k] = A.cost[e];
    const double dk = bitsd(A.dist[k]);
    if (A.cmatch[k] < 0) {
        if (dk == D) atomicMin(A.sink, k);
    } else if (dk <= D) {   // columns at D too: with reduced costs 0 the sink can lie behind them
        A.front[nxt][atomicAdd(&A.nfront[nxt], 1)] = k;
    }
}

// level 0: the free row's tight entries (one block); frontier buffers restart at 0
__global__ void sp_tree_seed_kernel(SpArgs A, int r) {
    const double D = bitsd(*A.best);
    const double ur = *A.ur;
    for (int64_t e = A.rp[r] + threadIdx.x; e < A.rp[r + 1]; e += kSpT) {
        const int k = A.col[e];
        if (dbits(sp_rc(A, e, ur)) == A.dist[k]) sp_claim(A, k, r, e, 0, D, 0);
    }
}

__global__ void sp_tree_reset_kernel(SpArgs A) {
    if (threadIdx.x == 0) A.nfront[0] = A.nfront[1] = A.nfront[2] = 0;
}

// level L + 1 from the columns of level L (buffer L % 3), one warp per column
__global__ void sp_tree_kernel(SpArgs A, int L) {
    const int lane = threadIdx.x & 31;
    const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int cur = L % 3, nxt = (L + 1) % 3;
    if (blockIdx.x == 0 && threadIdx.x == 0) A.nfront[(L + 2) % 3] = 0;
    if (w >= A.nfront[cur]) return;
    const double D = bitsd(*A.best);
    const int j = A.front[cur][w];
    const double dj = bitsd(A.dist[j]);
    const int i = A.cmatch[j];
    const double ui = A.mcost[i] - A.v[j];
    for (int64_t e = A.rp[i] + lane; e < A.rp[i + 1]; e += 32) {
        const int k = A.col[e];
        if (k == j) continue;
        if (dbits(dj + sp_rc(A, e, ui)) == A.dist[k]) sp_claim(A, k, i, e, L + 1, D, nxt);
    }
}

// prices of the columns closer than the path length, then the flip of the path
__global__ void sp_update_kernel(SpArgs A) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const double D = bitsd(*A.best);
    if (j < A.n) {
        const double dj = bitsd(A.dist[j]);
        if (dj < D) A.v[j] += dj - D;
    }
}

__global__ void sp_flip_kernel(SpArgs A, int r) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int j = *A.sink;
    if (j >= A.n) return;                 // no augmenting path: reported by the host
    for (int step = 0; step <= A.n; ++step) {   // a path has at most n columns
        const int i = A.pred[j];
        A.cmatch[j] = i;
        const int prev = A.rmatch[i];
        A.rmatch[i] = j;
        A.mcost[i] = A.pcost[j];
        if (i == r) return;
        j = prev;
    }
}

}  // namespace

sa_status ssp_device(void* user, SspState& st) {
    SspRun* run = (SspRun*)user;
    sa_ctx* ctx = run->ctx;
    const int n = st.n;
    std::vector<int> freel;
    for (int i = 0; i < n; ++i)
        if (st.rmatch[i] < 0) freel.push_back(i);
    if (freel.empty()) return SA_OK;
    cudaStream_t s = ctx->stream;
    const int64_t nnz = st.row_ptr[n];
    SpArgs A{};
    A.n = n;
    // device copies of the instance and the solver state
    char* base = nullptr;
    const size_t bytes = align_up(sizeof(int64_t) * (n + 1), 256) + align_up(sizeof(int32_t) * std::max<int64_t>(nnz, 1), 256) +
                         align_up(sizeof(double) * std::max<int64_t>(nnz, 1), 256) + 3 * align_up(sizeof(double) * n, 256) +
                         9 * align_up(sizeof(int32_t) * std::max(n, 4), 256) + align_up(sizeof(u64) * n, 256) + 1024;
    SA_CUDA(cudaMallocAsync((void**)&base, bytes, s));
    Carve cv(base);
    int64_t* rp = cv.take<int64_t>(n + 1);
    int32_t* col = cv.take<int32_t>(std::max<int64_t>(nnz, 1));
    double* cost = cv.take<double>(std::max<int64_t>(nnz, 1));
    A.v = cv.take<double>(n);
    A.mcost = cv.take<double>(n);
    A.pcost = cv.take<double>(n);
    A.rmatch = cv.take<int32_t>(n);
    A.cmatch = cv.take<int32_t>(n);
    A.pred = cv.take<int32_t>(n);
    A.mark = cv.take<int32_t>(n);
    A.level = cv.take<int32_t>(n);
    A.front[0] = cv.take<int32_t>(n);
    A.front[1] = cv.take<int32_t>(n);
    A.front[2] = cv.take<int32_t>(n);
    int32_t* misc = cv.take<int32_t>(std::max(n, 4));   // nfront[3], sink
    A.dist = cv.take<u64>(n);
    u64* misc64 = cv.take<u64>(4);         // best, ur
    A.nfront = misc;
    A.sink = misc + 3;
    A.best = misc64;
    A.ur = (double*)(misc64 + 1);
    A.rp = rp;
    A.col = col;
    A.cost = cost;
    std::vector<double> c(std::max<int64_t>(nnz, 1));
    for (int64_t e = 0; e < nnz; ++e) c[e] = -st.logw[e];
    SA_CUDA(cudaMemcpyAsync(rp, st.row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s));
    if (nnz > 0) {
        SA_CUDA(cudaMemcpyAsync(col, st.col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, s));
        SA_CUDA(cudaMemcpyAsync(cost, c.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    }
    SA_CUDA(cudaMemcpyAsync(A.v, st.v, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    SA_CUDA(cudaMemcpyAsync(A.mcost, st.mcost, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    SA_CUDA(cudaMemcpyAsync(A.rmatch, st.rmatch, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    SA_CUDA(cudaMemcpyAsync(A.cmatch, st.cmatch, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s));
    sa_status rc = ctx->pinned.reserve(64);
    if (rc) { cudaFreeAsync(base, s); return rc; }
    int32_t* h = (int32_t*)ctx->pinned.ptr;
    const int ge = (n + kSpT - 1) / kSpT;
    const int wpb = kSpT / 32;
    for (int r : freel) {
        ++run->searches;
        sp_reset_kernel<<<ge, kSpT, 0, s>>>(A);
        sp_seed_kernel<<<1, kSpT, 0, s>>>(A, r);
        count_launch(2);
        // rounds run in batches; each batch ends with a read of the next frontier's size
        const int gfull = (n + wpb - 1) / wpb;   // enough warps for any frontier
        for (int round = 0; round <= n; round += kBatch) {
            for (int b = 0; b < kBatch; ++b) sp_relax_kernel<<<gfull, kSpT, 0, s>>>(A, round + b);
            count_launch(kBatch);
            run->rounds += kBatch;
            SA_CUDA(cudaMemcpyAsync(h, A.nfront + (round + kBatch) % 3, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            SA_CUDA(cudaStreamSynchronize(s));
            if (*h == 0) break;   // an empty frontier stays empty
        }
        sp_tree_reset_kernel<<<1, 32, 0, s>>>(A);
        sp_tree_seed_kernel<<<1, kSpT, 0, s>>>(A, r);
        count_launch(2);
        for (int L = 0; L <= n; L += kBatch) {
            for (int b = 0; b < kBatch; ++b) sp_tree_kernel<<<gfull, kSpT, 0, s>>>(A, L + b);
            count_launch(kBatch);
            run->rounds += kBatch;
            SA_CUDA(cudaMemcpyAsync(h, A.nfront + (L + kBatch) % 3, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            SA_CUDA(cudaStreamSynchronize(s));
            if (*h == 0) break;
        }
        sp_update_kernel<<<ge, kSpT, 0, s>>>(A);
        sp_flip_kernel<<<1, 32, 0, s>>>(A, r);
        count_launch(2);
        SA_CUDA(cudaMemcpyAsync(h + 1, A.sink, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SA_CUDA(cudaStreamSynchronize(s));
        if (h[1] >= n) {
            cudaFreeAsync(base, s);
            set_error("reduced instance has no perfect matching (row %d cannot be assigned)", r);
            return SA_E_NO_PERFECT_MATCHING;
        }
    }
    SA_CUDA(cudaMemcpyAsync(st.v, A.v, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    SA_CUDA(cudaMemcpyAsync(st.mcost, A.mcost, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    SA_CUDA(cudaMemcpyAsync(st.rmatch, A.rmatch, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    SA_CUDA(cudaMemcpyAsync(st.cmatch, A.cmatch, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(base, s);
    SA_CUDA(cudaStreamSynchronize(s));
    return SA_OK;
}

}  // namespace sa
