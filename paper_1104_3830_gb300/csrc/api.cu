// api.cu -- the C ABI of libsa (include/sa.h): contexts, argument checks, the scaling
// driver, pruning, the exact solve of the reduced instance with its duality repair loop
// (Algorithm 1 of Sec. 4.2 with a fixed schedule), and host-input convenience entry.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "sa_internal.h"

namespace sa {

static thread_local std::string tl_err;
std::atomic<long long> g_kernel_launches{0};

void set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    tl_err = buf;
}

sa_status cuda_fail(cudaError_t e, const char* what) {
    set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
    if (e == cudaErrorMemoryAllocation) return SA_E_NOMEM;
    return SA_E_CUDA;
}

sa_status Workspace::reserve(size_t bytes) {
    if (bytes <= size) return SA_OK;
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    size = 0;
    size_t want = std::max(bytes, (size_t)1 << 20);
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        return cuda_fail(e, "cudaMalloc(workspace)");
    }
    size = want;
    return SA_OK;
}
void Workspace::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    size = 0;
}
Workspace::~Workspace() {
    if (ptr) cudaFree(ptr);
}

size_t assign_device_bound(int num_sms, int n) {
    const size_t nn = (size_t)n;
    const size_t ldk = align_up(nn, 4);
    const size_t npad = align_up(nn, 32);
    return 12 * nn * ldk                       // K and the log2 pairs of w (STEP; NEWTON: K)
           + 8 * nn * nn                       // prune: device column and weight arrays
           + 2 * (size_t)num_sms * npad * 4    // column partials, two blocks per SM
           + 512 * nn                          // per-row and per-column vectors of every stage
           + ((size_t)4 << 20);                // schedule, flags, certificate additions
}

void release_buffers(sa_ctx* ctx) {
    ctx->ws.release();
    ctx->input.release();
    ctx->keep.release();
}
sa_status PinnedBuf::reserve(size_t bytes) {
    if (bytes <= size) return SA_OK;
    if (ptr) cudaFreeHost(ptr);
    ptr = nullptr;
    size = 0;
    size_t want = std::max(bytes, (size_t)4096);
    cudaError_t e = cudaHostAlloc(&ptr, want, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        ptr = nullptr;
        return cuda_fail(e, "cudaHostAlloc");
    }
    size = want;
    return SA_OK;
}
PinnedBuf::~PinnedBuf() {
    if (ptr) cudaFreeHost(ptr);
}

sa_status csr_alloc(sa_csr* c, int n, int64_t nnz) {
    c->n = n;
    c->nnz = nnz;
    c->row_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    c->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
    c->w = (int32_t*)malloc(sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
    if (!c->row_ptr || !c->col || !c->w) {
        free(c->row_ptr);
        free(c->col);
        free(c->w);
        c->row_ptr = nullptr;
        c->col = nullptr;
        c->w = nullptr;
        set_error("host allocation of %lld CSR entries failed", (long long)nnz);
        return SA_E_NOMEM;
    }
    return SA_OK;
}

static sa_status check_matrix(const sa_matrix* a) {
    if (!a || !a->w) { set_error("null matrix"); return SA_E_INVALID; }
    if (a->n <= 0) { set_error("n must be positive (got %d)", a->n); return SA_E_INVALID; }
    if (a->ld < a->n) { set_error("ld (%lld) < n (%d)", (long long)a->ld, a->n); return SA_E_INVALID; }
    if (a->wtype != SA_I16 && a->wtype != SA_I32) { set_error("unknown weight type"); return SA_E_INVALID; }
    return SA_OK;
}

static sa_status check_opts(const sa_scale_opts* o) {
    if (!o || !o->p || o->n_p <= 0) { set_error("empty p schedule"); return SA_E_INVALID; }
    for (int k = 0; k < o->n_p; ++k) {
        if (!(o->p[k] > 0) || !std::isfinite(o->p[k])) { set_error("p[%d] must be finite and > 0", k); return SA_E_INVALID; }
        if (k > 0 && !(o->p[k] > o->p[k - 1])) { set_error("p schedule must increase strictly"); return SA_E_INVALID; }
    }
    if (!(o->tol > 0)) { set_error("tol must be > 0"); return SA_E_INVALID; }
    if (o->max_sweeps_per_p <= 0) { set_error("max_sweeps_per_p must be > 0"); return SA_E_INVALID; }
    if (o->resume_from < 0 || o->resume_from >= o->n_p) { set_error("resume_from out of range"); return SA_E_INVALID; }
    if (o->prec < SA_PREC_MIXED || o->prec > SA_PREC_FP64) { set_error("unknown precision"); return SA_E_INVALID; }
    if (o->kernel < SA_KERNEL_AUTO || o->kernel > SA_KERNEL_NEWTON) { set_error("unknown kernel"); return SA_E_INVALID; }
    return SA_OK;
}

struct DeviceGuard {
    explicit DeviceGuard(int dev) { cudaSetDevice(dev); }
};

static double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// union of two CSRs with ascending columns; entries of `b` already in `a` are dropped
static sa_status csr_union(const sa_csr& a, const sa_csr& b, sa_csr* out) {
    const int n = a.n;
    std::vector<int64_t> rp(n + 1, 0);
    std::vector<int32_t> cols, ws;
    cols.reserve(a.nnz + b.nnz);
    ws.reserve(a.nnz + b.nnz);
    for (int i = 0; i < n; ++i) {
        int64_t x = a.row_ptr[i], xe = a.row_ptr[i + 1];
        int64_t y = b.row_ptr[i], ye = b.row_ptr[i + 1];
        while (x < xe || y < ye) {
            if (y >= ye || (x < xe && a.col[x] < b.col[y])) { cols.push_back(a.col[x]); ws.push_back(a.w[x]); ++x; }
            else if (x >= xe || b.col[y] < a.col[x]) { cols.push_back(b.col[y]); ws.push_back(b.w[y]); ++y; }
            else { cols.push_back(a.col[x]); ws.push_back(a.w[x]); ++x; ++y; }
        }
        rp[i + 1] = (int64_t)cols.size();
    }
    sa_status rc = csr_alloc(out, n, (int64_t)cols.size());
    if (rc) return rc;
    memcpy(out->row_ptr, rp.data(), sizeof(int64_t) * (n + 1));
    if (!cols.empty()) {
        memcpy(out->col, cols.data(), sizeof(int32_t) * cols.size());
        memcpy(out->w, ws.data(), sizeof(int32_t) * ws.size());
    }
    return SA_OK;
}

static sa_status solve_csr(const sa_csr& b, int32_t* perm, double* sum_log_w, double* alpha,
                           double* beta, const double* price0 = nullptr, SspFn ssp = nullptr,
                           void* ssp_user = nullptr) {
    std::vector<double> lw((size_t)std::max<int64_t>(b.nnz, 1));
    for (int64_t e = 0; e < b.nnz; ++e)
        lw[e] = b.w[e] > 0 ? std::log((double)b.w[e]) : -std::numeric_limits<double>::infinity();
    sa_status rc = sparse_assign(b.n, b.row_ptr, b.col, lw.data(), perm, alpha, beta, price0, ssp, ssp_user);
    if (rc) return rc;
    if (sum_log_w) {
        double s = 0.0;
        for (int i = 0; i < b.n; ++i) {
            double best = -std::numeric_limits<double>::infinity();   // a repeated column: its best entry
            for (int64_t e = b.row_ptr[i]; e < b.row_ptr[i + 1]; ++e)
                if (b.col[e] == perm[i] && lw[e] > best) best = lw[e];
            s += best;
        }
        *sum_log_w = s;
    }
    return SA_OK;
}

// B solved from the column minima, then of its LP-optimal duals the largest beta <= beta0
// (maximisation form): the optimum of the cold start with duals as close to beta0 as the
// optimum allows.  alpha/beta may be NULL.
static sa_status solve_csr_near(const sa_csr& b, const double* beta0, int32_t* perm, double* sum_log_w,
                                double* alpha, double* beta) {
    std::vector<double> al(b.n), be(b.n);
    sa_status rc = solve_csr(b, perm, sum_log_w, al.data(), be.data());
    if (rc) return rc;
    std::vector<double> lw((size_t)std::max<int64_t>(b.nnz, 1));
    for (int64_t e = 0; e < b.nnz; ++e)
        lw[e] = b.w[e] > 0 ? std::log((double)b.w[e]) : -std::numeric_limits<double>::infinity();
    rc = project_duals(b.n, b.row_ptr, b.col, lw.data(), perm, beta0, al.data(), be.data());
    if (rc) return rc;
    if (alpha) std::copy(al.begin(), al.end(), alpha);
    if (beta) std::copy(be.begin(), be.end(), beta);
    return SA_OK;
}

constexpr int64_t kAuctionRounds = 1000;      // bidding rounds of one sa_solve_reduced_gpu
constexpr int64_t kAuctionMinNnz = 150000;    // sa_assign uses the auction from this size of B

// B solved exactly, the column prices first improved by the GPU auction.  price_max: host
// maximisation-form starting prices (may be null).
static sa_status solve_csr_gpu(sa_ctx* ctx, const sa_csr& b, const double* price_max, int32_t* perm,
                               double* sum_log_w, double* alpha, double* beta, sa_auction_info* info) {
    const int n = b.n;
    const int64_t nnz = b.nnz;
    sa_auction_info loc{};
    if (!info) info = &loc;
    *info = sa_auction_info{};
    std::vector<double> lw((size_t)std::max<int64_t>(nnz, 1));
    double vmin = INFINITY, vmax = -INFINITY;
    for (int64_t e = 0; e < nnz; ++e) {
        lw[e] = b.w[e] > 0 ? std::log((double)b.w[e]) : -std::numeric_limits<double>::infinity();
        if (std::isfinite(lw[e])) { vmin = std::min(vmin, lw[e]); vmax = std::max(vmax, lw[e]); }
    }
    std::vector<double> price(n, 0.0);
    if (price_max)
        for (int j = 0; j < n; ++j) price[j] = std::isfinite(price_max[j]) ? price_max[j] : 0.0;
    double pmin = *std::min_element(price.begin(), price.end());
    for (int j = 0; j < n; ++j) price[j] -= pmin;   // bids and prices stay >= 0
    const double range = std::isfinite(vmax - vmin) ? std::max(vmax - vmin, 1e-9) : 1.0;
    // a short auction: its prices are a starting point for the exact solver (whose searches
    // then run on the GPU), not the end;
    // measured on reduced instances of the serving distribution (n = 2048 / 4096, 91k / 362k
    // entries), 1000 rounds to eps = 1e-3 of the value range cut the exact solve of the
    // larger one from 1.33 s to 0.67 s and cost about as much as they saved on the smaller
    const double eps0 = price_max ? range / 256.0 : range / 4.0;
    const double eps_final = range * 1e-3;
    double t0 = now_ms();
    int64_t *d_rp = nullptr;
    int32_t* d_col = nullptr;
    double *d_val = nullptr, *d_price = nullptr;
    int* d_asg = nullptr;
    cudaStream_t st = ctx->stream;
    SA_CUDA(cudaMallocAsync((void**)&d_rp, sizeof(int64_t) * (n + 1), st));
    SA_CUDA(cudaMallocAsync((void**)&d_col, sizeof(int32_t) * std::max<int64_t>(nnz, 1), st));
    SA_CUDA(cudaMallocAsync((void**)&d_val, sizeof(double) * std::max<int64_t>(nnz, 1), st));
    SA_CUDA(cudaMallocAsync((void**)&d_price, sizeof(double) * n, st));
    SA_CUDA(cudaMallocAsync((void**)&d_asg, sizeof(int) * n, st));
    SA_CUDA(cudaMemcpyAsync(d_rp, b.row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
    if (nnz > 0) {
        SA_CUDA(cudaMemcpyAsync(d_col, b.col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
        SA_CUDA(cudaMemcpyAsync(d_val, lw.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice, st));
    }
    SA_CUDA(cudaMemcpyAsync(d_price, price.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
    int phases = 0, complete = 0;
    int64_t rounds = 0;
    sa_status rc = auction_device(ctx, n, d_rp, d_col, d_val, eps0, eps_final, kAuctionRounds, d_price, d_asg, &phases, &rounds,
                                  &complete);
    std::vector<int> asg(n, -1);
    if (rc == SA_OK) {
        cudaError_t e1 = cudaMemcpyAsync(price.data(), d_price, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
        cudaError_t e2 = cudaMemcpyAsync(asg.data(), d_asg, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
        cudaError_t e3 = cudaStreamSynchronize(st);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess)
            rc = cuda_fail(e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3, "auction result");
    }
    cudaFreeAsync(d_rp, st);
    cudaFreeAsync(d_col, st);
    cudaFreeAsync(d_val, st);
    cudaFreeAsync(d_price, st);
    cudaFreeAsync(d_asg, st);
    if (rc) return rc;
    double t1 = now_ms();
    info->phases = phases;
    info->rounds = rounds;
    info->complete = complete;
    info->eps_final = eps_final;
    info->auction_ms = t1 - t0;
    if (complete) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) {
            double best = -INFINITY;   // a repeated column: its best entry
            for (int64_t e = b.row_ptr[i]; e < b.row_ptr[i + 1]; ++e)
                if (b.col[e] == asg[i] && lw[e] > best) best = lw[e];
            s += best;
        }
        info->auction_sum_log_w = s;
    }
    // the exact solver from the auction's prices (its minimisation-form prices are -beta),
    // its shortest-augmenting-path searches on the GPU
    for (int j = 0; j < n; ++j) price[j] = -price[j];
    SspRun run{ctx};
    rc = solve_csr(b, perm, sum_log_w, alpha, beta, price.data(), ssp_device, &run);
    info->host_ms = now_ms() - t1;
    info->searches = run.searches;
    info->search_rounds = run.rounds;
    return rc;
}

}  // namespace sa

using namespace sa;

extern "C" {

const char* sa_last_error(void) { return tl_err.c_str(); }

int64_t sa_kernel_launches(void) { return (int64_t)g_kernel_launches.load(); }

const char* sa_version(void) {
    return "libsa 1.0 (sm_103a; fused single-read log-domain Sinkhorn, CSR prune, sparse SAP solve)";
}

sa_status sa_create(sa_ctx** ctx, int device, void* cuda_stream) {
    if (!ctx) { set_error("null ctx pointer"); return SA_E_INVALID; }
    *ctx = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) { set_error("device %d out of range (%d devices)", device, count); return SA_E_INVALID; }
    SA_CUDA(cudaSetDevice(device));
    sa_ctx* c = new sa_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaGetDeviceProperties"); }
    c->num_sms = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    if (!prop.cooperativeLaunch) { delete c; set_error("device lacks cooperative launch"); return SA_E_UNSUPPORTED; }
    *ctx = c;
    return SA_OK;
}

sa_status sa_set_option(sa_ctx* ctx, sa_option opt, int64_t value) {
    if (!ctx) { set_error("null context"); return SA_E_INVALID; }
    switch (opt) {
    case SA_OPT_WAIT_LIMIT_NS:
        if (value < 0) { set_error("wait limit must be >= 0 ns"); return SA_E_INVALID; }
        ctx->wait_ns = (uint64_t)value;
        return SA_OK;
    case SA_OPT_SOLVE_GPU:
        if (value != 0 && value != 1) { set_error("SA_OPT_SOLVE_GPU takes 0 or 1"); return SA_E_INVALID; }
        ctx->solve_gpu = (int)value;
        return SA_OK;
    case SA_OPT_STEP_SPARSE:
        if (value != 0 && value != 1) { set_error("SA_OPT_STEP_SPARSE takes 0 or 1"); return SA_E_INVALID; }
        ctx->step_sparse = (int)value;
        return SA_OK;
    case SA_OPT_MAX_GRID:
        if (value < 0 || value > (1 << 20)) { set_error("grid cap out of range"); return SA_E_INVALID; }
        ctx->max_grid = (int)value;
        return SA_OK;
    case SA_OPT_STEP_L2_BYTES:
        if (value < 0) { set_error("SA_OPT_STEP_L2_BYTES must be >= 0"); return SA_E_INVALID; }
        ctx->step_l2_bytes = (size_t)value;
        return SA_OK;
    case SA_OPT_TEST_UNREACHABLE_BARRIER:
        if (value != 0 && value != 1) { set_error("SA_OPT_TEST_UNREACHABLE_BARRIER takes 0 or 1"); return SA_E_INVALID; }
        ctx->test_unreachable_barrier = (int)value;
        return SA_OK;
    case SA_OPT_FUSED_THREADS:
        if (value != 256 && value != 512) { set_error("SA_OPT_FUSED_THREADS takes 256 or 512"); return SA_E_INVALID; }
        ctx->fused_nt = (int)value;
        return SA_OK;
    }
    set_error("unknown option %d", (int)opt);
    return SA_E_INVALID;
}

sa_status sa_set_batch_plan(sa_ctx* ctx, const sa_batch_plan* plan) {
    if (!ctx) { set_error("null context"); return SA_E_INVALID; }
    if (!plan) {
        ctx->batch_plan = default_batch_plan();
        return SA_OK;
    }
    if (plan->count < 1 || plan->count > SA_BATCH_MAX_BUCKETS) { set_error("plan needs 1 .. 8 buckets"); return SA_E_INVALID; }
    for (int b = 0; b < plan->count; ++b) {
        if (plan->n_hi[b] < 1 || (b > 0 && plan->n_hi[b] <= plan->n_hi[b - 1])) {
            set_error("plan bucket %d: n_hi must be positive and increasing", b);
            return SA_E_INVALID;
        }
        if (plan->path[b] == SA_BATCH_GROUP) {
            const int w = plan->warps[b], g = plan->per_block[b];
            if (plan->n_hi[b] > 128 || (w != 1 && w != 2 && w != 4) || g < 1 || w * g > 8) {
                set_error("plan bucket %d: the group path takes n_hi <= 128, 1, 2 or 4 warps per instance and "
                          "at most 8 warps per block", b);
                return SA_E_INVALID;
            }
        } else if (plan->path[b] == SA_BATCH_REGS) {
            const int w = plan->warps[b], g = plan->per_block[b], nh = plan->n_hi[b];
            const bool shape = (nh <= 32 && (w == 1 || w == 2 || w == 4)) || (nh <= 64 && (w == 4 || w == 8)) ||
                               (nh <= 128 && w == 16);
            if (!shape || g < 1 || w * g > 16) {
                set_error("plan bucket %d: the register path takes 1, 2 or 4 warps per instance up to n = 32, 4 or 8 "
                          "up to 64, 16 up to 128, and at most 16 warps per block", b);
                return SA_E_INVALID;
            }
        } else if (plan->path[b] != SA_BATCH_BLOCK && plan->path[b] != SA_BATCH_KROWS) {
            set_error("plan bucket %d: unknown path %d", b, plan->path[b]);
            return SA_E_INVALID;
        }
    }
    if (plan->n_hi[plan->count - 1] < 512) { set_error("the last bucket must reach n = 512"); return SA_E_INVALID; }
    ctx->batch_plan = *plan;
    return SA_OK;
}

void sa_destroy(sa_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (cudaStream_t& s : ctx->batch_streams)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t& e : ctx->batch_events)
        if (e) cudaEventDestroy(e);
    delete ctx;
}

sa_status sa_scale(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* d_u, double* d_v,
                   sa_scale_info* info) {
    if (!ctx) { set_error("null context"); return SA_E_INVALID; }
    sa_status rc = check_matrix(a);
    if (rc) return rc;
    if ((rc = check_opts(o))) return rc;
    if (!d_u || !d_v) { set_error("null potential buffers"); return SA_E_INVALID; }
    DeviceGuard g(ctx->device);
    sa_scale_info tmp{};
    if (!info) info = &tmp;
    memset(info, 0, sizeof(*info));
    const int n = a->n;
    sa_kernel kind = o->kernel;
    if (o->prec == SA_PREC_FP64) kind = SA_KERNEL_PLAIN;
    else if (kind == SA_KERNEL_AUTO) {
        if (o->prec == SA_PREC_MIXED && step_supported(ctx, a)) kind = SA_KERNEL_STEP;
        else kind = fused_supported(ctx, a) ? SA_KERNEL_FUSED : SA_KERNEL_PLAIN;
    }
    if (kind == SA_KERNEL_FUSED && !fused_supported(ctx, a)) {
        set_error("fused kernel needs a 16-byte aligned base, ld*sizeof(w) %% 16 == 0 and n <= 8192 (int16) / 4096 (int32)");
        return SA_E_UNSUPPORTED;
    }
    if (kind == SA_KERNEL_STEP && (o->prec != SA_PREC_MIXED || !step_supported(ctx, a))) {
        set_error("step kernel needs SA_PREC_MIXED, a 16-byte aligned base, ld*sizeof(w) %% 16 == 0 and n <= 24576");
        return SA_E_UNSUPPORTED;
    }
    if (kind == SA_KERNEL_NEWTON && (o->prec != SA_PREC_MIXED || !newton_supported(ctx, a))) {
        set_error("newton kernel needs SA_PREC_MIXED, a 16-byte aligned base and ld*sizeof(w) %% 16 == 0");
        return SA_E_UNSUPPORTED;
    }
    NvtxRange range("sa_scale n=%d kernel=%d p_steps=%d", n, (int)kind, o->n_p);
    // library units: log2.  A warm start is kept so that a failure leaves the caller's
    // potentials as they were given.
    if (o->resume_from > 0) {
        if ((rc = ctx->keep.reserve(2 * (size_t)n * sizeof(double)))) return rc;
        double* keep = (double*)ctx->keep.ptr;
        SA_CUDA(cudaMemcpyAsync(keep, d_u, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        SA_CUDA(cudaMemcpyAsync(keep + n, d_v, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
        launch_scale_vec(d_u, n, kLog2e, ctx->stream);
        launch_scale_vec(d_v, n, kLog2e, ctx->stream);
    }
    if (kind == SA_KERNEL_NEWTON) rc = scale_newton(ctx, a, o, d_u, d_v, info);
    else if (kind == SA_KERNEL_STEP) rc = scale_step(ctx, a, o, d_u, d_v, info);
    else if (kind == SA_KERNEL_FUSED) rc = scale_fused(ctx, a, o, d_u, d_v, info);
    else rc = scale_plain(ctx, a, o, d_u, d_v, info);
    if (rc == SA_OK || rc == SA_E_NOT_CONVERGED) {
        launch_scale_vec(d_u, n, kLn2, ctx->stream);
        launch_scale_vec(d_v, n, kLn2, ctx->stream);
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(e, "sa_scale");
    } else if (o->resume_from > 0) {
        const double* keep = (const double*)ctx->keep.ptr;
        cudaMemcpyAsync(d_u, keep, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
        cudaMemcpyAsync(d_v, keep + n, n * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream);
        cudaStreamSynchronize(ctx->stream);
    }
    return rc;
}

sa_status sa_verify(sa_ctx* ctx, const sa_matrix* a, double p, const double* d_u, const double* d_v,
                    double* d_rows, double* d_cols, double* max_row_err, double* max_col_err) {
    if (!ctx) { set_error("null context"); return SA_E_INVALID; }
    sa_status rc = check_matrix(a);
    if (rc) return rc;
    if (!d_u || !d_v || !(p > 0)) { set_error("bad potentials or p"); return SA_E_INVALID; }
    DeviceGuard g(ctx->device);
    return verify_device(ctx, a, p, d_u, d_v, d_rows, d_cols, max_row_err, max_col_err);
}

sa_status sa_prune(sa_ctx* ctx, const sa_matrix* a, double p, const double* d_u, const double* d_v, double t,
                   int32_t guard, sa_csr* out, double* log_ub) {
    if (!ctx || !out) { set_error("null context or output"); return SA_E_INVALID; }
    sa_status rc = check_matrix(a);
    if (rc) return rc;
    if (!d_u || !d_v || !(p > 0)) { set_error("bad potentials or p"); return SA_E_INVALID; }
    DeviceGuard g(ctx->device);
    memset(out, 0, sizeof(*out));
    return prune_device(ctx, a, p, d_u, d_v, t, guard, out, log_ub);
}

static sa_status check_csr(const sa_csr* b) {
    if (!b || b->n <= 0 || !b->row_ptr || (b->nnz > 0 && (!b->col || !b->w))) {
        set_error("bad reduced instance");
        return SA_E_INVALID;
    }
    for (int64_t e = 0; e < b->nnz; ++e)
        if (b->col[e] < 0 || b->col[e] >= b->n) { set_error("column index out of range"); return SA_E_INVALID; }
    return SA_OK;
}

sa_status sa_solve_reduced(const sa_csr* b, int32_t* perm, double* sum_log_w, double* alpha, double* beta) {
    if (!perm) { set_error("perm is NULL"); return SA_E_INVALID; }
    sa_status rc = check_csr(b);
    if (rc) return rc;
    return solve_csr(*b, perm, sum_log_w, alpha, beta);
}

sa_status sa_solve_reduced_near(const sa_csr* b, const double* beta0, int32_t* perm, double* sum_log_w,
                                double* alpha, double* beta) {
    if (!perm || !beta0) { set_error("perm or beta0 is NULL"); return SA_E_INVALID; }
    sa_status rc = check_csr(b);
    if (rc) return rc;
    return solve_csr_near(*b, beta0, perm, sum_log_w, alpha, beta);
}

sa_status sa_solve_reduced_warm(const sa_csr* b, const double* beta0, int32_t* perm, double* sum_log_w,
                                double* alpha, double* beta) {
    if (!perm || !beta0) { set_error("perm or beta0 is NULL"); return SA_E_INVALID; }
    sa_status rc = check_csr(b);
    if (rc) return rc;
    // minimisation-form starting prices -beta0 (non-finite entries: the column minimum)
    std::vector<double> price(b->n);
    for (int j = 0; j < b->n; ++j) price[j] = std::isfinite(beta0[j]) ? -beta0[j] : NAN;
    return solve_csr(*b, perm, sum_log_w, alpha, beta, price.data());
}

sa_status sa_solve_reduced_gpu(sa_ctx* ctx, const sa_csr* b, const double* price0, int32_t* perm, double* sum_log_w,
                               double* alpha, double* beta, sa_auction_info* info) {
    if (!ctx) { set_error("null context"); return SA_E_INVALID; }
    if (!b || !perm || b->n <= 0 || !b->row_ptr || (b->nnz > 0 && (!b->col || !b->w))) {
        set_error("bad reduced instance");
        return SA_E_INVALID;
    }
    // the kernels index by these: a malformed CSR is rejected here, not read on the device
    if (b->row_ptr[0] != 0 || b->row_ptr[b->n] != b->nnz) { set_error("row_ptr must run from 0 to nnz"); return SA_E_INVALID; }
    for (int i = 0; i < b->n; ++i)
        if (b->row_ptr[i + 1] < b->row_ptr[i]) { set_error("row_ptr decreases at row %d", i); return SA_E_INVALID; }
    for (int64_t e = 0; e < b->nnz; ++e)
        if (b->col[e] < 0 || b->col[e] >= b->n) { set_error("column index %d out of range", b->col[e]); return SA_E_INVALID; }
    DeviceGuard g(ctx->device);
    return solve_csr_gpu(ctx, *b, price0, perm, sum_log_w, alpha, beta, info);
}

sa_status sa_certify(sa_ctx* ctx, const sa_matrix* a, const double* alpha, const double* beta, double tau,
                     int64_t* n_viol, int64_t max_add, sa_csr* additions) {
    if (!ctx || !alpha || !beta || !n_viol) { set_error("null argument"); return SA_E_INVALID; }
    sa_status rc = check_matrix(a);
    if (rc) return rc;
    DeviceGuard g(ctx->device);
    if (additions) memset(additions, 0, sizeof(*additions));
    return certify_device(ctx, a, alpha, beta, tau, n_viol, max_add, additions);
}

void sa_csr_free(sa_csr* c) {
    if (!c) return;
    free(c->row_ptr);
    free(c->col);
    free(c->w);
    c->row_ptr = nullptr;
    c->col = nullptr;
    c->w = nullptr;
    c->nnz = 0;
}

sa_status sa_assign(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double t, sa_assign_result* res) {
    if (!ctx || !res || !res->perm) { set_error("null context or result"); return SA_E_INVALID; }
    sa_status rc = check_matrix(a);
    if (rc) return rc;
    if ((rc = check_opts(o))) return rc;
    DeviceGuard g(ctx->device);
    const int n = a->n;
    NvtxRange range("sa_assign n=%d", n);
    double* d_uv = nullptr;
    SA_CUDA(cudaMallocAsync((void**)&d_uv, 2 * sizeof(double) * n, ctx->stream));
    double* d_u = d_uv;
    double* d_v = d_uv + n;
    double t0 = now_ms();
    sa_scale_opts oo = *o;
    oo.resume_from = 0;
    rc = sa_scale(ctx, a, &oo, d_u, d_v, &res->scale);
    double t1 = now_ms();
    res->ms_scale = t1 - t0;
    if (rc != SA_OK && rc != SA_E_NOT_CONVERGED) { cudaFreeAsync(d_uv, ctx->stream); return rc; }
    const double p = o->p[o->n_p - 1];
    if (!(t > 0)) t = 1.0 / n;
    sa_csr B{};
    double log_ub = 0.0;
    std::vector<double> alpha(n), beta(n);
    // starting prices of the exact solve: -v/p (natural log), dual feasible since x <= 1
    std::vector<double> price(n);
    SA_CUDA(cudaMemcpyAsync(price.data(), d_v, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    SA_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int j = 0; j < n; ++j) price[j] = -price[j] / p;
    res->reprunes = 0;
    res->repairs = 0;
    res->ms_prune = res->ms_solve = res->ms_certify = 0.0;
    double first_sum = 0.0;
    bool have_first = false;
    // prune + solve, re-pruning at t/16 while B holds no permutation
    for (;;) {
        double a0 = now_ms();
        nvtxRangePushA("prune");
        rc = prune_device(ctx, a, p, d_u, d_v, t, 1, &B, have_first ? nullptr : &log_ub);
        nvtxRangePop();
        double a1 = now_ms();
        res->ms_prune += a1 - a0;
        if (rc) { cudaFreeAsync(d_uv, ctx->stream); return rc; }
        if (!have_first) res->nnz_first = B.nnz;
        NvtxRange solve_range("solve B nnz=%lld", (long long)B.nnz);
        if (ctx->solve_gpu && B.nnz >= kAuctionMinNnz) {
            std::vector<double> pmax(n);
            for (int j = 0; j < n; ++j) pmax[j] = -price[j];
            rc = solve_csr_gpu(ctx, B, pmax.data(), res->perm, &res->sum_log_w, alpha.data(), beta.data(), nullptr);
        } else {
            // B from the column minima, then the optimal duals closest below the scaling's
            // v/p: those hold on the rest of A as well (x <= 1 there), so the certificate
            // below rarely adds entries.  Starting the search from v/p instead gives such
            // duals too, but makes nearly every entry of B almost tight and the searches long
            // (measured on the host: 20.8 s against 22 ms on a Zipf-weighted B of n = 2048)
            std::vector<double> beta0(n);
            for (int j = 0; j < n; ++j) beta0[j] = -price[j];
            rc = solve_csr_near(B, beta0.data(), res->perm, &res->sum_log_w, alpha.data(), beta.data());
        }
        res->ms_solve += now_ms() - a1;
        if (rc == SA_OK) break;
        sa_csr_free(&B);
        if (rc != SA_E_NO_PERFECT_MATCHING) { cudaFreeAsync(d_uv, ctx->stream); return rc; }
        if (t == 0.0) { cudaFreeAsync(d_uv, ctx->stream); return rc; }   // all of A: no support
        res->reprunes++;
        t = t / 16.0;
        if (t < 1e-300) t = 0.0;
        have_first = true;   // gamma refers to the first successful B below
    }
    first_sum = res->sum_log_w;
    res->log_ub = log_ub;
    res->gamma = std::exp(log_ub - first_sum);
    // LP-duality repair: add violating entries of A until none is left
    for (int iter = 0;; ++iter) {
        NvtxRange cert_range("certify %d", iter);
        double c0 = now_ms();
        int64_t nv = 0;
        sa_csr add{};
        const int64_t max_add = std::max<int64_t>(4 * (int64_t)n, 1 << 16);
        rc = certify_device(ctx, a, alpha.data(), beta.data(), 1e-9, &nv, max_add, &add);
        res->ms_certify += now_ms() - c0;
        if (rc) { sa_csr_free(&B); cudaFreeAsync(d_uv, ctx->stream); return rc; }
        if (nv == 0) { sa_csr_free(&add); break; }
        sa_csr merged{};
        rc = csr_union(B, add, &merged);
        sa_csr_free(&add);
        sa_csr_free(&B);
        if (rc) { cudaFreeAsync(d_uv, ctx->stream); return rc; }
        B = merged;
        res->repairs++;
        double s0 = now_ms();
        // from the last optimal duals: only the added entries break their optimality
        for (int j = 0; j < n; ++j) price[j] = -beta[j];
        rc = solve_csr(B, res->perm, &res->sum_log_w, alpha.data(), beta.data(), price.data());
        res->ms_solve += now_ms() - s0;
        if (rc) { sa_csr_free(&B); cudaFreeAsync(d_uv, ctx->stream); return rc; }
        if (iter > 64) { set_error("duality repair did not settle"); sa_csr_free(&B); cudaFreeAsync(d_uv, ctx->stream); return SA_E_NOT_CONVERGED; }
    }
    res->nnz_final = B.nnz;
    sa_csr_free(&B);
    cudaFreeAsync(d_uv, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sa_assign");
    return SA_OK;
}

sa_status sa_algorithm1(sa_ctx* ctx, const sa_matrix* a, const sa_alg1_opts* o, sa_alg1_result* res) {
    if (!ctx || !o || !res || !res->perm) { set_error("null context, options or result"); return SA_E_INVALID; }
    sa_status rc = check_matrix(a);
    if (rc) return rc;
    if (!(o->opt_ratio > 1.0) || !(o->p0 > 0) || !(o->dp > 0) || o->max_rounds <= 0 || o->max_sweeps_per_p <= 0) {
        set_error("algorithm 1 needs opt_ratio > 1, p0 > 0, dp > 0, max_rounds > 0 and max_sweeps_per_p > 0");
        return SA_E_INVALID;
    }
    DeviceGuard g(ctx->device);
    const int n = a->n;
    int64_t wmin = 0, wmax = 0;
    if ((rc = weights_minmax(ctx, a, &wmin, &wmax))) return rc;
    // prescaling (Sec. 4.1.1): A^(m)/c has entries in [1, e]; X at p on that scale is X of A at p m
    const double ratio = (double)wmax / (double)wmin;
    const double m = ratio > std::exp(1.0) ? 1.0 / std::log(ratio) : 1.0;
    const double eps = o->eps > 0 ? o->eps : 1.0 / n;
    const double t = o->t > 0 ? o->t : 1.0 / n;
    double* d_uv = nullptr;
    SA_CUDA(cudaMallocAsync((void**)&d_uv, 2 * sizeof(double) * n, ctx->stream));
    double* d_u = d_uv;
    double* d_v = d_uv + n;
    std::vector<double> alpha(n), beta(n);
    std::vector<int32_t> perm(n);
    res->rounds = 0;
    res->sweeps_total = 0;
    res->gamma = INFINITY;
    double p = o->p0, p_prev_raw = 0.0;
    sa_status out = SA_E_NOT_CONVERGED;
    for (int r = 0; r < o->max_rounds; ++r, p += o->dp) {
        NvtxRange round_range("algorithm 1 round %d (p=%g)", r, p);
        const double p_raw = p * m;
        double sched[2] = {p_prev_raw, p_raw};
        sa_scale_opts so{};
        so.p = r == 0 ? sched + 1 : sched;
        so.n_p = r == 0 ? 1 : 2;
        so.tol = eps;
        so.max_sweeps_per_p = o->max_sweeps_per_p;
        so.prec = o->prec;
        so.kernel = o->kernel;
        so.warm_keep_v = 0;
        so.resume_from = r == 0 ? 0 : 1;   // warm start: (u, v) * p_raw / p_prev_raw
        sa_scale_info info{};
        rc = sa_scale(ctx, a, &so, d_u, d_v, &info);
        if (rc != SA_OK && rc != SA_E_NOT_CONVERGED) { out = rc; break; }
        res->sweeps_total += info.sweeps_total;
        res->rounds = r + 1;
        res->p_final = p;
        res->p_raw = p_raw;
        p_prev_raw = p_raw;
        sa_csr B{};
        double log_ub = 0.0;
        rc = prune_device(ctx, a, p_raw, d_u, d_v, t, 1, &B, &log_ub);
        if (rc) { out = rc; break; }
        double sum = 0.0;
        // from the column minima: no certificate follows here, and the scaling's duals leave
        // nearly every entry of B almost tight, which makes the searches long (measured on the
        // host: 22.5 s against 26 ms on a Zipf-weighted B of n = 2048)
        rc = solve_csr(B, perm.data(), &sum, alpha.data(), beta.data());
        const int64_t nnz = B.nnz;
        sa_csr_free(&B);
        if (rc != SA_OK && rc != SA_E_NO_PERFECT_MATCHING) { out = rc; break; }
        const double gam = rc == SA_OK ? std::exp(log_ub - sum) : INFINITY;
        if (rc == SA_OK) {
            std::copy(perm.begin(), perm.end(), res->perm);
            res->sum_log_w = sum;
            res->nnz = nnz;
        }
        res->gamma = gam;
        if (gam <= o->opt_ratio) { out = SA_OK; break; }
    }
    cudaFreeAsync(d_uv, ctx->stream);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sa_algorithm1");
    if (out == SA_E_NOT_CONVERGED) set_error("gamma above opt_ratio after %d rounds (last %g)", o->max_rounds, res->gamma);
    return out;
}

sa_status sa_assign_host(sa_ctx* ctx, const void* host_w, sa_wtype wtype, int32_t n, int64_t ld,
                         const sa_scale_opts* o, double t, sa_assign_result* res) {
    if (!ctx || !host_w || n <= 0 || ld < n) { set_error("bad host matrix"); return SA_E_INVALID; }
    DeviceGuard g(ctx->device);
    const int sz = wbytes(wtype);
    // device copy with a 16-byte aligned pitch so the fused kernel can take it
    const int64_t dld = (int64_t)align_up((size_t)n * sz, 16) / sz;
    sa_status rc = ctx->input.reserve((size_t)dld * n * sz);
    if (rc) return rc;
    SA_CUDA(cudaMemcpy2DAsync(ctx->input.ptr, (size_t)dld * sz, host_w, (size_t)ld * sz, (size_t)n * sz, n,
                              cudaMemcpyHostToDevice, ctx->stream));
    sa_matrix a{ctx->input.ptr, wtype, n, dld};
    return sa_assign(ctx, &a, o, t, res);
}

sa_status sa_narrow_i32_to_i16(sa_ctx* ctx, const int32_t* d_src, int64_t ld_src, int16_t* d_dst, int64_t ld_dst,
                               int32_t n, int64_t* n_bad) {
    if (!ctx || !d_src || !d_dst || n <= 0 || ld_src < n || ld_dst < n) { set_error("bad narrowing arguments"); return SA_E_INVALID; }
    DeviceGuard g(ctx->device);
    return narrow_device(ctx, d_src, ld_src, d_dst, ld_dst, n, n_bad);
}

}  // extern "C"
