// server.cpp -- continuous-batching server for assignment requests (sa_submit/sa_poll).
//
// Requests of mixed size arrive at any time.  A request is admitted when the device
// memory it can need (its int16/int32 matrix, potentials, the scaling workspace and the
// reduced instance's device arrays, bounded from above) fits in the budget next to the
// requests already resident, so new work joins while earlier work is still on the GPU.
// A large request's worker gives its context's buffers back to the device when the
// request finishes, with its share of the budget.  Worker threads, each with its own CUDA stream and library context, run admitted
// requests concurrently on the device:
//  - small requests (n <= 512) are drained from the queue in groups and scaled together
//    by one sa_batch_scale launch, then pruned, solved and certified one by one;
//  - larger requests run the whole path (sa_assign: fused sweep kernel, prune, exact
//    solve, duality repair) on a worker of their own.
// Every kernel launch is finite; results are kept until sa_result_release.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "sa_internal.h"

namespace {

constexpr int kSmallMax = 512;

struct Request {
    uint64_t ticket = 0;
    int n = 0;
    sa_wtype wtype = SA_I16;
    std::vector<unsigned char> host;   // n x n weights, row-major
    size_t dev_bytes = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    bool done = false;
    sa_status status = SA_PENDING;
    std::vector<int32_t> perm;
    double sum_log_w = 0, gamma = 0;
    int64_t sweeps = 0;
};

}  // namespace

struct sa_server {
    int device = 0;
    size_t budget = 0, used = 0;
    std::vector<double> sched;
    sa_scale_opts opts{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> queue;
    std::map<uint64_t, std::unique_ptr<Request>> all;
    std::vector<std::thread> workers;
    bool stop = false;
    uint64_t next_ticket = 1;
    std::chrono::steady_clock::time_point t0;
    int large_grid = 0;
    int num_sms = 0;

    double now() const {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Test hook (sa_debug_fail_allocs): this many of the next device allocations of the
// request paths fail as if the device were out of memory, without allocating.
std::atomic<int> g_fail_allocs{0};

cudaError_t srv_alloc(void** p, size_t bytes, cudaStream_t st) {
    int k = g_fail_allocs.load();
    while (k > 0) {
        if (g_fail_allocs.compare_exchange_weak(k, k - 1)) {
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMallocAsync(p, bytes, st);
}

// Device bytes a request can hold while it runs (an upper bound).  Small requests: the
// matrix, the potentials, the reduced instance's device arrays (8 bytes per kept entry,
// at most n^2), the batch launch's tables and, above n = 128, a slot of K.  Large ones: the matrix and everything
// sa_assign allocates (sa::assign_device_bound).  What is not counted is each worker
// context's small persistent state: the small workers' workspaces (a few MiB for
// n <= 512) and the CUDA streams.
size_t request_bytes(int n, sa_wtype wt, int num_sms) {
    const size_t sz = wt == SA_I16 ? 2 : 4;
    const size_t ld = sa::align_up((size_t)n * sz, 16) / sz;
    const size_t matrix = ld * n * sz;
    // above n = 128 the batched form may keep K in a global slot sized for the group's
    // largest instance (at most 4 * 512 * 512 bytes, one slot per instance at most)
    if (n <= kSmallMax)
        return matrix + 2 * sizeof(double) * n + 8 * (size_t)n * n + 64 + (1 << 20) +
               (n > 128 ? (size_t)4 * kSmallMax * kSmallMax : 0);
    return matrix + sa::assign_device_bound(num_sms, n);
}

// Take requests from the head of the queue while they fit the budget.  small_only picks
// a group of small requests (up to max_take); otherwise one request of any size.
std::vector<Request*> admit(sa_server* s, bool small_only, int max_take, std::unique_lock<std::mutex>& lk) {
    std::vector<Request*> got;
    for (auto it = s->queue.begin(); it != s->queue.end() && (int)got.size() < max_take;) {
        Request* r = *it;
        const bool small = r->n <= kSmallMax;
        // one launch takes one weight type
        if (small_only != small || (!got.empty() && r->wtype != got[0]->wtype)) { ++it; continue; }
        if (s->used + r->dev_bytes > s->budget) break;   // FIFO within a class: wait for memory
        s->used += r->dev_bytes;
        r->t_start = s->now();
        got.push_back(r);
        it = s->queue.erase(it);
    }
    (void)lk;
    return got;
}

void finish(sa_server* s, Request* r, sa_status st) {
    std::lock_guard<std::mutex> g(s->mu);
    r->status = st;
    r->t_done = s->now();
    r->done = true;
    s->used -= r->dev_bytes;
    r->host.clear();
    r->host.shrink_to_fit();
    s->cv.notify_all();
}

// copy a request into a device buffer with a 16-byte row pitch
sa_status upload(Request* r, cudaStream_t st, void** d_w, int64_t* ld) {
    const size_t sz = r->wtype == SA_I16 ? 2 : 4;
    *ld = (int64_t)(sa::align_up((size_t)r->n * sz, 16) / sz);
    SA_CUDA(srv_alloc(d_w, (size_t)(*ld) * r->n * sz, st));
    SA_CUDA(cudaMemcpy2DAsync(*d_w, (size_t)(*ld) * sz, r->host.data(), (size_t)r->n * sz, (size_t)r->n * sz, r->n,
                              cudaMemcpyHostToDevice, st));
    return SA_OK;
}

// prune + solve + certify one scaled instance (the tail of sa_assign)
sa_status finish_small(sa_ctx* ctx, Request* r, const sa_matrix* a, const double* d_u, const double* d_v,
                       double p) {
    // the scaling's column duals v/p: B is solved from the column minima and then given the
    // optimal duals closest below them, which hold on the rest of A as well (x <= 1 there),
    // so the certificate rarely adds entries
    std::vector<double> beta0(r->n);
    SA_CUDA(cudaMemcpyAsync(beta0.data(), d_v, sizeof(double) * r->n, cudaMemcpyDeviceToHost, ctx->stream));
    SA_CUDA(cudaStreamSynchronize(ctx->stream));
    for (double& x : beta0) x /= p;
    sa_csr B{};
    double log_ub = 0;
    sa_status rc = sa_prune(ctx, a, p, d_u, d_v, 0.0, 1, &B, &log_ub);
    if (rc) return rc;
    std::vector<double> al(r->n), be(r->n);
    r->perm.assign(r->n, -1);
    rc = sa_solve_reduced_near(&B, beta0.data(), r->perm.data(), &r->sum_log_w, al.data(), be.data());
    double t = 1.0 / r->n;
    while (rc == SA_E_NO_PERFECT_MATCHING && t > 0) {
        sa_csr_free(&B);
        t = t / 16 < 1e-300 ? 0.0 : t / 16;
        rc = sa_prune(ctx, a, p, d_u, d_v, t, 1, &B, nullptr);
        if (rc) return rc;
        rc = sa_solve_reduced_near(&B, beta0.data(), r->perm.data(), &r->sum_log_w, al.data(), be.data());
    }
    if (rc) { sa_csr_free(&B); return rc; }
    r->gamma = std::exp(log_ub - r->sum_log_w);
    bool certified = false;
    for (int iter = 0; iter < 64; ++iter) {
        int64_t nv = 0;
        sa_csr add{};
        rc = sa_certify(ctx, a, al.data(), be.data(), 1e-9, &nv, 1 << 16, &add);
        if (rc || nv == 0) {
            certified = rc == SA_OK;
            sa_csr_free(&add);
            break;
        }
        // merge and re-solve
        std::vector<int64_t> rp(r->n + 1, 0);
        std::vector<int32_t> cols, ws;
        for (int i = 0; i < r->n; ++i) {
            int64_t x = B.row_ptr[i], xe = B.row_ptr[i + 1], y = add.row_ptr[i], ye = add.row_ptr[i + 1];
            while (x < xe || y < ye) {
                if (y >= ye || (x < xe && B.col[x] < add.col[y])) { cols.push_back(B.col[x]); ws.push_back(B.w[x]); ++x; }
                else if (x >= xe || add.col[y] < B.col[x]) { cols.push_back(add.col[y]); ws.push_back(add.w[y]); ++y; }
                else { cols.push_back(B.col[x]); ws.push_back(B.w[x]); ++x; ++y; }
            }
            rp[i + 1] = (int64_t)cols.size();
        }
        sa_csr_free(&add);
        sa_csr_free(&B);
        sa_status ac = sa::csr_alloc(&B, r->n, (int64_t)cols.size());
        if (ac) return ac;
        memcpy(B.row_ptr, rp.data(), 8 * (r->n + 1));
        memcpy(B.col, cols.data(), 4 * cols.size());
        memcpy(B.w, ws.data(), 4 * ws.size());
        // from the last optimal duals: only the added entries break their optimality
        const std::vector<double> prev(be);
        rc = sa_solve_reduced_warm(&B, prev.data(), r->perm.data(), &r->sum_log_w, al.data(), be.data());
        if (rc) break;
    }
    sa_csr_free(&B);
    if (rc == SA_OK && !certified) {
        sa::set_error("duality repair did not settle");
        rc = SA_E_NOT_CONVERGED;
    }
    return rc;
}

void small_worker(sa_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    // without a context on the device the worker still takes its requests and fails each
    // with the creation status, so that no request of its class stays pending
    sa_ctx* ctx = nullptr;
    const sa_status crc = sa_create(&ctx, s->device, st);
    for (;;) {
        std::vector<Request*> group;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                if (s->stop) return true;
                for (Request* r : s->queue)
                    if (r->n <= kSmallMax) return s->used + r->dev_bytes <= s->budget;
                return false;
            });
            if (s->stop) break;
            group = admit(s, true, 256, lk);
        }
        if (group.empty()) continue;
        if (crc != SA_OK) {
            for (Request* r : group) finish(s, r, crc);
            continue;
        }
        const int k = (int)group.size();
        std::vector<void*> dw(k, nullptr);
        std::vector<int32_t> ns(k);
        std::vector<int64_t> lds(k), offs(k);
        int64_t tot = 0;
        sa_status rc = SA_OK;
        for (int q = 0; q < k && rc == SA_OK; ++q) {
            rc = upload(group[q], st, &dw[q], &lds[q]);
            ns[q] = group[q]->n;
            offs[q] = tot;
            tot += group[q]->n;
        }
        // d_uv (k * 16 n bytes in all) is within the group's charge: 16 n of each request
        // the group's tables (pointers, sizes, pitches, offsets) in one buffer, then the
        // potentials; every allocation and copy is checked, and a failure fails the group
        const size_t tab = sa::align_up(8 * (size_t)k, 256);
        unsigned char* d_tab = nullptr;
        double* d_uv = nullptr;
        if (rc == SA_OK) {
            cudaError_t e = srv_alloc((void**)&d_tab, 4 * tab, st);
            if (e == cudaSuccess) e = srv_alloc((void**)&d_uv, 16 * (size_t)tot, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab, dw.data(), 8 * k, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab + tab, ns.data(), 4 * k, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab + 2 * tab, lds.data(), 8 * k, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(d_tab + 3 * tab, offs.data(), 8 * k, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) rc = sa::cuda_fail(e, "server: group tables");
        }
        if (rc == SA_OK) {
            void** d_ptrs = (void**)d_tab;
            int32_t* d_n = (int32_t*)(d_tab + tab);
            int64_t* d_ld = (int64_t*)(d_tab + 2 * tab);
            int64_t* d_off = (int64_t*)(d_tab + 3 * tab);
            std::vector<int32_t> sw(k), stt(k);
            rc = sa_batch_scale(ctx, k, (const void* const*)d_ptrs, d_n, d_ld, d_off, group[0]->wtype, &s->opts, d_uv,
                                d_uv + tot, sw.data(), stt.data());
            const double p = s->sched.back();
            for (int q = 0; q < k; ++q) {
                Request* r = group[q];
                r->sweeps = sw[q];
                sa_status rq = (rc == SA_OK || rc == SA_E_NOT_CONVERGED) && stt[q] >= 0 ? SA_OK : (stt[q] < 0 ? SA_E_NONFINITE : rc);
                if (rq == SA_OK) {
                    sa_matrix a{dw[q], r->wtype, r->n, lds[q]};
                    rq = finish_small(ctx, r, &a, d_uv + offs[q], d_uv + tot + offs[q], p);
                }
                cudaFreeAsync(dw[q], st);
                cudaStreamSynchronize(st);
                finish(s, r, rq);
            }
            cudaFreeAsync(d_tab, st);
            cudaFreeAsync(d_uv, st);
            cudaStreamSynchronize(st);
            // the group's K slots were charged to its requests: keep only a small workspace
            if (ctx->ws.size > ((size_t)32 << 20)) sa::release_buffers(ctx);
        } else {
            if (d_tab) cudaFreeAsync(d_tab, st);
            if (d_uv) cudaFreeAsync(d_uv, st);
            for (int q = 0; q < k; ++q)
                if (dw[q]) cudaFreeAsync(dw[q], st);
            cudaStreamSynchronize(st);
            for (int q = 0; q < k; ++q) finish(s, group[q], rc);
        }
    }
    if (ctx) sa_destroy(ctx);
    cudaStreamDestroy(st);
}

void large_worker(sa_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    sa_ctx* ctx = nullptr;
    const sa_status crc = sa_create(&ctx, s->device, st);   // failing: as in small_worker
    if (crc == SA_OK) ctx->max_grid = s->large_grid;
    for (;;) {
        Request* r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                if (s->stop) return true;
                for (Request* q : s->queue)
                    if (q->n > kSmallMax) return s->used + q->dev_bytes <= s->budget;
                return false;
            });
            if (s->stop) break;
            auto got = admit(s, false, 1, lk);
            if (got.empty()) continue;
            r = got[0];
        }
        if (crc != SA_OK) {
            finish(s, r, crc);
            continue;
        }
        void* dw = nullptr;
        int64_t ld = 0;
        sa_status rc = upload(r, st, &dw, &ld);
        if (rc == SA_OK) {
            sa_matrix a{dw, r->wtype, r->n, ld};
            r->perm.assign(r->n, -1);
            sa_assign_result res{};
            res.perm = r->perm.data();
            rc = sa_assign(ctx, &a, &s->opts, 0.0, &res);
            r->sum_log_w = res.sum_log_w;
            r->gamma = res.gamma;
            r->sweeps = res.scale.sweeps_total;
        }
        if (dw) cudaFreeAsync(dw, st);
        cudaStreamSynchronize(st);
        // the request's share of the budget covered the context's buffers: give them back
        sa::release_buffers(ctx);
        finish(s, r, rc);
    }
    if (ctx) sa_destroy(ctx);
    cudaStreamDestroy(st);
}

}  // namespace

extern "C" {

sa_status sa_server_create(sa_server** out, int device, size_t hbm_budget, const sa_scale_opts* opts,
                           int32_t solver_threads) {
    if (!out || !opts || !opts->p || opts->n_p <= 0 || hbm_budget == 0) {
        sa::set_error("bad server arguments");
        return SA_E_INVALID;
    }
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        sa::set_error("bad device %d", device);
        return SA_E_INVALID;
    }
    sa_server* s = new sa_server();
    s->device = device;
    s->budget = hbm_budget;
    s->sched.assign(opts->p, opts->p + opts->n_p);
    s->opts = *opts;
    s->opts.p = s->sched.data();
    s->opts.resume_from = 0;
    s->t0 = std::chrono::steady_clock::now();
    const int large = std::max(1, solver_threads > 0 ? solver_threads : 2);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        delete s;
        sa::set_error("cudaGetDeviceProperties failed for device %d", device);
        return SA_E_CUDA;
    }
    s->num_sms = prop.multiProcessorCount;
    s->large_grid = std::max(8, prop.multiProcessorCount / large);
    for (int q = 0; q < 2; ++q) s->workers.emplace_back(small_worker, s);
    for (int q = 0; q < large; ++q) s->workers.emplace_back(large_worker, s);
    *out = s;
    return SA_OK;
}

void sa_server_destroy(sa_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    for (auto& t : s->workers) t.join();
    delete s;
}

sa_status sa_submit(sa_server* s, const void* host_w, sa_wtype wtype, int32_t n, uint64_t* ticket) {
    if (!s || !host_w || n <= 0 || !ticket || (wtype != SA_I16 && wtype != SA_I32)) {
        sa::set_error("bad request");
        return SA_E_INVALID;
    }
    auto r = std::make_unique<Request>();
    r->n = n;
    r->wtype = wtype;
    r->dev_bytes = request_bytes(n, wtype, s->num_sms);
    if (r->dev_bytes > s->budget) {
        sa::set_error("request of n=%d needs %zu bytes, over the %zu byte budget", n, r->dev_bytes, s->budget);
        return SA_E_BUDGET;
    }
    const size_t sz = wtype == SA_I16 ? 2 : 4;
    r->host.resize((size_t)n * n * sz);
    memcpy(r->host.data(), host_w, r->host.size());
    std::lock_guard<std::mutex> g(s->mu);
    r->ticket = s->next_ticket++;
    r->t_submit = s->now();
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->all[r->ticket] = std::move(r);
    s->cv.notify_all();
    return SA_OK;
}

sa_status sa_poll(sa_server* s, uint64_t ticket, sa_result* out) {
    if (!s || !out) { sa::set_error("bad poll"); return SA_E_INVALID; }
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) { sa::set_error("unknown ticket %llu", (unsigned long long)ticket); return SA_E_INVALID; }
    Request* r = it->second.get();
    if (!r->done) return SA_PENDING;
    out->n = r->n;
    out->perm = r->perm.empty() ? nullptr : r->perm.data();
    out->sum_log_w = r->sum_log_w;
    out->gamma = r->gamma;
    out->sweeps = r->sweeps;
    out->status = r->status;
    out->t_submit = r->t_submit;
    out->t_start = r->t_start;
    out->t_done = r->t_done;
    return r->status == SA_E_NOT_CONVERGED ? SA_OK : r->status;
}

void sa_result_release(sa_server* s, uint64_t ticket) {
    if (!s) return;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->all.find(ticket);
    if (it != s->all.end() && it->second->done) s->all.erase(it);
}

double sa_server_now(const sa_server* s) { return s ? s->now() : 0.0; }

size_t sa_server_request_bytes(const sa_server* s, sa_wtype wtype, int32_t n) {
    if (!s || n <= 0 || (wtype != SA_I16 && wtype != SA_I32)) return 0;
    return request_bytes(n, wtype, s->num_sms);
}

void sa_debug_fail_allocs(int32_t count) { g_fail_allocs.store(count > 0 ? count : 0); }

}  // extern "C"
