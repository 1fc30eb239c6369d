// server.cpp -- continuous-batching server for assignment requests (sa_submit/sa_poll).
//
// Requests of mixed size arrive at any time.  A request is admitted when the device
// memory it can need (its int16/int32 matrix, potentials, the scaling workspace and the
// reduced instance's device arrays, bounded from above) fits in the budget next to the
// requests already resident, so new work joins while earlier work is still on the GPU.
// A large request's worker gives its context's buffers back to the device when the
// request finishes, with its share of the budget.
//  - Small requests (n <= 512) go through a device-resident queue (serve_live.cu): a
//    worker uploads the matrix and publishes the request in a ring in host-mapped memory,
//    and the blocks of a persistent kernel take requests from the ring as they free up,
//    one request per block, so a request joins the scaling already under way instead of
//    waiting for a launch.  A dispatcher thread collects the completion flags, hands the
//    scaled requests to the workers (prune, exact solve and certificate, one by one) and
//    starts the queue's kernel when published requests find none running.
//  - Larger requests run the whole path (sa_assign: step sweep kernel, prune, exact
//    solve, duality repair) on a worker of their own, with a grid that leaves the
//    queue's blocks their SMs.
// Every kernel launch is finite; results are kept until sa_result_release.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
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
// small-request workers: each admits and uploads requests and runs the host-driven prune,
// exact solve and certificate of scaled ones (four measured slower than two: their prune
// and certificate kernels compete for the SMs the scaling kernels leave)
constexpr int kSmallWorkers = 2;

struct Request {
    uint64_t ticket = 0;
    int n = 0;
    sa_wtype wtype = SA_I16;
    std::vector<unsigned char> host;   // n x n weights, row-major
    size_t dev_bytes = 0;
    // small requests on the device-resident queue
    void* d_w = nullptr;                // device matrix
    int64_t ld = 0;
    double* d_uv = nullptr;             // device potentials u (n) then v (n)
    unsigned seq = 0;                   // position in the queue
    double t_pub = 0;                   // when it was published
    int32_t live_sweeps = 0, live_status = 0;
    sa_status live_rc = SA_OK;          // a failed launch of the queue's kernel
    double t_submit = 0, t_start = 0, t_done = 0, t_scaled = 0;
    bool done = false;
    sa_status status = SA_PENDING;
    std::vector<int32_t> perm;
    double sum_log_w = 0, gamma = 0;
    int64_t sweeps = 0;
};

// The device-resident queue of small requests: a ring in host-mapped memory, device
// counters, and two launch slots (stream, completion event, slots of K), so that a second
// kernel of the queue can start while the first one's blocks are all busy.
struct LiveQueue {
    static constexpr int kLaunchSlots = 2;
    int grid = 0;                        // most blocks of one launch (slots of K per launch slot)
    int sm_cap = 0;                      // most blocks (SMs) of one launch while large requests run
    int sms_run[kLaunchSlots] = {};      // SMs counted for each running launch (one per block:
                                         // the block scheduler may spread them)
    unsigned cap = 0;                    // ring slots
    unsigned char* host = nullptr;       // host-mapped ring and flags
    void* dev = nullptr;                 // head, busy, schedule, slots of K
    size_t dev_bytes = 0;
    sa::LiveArgs args{};                 // pointers as the device sees them
    unsigned* tail = nullptr;            // host views of the mapped words
    unsigned* stop = nullptr;
    unsigned* claimed = nullptr;
    unsigned* done = nullptr;
    int32_t* sweeps = nullptr;
    int32_t* status = nullptr;
    sa::LiveDesc* desc = nullptr;
    float* kbase = nullptr;              // launch slot s: kbase + s * grid * slot floats
    cudaStream_t stream[kLaunchSlots] = {};
    cudaEvent_t ev[kLaunchSlots] = {};
    bool running[kLaunchSlots] = {};
    unsigned published = 0;
    unsigned reserved = 0;               // admitted and not yet scaled (<= cap)
    std::vector<Request*> slot;          // in flight per ring slot
    int inflight = 0;
    int64_t launches = 0, served = 0;
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
    int large_grid = 0;                  // a large request's grid when the GPU is free
    int num_sms = 0;
    int sm_live = 0;                     // blocks of the request queue's running launches
    int sm_large = 0;                    // grids of the large requests' running scaling
    LiveQueue live;
    std::deque<Request*> scaled;         // small requests scaled on the queue, to finish
    std::thread dispatcher;

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
// at most n^2) and 1 MiB (the slots of K they are scaled on belong to the queue, whose
// device memory is charged once when the server starts).  Large ones: the matrix and
// everything sa_assign allocates (sa::assign_device_bound).  What is not counted is each
// worker context's small persistent state: the small workers' workspaces (a few MiB for
// n <= 512) and the CUDA streams.
size_t request_bytes(int n, sa_wtype wt, int num_sms) {
    const size_t sz = wt == SA_I16 ? 2 : 4;
    const size_t ld = sa::align_up((size_t)n * sz, 16) / sz;
    const size_t matrix = ld * n * sz;
    if (n <= kSmallMax) return matrix + 2 * sizeof(double) * n + 8 * (size_t)n * n + 64 + (1 << 20);
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
    // a failed request leaves a line on stderr with the worker's last error message
    if (st != SA_OK && st != SA_E_NOT_CONVERGED)
        fprintf(stderr, "sa_server: request %llu (n=%d) failed with status %d: %s\n", (unsigned long long)r->ticket, r->n,
                (int)st, sa_last_error());
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

// Publish an uploaded small request on the queue (lock held).  Request q takes ring slot
// q % cap, which request q - cap must have left: the caller waits for that (the dispatcher
// frees a slot when its request is scaled).
void live_publish(sa_server* s, Request* r) {
    LiveQueue& L = s->live;
    const unsigned q = L.published;
    const unsigned j = q % L.cap;
    sa::LiveDesc& d = L.desc[j];
    d.w = r->d_w;
    d.u = r->d_uv;
    d.v = r->d_uv + r->n;
    d.ld = r->ld;
    d.n = r->n;
    d.i16 = r->wtype == SA_I16;
    r->seq = q;
    r->t_pub = s->now();
    L.slot[j] = r;
    ++L.inflight;
    L.published = q + 1;
    __atomic_store_n(L.tail, q + 1, __ATOMIC_RELEASE);   // the descriptor before the tail
    s->cv.notify_all();
}

bool small_admissible(const sa_server* s) {
    for (const Request* r : s->queue)
        if (r->n <= kSmallMax) return s->used + r->dev_bytes <= s->budget;
    return false;
}

// Small-request worker: admits small requests in groups (upload, then publish on the
// queue) and finishes those the queue has scaled (prune, exact solve, certificate).
// Admission goes first: it is quick, and it keeps the queue's blocks supplied.
void small_worker(sa_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    // without a context on the device the worker still takes its requests and fails each
    // with the creation status, so that no request of its class stays pending
    sa_ctx* ctx = nullptr;
    const sa_status crc = sa_create(&ctx, s->device, st);
    LiveQueue& L = s->live;
    for (;;) {
        std::vector<Request*> adm;
        Request* fin = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [&] {
                return s->stop || !s->scaled.empty() || (L.reserved < L.cap && small_admissible(s));
            });
            if (s->stop) break;
            if (L.reserved < L.cap && small_admissible(s)) {
                adm = admit(s, true, (int)std::min<unsigned>(32u, L.cap - L.reserved), lk);
                L.reserved += (unsigned)adm.size();
            }
            if (adm.empty()) {
                if (s->scaled.empty()) continue;
                fin = s->scaled.front();
                s->scaled.pop_front();
            }
        }
        if (fin) {
            sa::NvtxRange range("server: finish request %llu n=%d", (unsigned long long)fin->ticket, fin->n);
            sa_status rq = fin->live_rc;
            if (rq == SA_OK) rq = fin->live_status >= 0 ? SA_OK : SA_E_NONFINITE;
            fin->sweeps = fin->live_sweeps;
            if (rq == SA_OK && crc != SA_OK) rq = crc;
            if (rq == SA_OK) {
                sa_matrix a{fin->d_w, fin->wtype, fin->n, fin->ld};
                rq = finish_small(ctx, fin, &a, fin->d_uv, fin->d_uv + fin->n, s->sched.back());
            }
            cudaFreeAsync(fin->d_w, st);
            cudaFreeAsync(fin->d_uv, st);
            cudaStreamSynchronize(st);
            fin->d_w = nullptr;
            fin->d_uv = nullptr;
            if (ctx && ctx->ws.size > ((size_t)16 << 20)) sa::release_buffers(ctx);
            finish(s, fin, rq);
            continue;
        }
        // upload the group's matrices and make room for their potentials; one
        // synchronisation, then each request that made it is published
        sa::NvtxRange range("server: admit %zu small requests", adm.size());
        std::vector<sa_status> rcs(adm.size(), SA_OK);
        for (size_t q = 0; q < adm.size(); ++q) {
            Request* r = adm[q];
            rcs[q] = upload(r, st, &r->d_w, &r->ld);
            if (rcs[q] == SA_OK) {
                const cudaError_t e = srv_alloc((void**)&r->d_uv, 16 * (size_t)r->n, st);
                if (e != cudaSuccess) rcs[q] = sa::cuda_fail(e, "server: potentials");
            }
        }
        const cudaError_t se = cudaStreamSynchronize(st);   // the matrices are on the device
        std::vector<Request*> failed;
        for (size_t q = 0; q < adm.size(); ++q) {
            Request* r = adm[q];
            if (rcs[q] == SA_OK && se != cudaSuccess) rcs[q] = sa::cuda_fail(se, "server: upload");
            if (rcs[q] == SA_OK) continue;
            if (r->d_w) cudaFreeAsync(r->d_w, st);
            if (r->d_uv) cudaFreeAsync(r->d_uv, st);
            failed.push_back(r);
        }
        if (!failed.empty()) {
            cudaStreamSynchronize(st);
            for (Request* r : failed) {
                r->d_w = nullptr;
                r->d_uv = nullptr;
            }
        }
        bool stopped = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            L.reserved -= (unsigned)failed.size();
            for (size_t q = 0; q < adm.size(); ++q) {
                if (rcs[q] != SA_OK) continue;
                s->cv.wait(lk, [&] { return s->stop || L.slot[L.published % L.cap] == nullptr; });
                if (s->stop) {   // the requests' buffers are freed with the server
                    stopped = true;
                    break;
                }
                live_publish(s, adm[q]);
            }
        }
        for (size_t q = 0; q < adm.size(); ++q)
            if (rcs[q] != SA_OK) finish(s, adm[q], rcs[q]);
        if (stopped) break;
    }
    if (ctx) sa_destroy(ctx);
    cudaStreamDestroy(st);
}

constexpr int kMinLiveGrid = 8;

// Dispatcher of the queue: moves scaled requests to the workers, and starts a kernel of
// the queue when published requests are unclaimed and no kernel of the queue runs, or
// when they stay unclaimed for 0.2 ms while all running blocks are busy; a launch takes
// the SMs that the large requests leave.
void live_dispatcher(sa_server* s) {
    cudaSetDevice(s->device);
    LiveQueue& L = s->live;
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        if (s->stop) break;
        int nrun = 0, free_slot = -1;
        for (int k = 0; k < LiveQueue::kLaunchSlots; ++k) {
            if (L.running[k] && cudaEventQuery(L.ev[k]) != cudaErrorNotReady) {
                L.running[k] = false;
                s->sm_live -= L.sms_run[k];
                s->cv.notify_all();   // SMs for the large requests
            }
            if (L.running[k]) ++nrun;
            else if (free_slot < 0) free_slot = k;
        }
        if (L.inflight == 0) {
            // idle: a running kernel leaves within its idle time; its SMs are counted free
            // as soon as it has ended
            if (nrun == 0) s->cv.wait_for(lk, std::chrono::milliseconds(5));
            else s->cv.wait_for(lk, std::chrono::microseconds(200));
            continue;
        }
        // completions (after the kernel-end check: an ended kernel's flags are final)
        double oldest_unclaimed = -1;
        for (unsigned j = 0; j < L.cap && L.inflight > 0; ++j) {
            Request* r = L.slot[j];
            if (!r) continue;
            if (__atomic_load_n(L.done + j, __ATOMIC_ACQUIRE) == r->seq + 1) {
                r->live_sweeps = L.sweeps[j];
                r->live_status = L.status[j];
                r->t_scaled = s->now();
                L.slot[j] = nullptr;
                --L.inflight;
                --L.reserved;
                ++L.served;
                s->scaled.push_back(r);
                s->cv.notify_all();
            } else if (__atomic_load_n(L.claimed + j, __ATOMIC_ACQUIRE) != r->seq + 1) {
                if (oldest_unclaimed < 0 || r->t_pub < oldest_unclaimed) oldest_unclaimed = r->t_pub;
            }
        }
        // A launch takes SMs that no large request's cooperative grid holds (a block per SM,
        // as the block scheduler may place them): the first at most a quarter of the GPU,
        // so that large requests keep the rest; a second one (the first's blocks all busy,
        // requests waiting 0.2 ms) only while no large request runs or waits, up to its
        // slots of K.  The queue's blocks leave only when idle.
        bool large_pending = s->sm_large > 0;
        for (const Request* r : s->queue)
            if (r->n > kSmallMax) large_pending = true;
        const int cap = nrun == 0 ? L.sm_cap : L.grid;
        const int grid = std::min(std::min(L.grid, cap), s->num_sms - s->sm_live - s->sm_large);
        const bool start = oldest_unclaimed >= 0 && free_slot >= 0 && grid >= std::min(L.grid, kMinLiveGrid) &&
                           (nrun == 0 || (!large_pending && s->now() - oldest_unclaimed > 2e-4));
        if (start) {
            nvtxMarkA("server: request queue launch");
            sa::LiveArgs a = L.args;
            a.kscr = L.kbase + (size_t)free_slot * L.grid * sa::live_slot_floats();
            sa_status rc = sa::live_launch(a, grid, L.stream[free_slot]);
            if (rc == SA_OK && cudaEventRecord(L.ev[free_slot], L.stream[free_slot]) != cudaSuccess) rc = SA_E_CUDA;
            if (rc == SA_OK) {
                L.running[free_slot] = true;
                L.sms_run[free_slot] = grid;
                s->sm_live += L.sms_run[free_slot];
                ++L.launches;
            } else if (nrun == 0) {
                // no kernel will take them: fail what is unclaimed
                for (unsigned j = 0; j < L.cap; ++j) {
                    Request* r = L.slot[j];
                    if (!r || __atomic_load_n(L.claimed + j, __ATOMIC_ACQUIRE) == r->seq + 1) continue;
                    r->live_rc = rc;
                    L.slot[j] = nullptr;
                    --L.inflight;
                    --L.reserved;
                    s->scaled.push_back(r);
                }
                s->cv.notify_all();
            }
        }
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
    }
    // stop: every kernel of the queue leaves at its next poll
    __atomic_store_n(L.stop, 1u, __ATOMIC_RELEASE);
    lk.unlock();
    for (int k = 0; k < LiveQueue::kLaunchSlots; ++k)
        if (L.stream[k]) cudaStreamSynchronize(L.stream[k]);
}

// Device and host-mapped memory of the queue; the caller charges L.dev_bytes.
sa_status live_setup(sa_server* s, int grid, unsigned cap, uint64_t idle_ns) {
    LiveQueue& L = s->live;
    L.grid = grid;
    L.cap = cap;
    L.slot.assign(cap, nullptr);
    const size_t ring = sa::align_up(sizeof(sa::LiveDesc) * cap, 256);
    const size_t words = sa::align_up(4 * (size_t)cap, 256);
    const size_t host_bytes = 256 + ring + 4 * words;
    SA_CUDA(cudaHostAlloc((void**)&L.host, host_bytes, cudaHostAllocMapped));
    memset(L.host, 0, host_bytes);
    unsigned char* hdev = nullptr;
    SA_CUDA(cudaHostGetDevicePointer((void**)&hdev, L.host, 0));
    L.tail = (unsigned*)L.host;
    L.stop = (unsigned*)(L.host + 128);
    L.desc = (sa::LiveDesc*)(L.host + 256);
    L.claimed = (unsigned*)(L.host + 256 + ring);
    L.done = (unsigned*)(L.host + 256 + ring + words);
    L.sweeps = (int32_t*)(L.host + 256 + ring + 2 * words);
    L.status = (int32_t*)(L.host + 256 + ring + 3 * words);
    const size_t kslot_bytes = sa::live_slot_floats() * sizeof(float);
    const size_t sched = sa::align_up(8 * s->sched.size(), 256);
    L.dev_bytes = 256 + sched + (size_t)LiveQueue::kLaunchSlots * grid * kslot_bytes;
    SA_CUDA(cudaMalloc(&L.dev, L.dev_bytes));
    SA_CUDA(cudaMemset(L.dev, 0, 256));
    unsigned char* d = (unsigned char*)L.dev;
    SA_CUDA(cudaMemcpy(d + 256, s->sched.data(), 8 * s->sched.size(), cudaMemcpyHostToDevice));
    L.kbase = (float*)(d + 256 + sched);
    sa::LiveArgs& a = L.args;
    a.desc = (const sa::LiveDesc*)(hdev + 256);
    a.tail = (const unsigned*)hdev;
    a.stop = (const unsigned*)(hdev + 128);
    a.claimed = (unsigned*)(hdev + 256 + ring);
    a.done = (unsigned*)(hdev + 256 + ring + words);
    a.sweeps = (int32_t*)(hdev + 256 + ring + 2 * words);
    a.status = (int32_t*)(hdev + 256 + ring + 3 * words);
    a.head = (unsigned*)d;
    a.busy = (unsigned*)(d + 128);
    a.cap = cap;
    a.P = (const double*)(d + 256);
    a.n_p = (int)s->sched.size();
    a.tol = s->opts.tol;
    a.max_sweeps = s->opts.max_sweeps_per_p;
    a.kscr = nullptr;   // per launch slot
    a.kscr_floats = sa::live_slot_floats();
    a.idle_ns = idle_ns;
    for (int k = 0; k < LiveQueue::kLaunchSlots; ++k) {
        SA_CUDA(cudaStreamCreateWithFlags(&L.stream[k], cudaStreamNonBlocking));
        SA_CUDA(cudaEventCreateWithFlags(&L.ev[k], cudaEventDisableTiming));
    }
    return SA_OK;
}

void live_teardown(LiveQueue& L) {
    for (int k = 0; k < LiveQueue::kLaunchSlots; ++k) {
        if (L.stream[k]) cudaStreamSynchronize(L.stream[k]);
        if (L.ev[k]) cudaEventDestroy(L.ev[k]);
        if (L.stream[k]) cudaStreamDestroy(L.stream[k]);
        L.ev[k] = nullptr;
        L.stream[k] = nullptr;
    }
    if (L.dev) cudaFree(L.dev);
    if (L.host) cudaFreeHost(L.host);
    L.dev = nullptr;
    L.host = nullptr;
}

constexpr int kMinLargeGrid = 8;

// The grid a large request's scaling kernel may take now (lock held): at most its share of
// the GPU, and only SMs that the request queue's blocks and the other large requests'
// grids leave; while small requests wait and no kernel of the queue runs, the SMs of one
// launch of the queue are kept free for it.
int large_grid_now(const sa_server* s) {
    const LiveQueue& L = s->live;
    bool small_waiting = L.inflight > 0;
    for (const Request* r : s->queue)
        if (r->n <= kSmallMax) small_waiting = true;
    const int keep = small_waiting && s->sm_live == 0 ? std::min(L.grid, L.sm_cap) : 0;
    return std::min(s->large_grid, s->num_sms - s->sm_live - s->sm_large - keep);
}

void large_worker(sa_server* s) {
    cudaSetDevice(s->device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    sa_ctx* ctx = nullptr;
    const sa_status crc = sa_create(&ctx, s->device, st);   // failing: as in small_worker
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
            // the scaling kernel's grid: SMs that neither the request queue nor the other
            // large requests hold (its blocks must all be resident at once)
            int grid = 0;
            {
                std::unique_lock<std::mutex> lk(s->mu);
                s->cv.wait(lk, [&] { return s->stop || large_grid_now(s) >= kMinLargeGrid; });
                if (!s->stop) {
                    grid = large_grid_now(s);
                    s->sm_large += grid;
                }
            }
            if (grid == 0) {
                rc = SA_E_INVALID;
                sa::set_error("server stopped");
            } else {
                sa::NvtxRange range("server: assign request %llu n=%d grid=%d", (unsigned long long)r->ticket, r->n, grid);
                ctx->max_grid = grid;
                sa_matrix a{dw, r->wtype, r->n, ld};
                r->perm.assign(r->n, -1);
                sa_assign_result res{};
                res.perm = r->perm.data();
                rc = sa_assign(ctx, &a, &s->opts, 0.0, &res);
                r->sum_log_w = res.sum_log_w;
                r->gamma = res.gamma;
                r->sweeps = res.scale.sweeps_total;
                std::lock_guard<std::mutex> g(s->mu);
                s->sm_large -= grid;
                s->cv.notify_all();
            }
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
    // a launch of the request queue takes up to a block per SM (a quarter of them while
    // large requests run); its slots of K (1 MiB a block, two launch slots) take at most
    // an eighth of the budget
    const int live_grid = (int)std::max<size_t>(4, std::min<size_t>(s->num_sms, hbm_budget / ((size_t)16 << 20)));
    s->live.sm_cap = std::max(1, s->num_sms / 4);
    s->large_grid = std::max(kMinLargeGrid, s->num_sms / large);
    if (cudaSetDevice(device) != cudaSuccess) {
        delete s;
        sa::set_error("cudaSetDevice(%d) failed", device);
        return SA_E_CUDA;
    }
    const sa_status lrc = live_setup(s, live_grid, 1024u, 2000000ull);
    if (lrc != SA_OK) {
        live_teardown(s->live);
        delete s;
        return lrc;
    }
    if (s->live.dev_bytes >= s->budget) {
        sa::set_error("the budget (%zu bytes) does not cover the request queue's %zu bytes", s->budget,
                      s->live.dev_bytes);
        live_teardown(s->live);
        delete s;
        return SA_E_BUDGET;
    }
    s->used = s->live.dev_bytes;
    s->dispatcher = std::thread(live_dispatcher, s);
    for (int q = 0; q < kSmallWorkers; ++q) s->workers.emplace_back(small_worker, s);
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
    if (s->dispatcher.joinable()) s->dispatcher.join();
    live_teardown(s->live);
    // device buffers of small requests that were still queued, in flight or unfinished
    for (auto& kv : s->all) {
        if (kv.second->d_w) cudaFree(kv.second->d_w);
        if (kv.second->d_uv) cudaFree(kv.second->d_uv);
    }
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
    out->t_scaled = r->t_scaled;
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

sa_status sa_server_get_stats(sa_server* s, sa_server_stats* out) {
    if (!s || !out) {
        sa::set_error("bad stats arguments");
        return SA_E_INVALID;
    }
    std::lock_guard<std::mutex> g(s->mu);
    out->live_launches = s->live.launches;
    out->live_requests = s->live.served;
    out->live_blocks = s->live.grid;
    out->live_capacity = (int32_t)s->live.cap;
    out->large_grid = s->large_grid;
    out->live_slots = LiveQueue::kLaunchSlots;
    out->live_device_bytes = (int64_t)s->live.dev_bytes;
    return SA_OK;
}

}  // extern "C"
