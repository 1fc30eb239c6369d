// sa_internal.h -- host-side internals of libsa shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/sa.h"

namespace sa {

// Device-side error codes written to an int flag by kernels (0 = none).
enum : int {
    kErrNone = 0,
    kErrTimeout = 1,     // a bounded wait gave up
    kErrNonfinite = 2,   // a row or column sum was zero / not finite
    kErrLaunch = 3,
};

constexpr double kLn2 = 0.69314718055994530942;
constexpr double kLog2e = 1.44269504088896340736;
constexpr uint64_t kWaitTimeoutNs = 2000000000ull;  // 2 s per device wait

void set_error(const char* fmt, ...);

// An NVTX range over a scope (host side: API calls, p steps of host-driven loops, server
// request phases).  Without a tool attached the NVTX calls return at once.
struct NvtxRange {
    explicit NvtxRange(const char* fmt, ...) {
        char buf[96];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Process-wide count of kernels this library has launched (sa_kernel_launches).
extern std::atomic<long long> g_kernel_launches;
inline void count_launch(int k = 1) { g_kernel_launches.fetch_add(k, std::memory_order_relaxed); }
sa_status cuda_fail(cudaError_t e, const char* what);

#define SA_CUDA(call)                                              \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::sa::cuda_fail(_e, #call);  \
    } while (0)

// Growable device workspace carved into named regions per call.
struct Workspace {
    void* ptr = nullptr;
    size_t size = 0;
    sa_status reserve(size_t bytes);
    void release();          // give the memory back to the device
    ~Workspace();
};

struct PinnedBuf {
    void* ptr = nullptr;
    size_t size = 0;
    sa_status reserve(size_t bytes);
    ~PinnedBuf();
};

// sa_batch_scale's plan when none is set (see sa_set_batch_plan)
inline sa_batch_plan default_batch_plan() {
    sa_batch_plan p{};
    p.count = 5;
    const int n_hi[5] = {32, 64, 128, 256, 512};
    const int path[5] = {SA_BATCH_REGS, SA_BATCH_REGS, SA_BATCH_REGS, SA_BATCH_KROWS, SA_BATCH_KROWS};
    const int warps[5] = {1, 4, 16, 0, 0}, per_block[5] = {2, 1, 1, 0, 0};
    for (int b = 0; b < 5; ++b) {
        p.n_hi[b] = n_hi[b];
        p.path[b] = path[b];
        p.warps[b] = warps[b];
        p.per_block[b] = per_block[b];
    }
    return p;
}

}  // namespace sa

struct sa_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 0;
    size_t smem_optin = 0;
    // options (sa_set_option)
    int max_grid = 0;        // cap on the persistent kernels' grid (0: all SMs)
    int fused_nt = 512;      // threads per block of the fused kernel when 512 < chunks <= 1024
    int step_sparse = 0;     // step kernel: allow sparse epochs
    int solve_gpu = 0;       // sa_assign: large reduced instances through the GPU path
    uint64_t wait_ns = sa::kWaitTimeoutNs;   // step kernel: limit of its barrier and ring waits
    size_t step_l2_bytes = (size_t)48 << 20;  // step kernel: bytes of K read with the default L2
                                              // policy (the rest "evict first")
    int test_unreachable_barrier = 0;         // testing hook (SA_OPT_TEST_UNREACHABLE_BARRIER)
    sa_batch_plan batch_plan = sa::default_batch_plan();
    cudaStream_t batch_streams[SA_BATCH_MAX_BUCKETS] = {};   // one per bucket launch (lazily made)
    cudaEvent_t batch_events[SA_BATCH_MAX_BUCKETS + 1] = {};
    sa::Workspace ws;        // scratch for sweeps, prune, certify
    sa::Workspace input;     // device copy of host inputs (sa_assign_host)
    sa::Workspace keep;      // sa_scale: the caller's warm-start potentials, restored on failure
    sa::PinnedBuf pinned;    // staging for small device->host results
};

namespace sa {

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Sets a kernel's dynamic shared-memory limit to the most it can take next to its static
// shared memory (optin: the device's per-block opt-in maximum).  Setting the size of each
// call instead would race between host threads that launch the same kernel with different
// sizes (one thread's smaller limit failing the other's occupancy query or launch).
template <typename Kern>
inline cudaError_t allow_dynamic_smem(Kern kern, size_t optin) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kern);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(optin - fa.sharedSizeBytes));
}
inline int wbytes(sa_wtype t) { return t == SA_I16 ? 2 : 4; }

// Bump allocator over a reserved workspace.
struct Carve {
    char* base;
    size_t off = 0;
    explicit Carve(void* p) : base((char*)p) {}
    template <typename T>
    T* take(size_t count) {
        off = align_up(off, 256);
        T* r = (T*)(base + off);
        off += count * sizeof(T);
        return r;
    }
};

// ---- sweeps (sweep_plain.cu, sweep_fused.cu) ------------------------------------------
// Potentials inside the library are FP64 in log2 units: U = u / ln 2, V = v / ln 2.
struct ScaleState {
    double* U;   // n
    double* V;   // n
};
sa_status scale_plain(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U,
                      double* V, sa_scale_info* info);
sa_status scale_fused(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U,
                      double* V, sa_scale_info* info);
sa_status scale_fp64(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U,
                     double* V, sa_scale_info* info);
bool fused_supported(const sa_ctx* ctx, const sa_matrix* a);
// sweep_step.cu: the per-step FP32 matrix path (SA_KERNEL_STEP)
sa_status scale_step(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U,
                     double* V, sa_scale_info* info);
bool step_supported(const sa_ctx* ctx, const sa_matrix* a);
size_t fused_workspace_bytes(const sa_ctx* ctx, const sa_matrix* a);
// newton.cu: Newton scaling of Sec. 5.3 on the per-step matrix (SA_KERNEL_NEWTON)
sa_status scale_newton(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U,
                       double* V, sa_scale_info* info);
bool newton_supported(const sa_ctx* ctx, const sa_matrix* a);

// natural <-> log2 units, in place on the device (n doubles), y = x * f
void launch_scale_vec(double* x, int n, double f, cudaStream_t s);
// Vh = float(V), Vc = 2^(Vh - V)
void launch_split_v(const double* V, float* Vh, float* Vc, int n, cudaStream_t s);

// ---- prune / certify / verify (prune.cu) --------------------------------------------
sa_status prune_device(sa_ctx* ctx, const sa_matrix* a, double p, const double* d_u,
                       const double* d_v, double t, int guard, sa_csr* out, double* log_ub);
sa_status certify_device(sa_ctx* ctx, const sa_matrix* a, const double* alpha,
                         const double* beta, double tau, int64_t* n_viol, int64_t max_add,
                         sa_csr* add);
sa_status verify_device(sa_ctx* ctx, const sa_matrix* a, double p, const double* d_u,
                        const double* d_v, double* d_rows, double* d_cols, double* max_row_err,
                        double* max_col_err);

// smallest positive and largest weight (prune.cu)
sa_status weights_minmax(sa_ctx* ctx, const sa_matrix* a, int64_t* wmin, int64_t* wmax);

sa_status narrow_device(sa_ctx* ctx, const int32_t* src, int64_t lds, int16_t* dst, int64_t ldd,
                        int n, int64_t* n_bad);

// ---- host exact solver (solve.cpp) ----------------------------------------------------
// Max sum of logw over perfect matchings of a CSR bipartite graph (rows -> cols).
// price0 (may be null): starting column prices of the minimisation form (-beta_j).
// Returns SA_OK / SA_E_NO_PERFECT_MATCHING.
// State handed to a replacement of the shortest-augmenting-path phase (ssp.cu): column
// prices v (minimisation form), the matching and the cost -log w of each row's assigned
// entry; every assigned row sits on a least-reduced-cost column.  The replacement assigns
// the free rows and keeps that invariant.
struct SspState {
    int n;
    const int64_t* row_ptr;
    const int32_t* col;
    const double* logw;
    double* v;
    int32_t* rmatch;
    int32_t* cmatch;
    double* mcost;
};
typedef sa_status (*SspFn)(void* user, SspState& st);
sa_status sparse_assign(int n, const int64_t* row_ptr, const int32_t* col, const double* logw,
                        int32_t* perm, double* alpha, double* beta, const double* price0 = nullptr,
                        SspFn ssp = nullptr, void* ssp_user = nullptr);
// of the LP-optimal duals of B for perm, the largest beta <= beta0 (alpha, beta in and out)
sa_status project_duals(int n, const int64_t* row_ptr, const int32_t* col, const double* logw,
                        const int32_t* perm, const double* beta0, double* alpha, double* beta);
// ssp.cu: the shortest-augmenting-path phase on the GPU (user = SspRun*)
struct SspRun {
    sa_ctx* ctx;
    int64_t searches = 0;        // shortest-path searches run on the GPU
    int64_t rounds = 0;          // label-correcting rounds and tree levels launched, in all
};
sa_status ssp_device(void* user, SspState& st);

// auction.cu: eps-scaling forward auction on a device CSR (prices >= 0 in and out)
sa_status auction_device(sa_ctx* ctx, int n, const int64_t* d_rp, const int32_t* d_col, const double* d_val,
                         double eps0, double eps_final, int64_t max_rounds, double* d_price, int* d_assigned,
                         int* phases, int64_t* rounds, int* complete);

// serve_live.cu: the server's device-resident queue of small requests (n <= 512).
// Ring entry of one request, in host-mapped memory.
struct LiveDesc {
    const void* w;     // device matrix, n x ld elements
    double* u;         // device FP64[n] outputs (natural units)
    double* v;
    int64_t ld;
    int32_t n;
    int32_t i16;       // weights are int16 (else int32)
};
struct LiveArgs {
    const LiveDesc* desc;   // host-mapped [cap]
    const unsigned* tail;   // host-mapped: requests published
    const unsigned* stop;   // host-mapped: nonzero ends the kernel
    unsigned* claimed;      // host-mapped [cap]: q + 1 once request q is claimed
    unsigned* done;         // host-mapped [cap]: q + 1 once request q is scaled
    int32_t* sweeps;        // host-mapped [cap]
    int32_t* status;        // host-mapped [cap]: 0 ok, 1 a step hit its cap, -6 non-finite
    unsigned* head;         // device: requests claimed
    unsigned* busy;         // device: blocks scaling a request
    unsigned cap;
    const double* P;        // device schedule
    int n_p;
    double tol;
    int max_sweeps;
    float* kscr;            // device: a slot of K per block
    size_t kscr_floats;     // floats per slot (live_slot_floats())
    uint64_t idle_ns;       // a block leaves after this long without a request
};
size_t live_slot_floats();
sa_status live_launch(const LiveArgs& args, int grid, cudaStream_t st);

// csr helpers (api.cu)
sa_status csr_alloc(sa_csr* c, int n, int64_t nnz);

// Upper bound of the device memory sa_assign allocates for an n x n matrix besides the
// matrix itself, on a device of num_sms SMs: the largest scaling workspace (the per-step
// matrix K of the STEP and NEWTON kernels and the STEP kernel's log2 w pairs, 12 n
// ceil(n/4)*4 bytes; column partials of up to two blocks per SM), the prune's device CSR
// arrays (8 bytes per kept entry, at most
// n^2 when the re-prune reaches t = 0), the potentials and the certificate's buffers.
size_t assign_device_bound(int num_sms, int n);
// Give a context's device buffers (workspace, input copy, warm-start copy) back to the
// device; they are allocated again by the next call that needs them.
void release_buffers(sa_ctx* ctx);

}  // namespace sa
