// sweep_step.cu -- fused Sinkhorn sweep over a per-step FP32 matrix (Sec. 4.1.2 log-domain
// iteration, Sec. 4.2 stopping rule, deformed warm start between p steps as in Sec. 4.1).
//
// At the start of every p step each block evaluates, for its own row stripe,
//     K_ij = 2^(p log2 w_ij - C_i - V_j)        (C_i ~ max_j (p log2 w_ij - V_j))
// once, with the exponent formed in float-pair arithmetic (log2 w to about 2^-40 from a
// 256-entry shared table and a series; exact two-product and two-sums), one SFU exp2, and
// stores K as FP32 in a global workspace.  K is the iterate X(p) at the step start, so every entry is
// in [0, ~1] and its relative error (about 2e-7) does not grow with p.  The launch's first
// evaluation also stores log2 w as a float pair (two FP32 planes); the later ones read the
// pairs (8 bytes per entry, no table lookups or series) and are bound by memory, not by
// the arithmetic of the logarithm.  Within the step
// the potentials move only through a column factor c_j = 2^(Vs_j - V_j) (Vs = V at the
// step start) and the fresh row sums, so a sweep is
//     s_i  = sum_j K_ij c_j,     S_j = c_j sum_i K_ij / s_i,     V_j += log2 S_j
// and U_i = C_i + log2 s_i.  No logarithm or exponential is evaluated per entry and sweep.
//
// Work split, ring and barriers follow the single-read sweep: block b owns the row stripe
// [b n/G, (b+1) n/G) and finalises the same index range of columns; each thread owns fixed
// 16-byte chunks (4 columns) of every row, keeping its column partial sums in registers;
// rows stream through a shared-memory ring by bulk copies (cp.async.bulk + mbarrier).
// Because K stays in the ring slot until the row sum is known, the second use of a row
// (the column accumulation) re-reads the slot: no stash of terms is needed.  The warp
// whose release completes a slot's count refills it with the row RING positions ahead.
//
// Every wait is bounded (2 s); on expiry the kernel records kErrTimeout, waits for its
// outstanding copies (bounded) and returns.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "common.cuh"
#include "log2pair.cuh"
#include "sa_internal.h"

#ifndef SA_STEP_STAMP
#define SA_STEP_STAMP(slot)   // phase timing hook (no-op in the library build)
#endif

namespace sa {

namespace {

constexpr int kStepNred = 4;      // row-sum publication buffers
constexpr int kStepMaxRps = 4;    // rows per ring stage at most
constexpr int kStepMaxRing = 16;  // ring slots at most; a slot holds one stage
// rows per ring stage of the dense ring mode.  A stage costs a fixed ~0.5 us (the
// publication of the warps' partial row sums and the slot's release) plus ~0.4 us per row
// at n = 8192, so two-row stages beat one-row stages (34.7 against 47.7 us per row pass)
// although a one-row ring keeps twice the rows in flight.  Where at most three two-row
// stages fit and two three-row stages do (rows of 27 to 35 KB), three-row stages are taken:
// at n = 8192 45.5 against 48.0 us per sweep (row pass 33.7 against 37.1 us), although the
// two-stage ring consumes each stage before forming the next one's partials.
constexpr int kDenseRowsPerStage = 2;
constexpr int kWideRowsPerStage = 3;

struct StepArgs {
    const void* w;
    int n;
    int64_t ld;            // elements
    int i16;               // weights are int16 (else int32)
    float* K;              // n x ldk, FP32
    float* Lh;             // n x ldk: log2 w as a float pair (head, tail; -inf head: w = 0),
    float* Ll;             //   written by the launch's first evaluation of K, read by the others
    int64_t ldk;           // floats, multiple of 4
    unsigned row_bytes;    // bytes copied per K row (multiple of 16)
    int ring;              // ring slots of a dense epoch (>= 4)
    unsigned region_bytes; // shared-memory region for the ring (and sparse c, S)
    uint2* rec;            // (column, value bits) records of K >= theta, rec_cap_row per row
    int64_t rec_cap_row;   // record capacity per row (even)
    unsigned long long* stats;   // [2][4]: records, longest row, overflow (per epoch parity)
    unsigned* crange;      // [2][2]: max and min column factor of a sweep (float bits)
    int* counters;         // [2]: sparse epochs, re-anchors
    int sparse_ok;         // build records and allow sparse epochs
    unsigned sparse_row_cap;            // longest stage (records of two rows) a sparse ring holds
    unsigned long long sparse_max_total; // most records for a sparse epoch
    float theta;           // entries of K below theta are dropped in sparse epochs
    float reanchor_ratio;  // re-evaluate K when max c / min c exceeds this
    const double* P;       // schedule
    int k0, n_p;
    double tol;
    int max_sweeps;
    int keep_v;
    double* U;             // n, log2 units
    double* V;             // n, log2 units
    double* Vs;            // n, V at the step start
    float* Cf;             // n, 2^(Vs - V)
    float* part;           // G x npad column partials
    int npad;
    float* rmax;           // 2 alternating residual words
    unsigned* bar;         // grid barrier counter
    int* err;
    int* sweeps_out;       // n_p
    double* resid_out;     // n_p
    int max_rows;
    uint64_t wait_ns;      // limit of the grid barriers' and the sweeps' ring waits (the
                           // waits for copies in flight before an exit keep kWaitTimeoutNs)
    int l2_keep_stages;    // stages of each stripe read with the default L2 policy; the
                           // others are read "evict first", so the kept ones stay in L2
    unsigned extra_arrivals;   // testing hook: arrivals the first grid barrier waits for
                               // beyond the grid (nothing provides them: it runs out)
};


__device__ __forceinline__ void load_w4(const StepArgs& A, int64_t row, int j, int cnt, int w[4]) {
    if (A.i16) {
        const int16_t* p = (const int16_t*)A.w + row * A.ld + j;
        if (cnt == 4) {
            const uint2 q = *(const uint2*)p;
            w[0] = (int16_t)(q.x & 0xffffu);
            w[1] = (int16_t)(q.x >> 16);
            w[2] = (int16_t)(q.y & 0xffffu);
            w[3] = (int16_t)(q.y >> 16);
        } else {
            for (int e = 0; e < 4; ++e) w[e] = e < cnt ? p[e] : 0;
        }
    } else {
        const int32_t* p = (const int32_t*)A.w + row * A.ld + j;
        if (cnt == 4) {
            const int4 q = *(const int4*)p;
            w[0] = q.x;
            w[1] = q.y;
            w[2] = q.z;
            w[3] = q.w;
        } else {
            for (int e = 0; e < 4; ++e) w[e] = e < cnt ? p[e] : 0;
        }
    }
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(p)), "r"(v) : "memory");
    return old;
}

// orders this thread's generic-proxy accesses (global and shared) before later bulk copies
__device__ __forceinline__ void fence_proxy_async_all() {
    asm volatile("fence.proxy.async;" ::: "memory");
}

// Grid barrier: thread 0 arrives with a release reduction (the block's writes, ordered
// before it by the block barrier, become visible with the arrival) and polls the counter
// with acquire loads.  The error word is read while polling, not after a completed wait:
// a block that fails sets it and leaves before its next arrival, so the others see it
// while they wait at that barrier (within 32 polls) and leave in turn.
__device__ __forceinline__ bool step_grid_sync(unsigned* ctr, unsigned target, int* err, int* s_ok,
                                               uint64_t wait_ns) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(ctr), "r"(1u) : "memory");
        if (ld_acquire(ctr) < target) {
            const uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (ld_acquire(ctr) < target) {
                if ((++spins & 31u) == 0) {
                    if (*(volatile int*)err != 0) { ok = 0; break; }
                    if (globaltimer_ns() - t0 > wait_ns) { atomicCAS(err, 0, kErrTimeout); ok = 0; break; }
                }
                __nanosleep(32);
            }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

struct KahanS {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// SP: sparse epochs possible.  RPS: rows per ring stage (three for rows of 27 to 35 KB, one
// for rows of more than 48 KB; two or three slots then).
template <int NT, int CH, bool SP, int RPS>
__global__ void __launch_bounds__(NT, 1) step_kernel(StepArgs A) {
    constexpr int NW = NT / 32;
    constexpr int M = CH * 4;   // columns owned per thread (dense mode)
    constexpr int NRED = kStepNred;
    constexpr int MAXR = kStepMaxRing;
    constexpr int FG = NT / 64;
    static_assert(NT % 64 == 0, "layout");
    static_assert(RPS >= 1 && RPS <= kStepMaxRps, "rows per stage");
    static_assert(!SP || RPS == 2, "sparse records come in stages of two rows");
    extern __shared__ __align__(128) unsigned char smem[];
    // [region: dense ring | or sparse c, S and ring] [barriers] [scratch]
    unsigned char* region = smem;
    uint64_t* mbar = (uint64_t*)(smem + A.region_bytes);   // [MAXR] copy arrivals
    uint64_t* mrow = mbar + MAXR;                           // [NRED] row-sum publication
    unsigned* rel_cnt = (unsigned*)(mrow + NRED);           // [MAXR] warp releases per slot
    unsigned* iss_cnt = rel_cnt + MAXR;                     // [MAXR] copies issued per slot
    // 8 (MAXR + NRED) + 8 MAXR bytes of barriers and counters end on a 16-byte boundary
    float* red = (float*)(iss_cnt + MAXR);                  // [NRED][RPS][NW] (16-aligned)
    double* crow = (double*)(red + NRED * kStepMaxRps * NW);   // [max_rows] row references
    double* redp = crow + A.max_rows;                       // [FG][64]
    double* redd = redp + FG * 64;                          // [NW]
    float* srow = (float*)(redd + NW);                      // [max_rows] row sums
    unsigned* rowoff = (unsigned*)(srow + A.max_rows);      // [max_rows] record offsets
    unsigned* rowlen = rowoff + A.max_rows;                 // [max_rows] padded record counts
    __shared__ int s_flag, s_ok, s_mode, s_reanchor;
    __shared__ float4 s_l2tab[256];
    __shared__ float s_res;
    __shared__ unsigned s_maxlen;   // longest stage (records of two rows) of this stripe

    const int n = A.n;
    const int G = gridDim.x;
    const int b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int r0 = (int)((int64_t)b * n / G);
    const int r1 = (int)((int64_t)(b + 1) * n / G);
    const int nrows = r1 - r0;
    const int c0 = r0, c1 = r1;
    const int NC = (n + 3) / 4;
    const unsigned char* kbase = (const unsigned char*)A.K;
    const size_t kpitch = (size_t)A.ldk * sizeof(float);
    uint2* recb = A.rec + (size_t)r0 * A.rec_cap_row;        // this block's records
    const size_t rec_cap = (size_t)nrows * A.rec_cap_row;
    const size_t cs_bytes = ((size_t)n * 8 + 15) & ~(size_t)15;   // sparse: c and S
    float* c_s = (float*)region;
    float* S_s = c_s + n;

    for (int j = tid; j < 256; j += NT) s_l2tab[j] = log2_tab_entry(j);
    if (tid == 0) {
        for (int s = 0; s < MAXR; ++s) rel_cnt[s] = iss_cnt[s] = 0u;
        for (int s = 0; s < NRED; ++s) mbar_init(&mrow[s], NW);
        mbar_fence_init();
        s_flag = 0;
    }
    __syncthreads();

    // ring geometry of the current epoch (one evaluation of K and the sweeps that use it)
    int sparse = 0;
    int ring_n = 4;
    unsigned slot_bytes = A.row_bytes;
    unsigned char* sbase = region;
    uint32_t its = 0;     // ring index of the current sweep's first stage (per epoch)
    uint32_t gbase = 0;   // row stages completed, over the whole launch
    unsigned nbar = 0;
    int rphase = 0;
    unsigned epoch = 0;
    // The ring holds stages (local rows 2g and 2g+1, contiguous in global memory: K rows, or
    // the records of the two rows) in fixed slots: ring index v is stage v % nst of its sweep,
    // in slot v % ring_n.  The warp whose release completes a slot's count refills it with
    // ring index v + ring_n: no thread waits to issue a copy.
    const int nst = (nrows + RPS - 1) / RPS;
    // Stage read at ring index v: the sweeps of an epoch alternate direction over the stripe,
    // so the rows a sweep reads last -- the ones most likely still in L2 (K is about twice
    // the L2 at n = 8192) -- are the rows the next sweep reads first.  The first sweep of an
    // epoch runs backwards: the evaluation of K wrote the stripe forwards.
    auto stage_of = [&](uint32_t v) -> int {
        const int g = (int)(v % (uint32_t)nst);
        return ((v / (uint32_t)nst) & 1u) ? g : nst - 1 - g;
    };
    auto issue_index = [&](uint32_t v) {   // one thread
        const uint32_t slot = v % (uint32_t)ring_n;
        const int stg = stage_of(v);
        const int q0 = RPS * stg;
        const int nr = min(RPS, nrows - q0);
        const void* src;
        unsigned bytes;
        if (SP && sparse) {
            src = recb + rowoff[q0];
            bytes = (rowlen[q0] + (nr > 1 ? rowlen[q0 + 1] : 0u)) * 8u;
        } else {
            src = kbase + (size_t)(r0 + q0) * kpitch;
            bytes = (unsigned)nr * A.row_bytes;
        }
        iss_cnt[slot] += 1;
        mbar_arrive_expect_tx(&mbar[slot], bytes);
        // K is larger than L2: the first l2_keep_stages stages of every stripe keep the
        // default policy and stay resident from sweep to sweep, the rest stream through
        if ((SP && sparse) || stg < A.l2_keep_stages)
            bulk_g2s(sbase + (size_t)slot * slot_bytes, src, bytes, &mbar[slot]);
        else
            bulk_g2s_hint(sbase + (size_t)slot * slot_bytes, src, bytes, &mbar[slot], l2_policy_evict_first());
    };
    auto release_index = [&](uint32_t v) {   // lane 0 after __syncwarp
        const uint32_t slot = v % (uint32_t)ring_n;
        const unsigned old = atom_add_acq_rel(&rel_cnt[slot], 1u);
        if ((old + 1u) % (unsigned)NW == 0u) {
            fence_proxy_async_smem();
            issue_index(v + (uint32_t)ring_n);
        }
    };
    auto wait_copies = [&]() {   // tid 0: the last copy issued into every slot
        for (int s = 0; s < MAXR; ++s) {
            const unsigned k = iss_cnt[s];
            if (k > 0u && !mbar_wait(&mbar[s], (k - 1u) & 1u, A.err, kWaitTimeoutNs)) break;
        }
    };
    auto drain = [&]() {
        __syncthreads();
        if (tid == 0) wait_copies();
        __syncthreads();
    };
    auto gsync = [&]() -> bool {
        ++nbar;
        return step_grid_sync(A.bar, nbar * (unsigned)G + A.extra_arrivals, A.err, &s_ok, A.wait_ns);
    };

    int cidx[CH];
    int nval[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        cidx[k] = tid + k * NT;
        nval[k] = cidx[k] < NC ? min(4, n - cidx[k] * 4) : 0;
    }
    float S[M], cf[M];

    // ---- one evaluation of this stripe's rows of K for p (V: the epoch's starting column
    //      potentials), dense rows in global memory plus, when enabled, the entries
    //      >= theta as (column, value) records ----
    // cscale > 0: the row references come from the previous step's row potentials,
    // C_i = cscale U_i (cscale = p_k / p_{k-1}): with (u, v) scaled by that ratio, C_i lies
    // within cscale log2 n above max_j (p log2 w_ij - V_j), so every entry of K stays in
    // [2^-(cscale log2 n + the range of the row), 1] and no per-row maximum pass is needed.
    // cscale = 0: the references are the FP32 row maxima (a cold start, a kept v, a
    // re-evaluation within a step).
    // FRESH (the launch's first evaluation): log2 w of every entry is formed from the
    // weights and stored as a float pair in Lh, Ll; later evaluations read the pairs back.
    auto prep = [&](double p, double cscale, auto fresh) {
        constexpr bool FRESH = decltype(fresh)::value;
        const float pf = (float)p;
        // the region is idle: stage V there as the FP32 head and tail of each entry, in two
        // arrays, so that a thread reads its four columns with one 16-byte load from each
        float* vhi = (float*)region;
        float* vlo = vhi + NC * 4;
        for (int j = tid; j < NC * 4; j += NT) {
            const double vj = j < n ? A.V[j] : 0.0;
            const float hi = (float)vj;
            vhi[j] = hi;
            vlo[j] = (float)(vj - (double)hi);
        }
        // p = ph + pl (pl = 0 for any p with at most 24 significant bits)
        const float ph = (float)p;
        const float pl = (float)(p - (double)ph);
        if (tid == 0) s_maxlen = 0u;
        __syncthreads();
        unsigned* wcnt = (unsigned*)red;   // [NW] per-warp kept counts (scratch)
        size_t roff = 0;                   // records written so far (block-relative)
        bool overflow = false;
        // the weights of row q + 1 are loaded while row q is evaluated (up to eight chunks a
        // thread: wider rows would spill the second set of registers)
        constexpr bool PREF = FRESH && CH <= 8;
        int wv[FRESH ? M : 1], wn[PREF ? M : 1];
        auto load_row = [&](int q, int* dst) {
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                int w4[4] = {0, 0, 0, 0};
                if (q < nrows && nval[k] > 0) load_w4(A, r0 + q, cidx[k] * 4, nval[k], w4);
#pragma unroll
                for (int e = 0; e < 4; ++e) dst[4 * k + e] = w4[e];
            }
        };
        if (PREF) load_row(0, wn);
        for (int q = 0; q < nrows; ++q) {
            const int64_t row = r0 + q;
            // the row's log2 pairs, every chunk's loads issued before the first is used (the
            // stores of K below could alias them for the compiler, which then keeps the
            // loads behind the stores)
            float4 lh4[FRESH ? 1 : CH], ll4[FRESH ? 1 : CH];
            if constexpr (!FRESH) {
                const float* lhr = A.Lh + row * A.ldk;
                const float* llr = A.Ll + row * A.ldk;
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                    lh4[k] = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
                    ll4[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (nval[k] > 0) {
                        lh4[k] = __ldcs((const float4*)(lhr + cidx[k] * 4));
                        ll4[k] = __ldcs((const float4*)(llr + cidx[k] * 4));
                    }
                }
            }
            if (PREF) {
#pragma unroll
                for (int x = 0; x < M; ++x) wv[x] = wn[PREF ? x : 0];
                load_row(q + 1, wn);
            } else if (FRESH) {
                load_row(q, wv);
            }
            double cref;
            if (cscale > 0.0) {
                cref = A.U[row] * cscale;
            } else {
                // reference C ~ max_j (p log2 w - V_j), an FP32 estimate (only a scale; C itself
                // enters the row potential exactly)
                float mloc = -INFINITY;
#pragma unroll
                for (int k = 0; k < CH; ++k) {
                    if (nval[k] == 0) continue;
                    const float4 vh4 = *(const float4*)(vhi + cidx[k] * 4);
                    const float vh[4] = {vh4.x, vh4.y, vh4.z, vh4.w};
                    if constexpr (FRESH) {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (e < nval[k] && wv[4 * k + e] > 0)
                                mloc = fmaxf(mloc, fmaf(pf, lg2_approx((float)wv[4 * k + e]), -vh[e]));
                    } else {
                        const float4 l4 = lh4[FRESH ? 0 : k];
                        const float lh[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (lh[e] > -INFINITY) mloc = fmaxf(mloc, fmaf(pf, lh[e], -vh[e]));
                    }
                }
                mloc = warp_max(mloc);
                float* smx = (float*)redd;
                if (lane == 0) smx[wid] = mloc;
                __syncthreads();
                float mf = -INFINITY;
#pragma unroll
                for (int x = 0; x < NW; ++x) mf = fmaxf(mf, smx[x]);
                if (!(mf > -INFINITY)) {
                    if (tid == 0) atomicCAS(A.err, 0, kErrNonfinite);
                    mf = 0.0f;
                }
                cref = (double)mf;
                __syncthreads();   // smx is rewritten by the next row
            }
            if (tid == 0) crow[q] = cref;
            const float mh = (float)cref, ml = (float)(cref - (double)mh);
            float* krow = A.K + row * A.ldk;
            float kvs[M];
#pragma unroll
            for (int k = 0; k < CH; ++k) {
                float kv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                float vh[4] = {0.0f, 0.0f, 0.0f, 0.0f}, vl[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                if (nval[k] > 0) {
                    const float4 h4 = *(const float4*)(vhi + cidx[k] * 4);
                    const float4 l4 = *(const float4*)(vlo + cidx[k] * 4);
                    vh[0] = h4.x; vh[1] = h4.y; vh[2] = h4.z; vh[3] = h4.w;
                    vl[0] = l4.x; vl[1] = l4.y; vl[2] = l4.z; vl[3] = l4.w;
                }
                // log2 w of the chunk's entries as float pairs (-inf: no entry)
                float lh[4], ll[4];
                if constexpr (FRESH) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        lh[e] = -INFINITY;
                        ll[e] = 0.0f;
                        if (e < nval[k] && wv[4 * k + e] > 0) {
                            const float2 lw = wlog2(s_l2tab, wv[4 * k + e]);
                            lh[e] = lw.x;
                            ll[e] = lw.y;
                        }
                    }
                    if (cidx[k] < NC) {
                        *(float4*)(A.Lh + row * A.ldk + cidx[k] * 4) = make_float4(lh[0], lh[1], lh[2], lh[3]);
                        *(float4*)(A.Ll + row * A.ldk + cidx[k] * 4) = make_float4(ll[0], ll[1], ll[2], ll[3]);
                    }
                } else {
                    const float4 h4 = lh4[FRESH ? 0 : k], l4 = ll4[FRESH ? 0 : k];
                    lh[0] = h4.x; lh[1] = h4.y; lh[2] = h4.z; lh[3] = h4.w;
                    ll[0] = l4.x; ll[1] = l4.y; ll[2] = l4.z; ll[3] = l4.w;
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (lh[e] > -INFINITY) {
                        // x = p log2 w - V_j - m with 48-bit operands: the large leading
                        // parts cancel exactly (two-product, two-sums), the small ones are
                        // added after; x is then exact to about 2^-24 |x|
                        const float2 lw = make_float2(lh[e], ll[e]);
                        const float2 vj = make_float2(vh[e], vl[e]);
                        const float t = ph * lw.x;
                        const float te = fmaf(ph, lw.x, -t);
                        float e1, e2;
                        const float s1 = two_sum(t, -vj.x, &e1);
                        const float s2 = two_sum(s1, -mh, &e2);
                        const float rest = ((te + e1) + e2) + (fmaf(ph, lw.y, pl * lw.x) - vj.y - ml);
                        kv[e] = ex2_approx(s2 + rest);
                    }
                }
                if (cidx[k] < NC) *(float4*)(krow + cidx[k] * 4) = make_float4(kv[0], kv[1], kv[2], kv[3]);
#pragma unroll
                for (int e = 0; e < 4; ++e) kvs[4 * k + e] = kv[e];
            }
            if (SP && A.sparse_ok) {
                // compaction of the entries >= theta: warp scan of the per-thread counts
                unsigned c = 0;
#pragma unroll
                for (int x = 0; x < M; ++x) c += kvs[x] >= A.theta ? 1u : 0u;
                unsigned incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane == 31) wcnt[wid] = incl;
                __syncthreads();
                unsigned wbase = 0, tot = 0;
                for (int x = 0; x < NW; ++x) {
                    const unsigned t = wcnt[x];
                    if (x < wid) wbase += t;
                    tot += t;
                }
                const unsigned padded = tot < 2u ? 2u : tot + (tot & 1u);
                const bool fits = !overflow && roff + padded <= rec_cap;
                if (fits) {
                    size_t o = roff + wbase + incl - c;
#pragma unroll
                    for (int x = 0; x < M; ++x)
                        if (kvs[x] >= A.theta)
                            recb[o++] = make_uint2((unsigned)(cidx[x / 4] * 4 + (x % 4)), __float_as_uint(kvs[x]));
                    if (tid == 0)
                        for (unsigned e = tot; e < padded; ++e) recb[roff + e] = make_uint2(0u, 0u);
                }
                if (tid == 0) {
                    rowoff[q] = (unsigned)roff;
                    rowlen[q] = padded;
                    // stage records: rows 2g and 2g+1 are contiguous
                    const unsigned stage = (q & 1) ? rowlen[q - 1] + padded : padded;
                    if (stage > s_maxlen) s_maxlen = stage;
                }
                if (fits) roff += padded;
                else overflow = true;
                __syncthreads();   // wcnt is reused by the next row
            }
        }
        if (SP && A.sparse_ok && tid == 0) {
            unsigned long long* st = A.stats + 4 * (epoch & 1u);
            atomicAdd(st + 0, (unsigned long long)roff);
            atomicMax(st + 1, (unsigned long long)s_maxlen);
            if (overflow) atomicMax(st + 2, 1ull);
        }
        fence_proxy_async_all();   // K rows are read back, and the region overwritten, by bulk copies
        __syncthreads();
    };

    bool l_ready = false;   // this launch has stored its stripe's log2 pairs
    for (int k = A.k0; k < A.n_p; ++k) {
        const double p = A.P[k];
        int sweeps = 0;
        float resid = INFINITY;
        int step_reanchors = 0;   // after two re-anchors the step finishes dense
        for (;;) {   // epochs of step k: one evaluation of K, then sweeps until done or re-anchor
            // every copy of the previous epoch has landed; reset the ring
            __syncthreads();
            if (tid == 0) wait_copies();
            __syncthreads();
            if (s_flag) { drain(); return; }
            if (tid == 0) {
                for (int s = 0; s < MAXR; ++s) {
                    if (epoch > 0u) mbar_inval(&mbar[s]);   // initialised by the previous epoch
                    mbar_init(&mbar[s], 1);
                    rel_cnt[s] = iss_cnt[s] = 0u;
                }
                mbar_fence_init();
            }
            for (int j = c0 + tid; j < c1; j += NT) {
                A.Vs[j] = A.V[j];
                A.Cf[j] = 1.0f;
            }
            // the first evaluation of a step after a step (or a resumed one) scaled (u, v):
            // row references from U; otherwise the row maxima
            {
                const double cs = (k > 0 && !A.keep_v && step_reanchors == 0) ? p / A.P[k - 1] : 0.0;
                if (l_ready) {
                    prep(p, cs, std::false_type{});
                } else {
                    prep(p, cs, std::true_type{});
                    l_ready = true;
                }
            }
            if (!gsync()) { drain(); return; }
            // mode of this epoch, identical in every block
            if (tid == 0) {
                int sp = 0;
                if (SP && A.sparse_ok) {
                    const volatile unsigned long long* st = A.stats + 4 * (epoch & 1u);
                    sp = st[2] == 0ull && st[0] <= A.sparse_max_total && st[1] <= (unsigned long long)A.sparse_row_cap &&
                         step_reanchors < 2;
                    if (b == 0) {
                        unsigned long long* nx = A.stats + 4 * ((epoch + 1u) & 1u);
                        nx[0] = nx[1] = nx[2] = 0ull;
                    }
                    if (b == 0 && sp) atomicAdd(A.counters + 0, 1);
                }
                s_mode = sp;
            }
            __syncthreads();
            sparse = s_mode;
            ++epoch;
            its = 0;
            if (SP && sparse) {
                for (int j = tid; j < n; j += NT) {
                    c_s[j] = 1.0f;
                    S_s[j] = 0.0f;
                }
                slot_bytes = s_maxlen * 8u;
                sbase = region + cs_bytes;
                ring_n = (int)min((size_t)MAXR, ((size_t)A.region_bytes - cs_bytes) / slot_bytes);
            } else {
                slot_bytes = (unsigned)RPS * A.row_bytes;
                sbase = region;
                ring_n = A.ring / RPS;
#pragma unroll
                for (int m = 0; m < M; ++m) cf[m] = (m % 4) < nval[m / 4] ? 1.0f : 0.0f;
            }
            __syncthreads();
            if (tid == 0 && nrows > 0)
                for (uint32_t v = 0; v < (uint32_t)ring_n; ++v) issue_index(v);
            bool done = false, reanchor = false;
            while (!done && !reanchor) {
                SA_STEP_STAMP(0);
#pragma unroll
                for (int m = 0; m < M; ++m) S[m] = 0.0f;
                // ---------------- row pass ----------------
                // stage g = local rows 2g, 2g+1.  produce(g): partial row sums, published on
                // mrow[g % NRED]; consume(g): wait for every warp's partials, accumulate the
                // normalised rows into the column sums, release the slots.
                // row r (0, 1) of the stage at ring index v
                // row r of the stage in slot v % ring_n: dense rows at r row pitches; a sparse
                // stage (two rows) holds the records of its first row, then its second's
                auto row_of = [&](uint32_t v, int q0, int r) -> const unsigned char* {
                    const unsigned char* base = sbase + (size_t)(v % (uint32_t)ring_n) * slot_bytes;
                    if (r == 0) return base;
                    if (SP && sparse) return base + rowlen[q0] * 8u;
                    return base + (size_t)r * A.row_bytes;
                };
                auto row_partial = [&](const unsigned char* rowp, int q) -> float {
                    float a0 = 0.0f, a1 = 0.0f;
                    if (SP && sparse) {
                        const uint2* rp = (const uint2*)rowp;
                        const unsigned len = rowlen[q];
                        for (unsigned e = tid; e < len; e += NT) {
                            const uint2 r = rp[e];
                            a0 = fmaf(__uint_as_float(r.y), c_s[r.x], a0);
                        }
                        return a0;
                    }
#pragma unroll
                    for (int kk = 0; kk < CH; ++kk) {
                        if (nval[kk] == 0) continue;   // chunk beyond the row: not in the slot
                        const float4 kv = *(const float4*)(rowp + (size_t)cidx[kk] * 16);
                        a0 = fmaf(kv.x, cf[4 * kk], a0);
                        a1 = fmaf(kv.y, cf[4 * kk + 1], a1);
                        a0 = fmaf(kv.z, cf[4 * kk + 2], a0);
                        a1 = fmaf(kv.w, cf[4 * kk + 3], a1);
                    }
                    return a0 + a1;
                };
                auto produce = [&](int g) {
                    const uint32_t v = its + g;
                    const int q0 = RPS * stage_of(v);
                    const int nr = min(RPS, nrows - q0);   // rows of the stage (the last may be short)
                    const uint32_t rn = (uint32_t)ring_n;
                    if (!mbar_wait(&mbar[v % rn], (v / rn) & 1u, A.err, A.wait_ns)) {
                        s_flag = 1;   // this thread's copy is not in: its warp never releases the slot
                    }
                    float sp[RPS];
#pragma unroll
                    for (int r = 0; r < RPS; ++r) sp[r] = r < nr ? row_partial(row_of(v, q0, r), q0 + r) : 0.0f;
#pragma unroll
                    for (int r = 0; r < RPS; ++r) sp[r] = warp_sum(sp[r]);
                    if (lane == 0) {
                        const uint32_t gs = gbase + g;
#pragma unroll
                        for (int r = 0; r < RPS; ++r) red[((gs % NRED) * RPS + r) * NW + wid] = sp[r];
                        mbar_arrive(&mrow[gs % NRED]);
                    }
                };
                auto consume = [&](int g) -> bool {
                    const uint32_t v = its + g;
                    const int q0 = RPS * stage_of(v);
                    const int nr = min(RPS, nrows - q0);
                    const uint32_t gs = gbase + g;
                    if (!mbar_wait(&mrow[gs % NRED], (gs / NRED) & 1u, A.err, A.wait_ns)) s_flag = 1;
                    // warp-uniform: a warp either releases the stage (every lane got its copy
                    // and every partial) or leaves the pass as a whole
                    if (__any_sync(0xffffffffu, *(volatile int*)&s_flag != 0)) return false;
                    float ss[RPS];
                    bool ss_bad = false;
#pragma unroll
                    for (int r = 0; r < RPS; ++r) {
                        const float4* rv = (const float4*)(red + ((gs % NRED) * RPS + r) * NW);
                        float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
#pragma unroll
                        for (int x = 0; x < NW / 4; ++x) {
                            const float4 q4 = rv[x];
                            a0 += q4.x;
                            a1 += q4.y;
                            a2 += q4.z;
                            a3 += q4.w;
                        }
                        ss[r] = (a0 + a1) + (a2 + a3);
                        if (r < nr && !(ss[r] >= 0x1p-120f && ss[r] <= 0x1p120f)) ss_bad = true;
                    }
                    if (ss_bad) {
                        if (tid == 0) atomicCAS(A.err, 0, kErrNonfinite);
                        s_flag = 1;
                        return false;
                    }
                    if (tid == 0) {
#pragma unroll
                        for (int r = 0; r < RPS; ++r)
                            if (r < nr) srow[q0 + r] = ss[r];
                    }
#pragma unroll
                    for (int r = 0; r < RPS; ++r) {
                        if (r >= nr) break;
                        const float inv = rcp_approx(ss[r]);
                        const unsigned char* rowp = row_of(v, q0, r);
                        if (SP && sparse) {
                            const uint2* rp = (const uint2*)rowp;
                            const unsigned len = rowlen[q0 + r];
                            for (unsigned e = tid; e < len; e += NT) {
                                const uint2 rr = rp[e];
                                atomicAdd(&S_s[rr.x], __uint_as_float(rr.y) * inv);
                            }
                            continue;
                        }
#pragma unroll
                        for (int kk = 0; kk < CH; ++kk) {
                            if (nval[kk] == 0) continue;
                            const float4 kv = *(const float4*)(rowp + (size_t)cidx[kk] * 16);
                            S[4 * kk] = fmaf(kv.x, inv, S[4 * kk]);
                            S[4 * kk + 1] = fmaf(kv.y, inv, S[4 * kk + 1]);
                            S[4 * kk + 2] = fmaf(kv.z, inv, S[4 * kk + 2]);
                            S[4 * kk + 3] = fmaf(kv.w, inv, S[4 * kk + 3]);
                        }
                    }
                    __syncwarp();
                    if (lane == 0) release_index(v);
                    return true;
                };
                // With three or more ring stages the partial row sums of stage g + 1 are
                // formed while the other warps' partials of stage g are still arriving.  A
                // two-stage ring cannot look ahead: the slot of g + 1 is refilled only when
                // g + 1 - 2 is released, so each stage is consumed first and its copy for
                // g + 2 is in flight while the next stage is read.  (Forming g + 1's partials
                // first whenever its copy had already landed measured slower: 46.7 against
                // 45.5 us per sweep at n = 8192 with three-row stages.)
                if ((SP && sparse) || ring_n > 2) {
                    if (nst > 0) produce(0);
                    for (int g = 0; g < nst; ++g) {
                        if (g + 1 < nst) produce(g + 1);
                        if (!consume(g)) break;
                    }
                } else {
                    for (int g = 0; g < nst; ++g) {
                        produce(g);
                        if (!consume(g)) break;
                    }
                }
                __syncthreads();
                SA_STEP_STAMP(1);
                if (s_flag) { drain(); return; }
                its += (uint32_t)nst;
                gbase += (uint32_t)nst;
                float* pb = A.part + (size_t)b * A.npad;
                if (SP && sparse) {
                    for (int j = tid; j < n; j += NT) {
                        pb[j] = S_s[j] * c_s[j];
                        S_s[j] = 0.0f;
                    }
                } else {
#pragma unroll
                    for (int kk = 0; kk < CH; ++kk) {
                        if (nval[kk] > 0)
                            *(float4*)(pb + (size_t)cidx[kk] * 4) =
                                make_float4(S[4 * kk] * cf[4 * kk], S[4 * kk + 1] * cf[4 * kk + 1],
                                            S[4 * kk + 2] * cf[4 * kk + 2], S[4 * kk + 3] * cf[4 * kk + 3]);
                    }
                }
                ++sweeps;
                if (!gsync()) { drain(); return; }
                SA_STEP_STAMP(2);
                // ---------------- column finalisation of columns [c0, c1) ----------------
                const int par = (sweeps + rphase) & 1;
                float* rmax_word = A.rmax + par;
                float rmax = 0.0f, cmx = 0.0f, cmn = INFINITY;
                for (int cb = c0; cb < c1; cb += 64) {
                    const int j = cb + (tid & 63);
                    const int grp = tid >> 6;
                    KahanS acc;
                    if (j < c1) {
                        // every load of a batch is issued before the first is used: one L2
                        // round trip per 24 partial rows (FG * 24 >= 192 rows at 512 threads)
                        const float* pj = A.part + j;
                        for (int g0 = grp; g0 < G; g0 += FG * 24) {
                            float a[24];
#pragma unroll
                            for (int x = 0; x < 24; ++x) {
                                const int g = g0 + x * FG;
                                a[x] = g < G ? __ldcg(pj + (size_t)g * A.npad) : 0.0f;
                            }
#pragma unroll
                            for (int x = 0; x < 24; ++x) acc.add(a[x]);
                        }
                    }
                    redp[grp * 64 + (tid & 63)] = (double)acc.s - (double)acc.c;
                    __syncthreads();
                    if (tid < 64 && j < c1) {
                        double Sj = 0.0;
#pragma unroll
                        for (int x = 0; x < FG; ++x) Sj += redp[x * 64 + tid];
                        if (!(Sj > 0.0) || !isfinite(Sj)) atomicCAS(A.err, 0, kErrNonfinite);
                        const double d = Sj - 1.0;
                        rmax = fmaxf(rmax, (float)fabs(d));
                        double lg;
                        if (fabs(d) < 1e-3) {
                            // log2(1 + d) by its series in FP64 (|d| < 1e-3: five terms reach 1e-17)
                            lg = d * (1.0 + d * (-0.5 + d * (1.0 / 3.0 + d * (-0.25 + d * 0.2)))) * kLog2e;
                        } else {
                            lg = log2(Sj);
                        }
                        const double v = A.V[j] + lg;
                        A.V[j] = v;
                        const float cnew = ex2_approx((float)(A.Vs[j] - v));
                        A.Cf[j] = cnew;
                        cmx = fmaxf(cmx, cnew);
                        cmn = fminf(cmn, cnew);
                    }
                    __syncthreads();
                }
                if (wid < 2) {
                    rmax = warp_max(rmax);
                    if (lane == 0 && rmax > 0.0f) atomicMax((unsigned*)rmax_word, __float_as_uint(rmax));
                    if (SP && sparse) {
                        cmx = warp_max(cmx);
                        cmn = -warp_max(-cmn);
                        // positive floats order like their bit patterns
                        if (lane == 0 && cmx > 0.0f) atomicMax(A.crange + 2 * par, __float_as_uint(cmx));
                        if (lane == 0 && cmn < INFINITY) atomicMin(A.crange + 2 * par + 1, __float_as_uint(cmn));
                    }
                }
                if (!gsync()) { drain(); return; }
                SA_STEP_STAMP(3);
                // ---------------- decision (identical in every block) ----------------
                // the next sweep's column factors are loaded while the residual word is
                // read (one L2 round trip for both); the old ones are dead once the partials
                // are written, and a new epoch resets them if the step ends here
                if (!(SP && sparse)) {
#pragma unroll
                    for (int kk = 0; kk < CH; ++kk)
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            cf[4 * kk + e] = e < nval[kk] ? __ldcg(A.Cf + cidx[kk] * 4 + e) : 0.0f;
                }
                if (tid == 0) {
                    s_res = __uint_as_float(ld_acquire((const unsigned*)rmax_word));
                    int ra = 0;
                    if (SP && sparse) {
                        const float hi = __uint_as_float(ld_acquire(A.crange + 2 * par));
                        const float lo = __uint_as_float(ld_acquire(A.crange + 2 * par + 1));
                        ra = !(hi <= A.reanchor_ratio * lo);
                    }
                    s_reanchor = ra;
                    if (b == 0) {
                        A.rmax[par ^ 1] = 0.0f;
                        A.crange[2 * (par ^ 1)] = 0u;
                        A.crange[2 * (par ^ 1) + 1] = 0x7f800000u;
                    }
                }
                __syncthreads();
                resid = s_res;
                done = (resid <= A.tol) || (sweeps >= A.max_sweeps);
                reanchor = !done && s_reanchor;
                if (!done && !reanchor) {
                    if (SP && sparse) {
                        for (int j = tid; j < n; j += NT) c_s[j] = __ldcg(A.Cf + j);
                        __syncthreads();
                    }
                }
                SA_STEP_STAMP(4);
            }
            if (!reanchor) break;
            ++step_reanchors;
            if (b == 0 && tid == 0) atomicAdd(A.counters + 1, 1);
        }
        rphase += sweeps;
        for (int q = tid; q < nrows; q += NT) A.U[r0 + q] = crow[q] + log2((double)srow[q]);
        if (b == 0 && tid == 0) {
            A.sweeps_out[k] = sweeps;
            A.resid_out[k] = resid;
        }
        if (k + 1 < A.n_p) {
            const double f = A.keep_v ? 1.0 : A.P[k + 1] / p;
            for (int j = c0 + tid; j < c1; j += NT) A.V[j] *= f;
            if (!gsync()) { drain(); return; }
        }
    }
    drain();
}

struct StepCfg {
    int nt, ch, ring;
    int rps;   // rows per ring stage
};

size_t step_smem_bytes(int nt, size_t region_bytes, int max_rows) {
    const int nw = nt / 32;
    const int fg = nt / 64;
    return region_bytes + 8 * (size_t)(kStepMaxRing + kStepNred) + 8 * (size_t)kStepMaxRing +
           4 * (size_t)(kStepNred * kStepMaxRps * nw) +
           8 * (size_t)(max_rows + fg * 64 + nw) + 4 * (size_t)max_rows + 8 * (size_t)max_rows + 4096 + 1024;
}

int step_max_rows(const sa_ctx* ctx, int n) {
    int gmin = std::max(1, std::min(ctx->num_sms, n / 8));
    if (ctx->max_grid > 0) gmin = std::max(1, std::min(gmin, ctx->max_grid));
    return (n + gmin - 1) / gmin + 1;
}

StepCfg pick_step(const sa_ctx* ctx, int n) {
    const int nc = (n + 3) / 4;
    const int R = kDenseRowsPerStage;
    StepCfg c{0, 0, 0, R};
    if (nc <= 128) c = {128, 1, 0, R};
    else if (nc <= 256) c = {256, 1, 0, R};
    else if (nc <= 512) c = {512, 1, 0, R};
    else if (nc <= 1024) c = {512, 2, 0, R};
    else if (nc <= 2048) c = {512, 4, 0, R};
    else if (nc <= 3072) c = {512, 6, 0, R};
    else if (nc <= 4096) c = {512, 8, 0, 1};
    else if (nc <= 5120) c = {512, 10, 0, 1};
    else if (nc <= 6144) c = {512, 12, 0, 1};
    else return c;
    const unsigned row_bytes = (unsigned)align_up((size_t)n * 4, 16);
    const int max_rows = step_max_rows(ctx, n);
    auto fits = [&](int ring) {
        return step_smem_bytes(c.nt, (size_t)ring * row_bytes, max_rows) <= ctx->smem_optin;
    };
    // ring slots in rows, a whole number of stages, at least two: one-row stages for rows of
    // 48 to 96 KB (two or three fit); else two-row stages, up to four, unless at most three
    // of them fit and two three-row stages do.  The ring doubles as scratch for V
    // (8 ceil(n/4)*4 bytes = two rows) during the per-step evaluation of K.
    if (c.rps == 1) {
        for (int st = 3; st >= 2; --st)
            if (fits(st)) {
                c.ring = st;
                return c;
            }
    } else {
        int st2 = 0;
        for (int st = 4; st >= 2 && st2 == 0; --st)
            if (fits(st * kDenseRowsPerStage)) st2 = st;
        if (st2 <= 3 && (c.ch == 4 || c.ch == 6) && fits(2 * kWideRowsPerStage)) {
            c.rps = kWideRowsPerStage;
            c.ring = 2 * kWideRowsPerStage;
            return c;
        }
        if (st2 >= 2) {
            c.ring = st2 * kDenseRowsPerStage;
            return c;
        }
    }
    c.nt = 0;
    return c;
}

template <int NT, int CH, int RPS = kDenseRowsPerStage>
sa_status launch_step(sa_ctx* ctx, const StepArgs& args, size_t smem, int* grid_out) {
    // the dense-only instantiation carries none of the sparse code (sparse epochs need
    // two-row stages)
    void (*kern)(StepArgs);
    if constexpr (RPS == 2)
        kern = args.sparse_ok ? step_kernel<NT, CH, true, 2> : step_kernel<NT, CH, false, 2>;
    else
        kern = step_kernel<NT, CH, false, RPS>;
    SA_CUDA(allow_dynamic_smem(kern, ctx->smem_optin));
    int per_sm = 0;
    SA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    if (per_sm < 1) {
        set_error("step sweep: kernel does not fit on an SM (smem %zu)", smem);
        return SA_E_UNSUPPORTED;
    }
    int G = ctx->num_sms * per_sm;
    const int gmax_rows = args.n / 8 > 0 ? args.n / 8 : 1;
    if (G > gmax_rows) G = gmax_rows;
    if (*grid_out > 0 && *grid_out < G) G = *grid_out;
    if ((args.n + G - 1) / G > args.max_rows) {
        set_error("step sweep: grid of %d blocks leaves stripes longer than %d rows", G, args.max_rows);
        return SA_E_UNSUPPORTED;
    }
    *grid_out = G;
    StepArgs a = args;
    // stages of each stripe that stay L2-resident: the context's byte budget over the grid
    const size_t stage_bytes = (size_t)RPS * args.row_bytes;
    const size_t keep = ctx->step_l2_bytes / ((size_t)G * stage_bytes);
    a.l2_keep_stages = (int)std::min<size_t>(keep, (size_t)args.n);
    void* params[] = {&a};
    SA_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(NT), params, smem, ctx->stream));
    count_launch();
    return SA_OK;
}

}  // namespace

bool step_supported(const sa_ctx* ctx, const sa_matrix* a) {
    const int sz = wbytes(a->wtype);
    if (((uintptr_t)a->w & 15) != 0) return false;
    if (((size_t)a->ld * sz) % 16 != 0) return false;
    return pick_step(ctx, a->n).nt > 0;
}

// records per row reserved for sparse epochs: a quarter of the row (denser steps run dense)
int64_t step_rec_cap_row(int n) { return (int64_t)align_up((size_t)n / 4 + 2, 2); }

size_t step_workspace_bytes(const sa_ctx* ctx, const sa_matrix* a, int n_p) {
    const int n = a->n;
    const size_t ldk = align_up((size_t)n, 4);
    const int G_max = ctx->num_sms * 2;
    const size_t npad = align_up((size_t)n, 32);
    const size_t recs = ctx->step_sparse ? (size_t)n * step_rec_cap_row(n) : 2;
    return (size_t)n * ldk * 12 + recs * 8 + (size_t)G_max * npad * 4 +
           2 * align_up((size_t)n * 8, 256) + align_up((size_t)n * 4, 256) + (size_t)n_p * 16 + 32768;
}

sa_status scale_step(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U, double* V,
                     sa_scale_info* info) {
    const int n = a->n;
    const StepCfg cfg = pick_step(ctx, n);
    if (cfg.nt == 0) {
        set_error("step sweep: n=%d not supported", n);
        return SA_E_UNSUPPORTED;
    }
    cudaStream_t st = ctx->stream;
    const int G_max = ctx->num_sms * 2;
    const int npad = (int)align_up((size_t)n, 32);
    const int64_t ldk = (int64_t)align_up((size_t)n, 4);
    sa_status rc = ctx->ws.reserve(step_workspace_bytes(ctx, a, o->n_p));
    if (rc) return rc;
    Carve cv(ctx->ws.ptr);
    float* K = cv.take<float>((size_t)n * ldk);
    float* Lh = cv.take<float>((size_t)n * ldk);
    float* Ll = cv.take<float>((size_t)n * ldk);
    const int64_t rec_cap_row = ctx->step_sparse ? step_rec_cap_row(n) : 0;
    uint2* rec = cv.take<uint2>(ctx->step_sparse ? (size_t)n * rec_cap_row : 2);
    float* part = cv.take<float>((size_t)G_max * npad);
    double* Vs = cv.take<double>(n);
    float* Cf = cv.take<float>(n);
    float* rmax = cv.take<float>(2);
    double* P = cv.take<double>(o->n_p);
    double* resid_out = cv.take<double>(o->n_p);
    int* sweeps_out = cv.take<int>(o->n_p);
    unsigned* bar = cv.take<unsigned>(2);
    int* err = cv.take<int>(1);
    unsigned long long* stats = cv.take<unsigned long long>(8);
    unsigned* crange = cv.take<unsigned>(4);
    int* counters = cv.take<int>(2);
    SA_CUDA(cudaMemcpyAsync(P, o->p, o->n_p * sizeof(double), cudaMemcpyHostToDevice, st));
    SA_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
    SA_CUDA(cudaMemsetAsync(rmax, 0, 2 * sizeof(float), st));
    SA_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    SA_CUDA(cudaMemsetAsync(sweeps_out, 0, o->n_p * sizeof(int), st));
    SA_CUDA(cudaMemsetAsync(stats, 0, 8 * sizeof(unsigned long long), st));
    SA_CUDA(cudaMemsetAsync(counters, 0, 2 * sizeof(int), st));
    {
        // crange words: max = 0, min = +inf (bits of positive floats order like the floats)
        static const unsigned init[4] = {0u, 0x7f800000u, 0u, 0x7f800000u};
        SA_CUDA(cudaMemcpyAsync(crange, init, sizeof(init), cudaMemcpyHostToDevice, st));
    }
    const int k0 = o->resume_from > 0 ? o->resume_from : 0;
    if (k0 == 0) {
        SA_CUDA(cudaMemsetAsync(U, 0, n * sizeof(double), st));
        SA_CUDA(cudaMemsetAsync(V, 0, n * sizeof(double), st));
    } else if (!o->warm_keep_v) {
        launch_scale_vec(V, n, o->p[k0] / o->p[k0 - 1], st);
    }
    const size_t region = (size_t)cfg.ring * align_up((size_t)n * 4, 16);
    const size_t cs_bytes = align_up((size_t)n * 8, 16);
    StepArgs args{};
    args.w = a->w;
    args.n = n;
    args.ld = a->ld;
    args.i16 = a->wtype == SA_I16;
    args.K = K;
    args.Lh = Lh;
    args.Ll = Ll;
    args.ldk = ldk;
    args.row_bytes = (unsigned)align_up((size_t)n * 4, 16);
    args.ring = cfg.ring;
    args.region_bytes = (unsigned)region;
    args.rec = rec;
    args.rec_cap_row = rec_cap_row;
    args.stats = stats;
    args.crange = crange;
    args.counters = counters;
    // a sparse epoch's ring (next to c and S) needs >= 3 slots of its longest stage: two in
    // use and one in flight
    args.sparse_row_cap = region > cs_bytes ? (unsigned)(((region - cs_bytes) / (3 * 8)) & ~(size_t)1) : 0u;
    args.sparse_ok = ctx->step_sparse && cfg.rps == 2 && args.sparse_row_cap >= 2;
    args.sparse_max_total = (unsigned long long)n * (unsigned long long)n / 4ull;
    // dropped entries of a row sum to at most n * theta * (max c / min c) of its mass
    // (the largest entry of K in a row is about 1): n * 2^-70 * 2^20 <= 2^-36 for n <= 2^14
    args.theta = 0x1p-70f;
    args.reanchor_ratio = 0x1p20f;
    args.P = P;
    args.k0 = k0;
    args.n_p = o->n_p;
    args.tol = o->tol;
    args.max_sweeps = o->max_sweeps_per_p;
    args.keep_v = o->warm_keep_v;
    args.U = U;
    args.V = V;
    args.Vs = Vs;
    args.Cf = Cf;
    args.part = part;
    args.npad = npad;
    args.rmax = rmax;
    args.bar = bar;
    args.err = err;
    args.sweeps_out = sweeps_out;
    args.resid_out = resid_out;
    args.max_rows = step_max_rows(ctx, n);
    args.wait_ns = ctx->wait_ns;
    args.extra_arrivals = ctx->test_unreachable_barrier ? 1u : 0u;
    const size_t smem = step_smem_bytes(cfg.nt, region, args.max_rows);
    int G = ctx->max_grid > 0 ? std::min(G_max, ctx->max_grid) : G_max;
    cudaEvent_t ev0, ev1;
    SA_CUDA(cudaEventCreate(&ev0));
    SA_CUDA(cudaEventCreate(&ev1));
    SA_CUDA(cudaEventRecord(ev0, st));
    if (cfg.nt == 128) rc = launch_step<128, 1>(ctx, args, smem, &G);
    else if (cfg.nt == 256) rc = launch_step<256, 1>(ctx, args, smem, &G);
    else if (cfg.ch == 1) rc = launch_step<512, 1>(ctx, args, smem, &G);
    else if (cfg.ch == 2) rc = launch_step<512, 2>(ctx, args, smem, &G);
    else if (cfg.ch == 4 && cfg.rps == kWideRowsPerStage) rc = launch_step<512, 4, kWideRowsPerStage>(ctx, args, smem, &G);
    else if (cfg.ch == 4) rc = launch_step<512, 4>(ctx, args, smem, &G);
    else if (cfg.ch == 6 && cfg.rps == kWideRowsPerStage) rc = launch_step<512, 6, kWideRowsPerStage>(ctx, args, smem, &G);
    else if (cfg.ch == 6) rc = launch_step<512, 6>(ctx, args, smem, &G);
    else if (cfg.ch == 8) rc = launch_step<512, 8, 1>(ctx, args, smem, &G);
    else if (cfg.ch == 10) rc = launch_step<512, 10, 1>(ctx, args, smem, &G);
    else rc = launch_step<512, 12, 1>(ctx, args, smem, &G);
    if (rc) { cudaEventDestroy(ev0); cudaEventDestroy(ev1); return rc; }
    SA_CUDA(cudaEventRecord(ev1, st));
    sa_status prc = ctx->pinned.reserve(4096 + (size_t)o->n_p * 16);
    if (prc) return prc;
    char* hp = (char*)ctx->pinned.ptr;
    int* h_err = (int*)hp;
    int* h_cnt = (int*)(hp + 16);
    int* h_sw = (int*)(hp + 64);
    double* h_rs = (double*)(hp + 64 + align_up((size_t)o->n_p * 4, 64));
    SA_CUDA(cudaMemcpyAsync(h_err, err, 4, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(h_cnt, counters, 8, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(h_sw, sweeps_out, o->n_p * 4, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(h_rs, resid_out, o->n_p * 8, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaStreamSynchronize(st));
    float kms = 0.0f;
    SA_CUDA(cudaEventElapsedTime(&kms, ev0, ev1));
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    int64_t total = 0;
    int conv = 1;
    for (int k = k0; k < o->n_p; ++k) {
        total += h_sw[k];
        if (!(h_rs[k] <= o->tol)) conv = 0;
    }
    if (info) {
        info->sweeps_total = total;
        info->residual = h_rs[o->n_p - 1];
        info->p_final = o->p[o->n_p - 1];
        info->converged = conv;
        info->steps_done = o->n_p - k0;
        info->fallback_rows = 0;
        info->kernel_used = SA_KERNEL_STEP;
        info->kernel_ms = kms;
        info->sparse_epochs = h_cnt[0];
        info->reanchors = h_cnt[1];
    }
    if (*h_err == kErrTimeout) {
        set_error("step sweep: a bounded device wait timed out (grid of %d blocks)", G);
        return SA_E_TIMEOUT;
    }
    if (*h_err == kErrNonfinite) {
        set_error("step sweep: a row or column sum left the FP32 range (matrix without support?)");
        return SA_E_NONFINITE;
    }
    return conv ? SA_OK : SA_E_NOT_CONVERGED;
}

}  // namespace sa
