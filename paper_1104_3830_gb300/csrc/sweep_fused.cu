// sweep_fused.cu -- the single-read Sinkhorn sweep: one persistent cooperative kernel
// runs every sweep of every p step of the schedule (Sec. 4.1.2 log-domain iteration,
// Sec. 4.2 stopping rule) and reads A once per sweep.
//
// Work split.  Block b owns the row stripe [b*n/G, (b+1)*n/G).  Within a block every
// compute thread owns a fixed set of 16-byte column chunks, so the column partial sums of
// the stripe live in registers for the whole sweep.  Rows stream through a shared-memory
// ring filled by the bulk-copy engine (cp.async.bulk + mbarrier).  Each warp counts its
// release of a slot on a shared counter; the warp whose release completes the count
// refills the slot at once with the row RING positions ahead, so nobody waits to issue a
// copy and a slot is reused as soon as the last reader is done with it.
//
// One sweep, in log2 units (U = u/ln2, V = v/ln2, L = log2 w):
//   row i   t_ij = 2^(p log2(w_ij a_i) - Vh_j) * c_j          (FP32, SFU ex2/lg2)
//           s_i  = sum_j t_ij                                   (block reduction)
//           S_j += t_ij / s_i        (column sums of the row-stochastic iterate)
//           U_i  = -p log2 a_i + log2 s_i                       (row update, dad2)
//   grid barrier; block b finalises a slice of columns:
//           S_j  = sum_b S_j^(b)     (FP64, fixed order: deterministic)
//           V_j += log2 S_j          (column update, dad3, FP64)
//           residual = max_j |S_j - 1|  (eps-bistochastic measure, Sec. 4.2, FP64)
//   grid barrier; every block reads the residual and takes the same decision.
// a_i = float(2^(-U_i/p)) is a per-row FP32 scale frozen during a p step: the row
// normalisation cancels it exactly, and it keeps log2(w a) small for the entries that
// matter, so the SFU logarithm's absolute error stays small.  w a is formed exactly up to
// one rounding (int16: the integer is decoded by a byte permute into a float with a
// 2^23 bias and one FMA removes the bias and applies a).  V_j is exact in FP64; the kernel
// applies it as an FP32 head Vh_j = float(V_j) (frozen per step) times c_j = 2^(Vh_j - V_j),
// so column updates smaller than an FP32 ulp of V are not lost.
//
// Rows whose sum leaves [2^-64, 2^64] (a stale shift, e.g. the first sweep at a large
// p) are recomputed with the exact max shift of the paper and re-anchor Lr_i.
//
// Every wait is bounded (2 s); on expiry the kernel records kErrTimeout, drains its
// outstanding bulk copies and returns.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "sa_internal.h"

namespace sa {

struct FusedArgs {
    const void* w;
    int n;
    int64_t ld;
    unsigned row_bytes;   // bytes copied per row (multiple of 16)
    const double* P;      // device copy of the schedule
    int k0, n_p;
    double tol;
    int max_sweeps;
    int keep_v;
    int f32_potentials;   // SA_PREC_FP32: round U, V to FP32 after every update
    double* U;            // n, log2 units
    double* V;            // n, log2 units
    float* Vh;            // n, FP32 head of V (frozen per step)
    float* Vc;            // n, 2^(Vh - V)
    float* part;          // G x npad column partials
    int npad;
    float* rmax;          // 2 alternating words: max_j |S_j - 1| of a sweep (atomicMax)
    unsigned* bar;        // grid barrier words
    int* err;
    int* fallback;
    int* sweeps_out;      // n_p
    double* resid_out;    // n_p
    int max_rows;         // max rows in any stripe (smem arrays)
};

namespace {

template <typename WT>
struct Vec;
template <>
struct Vec<int16_t> {
    static constexpr int N = 8;
    // log2(w * a) of 8 weights: the byte permute places w in the mantissa of 2^23, and one
    // FMA forms (2^23 + w) a - 2^23 a = w a exactly rounded (ca = -2^23 a is exact)
    __device__ static __forceinline__ void log2w(const uint4& q, float a, float ca, float* L) {
        const uint32_t wd[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            L[2 * k] = lg2_approx(fmaf(__uint_as_float(__byte_perm(wd[k], 0x4B00u, 0x5410u)), a, ca));
            L[2 * k + 1] = lg2_approx(fmaf(__uint_as_float(__byte_perm(wd[k], 0x4B00u, 0x5432u)), a, ca));
        }
    }
};
template <>
struct Vec<int32_t> {
    static constexpr int N = 4;
    __device__ static __forceinline__ void log2w(const uint4& q, float a, float, float* L) {
        L[0] = lg2_approx((float)(int)q.x * a);
        L[1] = lg2_approx((float)(int)q.y * a);
        L[2] = lg2_approx((float)(int)q.z * a);
        L[3] = lg2_approx((float)(int)q.w * a);
    }
};

#ifndef SA_STAMP
#define SA_STAMP(slot)   // phase timing hook (no-op in the library build)
#endif

// Kahan-compensated FP32 accumulation
struct KahanF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Grid barrier on a monotonic arrival counter: barrier number `k` (0, 1, 2, ...) completes
// when the counter reaches (k + 1) * nblocks.  Bounded wait; false on timeout or error.
__device__ __forceinline__ bool grid_sync(unsigned* ctr, unsigned target, int* err, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(ctr, 1u);
        if (ld_acquire(ctr) < target) {
            const uint64_t t0 = globaltimer_ns();
            unsigned spins = 0;
            while (ld_acquire(ctr) < target) {
                if ((++spins & 31u) == 0) {
                    if (*(volatile int*)err != 0) { ok = 0; break; }
                    if (globaltimer_ns() - t0 > kWaitTimeoutNs) { atomicCAS(err, 0, kErrTimeout); ok = 0; break; }
                }
                __nanosleep(32);
            }
        }
        if (*(volatile int*)err != 0) ok = 0;
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// Shared-memory fetch-and-add with acquire-release semantics at CTA scope: the caller's
// earlier reads are ordered before it, and the releases it observes before what follows.
__device__ __forceinline__ unsigned atom_add_acq_rel_cta(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(smem_u32(p)), "r"(v) : "memory");
    return old;
}

template <typename WT, int NT, int CH, int RING, int R>
__global__ void __launch_bounds__(NT, 1) fused_kernel(FusedArgs A) {
    constexpr int VEC = Vec<WT>::N;
    constexpr int NW = NT / 32;
    constexpr int M = CH * VEC;   // columns owned per thread
    constexpr int M4 = M / 4;
    constexpr int NRED = 4;       // row-sum buffers in flight (see the pipeline note below)
    constexpr int FG = NT / 64;   // column-finalisation groups of 64 threads
    static_assert(M % 4 == 0 && NT % 64 == 0, "layout");
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char* ring = smem;
    uint64_t* mbar = (uint64_t*)(smem + (size_t)RING * A.row_bytes);   // [RING] bulk-copy arrivals (full)
    uint64_t* mrow = mbar + RING;                                      // [NRED] row-sum publication
    unsigned* rel_cnt = (unsigned*)(mrow + NRED);                      // [RING] warp releases per slot
    unsigned* iss_cnt = rel_cnt + RING;                                // [RING] copies issued per slot
    float4* tbuf = (float4*)(mrow + NRED + RING + ((2 * RING + NRED) & 1));   // [4][M4][NT]
    float* red = (float*)(tbuf + (size_t)4 * M4 * NT);                 // [NRED][2][NW]
    float* red2 = red + NRED * 2 * NW;                                 // [NW] slow path
    float* Lr = red2 + NW;                                             // [max_rows]
    float* srow = Lr + A.max_rows;                                     // [max_rows]
    double* redp = (double*)(srow + A.max_rows);   // [FG][64] (offset 4*(9 NW + 2 max_rows): 8-aligned)
    __shared__ int s_flag, s_ok;
    __shared__ float s_res;

    const int n = A.n;
    const int G = gridDim.x;
    const int b = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int r0 = (int)((int64_t)b * n / G);
    const int r1 = (int)((int64_t)(b + 1) * n / G);
    const int nrows = r1 - r0;
    const int c0 = r0, c1 = r1;   // this block finalises the same index range of columns
    const int NC = (n + VEC - 1) / VEC;
    const unsigned char* wbase = (const unsigned char*)A.w;
    const size_t pitch = (size_t)A.ld * sizeof(WT);

    if (tid == 0) {
        for (int s = 0; s < RING; ++s) mbar_init(&mbar[s], 1);
        for (int s = 0; s < RING; ++s) rel_cnt[s] = iss_cnt[s] = 0;
        for (int s = 0; s < NRED; ++s) mbar_init(&mrow[s], NW);
        mbar_fence_init();
        s_flag = 0;
    }
    __syncthreads();

    uint32_t it = 0;            // rows consumed by this block, over all sweeps
    uint32_t gbase = 0;         // row stages completed by this block, over all sweeps
    unsigned nbar = 0;          // grid barriers passed
    int rphase = 0;             // sweeps of earlier steps (selects the residual word)
    // Consumption index u holds local row u % nrows in slot u % RING (phase u / RING).
    auto issue_index = [&](uint32_t u) {   // one thread
        const uint32_t slot = u % RING;
        const int q = (int)(u % (uint32_t)nrows);
        iss_cnt[slot] += 1;
        mbar_arrive_expect_tx(&mbar[slot], A.row_bytes);
        bulk_g2s(ring + (size_t)slot * A.row_bytes, wbase + (size_t)(r0 + q) * pitch, A.row_bytes, &mbar[slot]);
    };
    // lane 0, after __syncwarp: the warp is done reading index u; the last of the NW
    // warps refills the slot with index u + RING
    auto release_index = [&](uint32_t u) {
        const uint32_t slot = u % RING;
        const unsigned old = atom_add_acq_rel_cta(&rel_cnt[slot], 1u);
        if ((old + 1u) % (unsigned)NW == 0u) {
            fence_proxy_async_smem();
            issue_index(u + RING);
        }
    };
    // wait for the last copy issued into every slot (bounded), so none is in flight at exit
    auto drain = [&]() {
        __syncthreads();
        if (tid == 0) {
            for (int s = 0; s < RING; ++s) {
                const unsigned k = iss_cnt[s];
                if (k > 0u && !mbar_wait(&mbar[s], (k - 1u) & 1u, A.err, kWaitTimeoutNs)) break;
            }
        }
        __syncthreads();
    };
    auto gsync = [&]() -> bool {
        ++nbar;
        return grid_sync(A.bar, nbar * (unsigned)G, A.err, &s_ok);
    };

    if (tid == 0 && nrows > 0)
        for (uint32_t u = 0; u < (uint32_t)RING; ++u) issue_index(u);   // the first RING rows

    int cidx[CH];
    int nval[CH];
#pragma unroll
    for (int k = 0; k < CH; ++k) {
        cidx[k] = tid + k * NT;
        nval[k] = cidx[k] < NC ? min(VEC, n - cidx[k] * VEC) : 0;
    }

    float S[M], vh[M], vc[M];
    auto load_cols = [&]() {
#pragma unroll
        for (int k = 0; k < CH; ++k)
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int j = cidx[k] * VEC + e;
                const bool ok = e < nval[k];
                vh[k * VEC + e] = ok ? __ldcg(A.Vh + j) : 0.0f;
                vc[k * VEC + e] = ok ? __ldcg(A.Vc + j) : 0.0f;   // c = 0 masks the column
            }
    };

    // Terms t_ij = 2^(p log2(w_ij a_i) - Vh_j) of this thread's columns into tbuf[slot];
    // a_i = 2^-Lr_i is the row's scale (log2(w a) is small for the entries that matter).
    // Returns the partial row sum of t_ij c_j (c_j is applied to the column sums later).
    auto row_terms = [&](const unsigned char* rowp, float a, float pf, int slot) -> float {
        const float ca = -8388608.0f * a;
        float sp0 = 0.0f, sp1 = 0.0f;
#pragma unroll
        for (int kk = 0; kk < CH; ++kk) {
            float t[VEC];
            if (nval[kk] == VEC) {
                float L[VEC];
                Vec<WT>::log2w(*(const uint4*)(rowp + (size_t)cidx[kk] * 16), a, ca, L);
#pragma unroll
                for (int e = 0; e < VEC; ++e) t[e] = ex2_approx(fmaf(pf, L[e], -vh[kk * VEC + e]));
            } else {
#pragma unroll
                for (int e = 0; e < VEC; ++e) t[e] = 0.0f;
                if (nval[kk] > 0) {
                    float L[VEC];
                    Vec<WT>::log2w(*(const uint4*)(rowp + (size_t)cidx[kk] * 16), a, ca, L);
#pragma unroll
                    for (int e = 0; e < VEC; ++e)
                        if (e < nval[kk]) t[e] = ex2_approx(fmaf(pf, L[e], -vh[kk * VEC + e]));
                }
            }
#pragma unroll
            for (int e = 0; e < VEC; e += 2) {
                sp0 = fmaf(t[e], vc[kk * VEC + e], sp0);
                sp1 = fmaf(t[e + 1], vc[kk * VEC + e + 1], sp1);
            }
#pragma unroll
            for (int h = 0; h < VEC / 4; ++h)
                tbuf[((size_t)slot * M4 + kk * (VEC / 4) + h) * NT + tid] =
                    make_float4(t[4 * h], t[4 * h + 1], t[4 * h + 2], t[4 * h + 3]);
        }
        return sp0 + sp1;
    };

    // Stage g = local rows 2g and 2g+1: wait for their bytes, form their terms (tbuf slots
    // 2(g&1) and 2(g&1)+1), and publish the warp's two partial row sums on mrow[g % NRED].
    // Two rows per stage halve the reductions, waits and copy issues per row, and give each
    // warp two independent rows of work to interleave.
    auto produce = [&](int g, float pf) {
        const int q0 = 2 * g;
        const bool two = q0 + 1 < nrows;
        const uint32_t u0 = it + q0;
        bool ok = mbar_wait(&mbar[u0 % RING], (u0 / RING) & 1u, A.err, kWaitTimeoutNs);
        if (two) ok = mbar_wait(&mbar[(u0 + 1) % RING], ((u0 + 1) / RING) & 1u, A.err, kWaitTimeoutNs) && ok;
        if (!ok) s_flag = 1;
        const int ts = (g & 1) * 2;
        const float sp0 = row_terms(ring + (size_t)(u0 % RING) * A.row_bytes, Lr[q0], pf, ts);
        const float sp1 = two ? row_terms(ring + (size_t)((u0 + 1) % RING) * A.row_bytes, Lr[q0 + 1], pf, ts + 1) : 0.0f;
        // this warp is done with the rows' slots (an exact-max redo reads the row from
        // global memory): release them
        __syncwarp();
        if (lane == 0) {
            release_index(u0);
            if (two) release_index(u0 + 1);
        }

        const float w0 = warp_sum(sp0);
        const float w1 = warp_sum(sp1);
        if (lane == 0) {
            const uint32_t gs = gbase + g;   // stage count over all sweeps: mbarrier phase
            red[((gs % NRED) * 2) * NW + wid] = w0;
            red[((gs % NRED) * 2 + 1) * NW + wid] = w1;
            mbar_arrive(&mrow[gs % NRED]);
        }
    };

    // exact max shift for row q (the paper's form), block-wide; terms into tbuf[q & 1]
    auto row_exact = [&](const unsigned char* rowp, float a, float pf, int slot, float* gm_out) -> float {
        float e_loc[M];
        float mx = -INFINITY;
        const float ca = -8388608.0f * a;
#pragma unroll
        for (int kk = 0; kk < CH; ++kk) {
            float L[VEC];
            if (nval[kk] > 0) Vec<WT>::log2w(*(const uint4*)(rowp + (size_t)cidx[kk] * 16), a, ca, L);
#pragma unroll
            for (int e = 0; e < VEC; ++e) {
                const int m = kk * VEC + e;
                float ev = -INFINITY;
                if (e < nval[kk] && vc[m] > 0.0f) ev = fmaf(pf, L[e], -vh[m]) + log2f(vc[m]);
                e_loc[m] = ev;
                mx = fmaxf(mx, ev);
            }
        }
        mx = warp_max(mx);
        __syncthreads();
        if (lane == 0) red2[wid] = mx;
        __syncthreads();
        float gm = -INFINITY;
        for (int x = 0; x < NW; ++x) gm = fmaxf(gm, red2[x]);
        float s2 = 0.0f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            // tbuf holds terms before the column factor: divide it back out
            const float tv = (gm > -INFINITY && vc[m] > 0.0f) ? ex2_approx(e_loc[m] - gm) : 0.0f;
            s2 += tv;
            e_loc[m] = vc[m] > 0.0f ? tv / vc[m] : 0.0f;
        }
#pragma unroll
        for (int m4 = 0; m4 < M4; ++m4)
            tbuf[((size_t)slot * M4 + m4) * NT + tid] =
                make_float4(e_loc[4 * m4], e_loc[4 * m4 + 1], e_loc[4 * m4 + 2], e_loc[4 * m4 + 3]);
        s2 = warp_sum(s2);
        __syncthreads();
        if (lane == 0) red2[wid] = s2;
        __syncthreads();
        float ss = 0.0f;
        for (int x = 0; x < NW; ++x) ss += red2[x];
        *gm_out = gm;
        return ss;
    };

    for (int k = A.k0; k < A.n_p; ++k) {
        const double p = A.P[k];
        const float pf = (float)p;
        // per-step row references: U holds the row potentials reached at p[k-1]
        // (zero on a fresh start), so U/p[k-1] is the per-row level of log2 w
        // (Lr holds the row scale a_i = 2^-(U_i/p[k-1]) as an FP32 number; the row's
        //  potential is recovered exactly as U_i = -p log2(a_i) + log2(s_i) in FP64)
        {
            const double pprev = (k > 0) ? A.P[k - 1] : p;
            for (int q = tid; q < nrows; q += NT) Lr[q] = (float)exp2(-fmin(fmax(A.U[r0 + q] / pprev, -120.0), 120.0));
        }
        __syncthreads();
        load_cols();
        int sweeps = 0;
        float resid = INFINITY;
        bool done = false;
        while (!done) {
            SA_STAMP(0);
#pragma unroll
            for (int m = 0; m < M; ++m) S[m] = 0.0f;
            // ---------------- row pass ----------------
            // Two-stage pipeline without block barriers: a warp forms the terms of row q+1,
            // publishes its partial sum on mrow, then waits for every warp's partial of row
            // q and accumulates row q's normalised terms into its column sums.  NRED = 4
            // buffers: a warp can publish row q+3 only after all warps published q+1, i.e.
            // after they read the sums of row q-1, the last reader of that buffer.
            const int nst = (nrows + 1) / 2;
            if (nst > 0) produce(0, pf);
            for (int g = 0; g < nst; ++g) {
                const int q0 = 2 * g;
                const int nr = min(2, nrows - q0);
                if (g + 1 < nst) produce(g + 1, pf);
                const uint32_t gs = gbase + g;
                if (!mbar_wait(&mrow[gs % NRED], (gs / NRED) & 1u, A.err, kWaitTimeoutNs)) s_flag = 1;
                if (s_flag) break;
                float srs[2];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float4* rv = (const float4*)(red + ((gs % NRED) * 2 + r) * NW);
                    float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
                    for (int x = 0; x < NW / 4; ++x) {
                        const float4 q4 = rv[x];
                        a0 += q4.x + q4.y;
                        a1 += q4.z + q4.w;
                    }
                    srs[r] = a0 + a1;
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    if (r >= nr || (srs[r] >= 0x1p-64f && srs[r] <= 0x1p64f)) continue;
                    // the stale shift left the range (uniform decision): exact max shift
                    const int q = q0 + r;
                    const float ar = Lr[q];
                    float gm;
                    float ss = row_exact(wbase + (size_t)(r0 + q) * pitch, ar, pf, (g & 1) * 2 + r, &gm);
                    if (!(gm > -INFINITY) || !(ss > 0.0f)) {
                        if (tid == 0) atomicCAS(A.err, 0, kErrNonfinite);
                        ss = 1.0f;
                        gm = 0.0f;
                    }
                    srs[r] = -ss;   // marks a re-anchored row (negative: srow already set)
                    if (tid == 0) {
                        // re-anchor the row scale at the exact row potential
                        const double un = -p * log2((double)ar) + (double)gm + log2((double)ss);
                        const float an = (float)exp2(-un / p);
                        Lr[q] = an;
                        srow[q] = (float)exp2(un + p * log2((double)an));
                        atomicAdd(A.fallback, 1);
                    }
                    __syncthreads();
                }
                if (tid == 0) {
                    for (int r = 0; r < nr; ++r)
                        if (srs[r] > 0.0f) srow[q0 + r] = srs[r];
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    if (r >= nr) break;
                    const float inv = rcp_approx(fabsf(srs[r]));
                    const float4* tb = tbuf + (size_t)((g & 1) * 2 + r) * M4 * NT + tid;
#pragma unroll
                    for (int m4 = 0; m4 < M4; ++m4) {
                        const float4 t4 = tb[(size_t)m4 * NT];
                        S[4 * m4] = fmaf(t4.x, inv, S[4 * m4]);
                        S[4 * m4 + 1] = fmaf(t4.y, inv, S[4 * m4 + 1]);
                        S[4 * m4 + 2] = fmaf(t4.z, inv, S[4 * m4 + 2]);
                        S[4 * m4 + 3] = fmaf(t4.w, inv, S[4 * m4 + 3]);
                    }
                }
            }
            __syncthreads();
            if (s_flag) { drain(); return; }
            it += nrows;
            gbase += (nrows + 1) / 2;
            SA_STAMP(1);
            float* pb = A.part + (size_t)b * A.npad;
#pragma unroll
            for (int kk = 0; kk < CH; ++kk) {
                if (nval[kk] > 0) {
#pragma unroll
                    for (int e = 0; e < VEC; e += 4)
                        *(float4*)(pb + (size_t)cidx[kk] * VEC + e) =
                            make_float4(S[kk * VEC + e] * vc[kk * VEC + e], S[kk * VEC + e + 1] * vc[kk * VEC + e + 1],
                                        S[kk * VEC + e + 2] * vc[kk * VEC + e + 2],
                                        S[kk * VEC + e + 3] * vc[kk * VEC + e + 3]);
                }
            }
            ++sweeps;
            if (!gsync()) { drain(); return; }
            SA_STAMP(2);
            // ---------------- column finalisation of columns [c0, c1) ----------------
            float* rmax_word = A.rmax + ((sweeps + rphase) & 1);
            float rmax = 0.0f;
            for (int cb = c0; cb < c1; cb += 64) {
                const int j = cb + (tid & 63);
                const int grp = tid >> 6;
                KahanF acc;
                if (j < c1) {
                    const float* pj = A.part + j;
                    for (int g0 = grp; g0 < G; g0 += FG * 20) {
                        float a[20];
#pragma unroll
                        for (int x = 0; x < 20; ++x) {
                            const int g = g0 + x * FG;
                            a[x] = g < G ? __ldcg(pj + (size_t)g * A.npad) : 0.0f;
                        }
#pragma unroll
                        for (int x = 0; x < 20; ++x) acc.add(a[x]);
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
                        // log2(1 + d) by its series, FP64 (|d| < 1e-3: 5 terms reach 1e-17)
                        lg = d * (1.0 + d * (-0.5 + d * (1.0 / 3.0 + d * (-0.25 + d * 0.2)))) * kLog2e;
                    } else {
                        lg = log2(Sj);
                    }
                    double v = A.V[j] + lg;
                    if (A.f32_potentials) v = (double)(float)v;
                    A.V[j] = v;
                    float h = A.Vh[j];
                    if (A.f32_potentials || fabs((double)h - v) > 16.0) { h = (float)v; A.Vh[j] = h; }
                    A.Vc[j] = ex2_approx((float)((double)h - v));
                }
                __syncthreads();
            }
            if (wid < 2) {
                rmax = warp_max(rmax);
                if (lane == 0 && rmax > 0.0f) atomicMax((unsigned*)rmax_word, __float_as_uint(rmax));
            }
            if (!gsync()) { drain(); return; }
            SA_STAMP(3);
            // ---------------- decision (identical in every block) ----------------
            if (tid == 0) {
                s_res = __uint_as_float(ld_acquire((const unsigned*)rmax_word));
                if (b == 0) A.rmax[((sweeps + rphase) + 1) & 1] = 0.0f;   // next sweep's word
            }
            __syncthreads();
            resid = s_res;
            done = (resid <= A.tol) || (sweeps >= A.max_sweeps);
            if (!done) load_cols();
            SA_STAMP(4);
        }
        rphase += sweeps;
        for (int q = tid; q < nrows; q += NT) {
            double uu = -p * log2((double)Lr[q]) + log2((double)srow[q]);
            if (A.f32_potentials) uu = (double)(float)uu;
            A.U[r0 + q] = uu;
        }
        if (b == 0 && tid == 0) {
            A.sweeps_out[k] = sweeps;
            A.resid_out[k] = resid;
        }
        if (k + 1 < A.n_p) {
            // warm start of the next step: (U, V) *= p_{k+1}/p_k unless v is kept
            const double f = A.keep_v ? 1.0 : A.P[k + 1] / p;
            for (int j = c0 + tid; j < c1; j += NT) {
                double v = A.V[j] * f;
                A.V[j] = v;
                float h = (float)v;
                A.Vh[j] = h;
                A.Vc[j] = ex2_approx((float)((double)h - v));
            }
            if (!gsync()) { drain(); return; }
        }
    }
    drain();
}

template <typename WT, int NT, int CH, int RING, int R>
sa_status launch_fused(sa_ctx* ctx, const FusedArgs& args, size_t smem, int* grid_out) {
    auto kern = fused_kernel<WT, NT, CH, RING, R>;
    SA_CUDA(allow_dynamic_smem(kern, ctx->smem_optin));
    int per_sm = 0;
    SA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem));
    if (per_sm < 1) {
        set_error("fused sweep: kernel does not fit on an SM (smem %zu)", smem);
        return SA_E_UNSUPPORTED;
    }
    int G = ctx->num_sms * per_sm;
    // at least 8 rows per block (fewer blocks share each barrier for small n)
    const int gmax_rows = args.n / 8 > 0 ? args.n / 8 : 1;
    if (G > gmax_rows) G = gmax_rows;
    if (*grid_out > 0 && *grid_out < G) G = *grid_out;
    if ((args.n + G - 1) / G > args.max_rows) {
        set_error("fused sweep: grid of %d blocks leaves stripes longer than %d rows", G, args.max_rows);
        return SA_E_UNSUPPORTED;
    }
    *grid_out = G;
    FusedArgs a = args;
    void* params[] = {&a};
    SA_CUDA(cudaLaunchCooperativeKernel((const void*)kern, dim3(G), dim3(NT), params, smem, ctx->stream));
    count_launch();
    return SA_OK;
}

struct FusedCfg {
    int nt, ch, ring, r;
};

#ifndef SA_ROWS_PER_SYNC
#define SA_ROWS_PER_SYNC 2
#endif
constexpr int kRowsPerSync = SA_ROWS_PER_SYNC;

size_t fused_smem_bytes(const FusedCfg& c, unsigned row_bytes, int vec, int max_rows) {
    const int nw = c.nt / 32;
    const int m4 = c.ch * vec / 4;
    const size_t head = (size_t)c.ring * row_bytes + 8 * (size_t)(2 * c.ring + 4 + ((2 * c.ring + 4) & 1));
    const size_t fg = c.nt / 64;
    // + 1 KiB for the kernel's static shared variables and alignment
    return head + 16 * (size_t)4 * m4 * c.nt + 4 * (size_t)(8 * nw + nw + 2 * max_rows) + 8 + 8 * fg * 64 + 1024;
}

// nt_pref: threads per block for 512 < chunks <= 1024 (256 x 4 or 512 x 2 chunks)
FusedCfg pick_cfg(const sa_matrix* a, size_t smem_optin, int max_rows, int nt_pref = 512) {
    const int vec = 16 / wbytes(a->wtype);
    const int nc = (a->n + vec - 1) / vec;
    FusedCfg c{0, 0, 0, kRowsPerSync};
    if (nc <= 128) c = {128, 1, 0, kRowsPerSync};
    else if (nc <= 256) c = {256, 1, 0, kRowsPerSync};
    else if (nc <= 512) c = {512, 1, 0, kRowsPerSync};
    else if (nc <= 1024) {
        if (nt_pref == 256) c = {256, 4, 0, kRowsPerSync};
        else c = {512, 2, 0, kRowsPerSync};
    } else return c;
    const unsigned row_bytes = (unsigned)align_up((size_t)a->n * wbytes(a->wtype), 16);
    for (int ring : {6, 5, 4}) {
        c.ring = ring;
        if (fused_smem_bytes(c, row_bytes, vec, max_rows) <= smem_optin) return c;
    }
    c.nt = 0;
    return c;
}

int fused_max_rows(const sa_ctx* ctx, int n) {
    // any grid has >= min(num_sms, n/8, max_grid) blocks, so no stripe exceeds this many rows
    int gmin = std::max(1, std::min(ctx->num_sms, n / 8));
    if (ctx->max_grid > 0) gmin = std::max(1, std::min(gmin, ctx->max_grid));
    return (n + gmin - 1) / gmin + 1;
}

}  // namespace

bool fused_supported(const sa_ctx* ctx, const sa_matrix* a) {
    const int sz = wbytes(a->wtype);
    if (((uintptr_t)a->w & 15) != 0) return false;
    if (((size_t)a->ld * sz) % 16 != 0) return false;
    if ((size_t)a->ld * sz < align_up((size_t)a->n * sz, 16)) return false;
    return pick_cfg(a, ctx->smem_optin, fused_max_rows(ctx, a->n)).nt > 0;
}

sa_status scale_fused(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* o, double* U,
                      double* V, sa_scale_info* info) {
    const int n = a->n;
    const int max_rows = fused_max_rows(ctx, n);
    FusedCfg cfg = pick_cfg(a, ctx->smem_optin, max_rows, ctx->fused_nt);
    if (cfg.nt == 0) {
        set_error("fused sweep: n=%d not supported by the fused kernel", n);
        return SA_E_UNSUPPORTED;
    }
    cudaStream_t st = ctx->stream;
    const int G_max = ctx->num_sms * 2;
    const int npad = (int)align_up((size_t)n, 32);
    size_t need = (size_t)G_max * npad * 4 + (size_t)G_max * 8 + 2 * align_up((size_t)n * 4, 256) +
                  (size_t)o->n_p * 16 + 8192;
    sa_status rc = ctx->ws.reserve(need);
    if (rc) return rc;
    Carve cv(ctx->ws.ptr);
    float* part = cv.take<float>((size_t)G_max * npad);
    float* rmax = cv.take<float>(2);
    float* Vh = cv.take<float>(n);
    float* Vc = cv.take<float>(n);
    double* P = cv.take<double>(o->n_p);
    double* resid_out = cv.take<double>(o->n_p);
    int* sweeps_out = cv.take<int>(o->n_p);
    unsigned* bar = cv.take<unsigned>(2);
    int* err = cv.take<int>(1);
    int* fallback = cv.take<int>(1);
    SA_CUDA(cudaMemcpyAsync(P, o->p, o->n_p * sizeof(double), cudaMemcpyHostToDevice, st));
    SA_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
    SA_CUDA(cudaMemsetAsync(rmax, 0, 2 * sizeof(float), st));
    SA_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    SA_CUDA(cudaMemsetAsync(fallback, 0, sizeof(int), st));
    SA_CUDA(cudaMemsetAsync(sweeps_out, 0, o->n_p * sizeof(int), st));
    const int k0 = o->resume_from > 0 ? o->resume_from : 0;
    if (k0 == 0) {
        SA_CUDA(cudaMemsetAsync(U, 0, n * sizeof(double), st));
        SA_CUDA(cudaMemsetAsync(V, 0, n * sizeof(double), st));
    } else if (!o->warm_keep_v) {
        // warm start from step k0-1: scale to p[k0]; the kernel's first-step row
        // reference divides U by p[k0-1] (the unscaled value), so scale V only.
        launch_scale_vec(V, n, o->p[k0] / o->p[k0 - 1], st);
    }
    // Vh = float(V), Vc = 2^(Vh - V)
    launch_split_v(V, Vh, Vc, n, st);
    FusedArgs args{};
    args.w = a->w;
    args.n = n;
    args.ld = a->ld;
    args.row_bytes = (unsigned)align_up((size_t)n * wbytes(a->wtype), 16);
    args.P = P;
    args.k0 = k0;
    args.n_p = o->n_p;
    args.tol = o->tol;
    args.max_sweeps = o->max_sweeps_per_p;
    args.keep_v = o->warm_keep_v;
    args.f32_potentials = o->prec == SA_PREC_FP32;
    args.U = U;
    args.V = V;
    args.Vh = Vh;
    args.Vc = Vc;
    args.part = part;
    args.npad = npad;
    args.rmax = rmax;
    args.bar = bar;
    args.err = err;
    args.fallback = fallback;
    args.sweeps_out = sweeps_out;
    args.resid_out = resid_out;
    args.max_rows = max_rows;
    const size_t smem = fused_smem_bytes(cfg, args.row_bytes, 16 / wbytes(a->wtype), max_rows);
    int G = ctx->max_grid > 0 ? std::min(G_max, ctx->max_grid) : G_max;
    const bool i16 = a->wtype == SA_I16;
    cudaEvent_t ev0, ev1;
    SA_CUDA(cudaEventCreate(&ev0));
    SA_CUDA(cudaEventCreate(&ev1));
    SA_CUDA(cudaEventRecord(ev0, st));
#define SA_LAUNCH(NT_, CH_, RING_)                                                              \
    rc = i16 ? launch_fused<int16_t, NT_, CH_, RING_, kRowsPerSync>(ctx, args, smem, &G)       \
             : launch_fused<int32_t, NT_, CH_, RING_, kRowsPerSync>(ctx, args, smem, &G)
    if (cfg.ring == 6) {
        if (cfg.nt == 128) SA_LAUNCH(128, 1, 6);
        else if (cfg.nt == 256 && cfg.ch == 1) SA_LAUNCH(256, 1, 6);
        else if (cfg.nt == 256) SA_LAUNCH(256, 4, 6);
        else if (cfg.ch == 1) SA_LAUNCH(512, 1, 6);
        else SA_LAUNCH(512, 2, 6);
    } else if (cfg.ring == 5) {
        if (cfg.nt == 256) SA_LAUNCH(256, 4, 5);
        else SA_LAUNCH(512, 2, 5);
    } else {
        if (cfg.nt == 256) SA_LAUNCH(256, 4, 4);
        else SA_LAUNCH(512, 2, 4);
    }
#undef SA_LAUNCH
    if (rc) { cudaEventDestroy(ev0); cudaEventDestroy(ev1); return rc; }
    SA_CUDA(cudaEventRecord(ev1, st));
    // results
    sa_status prc = ctx->pinned.reserve(4096 + (size_t)o->n_p * 16);
    if (prc) return prc;
    char* hp = (char*)ctx->pinned.ptr;
    int* h_err = (int*)hp;
    int* h_fb = (int*)(hp + 8);
    int* h_sw = (int*)(hp + 64);
    double* h_rs = (double*)(hp + 64 + align_up((size_t)o->n_p * 4, 64));
    SA_CUDA(cudaMemcpyAsync(h_err, err, 4, cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(h_fb, fallback, 4, cudaMemcpyDeviceToHost, st));
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
        info->fallback_rows = *h_fb;
        info->kernel_used = SA_KERNEL_FUSED;
        info->kernel_ms = kms;
    }
    if (*h_err == kErrTimeout) {
        set_error("fused sweep: a bounded device wait timed out (grid of %d blocks)", G);
        return SA_E_TIMEOUT;
    }
    if (*h_err == kErrNonfinite) {
        set_error("fused sweep: a row or column lost all mass (matrix without support?)");
        return SA_E_NONFINITE;
    }
    return conv ? SA_OK : SA_E_NOT_CONVERGED;
}

__global__ void split_v_kernel(const double* V, float* Vh, float* Vc, int n) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) {
        double v = V[j];
        float h = (float)v;
        Vh[j] = h;
        Vc[j] = ex2_approx((float)((double)h - v));
    }
}

void launch_split_v(const double* V, float* Vh, float* Vc, int n, cudaStream_t s) {
    if (n > 0) split_v_kernel<<<(n + 255) / 256, 256, 0, s>>>(V, Vh, Vc, n);
    count_launch();
}

}  // namespace sa

// ---------------------------------------------------------------------------------------
// Allocation-free variant of the fused scaling (sa_scale_noalloc).
//
// Some callers cannot allocate device memory at the point where they need a scaling:
// their device memory is planned up front (a fixed budget, a pre-sized pool, an
// allocator that must not grow), or they cannot take the device-wide synchronisation
// that cudaMalloc and cudaFree bring.  For them the scratch of the fused kernel (column
// partials, the FP32 head/factor of V, the schedule, barrier and status words, and a copy
// of the caller's warm-start potentials) lives in this file-scope device array instead
// of a context workspace.  Every device that loads the library holds the array until
// the process exits.  All calls share it: two calls whose work overlaps on the GPU race
// on it and must be serialised by the caller (one stream, or events).
// ---------------------------------------------------------------------------------------
namespace sa {
namespace {

constexpr int kNoAllocMaxN = 4096;      // largest n accepted
constexpr int kNoAllocMaxGrid = 160;    // grid cap (one block per SM on GB300: 152)
constexpr int kNoAllocMaxSteps = 64;    // longest p schedule accepted
constexpr size_t kNoAllocPartFloats = (size_t)kNoAllocMaxGrid * kNoAllocMaxN;
constexpr size_t kNoAllocBytes =
    kNoAllocPartFloats * 4 + 2 * (size_t)kNoAllocMaxN * 4 + 2 * (size_t)kNoAllocMaxSteps * 8 +
    (size_t)kNoAllocMaxSteps * 4 + 256 * 4 + 2 * (size_t)kNoAllocMaxN * 8;   // about 2.7 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
    bool ready = false;
    unsigned char* scratch = nullptr;   // device address of g_noalloc_scratch on this device
    int num_sms = 0;
    size_t smem_optin = 0;
};
std::mutex g_noalloc_mu;
NoAllocDevice g_noalloc_dev[64];

}  // namespace

}  // namespace sa

using namespace sa;

extern "C" sa_status sa_scale_noalloc(const sa_matrix* a, const sa_scale_opts* o, void* cuda_stream, double* d_u,
                                      double* d_v, sa_scale_info* info) {
    if (!a || !a->w || !o || !o->p || !d_u || !d_v) { set_error("null argument"); return SA_E_INVALID; }
    if (a->n <= 0 || a->ld < a->n || (a->wtype != SA_I16 && a->wtype != SA_I32)) { set_error("bad matrix"); return SA_E_INVALID; }
    if (a->n > kNoAllocMaxN) {
        set_error("sa_scale_noalloc: n=%d exceeds the static scratch limit n <= %d", a->n, kNoAllocMaxN);
        return SA_E_UNSUPPORTED;
    }
    if (o->n_p <= 0 || o->n_p > kNoAllocMaxSteps) {
        set_error("sa_scale_noalloc: schedule of %d steps (1..%d supported)", o->n_p, kNoAllocMaxSteps);
        return o->n_p <= 0 ? SA_E_INVALID : SA_E_UNSUPPORTED;
    }
    for (int k = 0; k < o->n_p; ++k)
        if (!(o->p[k] > 0) || !std::isfinite(o->p[k]) || (k > 0 && !(o->p[k] > o->p[k - 1]))) {
            set_error("p schedule must be finite, positive and increasing");
            return SA_E_INVALID;
        }
    if (!(o->tol > 0) || o->max_sweeps_per_p <= 0 || o->resume_from < 0 || o->resume_from >= o->n_p ||
        o->prec == SA_PREC_FP64) {
        set_error("sa_scale_noalloc: bad tol/cap/resume or FP64 precision (fused kernel only)");
        return SA_E_INVALID;
    }
    int dev = 0;
    SA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("device index %d out of range", dev); return SA_E_INVALID; }
    NoAllocDevice nd;
    {
        // once per device, with that device current: the device address of the array
        std::lock_guard<std::mutex> g(g_noalloc_mu);
        NoAllocDevice& d = g_noalloc_dev[dev];
        if (!d.ready) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
            cudaDeviceProp prop;
            e = cudaGetDeviceProperties(&prop, dev);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
            d.scratch = (unsigned char*)ptr;
            d.num_sms = prop.multiProcessorCount;
            d.smem_optin = prop.sharedMemPerBlockOptin;
            d.ready = true;
        }
        nd = d;
    }
    // a context on the stack: no workspace is reserved through it
    sa_ctx ctx;
    ctx.device = dev;
    ctx.stream = (cudaStream_t)cuda_stream;
    ctx.num_sms = nd.num_sms;
    ctx.smem_optin = nd.smem_optin;
    ctx.max_grid = kNoAllocMaxGrid;
    const int n = a->n;
    if (!fused_supported(&ctx, a)) {
        set_error("sa_scale_noalloc: layout not supported by the fused kernel (16-byte aligned rows needed)");
        return SA_E_UNSUPPORTED;
    }
    const int max_rows = fused_max_rows(&ctx, n);
    FusedCfg cfg = pick_cfg(a, ctx.smem_optin, max_rows, 512);
    cudaStream_t st = ctx.stream;
    const int npad = (int)align_up((size_t)n, 32);
    // carve the static array
    unsigned char* base = nd.scratch;
    float* part = (float*)base;
    float* Vh = part + kNoAllocPartFloats;
    float* Vc = Vh + kNoAllocMaxN;
    double* P = (double*)(Vc + kNoAllocMaxN);
    double* resid_out = P + kNoAllocMaxSteps;
    int* sweeps_out = (int*)(resid_out + kNoAllocMaxSteps);
    unsigned* words = (unsigned*)(sweeps_out + kNoAllocMaxSteps);   // bar[2], err, fallback, rmax[2]
    unsigned* bar = words;
    int* err = (int*)(words + 2);
    int* fallback = (int*)(words + 3);
    float* rmax = (float*)(words + 4);
    double* keep_u = (double*)(words + 256);   // the caller's warm start, restored on failure
    double* keep_v = keep_u + kNoAllocMaxN;
    if ((size_t)npad * kNoAllocMaxGrid > kNoAllocPartFloats) { set_error("scratch too small"); return SA_E_UNSUPPORTED; }
    const int k0 = o->resume_from;
    // a failure after this point puts the caller's potentials back as they were given
    auto restore = [&](sa_status rc) -> sa_status {
        if (k0 > 0) {
            cudaMemcpyAsync(d_u, keep_u, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(d_v, keep_v, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
            cudaStreamSynchronize(st);
        }
        return rc;
    };
    // the previous call's contents stay in the array: clear what must start at zero, and
    // mark every step's residual unknown (NaN) until the kernel writes it
    SA_CUDA(cudaMemcpyAsync(P, o->p, o->n_p * sizeof(double), cudaMemcpyHostToDevice, st));
    SA_CUDA(cudaMemsetAsync(words, 0, 8 * sizeof(unsigned), st));
    SA_CUDA(cudaMemsetAsync(sweeps_out, 0, o->n_p * sizeof(int), st));
    SA_CUDA(cudaMemsetAsync(resid_out, 0xFF, o->n_p * sizeof(double), st));
    if (k0 > 0) {
        SA_CUDA(cudaMemcpyAsync(keep_u, d_u, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        SA_CUDA(cudaMemcpyAsync(keep_v, d_v, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        launch_scale_vec(d_u, n, kLog2e, st);
        launch_scale_vec(d_v, n, kLog2e, st);
        if (!o->warm_keep_v) launch_scale_vec(d_v, n, o->p[k0] / o->p[k0 - 1], st);
    } else {
        SA_CUDA(cudaMemsetAsync(d_u, 0, n * sizeof(double), st));
        SA_CUDA(cudaMemsetAsync(d_v, 0, n * sizeof(double), st));
    }
    launch_split_v(d_v, Vh, Vc, n, st);
    FusedArgs args{};
    args.w = a->w;
    args.n = n;
    args.ld = a->ld;
    args.row_bytes = (unsigned)align_up((size_t)n * wbytes(a->wtype), 16);
    args.P = P;
    args.k0 = k0;
    args.n_p = o->n_p;
    args.tol = o->tol;
    args.max_sweeps = o->max_sweeps_per_p;
    args.keep_v = o->warm_keep_v;
    args.f32_potentials = o->prec == SA_PREC_FP32;
    args.U = d_u;
    args.V = d_v;
    args.Vh = Vh;
    args.Vc = Vc;
    args.part = part;
    args.npad = npad;
    args.rmax = rmax;
    args.bar = bar;
    args.err = err;
    args.fallback = fallback;
    args.sweeps_out = sweeps_out;
    args.resid_out = resid_out;
    args.max_rows = max_rows;
    const size_t smem = fused_smem_bytes(cfg, args.row_bytes, 16 / wbytes(a->wtype), max_rows);
    int G = kNoAllocMaxGrid;
    const bool i16 = a->wtype == SA_I16;
    sa_status rc;
    // n <= 4096: int16 has at most 512 chunks (one per thread), int32 up to 1024 (512 x 2)
    if (cfg.nt == 128) rc = i16 ? launch_fused<int16_t, 128, 1, 6, kRowsPerSync>(&ctx, args, smem, &G)
                                : launch_fused<int32_t, 128, 1, 6, kRowsPerSync>(&ctx, args, smem, &G);
    else if (cfg.nt == 256) rc = i16 ? launch_fused<int16_t, 256, 1, 6, kRowsPerSync>(&ctx, args, smem, &G)
                                     : launch_fused<int32_t, 256, 1, 6, kRowsPerSync>(&ctx, args, smem, &G);
    else if (cfg.ch == 1) rc = i16 ? launch_fused<int16_t, 512, 1, 6, kRowsPerSync>(&ctx, args, smem, &G)
                                   : launch_fused<int32_t, 512, 1, 6, kRowsPerSync>(&ctx, args, smem, &G);
    else if (cfg.ring == 6) rc = i16 ? launch_fused<int16_t, 512, 2, 6, kRowsPerSync>(&ctx, args, smem, &G)
                                     : launch_fused<int32_t, 512, 2, 6, kRowsPerSync>(&ctx, args, smem, &G);
    else if (cfg.ring == 5) rc = i16 ? launch_fused<int16_t, 512, 2, 5, kRowsPerSync>(&ctx, args, smem, &G)
                                     : launch_fused<int32_t, 512, 2, 5, kRowsPerSync>(&ctx, args, smem, &G);
    else rc = i16 ? launch_fused<int16_t, 512, 2, 4, kRowsPerSync>(&ctx, args, smem, &G)
                  : launch_fused<int32_t, 512, 2, 4, kRowsPerSync>(&ctx, args, smem, &G);
    if (rc) return restore(rc);
    // results through pageable host memory (no pinned allocation)
    int h_words[4] = {0, 0, 0, 0};
    int h_sw[kNoAllocMaxSteps];
    double h_rs[kNoAllocMaxSteps];
    SA_CUDA(cudaMemcpyAsync(h_words, words, sizeof(h_words), cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(h_sw, sweeps_out, o->n_p * sizeof(int), cudaMemcpyDeviceToHost, st));
    SA_CUDA(cudaMemcpyAsync(h_rs, resid_out, o->n_p * sizeof(double), cudaMemcpyDeviceToHost, st));
    launch_scale_vec(d_u, n, kLn2, st);
    launch_scale_vec(d_v, n, kLn2, st);
    SA_CUDA(cudaStreamSynchronize(st));
    int64_t total = 0;
    // a step the kernel did not finish keeps its NaN residual, so it never counts as converged
    int conv = h_words[2] == 0;
    for (int k = k0; k < o->n_p; ++k) {
        total += h_sw[k];
        if (!(h_rs[k] <= o->tol)) conv = 0;
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->sweeps_total = total;
        info->residual = h_rs[o->n_p - 1];
        info->p_final = o->p[o->n_p - 1];
        info->converged = conv;
        info->steps_done = o->n_p - k0;
        info->fallback_rows = h_words[3];
        info->kernel_used = SA_KERNEL_FUSED;
        info->kernel_ms = 0.0;
    }
    if (h_words[2] == kErrTimeout) { set_error("sa_scale_noalloc: a bounded device wait timed out"); return restore(SA_E_TIMEOUT); }
    if (h_words[2] == kErrNonfinite) { set_error("sa_scale_noalloc: a row or column lost all mass"); return restore(SA_E_NONFINITE); }
    return conv ? SA_OK : SA_E_NOT_CONVERGED;
}

