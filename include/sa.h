/*
 * sa.h -- C ABI of libsa: Sinkhorn diagonal-scaling preprocessing for the optimal
 * assignment problem on one GB300 GPU (sm_103a).
 *
 * Method: Sharify, Gaubert, Grigori, "Solution of the optimal assignment problem by
 * diagonal scaling algorithms", arXiv:1104.3830.  Given an n x n non-negative matrix A,
 * find a permutation sigma maximising prod_i a_{i sigma(i)} (Sec. 2.2).  The library
 * scales the Hadamard power A^(p) = (a_ij^p) to the bistochastic matrix X(p) of maximal
 * entropy (Eq. pentropyopt, Thm. prop-borweinlewisnussbaum) with the log-domain Sinkhorn
 * iteration (Sec. 4.1.2) under an increasing p schedule, deletes the entries with
 * x_ij(p) < t (Eq. matrixred), compacts the survivors into CSR, solves that reduced
 * instance exactly and proves the result optimal for A by LP duality.
 *
 * Conventions used by every entry point.
 *  - Weights are integers w_ij >= 0 with a_ij = w_ij; w = 0 marks a forbidden entry
 *    (b_ij = log a_ij = -inf, Eq. pentropyopt).  int16 weights must be <= 32767.
 *  - Matrices are row-major on the device with a leading dimension ld >= n (elements).
 *    The fused kernels need ld * sizeof(weight) to be a multiple of 16 bytes and the base
 *    16-byte aligned; other layouts run on the plain kernels.
 *  - Potentials are FP64 natural-log vectors u (rows) and v (columns) with
 *        x_ij(p) = exp(p * log w_ij - u_i - v_j),
 *    i.e. u_i = -log (D_r)_ii and v_j = -log (D_c)_jj for X(p) = D_r A^(p) D_c; in the
 *    paper's log coordinates (Sec. 4.1.2) u = -p * ubar and v = -p * vbar.  (u + c, v - c)
 *    describe the same X (P gauge), so compare X or u_i + v_j, never raw u or v.
 *  - All device work of a context runs in order on the context's CUDA stream.  Calls
 *    that return host results synchronise that stream before returning.
 *  - Errors are returned as sa_status codes; nothing crosses the ABI as an exception.
 *    sa_last_error() gives a message for the calling thread's last failure.
 *  - Pointers named d_* are device pointers; all others are host pointers.  Unless a
 *    comment says otherwise the caller owns every buffer it passes.
 */
#ifndef SA_H
#define SA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SA_OK = 0,
    SA_PENDING = 1,               /* sa_poll: the request is not finished yet */
    SA_E_INVALID = -1,            /* bad argument (null pointer, n <= 0, bad schedule, ...) */
    SA_E_NOMEM = -2,              /* device or host allocation failed */
    SA_E_CUDA = -3,               /* a CUDA call failed; sa_last_error has the CUDA message */
    SA_E_NOT_CONVERGED = -4,      /* some p step hit max_sweeps_per_p before tol */
    SA_E_NO_PERFECT_MATCHING = -5,/* the allowed entries contain no permutation */
    SA_E_NONFINITE = -6,          /* a row or column lost all mass (no support, Sec. 2.1) */
    SA_E_BUDGET = -7,             /* request larger than the server's memory budget */
    SA_E_TIMEOUT = -8,            /* a bounded device wait gave up (kernel returned early) */
    SA_E_UNSUPPORTED = -9         /* valid request the library does not support (e.g. n too large) */
} sa_status;

typedef enum { SA_I16 = 0, SA_I32 = 1 } sa_wtype;

/* Arithmetic of the sweeps.  MIXED: per-element FP32 (exp2/log2 on the SFU), potentials
 * and stopping residual in FP64.  FP32: potentials in FP32 as well.  FP64: every step
 * in FP64 (slow on GB300; a reference for the error of the other two). */
typedef enum { SA_PREC_MIXED = 0, SA_PREC_FP32 = 1, SA_PREC_FP64 = 2 } sa_prec;

/* Which sweep implementation sa_scale uses.
 * FUSED: one persistent cooperative kernel runs the whole schedule, one read of the
 *   integer matrix per sweep, exp2/log2 of every element on the SFU in FP32.  The SFU
 *   logarithm's absolute error (about 2^-21) is multiplied by p in the exponent, so the
 *   FP64-checked row and column sums of the result are off by about 1.3e-7 p.
 * PLAIN: separate row and column kernels per sweep launched from the host (two reads of
 *   the matrix per sweep), the comparison path; the only path for SA_PREC_FP64.
 * STEP: one persistent cooperative kernel; at the start of every p step it evaluates
 *   K = 2^(p log2 w - C_i - V_j) once (exponent in float-pair arithmetic, log2 w to about
 *   2^-40, one SFU exp2) into a workspace of n * ceil(n/4)*4 floats, and each sweep reads K once
 *   (4 bytes per element): no per-element SFU work in the sweeps and an error that does
 *   not grow with p.  The first evaluation of a call also keeps log2 w as a float pair
 *   (8 bytes per element), which the later ones read instead of the weights.  Needs
 *   n <= 24576 (above 12288 the shared-memory ring holds one row per stage).
 * NEWTON: the Newton variant of Sec. 5.3 (Knight-Ruiz iteration on the symmetric
 *   embedding S = [[0, A], [A^T, 0]], conjugate gradients for each Newton system).  At
 *   every p step it evaluates the same K as STEP, then iterates on K; each CG iteration
 *   and each residual check reads K once.  sweeps_total counts these operator
 *   applications (the paper's "No.it." of Tables 2-3), and the stop test is
 *   max(|row sum - 1|, |column sum - 1|) <= tol over rows and columns.  SA_PREC_MIXED
 *   only; same layout needs as STEP; never chosen by AUTO.
 * AUTO: STEP for SA_PREC_MIXED when it applies, else FUSED when it applies, else PLAIN;
 *   PLAIN for SA_PREC_FP64. */
typedef enum { SA_KERNEL_AUTO = 0, SA_KERNEL_FUSED = 1, SA_KERNEL_PLAIN = 2, SA_KERNEL_STEP = 3,
               SA_KERNEL_NEWTON = 4 } sa_kernel;

/* A device matrix: w points to n rows of ld weights of type wtype. */
typedef struct {
    const void* w;
    sa_wtype wtype;
    int32_t n;
    int64_t ld;
} sa_matrix;

/* Options of the scaling phase (Sec. 4.2, Algorithm 1 with a fixed schedule). */
typedef struct {
    const double* p;          /* host array of n_p strictly increasing values > 0 */
    int32_t n_p;
    double tol;               /* eps of the eps-bistochastic stop (Sec. 4.2), per p step */
    int32_t max_sweeps_per_p; /* cap per p step; reaching it sets converged = 0 */
    sa_prec prec;
    sa_kernel kernel;
    int32_t warm_keep_v;      /* 0: multiply (u, v) by p_k / p_{k-1} between steps;
                                 1: keep v as the deformed iteration of Sec. 3.2 does */
    int32_t resume_from;      /* 0: start from v = 0 (v_0 = 1, Eq. dad1);  k > 0: d_u, d_v
                                 hold potentials reached at p[k-1]; run steps k..n_p-1 */
} sa_scale_opts;

typedef struct {
    int64_t sweeps_total;     /* sweeps over all steps run by this call */
    double residual;          /* last stopping residual, max_j |c_j - 1| (FP64) */
    double p_final;           /* p of the last step run */
    int32_t converged;        /* 1 if every step reached tol */
    int32_t steps_done;
    int32_t fallback_rows;    /* rows recomputed with an exact max shift (range guard) */
    int32_t kernel_used;      /* sa_kernel actually used */
    double kernel_ms;         /* device time of the sweep kernels (CUDA events on the
                                 context stream), excluding set-up and unit conversion */
    int32_t sparse_epochs;    /* STEP: evaluations of K whose sweeps ran on the entries
                                 >= 2^-70 of their row only (0 for the other kernels) */
    int32_t reanchors;        /* STEP: re-evaluations of K within a p step because the
                                 column factors spread beyond 2^20 in a sparse epoch */
} sa_scale_info;

/* Reduced instance B in CSR (Eq. matrixred).  Arrays are host memory owned by the
 * library: release them with sa_csr_free.  Columns ascend within each row; w holds the
 * original weights. */
typedef struct {
    int32_t n;
    int64_t nnz;
    int64_t* row_ptr;         /* n + 1 */
    int32_t* col;             /* nnz */
    int32_t* w;               /* nnz */
} sa_csr;

typedef struct sa_ctx sa_ctx;

/* Create a context on CUDA device `device` using stream `cuda_stream` (a cudaStream_t,
 * NULL for the legacy default stream).  The context owns a growing device workspace. */
sa_status sa_create(sa_ctx** ctx, int device, void* cuda_stream);
void sa_destroy(sa_ctx* ctx);

/* Options of a context (deployment settings; the paper has no counterpart).  Each applies
 * to the calls made on the context after it is set. */
typedef enum {
    SA_OPT_WAIT_LIMIT_NS = 0, /* limit in ns of each grid barrier and ring wait of the STEP
                                 kernel's evaluations of K and sweeps (default 2e9, i.e. 2 s;
                                 >= 0; a wait checks its clock every few dozen polls, so a
                                 wait shorter than that never runs out).  A wait that runs out makes the kernel record the
                                 failure, wait (up to 2 s) for its own copies in flight and
                                 return: the call returns SA_E_TIMEOUT and the context stays
                                 usable.  The other kernels keep 2 s. */
    SA_OPT_SOLVE_GPU = 1,     /* 1: sa_assign solves a B of at least 150000 entries with
                                 sa_solve_reduced_gpu from the scaling's duals; 0 (default):
                                 on the host with sa_solve_reduced_near */
    SA_OPT_STEP_SPARSE = 2,   /* 1: the STEP kernel may sweep only the entries >= 2^-70 of
                                 their row when K is sparse enough (where its ring has
                                 two-row stages: n <= 6700 or 8900 < n <= 12288 on a GB300);
                                 0 (default): dense */
    SA_OPT_MAX_GRID = 3,      /* cap on the blocks of the persistent kernels (0, the
                                 default: one or two per SM) */
    SA_OPT_FUSED_THREADS = 4, /* threads per block of the FUSED kernel for rows of 513 to
                                 1024 chunks of 16 bytes: 256 or 512 (default) */
    SA_OPT_STEP_L2_BYTES = 5, /* bytes of the STEP kernel's per-step matrix K that its sweeps
                                 read with the default L2 policy (default 48 MiB); the rest of
                                 K is read "evict first", so that this part stays in L2 from
                                 one sweep to the next.  A value >= the size of K reads all of
                                 it with the default policy.  Speed only: results are equal. */
    SA_OPT_TEST_UNREACHABLE_BARRIER = 6 /* testing hook for failure handling without a
                                 device fault (not part of the method): 1 makes the STEP
                                 kernel's first grid barrier wait for one arrival more than its
                                 grid provides, so the wait runs out after SA_OPT_WAIT_LIMIT_NS
                                 and the call returns SA_E_TIMEOUT; 0 (default) off */
} sa_option;

/* Set one option; SA_E_INVALID for an unknown option or a value out of range. */
sa_status sa_set_option(sa_ctx* ctx, sa_option opt, int64_t value);

/* Message of the calling thread's most recent failure ("" if none). */
const char* sa_last_error(void);

/* Library build string (compile flags, arch). */
const char* sa_version(void);

/* Number of CUDA kernels this library has launched in the process so far (all
 * contexts); a launch-count probe for benchmarks. */
int64_t sa_kernel_launches(void);

/*
 * sa_scale: log-domain Sinkhorn (Sec. 4.1.2, Eqs. dad1-dad3 in log coordinates) for
 * each p of opts->p in turn, each step until max_j |c_j - 1| <= tol for the row-
 * stochastic iterate (the eps-bistochastic measure of Sec. 4.2) or max_sweeps_per_p.
 *   d_u, d_v  device FP64[n], caller-owned.  Read as the warm start when
 *             opts->resume_from > 0; written with the potentials at the last p run.
 *   info      may be NULL.
 * Returns SA_OK, SA_E_NOT_CONVERGED (potentials still written), SA_E_NONFINITE,
 * SA_E_TIMEOUT, or an argument/CUDA error.  On any error other than SA_E_NOT_CONVERGED a
 * warm start (resume_from > 0) is left in d_u, d_v as it was given; after a cold start
 * their contents are then unspecified.  Synchronises the context stream.
 */
sa_status sa_scale(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* opts, double* d_u,
                   double* d_v, sa_scale_info* info);

/*
 * sa_scale_noalloc: sa_scale on the fused kernel without allocating anything.  The paper
 * has no counterpart: this is a deployment entry point for callers that cannot allocate
 * device memory when they scale -- callers whose memory is planned up front (a fixed
 * budget or a pre-sized pool) and callers that cannot afford the device-wide
 * synchronisation that cudaMalloc/cudaFree bring.  The fused kernel's scratch (column
 * partials, FP32 head and factor of v, schedule, barrier and status words, a copy of a
 * warm start) then lives in a static device array of the library, about 2.7 MiB, which
 * every GPU that loads the library holds until the process exits.  The caller still passes the matrix, the
 * potentials d_u, d_v (device FP64[n], as for sa_scale) and a CUDA stream (NULL: the
 * legacy default stream); the device is the calling thread's current device.
 *   Limits: n <= 4096, at most 64 p steps, MIXED or FP32 precision, and a layout the
 *   fused kernel reads (16-byte aligned base and row pitch).  Anything else returns
 *   SA_E_UNSUPPORTED or SA_E_INVALID with a message and runs nothing.
 *   The first call on a device looks the array's device address up (once per device,
 *   with that device current).
 *   All calls share the array and find the previous call's contents in it; each call
 *   clears what must start at zero, but calls whose work overlaps on the GPU race on
 *   the array, so serialise them (one stream, or events).
 *   Synchronises the stream before returning; info->kernel_ms is 0 (no events are made).
 *   A failure after the arguments were accepted leaves a warm start (resume_from > 0) in
 *   d_u, d_v as it was given; a step the kernel did not finish reports a NaN residual.
 *   It calls no cudaMalloc, cudaFree, cudaHostAlloc or other allocating routine.
 */
sa_status sa_scale_noalloc(const sa_matrix* a, const sa_scale_opts* opts, void* cuda_stream,
                           double* d_u, double* d_v, sa_scale_info* info);

/*
 * sa_verify: FP64 row and column sums of X(p) from the potentials (one read of A).
 *   d_rows, d_cols  device FP64[n] outputs (either may be NULL).
 *   max_row_err, max_col_err  host outputs max |sum - 1| (either may be NULL).
 */
sa_status sa_verify(sa_ctx* ctx, const sa_matrix* a, double p, const double* d_u,
                    const double* d_v, double* d_rows, double* d_cols, double* max_row_err,
                    double* max_col_err);

/*
 * sa_prune: the reduced matrix B_ij = A_ij if x_ij(p) >= t, else 0 (Eq. matrixred),
 * compacted to CSR.  t <= 0 selects t = 1/n (Sec. 4.2).  With guard != 0 the largest
 * entry of every row and of every column of X(p) is kept as well (the paper leaves
 * empty rows and columns open).  The keep test is p*log w - u - v >= log t, screened
 * in FP32 and decided in FP64 near the threshold.
 *   out     filled with library-owned host arrays (sa_csr_free).
 *   log_ub  may be NULL; receives the approximate optimality certificate of Prop. aoc,
 *           (1/p) (sum_i max_j (p log w_ij - v_j) + sum_j v_j) >= log w_opt(A).
 */
sa_status sa_prune(sa_ctx* ctx, const sa_matrix* a, double p, const double* d_u,
                   const double* d_v, double t, int32_t guard, sa_csr* out, double* log_ub);

/*
 * sa_solve_reduced: exact max sum_i log w_{i sigma(i)} over permutations supported by B
 * (host, sparse shortest augmenting paths; the sequential solve of B in Sec. 4.2).
 *   perm       host int32[n] out: column of row i
 *   sum_log_w  host out (may be NULL): sum_i log w_{i perm(i)}
 *   alpha,beta host FP64[n] out (may be NULL): LP duals, alpha_i + beta_j >= log w_ij on
 *              B with equality on the assignment
 * Returns SA_E_NO_PERFECT_MATCHING when B holds no permutation.  A column listed more
 * than once in a row counts with its largest weight; entries with w = 0 are forbidden.
 * Host only: needs no context and no GPU.
 */
sa_status sa_solve_reduced(const sa_csr* b, int32_t* perm, double* sum_log_w, double* alpha,
                           double* beta);

/*
 * sa_solve_reduced_warm: sa_solve_reduced started from given column duals instead of the
 * column minima: the same exact optimum (ties may pick another optimal permutation) and LP
 * duals.  Exact duals of a nearby instance (sa_assign's re-solve after its certificate
 * added entries) make it fast.  The scaling's approximate duals v/p make nearly every
 * entry of B almost tight and can make the solve much slower than the cold start
 * (measured 22.5 s against 26 ms on a Zipf-weighted B of n = 2048): for duals near v/p
 * use sa_solve_reduced_near.
 *   beta0  host FP64[n] in: maximisation-form column duals (natural log units); a
 *          non-finite entry falls back to that column's minimum cost.
 *   perm, sum_log_w, alpha, beta  as sa_solve_reduced.  Host only.
 */
sa_status sa_solve_reduced_warm(const sa_csr* b, const double* beta0, int32_t* perm, double* sum_log_w,
                                double* alpha, double* beta);

/*
 * sa_solve_reduced_near: the optimum of B as sa_solve_reduced computes it (from the column
 * minima), then, of all LP-optimal duals of B for that assignment, the one with the
 * componentwise largest beta <= beta0.  With the assignment sigma fixed, optimality reads
 * alpha_i = log w_{i sigma(i)} - beta_{sigma(i)} and
 * beta_{sigma(i)} - beta_j <= log w_{i sigma(i)} - log w_ij on every entry (i, j) of B,
 * difference constraints whose largest solution below beta0 is a shortest-path labelling
 * (Dijkstra over the columns).  With beta0 = the scaling's v/p (Sec. 4.2: x_ij(p) <= 1
 * makes (u/p, v/p) nearly feasible on all of A) the returned duals also tend to hold on
 * the rest of A, which is what sa_assign's certificate checks; sa_assign solves its first
 * B this way.
 *   beta0  host FP64[n] in: maximisation-form column duals to stay below; a non-finite
 *          entry leaves that column's dual where the cold solve put it.
 *   perm, sum_log_w, alpha, beta  as sa_solve_reduced.  Host only.
 */
sa_status sa_solve_reduced_near(const sa_csr* b, const double* beta0, int32_t* perm, double* sum_log_w,
                                double* alpha, double* beta);

/* Statistics of sa_solve_reduced_gpu. */
typedef struct {
    int32_t phases;           /* eps-scaling phases of the auction */
    int64_t rounds;           /* bidding rounds (three kernel launches each) */
    int32_t complete;         /* 1: the auction assigned every row at the final eps */
    double auction_sum_log_w; /* sum_i log w of the auction's own assignment (if complete):
                                 within n * eps_final of the optimum */
    double eps_final;
    double auction_ms;        /* wall time of the auction */
    double host_ms;           /* wall time of the exact phase after it: greedy pass and row
                                 reduction on the host, shortest-path searches on the GPU */
    int64_t searches;         /* shortest augmenting path searches run on the GPU */
    int64_t search_rounds;    /* their label-correcting rounds and tree levels, in all */
} sa_auction_info;

/*
 * sa_solve_reduced_gpu: the same exact optimum and LP duals as sa_solve_reduced, on the
 * GPU where it pays: the column prices first moved toward an optimal dual by a forward
 * auction with eps-scaling (all free rows bid in parallel each round; at most 1000 rounds,
 * down to eps = 1e-3 of the range of log w), then the exact solver's greedy pass and row
 * reduction on the host, and each of its shortest-augmenting-path searches on the GPU
 * (label-correcting search, then the dual update and the path flip on the device).
 * Measured: 3.9x on a B of 362k entries, slower than the host below about 100k.  Not in
 * the paper, which solves B sequentially (Sec. 4.2).
 *   b       host CSR (as from sa_prune); copied to the device for the call
 *   price0  host FP64[n] or NULL: starting column prices in the maximisation form (beta;
 *           e.g. v/p of the scaling); NULL starts from zero
 *   perm, sum_log_w, alpha, beta  as sa_solve_reduced
 *   info    may be NULL
 * Returns SA_E_NO_PERFECT_MATCHING when B holds no permutation (the auction then stops at
 * its round cap and the exact solver reports it).
 */
sa_status sa_solve_reduced_gpu(sa_ctx* ctx, const sa_csr* b, const double* price0, int32_t* perm,
                               double* sum_log_w, double* alpha, double* beta, sa_auction_info* info);

/*
 * sa_certify: LP-duality check of (alpha, beta) against the whole of A (one read):
 * entries with log w_ij - alpha_i - beta_j > tau violate dual feasibility.  No
 * violation means an assignment tight for (alpha, beta) is optimal for A.  (Not in the
 * paper: it turns the heuristic prune of Sec. 4.2 into an exact method.)
 *   alpha, beta  host FP64[n]
 *   n_viol       host out: number of violating entries
 *   additions    may be NULL; receives up to max_add violating entries as CSR
 */
sa_status sa_certify(sa_ctx* ctx, const sa_matrix* a, const double* alpha, const double* beta,
                     double tau, int64_t* n_viol, int64_t max_add, sa_csr* additions);

void sa_csr_free(sa_csr* c);

/* Result of the whole preprocessing + exact solve (Algorithm 1, fixed schedule). */
typedef struct {
    int32_t* perm;            /* caller-owned host int32[n]: optimal column of each row */
    double sum_log_w;         /* sum_i log w_{i perm(i)} */
    double log_ub;            /* certificate of Prop. aoc at the last p */
    double gamma;             /* Eq. optratio: exp(log_ub - log w_opt(B_first)) */
    int64_t nnz_first;        /* entries kept by the first prune */
    int64_t nnz_final;        /* entries of the last reduced instance solved */
    int32_t repairs;          /* certificate-driven re-solves */
    int32_t reprunes;         /* re-prunes at t/16 after no perfect matching */
    sa_scale_info scale;
    double ms_scale, ms_prune, ms_solve, ms_certify;
} sa_assign_result;

/*
 * sa_assign: scale (sa_scale), prune at t (sa_prune, guard on), solve B
 * (sa_solve_reduced_near toward the scaling's duals v/p; sa_solve_reduced_gpu from those
 * duals when the context's SA_OPT_SOLVE_GPU is 1 and B has at least 150000 entries),
 * then certify on A (sa_certify, tau = 1e-9) and re-solve from the last duals
 * with the violating entries added until none is left (SA_E_NOT_CONVERGED if that does
 * not settle); the result is optimal for A.  If B has no perfect matching, re-prune at
 * t/16 (finally t = 0, i.e. all of A).
 */
sa_status sa_assign(sa_ctx* ctx, const sa_matrix* a, const sa_scale_opts* opts, double t,
                    sa_assign_result* res);

/* ---- Algorithm 1 with adaptive p (Sec. 4.2, Algorithm 1) ----------------------------- */

/* Options of the preprocessing loop: prescale A to [1, e] (Sec. 4.1.1), then for
 * p = p0, p0 + dp, ...: scale A^(p) to an eps-bistochastic X, prune B = {x_ij >= t}
 * (Eq. matrixred), solve B exactly and evaluate gamma (Eq. optratio); stop at the first p
 * with gamma <= opt_ratio.  p is on the prescaled scale; the raw-weight equivalent is
 * p / log(max w / min w) when max/min > e (the identity X(A^(m)/c, p) = X(A, p m)). */
typedef struct {
    double opt_ratio;         /* required gamma, > 1 (the paper uses about 2) */
    double p0;                /* first p (the paper: 100) */
    double dp;                /* increase of p per round (the paper: 50) */
    int32_t max_rounds;       /* SA_E_NOT_CONVERGED after this many rounds without success */
    double eps;               /* eps of the eps-bistochastic stop; <= 0: 1/n (the paper's) */
    double t;                 /* pruning threshold; <= 0: 1/n (the paper's) */
    int32_t max_sweeps_per_p; /* cap of the scaling at each p */
    sa_prec prec;
    sa_kernel kernel;
} sa_alg1_opts;

typedef struct {
    int32_t* perm;            /* caller-owned host int32[n]: an optimal permutation of the final B */
    double sum_log_w;         /* sum_i log w_{i perm(i)} */
    double gamma;             /* Eq. optratio at the final p (<= opt_ratio on success) */
    double p_final;           /* final p on the prescaled scale */
    double p_raw;             /* the same p applied to the raw weights */
    int32_t rounds;           /* values of p tried */
    int64_t sweeps_total;     /* scaling sweeps over all rounds */
    int64_t nnz;              /* entries of the final B (row and column maxima always kept) */
} sa_alg1_result;

/*
 * sa_algorithm1: the paper's preprocessing algorithm on a device matrix.  Each round
 * warm-starts the scaling from the previous round's potentials (scaled by the ratio of the
 * p values); its B is solved exactly from the column minima (sa_solve_reduced), since
 * gamma needs only B's optimal weight.  A round whose B holds no permutation counts as
 * gamma = +inf.  Returns SA_OK
 * with gamma <= opt_ratio, or SA_E_NOT_CONVERGED after max_rounds (res filled with the
 * last round).  Unlike sa_assign the result is only certified to within gamma.
 */
sa_status sa_algorithm1(sa_ctx* ctx, const sa_matrix* a, const sa_alg1_opts* opts, sa_alg1_result* res);

/*
 * sa_assign_host: sa_assign on a HOST matrix (n x ld weights): copies it into a
 * context-owned device buffer on the context stream first.  For end-to-end timing.
 */
sa_status sa_assign_host(sa_ctx* ctx, const void* host_w, sa_wtype wtype, int32_t n, int64_t ld,
                         const sa_scale_opts* opts, double t, sa_assign_result* res);

/*
 * sa_narrow_i32_to_i16: exact int32 -> int16 copy (values must lie in [0, 32767]),
 * halving the bytes the sweeps read.  d_dst has n rows of ld_dst.  *n_bad counts values
 * out of range (those are clamped; treat n_bad > 0 as failure).
 */
sa_status sa_narrow_i32_to_i16(sa_ctx* ctx, const int32_t* d_src, int64_t ld_src, int16_t* d_dst,
                               int64_t ld_dst, int32_t n, int64_t* n_bad);

/* ---- Batched scaling of many independent small instances (one launch) -------------- */

/* How sa_batch_scale runs an instance (a deployment choice; the paper has no counterpart).
 * BLOCK: one thread block of 256 threads per instance; every sweep forms each term with an
 *   SFU exp2 of an FP32 exponent (the log2 table of the instance in shared memory when it
 *   fits), so the error of the sums grows like 1.3e-7 p.
 * GROUP: a group of 1, 2 or 4 warps per instance (n <= 128), with the per-step matrix K of
 *   the STEP path in a shared-memory slot of the group (exponent in float-pair arithmetic
 *   once per p step); the sweeps multiply and add only, the group's warps meet at a named
 *   barrier of their own, and the error does not grow with p.
 * REGS: as GROUP, with K in registers during the sweeps (each row and column of K split
 *   over 32 G / NMAX adjacent lanes): 1, 2 or 4 warps for n <= 32, 4 or 8 for n <= 64, 16
 *   for n <= 128.
 * KROWS: one block of 256 threads per instance (n <= 512) on the same K, kept in a global
 *   slot of n x ceil(n/4)*4 FP32 per block (taken from the context workspace: up to two
 *   blocks per SM); each warp evaluates and reads whole rows, so a row sum needs no block
 *   barrier, and a sweep has one; the error does not grow with p. */
typedef enum { SA_BATCH_BLOCK = 0, SA_BATCH_GROUP = 1, SA_BATCH_REGS = 2, SA_BATCH_KROWS = 3 } sa_batch_path;

/* A launch plan: instances are grouped by n into buckets (n_hi[b-1], n_hi[b]] (n_hi
 * increasing, the last >= 512), and each bucket runs on its path in a persistent launch of
 * its own; the launches of the buckets run side by side on the device.  The project's
 * autotuner (paper_1104_3830_gb300/autotune.py) picks a plan per GPU and weight type by
 * timing the candidates, and caches it. */
#define SA_BATCH_MAX_BUCKETS 8
typedef struct {
    int32_t count;                          /* buckets in use, 1 .. SA_BATCH_MAX_BUCKETS */
    int32_t n_hi[SA_BATCH_MAX_BUCKETS];     /* largest n of each bucket */
    int32_t path[SA_BATCH_MAX_BUCKETS];     /* sa_batch_path; GROUP and REGS for n_hi <= 128 */
    int32_t warps[SA_BATCH_MAX_BUCKETS];    /* GROUP: warps per instance, 1, 2 or 4;
                                               REGS: 1, 2, 4, 8 or 16 (as above) */
    int32_t per_block[SA_BATCH_MAX_BUCKETS];/* groups per block: GROUP warps * per_block <= 8,
                                               REGS <= 16 warps per block */
} sa_batch_plan;

/* Set the context's plan (copied); NULL restores the default (the autotuner's choice on a
 * GB300): the register path with one warp per instance (two per block) up to n = 32, four
 * warps up to 64 and sixteen up to 128, the K rows path in two buckets up to 256 and 512.
 * SA_E_INVALID for a plan that breaks the rules above. */
sa_status sa_set_batch_plan(sa_ctx* ctx, const sa_batch_plan* plan);

/*
 * sa_batch_scale: scale k independent instances, each bucket of the context's plan in one
 * persistent launch (Sec. 4.1.2 iteration and Sec. 4.2 stop rule per instance, p schedule
 * and warm start as sa_scale).  Instance i is the device matrix d_w[i] (n[i] x ld[i] int16
 * or int32 per wtype, all the same type); its potentials go to d_u + off[i], d_v + off[i]
 * (device FP64, natural units).  The schedule, tol and cap are shared.  Instances with
 * n <= 512 are supported; larger ones return SA_E_UNSUPPORTED.  Per-instance sweeps and
 * status (0 converged, 1 a step hit the cap, -6 a row or column lost all mass) go to the
 * host arrays sweeps[k] and status[k] (may be NULL).
 *   d_w, d_n, d_ld, d_off  device arrays of length k (pointers, int32, int64, int64)
 */
sa_status sa_batch_scale(sa_ctx* ctx, int32_t k, const void* const* d_w, const int32_t* d_n,
                         const int64_t* d_ld, const int64_t* d_off, sa_wtype wtype,
                         const sa_scale_opts* opts, double* d_u, double* d_v, int32_t* sweeps,
                         int32_t* status);

/* ---- Continuous-batching server ---------------------------------------------------- */
/* Not part of the paper: a serving layer around the same path.  Small requests (n <= 512)
 * are scaled on a device-resident queue: the blocks of a persistent kernel take published
 * requests one per block as they free up (the K rows form of the batched path), so a
 * request joins the scaling already under way; a block leaves after 2 ms without a
 * request while none is busy, and the next request starts the kernel again.  Each scaled
 * request is then pruned, solved exactly and certified on the host side of the path.
 * Larger requests run sa_assign on workers of their own. */

typedef struct sa_server sa_server;

typedef struct {
    int32_t n;
    int32_t* perm;            /* library-owned until sa_result_release */
    double sum_log_w;
    double gamma;
    int64_t sweeps;
    int32_t status;           /* sa_status of the request */
    double t_submit, t_start, t_done;  /* seconds on the server's monotonic clock */
    double t_scaled;          /* small requests: when the request queue had scaled it; else 0 */
} sa_result;

/* Start a server on `device` with a device-memory budget for resident requests.  Each
 * admitted request is charged an upper bound of the device memory it can hold while it
 * runs (sa_server_request_bytes), and is admitted only while the charges of the requests
 * on the device stay within hbm_budget.  SMs are shared the same way: a large request's
 * scaling kernel (a cooperative grid of at most num_sms / solver_threads blocks) takes only
 * SMs that the request queue's running blocks and the other large requests leave, and
 * while small requests wait for the queue, the SMs of one launch of it are kept free.  The
 * request queue's device memory (its slots of K, one 1 MiB slot per block of each of its
 * two launch slots, at most an eighth of hbm_budget) is charged once, here; SA_E_BUDGET if
 * hbm_budget does not exceed it.  Outside the budget the server holds only its workers'
 * small persistent state: per small-request worker (two) a context workspace of at most
 * 16 MiB, and a CUDA stream per worker. */
sa_status sa_server_create(sa_server** s, int device, size_t hbm_budget, const sa_scale_opts* opts,
                           int32_t solver_threads);
void sa_server_destroy(sa_server* s);

/* Submit an n x n host matrix (row-major, ld = n); the weights are copied before return.
 * Returns SA_E_BUDGET if the request alone exceeds the budget. */
sa_status sa_submit(sa_server* s, const void* host_w, sa_wtype wtype, int32_t n, uint64_t* ticket);

/* SA_PENDING until the request is done; then SA_OK (or its error) with *out filled.  Every
 * finished request's permutation is the certified optimum of its matrix, as from sa_assign
 * (small requests: scaling on the request queue, then sa_solve_reduced_near toward v/p, the
 * certificate and its repairs; SA_E_NOT_CONVERGED if the repairs do not settle). */
sa_status sa_poll(sa_server* s, uint64_t ticket, sa_result* out);
void sa_result_release(sa_server* s, uint64_t ticket);

/* Server clock (seconds), the one t_submit/t_start/t_done use. */
double sa_server_now(const sa_server* s);

/* Bytes of the budget an n x n request of this weight type is charged: its matrix (16-byte
 * row pitch) plus, for n <= 512, its potentials, the reduced instance's device arrays (8
 * bytes per kept entry, at most n^2) and 1 MiB; for larger n, everything sa_assign can
 * allocate (the per-step matrix K and the log2 w pairs, 12 n ceil(n/4)*4 bytes, the reduced instance's device
 * arrays up to 8 n^2 bytes, column partials, vectors).  0 for bad arguments. */
size_t sa_server_request_bytes(const sa_server* s, sa_wtype wtype, int32_t n);

/* Testing hook for failure handling without a device fault (not part of the method): the
 * next `count` device allocations made by the server's request paths fail as if the device
 * were out of memory, without allocating; the requests concerned finish with SA_E_NOMEM.
 * Process-wide; 0 clears it. */
void sa_debug_fail_allocs(int32_t count);

/* Counters of a server's request queue and its launch geometry. */
typedef struct {
    int64_t live_launches;      /* launches of the queue's kernel so far */
    int64_t live_requests;      /* small requests it has scaled */
    int64_t live_device_bytes;  /* device memory of the queue (charged at creation) */
    int32_t live_blocks;        /* blocks per launch */
    int32_t live_slots;         /* launches that may run at once */
    int32_t live_capacity;      /* requests published and not yet scaled, at most */
    int32_t large_grid;         /* grid of a large request's scaling kernel on a free GPU */
} sa_server_stats;
sa_status sa_server_get_stats(sa_server* s, sa_server_stats* out);

#ifdef __cplusplus
}
#endif
#endif /* SA_H */
