/*
 * orc.c -- FP64 CPU oracle for the diagonal-scaling preprocessing of the optimal
 * assignment problem (Sharify, Gaubert, Grigori, "Solution of the optimal assignment
 * problem by diagonal scaling algorithms", arXiv:1104.3830).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls this
 * file: only the test suite, the smoke check and the benchmark's CPU-baseline leg use it.
 * It shares no code, header, table or helper with the CUDA library; it is written to be
 * read against the paper, not to be fast.  Loops are plain and in the order the paper
 * states them; OpenMP only splits independent rows or columns across threads.
 *
 * Notation.  b_ij = log a_ij (Eq. pentropyopt, Sec. 2.1), b_ij = -inf for a_ij = 0.
 * X(p) = D_r A^(p) D_c (Thm. prop-borweinlewisnussbaum) is stored through potentials
 *     x_ij = exp(p*b_ij - u_i - v_j),   u_i = -log (D_r)_ii,  v_j = -log (D_c)_jj,
 * so u = -p*ubar and v = -p*vbar in the paper's log coordinates of Sec. 4.1.2.
 *
 * Every function returns 0 on success and a negative code on invalid input.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_NOT_CONVERGED 1
#define ORC_E_INVALID (-1)
#define ORC_E_NO_SUPPORT (-2)
#define ORC_E_INFEASIBLE (-3)

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the later parallel loops (k >= 1); the arithmetic does not depend on it */
void orc_set_num_threads(int k) {
#ifdef _OPENMP
    omp_set_num_threads(k >= 1 ? k : 1);
#else
    (void)k;
#endif
}

/* ------------------------------------------------------------------------------------
 * Log-domain Sinkhorn iteration at a fixed p (Sec. 4.1.2, "logarithmic p-Sinkhorn"),
 * which is the iteration of Eqs. dad1-dad3 written in log coordinates with the row and
 * column maxima factored out.  One sweep = one row update followed by one column update.
 * ------------------------------------------------------------------------------------ */

/* Row update: u_i = m_i + log sum_j exp(p*b_ij - v_j - m_i), m_i = max_j (p*b_ij - v_j). */
static int row_update(int n, const double* b, double p, const double* v, double* u) {
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int i = 0; i < n; ++i) {
        const double* bi = b + (int64_t)i * n;
        double m = -INFINITY;
        for (int j = 0; j < n; ++j) {
            double e = p * bi[j] - v[j];
            if (e > m) m = e;
        }
        if (m == -INFINITY) { bad = 1; continue; }
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += exp(p * bi[j] - v[j] - m);
        u[i] = m + log(s);
    }
    return bad ? ORC_E_NO_SUPPORT : ORC_OK;
}

/* Column update: v_j = m_j + log sum_i exp(p*b_ij - u_i - m_j), m_j = max_i (p*b_ij - u_i). */
static int col_update(int n, const double* b, double p, const double* u, double* v) {
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int j = 0; j < n; ++j) {
        double m = -INFINITY;
        for (int i = 0; i < n; ++i) {
            double e = p * b[(int64_t)i * n + j] - u[i];
            if (e > m) m = e;
        }
        if (m == -INFINITY) { bad = 1; continue; }
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += exp(p * b[(int64_t)i * n + j] - u[i] - m);
        v[j] = m + log(s);
    }
    return bad ? ORC_E_NO_SUPPORT : ORC_OK;
}

/* Distance to bistochastic of a column-stochastic X (Sec. 4.2): max_i |r_i - 1|,
 * with r_i the i-th row sum. */
static double row_residual(int n, const double* b, double p, const double* u, const double* v) {
    double worst = 0.0;
#pragma omp parallel for schedule(static) reduction(max : worst)
    for (int i = 0; i < n; ++i) {
        const double* bi = b + (int64_t)i * n;
        double r = 0.0;
        for (int j = 0; j < n; ++j) r += exp(p * bi[j] - u[i] - v[j]);
        double d = fabs(r - 1.0);
        if (d > worst) worst = d;
    }
    return worst;
}

/*
 * orc_sinkhorn: run the log-domain Sinkhorn iteration for each p in the increasing
 * schedule p[0..n_p), each step to an eps-bistochastic matrix with eps = tol (Sec. 4.2),
 * capped at max_sweeps sweeps per step.
 *   b            n x n row-major log weights (-inf allowed where a_ij = 0)
 *   warm_keep_v  0: between steps scale (u, v) by p_k/p_{k-1}, so that x_ij(p_{k-1})
 *                   becomes x_ij(p_{k-1})^(p_k/p_{k-1});  1: keep v as the deformed
 *                   iteration does (Sec. 3.2).  v starts at 0 (v_0 = 1, Eq. dad1).
 *   u, v         out: FP64 potentials at p[n_p-1]
 *   sweeps       out (may be NULL): sweeps spent at each p step
 *   resid        out (may be NULL): final residual at each p step
 * Returns ORC_OK, ORC_NOT_CONVERGED (some step hit the cap), or a negative error.
 */
int orc_sinkhorn(int n, const double* b, const double* p, int n_p, double tol, int max_sweeps,
                 int warm_keep_v, double* u, double* v, int32_t* sweeps, double* resid) {
    if (n <= 0 || n_p <= 0 || max_sweeps <= 0 || !(tol > 0)) return ORC_E_INVALID;
    for (int k = 0; k < n_p; ++k)
        if (!(p[k] > 0) || (k > 0 && !(p[k] > p[k - 1]))) return ORC_E_INVALID;
    for (int j = 0; j < n; ++j) v[j] = 0.0;
    for (int i = 0; i < n; ++i) u[i] = 0.0;
    int status = ORC_OK;
    for (int k = 0; k < n_p; ++k) {
        if (k > 0 && !warm_keep_v) {
            double r = p[k] / p[k - 1];
            for (int i = 0; i < n; ++i) u[i] *= r;
            for (int j = 0; j < n; ++j) v[j] *= r;
        }
        int s = 0;
        double res = INFINITY;
        while (s < max_sweeps) {
            int rc = row_update(n, b, p[k], v, u);
            if (rc) return rc;
            rc = col_update(n, b, p[k], u, v);
            if (rc) return rc;
            ++s;
            res = row_residual(n, b, p[k], u, v);
            if (res <= tol) break;
        }
        if (!(res <= tol)) status = ORC_NOT_CONVERGED;
        if (sweeps) sweeps[k] = s;
        if (resid) resid[k] = res;
    }
    return status;
}

/* Continue the iteration at one fixed p from given potentials (no reset): used by tests
 * that check independence from the starting point. */
int orc_sinkhorn_from(int n, const double* b, double p, double tol, int max_sweeps, double* u,
                      double* v, int32_t* sweeps, double* resid) {
    if (n <= 0 || max_sweeps <= 0 || !(p > 0) || !(tol > 0)) return ORC_E_INVALID;
    int s = 0;
    double res = INFINITY;
    while (s < max_sweeps) {
        int rc = row_update(n, b, p, v, u);
        if (rc) return rc;
        rc = col_update(n, b, p, u, v);
        if (rc) return rc;
        ++s;
        res = row_residual(n, b, p, u, v);
        if (res <= tol) break;
    }
    if (sweeps) *sweeps = s;
    if (resid) *resid = res;
    return res <= tol ? ORC_OK : ORC_NOT_CONVERGED;
}

/* x_ij = exp(p*b_ij - u_i - v_j) for the whole matrix (row-major, n x n). */
int orc_xmatrix(int n, const double* b, double p, const double* u, const double* v, double* x) {
    if (n <= 0) return ORC_E_INVALID;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            x[(int64_t)i * n + j] = exp(p * b[(int64_t)i * n + j] - u[i] - v[j]);
    return ORC_OK;
}

/* Row and column sums of X(p) recomputed in FP64 from the potentials. */
int orc_sums(int n, const double* b, double p, const double* u, const double* v, double* rows,
             double* cols) {
    if (n <= 0) return ORC_E_INVALID;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        for (int j = 0; j < n; ++j) r += exp(p * b[(int64_t)i * n + j] - u[i] - v[j]);
        rows[i] = r;
    }
#pragma omp parallel for schedule(static)
    for (int j = 0; j < n; ++j) {
        double c = 0.0;
        for (int i = 0; i < n; ++i) c += exp(p * b[(int64_t)i * n + j] - u[i] - v[j]);
        cols[j] = c;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Pruning (Eq. matrixred, Sec. 4.2): B_ij = A_ij if x_ij(p) >= t, else 0, with the test
 * taken in log form, p*b_ij - u_i - v_j >= log t.  With guard != 0 the entry of largest
 * x in every row and in every column is kept as well (lowest index on ties), so that no
 * row or column of B is empty; the paper leaves that case open.
 * mask: n x n bytes, 1 = kept.
 * ------------------------------------------------------------------------------------ */
int orc_prune_mask(int n, const double* b, double p, const double* u, const double* v,
                   double log_t, int guard, uint8_t* mask) {
    if (n <= 0) return ORC_E_INVALID;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        int best = 0;
        double best_e = -INFINITY;
        for (int j = 0; j < n; ++j) {
            double e = p * b[(int64_t)i * n + j] - u[i] - v[j];
            mask[(int64_t)i * n + j] = (uint8_t)(e >= log_t);
            if (e > best_e) { best_e = e; best = j; }
        }
        if (guard && best_e > -INFINITY) mask[(int64_t)i * n + best] = 1;
    }
    if (guard) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < n; ++j) {
            int best = 0;
            double best_e = -INFINITY;
            for (int i = 0; i < n; ++i) {
                double e = p * b[(int64_t)i * n + j] - u[i] - v[j];
                if (e > best_e) { best_e = e; best = i; }
            }
            if (best_e > -INFINITY) mask[(int64_t)best * n + j] = 1;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------
 * Approximate optimality certificate (Prop. aoc, Eq. e-certificate):
 *   log w_opt(A) <= (1/p) ( sum_i max_j log x_ij - sum_i log d_r,i - sum_j log d_c,j ).
 * With log x_ij = p*b_ij - u_i - v_j, log d_r,i = -u_i and log d_c,j = -v_j the right
 * side is (1/p) ( sum_i max_j (p*b_ij - v_j) + sum_j v_j ); it holds for any potentials.
 * ------------------------------------------------------------------------------------ */
double orc_log_ub(int n, const double* b, double p, const double* v) {
    double acc = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : acc)
    for (int i = 0; i < n; ++i) {
        double m = -INFINITY;
        for (int j = 0; j < n; ++j) {
            double e = p * b[(int64_t)i * n + j] - v[j];
            if (e > m) m = e;
        }
        acc += m;
    }
    for (int j = 0; j < n; ++j) acc += v[j];
    return acc / p;
}

/* Prescaling of Sec. 4.1.1 applied to a positive-pattern matrix a (zeros stay zero):
 * if max/min > e then a <- a^(m)/c with m = 1/log(max/min), c = exp(log(min)/log(max/min)),
 * else a <- a/min.  Writes the result to out and returns m (the exponent), c in *c_out
 * (c = min in the second branch, m = 1 there). */
double orc_prescale(int n, const double* a, double* out, double* c_out) {
    double mx = -INFINITY, mn = INFINITY;
    for (int64_t k = 0; k < (int64_t)n * n; ++k)
        if (a[k] > 0) {
            if (a[k] > mx) mx = a[k];
            if (a[k] < mn) mn = a[k];
        }
    double m = 1.0, c = mn;
    if (mx / mn > exp(1.0)) {
        m = 1.0 / log(mx / mn);
        c = exp(log(mn) / log(mx / mn));
    }
    for (int64_t k = 0; k < (int64_t)n * n; ++k)
        out[k] = a[k] > 0 ? pow(a[k], m) / c : 0.0;
    if (c_out) *c_out = c;
    return m;
}

/* ------------------------------------------------------------------------------------
 * Exact solvers of the optimal assignment problem max_sigma sum_i b_{i sigma(i)}
 * (Sec. 2.2: the LP over bistochastic matrices), i.e. max prod_i a_{i sigma(i)}.
 * Both work on costs c = -b; entries with b = -inf are forbidden.
 * ------------------------------------------------------------------------------------ */

/*
 * orc_hungarian: O(n^3) Hungarian method with potentials (Kuhn-Munkres; shortest
 * augmenting paths with reduced costs).  Rows are inserted one at a time; for each new
 * row a Dijkstra-like search over columns grows an alternating tree until it reaches a
 * free column, then the path is flipped.  perm[i] = column of row i.
 * alpha, beta (may be NULL): optimal duals of the maximisation, alpha_i + beta_j >= b_ij
 * on allowed entries, with equality on (i, perm[i]).
 * Returns ORC_E_INFEASIBLE if no permutation avoids every forbidden entry.
 */
int orc_hungarian(int n, const double* b, int32_t* perm, double* alpha, double* beta) {
    if (n <= 0) return ORC_E_INVALID;
    /* 1-based arrays; column 0 is a virtual column holding the row being inserted. */
    double* pu = (double*)calloc((size_t)n + 1, sizeof(double));     /* row potentials */
    double* pv = (double*)calloc((size_t)n + 1, sizeof(double));     /* column potentials */
    int* match = (int*)calloc((size_t)n + 1, sizeof(int));           /* column -> row */
    int* prev = (int*)calloc((size_t)n + 1, sizeof(int));            /* tree parent column */
    double* slack = (double*)malloc(((size_t)n + 1) * sizeof(double));
    char* used = (char*)malloc((size_t)n + 1);
    int rc = ORC_OK;
    for (int r = 1; r <= n && rc == ORC_OK; ++r) {
        match[0] = r;
        int j0 = 0;
        for (int j = 0; j <= n; ++j) { slack[j] = INFINITY; used[j] = 0; }
        do {
            used[j0] = 1;
            int i0 = match[j0];
            double delta = INFINITY;
            int j1 = -1;
            for (int j = 1; j <= n; ++j) {
                if (used[j]) continue;
                double bij = b[(int64_t)(i0 - 1) * n + (j - 1)];
                if (bij > -INFINITY) {
                    double cur = -bij - pu[i0] - pv[j];
                    if (cur < slack[j]) { slack[j] = cur; prev[j] = j0; }
                }
                if (slack[j] < delta) { delta = slack[j]; j1 = j; }
            }
            if (j1 < 0 || delta == INFINITY) { rc = ORC_E_INFEASIBLE; break; }
            for (int j = 0; j <= n; ++j) {
                if (used[j]) { pu[match[j]] += delta; pv[j] -= delta; }
                else slack[j] -= delta;
            }
            j0 = j1;
        } while (match[j0] != 0);
        if (rc != ORC_OK) break;
        do { /* flip the augmenting path back to the virtual column */
            int j1 = prev[j0];
            match[j0] = match[j1];
            j0 = j1;
        } while (j0 != 0);
    }
    if (rc == ORC_OK) {
        for (int j = 1; j <= n; ++j) perm[match[j] - 1] = j - 1;
        /* minimisation duals satisfy -b_ij - pu_i - pv_j >= 0; negate for maximisation */
        if (alpha) for (int i = 0; i < n; ++i) alpha[i] = -pu[i + 1];
        if (beta) for (int j = 0; j < n; ++j) beta[j] = -pv[j + 1];
    }
    free(pu); free(pv); free(match); free(prev); free(slack); free(used);
    return rc;
}

/*
 * orc_lapjv: dense Jonker-Volgenant (1987) for the same problem, written independently
 * of orc_hungarian: column reduction, reduction transfer, two rounds of augmenting row
 * reduction, then shortest augmenting paths for the rows still free.  Needs every entry
 * allowed (finite b); returns ORC_E_INVALID otherwise.  perm[i] = column of row i.
 */
int orc_lapjv(int n, const double* b, int32_t* perm) {
    if (n <= 0) return ORC_E_INVALID;
    for (int64_t k = 0; k < (int64_t)n * n; ++k)
        if (!(b[k] > -INFINITY) || !(b[k] < INFINITY)) return ORC_E_INVALID;
#define C(i, j) (-b[(int64_t)(i) * n + (j)])
    int* x = (int*)malloc((size_t)n * sizeof(int));      /* row -> column, -1 free */
    int* y = (int*)malloc((size_t)n * sizeof(int));      /* column -> row, -1 free */
    double* v = (double*)malloc((size_t)n * sizeof(double));
    int* freerows = (int*)malloc((size_t)n * sizeof(int));
    int* matches = (int*)calloc((size_t)n, sizeof(int));
    for (int i = 0; i < n; ++i) x[i] = -1;
    /* column reduction: v_j = min_i c_ij, give column j to its argmin row if that row
       has no column yet (scan columns from last to first) */
    for (int j = n - 1; j >= 0; --j) {
        int imin = 0;
        double mn = C(0, j);
        for (int i = 1; i < n; ++i)
            if (C(i, j) < mn) { mn = C(i, j); imin = i; }
        v[j] = mn;
        if (++matches[imin] == 1) { x[imin] = j; y[j] = imin; }
        else y[j] = -1;
    }
    /* reduction transfer from rows matched exactly once */
    int nfree = 0;
    for (int i = 0; i < n; ++i) {
        if (matches[i] == 0) { freerows[nfree++] = i; continue; }
        if (matches[i] == 1) {
            int j1 = x[i];
            double mn = INFINITY;
            for (int j = 0; j < n; ++j)
                if (j != j1 && C(i, j) - v[j] < mn) mn = C(i, j) - v[j];
            if (mn < INFINITY) v[j1] -= mn;
        }
    }
    /* augmenting row reduction, two rounds */
    for (int round = 0; round < 2; ++round) {
        int k = 0, prvnfree = nfree;
        nfree = 0;
        int guard = 0;
        while (k < prvnfree) {
            int i = freerows[k++];
            double u1 = INFINITY, u2 = INFINITY;
            int j1 = 0, j2 = -1;
            for (int j = 0; j < n; ++j) {
                double h = C(i, j) - v[j];
                if (h < u2) {
                    if (h >= u1) { u2 = h; j2 = j; }
                    else { u2 = u1; j2 = j1; u1 = h; j1 = j; }
                }
            }
            int i0 = y[j1];
            if (j2 >= 0 && u1 < u2) v[j1] = v[j1] - (u2 - u1);
            else if (i0 >= 0 && j2 >= 0) { j1 = j2; i0 = y[j2]; }
            x[i] = j1;
            y[j1] = i;
            if (i0 >= 0) {
                x[i0] = -1;
                if (u1 < u2 && ++guard < 4 * n) freerows[--k] = i0;
                else freerows[nfree++] = i0;
            }
        }
    }
    /* shortest augmenting path for each remaining free row (dense Dijkstra) */
    double* d = (double*)malloc((size_t)n * sizeof(double));
    int* pred = (int*)malloc((size_t)n * sizeof(int));
    int* col = (int*)malloc((size_t)n * sizeof(int));
    for (int f = 0; f < nfree; ++f) {
        int fr = freerows[f];
        for (int j = 0; j < n; ++j) { col[j] = j; d[j] = C(fr, j) - v[j]; pred[j] = fr; }
        int low = 0, up = 0, last = 0, endofpath = -1;
        double mn = 0;
        while (endofpath < 0) {
            if (up == low) {
                last = low - 1;
                mn = d[col[up++]];
                for (int k = up; k < n; ++k) {
                    int j = col[k];
                    double h = d[j];
                    if (h <= mn) {
                        if (h < mn) { up = low; mn = h; }
                        col[k] = col[up];
                        col[up++] = j;
                    }
                }
                for (int k = low; k < up; ++k)
                    if (y[col[k]] < 0) { endofpath = col[k]; break; }
            }
            if (endofpath < 0) {
                int j1 = col[low++];
                int i = y[j1];
                double u1 = C(i, j1) - v[j1] - mn;
                for (int k = up; k < n; ++k) {
                    int j = col[k];
                    double h = C(i, j) - v[j] - u1;
                    if (h < d[j]) {
                        d[j] = h;
                        pred[j] = i;
                        if (h == mn) {
                            if (y[j] < 0) { endofpath = j; break; }
                            col[k] = col[up];
                            col[up++] = j;
                        }
                    }
                }
            }
        }
        for (int k = 0; k <= last; ++k) {
            int j = col[k];
            v[j] += d[j] - mn;
        }
        int j = endofpath;
        for (;;) {
            int i = pred[j];
            y[j] = i;
            int tmp = x[i];
            x[i] = j;
            j = tmp;
            if (i == fr) break;
        }
    }
    for (int i = 0; i < n; ++i) perm[i] = x[i];
    free(d); free(pred); free(col);
    free(x); free(y); free(v); free(freerows); free(matches);
#undef C
    return ORC_OK;
}

/* Exhaustive search over all n! permutations (n <= 10) for max sum_i b_{i sigma(i)};
 * lexicographically first optimum.  Returns the optimum in *best. */
static void bf_rec(int n, const double* b, int row, int32_t* cur, char* used, double acc,
                   double* best, int32_t* perm) {
    if (row == n) {
        if (acc > *best) { *best = acc; memcpy(perm, cur, (size_t)n * sizeof(int32_t)); }
        return;
    }
    for (int j = 0; j < n; ++j) {
        if (used[j]) continue;
        double bij = b[(int64_t)row * n + j];
        if (!(bij > -INFINITY)) continue;
        used[j] = 1;
        cur[row] = j;
        bf_rec(n, b, row + 1, cur, used, acc + bij, best, perm);
        used[j] = 0;
    }
}

int orc_bruteforce(int n, const double* b, int32_t* perm, double* best) {
    if (n <= 0 || n > 10) return ORC_E_INVALID;
    int32_t cur[10];
    char used[10] = {0};
    *best = -INFINITY;
    bf_rec(n, b, 0, cur, used, 0.0, best, perm);
    return *best > -INFINITY ? ORC_OK : ORC_E_INFEASIBLE;
}

/* LP-duality check for max sum b over permutations: counts allowed entries with
 * alpha_i + beta_j < b_ij - tau (dual infeasible) and returns the largest such gap in
 * *max_gap.  A permutation sigma with alpha_i + beta_{sigma(i)} = b_{i sigma(i)} and no
 * violation is optimal (weak duality). */
int64_t orc_dual_violations(int n, const double* b, const double* alpha, const double* beta,
                            double tau, double* max_gap) {
    int64_t cnt = 0;
    double worst = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : cnt) reduction(max : worst)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double bij = b[(int64_t)i * n + j];
            if (!(bij > -INFINITY)) continue;
            double gap = bij - alpha[i] - beta[j];
            if (gap > tau) {
                ++cnt;
                if (gap > worst) worst = gap;
            }
        }
    if (max_gap) *max_gap = worst;
    return cnt;
}
