// solve.cpp -- exact solve of the reduced instance B on the host (the sequential solve
// of Sec. 4.2), by shortest augmenting paths on the sparse bipartite graph of B.
//
// Minimisation form: cost c_e = -log w_e on each kept entry.  Column prices v_j are kept
// such that every assigned row i sits on a column of least reduced cost c_ij - v_j
// (Jonker-Volgenant invariant).  Start: v_j = min_i c_ij, or caller-supplied prices (any
// prices keep the invariant once every row takes its least-reduced-cost column).  The
// exact duals of a nearby instance (a re-solve after entries were added) leave few
// conflicts.  The scaling's approximate duals -v/p give duals that also hold on the rest
// of A (what the certificate of sa_assign checks), but under them nearly every entry of B
// is almost tight, the greedy pass collides and the searches can sweep wide near-tied
// regions; solves that need no certificate start from the column minima.  Then a greedy
// assignment on each
// row's least-reduced-cost column and augmenting row reduction; each free row then runs
// Dijkstra over columns with a binary heap until no column in the heap is nearer than the
// nearest free column reached; the prices of the columns finalised before it are lowered
// by (d_target - d_j) and the path is flipped.  At the end
// u_i = c_{i,sigma(i)} - v_{sigma(i)} and (alpha, beta) = (-u, -v) are optimal LP duals
// of the maximisation: alpha_i + beta_j >= log w_ij on B, with equality on sigma.
#include <cmath>
#include <cstdint>
#include <limits>
#include <queue>
#include <utility>
#include <vector>

#include "sa_internal.h"

namespace sa {

sa_status sparse_assign(int n, const int64_t* row_ptr, const int32_t* col, const double* logw,
                        int32_t* perm, double* alpha, double* beta, const double* price0, SspFn ssp,
                        void* ssp_user) {
    const double INF = std::numeric_limits<double>::infinity();
    // a compacted copy of B for every loop below: allowed entries only, with their costs
    std::vector<int64_t> srp(n + 1, 0);
    std::vector<int32_t> scol;
    std::vector<double> scost;
    scol.reserve((size_t)row_ptr[n]);
    scost.reserve((size_t)row_ptr[n]);
    for (int i = 0; i < n; ++i) {
        for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e)
            if (logw[e] > -INF) {
                scol.push_back(col[e]);
                scost.push_back(-logw[e]);
            }
        srp[i + 1] = (int64_t)scol.size();
    }
    std::vector<double> v(n, INF);
    for (size_t e = 0; e < scol.size(); ++e)
        if (scost[e] < v[scol[e]]) v[scol[e]] = scost[e];
    for (int j = 0; j < n; ++j)
        if (v[j] == INF) {
            set_error("reduced instance: column %d has no allowed entry", j);
            return SA_E_NO_PERFECT_MATCHING;
        }
    if (price0)
        for (int j = 0; j < n; ++j)
            if (std::isfinite(price0[j])) v[j] = price0[j];
    std::vector<int32_t> rmatch(n, -1), cmatch(n, -1);
    std::vector<double> mcost(n, INF);   // cost -log w of each row's assigned entry
    // greedy assignment on least-reduced-cost columns
    for (int i = 0; i < n; ++i) {
        double best = INF, bc = INF;
        int bj = -1;
        for (int64_t e = srp[i]; e < srp[i + 1]; ++e) {
            const double h = scost[e] - v[scol[e]];
            if (h < best) { best = h; bj = scol[e]; bc = scost[e]; }
        }
        if (bj < 0) {
            set_error("reduced instance: row %d has no allowed entry", i);
            return SA_E_NO_PERFECT_MATCHING;
        }
        if (cmatch[bj] < 0) { cmatch[bj] = i; rmatch[i] = bj; mcost[i] = bc; }
    }
    // Augmenting row reduction (Jonker and Volgenant, 1987): a free row takes its least
    // reduced-cost column j1; when that is strictly below the second least, the price of j1
    // drops by the difference, so j1 stays the row's least after the change and the row
    // displaced from j1 (if any) is tried next.  Prices only drop, which keeps every
    // assigned row on a least-reduced-cost column.  Two passes, each bounded in work.
    {
        std::vector<int32_t> freel;
        for (int pass = 0; pass < 2; ++pass) {
            freel.clear();
            for (int i = 0; i < n; ++i)
                if (rmatch[i] < 0) freel.push_back(i);
            size_t k = 0;
            int64_t budget = 8 * (int64_t)n + 64;
            while (k < freel.size() && budget-- > 0) {
                const int i = freel[k++];
                double u1 = INF, u2 = INF, c1 = INF, c2 = INF;
                int j1 = -1, j2 = -1;
                for (int64_t e = srp[i]; e < srp[i + 1]; ++e) {
                    const int j = scol[e];
                    const double h = scost[e] - v[j];
                    if (h < u1) {
                        u2 = u1; j2 = j1; c2 = c1;
                        u1 = h; j1 = j; c1 = scost[e];
                    } else if (h < u2) {
                        u2 = h; j2 = j; c2 = scost[e];
                    }
                }
                if (j1 < 0) break;   // no allowed entry: reported by the search below
                int i0 = cmatch[j1];
                if (u1 < u2) {
                    if (j2 >= 0) v[j1] -= u2 - u1;
                } else if (i0 >= 0 && j2 >= 0) {
                    j1 = j2;   // tie: take the second column instead of displacing
                    c1 = c2;
                    i0 = cmatch[j1];
                }
                if (i0 >= 0) {
                    rmatch[i0] = -1;
                    if (u1 < u2 && k > 0) freel[--k] = i0;   // try the displaced row at once
                    else freel.push_back(i0);
                }
                cmatch[j1] = i;
                rmatch[i] = j1;
                mcost[i] = c1;
            }
        }
    }
    if (ssp) {
        SspState st{n, row_ptr, col, logw, v.data(), rmatch.data(), cmatch.data(), mcost.data()};
        const sa_status rc = ssp(ssp_user, st);
        if (rc) return rc;
    }
    // per column and search: state 2*epoch once reached (dist, pred, pcost valid), 2*epoch+1
    // once scanned; pcost is the cost of the entry (pred, j)
    std::vector<double> dist(n, INF), pcost(n, INF);
    std::vector<int32_t> pred(n, -1), scanned;
    std::vector<int64_t> state(n, 0);
    scanned.reserve(n);
    typedef std::pair<double, int32_t> Item;
    std::vector<Item> heapbuf;
    int64_t epoch = 0;
    for (int r = 0; r < n; ++r) {
        if (rmatch[r] >= 0) continue;
        ++epoch;
        const int64_t reached = 2 * epoch, finished = 2 * epoch + 1;
        scanned.clear();
        heapbuf.clear();
        std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap(std::greater<Item>(), std::move(heapbuf));
        // the nearest free column reached so far: it goes to no heap, and the search ends
        // as soon as no column in the heap is strictly nearer (Dijkstra's stopping rule at
        // the first target; on ties it saves scanning every matched column at that distance)
        int sink = -1;
        double dmin = INF;
        for (int64_t e = srp[r]; e < srp[r + 1]; ++e) {
            const int j = scol[e];
            const double d = scost[e] - v[j];
            if (state[j] != reached || d < dist[j]) {
                state[j] = reached;
                dist[j] = d;
                pred[j] = r;
                pcost[j] = scost[e];
                if (cmatch[j] < 0) {
                    if (d < dmin) { dmin = d; sink = j; }
                } else {
                    heap.push(Item(d, j));
                }
            }
        }
        while (!heap.empty()) {
            const Item top = heap.top();
            if (top.first >= dmin) break;
            heap.pop();
            const int j = top.second;
            if (state[j] == finished || top.first > dist[j]) continue;
            state[j] = finished;
            scanned.push_back(j);
            const int i = cmatch[j];
            // reduced cost of the assigned entry (i, j); zero-length step through row i
            const double ui = mcost[i] - v[j];
            const double dj = dist[j];
            for (int64_t e = srp[i]; e < srp[i + 1]; ++e) {
                const int k = scol[e];
                const double nd = dj + (scost[e] - v[k]) - ui;
                // a column not nearer than the nearest free one is never scanned and keeps
                // its price: its label does not matter
                if (!(nd < dmin)) continue;
                const int64_t sk = state[k];
                if (sk == finished || (sk == reached && !(nd < dist[k]))) continue;
                state[k] = reached;
                dist[k] = nd;
                pred[k] = i;
                pcost[k] = scost[e];
                if (cmatch[k] < 0) {
                    dmin = nd;
                    sink = k;
                } else {
                    heap.push(Item(nd, k));
                }
            }
        }
        if (sink < 0) {
            set_error("reduced instance has no perfect matching (row %d cannot be assigned)", r);
            return SA_E_NO_PERFECT_MATCHING;
        }
        for (int j : scanned) v[j] += dist[j] - dmin;
        // flip the alternating path ending at sink
        int j = sink;
        for (;;) {
            const int i = pred[j];
            cmatch[j] = i;
            const int prev = rmatch[i];
            rmatch[i] = j;
            mcost[i] = pcost[j];
            if (i == r) break;
            j = prev;
        }
    }
    for (int i = 0; i < n; ++i) perm[i] = rmatch[i];
    if (alpha || beta) {
        std::vector<double> u(n, 0.0);
        for (int i = 0; i < n; ++i) u[i] = mcost[i] - v[rmatch[i]];
        if (alpha) for (int i = 0; i < n; ++i) alpha[i] = -u[i];
        if (beta) for (int j = 0; j < n; ++j) beta[j] = -v[j];
    }
    return SA_OK;
}

// Of all LP-optimal duals of B for the optimal assignment perm, the componentwise largest
// beta with beta <= beta0 (beta0: maximisation-form column duals to stay close to, e.g. the
// scaling's v/p).  With the assignment fixed, optimality of (alpha, beta) is
//     alpha_i = log w_{i perm(i)} - beta_{perm(i)},
//     beta_{perm(i)} <= beta_j + (log w_{i perm(i)} - log w_ij)   for every entry (i, j),
// a system of difference constraints over the columns: edge j -> perm(i) of that length.
// Its largest solution below beta0 is the shortest-path labelling with beta0 as the
// starting label of every column.  Written relative to the given optimal duals
// (y = beta - beta_in) every edge length becomes the slack alpha_i + beta_j - log w_ij >= 0,
// so Dijkstra from all columns at once applies.  Columns whose beta0 is not finite keep
// their dual.  alpha and beta (in: optimal duals for perm, out: the projected ones).
sa_status project_duals(int n, const int64_t* row_ptr, const int32_t* col, const double* logw,
                        const int32_t* perm, const double* beta0, double* alpha, double* beta) {
    const double INF = std::numeric_limits<double>::infinity();
    const int64_t nnz = row_ptr[n];
    // columns of B: the rows holding an entry in each column, and that entry's log w
    std::vector<int64_t> cptr(n + 1, 0);
    for (int64_t e = 0; e < nnz; ++e) ++cptr[col[e] + 1];
    for (int j = 0; j < n; ++j) cptr[j + 1] += cptr[j];
    std::vector<int32_t> crow((size_t)std::max<int64_t>(nnz, 1));
    std::vector<double> clw((size_t)std::max<int64_t>(nnz, 1));
    std::vector<double> bsig(n, -INF);   // log w of each row's assigned entry
    {
        std::vector<int64_t> fill(cptr.begin(), cptr.end() - 1);
        for (int i = 0; i < n; ++i)
            for (int64_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
                const int64_t q = fill[col[e]]++;
                crow[q] = i;
                clw[q] = logw[e];
                if (col[e] == perm[i] && logw[e] > bsig[i]) bsig[i] = logw[e];   // repeated columns: the best
            }
    }
    for (int i = 0; i < n; ++i)
        if (!(bsig[i] > -INF)) {
            set_error("project_duals: row %d is not assigned to an allowed entry", i);
            return SA_E_INVALID;
        }
    std::vector<double> y(n);
    std::vector<char> done(n, 0);
    typedef std::pair<double, int32_t> Item;
    std::priority_queue<Item, std::vector<Item>, std::greater<Item>> heap;
    for (int j = 0; j < n; ++j) {
        y[j] = std::isfinite(beta0[j]) ? beta0[j] - beta[j] : 0.0;
        heap.push(Item(y[j], j));
    }
    while (!heap.empty()) {
        const Item top = heap.top();
        heap.pop();
        const int j = top.second;
        if (done[j] || top.first > y[j]) continue;
        done[j] = 1;
        for (int64_t q = cptr[j]; q < cptr[j + 1]; ++q) {
            if (!(clw[q] > -INF)) continue;
            const int i = crow[q];
            const int k = perm[i];
            if (k == j || done[k]) continue;
            const double slack = alpha[i] + beta[j] - clw[q];
            const double nd = y[j] + (slack > 0.0 ? slack : 0.0);
            if (nd < y[k]) {
                y[k] = nd;
                heap.push(Item(nd, k));
            }
        }
    }
    for (int j = 0; j < n; ++j) beta[j] += y[j];
    for (int i = 0; i < n; ++i) alpha[i] = bsig[i] - beta[perm[i]];
    return SA_OK;
}

}  // namespace sa
