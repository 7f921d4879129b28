/*
 * d2_oracle.c -- plain FP64 CPU oracle for the D2-clustering assignment step
 * (Zhang, Wang & Li, "Parallel D2-Clustering", arXiv 1302.0435).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  The product path
 * (paper_1302_0435_gb300/) never links, imports or calls it, and this file
 * shares no code, header, table or constant with the CUDA path.
 *
 * What it computes, each function citing the passage it follows:
 *   - weight normalisation so that every bag has total mass 1 (the equal-mass
 *     constraint of Eq. (D2opt): sum_r p_z^(r) = 1 and the row/column
 *     marginal constraints imply sum_alpha p_v^(alpha) = 1);
 *   - the ground cost c = ||z^(r) - v^(alpha)||^2 by explicit differences
 *     (Eq. (D2opt), objective);
 *   - the Mallows distance D^2 as the exact optimum of the transportation LP
 *     of Eq. (D2opt) with the centroid z fixed (the text right after
 *     Eq. (D2opt): "if z is fixed, D is the Mallows distance");
 *   - the nearest-centroid label of Alg. 2 Step 2.
 * The LP solver is the textbook transportation simplex (northwest-corner
 * start, u-v / MODI duals, most-negative reduced cost entering, min-ratio
 * leaving), written as dense loops with no blocking or fusion.  The paper
 * names no LP solver; any exact solver gives the same optimum value.
 *
 * Rounding: IEEE FP64, compile with -ffp-contract=off (no FMA contraction),
 * fixed summation orders.  Single-threaded per pair; the multi-pair entry
 * points spread independent pairs over POSIX threads (a harness around the
 * per-pair solve, not part of the arithmetic).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define D2O_OK 0
#define D2O_EINVAL (-1)
#define D2O_ENOMEM (-2)
#define D2O_ENOTCONVERGED (-3)

/* ------------------------------------------------------------------ */
/* Weight normalisation.  Eq. (D2opt) requires the centroid weights to */
/* sum to one and the marginal constraints then force the same total   */
/* for every object.  Inputs that are only approximately normalised   */
/* are divided by their sum; negative, NaN or zero-sum bags are        */
/* rejected.                                                           */
/* ------------------------------------------------------------------ */
int d2o_normalise(const double* w, int64_t m, double* out)
{
    if (m <= 0) return D2O_EINVAL;
    double s = 0.0;
    for (int64_t a = 0; a < m; ++a) {
        double x = w[a];
        if (!(x >= 0.0) || isinf(x)) return D2O_EINVAL; /* rejects NaN too */
        s += x;
    }
    if (!(s > 0.0) || isinf(s)) return D2O_EINVAL;
    for (int64_t a = 0; a < m; ++a) out[a] = w[a] / s;
    return D2O_OK;
}

/* ------------------------------------------------------------------ */
/* Ground cost of Eq. (D2opt): c[a][r] = ||x_a - y_r||^2, summed over   */
/* the coordinates in order, by explicit differences.                  */
/* ------------------------------------------------------------------ */
void d2o_cost(const double* x, int64_t m, const double* y, int64_t n, int32_t d, double* C)
{
    for (int64_t a = 0; a < m; ++a)
        for (int64_t r = 0; r < n; ++r) {
            double s = 0.0;
            for (int32_t k = 0; k < d; ++k) {
                double t = x[a * d + k] - y[r * d + k];
                s += t * t;
            }
            C[a * n + r] = s;
        }
}

/* Bipartite basis graph helpers: node a in [0,m) is row a, node m+r is
 * column r; an edge is a basic cell (a,r). */

/* Duals of the current basis: u_a + v_r = C[a][r] on every basic cell,
 * anchored at u_0 = 0 (the u-v method).  Breadth-first over the basis tree. */
static void solve_duals(const double* C, const unsigned char* B, int m, int n,
                        double* u, double* v, int* queue, unsigned char* seen)
{
    memset(seen, 0, (size_t)(m + n));
    int head = 0, tail = 0;
    u[0] = 0.0;
    seen[0] = 1;
    queue[tail++] = 0;
    while (head < tail) {
        int node = queue[head++];
        if (node < m) {
            int a = node;
            for (int r = 0; r < n; ++r)
                if (B[a * n + r] && !seen[m + r]) {
                    v[r] = C[a * n + r] - u[a];
                    seen[m + r] = 1;
                    queue[tail++] = m + r;
                }
        } else {
            int r = node - m;
            for (int a = 0; a < m; ++a)
                if (B[a * n + r] && !seen[a]) {
                    u[a] = C[a * n + r] - v[r];
                    seen[a] = 1;
                    queue[tail++] = a;
                }
        }
    }
}

/* The unique cycle closed by the entering cell (ea, er): the basis-tree path
 * from column er back to row ea.  Returned as the list of cells on that
 * path, starting at the cell touching column er.  Breadth-first search from
 * row ea with predecessor links. */
static int tree_path(const unsigned char* B, int m, int n, int ea, int er,
                     int* path_cells, int* queue, int* pred_cell, unsigned char* seen)
{
    memset(seen, 0, (size_t)(m + n));
    int head = 0, tail = 0;
    seen[ea] = 1;
    pred_cell[ea] = -1;
    queue[tail++] = ea;
    while (head < tail) {
        int node = queue[head++];
        if (node == m + er) break;
        if (node < m) {
            int a = node;
            for (int r = 0; r < n; ++r)
                if (B[a * n + r] && !seen[m + r]) {
                    seen[m + r] = 1;
                    pred_cell[m + r] = a * n + r;
                    queue[tail++] = m + r;
                }
        } else {
            int r = node - m;
            for (int a = 0; a < m; ++a)
                if (B[a * n + r] && !seen[a]) {
                    seen[a] = 1;
                    pred_cell[a] = a * n + r;
                    queue[tail++] = a;
                }
        }
    }
    if (!seen[m + er]) return -1; /* basis not spanning: cannot happen */
    int len = 0;
    int node = m + er;
    while (node != ea) {
        int cell = pred_cell[node];
        path_cells[len++] = cell;
        int a = cell / n, r = cell % n;
        node = (node == m + r) ? a : m + r;
    }
    return len;
}

/* ------------------------------------------------------------------ */
/* Exact transportation LP of Eq. (D2opt) with z fixed:                 */
/*   min sum_{a,r} w[a][r] C[a][r]  s.t.  sum_r w[a][r] = p[a],         */
/*   sum_a w[a][r] = q[r],  w >= 0.                                     */
/* Transportation simplex:                                              */
/*   1. northwest-corner basic feasible solution with m+n-1 basic cells */
/*      (degenerate zero-flow cells kept, so the basis is a tree);      */
/*   2. duals u, v with u_a + v_r = C on basic cells;                   */
/*   3. reduced costs C - u - v; stop when all >= -tol,                 */
/*      tol = 1e-12 * max(1, max C);                                    */
/*   4. enter the most negative cell (ties: smallest a*n+r); after      */
/*      2(m+n) consecutive degenerate pivots use Bland's rule (smallest */
/*      index with negative reduced cost) until a pivot moves flow;     */
/*   5. the cycle through the entering cell; alternate +/-; the leaving */
/*      cell is the "-" cell of least flow (ties: smallest a*n+r);      */
/*   6. shift that flow around the cycle.                               */
/* Objective: sum over basic cells in index order, compensated (Kahan). */
/* Outputs w (m*n dense), u (m), v (n), the objective and the pivot     */
/* count.  Returns D2O_ENOTCONVERGED if the pivot cap is reached.       */
/* ------------------------------------------------------------------ */
int d2o_transport(const double* C, const double* p, int64_t m64, const double* q, int64_t n64,
                  double* w, double* u, double* v, double* obj, int64_t* pivots_out)
{
    if (m64 <= 0 || n64 <= 0 || m64 > 4096 || n64 > 4096) return D2O_EINVAL;
    int m = (int)m64, n = (int)n64;
    int N = m + n;
    unsigned char* B = (unsigned char*)calloc((size_t)m * n, 1);
    double* rs = (double*)malloc(sizeof(double) * (size_t)m);
    double* cs = (double*)malloc(sizeof(double) * (size_t)n);
    int* queue = (int*)malloc(sizeof(int) * (size_t)N);
    int* pred = (int*)malloc(sizeof(int) * (size_t)N);
    int* path = (int*)malloc(sizeof(int) * (size_t)N);
    unsigned char* seen = (unsigned char*)malloc((size_t)N);
    if (!B || !rs || !cs || !queue || !pred || !path || !seen) {
        free(B); free(rs); free(cs); free(queue); free(pred); free(path); free(seen);
        return D2O_ENOMEM;
    }
    memset(w, 0, sizeof(double) * (size_t)m * n);
    for (int a = 0; a < m; ++a) rs[a] = p[a];
    for (int r = 0; r < n; ++r) cs[r] = q[r];

    /* 1. northwest corner: walk right/down from (0,0), m+n-1 cells */
    {
        int a = 0, r = 0;
        for (int s = 0; s < m + n - 1; ++s) {
            double t = rs[a] < cs[r] ? rs[a] : cs[r];
            w[a * n + r] = t;
            B[a * n + r] = 1;
            rs[a] -= t;
            cs[r] -= t;
            if (s == m + n - 2) break;
            if (a < m - 1 && (r == n - 1 || rs[a] <= cs[r])) ++a; else ++r;
        }
    }

    double cmax = 0.0;
    for (int64_t t = 0; t < (int64_t)m * n; ++t) if (C[t] > cmax) cmax = C[t];
    const double tol = 1e-12 * (cmax > 1.0 ? cmax : 1.0);
    const int64_t cap = 1000LL * N + 100000LL;
    int64_t pivots = 0;
    int degenerate_run = 0;
    int bland = 0;
    int status = D2O_OK;

    for (;;) {
        /* 2. duals */
        solve_duals(C, B, m, n, u, v, queue, seen);
        /* 3./4. pricing */
        int enter = -1;
        double best = -tol;
        for (int a = 0; a < m && !(bland && enter >= 0); ++a)
            for (int r = 0; r < n; ++r) {
                if (B[a * n + r]) continue;
                double red = C[a * n + r] - u[a] - v[r];
                if (bland) {
                    if (red < -tol) { enter = a * n + r; break; }
                } else if (red < best) {
                    best = red;
                    enter = a * n + r;
                }
            }
        if (enter < 0) break; /* optimal */
        if (pivots >= cap) { status = D2O_ENOTCONVERGED; break; }
        ++pivots;

        /* 5. cycle and ratio test */
        int ea = enter / n, er = enter % n;
        int len = tree_path(B, m, n, ea, er, path, queue, pred, seen);
        if (len < 0) { status = D2O_EINVAL; break; }
        /* path[0] touches column er and gets "-", then alternate */
        int leave = -1;
        double theta = 0.0;
        for (int k = 0; k < len; k += 2) {
            int cell = path[k];
            if (leave < 0 || w[cell] < theta || (w[cell] == theta && cell < leave)) {
                leave = cell;
                theta = w[cell];
            }
        }
        if (leave < 0) { status = D2O_EINVAL; break; } /* empty cycle: cannot happen */
        /* 6. shift flow */
        for (int k = 0; k < len; ++k) {
            int cell = path[k];
            if (k % 2 == 0) w[cell] -= theta; else w[cell] += theta;
        }
        w[enter] = theta;
        B[enter] = 1;
        B[leave] = 0;
        w[leave] = 0.0;

        if (theta == 0.0) {
            if (++degenerate_run >= 2 * N) bland = 1;
        } else {
            degenerate_run = 0;
            bland = 0;
        }
    }

    /* objective: compensated sum over basic cells in index order */
    double s = 0.0, comp = 0.0;
    for (int64_t t = 0; t < (int64_t)m * n; ++t) {
        if (!B[t]) continue;
        double term = w[t] * C[t] - comp;
        double nxt = s + term;
        comp = (nxt - s) - term;
        s = nxt;
    }
    *obj = s;
    if (pivots_out) *pivots_out = pivots;
    free(B); free(rs); free(cs); free(queue); free(pred); free(path); free(seen);
    return status;
}

/* Mallows distance D^2 between two bags (Eq. (D2opt) with z fixed):
 * normalise both weight vectors, build the cost, solve the LP.
 * flow (m*n), u (m), v (n) and pivots may be NULL. */
int d2o_mallows(const double* x, const double* wx, int64_t m, const double* y, const double* wy,
                int64_t n, int32_t d, double* dist2, double* flow, double* u, double* v,
                int64_t* pivots)
{
    if (m <= 0 || n <= 0 || d <= 0) return D2O_EINVAL;
    double* p = (double*)malloc(sizeof(double) * (size_t)m);
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    double* C = (double*)malloc(sizeof(double) * (size_t)(m * n));
    double* W = flow ? flow : (double*)malloc(sizeof(double) * (size_t)(m * n));
    double* U = u ? u : (double*)malloc(sizeof(double) * (size_t)m);
    double* V = v ? v : (double*)malloc(sizeof(double) * (size_t)n);
    int st = D2O_ENOMEM;
    if (p && q && C && W && U && V) {
        st = d2o_normalise(wx, m, p);
        if (st == D2O_OK) st = d2o_normalise(wy, n, q);
        if (st == D2O_OK) {
            d2o_cost(x, m, y, n, d, C);
            st = d2o_transport(C, p, m, q, n, W, U, V, dist2, pivots);
        }
    }
    free(p); free(q); free(C);
    if (!flow) free(W);
    if (!u) free(U);
    if (!v) free(V);
    return st;
}

/* ------------------------------------------------------------------ */
/* Pair lists and nearest-centroid labels.                              */
/* Bags are CSR: bag b owns supports [off[b], off[b+1]) of loc (row-    */
/* major, d per support) and w.                                         */
/* ------------------------------------------------------------------ */
typedef struct {
    const double *xloc, *xw; const int64_t* xoff;
    const double *yloc, *yw; const int64_t* yoff;
    int32_t d;
    /* pair mode */
    const int64_t *pi, *pj; int64_t npairs; double* out; int32_t* st_out; int64_t* piv_out;
    /* assign mode */
    int64_t N, K; int32_t* labels; double* dist2; double* all;
    /* work split */
    int64_t begin, end;
    int status;
} job_t;

static int solve_pair(const job_t* J, int64_t i, int64_t j, double* out, int64_t* piv)
{
    int64_t m = J->xoff[i + 1] - J->xoff[i];
    int64_t n = J->yoff[j + 1] - J->yoff[j];
    return d2o_mallows(J->xloc + J->xoff[i] * J->d, J->xw + J->xoff[i], m,
                       J->yloc + J->yoff[j] * J->d, J->yw + J->yoff[j], n, J->d,
                       out, NULL, NULL, NULL, piv);
}

static void* pairs_worker(void* arg)
{
    job_t* J = (job_t*)arg;
    for (int64_t t = J->begin; t < J->end; ++t) {
        double dd = NAN;
        int64_t piv = 0;
        int st = solve_pair(J, J->pi[t], J->pj[t], &dd, &piv);
        J->out[t] = dd;
        if (J->piv_out) J->piv_out[t] = piv;
        if (J->st_out) J->st_out[t] = st;
        if (st != D2O_OK && J->status == D2O_OK) J->status = st;
    }
    return NULL;
}

/* Alg. 2 Step 2: C(i) = argmin_j D(v_i, z_j).  Ties go to the smallest j
 * (the paper does not say; any smallest-index rule is a valid argmin). */
static void* assign_worker(void* arg)
{
    job_t* J = (job_t*)arg;
    for (int64_t i = J->begin; i < J->end; ++i) {
        int32_t best_j = -1;
        double best = INFINITY;
        for (int64_t j = 0; j < J->K; ++j) {
            double dd = NAN;
            int st = solve_pair(J, i, j, &dd, NULL);
            if (st != D2O_OK && J->status == D2O_OK) J->status = st;
            if (J->all) J->all[i * J->K + j] = dd;
            if (dd < best) { best = dd; best_j = (int32_t)j; }
        }
        J->labels[i] = best_j;
        J->dist2[i] = best;
    }
    return NULL;
}

static int run_threads(job_t* base, int64_t count, int32_t nthreads, void* (*fn)(void*))
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (count < nthreads) nthreads = count > 0 ? (int32_t)count : 1;
    job_t jobs[256];
    pthread_t th[256];
    int64_t chunk = (count + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *base;
        jobs[t].begin = t * chunk < count ? t * chunk : count;
        jobs[t].end = (t + 1) * chunk < count ? (t + 1) * chunk : count;
        jobs[t].status = D2O_OK;
    }
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) break;
        started = t;
    }
    fn(&jobs[0]);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    for (int t = started + 1; t < nthreads; ++t) fn(&jobs[t]); /* threads that failed to start */
    int st = D2O_OK;
    for (int t = 0; t < nthreads; ++t) if (jobs[t].status != D2O_OK) st = jobs[t].status;
    return st;
}

/* D^2 for a list of (object, centroid) pairs; status and pivots (per pair)
 * may be NULL. */
int d2o_mallows_pairs(const double* xloc, const double* xw, const int64_t* xoff,
                      const double* yloc, const double* yw, const int64_t* yoff, int32_t d,
                      const int64_t* pi, const int64_t* pj, int64_t npairs, int32_t nthreads,
                      double* dist2, int32_t* status, int64_t* pivots)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.xloc = xloc; J.xw = xw; J.xoff = xoff; J.yloc = yloc; J.yw = yw; J.yoff = yoff; J.d = d;
    J.pi = pi; J.pj = pj; J.npairs = npairs; J.out = dist2; J.st_out = status; J.piv_out = pivots;
    return run_threads(&J, npairs, nthreads, pairs_worker);
}

/* Labels and distances of Alg. 2 Step 2 for N objects against K centroids.
 * all_dist2 (N*K, row-major) may be NULL. */
int d2o_assign(const double* xloc, const double* xw, const int64_t* xoff, int64_t N,
               const double* yloc, const double* yw, const int64_t* yoff, int64_t K, int32_t d,
               int32_t nthreads, int32_t* labels, double* dist2, double* all_dist2)
{
    job_t J;
    memset(&J, 0, sizeof J);
    J.xloc = xloc; J.xw = xw; J.xoff = xoff; J.yloc = yloc; J.yw = yw; J.yoff = yoff; J.d = d;
    J.N = N; J.K = K; J.labels = labels; J.dist2 = dist2; J.all = all_dist2;
    return run_threads(&J, N, nthreads, assign_worker);
}
