/* Host sanitizer driver for the FP64 oracle (test infrastructure): runs the
 * oracle's transportation simplex, Mallows distance and threaded
 * assignment on random, degenerate and zero-weight problems, and checks
 * each result against its own certificate (feasible flows, dual
 * feasibility, zero duality gap), so that the address, undefined-behaviour
 * and thread sanitizers see every code path of the solver.  Exit status 0
 * when every check passes. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

int d2o_transport(const double* C, const double* p, int64_t m, const double* q, int64_t n,
                  double* w, double* u, double* v, double* obj, int64_t* pivots);
int d2o_mallows(const double* x, const double* wx, int64_t m, const double* y, const double* wy,
                int64_t n, int32_t d, double* dist2, double* flow, double* u, double* v,
                int64_t* pivots);
int d2o_assign(const double* xloc, const double* xw, const int64_t* xoff, int64_t N,
               const double* yloc, const double* yw, const int64_t* yoff, int64_t K, int32_t d,
               int32_t nthreads, int32_t* labels, double* dist2, double* all_dist2);

static uint64_t rs = 88172645463325252ull;
static double urand(void) {  /* xorshift64 */
  rs ^= rs << 13; rs ^= rs >> 7; rs ^= rs << 17;
  return (double)(rs >> 11) * 0x1p-53;
}

static int check_lp(int m, int n, const double* C, const double* p, const double* q) {
  double* w = malloc(sizeof(double) * m * n);
  double* u = malloc(sizeof(double) * m);
  double* v = malloc(sizeof(double) * n);
  double obj = 0.0, cmax = 0.0;
  int64_t piv = 0;
  int bad = d2o_transport(C, p, m, q, n, w, u, v, &obj, &piv) != 0;
  for (int k = 0; k < m * n; ++k) cmax = fmax(cmax, fabs(C[k]));
  const double tol = 1e-9 * (1.0 + cmax);
  double dual = 0.0;
  for (int a = 0; a < m; ++a) {
    double rsum = 0.0;
    for (int r = 0; r < n; ++r) {
      rsum += w[a * n + r];
      if (w[a * n + r] < -1e-12 || C[a * n + r] - u[a] - v[r] < -tol) bad = 1;
    }
    if (fabs(rsum - p[a]) > 1e-9) bad = 1;
    dual += p[a] * u[a];
  }
  for (int r = 0; r < n; ++r) {
    double csum = 0.0;
    for (int a = 0; a < m; ++a) csum += w[a * n + r];
    if (fabs(csum - q[r]) > 1e-9) bad = 1;
    dual += q[r] * v[r];
  }
  if (fabs(dual - obj) > tol) bad = 1;
  free(w); free(u); free(v);
  return bad;
}

int main(void) {
  int fails = 0;
  for (int t = 0; t < 400; ++t) {
    const int m = 1 + (int)(urand() * 12), n = 1 + (int)(urand() * 12);
    double* C = malloc(sizeof(double) * m * n);
    double* p = malloc(sizeof(double) * m);
    double* q = malloc(sizeof(double) * n);
    const int kind = t % 4;  /* 0 random, 1 integer (degenerate), 2 zero weights, 3 uniform */
    double sp = 0.0, sq = 0.0;
    for (int k = 0; k < m * n; ++k) C[k] = kind == 1 ? (double)(int)(urand() * 4) : urand() * 10;
    for (int a = 0; a < m; ++a) {
      p[a] = kind == 1 ? 1.0 + (int)(urand() * 3) : (kind == 2 && urand() < 0.4 ? 0.0 : urand());
      if (kind == 3) p[a] = 1.0;
      sp += p[a];
    }
    for (int r = 0; r < n; ++r) {
      q[r] = kind == 1 ? 1.0 + (int)(urand() * 3) : (kind == 2 && urand() < 0.4 ? 0.0 : urand());
      if (kind == 3) q[r] = 1.0;
      sq += q[r];
    }
    if (sp == 0.0) { p[0] = 1.0; sp = 1.0; }
    if (sq == 0.0) { q[0] = 1.0; sq = 1.0; }
    for (int a = 0; a < m; ++a) p[a] /= sp;
    for (int r = 0; r < n; ++r) q[r] /= sq;
    fails += check_lp(m, n, C, p, q);
    free(C); free(p); free(q);
  }
  /* bags through the Mallows entry point and the threaded assignment */
  enum { N = 300, K = 7, D = 3 };
  int64_t xoff[N + 1], yoff[K + 1];
  xoff[0] = 0;
  for (int i = 0; i < N; ++i) xoff[i + 1] = xoff[i] + 1 + (int64_t)(urand() * 9);
  yoff[0] = 0;
  for (int j = 0; j < K; ++j) yoff[j + 1] = yoff[j] + 1 + (int64_t)(urand() * 6);
  double* xl = malloc(sizeof(double) * xoff[N] * D);
  double* xw = malloc(sizeof(double) * xoff[N]);
  double* yl = malloc(sizeof(double) * yoff[K] * D);
  double* yw = malloc(sizeof(double) * yoff[K]);
  for (int64_t k = 0; k < xoff[N] * D; ++k) xl[k] = urand() * 4;
  for (int64_t k = 0; k < xoff[N]; ++k) xw[k] = urand() + 1e-3;
  for (int64_t k = 0; k < yoff[K] * D; ++k) yl[k] = urand() * 4;
  for (int64_t k = 0; k < yoff[K]; ++k) yw[k] = urand() + 1e-3;
  int32_t lab1[N], lab4[N];
  double d1[N], d4[N];
  double* all = malloc(sizeof(double) * N * K);
  fails += d2o_assign(xl, xw, xoff, N, yl, yw, yoff, K, D, 1, lab1, d1, NULL) != 0;
  fails += d2o_assign(xl, xw, xoff, N, yl, yw, yoff, K, D, 4, lab4, d4, all) != 0;
  for (int i = 0; i < N; ++i) {
    if (lab1[i] != lab4[i] || d1[i] != d4[i]) ++fails;  /* thread count must not matter */
    const int64_t j = lab1[i];
    double dd = 0.0, flow[64 * 64], u[64], v[64];
    int64_t piv = 0;
    fails += d2o_mallows(xl + xoff[i] * D, xw + xoff[i], xoff[i + 1] - xoff[i], yl + yoff[j] * D,
                         yw + yoff[j], yoff[j + 1] - yoff[j], D, &dd, flow, u, v, &piv) != 0;
    if (dd != d1[i] || all[i * K + j] != d1[i]) ++fails;
  }
  free(xl); free(xw); free(yl); free(yw); free(all);
  printf("oracle sanitize driver: %d failures\n", fails);
  return fails != 0;
}
