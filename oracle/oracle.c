/*
 * CPU oracle for the tridiagonal partition method (Veneva, "ML-Based Optimum
 * Sub-system Size for the GPU Implementation of the Tridiagonal Partition
 * Method", arXiv 2510.27351).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only tests, the smoke check and the bench's
 * CPU-baseline leg may load it; the product library never links it and shares
 * no code, header or constant with it.
 *
 * Conventions (all functions):
 *   row i of A reads  a[i] x[i-1] + b[i] x[i] + c[i] x[i+1] = d[i],
 *   a[0] and c[n-1] are ignored (treated as 0).  Arithmetic is IEEE binary64
 *   unless the name says otherwise; the dense solver uses long double.
 *   Return value 0 = success, 1 = zero pivot, 2 = bad argument.
 *
 * Pins (which independent facts hold each function in place) are listed per
 * function; the tests under tests/test_oracle_*.py implement them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_ZERO_PIVOT 1
#define OR_BADARG 2

/* ------------------------------------------------------------------------ */
/* Thomas algorithm (sequential LU of a tridiagonal matrix without pivoting). */
/* The paper solves the interface system of Stage 2 sequentially on the host  */
/* (Sec. I, Fig. 3); Thomas is the sequential direct solver used for it here. */
/* Pinned by: long-double dense elimination (n <= 64), LAPACK banded solve,   */
/* manufactured solutions, the DST closed form for constant diagonals.        */
/* ------------------------------------------------------------------------ */
int or_thomas(int64_t n, const double* a, const double* b, const double* c, const double* d, double* x) {
  if (n < 1) return OR_BADARG;
  double* cp = (double*)malloc(sizeof(double) * (size_t)n);
  double* dp = (double*)malloc(sizeof(double) * (size_t)n);
  if (!cp || !dp) { free(cp); free(dp); return OR_BADARG; }
  int rc = OR_OK;
  /* forward elimination: row i becomes x[i] + cp[i] x[i+1] = dp[i] */
  double den = b[0];
  if (den == 0.0) rc = OR_ZERO_PIVOT;
  cp[0] = (n > 1 ? c[0] : 0.0) / den;
  dp[0] = d[0] / den;
  for (int64_t i = 1; i < n; i++) {
    den = b[i] - a[i] * cp[i - 1];
    if (den == 0.0) rc = OR_ZERO_PIVOT;
    cp[i] = (i < n - 1 ? c[i] : 0.0) / den;
    dp[i] = (d[i] - a[i] * dp[i - 1]) / den;
  }
  /* back substitution */
  x[n - 1] = dp[n - 1];
  for (int64_t i = n - 2; i >= 0; i--) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
  return rc;
}

/* Same algorithm in binary32 arithmetic (inputs and outputs binary32).  Used
 * to bound the error a single-precision solve may have before refinement. */
int or_thomas_f32(int64_t n, const float* a, const float* b, const float* c, const float* d, float* x) {
  if (n < 1) return OR_BADARG;
  float* cp = (float*)malloc(sizeof(float) * (size_t)n);
  float* dp = (float*)malloc(sizeof(float) * (size_t)n);
  if (!cp || !dp) { free(cp); free(dp); return OR_BADARG; }
  int rc = OR_OK;
  float den = b[0];
  if (den == 0.0f) rc = OR_ZERO_PIVOT;
  cp[0] = (n > 1 ? c[0] : 0.0f) / den;
  dp[0] = d[0] / den;
  for (int64_t i = 1; i < n; i++) {
    den = b[i] - a[i] * cp[i - 1];
    if (den == 0.0f) rc = OR_ZERO_PIVOT;
    cp[i] = (i < n - 1 ? c[i] : 0.0f) / den;
    dp[i] = (d[i] - a[i] * dp[i - 1]) / den;
  }
  x[n - 1] = dp[n - 1];
  for (int64_t i = n - 2; i >= 0; i--) x[i] = dp[i] - cp[i] * x[i + 1];
  free(cp);
  free(dp);
  return rc;
}

/* Thomas on each system of a batch.  System j occupies elements
 *   base[j] + i*elem_stride, i = 0..len[j]-1
 * of every array.  Contiguous uneven batches use base = offsets[j],
 * len = offsets[j+1]-offsets[j], elem_stride = 1. */
int or_thomas_batched(int32_t B, const int64_t* base, const int64_t* len, int64_t elem_stride,
                      const double* a, const double* b, const double* c, const double* d, double* x) {
  int rc = OR_OK;
  for (int32_t j = 0; j < B; j++) {
    int64_t n = len[j];
    if (n < 1) continue;
    double* buf = (double*)malloc(sizeof(double) * 5 * (size_t)n);
    if (!buf) return OR_BADARG;
    double *aa = buf, *bb = buf + n, *cc = buf + 2 * n, *dd = buf + 3 * n, *xx = buf + 4 * n;
    for (int64_t i = 0; i < n; i++) {
      int64_t p = base[j] + i * elem_stride;
      aa[i] = a[p]; bb[i] = b[p]; cc[i] = c[p]; dd[i] = d[p];
    }
    int r = or_thomas(n, aa, bb, cc, dd, xx);
    if (r) rc = r;
    for (int64_t i = 0; i < n; i++) x[base[j] + i * elem_stride] = xx[i];
    free(buf);
  }
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Parallel partition method, non-recursive (Sec. I: three stages).          */
/*                                                                           */
/* Stage 1: split the n unknowns into consecutive sub-systems of s rows      */
/*   (block k holds rows L_k = k*s .. R_k = min(n,(k+1)s)-1; the last block  */
/*   may be shorter).  For every block, eliminate its interior rows           */
/*   L_k+1..R_k-1 so that two "interface equations" remain, one for x[L_k]   */
/*   and one for x[R_k].  With T_k the interior matrix, the interior values  */
/*   are x_int = g + v x[L_k] + w x[R_k], where                              */
/*       T_k g = d_int,  T_k v = -a[L_k+1] e_first,  T_k w = -c[R_k-1] e_last. */
/*   Substituting x[L_k+1] and x[R_k-1] into rows L_k and R_k gives           */
/*     a[L] x[L-1] + (b[L] + c[L] v_1) x[L] + c[L] w_1 x[R] = d[L] - c[L] g_1  */
/*     a[R] v_e x[L] + (b[R] + a[R] w_e) x[R] + c[R] x[R+1] = d[R] - a[R] g_e  */
/*   (index 1 = first interior row, e = last interior row).                  */
/*   A block of 2 rows has no interior: its two rows are copied.  A block of */
/*   1 row contributes that row.                                             */
/* Stage 2: the interface equations, in the order x[L_0], x[R_0], x[L_1], ... */
/*   form a tridiagonal interface system (Sec. I), solved here by Thomas.    */
/* Stage 3: with x[L_k], x[R_k] known, each interior is the independent      */
/*   system T_k x_int = d_int - a[L+1] x[L] e_first - c[R-1] x[R] e_last.     */
/*                                                                           */
/* Outputs: x (length n); optionally the interface system (ra, rb, rc, rd of */
/* length *M) and the global row index of each interface unknown (ridx).     */
/* Pinned by: equality with Thomas; s >= n and s == 2 special cases; the     */
/* interface system equals the dense Schur complement onto the interface     */
/* indices (computed with numpy); strict diagonal dominance (Sec. I claim).  */
/* ------------------------------------------------------------------------ */
int or_partition(int64_t n, int64_t s, const double* a, const double* b, const double* c, const double* d,
                 double* x, double* ra, double* rb, double* rc, double* rd, int64_t* ridx, int64_t* M_out) {
  if (n < 1 || s < 2) return OR_BADARG;
  int64_t m = (n + s - 1) / s;
  int64_t Mmax = 2 * m;
  double* A2 = (double*)calloc((size_t)Mmax, sizeof(double));
  double* B2 = (double*)calloc((size_t)Mmax, sizeof(double));
  double* C2 = (double*)calloc((size_t)Mmax, sizeof(double));
  double* D2 = (double*)calloc((size_t)Mmax, sizeof(double));
  double* Y = (double*)calloc((size_t)Mmax, sizeof(double));
  int64_t* I2 = (int64_t*)calloc((size_t)Mmax, sizeof(int64_t));
  /* scratch for the interior solves: three right-hand sides */
  double* ta = (double*)malloc(sizeof(double) * (size_t)s);
  double* tb = (double*)malloc(sizeof(double) * (size_t)s);
  double* tc = (double*)malloc(sizeof(double) * (size_t)s);
  double* rhs = (double*)malloc(sizeof(double) * (size_t)s);
  double* g = (double*)malloc(sizeof(double) * (size_t)s);
  double* v = (double*)malloc(sizeof(double) * (size_t)s);
  double* w = (double*)malloc(sizeof(double) * (size_t)s);
  int rcode = OR_OK;
  if (!A2 || !B2 || !C2 || !D2 || !Y || !I2 || !ta || !tb || !tc || !rhs || !g || !v || !w) { rcode = OR_BADARG; goto done; }

  /* effective coefficients: a[0] = c[n-1] = 0 */
#define AA(i) ((i) == 0 ? 0.0 : a[(i)])
#define CC(i) ((i) == n - 1 ? 0.0 : c[(i)])

  int64_t M = 0;
  /* ---- Stage 1 ---- */
  for (int64_t k = 0; k < m; k++) {
    int64_t L = k * s, R = (k + 1) * s - 1;
    if (R > n - 1) R = n - 1;
    int64_t nk = R - L + 1;
    if (nk == 1) {
      A2[M] = AA(L); B2[M] = b[L]; C2[M] = CC(L); D2[M] = d[L]; I2[M] = L; M++;
      continue;
    }
    if (nk == 2) {
      A2[M] = AA(L); B2[M] = b[L]; C2[M] = CC(L); D2[M] = d[L]; I2[M] = L; M++;
      A2[M] = AA(R); B2[M] = b[R]; C2[M] = CC(R); D2[M] = d[R]; I2[M] = R; M++;
      continue;
    }
    int64_t ni = nk - 2; /* interior rows L+1..R-1 */
    for (int64_t i = 0; i < ni; i++) {
      ta[i] = a[L + 1 + i]; tb[i] = b[L + 1 + i]; tc[i] = c[L + 1 + i];
    }
    /* T g = d_int */
    for (int64_t i = 0; i < ni; i++) rhs[i] = d[L + 1 + i];
    int r1 = or_thomas(ni, ta, tb, tc, rhs, g);
    /* T v = -a[L+1] e_first */
    for (int64_t i = 0; i < ni; i++) rhs[i] = 0.0;
    rhs[0] = -a[L + 1];
    int r2 = or_thomas(ni, ta, tb, tc, rhs, v);
    /* T w = -c[R-1] e_last */
    for (int64_t i = 0; i < ni; i++) rhs[i] = 0.0;
    rhs[ni - 1] = -c[R - 1];
    int r3 = or_thomas(ni, ta, tb, tc, rhs, w);
    if (r1 || r2 || r3) rcode = OR_ZERO_PIVOT;
    /* interface equation for x[L] */
    A2[M] = AA(L);
    B2[M] = b[L] + c[L] * v[0];
    C2[M] = c[L] * w[0];
    D2[M] = d[L] - c[L] * g[0];
    I2[M] = L;
    M++;
    /* interface equation for x[R] */
    A2[M] = a[R] * v[ni - 1];
    B2[M] = b[R] + a[R] * w[ni - 1];
    C2[M] = CC(R);
    D2[M] = d[R] - a[R] * g[ni - 1];
    I2[M] = R;
    M++;
  }
  /* ---- Stage 2 ---- */
  if (or_thomas(M, A2, B2, C2, D2, Y)) rcode = OR_ZERO_PIVOT;
  for (int64_t j = 0; j < M; j++) x[I2[j]] = Y[j];
  /* ---- Stage 3 ---- */
  for (int64_t k = 0; k < m; k++) {
    int64_t L = k * s, R = (k + 1) * s - 1;
    if (R > n - 1) R = n - 1;
    int64_t nk = R - L + 1;
    if (nk < 3) continue;
    int64_t ni = nk - 2;
    for (int64_t i = 0; i < ni; i++) {
      ta[i] = a[L + 1 + i]; tb[i] = b[L + 1 + i]; tc[i] = c[L + 1 + i]; rhs[i] = d[L + 1 + i];
    }
    rhs[0] -= a[L + 1] * x[L];
    rhs[ni - 1] -= c[R - 1] * x[R];
    if (or_thomas(ni, ta, tb, tc, rhs, g)) rcode = OR_ZERO_PIVOT;
    for (int64_t i = 0; i < ni; i++) x[L + 1 + i] = g[i];
  }
#undef AA
#undef CC
  if (ra) memcpy(ra, A2, sizeof(double) * (size_t)M);
  if (rb) memcpy(rb, B2, sizeof(double) * (size_t)M);
  if (rc) memcpy(rc, C2, sizeof(double) * (size_t)M);
  if (rd) memcpy(rd, D2, sizeof(double) * (size_t)M);
  if (ridx) memcpy(ridx, I2, sizeof(int64_t) * (size_t)M);
  if (M_out) *M_out = M;
done:
  free(A2); free(B2); free(C2); free(D2); free(Y); free(I2);
  free(ta); free(tb); free(tc); free(rhs); free(g); free(v); free(w);
  return rcode;
}

/* ------------------------------------------------------------------------ */
/* Dense Gaussian elimination with partial pivoting in long double, on the   */
/* full n x n matrix (row-major).  Textbook algorithm; the brute-force check */
/* for small systems.  Pinned by: LAPACK (numpy.linalg.solve) on random      */
/* dense matrices and by the residual of its own answer.                     */
/* ------------------------------------------------------------------------ */
int or_dense_ld_full(int64_t n, const double* Ain, const double* rhs, double* x) {
  if (n < 1) return OR_BADARG;
  long double* A = (long double*)malloc(sizeof(long double) * (size_t)(n * n));
  long double* y = (long double*)malloc(sizeof(long double) * (size_t)n);
  if (!A || !y) { free(A); free(y); return OR_BADARG; }
  for (int64_t i = 0; i < n * n; i++) A[i] = (long double)Ain[i];
  for (int64_t i = 0; i < n; i++) y[i] = (long double)rhs[i];
  int rc = OR_OK;
  for (int64_t k = 0; k < n; k++) {
    int64_t p = k;
    long double best = fabsl(A[k * n + k]);
    for (int64_t i = k + 1; i < n; i++) {
      long double v = fabsl(A[i * n + k]);
      if (v > best) { best = v; p = i; }
    }
    if (best == 0.0L) { rc = OR_ZERO_PIVOT; break; }
    if (p != k) {
      for (int64_t j = 0; j < n; j++) { long double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
      long double t = y[k]; y[k] = y[p]; y[p] = t;
    }
    for (int64_t i = k + 1; i < n; i++) {
      long double f = A[i * n + k] / A[k * n + k];
      if (f == 0.0L) continue;
      for (int64_t j = k; j < n; j++) A[i * n + j] -= f * A[k * n + j];
      y[i] -= f * y[k];
    }
  }
  if (rc == OR_OK) {
    for (int64_t i = n - 1; i >= 0; i--) {
      long double acc = y[i];
      for (int64_t j = i + 1; j < n; j++) acc -= A[i * n + j] * y[j];
      y[i] = acc / A[i * n + i];
    }
    for (int64_t i = 0; i < n; i++) x[i] = (double)y[i];
  }
  free(A);
  free(y);
  return rc;
}

/* Tridiagonal system solved by dense long-double elimination (n <= a few hundred). */
int or_dense_ld(int64_t n, const double* a, const double* b, const double* c, const double* d, double* x) {
  if (n < 1) return OR_BADARG;
  double* A = (double*)calloc((size_t)(n * n), sizeof(double));
  if (!A) return OR_BADARG;
  for (int64_t i = 0; i < n; i++) {
    if (i > 0) A[i * n + i - 1] = a[i];
    A[i * n + i] = b[i];
    if (i < n - 1) A[i * n + i + 1] = c[i];
  }
  int rc = or_dense_ld_full(n, A, d, x);
  free(A);
  return rc;
}

/* r = d - A x, each row accumulated in long double then rounded. */
void or_residual(int64_t n, const double* a, const double* b, const double* c, const double* d, const double* x,
                 double* r) {
  for (int64_t i = 0; i < n; i++) {
    long double acc = (long double)d[i] - (long double)b[i] * (long double)x[i];
    if (i > 0) acc -= (long double)a[i] * (long double)x[i - 1];
    if (i < n - 1) acc -= (long double)c[i] * (long double)x[i + 1];
    r[i] = (double)acc;
  }
}

/* y = A x (binary64, the natural row order), used to manufacture d = A x*. */
void or_matvec(int64_t n, const double* a, const double* b, const double* c, const double* x, double* y) {
  for (int64_t i = 0; i < n; i++) {
    double acc = b[i] * x[i];
    if (i > 0) acc += a[i] * x[i - 1];
    if (i < n - 1) acc += c[i] * x[i + 1];
    y[i] = acc;
  }
}

/* ------------------------------------------------------------------------ */
/* Mixed-precision iterative refinement (the library's binary32 solve with  */
/* binary64 residual; not in the paper, which runs FP32 and FP64 separately */
/* in Sec. IV-B).  Textbook scheme:                                          */
/*   x0 = solve32(A, d);  repeat: r = d - A x (binary64),                   */
/*   delta = solve32(A, r), x += delta (binary64),                          */
/* until ||r||inf / ||d||inf <= tol or max_iter corrections.  hist[k] holds  */
/* ||r_k||inf / ||d||inf for k = 0..iters (r_k is the residual of x_k).      */
/* Pinned by: converging to the binary64 Thomas answer within 1e-12; the     */
/* residual history shrinking by about kappa*eps32 per step.                  */
/* ------------------------------------------------------------------------ */
int or_refine(int64_t n, const double* a, const double* b, const double* c, const double* d, double* x,
              int max_iter, double tol, double* hist, int* iters_out) {
  if (n < 1) return OR_BADARG;
  float* fa = (float*)malloc(sizeof(float) * (size_t)n);
  float* fb = (float*)malloc(sizeof(float) * (size_t)n);
  float* fc = (float*)malloc(sizeof(float) * (size_t)n);
  float* fr = (float*)malloc(sizeof(float) * (size_t)n);
  float* fx = (float*)malloc(sizeof(float) * (size_t)n);
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  if (!fa || !fb || !fc || !fr || !fx || !r) { free(fa); free(fb); free(fc); free(fr); free(fx); free(r); return OR_BADARG; }
  for (int64_t i = 0; i < n; i++) { fa[i] = (float)a[i]; fb[i] = (float)b[i]; fc[i] = (float)c[i]; fr[i] = (float)d[i]; }
  int rc = or_thomas_f32(n, fa, fb, fc, fr, fx);
  for (int64_t i = 0; i < n; i++) x[i] = (double)fx[i];
  double dn = 0.0;
  for (int64_t i = 0; i < n; i++) dn = fmax(dn, fabs(d[i]));
  if (dn == 0.0) dn = 1.0;
  int it = 0;
  for (;;) {
    for (int64_t i = 0; i < n; i++) {
      double acc = d[i] - b[i] * x[i];
      if (i > 0) acc -= a[i] * x[i - 1];
      if (i < n - 1) acc -= c[i] * x[i + 1];
      r[i] = acc;
    }
    double rn = 0.0;
    for (int64_t i = 0; i < n; i++) rn = fmax(rn, fabs(r[i]));
    if (hist) hist[it] = rn / dn;
    if (rn / dn <= tol || it >= max_iter) break;
    for (int64_t i = 0; i < n; i++) fr[i] = (float)r[i];
    if (or_thomas_f32(n, fa, fb, fc, fr, fx)) rc = OR_ZERO_PIVOT;
    for (int64_t i = 0; i < n; i++) x[i] += (double)fx[i];
    it++;
  }
  if (iters_out) *iters_out = it;
  free(fa); free(fb); free(fc); free(fr); free(fx); free(r);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Adjoint of the solve (not in the paper).  For x = A^{-1} d and a loss L   */
/* with gradient g = dL/dx:                                                  */
/*   lambda = A^{-T} g,  dL/dd = lambda,  dL/dA = -lambda x^T,               */
/* restricted to the three diagonals:                                        */
/*   grad_a[i] = -lambda[i] x[i-1] (0 at i=0), grad_b[i] = -lambda[i] x[i],  */
/*   grad_c[i] = -lambda[i] x[i+1] (0 at i=n-1).                             */
/* A^T is tridiagonal with sub-diagonal c[i-1], diagonal b[i], super-        */
/* diagonal a[i+1]; it is solved by Thomas.                                  */
/* Pinned by: <w,x> = <lambda,d>; central finite differences; dense numpy.   */
/* ------------------------------------------------------------------------ */
int or_adjoint(int64_t n, const double* a, const double* b, const double* c, const double* x, const double* g,
               double* lam, double* ga, double* gb, double* gc, double* gd) {
  if (n < 1) return OR_BADARG;
  double* ta = (double*)malloc(sizeof(double) * (size_t)n);
  double* tc = (double*)malloc(sizeof(double) * (size_t)n);
  if (!ta || !tc) { free(ta); free(tc); return OR_BADARG; }
  for (int64_t i = 0; i < n; i++) {
    ta[i] = (i > 0) ? c[i - 1] : 0.0;
    tc[i] = (i < n - 1) ? a[i + 1] : 0.0;
  }
  int rc = or_thomas(n, ta, b, tc, g, lam);
  for (int64_t i = 0; i < n; i++) {
    ga[i] = (i > 0) ? -lam[i] * x[i - 1] : 0.0;
    gb[i] = -lam[i] * x[i];
    gc[i] = (i < n - 1) ? -lam[i] * x[i + 1] : 0.0;
    gd[i] = lam[i];
  }
  free(ta);
  free(tc);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Closed form for the constant-coefficient matrix tridiag(-r, 1+2r, -r) of  */
/* the implicit heat step: eigenvalues 1 + 4 r sin^2(j pi / (2(n+1))),       */
/* eigenvectors sin(i j pi / (n+1)) (a discrete sine transform), so         */
/*   x = (2/(n+1)) sum_j [ (v_j . d) / lambda_j ] v_j.                        */
/* O(n^2), long-double accumulation.  Independent of Thomas: pins it.        */
/* ------------------------------------------------------------------------ */
void or_dst_const(int64_t n, double r, const double* d, double* x) {
  long double pi = 3.141592653589793238462643383279502884L;
  int64_t P = 2 * (n + 1); /* sin(k pi/(n+1)) has period 2(n+1) in k */
  long double* S = (long double*)malloc(sizeof(long double) * (size_t)P);
  long double* coef = (long double*)malloc(sizeof(long double) * (size_t)n);
  for (int64_t k = 0; k < P; k++) S[k] = sinl((long double)k * pi / (long double)(n + 1));
  for (int64_t j = 1; j <= n; j++) {
    long double acc = 0.0L;
    for (int64_t i = 1; i <= n; i++) acc += S[(i * j) % P] * (long double)d[i - 1];
    long double sj = sinl((long double)j * pi / (2.0L * (long double)(n + 1)));
    long double lam = 1.0L + 4.0L * (long double)r * sj * sj;
    coef[j - 1] = acc / lam;
  }
  for (int64_t i = 1; i <= n; i++) {
    long double acc = 0.0L;
    for (int64_t j = 1; j <= n; j++) acc += coef[j - 1] * S[(i * j) % P];
    x[i - 1] = (double)(acc * 2.0L / (long double)(n + 1));
  }
  free(S);
  free(coef);
}
