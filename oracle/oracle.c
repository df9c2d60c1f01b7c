/*
 * oracle.c -- plain, slow, FP64 CPU reference for the Hermitian-definite
 * generalized eigenproblem  A x = lambda B x  (A Hermitian, B Hermitian
 * positive definite), as set out in the paper's Algorithm 1 (Cholesky,
 * reduction to standard form, standard eigensolver, back-substitution) and
 * Algorithm 2 (tridiagonal reduction, tridiagonal eigensolver, eigenvector
 * back-transformation) with a single stage (Section 4.1).
 *
 * THIS IS TEST INFRASTRUCTURE.  It exists only to check the CUDA path; only
 * the test suite, the smoke check and the benchmark's CPU-baseline leg load
 * it.  It shares no code, header, table or helper with the CUDA library.
 *
 * Conventions (the paper is silent on them; these are the LAPACK ones):
 *   - complex128 (C99 double complex), column-major, leading dimension ld;
 *   - Hermitian inputs are read from their LOWER triangle only;
 *   - Householder reflector H = I - tau v v^H with v(0) = 1, chosen so that
 *     H^H (alpha, x)^T = (beta, 0)^T with beta REAL; this makes the
 *     tridiagonal matrix real symmetric directly;
 *   - eigenvalues ascending, ties broken by original index (stable sort).
 *
 * The tridiagonal eigensolver here is the implicit symmetric QR iteration
 * with a Wilkinson shift, deliberately a different algorithm from the divide
 * and conquer method the paper uses (Section 4.3) so that agreement between
 * the two is a real test.
 *
 * Loops are written straight from the definitions; the only concession to
 * speed is "omp parallel for" over independent columns.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;
#define AT(M, i, j, ld) (M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)]

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Algorithm 1, step 1: B = L L^H, L lower triangular with real positive
 * diagonal, overwriting the lower triangle of B (right-looking, unblocked).
 * Returns 0, or k (1-based) if the leading minor of order k is not positive
 * definite.  The strictly upper triangle is left untouched. */
int orc_potrf(int n, zc* B, int ldb) {
  for (int k = 0; k < n; ++k) {
    double d = creal(AT(B, k, k, ldb));
    if (!(d > 0.0) || !isfinite(d)) return k + 1;
    d = sqrt(d);
    AT(B, k, k, ldb) = d;
    for (int i = k + 1; i < n; ++i) AT(B, i, k, ldb) /= d;
#pragma omp parallel for schedule(dynamic, 8)
    for (int j = k + 1; j < n; ++j) {
      zc ljk = conj(AT(B, j, k, ldb));
      for (int i = j; i < n; ++i) AT(B, i, j, ldb) -= AT(B, i, k, ldb) * ljk;
      AT(B, j, j, ldb) = creal(AT(B, j, j, ldb));
    }
  }
  return 0;
}

/* Forward substitution L Y = R for all n columns of R (in place, n x n). */
static void lower_solve_inplace(int n, const zc* L, int ldl, zc* R, int ldr) {
#pragma omp parallel for schedule(static)
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) {
      zc s = AT(R, i, c, ldr);
      for (int j = 0; j < i; ++j) s -= AT(L, i, j, ldl) * AT(R, j, c, ldr);
      AT(R, i, c, ldr) = s / AT(L, i, i, ldl);
    }
  }
}

/* Algorithm 1, step 2: A' = L^{-1} A L^{-H}.  A is read from its lower
 * triangle; on return A holds the FULL Hermitian A' (both triangles, real
 * diagonal).  Two forward substitutions:
 *   W = L^{-1} A,   A'^H = L^{-1} W^H,  then A' := (A' + A'^H)/2. */
void orc_hegst(int n, zc* A, int lda, const zc* L, int ldl) {
  zc* W = (zc*)malloc(sizeof(zc) * (size_t)n * n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i)
      AT(W, i, j, n) = (i >= j) ? AT(A, i, j, lda) : conj(AT(A, j, i, lda));
  for (int i = 0; i < n; ++i) AT(W, i, i, n) = creal(AT(W, i, i, n));
  lower_solve_inplace(n, L, ldl, W, n);           /* W = L^{-1} A          */
  zc* Y = (zc*)malloc(sizeof(zc) * (size_t)n * n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) AT(Y, i, j, n) = conj(AT(W, j, i, n));
  lower_solve_inplace(n, L, ldl, Y, n);           /* Y = L^{-1} W^H = A'^H */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i)
      AT(A, i, j, lda) = 0.5 * (conj(AT(Y, j, i, n)) + AT(Y, i, j, n));
  for (int i = 0; i < n; ++i) AT(A, i, i, lda) = creal(AT(A, i, i, lda));
  free(W);
  free(Y);
}

/* Householder reflector for the vector (alpha, x) of length len >= 1:
 * returns tau and beta (real) and overwrites x with v(1:len-1) (v(0) = 1),
 * so that H^H (alpha, x) = (beta, 0) with H = I - tau v v^H.
 * tau = 0 (H = I) when x = 0 and alpha is already real. */
static zc make_reflector(int len, zc alpha, zc* x, double* beta_out) {
  double xnorm2 = 0.0;
  for (int i = 0; i < len - 1; ++i) xnorm2 += creal(x[i] * conj(x[i]));
  if (xnorm2 == 0.0 && cimag(alpha) == 0.0) {
    *beta_out = creal(alpha);
    return 0.0;
  }
  double nrm = sqrt(creal(alpha) * creal(alpha) + cimag(alpha) * cimag(alpha) + xnorm2);
  double beta = (creal(alpha) >= 0.0) ? -nrm : nrm;
  zc tau = (beta - alpha) / beta;
  zc scal = 1.0 / (alpha - beta);
  for (int i = 0; i < len - 1; ++i) x[i] *= scal;
  *beta_out = beta;
  return tau;
}

/* Algorithm 2, step 1 with one stage (Section 4.1): Householder reduction of
 * the full Hermitian A (n x n, both triangles valid) to real symmetric
 * tridiagonal T = Q^H A Q, Q = H_0 H_1 ... H_{n-2}.  For column k the
 * reflector H_k acts on rows k+1..n-1; its vector is stored in V (column k,
 * rows k+1..n-1, V(k+1,k) = 1) and its scalar in tau[k].  On return d (n)
 * and e (n-1) hold the diagonal and subdiagonal of T.  A is destroyed. */
void orc_hetrd(int n, zc* A, int lda, double* d, double* e, zc* V, int ldv, zc* tau) {
  zc* p = (zc*)malloc(sizeof(zc) * (size_t)(n > 0 ? n : 1));
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) AT(V, i, j, ldv) = 0.0;
  for (int k = 0; k + 1 < n; ++k) {
    int len = n - k - 1; /* rows k+1..n-1 */
    zc* x = &AT(A, k + 1, k, lda);
    double beta;
    zc t = make_reflector(len, x[0], x + 1, &beta);
    tau[k] = t;
    AT(V, k + 1, k, ldv) = 1.0;
    for (int i = 1; i < len; ++i) AT(V, k + 1 + i, k, ldv) = x[i];
    e[k] = beta;
    /* A22 <- H^H A22 H = A22 - v w^H - w v^H, with
     * p = tau A22 v, w = p - (tau/2)(p^H v) v. */
    const zc* v = &AT(V, k + 1, k, ldv);
    int o = k + 1;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < len; ++i) {
      zc s = 0.0;
      for (int j = 0; j < len; ++j) s += conj(AT(A, o + j, o + i, lda)) * v[j];
      p[i] = t * s;
    }
    zc pv = 0.0;
    for (int i = 0; i < len; ++i) pv += conj(p[i]) * v[i];
    zc half = 0.5 * t * pv;
    for (int i = 0; i < len; ++i) p[i] -= half * v[i]; /* p := w */
#pragma omp parallel for schedule(static)
    for (int j = 0; j < len; ++j)
      for (int i = 0; i < len; ++i)
        AT(A, o + i, o + j, lda) -= v[i] * conj(p[j]) + p[i] * conj(v[j]);
    for (int i = 0; i < len; ++i) AT(A, o + i, o + i, lda) = creal(AT(A, o + i, o + i, lda));
  }
  for (int k = 0; k < n; ++k) d[k] = creal(AT(A, k, k, lda));
  if (n >= 1) tau[n - 1] = 0.0;
  free(p);
}

/* Algorithm 2, step 2 (oracle variant): implicit symmetric QR iteration with
 * Wilkinson shift on the real symmetric tridiagonal (d, e), e[i] coupling rows
 * i and i+1.  Each step applies plane rotations G_k (rows/cols k, k+1) as the
 * similarity T <- G_k^T T G_k, chasing the bulge element down the block; the
 * first rotation is fixed by the shift (implicit Q theorem).  Z (n x n) holds
 * an orthogonal matrix on entry (normally I); the rotations are accumulated
 * as Z <- Z G_k so that on return T = Z diag(d) Z^T.  Off-diagonals with
 * |e_i| <= eps (|d_i| + |d_{i+1}|) are set to zero (deflation).
 * Eigenvalues are NOT sorted here.  Returns 0, or 1 if the iteration count
 * exceeded 40 n. */
int orc_steqr(int n, double* d, const double* e_in, double* Z, int ldz) {
  if (n <= 1) return 0;
  double* e = (double*)malloc(sizeof(double) * (size_t)n);
  for (int i = 0; i + 1 < n; ++i) e[i] = e_in[i];
  const double eps = 2.220446049250313e-16;
  long iter = 0, maxit = 40L * n;
  int hi = n - 1;
  while (hi > 0) {
    for (int i = 0; i < hi; ++i)
      if (fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1]))) e[i] = 0.0;
    if (e[hi - 1] == 0.0) { --hi; continue; }
    int lo = hi - 1;
    while (lo > 0 && e[lo - 1] != 0.0) --lo;
    if (++iter > maxit) { free(e); return 1; }
    /* Wilkinson shift: eigenvalue of the trailing 2x2 of the block closer
     * to d[hi]. */
    double dd = 0.5 * (d[hi - 1] - d[hi]);
    double bb = e[hi - 1];
    double den = dd + (dd >= 0.0 ? hypot(dd, bb) : -hypot(dd, bb));
    double mu = d[hi] - bb * bb / den;
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      /* G^T (x, z)^T = (r, 0)^T with G = [[c, -s], [s, c]] on (k, k+1). */
      double r = hypot(x, z);
      double c = 1.0, s = 0.0;
      if (r != 0.0) { c = x / r; s = z / r; }
      if (k > lo) e[k - 1] = r; /* bulge at (k+1, k-1) annihilated */
      double a = d[k], b = e[k], cc = d[k + 1];
      d[k] = c * c * a + 2.0 * c * s * b + s * s * cc;
      d[k + 1] = s * s * a - 2.0 * c * s * b + c * c * cc;
      e[k] = c * s * (cc - a) + (c * c - s * s) * b;
      if (k + 1 < hi) {
        z = s * e[k + 1];     /* new bulge at (k+2, k) */
        e[k + 1] = c * e[k + 1];
        x = e[k];
      }
      for (int row = 0; row < n; ++row) {
        double zk = AT(Z, row, k, ldz), zk1 = AT(Z, row, k + 1, ldz);
        AT(Z, row, k, ldz) = c * zk + s * zk1;
        AT(Z, row, k + 1, ldz) = -s * zk + c * zk1;
      }
    }
  }
  free(e);
  return 0;
}

/* Sort eigenvalues ascending (stable: equal values keep index order) and
 * permute the columns of Z to match.  Insertion sort on an index array. */
void orc_sort_eig(int n, double* w, double* Z, int ldz) {
  int* idx = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 1; i < n; ++i) {
    int t = idx[i];
    int j = i - 1;
    while (j >= 0 && w[idx[j]] > w[t]) { idx[j + 1] = idx[j]; --j; }
    idx[j + 1] = t;
  }
  double* w2 = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* Z2 = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(n > 0 ? n : 1));
  for (int c = 0; c < n; ++c) {
    w2[c] = w[idx[c]];
    for (int r = 0; r < n; ++r) AT(Z2, r, c, n) = AT(Z, r, idx[c], ldz);
  }
  for (int c = 0; c < n; ++c) {
    w[c] = w2[c];
    for (int r = 0; r < n; ++r) AT(Z, r, c, ldz) = AT(Z2, r, c, n);
  }
  free(idx); free(w2); free(Z2);
}

/* Algorithm 2, step 3: Y := Q Y = H_0 H_1 ... H_{n-2} Y for the m columns of
 * Y (n x m), applying the last reflector first. */
void orc_unmtr(int n, int m, const zc* V, int ldv, const zc* tau, zc* Y, int ldy) {
  for (int k = n - 2; k >= 0; --k) {
    zc t = tau[k];
    if (t == 0.0) continue;
    int o = k + 1, len = n - k - 1;
    const zc* v = &AT(V, o, k, ldv);
#pragma omp parallel for schedule(static)
    for (int c = 0; c < m; ++c) {
      zc s = 0.0;
      for (int i = 0; i < len; ++i) s += conj(v[i]) * AT(Y, o + i, c, ldy);
      s *= t;
      for (int i = 0; i < len; ++i) AT(Y, o + i, c, ldy) -= v[i] * s;
    }
  }
}

/* Algorithm 1, step 4: X = L^{-H} Y (back substitution with L^H, upper),
 * in place on the m columns of X (n x m). */
void orc_trsm_lh(int n, int m, const zc* L, int ldl, zc* X, int ldx) {
#pragma omp parallel for schedule(static)
  for (int c = 0; c < m; ++c) {
    for (int i = n - 1; i >= 0; --i) {
      zc s = AT(X, i, c, ldx);
      for (int j = i + 1; j < n; ++j) s -= conj(AT(L, j, i, ldl)) * AT(X, j, c, ldx);
      AT(X, i, c, ldx) = s / conj(AT(L, i, i, ldl));
    }
  }
}

/* Full driver (Algorithm 1 around Algorithm 2, one-stage):
 * eigenpairs il..iu (1-based, inclusive, ascending) of A x = lambda B x.
 * A (lower triangle read) and B (lower triangle read; overwritten by L) are
 * n x n; w receives m = iu-il+1 eigenvalues, X (n x m) the B-orthonormal
 * eigenvectors.  Returns 0; k>0 if B is not positive definite (minor k);
 * -1 bad arguments; n+1 if the tridiagonal QR iteration did not converge. */
int orc_hegv(int n, zc* A, int lda, zc* B, int ldb, int il, int iu, double* w, zc* X, int ldx) {
  if (n < 0 || il < 1 || iu < il - 1 || iu > n) return -1;
  if (n == 0) return 0;
  int info = orc_potrf(n, B, ldb);
  if (info) return info;
  orc_hegst(n, A, lda, B, ldb);
  double* d = (double*)malloc(sizeof(double) * (size_t)n);
  double* e = (double*)malloc(sizeof(double) * (size_t)n);
  zc* V = (zc*)malloc(sizeof(zc) * (size_t)n * n);
  zc* tau = (zc*)malloc(sizeof(zc) * (size_t)n);
  orc_hetrd(n, A, lda, d, e, V, n, tau);
  double* Z = (double*)calloc((size_t)n * n, sizeof(double));
  for (int i = 0; i < n; ++i) AT(Z, i, i, n) = 1.0;
  info = orc_steqr(n, d, e, Z, n);
  if (info) {
    free(d); free(e); free(V); free(tau); free(Z);
    return n + info;
  }
  orc_sort_eig(n, d, Z, n);
  int m = iu - il + 1;
  for (int c = 0; c < m; ++c) {
    w[c] = d[il - 1 + c];
    for (int r = 0; r < n; ++r) AT(X, r, c, ldx) = AT(Z, r, il - 1 + c, n);
  }
  orc_unmtr(n, m, V, n, tau, X, ldx);
  orc_trsm_lh(n, m, B, ldb, X, ldx);
  free(d); free(e); free(V); free(tau); free(Z);
  return 0;
}
