/*
 * Plain CPU oracle for TSQR / CAQR: unblocked FP64 Householder QR.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this file; only the test suite, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or constant with the CUDA
 * library.
 *
 * What it computes.  The paper's TSQR (Section 2.1, Eqs. TSQR_binarytree_1..4)
 * returns the R factor of A and a tree-structured Q whose product with R is A.
 * By uniqueness of the QR factorisation up to the signs of diag(R) (Section
 * 2.1, the paragraph after Eq. TSQR_binarytree_4) every reduction tree yields
 * the same factorisation; the "trivial tree" of the same section is
 * conventional Householder QR.  So the oracle is that plain definition: one
 * Householder reflector per column, applied column by column, no blocking.
 *
 * Conventions (all matrices column-major, element (i,j) at a[i + j*lda]):
 *   - reflector H_j = I - tau_j v_j v_j^T with the topmost nonzero entry of
 *     v_j equal to one (Section 4, the list of Q representations in the
 *     lower-bound argument); v_j(j) = 1 is implicit, v_j(j+1:m) is stored
 *     below the diagonal of column j;
 *   - beta_j = -sign(alpha_j) * ||x_j|| so that alpha_j - beta_j never cancels;
 *     a column whose tail below the diagonal is exactly zero gets tau_j = 0
 *     (H_j = I) and keeps alpha_j as its diagonal entry;
 *   - 2-norms use a scaled sum of squares (largest magnitude factored out)
 *     so that entries near 1e+-150 neither overflow nor underflow;
 *   - sign normalisation: d_j = sign(R_jj) with sign(0) = +1, R <- D R, and
 *     the explicit Q carries D: A = (Q D)(D R).
 *
 * Compiled with -O2 -ffp-contract=off so that every product and sum is a
 * separately rounded IEEE operation in the order written here.
 *
 * Parity pins: closed forms for 2x2 and 3x2 inputs, exact rational QR of tiny
 * integer matrices, R^T R = A^T A (Cholesky of the Gram matrix, Section 4 lower
 * bound argument), LAPACK QR run as a library, orthogonality and residual
 * bounds, and row-permutation / tree-shape invariance.  The T factor of the
 * compact WY form is pinned against the explicit product of reflectors; the
 * QR adjoint is pinned by central finite differences; least squares by the
 * closed-form straight-line fit, the normal equations A^T (A x - b) = 0, exact
 * recovery of consistent systems and LAPACK's least-squares solver run as a
 * library.  Intermediate tree data
 * (Y, tau, T of a given tree) are not part of any pin: they depend on the tree.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* Scaled 2-norm of x[0..len) with stride 1. */
static double scaled_nrm2(const double* x, int64_t len) {
  double scale = 0.0;
  for (int64_t i = 0; i < len; ++i) {
    double a = fabs(x[i]);
    if (a > scale) scale = a;
  }
  if (scale == 0.0) return 0.0;
  double ssq = 0.0;
  for (int64_t i = 0; i < len; ++i) {
    double t = x[i] / scale;
    ssq += t * t;
  }
  return scale * sqrt(ssq);
}

/* sqrt(a^2 + b^2) without overflow, for a >= 0, b >= 0. */
static double scaled_hypot(double a, double b) {
  double t = a > b ? a : b;
  if (t == 0.0) return 0.0;
  double x = a / t, y = b / t;
  return t * sqrt(x * x + y * y);
}

/*
 * Householder QR of the m x n matrix A (m >= n >= 0), in place.
 * On exit the upper triangle holds R (before sign normalisation), the strict
 * lower trapezoid holds v_j(j+1:m), and tau[0..n) the reflector scalars.
 * Trailing columns are updated one at a time: w = v^T a_c, a_c -= tau w v.
 * With OpenMP the loop over trailing columns c runs in parallel; each column's
 * arithmetic and its order are unchanged.
 */
void oracle_geqr2(int64_t m, int64_t n, double* A, int64_t lda, double* tau) {
  for (int64_t j = 0; j < n; ++j) {
    double* x = &A[IDX(j, j, lda)];
    int64_t len = m - j;
    double alpha = x[0];
    double xnorm = scaled_nrm2(x + 1, len - 1);
    if (xnorm == 0.0) {
      tau[j] = 0.0;
      continue;
    }
    double nrm = scaled_hypot(fabs(alpha), xnorm);
    double beta = alpha >= 0.0 ? -nrm : nrm;
    double t = (beta - alpha) / beta;
    double denom = alpha - beta;
    for (int64_t i = 1; i < len; ++i) x[i] = x[i] / denom;
    x[0] = beta;
    tau[j] = t;
#pragma omp parallel for schedule(static) if ((n - j) * len > 65536)
    for (int64_t c = j + 1; c < n; ++c) {
      double* a = &A[IDX(j, c, lda)];
      double w = a[0];
      for (int64_t i = 1; i < len; ++i) w += x[i] * a[i];
      double tw = t * w;
      a[0] -= tw;
      for (int64_t i = 1; i < len; ++i) a[i] -= tw * x[i];
    }
  }
}

/*
 * Sign normalisation: d_j = sign(R_jj), sign(0) = +1.  Writes d[0..n) and
 * R (n x n, ldr) = D * triu(A(0:n, 0:n)); entries below the diagonal of R are
 * set to zero.
 */
void oracle_extract_r(int64_t n, const double* A, int64_t lda, double* d, double* R, int64_t ldr) {
  for (int64_t j = 0; j < n; ++j) d[j] = A[IDX(j, j, lda)] < 0.0 ? -1.0 : 1.0;
  for (int64_t c = 0; c < n; ++c)
    for (int64_t i = 0; i < n; ++i) R[IDX(i, c, ldr)] = i <= c ? d[i] * A[IDX(i, c, lda)] : 0.0;
}

/* Apply H_j = I - tau v v^T (v from column j of Y, v(j) = 1) to rows j..m-1 of C. */
static void apply_reflector(int64_t m, int64_t j, const double* Y, int64_t ldy, double t, int64_t k,
                            double* C, int64_t ldc) {
  if (t == 0.0) return;
  const double* v = &Y[IDX(j, j, ldy)];
  int64_t len = m - j;
#pragma omp parallel for schedule(static) if (k * len > 65536)
  for (int64_t c = 0; c < k; ++c) {
    double* a = &C[IDX(j, c, ldc)];
    double w = a[0];
    for (int64_t i = 1; i < len; ++i) w += v[i] * a[i];
    double tw = t * w;
    a[0] -= tw;
    for (int64_t i = 1; i < len; ++i) a[i] -= tw * v[i];
  }
}

/*
 * C (m x k) <- Q^T C with the square Q = H_0 H_1 ... H_{n-1} diag(d, I):
 * first H_0, then H_1, ..., then rows 0..n-1 scaled by d.
 */
void oracle_apply_qt(int64_t m, int64_t n, const double* Y, int64_t ldy, const double* tau, const double* d,
                     int64_t k, double* C, int64_t ldc) {
  for (int64_t j = 0; j < n; ++j) apply_reflector(m, j, Y, ldy, tau[j], k, C, ldc);
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < n; ++i) C[IDX(i, c, ldc)] *= d[i];
}

/* C (m x k) <- Q C, the reverse of oracle_apply_qt. */
void oracle_apply_q(int64_t m, int64_t n, const double* Y, int64_t ldy, const double* tau, const double* d,
                    int64_t k, double* C, int64_t ldc) {
  for (int64_t c = 0; c < k; ++c)
    for (int64_t i = 0; i < n; ++i) C[IDX(i, c, ldc)] *= d[i];
  for (int64_t j = n - 1; j >= 0; --j) apply_reflector(m, j, Y, ldy, tau[j], k, C, ldc);
}

/* Thin Q (m x n) = H_0 ... H_{n-1} [I_n; 0] diag(d). */
void oracle_form_q(int64_t m, int64_t n, const double* Y, int64_t ldy, const double* tau, const double* d,
                   double* Q, int64_t ldq) {
  for (int64_t c = 0; c < n; ++c)
    for (int64_t i = 0; i < m; ++i) Q[IDX(i, c, ldq)] = (i == c) ? d[c] : 0.0;
  for (int64_t j = n - 1; j >= 0; --j) apply_reflector(m, j, Y, ldy, tau[j], n, Q, ldq);
}

/*
 * Compact WY factor (Schreiber and Van Loan, cited in Section 2.1): the
 * upper-triangular T (n x n) with H_0 H_1 ... H_{n-1} = I - Y T Y^T, built by
 * the forward recurrence T_jj = tau_j, T(0:j, j) = -tau_j T(0:j,0:j) (Y(:,0:j)^T y_j).
 */
void oracle_larft(int64_t m, int64_t n, const double* Y, int64_t ldy, const double* tau, double* T, int64_t ldt) {
  double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int64_t j = 0; j < n; ++j) {
    for (int64_t i = 0; i < n; ++i) T[IDX(i, j, ldt)] = 0.0;
    /* z(p) = y_p^T y_j for p < j; y_p has unit entry p and y_j is zero above row j. */
    for (int64_t p = 0; p < j; ++p) {
      double s = Y[IDX(j, p, ldy)]; /* y_p(j) * y_j(j), y_j(j) = 1 */
      for (int64_t i = j + 1; i < m; ++i) s += Y[IDX(i, p, ldy)] * Y[IDX(i, j, ldy)];
      z[p] = s;
    }
    for (int64_t p = 0; p < j; ++p) {
      double s = 0.0;
      for (int64_t q = p; q < j; ++q) s += T[IDX(p, q, ldt)] * z[q];
      T[IDX(p, j, ldt)] = -tau[j] * s;
    }
    T[IDX(j, j, ldt)] = tau[j];
  }
  free(z);
}

/*
 * Full QR: copies A (m x n) into Y, factors it, normalises signs, writes
 * R (n x n) with diag(R) >= 0 and, when Q is non-null, the thin Q (m x n).
 * tau and d (length n) are outputs too.
 */
void oracle_qr(int64_t m, int64_t n, const double* A, int64_t lda, double* Y, int64_t ldy, double* tau,
               double* d, double* R, int64_t ldr, double* Q, int64_t ldq) {
  for (int64_t c = 0; c < n; ++c) memcpy(&Y[IDX(0, c, ldy)], &A[IDX(0, c, lda)], sizeof(double) * (size_t)m);
  oracle_geqr2(m, n, Y, ldy, tau);
  oracle_extract_r(n, Y, ldy, d, R, ldr);
  if (Q) oracle_form_q(m, n, Y, ldy, tau, d, Q, ldq);
}

/*
 * Adjoint of the thin QR with diag(R) > 0 (the training-system add-on; the
 * paper has no gradient):
 *   M  = R dR^T - dQ^T Q                      (n x n)
 *   B  = dQ + Q copyltu(M),  copyltu(M) = tril(M) + tril(M,-1)^T
 *   dA = B R^{-T}   (row i of dA solves R x = B(i,:)^T by back substitution)
 * Q, dQ, dA are m x n (ld = m), R and dR are n x n (ld = n).  dA may not alias.
 */
void oracle_qr_backward(int64_t m, int64_t n, const double* Q, const double* R, const double* dQ, const double* dR,
                        double* dA) {
  double* M = (double*)malloc(sizeof(double) * (size_t)(n * n > 0 ? n * n : 1));
  double* S = (double*)malloc(sizeof(double) * (size_t)(n * n > 0 ? n * n : 1));
#pragma omp parallel for schedule(dynamic) if (m * n * n > 1000000)
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      double a = 0.0; /* (R dR^T)_ij = sum_k R_ik dR_jk */
      for (int64_t k = 0; k < n; ++k) a += R[IDX(i, k, n)] * dR[IDX(j, k, n)];
      double b = 0.0; /* (dQ^T Q)_ij = sum_r dQ_ri Q_rj */
      for (int64_t r = 0; r < m; ++r) b += dQ[IDX(r, i, m)] * Q[IDX(r, j, m)];
      M[IDX(i, j, n)] = a - b;
    }
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) S[IDX(i, j, n)] = i >= j ? M[IDX(i, j, n)] : M[IDX(j, i, n)];
#pragma omp parallel for schedule(static) if (m * n * n > 1000000)
  for (int64_t r = 0; r < m; ++r) {
    double b[512];
    double* bb = n <= 512 ? b : (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t j = 0; j < n; ++j) {
      double s = dQ[IDX(r, j, m)];
      for (int64_t k = 0; k < n; ++k) s += Q[IDX(r, k, m)] * S[IDX(k, j, n)];
      bb[j] = s;
    }
    /* x R^T = b  <=>  R x^T = b^T: back substitution from the last column. */
    for (int64_t j = n - 1; j >= 0; --j) {
      double s = bb[j];
      for (int64_t k = j + 1; k < n; ++k) s -= R[IDX(j, k, n)] * dA[IDX(r, k, m)];
      dA[IDX(r, j, m)] = s / R[IDX(j, j, n)];
    }
    if (bb != b) free(bb);
  }
  free(M);
  free(S);
}

/*
 * Least squares min ||A x_c - b_c||_2 for the k columns of B (Section 1: the
 * tall-skinny least-squares problem that TSQR serves), the textbook way:
 * Householder QR of a copy of A (oracle_geqr2), Q^T B by H_0, ..., H_{n-1} in
 * order (no sign normalisation: R and Q^T B then carry the same signs), back
 * substitution with R = triu(A(0:n, 0:n)) for X (n x k, ldx), and the
 * residual norms rnorm[c] = ||(Q^T b_c)(n:m)||_2 (scaled norm).  A zero
 * diagonal entry of R (rank-deficient A) gives inf or NaN in X.
 */
void oracle_lstsq(int64_t m, int64_t n, const double* A, int64_t lda, int64_t k, const double* B, int64_t ldb,
                  double* X, int64_t ldx, double* rnorm) {
  double* Y = (double*)malloc(sizeof(double) * (size_t)(m * n > 0 ? m * n : 1));
  double* tau = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* C = (double*)malloc(sizeof(double) * (size_t)(m * k > 0 ? m * k : 1));
  for (int64_t c = 0; c < n; ++c) memcpy(&Y[IDX(0, c, m)], &A[IDX(0, c, lda)], sizeof(double) * (size_t)m);
  for (int64_t c = 0; c < k; ++c) memcpy(&C[IDX(0, c, m)], &B[IDX(0, c, ldb)], sizeof(double) * (size_t)m);
  oracle_geqr2(m, n, Y, m, tau);
  for (int64_t j = 0; j < n; ++j) apply_reflector(m, j, Y, m, tau[j], k, C, m);
  for (int64_t c = 0; c < k; ++c) {
    double* x = &X[IDX(0, c, ldx)];
    const double* y = &C[IDX(0, c, m)];
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int64_t j = i + 1; j < n; ++j) s -= Y[IDX(i, j, m)] * x[j];
      x[i] = s / Y[IDX(i, i, m)];
    }
    if (rnorm) rnorm[c] = scaled_nrm2(y + n, m - n);
  }
  free(Y);
  free(tau);
  free(C);
}

/* Number of OpenMP threads the oracle would use (1 without OpenMP). */
int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Sets the number of OpenMP threads for later calls (no effect without
 * OpenMP); for timing the oracle on one core beside all of them. */
void oracle_set_num_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
}
