/*
 * msts_oracle.c -- plain, slow, obviously-correct CPU reference for the
 * blocked multi-shift triangular solve of Moon & Poulson (arXiv:1607.01477).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA library is
 * checked against.  Only the tests, the package smoke check and the bench's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA library, and the library never calls it.
 *
 * Arithmetic: IEEE binary64 throughout, complex numbers as (re, im) pairs,
 * compiled with -ffp-contract=off so that every a*b+c rounds twice.
 * Matrices are column-major with a leading dimension (element (r,c) of A is
 * A[r + c*lda]).  Only the upper triangle of U / T is read.
 * OpenMP is used only across independent shifts / grid points.
 *
 * Readings of the paper fixed here (the CUDA library takes the same ones):
 *   - Omega (the overflow threshold of Alg. 4 and Alg. 5) is 2^960.
 *   - Magnitudes in all growth bounds are complex moduli |z| (hypot).
 *   - A pivot U(i,i)-lambda that is exactly zero is replaced by the real
 *     number delta = max(eps*||U||_inf, DBL_MIN), eps = 2^-52 (Sec. 3).
 *   - Every scale factor t is a power of two 2^-k with k the smallest k >= 1
 *     for which the rescaled quantity is below Omega; scale factors are kept
 *     as integer exponents e (s = 2^-e) so that they cannot underflow, and
 *     t * x is applied as an exponent shift of x (exact unless x * 2^-k
 *     itself underflows), never as a multiplication by a rounded t.
 *   - The ratio |b(i)|/|U(i,i)| is evaluated through a mantissa/exponent
 *     split so that it can be compared with Omega without overflowing.
 *   - After the diagonal step, M is the modulus of the computed x(i).
 *   - Blocks are cut from the bottom; when m is not a multiple of n_b the
 *     ragged block of m mod n_b rows is the top one.
 */
#include <math.h>
#include <float.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double re, im; } oz;

/* Reading: Omega = 2^960 leaves 2^63 of headroom below DBL_MAX. */
#define OR_OMEGA_EXP 960

static inline oz oz_make(double re, double im) { oz z; z.re = re; z.im = im; return z; }
static inline oz oz_add(oz a, oz b) { return oz_make(a.re + b.re, a.im + b.im); }
static inline oz oz_sub(oz a, oz b) { return oz_make(a.re - b.re, a.im - b.im); }
static inline oz oz_mul(oz a, oz b) {
  return oz_make(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
static inline oz oz_conj(oz a) { return oz_make(a.re, -a.im); }
static inline oz oz_scale(oz a, double s) { return oz_make(a.re * s, a.im * s); }
static inline double oz_abs(oz a) { return hypot(a.re, a.im); }
static inline int oz_is_zero(oz a) { return a.re == 0.0 && a.im == 0.0; }
/* a * 2^k applied to the exponent of each part (exact unless it underflows). */
static inline oz oz_ldexp(oz a, int k) { return oz_make(ldexp(a.re, k), ldexp(a.im, k)); }

/* Complex division a/b by Smith's algorithm (R. L. Smith, CACM 5(8), 1962). */
static oz oz_div(oz a, oz b) {
  if (fabs(b.re) >= fabs(b.im)) {
    double r = b.im / b.re;
    double d = b.re + b.im * r;
    return oz_make((a.re + a.im * r) / d, (a.im - a.re * r) / d);
  } else {
    double r = b.re / b.im;
    double d = b.re * r + b.im;
    return oz_make((a.re * r + a.im) / d, (a.im * r - a.re) / d);
  }
}

#define AT(A, ld, r, c) ((A)[(size_t)(r) + (size_t)(c) * (size_t)(ld)])

static double omega(void) { return ldexp(1.0, OR_OMEGA_EXP); }

/* Smallest k >= 1 with 2^-k * x < Omega, for a finite x >= Omega. */
static int choose_k(double x) {
  int e = ilogb(x);
  int k = e - (OR_OMEGA_EXP - 1);
  return k < 1 ? 1 : k;
}

/* The ratio q = |a|/|b| as (mantissa ratio, exponent) so that it never
 * overflows: returns e = floor(log2 q) and writes the ratio scaled by 2^-kk
 * (kk >= 0) into *scaled.  For a == 0 returns INT_MIN-ish and *scaled = 0. */
static int split_ratio(double a, double b, int kk, double *scaled) {
  if (a == 0.0) { *scaled = 0.0; return -100000; }
  int ea = ilogb(a), eb = ilogb(b);
  double q = ldexp(a, -ea) / ldexp(b, -eb);
  *scaled = ldexp(q, ea - eb - kk);
  return ilogb(q) + ea - eb;
}

/* ||U||_inf over the upper triangle (max row sum of moduli). */
double or_norm_inf_upper(int64_t m, const oz *U, int64_t ldu) {
  double best = 0.0;
  for (int64_t r = 0; r < m; ++r) {
    double s = 0.0;
    for (int64_t c = r; c < m; ++c) s += oz_abs(AT(U, ldu, r, c));
    if (s > best) best = s;
  }
  return best;
}

/* delta of Sec. 3: the replacement for an exactly-zero pivot. */
double or_delta(int64_t m, const oz *U, int64_t ldu) {
  double d = DBL_EPSILON * or_norm_inf_upper(m, U, ldu);
  return d < DBL_MIN ? DBL_MIN : d;
}

/* ------------------------------------------------------------------------
 * Alg. 1 with a shift (Eq. 2): unblocked back substitution on U - lambda*I.
 * This is the plain definition x = (U - lambda I)^{-1} b.
 * ---------------------------------------------------------------------- */
static void trsv_shift(int64_t m, const oz *U, int64_t ldu, oz lambda, oz *b) {
  for (int64_t i = m - 1; i >= 0; --i) {
    b[i] = oz_div(b[i], oz_sub(AT(U, ldu, i, i), lambda));  /* diagonal step */
    oz xi = b[i];
    for (int64_t r = 0; r < i; ++r)                            /* AXPY */
      b[r] = oz_sub(b[r], oz_mul(xi, AT(U, ldu, r, i)));
  }
}

/* Forward substitution on U^H - conj(lambda) I (the lower-triangular case of
 * the footnote in Sec. 2): row r of U^H is conj(U(0:r, r))^T. */
static void trsv_shift_conj_trans(int64_t m, const oz *U, int64_t ldu, oz lambda, oz *b) {
  for (int64_t i = 0; i < m; ++i) {
    oz piv = oz_sub(oz_conj(AT(U, ldu, i, i)), oz_conj(lambda));
    b[i] = oz_div(b[i], piv);
    oz xi = b[i];
    for (int64_t r = i + 1; r < m; ++r)          /* (U^H)(r,i) = conj(U(i,r)) */
      b[r] = oz_sub(b[r], oz_mul(xi, oz_conj(AT(U, ldu, i, r))));
  }
}

/* Multi-shift solve, plain definition: every column j is solved on its own
 * with U - shifts[j] I (Eq. 2) or, when conj_trans, with U^H - conj(shifts[j]) I. */
void or_multishift_solve(int64_t m, const oz *U, int64_t ldu, int64_t n,
                         const oz *shifts, oz *B, int64_t ldb, int conj_trans) {
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; ++j) {
    if (conj_trans) trsv_shift_conj_trans(m, U, ldu, shifts[j], &AT(B, ldb, 0, j));
    else trsv_shift(m, U, ldu, shifts[j], &AT(B, ldb, 0, j));
  }
}

/* ------------------------------------------------------------------------
 * Alg. 4 (SafeTrsv) on the k x k upper-triangular matrix A - lambda I whose
 * top-left element is A[0].  cnorm[i] = max_{r<i} |A(r,i)| are the norms of
 * the columns of A excluding the diagonal (Sec. 3).  b (length k) is
 * overwritten with x; the returned integer kexp gives t = 2^-kexp with
 * (A - lambda I) x = t b.
 * ---------------------------------------------------------------------- */
static int safe_trsv(int64_t k, const oz *A, int64_t lda, oz lambda, double delta,
                     const double *cnorm, oz *b) {
  const double OM = omega();
  if (k <= 0) return 0;
  oz *piv = (oz *)malloc(sizeof(oz) * (size_t)k);
  for (int64_t i = 0; i < k; ++i) {
    piv[i] = oz_sub(AT(A, lda, i, i), lambda);
    if (oz_is_zero(piv[i])) piv[i] = oz_make(delta, 0.0);   /* U(i,i)=0 -> delta */
  }
  /* Growth bounds (the recursions for M(i), G(i) in Sec. 3). */
  double M = 0.0, G = 0.0;
  for (int64_t i = 0; i < k; ++i) { double a = oz_abs(b[i]); if (a > G) G = a; }
  for (int64_t i = k - 1; i >= 0; --i) {
    double ap = oz_abs(piv[i]);
    double q = G / ap;
    if (q > M) M = q;
    G = G * (1.0 + cnorm[i] / ap);
  }
  int kexp = 0;
  if (M < OM && G < OM) {
    /* Well-conditioned case: plain back substitution (Alg. 1). */
    for (int64_t i = k - 1; i >= 0; --i) {
      b[i] = oz_div(b[i], piv[i]);
      oz xi = b[i];
      for (int64_t r = 0; r < i; ++r) b[r] = oz_sub(b[r], oz_mul(xi, AT(A, lda, r, i)));
    }
    free(piv);
    return 0;
  }
  /* Safeguarded back substitution. */
  G = 0.0;
  for (int64_t i = 0; i < k; ++i) { double a = oz_abs(b[i]); if (a > G) G = a; }
  for (int64_t i = k - 1; i >= 0; --i) {
    double Mi;
    int eM = split_ratio(oz_abs(b[i]), oz_abs(piv[i]), 0, &Mi);
    if (eM >= OR_OMEGA_EXP) {                 /* M >= Omega: rescale before dividing */
      int kk = eM - (OR_OMEGA_EXP - 1);
      if (kk < 1) kk = 1;
      for (int64_t r = 0; r < k; ++r) b[r] = oz_ldexp(b[r], -kk);
      kexp += kk;
      G = ldexp(G, -kk);
    }
    b[i] = oz_div(b[i], piv[i]);              /* diagonal step */
    M = oz_abs(b[i]);
    G = G + M * cnorm[i];
    if (G >= OM) {                            /* protect the substitution step */
      int kk = choose_k(G);
      for (int64_t r = 0; r < k; ++r) b[r] = oz_ldexp(b[r], -kk);
      kexp += kk;
      M = ldexp(M, -kk);
      G = ldexp(G, -kk);
    }
    oz xi = b[i];
    for (int64_t r = 0; r < i; ++r) b[r] = oz_sub(b[r], oz_mul(xi, AT(A, lda, r, i)));
  }
  free(piv);
  return kexp;
}

/* Unblocked SafeTrsv (Alg. 4) on the whole U - shifts[j] I for every column:
 * the second, block-free reference for the safe solve. */
void or_safe_trsv_unblocked(int64_t m, const oz *U, int64_t ldu, int64_t n,
                            const oz *shifts, oz *B, int64_t ldb, int32_t *scale_exp) {
  double delta = or_delta(m, U, ldu);
  double *cn = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  for (int64_t i = 0; i < m; ++i) {
    double c = 0.0;
    for (int64_t r = 0; r < i; ++r) { double a = oz_abs(AT(U, ldu, r, i)); if (a > c) c = a; }
    cn[i] = c;
  }
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; ++j)
    scale_exp[j] = safe_trsv(m, U, ldu, shifts[j], delta, cn, &AT(B, ldb, 0, j));
  free(cn);
}

/* ------------------------------------------------------------------------
 * Alg. 5 (SafeMultiShiftTrsm), blocked from the bottom with block size nb.
 * Alg. 5 never mixes columns: the diagonal-block step, the two rescalings and
 * the substitution GEMM act on column j only through column j, so each column
 * is run through the block loop on its own (the GEMM restricted to column j
 * is B(I0,j) -= U(I0,I1) B(I1,j)).
 *
 * shortcut != 0 declares column j of B zero in rows >= j (the strictly upper
 * right-hand sides of Alg. 6); then column j only visits rows < j: blocks
 * that start at or below row j are skipped and the block holding row j-1 is
 * cut at row j (Sec. 4, the footnote on trailing zeros).
 *
 * Per block, the bound of Alg. 5 is G(j) += C_blk * ||B(I1,j)||_inf with the
 * single scalar C_blk = sum_{k in I1} ||U(I0,k)||_inf of the full block.
 * ---------------------------------------------------------------------- */
/* Shift-independent data of Alg. 5: within-block column norms (Sec. 3, the
 * note after Alg. 5 on reusing them for every right-hand side), C_blk per
 * block, and delta. */
typedef struct { double *cin, *cblk; double delta; int64_t nblk; } safe_prep;

static safe_prep safe_prepare(int64_t m, const oz *U, int64_t ldu, int64_t nb) {
  safe_prep P;
  P.delta = or_delta(m, U, ldu);
  P.nblk = (m + nb - 1) / nb;
  P.cin = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  P.cblk = (double *)malloc(sizeof(double) * (size_t)(P.nblk > 0 ? P.nblk : 1));
  for (int64_t b = 0; b < P.nblk; ++b) {
    int64_t hi = m - b * nb, lo = hi - nb < 0 ? 0 : hi - nb;
    double C = 0.0;
    for (int64_t k = lo; k < hi; ++k) {
      double c = 0.0, cu = 0.0;
      for (int64_t r = lo; r < k; ++r) { double a = oz_abs(AT(U, ldu, r, k)); if (a > c) c = a; }
      for (int64_t r = 0; r < lo; ++r) { double a = oz_abs(AT(U, ldu, r, k)); if (a > cu) cu = a; }
      P.cin[k] = c;
      C += cu;
    }
    P.cblk[b] = C;
  }
  return P;
}

static void safe_release(safe_prep *P) { free(P->cin); free(P->cblk); }

/* Alg. 5 for one column x (length m) with shift lambda; rows >= end are zero
 * and never visited.  Returns the scale exponent e (s = 2^-e). */
static int safe_column(int64_t m, const oz *U, int64_t ldu, int64_t nb, const safe_prep *P,
                       oz lambda, oz *x, int64_t end) {
  const double OM = omega();
  int e = 0;
  double G = 0.0;                                  /* G(j) = ||B(:,j)||_inf */
  for (int64_t r = 0; r < end; ++r) { double a = oz_abs(x[r]); if (a > G) G = a; }
  for (int64_t b = 0; b < P->nblk; ++b) {
    int64_t hi = m - b * nb, lo = hi - nb < 0 ? 0 : hi - nb;
    if (lo >= end) continue;                       /* all-zero block of this column */
    int64_t hie = hi < end ? hi : end;
    /* Diagonal block step: SafeTrsv(U(I1,I1) - lambda I, B(I1,j), t). */
    int kk = safe_trsv(hie - lo, &AT(U, ldu, lo, lo), ldu, lambda, P->delta, &P->cin[lo], &x[lo]);
    if (kk > 0) {                                  /* t < 1: rescale I0 and I2 */
      for (int64_t r = 0; r < lo; ++r) x[r] = oz_ldexp(x[r], -kk);
      for (int64_t r = hie; r < end; ++r) x[r] = oz_ldexp(x[r], -kk);
      e += kk;
      G = ldexp(G, -kk);
    }
    double N = 0.0;
    for (int64_t r = lo; r < hie; ++r) { double a = oz_abs(x[r]); if (a > N) N = a; }
    G = G + P->cblk[b] * N;
    if (G >= OM) {                                 /* rescale the whole column */
      int k2 = choose_k(G);
      for (int64_t r = 0; r < end; ++r) x[r] = oz_ldexp(x[r], -k2);
      e += k2;
      G = ldexp(G, -k2);
    }
    /* Substitution step (xGEMM restricted to this column). */
    for (int64_t k = lo; k < hie; ++k) {
      oz xk = x[k];
      for (int64_t r = 0; r < lo; ++r) x[r] = oz_sub(x[r], oz_mul(AT(U, ldu, r, k), xk));
    }
  }
  return e;
}

void or_safe_multishift_solve(int64_t m, const oz *U, int64_t ldu, int64_t n,
                              const oz *shifts, oz *B, int64_t ldb, int64_t nb,
                              int shortcut, int32_t *scale_exp) {
  safe_prep P = safe_prepare(m, U, ldu, nb);
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; ++j) {
    int64_t end = shortcut ? (j < m ? j : m) : m;   /* active rows [0, end) */
    scale_exp[j] = safe_column(m, U, ldu, nb, &P, shifts[j], &AT(B, ldb, 0, j), end);
  }
  safe_release(&P);
}

/* Alg. 6 restricted to the listed columns cols[0..ncols): column c of Zc
 * (m x ncols) receives eigenvector cols[c] exactly as or_trevc computes it. */
void or_trevc_columns(int64_t m, const oz *T, int64_t ldt, int64_t ncols, const int64_t *cols,
                      oz *Zc, int64_t ldzc, int64_t nb, int32_t *scale_exp) {
  safe_prep P = safe_prepare(m, T, ldt, nb);
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < ncols; ++c) {
    int64_t j = cols[c];
    oz *x = &AT(Zc, ldzc, 0, c);
    for (int64_t r = 0; r < m; ++r)
      x[r] = r < j ? oz_make(-AT(T, ldt, r, j).re, -AT(T, ldt, r, j).im) : oz_make(0.0, 0.0);
    scale_exp[c] = safe_column(m, T, ldt, nb, &P, AT(T, ldt, j, j), x, j);
    x[j] = oz_make(ldexp(1.0, -scale_exp[c]), 0.0);
  }
  safe_release(&P);
}

/* Alg. 3 (MultiShiftTrsm), blocked from the bottom: the same block loop as
 * above without the safeguards.  Used to pin that blocking changes rounding
 * only (Sec. 2). */
void or_multishift_solve_blocked(int64_t m, const oz *U, int64_t ldu, int64_t n,
                                 const oz *shifts, oz *B, int64_t ldb, int64_t nb) {
  int64_t nblk = (m + nb - 1) / nb;
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; ++j) {
    oz *x = &AT(B, ldb, 0, j);
    for (int64_t b = 0; b < nblk; ++b) {
      int64_t hi = m - b * nb, lo = hi - nb < 0 ? 0 : hi - nb;
      trsv_shift(hi - lo, &AT(U, ldu, lo, lo), ldu, shifts[j], &x[lo]);
      for (int64_t k = lo; k < hi; ++k) {
        oz xk = x[k];
        for (int64_t r = 0; r < lo; ++r) x[r] = oz_sub(x[r], oz_mul(AT(U, ldu, r, k), xk));
      }
    }
  }
}

/* ------------------------------------------------------------------------
 * Alg. 6 (TriangEig): lambda = diag(T); Z = -T with diag(Z) = 0 (and zero
 * below the diagonal); SafeMultiShiftTrsm with the strictly-upper shortcut;
 * diag(Z) = s.  scales[j] = 2^-scale_exp[j] (0 once it underflows).
 * ---------------------------------------------------------------------- */
void or_trevc(int64_t m, const oz *T, int64_t ldt, oz *Z, int64_t ldz, int64_t nb,
              int32_t *scale_exp, double *scales) {
  oz *lam = (oz *)calloc((size_t)(m > 0 ? m : 1), sizeof(oz));
  for (int64_t j = 0; j < m; ++j) {
    lam[j] = AT(T, ldt, j, j);
    for (int64_t r = 0; r < m; ++r)
      AT(Z, ldz, r, j) = r < j ? oz_make(-AT(T, ldt, r, j).re, -AT(T, ldt, r, j).im)
                               : oz_make(0.0, 0.0);
  }
  or_safe_multishift_solve(m, T, ldt, m, lam, Z, ldz, nb, 1, scale_exp);
  for (int64_t j = 0; j < m; ++j) {
    scales[j] = ldexp(1.0, -scale_exp[j]);
    AT(Z, ldz, j, j) = oz_make(scales[j], 0.0);
  }
  free(lam);
}

/* ------------------------------------------------------------------------
 * Largest eigenvalue of the real symmetric tridiagonal matrix with diagonal
 * a[0..k) and off-diagonal b[0..k-1), by bisection on Sturm counts
 * (Barth, Martin & Wilkinson, Numer. Math. 9, 1967).  count(x) is the number
 * of eigenvalues below x, read off as the negative pivots of the LDL^T
 * factorisation of (tridiag - x I).
 * ---------------------------------------------------------------------- */
static int sturm_count(int k, const double *a, const double *b, double x, double pivmin) {
  int c = 0;
  double d = a[0] - x;
  if (d < 0.0) ++c;
  for (int i = 1; i < k; ++i) {
    if (fabs(d) < pivmin) d = -pivmin;
    d = (a[i] - x) - b[i - 1] * b[i - 1] / d;
    if (d < 0.0) ++c;
  }
  return c;
}

double or_tridiag_max_eig(int k, const double *a, const double *b) {
  if (k <= 0) return 0.0;
  double lo = a[0], hi = a[0], bmax2 = 0.0;
  for (int i = 0; i < k; ++i) {
    double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < k ? fabs(b[i]) : 0.0);
    if (a[i] - r < lo) lo = a[i] - r;
    if (a[i] + r > hi) hi = a[i] + r;
    if (i + 1 < k && b[i] * b[i] > bmax2) bmax2 = b[i] * b[i];
  }
  double pivmin = DBL_MIN * (bmax2 > 1.0 ? bmax2 : 1.0);
  /* Widen the Gershgorin interval slightly so that it strictly brackets. */
  double w = fabs(hi) > fabs(lo) ? fabs(hi) : fabs(lo);
  lo -= 4.0 * DBL_EPSILON * w + pivmin;
  hi += 4.0 * DBL_EPSILON * w + pivmin;
  for (int it = 0; it < 4096; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(k, a, b, mid, pivmin) >= k) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------
 * Alg. 7 (Van Loan / Lui) on a triangular T: for every grid point z_p the
 * largest eigenvalue of (T - z I)^{-H} (T - z I)^{-1} is estimated by Lanczos
 * and sigma_min(T - z I) = 1/sqrt(theta_max) (Sec. 5).  Each operator apply is
 * two triangular solves: upper with T - z I, then lower with (T - z I)^H.
 *
 * Readings: the start vector of point p is column p of V0, normalised; the
 * Lanczos vectors are fully reorthogonalised by classical Gram-Schmidt, run a
 * second time only when the first pass removed more than half of ||w||^2
 * (Kahan-Parlett "twice is enough"); exactly min(iters, m) steps are taken,
 * stopping earlier only when beta_k <= 1e-14 * max_{i<=k} |alpha_i|.  alpha/beta (iters x N, column p
 * for point p; may be NULL) receive the tridiagonal, steps[p] its order.
 * ---------------------------------------------------------------------- */
void or_pseudospectra(int64_t m, const oz *T, int64_t ldt, int64_t N, const oz *z,
                      const oz *V0, int64_t ldv, int iters, double *sigma_min,
                      double *alpha_out, double *beta_out, int32_t *steps_out) {
  int K = iters < m ? iters : (int)m;
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < N; ++p) {
    oz *V = (oz *)calloc((size_t)(K + 1) * (size_t)m, sizeof(oz));
    oz *w = (oz *)malloc(sizeof(oz) * (size_t)m);
    double *al = (double *)calloc((size_t)K + 1, sizeof(double));
    double *be = (double *)calloc((size_t)K + 1, sizeof(double));
    double nv = 0.0;
    for (int64_t r = 0; r < m; ++r) { oz v = AT(V0, ldv, r, p); nv += v.re * v.re + v.im * v.im; }
    nv = sqrt(nv);
    for (int64_t r = 0; r < m; ++r) V[r] = oz_scale(AT(V0, ldv, r, p), 1.0 / nv);
    int steps = 0;
    double amax = 0.0;
    for (int k = 0; k < K; ++k) {
      oz *vk = &V[(size_t)k * m];
      memcpy(w, vk, sizeof(oz) * (size_t)m);
      trsv_shift(m, T, ldt, z[p], w);              /* y = (T - zI)^{-1} v_k   */
      trsv_shift_conj_trans(m, T, ldt, z[p], w);   /* w = (T - zI)^{-H} y     */
      double a = 0.0;                              /* alpha_k = Re(v_k^H w)   */
      for (int64_t r = 0; r < m; ++r) a += vk[r].re * w[r].re + vk[r].im * w[r].im;
      al[k] = a;
      if (fabs(a) > amax) amax = fabs(a);
      for (int64_t r = 0; r < m; ++r) w[r] = oz_sub(w[r], oz_scale(vk[r], a));
      if (k > 0) {
        oz *vp = &V[(size_t)(k - 1) * m];
        for (int64_t r = 0; r < m; ++r) w[r] = oz_sub(w[r], oz_scale(vp[r], be[k - 1]));
      }
      /* classical Gram-Schmidt against v_0..v_k, repeated once when the first
       * pass removed more than half of ||w||^2 ("twice is enough") */
      double n0 = 0.0;
      for (int64_t r = 0; r < m; ++r) n0 += w[r].re * w[r].re + w[r].im * w[r].im;
      for (int pass = 0; pass < 2; ++pass) {
        oz h[64];
        oz *hh = (k + 1 <= 64) ? h : (oz *)malloc(sizeof(oz) * (size_t)(k + 1));
        for (int i = 0; i <= k; ++i) {
          oz *vi = &V[(size_t)i * m];
          oz s = oz_make(0.0, 0.0);
          for (int64_t r = 0; r < m; ++r) s = oz_add(s, oz_mul(oz_conj(vi[r]), w[r]));
          hh[i] = s;
        }
        for (int i = 0; i <= k; ++i) {
          oz *vi = &V[(size_t)i * m];
          for (int64_t r = 0; r < m; ++r) w[r] = oz_sub(w[r], oz_mul(vi[r], hh[i]));
        }
        if (hh != h) free(hh);
        if (pass == 0) {
          double n1 = 0.0;
          for (int64_t r = 0; r < m; ++r) n1 += w[r].re * w[r].re + w[r].im * w[r].im;
          if (!(n1 < 0.5 * n0)) break;
        }
      }
      double bn = 0.0;
      for (int64_t r = 0; r < m; ++r) bn += w[r].re * w[r].re + w[r].im * w[r].im;
      bn = sqrt(bn);
      be[k] = bn;
      steps = k + 1;
      if (k == K - 1) break;
      if (bn <= 1e-14 * amax) break;               /* invariant subspace found */
      oz *vn = &V[(size_t)(k + 1) * m];
      for (int64_t r = 0; r < m; ++r) vn[r] = oz_scale(w[r], 1.0 / bn);
    }
    double theta = or_tridiag_max_eig(steps, al, be);
    sigma_min[p] = 1.0 / sqrt(theta);
    if (alpha_out)
      for (int k = 0; k < iters; ++k) alpha_out[(size_t)p * iters + k] = k < steps ? al[k] : 0.0;
    if (beta_out)
      for (int k = 0; k < iters; ++k) beta_out[(size_t)p * iters + k] = k < steps ? be[k] : 0.0;
    if (steps_out) steps_out[p] = steps;
    free(V); free(w); free(al); free(be);
  }
}

/* ------------------------------------------------------------------------
 * Adjoint of X = MultiShiftTrsm(U, s, B) for a real loss L, with the complex
 * gradient convention g = dL/dRe + i dL/dIm, so that dL = Re<g, d.>:
 *   lambda_j = (U - s_j I)^{-H} g_j     (a multi-shift solve with U^H, conj s)
 *   dL/dB    = Lambda
 *   dL/dU    = -triu(Lambda X^H)        (only the upper triangle is a parameter)
 *   dL/ds_j  = x_j^H lambda_j
 * which follows from dx_j = (U - s_j I)^{-1} (db_j - dU x_j + ds_j x_j).
 * X is recomputed here from U, s and B.
 * ---------------------------------------------------------------------- */
void or_adjoint(int64_t m, const oz *U, int64_t ldu, int64_t n, const oz *shifts,
                const oz *B, int64_t ldb, const oz *GX, int64_t ldg,
                oz *dU, int64_t lddu, oz *dB, int64_t lddb, oz *ds) {
  oz *X = (oz *)malloc(sizeof(oz) * (size_t)(m > 0 ? m : 1) * (size_t)(n > 0 ? n : 1));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t r = 0; r < m; ++r) {
      X[r + j * m] = AT(B, ldb, r, j);
      AT(dB, lddb, r, j) = AT(GX, ldg, r, j);
    }
  or_multishift_solve(m, U, ldu, n, shifts, X, m, 0);
  or_multishift_solve(m, U, ldu, n, shifts, dB, lddb, 1);
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < m; ++c)
    for (int64_t r = 0; r < m; ++r) {
      oz acc = oz_make(0.0, 0.0);
      if (r <= c)
        for (int64_t j = 0; j < n; ++j)
          acc = oz_add(acc, oz_mul(AT(dB, lddb, r, j), oz_conj(X[c + j * m])));
      AT(dU, lddu, r, c) = oz_make(-acc.re, -acc.im);
    }
  for (int64_t j = 0; j < n; ++j) {
    oz acc = oz_make(0.0, 0.0);
    for (int64_t r = 0; r < m; ++r) acc = oz_add(acc, oz_mul(oz_conj(X[r + j * m]), AT(dB, lddb, r, j)));
    ds[j] = acc;
  }
  free(X);
}

/* Number of OpenMP threads the oracle runs with (1 without OpenMP). */
/* ------------------------------------------------------------------------
 * Generalized multi-shift triangular solve (appendix, Alg. 8):
 * (U - lambda_j V) x_j = b_j with U, V upper triangular.  Plain definition,
 * per shift: unblocked back substitution on U - lambda V, whose entries are
 * formed as U(r,i) - lambda V(r,i).
 * ---------------------------------------------------------------------- */
static inline oz gentry(const oz *U, int64_t ldu, const oz *V, int64_t ldv, oz lambda, int64_t r, int64_t c) {
  return oz_sub(AT(U, ldu, r, c), oz_mul(lambda, AT(V, ldv, r, c)));
}

static void trsv_gshift(int64_t m, const oz *U, int64_t ldu, const oz *V, int64_t ldv, oz lambda, oz *b) {
  for (int64_t i = m - 1; i >= 0; --i) {
    b[i] = oz_div(b[i], gentry(U, ldu, V, ldv, lambda, i, i));   /* diagonal step */
    oz xi = b[i];
    for (int64_t r = 0; r < i; ++r)                               /* AXPY */
      b[r] = oz_sub(b[r], oz_mul(xi, gentry(U, ldu, V, ldv, lambda, r, i)));
  }
}

void or_gmultishift_solve(int64_t m, const oz *U, int64_t ldu, const oz *V, int64_t ldv, int64_t n,
                          const oz *shifts, oz *B, int64_t ldb) {
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; ++j) trsv_gshift(m, U, ldu, V, ldv, shifts[j], &AT(B, ldb, 0, j));
}

/* Alg. 4 on the k x k block U' = A - lambda W (A, W the diagonal blocks of U
 * and V): as safe_trsv, with the pivots and AXPY entries of U' and the column
 * bounds cnorm[i] = cnU[i] + |lambda| cnV[i] >= max_{r<i} |U'(r,i)|. */
static int safe_gtrsv(int64_t k, const oz *A, int64_t lda, const oz *Wv, int64_t ldw, oz lambda,
                      double delta, const double *cnU, const double *cnV, oz *b) {
  const double OM = omega();
  if (k <= 0) return 0;
  const double al = oz_abs(lambda);
  oz *piv = (oz *)malloc(sizeof(oz) * (size_t)k);
  double *cnorm = (double *)malloc(sizeof(double) * (size_t)k);
  for (int64_t i = 0; i < k; ++i) {
    piv[i] = gentry(A, lda, Wv, ldw, lambda, i, i);
    if (oz_is_zero(piv[i])) piv[i] = oz_make(delta, 0.0);   /* U'(i,i)=0 -> delta */
    cnorm[i] = cnU[i] + al * cnV[i];
  }
  double M = 0.0, G = 0.0;
  for (int64_t i = 0; i < k; ++i) { double a = oz_abs(b[i]); if (a > G) G = a; }
  for (int64_t i = k - 1; i >= 0; --i) {
    double ap = oz_abs(piv[i]);
    double q = G / ap;
    if (q > M) M = q;
    G = G * (1.0 + cnorm[i] / ap);
  }
  int kexp = 0;
  if (M < OM && G < OM) {
    for (int64_t i = k - 1; i >= 0; --i) {
      b[i] = oz_div(b[i], piv[i]);
      oz xi = b[i];
      for (int64_t r = 0; r < i; ++r) b[r] = oz_sub(b[r], oz_mul(xi, gentry(A, lda, Wv, ldw, lambda, r, i)));
    }
    free(piv); free(cnorm);
    return 0;
  }
  G = 0.0;
  for (int64_t i = 0; i < k; ++i) { double a = oz_abs(b[i]); if (a > G) G = a; }
  for (int64_t i = k - 1; i >= 0; --i) {
    double Mi;
    int eM = split_ratio(oz_abs(b[i]), oz_abs(piv[i]), 0, &Mi);
    if (eM >= OR_OMEGA_EXP) {
      int kk = eM - (OR_OMEGA_EXP - 1);
      if (kk < 1) kk = 1;
      for (int64_t r = 0; r < k; ++r) b[r] = oz_ldexp(b[r], -kk);
      kexp += kk;
      G = ldexp(G, -kk);
    }
    b[i] = oz_div(b[i], piv[i]);
    M = oz_abs(b[i]);
    G = G + M * cnorm[i];
    if (G >= OM) {
      int kk = choose_k(G);
      for (int64_t r = 0; r < k; ++r) b[r] = oz_ldexp(b[r], -kk);
      kexp += kk;
      M = ldexp(M, -kk);
      G = ldexp(G, -kk);
    }
    oz xi = b[i];
    for (int64_t r = 0; r < i; ++r) b[r] = oz_sub(b[r], oz_mul(xi, gentry(A, lda, Wv, ldw, lambda, r, i)));
  }
  free(piv); free(cnorm);
  return kexp;
}

/* Shift-independent data of Alg. 9: within-block column norms and the block
 * sums C_blk of U and of V, and ||U||_inf, ||V||_inf for delta. */
typedef struct { double *cinU, *cinV, *cblkU, *cblkV; double nU, nV; int64_t nblk; } gsafe_prep;

static void colnorm_blocks(int64_t m, const oz *U, int64_t ldu, int64_t nb, int64_t nblk, double *cin,
                           double *cblk) {
  for (int64_t b = 0; b < nblk; ++b) {
    int64_t hi = m - b * nb, lo = hi - nb < 0 ? 0 : hi - nb;
    double C = 0.0;
    for (int64_t k = lo; k < hi; ++k) {
      double c = 0.0, cu = 0.0;
      for (int64_t r = lo; r < k; ++r) { double a = oz_abs(AT(U, ldu, r, k)); if (a > c) c = a; }
      for (int64_t r = 0; r < lo; ++r) { double a = oz_abs(AT(U, ldu, r, k)); if (a > cu) cu = a; }
      cin[k] = c;
      C += cu;
    }
    cblk[b] = C;
  }
}

static gsafe_prep gsafe_prepare(int64_t m, const oz *U, int64_t ldu, const oz *V, int64_t ldv, int64_t nb) {
  gsafe_prep P;
  P.nblk = (m + nb - 1) / nb;
  size_t mm = (size_t)(m > 0 ? m : 1), nn = (size_t)(P.nblk > 0 ? P.nblk : 1);
  P.cinU = (double *)malloc(sizeof(double) * mm);
  P.cinV = (double *)malloc(sizeof(double) * mm);
  P.cblkU = (double *)malloc(sizeof(double) * nn);
  P.cblkV = (double *)malloc(sizeof(double) * nn);
  colnorm_blocks(m, U, ldu, nb, P.nblk, P.cinU, P.cblkU);
  colnorm_blocks(m, V, ldv, nb, P.nblk, P.cinV, P.cblkV);
  P.nU = or_norm_inf_upper(m, U, ldu);
  P.nV = or_norm_inf_upper(m, V, ldv);
  return P;
}

static void gsafe_release(gsafe_prep *P) { free(P->cinU); free(P->cinV); free(P->cblkU); free(P->cblkV); }

/* Alg. 9 for one column x with shift lambda; rows >= end are zero and never
 * visited.  Readings: the within-block SafeTrsv uses the column bounds of
 * safe_gtrsv; delta_j = max(eps (||U||_inf + |lambda| ||V||_inf), DBL_MIN); the
 * block bound is (C_blk(U) + |lambda| C_blk(V)) ||B(I1,j)||_inf, and the
 * update subtracts U(I0,I1) X(I1,j) and then adds V(I0,I1) (lambda X(I1,j)). */
static int gsafe_column(int64_t m, const oz *U, int64_t ldu, const oz *V, int64_t ldv, int64_t nb,
                        const gsafe_prep *P, oz lambda, oz *x, int64_t end) {
  const double OM = omega();
  const double al = oz_abs(lambda);
  double delta = DBL_EPSILON * (P->nU + al * P->nV);
  if (delta < DBL_MIN) delta = DBL_MIN;
  int e = 0;
  double G = 0.0;
  for (int64_t r = 0; r < end; ++r) { double a = oz_abs(x[r]); if (a > G) G = a; }
  for (int64_t b = 0; b < P->nblk; ++b) {
    int64_t hi = m - b * nb, lo = hi - nb < 0 ? 0 : hi - nb;
    if (lo >= end) continue;
    int64_t hie = hi < end ? hi : end;
    int kk = safe_gtrsv(hie - lo, &AT(U, ldu, lo, lo), ldu, &AT(V, ldv, lo, lo), ldv, lambda, delta,
                        &P->cinU[lo], &P->cinV[lo], &x[lo]);
    if (kk > 0) {
      for (int64_t r = 0; r < lo; ++r) x[r] = oz_ldexp(x[r], -kk);
      for (int64_t r = hie; r < end; ++r) x[r] = oz_ldexp(x[r], -kk);
      e += kk;
      G = ldexp(G, -kk);
    }
    double N = 0.0;
    for (int64_t r = lo; r < hie; ++r) { double a = oz_abs(x[r]); if (a > N) N = a; }
    G = G + (P->cblkU[b] + al * P->cblkV[b]) * N;
    if (G >= OM) {
      int k2 = choose_k(G);
      for (int64_t r = 0; r < end; ++r) x[r] = oz_ldexp(x[r], -k2);
      e += k2;
      G = ldexp(G, -k2);
    }
    for (int64_t k = lo; k < hie; ++k) {                     /* B(I0,j) -= U(I0,I1) X(I1,j) */
      oz xk = x[k];
      for (int64_t r = 0; r < lo; ++r) x[r] = oz_sub(x[r], oz_mul(AT(U, ldu, r, k), xk));
    }
    for (int64_t k = lo; k < hie; ++k) {                     /* B(I0,j) += V(I0,I1) C(:,j) */
      oz ck = oz_mul(lambda, x[k]);
      for (int64_t r = 0; r < lo; ++r) x[r] = oz_add(x[r], oz_mul(AT(V, ldv, r, k), ck));
    }
  }
  return e;
}

void or_safe_gmultishift_solve(int64_t m, const oz *U, int64_t ldu, const oz *V, int64_t ldv, int64_t n,
                               const oz *shifts, oz *B, int64_t ldb, int64_t nb, int shortcut,
                               int32_t *scale_exp) {
  gsafe_prep P = gsafe_prepare(m, U, ldu, V, ldv, nb);
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; ++j) {
    int64_t end = shortcut ? (j < m ? j : m) : m;
    scale_exp[j] = gsafe_column(m, U, ldu, V, ldv, nb, &P, shifts[j], &AT(B, ldb, 0, j), end);
  }
  gsafe_release(&P);
}

/* Alg. 10 (GeneralizedTriangEig): lambda = diag(T) ./ diag(S) (S(j,j) != 0);
 * Z = -T + S diag(lambda) strictly above the diagonal, zero elsewhere;
 * SafeGeneralizedMultiShiftTrsm with the strictly-upper shortcut; diag(Z) = s. */
void or_gtrevc(int64_t m, const oz *T, int64_t ldt, const oz *S, int64_t lds, oz *Z, int64_t ldz,
               oz *lam, int64_t nb, int32_t *scale_exp, double *scales) {
  for (int64_t j = 0; j < m; ++j) {
    lam[j] = oz_div(AT(T, ldt, j, j), AT(S, lds, j, j));
    for (int64_t r = 0; r < m; ++r)
      AT(Z, ldz, r, j) = r < j ? oz_sub(oz_mul(lam[j], AT(S, lds, r, j)), AT(T, ldt, r, j)) : oz_make(0.0, 0.0);
  }
  or_safe_gmultishift_solve(m, T, ldt, S, lds, m, lam, Z, ldz, nb, 1, scale_exp);
  for (int64_t j = 0; j < m; ++j) {
    scales[j] = ldexp(1.0, -scale_exp[j]);
    AT(Z, ldz, j, j) = oz_make(scales[j], 0.0);
  }
}

/* Alg. 10 for the listed columns only, each exactly as or_gtrevc computes it
 * (the same block partition and bounds): Zc(:, c) is eigenvector cols[c]. */
void or_gtrevc_columns(int64_t m, const oz *T, int64_t ldt, const oz *S, int64_t lds, int64_t ncols,
                       const int64_t *cols, oz *Zc, int64_t ldzc, oz *lam, int64_t nb, int32_t *scale_exp) {
  gsafe_prep P = gsafe_prepare(m, T, ldt, S, lds, nb);
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < ncols; ++c) {
    int64_t j = cols[c];
    oz l = oz_div(AT(T, ldt, j, j), AT(S, lds, j, j));
    oz *x = &AT(Zc, ldzc, 0, c);
    for (int64_t r = 0; r < m; ++r)
      x[r] = r < j ? oz_sub(oz_mul(l, AT(S, lds, r, j)), AT(T, ldt, r, j)) : oz_make(0.0, 0.0);
    scale_exp[c] = gsafe_column(m, T, ldt, S, lds, nb, &P, l, x, j);
    x[j] = oz_make(ldexp(1.0, -scale_exp[c]), 0.0);
    lam[c] = l;
  }
  gsafe_release(&P);
}

/* ------------------------------------------------------------------------
 * Back-transformation (Sec. 4, Alg. 6 "Eig"): the eigenvectors of
 * A = Q T Q^H are X = Q Z, Z upper triangular (only its upper triangle is
 * read).  Plain definition: X(i,j) = sum_{k <= j} Q(i,k) Z(k,j), summed in
 * increasing k.
 * ---------------------------------------------------------------------- */
void or_back_transform(int64_t m, const oz *Q, int64_t ldq, const oz *Z, int64_t ldz, oz *X, int64_t ldx) {
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < m; ++j)
    for (int64_t i = 0; i < m; ++i) {
      oz s = oz_make(0.0, 0.0);
      for (int64_t k = 0; k <= j; ++k) s = oz_add(s, oz_mul(AT(Q, ldq, i, k), AT(Z, ldz, k, j)));
      AT(X, ldx, i, j) = s;
    }
}

/* ------------------------------------------------------------------------
 * The other triangular variants (footnote to Sec. 2: the lower-triangular
 * and right-hand cases).  The operator is M_j = op(A) - s_j I, op(A) = A, A^T
 * or A^H (trans = 0, 1, 2), A upper (uplo = 0) or lower (uplo = 1)
 * triangular; only that triangle of A is read.
 *   left  (side = 0): M_j x_j = b_j,       x_j, b_j column j of the m x n B;
 *   right (side = 1): x_j^T M_j = b_j^T,   x_j, b_j row j of the n x m B.
 * A right-side system is the left-side system with the transposed operator
 * M_j^T = op'(A) - s_j I, where op' maps A -> A^T, A^T -> A and A^H -> conj(A)
 * (internal code 3).  Plain definition per shift: unblocked substitution in
 * the order the triangle of M_j fixes -- back substitution when M_j is upper
 * triangular, forward substitution when it is lower triangular.
 * ---------------------------------------------------------------------- */
static inline oz op_entry(const oz *A, int64_t lda, int op, int64_t r, int64_t c) {
  if (op == 0) return AT(A, lda, r, c);
  if (op == 3) return oz_conj(AT(A, lda, r, c));
  oz a = AT(A, lda, c, r);
  return op == 2 ? oz_conj(a) : a;
}

/* op(A) is upper triangular when A is upper and op keeps the triangle
 * (op = A or conj(A)), or A is lower and op transposes. */
static inline int op_is_upper(int uplo, int op) { return (uplo == 0) == (op == 0 || op == 3); }

static int right_op(int trans) { return trans == 0 ? 1 : (trans == 1 ? 0 : 3); }

static void trsv_op_shift(int64_t m, const oz *A, int64_t lda, int uplo, int op, oz s, oz *x) {
  if (op_is_upper(uplo, op)) {
    for (int64_t i = m - 1; i >= 0; --i) {
      x[i] = oz_div(x[i], oz_sub(op_entry(A, lda, op, i, i), s));
      oz xi = x[i];
      for (int64_t r = 0; r < i; ++r) x[r] = oz_sub(x[r], oz_mul(xi, op_entry(A, lda, op, r, i)));
    }
  } else {
    for (int64_t i = 0; i < m; ++i) {
      x[i] = oz_div(x[i], oz_sub(op_entry(A, lda, op, i, i), s));
      oz xi = x[i];
      for (int64_t r = i + 1; r < m; ++r) x[r] = oz_sub(x[r], oz_mul(xi, op_entry(A, lda, op, r, i)));
    }
  }
}

void or_solve_variant(int side, int uplo, int trans, int64_t m, int64_t n, const oz *A, int64_t lda,
                      const oz *shifts, oz *B, int64_t ldb) {
  const int op = side == 0 ? trans : right_op(trans);
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t j = 0; j < n; ++j) {
    if (side == 0) {
      trsv_op_shift(m, A, lda, uplo, op, shifts[j], &AT(B, ldb, 0, j));
    } else {
      oz *x = (oz *)malloc(sizeof(oz) * (size_t)(m > 0 ? m : 1));
      for (int64_t c = 0; c < m; ++c) x[c] = AT(B, ldb, j, c);
      trsv_op_shift(m, A, lda, uplo, op, shifts[j], x);
      for (int64_t c = 0; c < m; ++c) AT(B, ldb, j, c) = x[c];
      free(x);
    }
  }
}

/* Safe form of every variant: Alg. 5 run in the variant's own substitution
 * order.  The operator is first written as an upper-triangular matrix U in
 * that order -- U = op'(A) when it is upper triangular, else the reversal
 * U(r,c) = op'(A)(m-1-r, m-1-c) with the right-hand side reversed alike --
 * so the blocks are cut from the end where the substitution starts (the
 * ragged block is the last one visited), and SafeMultiShiftTrsm runs on it. */
void or_safe_solve_variant(int side, int uplo, int trans, int64_t m, int64_t n, const oz *A, int64_t lda,
                           const oz *shifts, oz *B, int64_t ldb, int64_t nb, int32_t *scale_exp) {
  const int op = side == 0 ? trans : right_op(trans);
  const int rev = !op_is_upper(uplo, op);
  size_t mm = (size_t)(m > 0 ? m : 1), nn = (size_t)(n > 0 ? n : 1);
  oz *U = (oz *)calloc(mm * mm, sizeof(oz));
  oz *X = (oz *)malloc(sizeof(oz) * mm * nn);
  for (int64_t c = 0; c < m; ++c)
    for (int64_t r = 0; r <= c; ++r)
      U[r + c * (int64_t)mm] = rev ? op_entry(A, lda, op, m - 1 - r, m - 1 - c) : op_entry(A, lda, op, r, c);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t r = 0; r < m; ++r) {
      int64_t q = rev ? m - 1 - r : r;
      X[r + j * (int64_t)mm] = side == 0 ? AT(B, ldb, q, j) : AT(B, ldb, j, q);
    }
  or_safe_multishift_solve(m, U, (int64_t)mm, n, shifts, X, (int64_t)mm, nb, 0, scale_exp);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t r = 0; r < m; ++r) {
      int64_t q = rev ? m - 1 - r : r;
      if (side == 0) AT(B, ldb, q, j) = X[r + j * (int64_t)mm];
      else AT(B, ldb, j, q) = X[r + j * (int64_t)mm];
    }
  free(U);
  free(X);
}

/* ------------------------------------------------------------------------
 * 1-norm pseudospectra (the footnote to Sec. 5: Hager's estimator as refined
 * by Higham, driven by shifted triangular solves with the grid points as
 * shifts).  For each grid point z, an estimate of ||R||_1 with
 * R = Q (T - zI)^{-1} Q^H, i.e. the resolvent norm ||(zI - A)^{-1}||_1 of
 * A = Q T Q^H (Q = I when Q is NULL; the sign of the resolvent does not
 * change any norm).
 *
 * Estimator (t = 1 column, at most 5 gradient steps), with y = R x,
 * g = ||y||_1 and sign(y)_i = y_i/|y_i| (1 where y_i = 0):
 *   x = (1/m) e;  y = R x;  est = g;  kind = -1
 *   repeat up to 5 times:
 *     w = R^H sign(y);  j = the first index of max_i |w_i|
 *     stop if |w_j| <= g                 (x is a local maximum of ||R x||_1:
 *                                          w^H x = ||R x||_1 for every x)
 *     x = e_j;  y = R x;  g = ||y||_1
 *     stop if g <= est                   (no increase)
 *     est = g;  kind = j
 *   alternative vector x_i = (-1)^i (1 + i/(m-1)), i = 0..m-1 (m >= 2):
 *     est = max(est, 2 ||R x||_1 / (3m)), kind = -2 when it wins.
 * steps[p] = the number of R^H applications.  ||y||_1 sums the moduli in
 * increasing row order.
 * ---------------------------------------------------------------------- */
static void apply_resolvent(int64_t m, const oz *T, int64_t ldt, const oz *Q, int64_t ldq, oz z, int adj,
                            oz *x, oz *tmp) {
  if (Q) {
    for (int64_t i = 0; i < m; ++i) {                 /* tmp = Q^H x */
      oz s = oz_make(0.0, 0.0);
      for (int64_t r = 0; r < m; ++r) s = oz_add(s, oz_mul(oz_conj(AT(Q, ldq, r, i)), x[r]));
      tmp[i] = s;
    }
  } else {
    memcpy(tmp, x, sizeof(oz) * (size_t)m);
  }
  if (adj) trsv_shift_conj_trans(m, T, ldt, z, tmp);  /* (T - zI)^{-H}: (T^H - conj(z) I)^{-1} */
  else trsv_shift(m, T, ldt, z, tmp);
  if (Q) {
    for (int64_t r = 0; r < m; ++r) {                 /* x = Q tmp */
      oz s = oz_make(0.0, 0.0);
      for (int64_t i = 0; i < m; ++i) s = oz_add(s, oz_mul(AT(Q, ldq, r, i), tmp[i]));
      x[r] = s;
    }
  } else {
    memcpy(x, tmp, sizeof(oz) * (size_t)m);
  }
}

static double norm1_vec(int64_t m, const oz *y) {
  double s = 0.0;
  for (int64_t i = 0; i < m; ++i) s += oz_abs(y[i]);
  return s;
}

static void sign_vec(int64_t m, oz *y) {
  for (int64_t i = 0; i < m; ++i) {
    double a = oz_abs(y[i]);
    y[i] = a == 0.0 ? oz_make(1.0, 0.0) : oz_make(y[i].re / a, y[i].im / a);
  }
}

void or_pseudospectra_1norm(int64_t m, const oz *T, int64_t ldt, const oz *Q, int64_t ldq, int64_t N,
                            const oz *z, double *est_out, int32_t *kind_out, int32_t *steps_out) {
  #pragma omp parallel for schedule(dynamic, 1)
  for (int64_t p = 0; p < N; ++p) {
    oz *y = (oz *)malloc(sizeof(oz) * (size_t)(m > 0 ? m : 1));
    oz *tmp = (oz *)malloc(sizeof(oz) * (size_t)(m > 0 ? m : 1));
    for (int64_t i = 0; i < m; ++i) y[i] = oz_make(1.0 / (double)m, 0.0);
    apply_resolvent(m, T, ldt, Q, ldq, z[p], 0, y, tmp);
    double g = norm1_vec(m, y), est = g;
    int kind = -1, steps = 0;
    for (int it = 0; it < 5 && m > 1; ++it) {
      sign_vec(m, y);
      apply_resolvent(m, T, ldt, Q, ldq, z[p], 1, y, tmp);       /* w = R^H sign(y) */
      ++steps;
      int64_t j = 0;
      double wj = -1.0;
      for (int64_t i = 0; i < m; ++i) { double a = oz_abs(y[i]); if (a > wj) { wj = a; j = i; } }
      if (wj <= g) break;
      for (int64_t i = 0; i < m; ++i) y[i] = oz_make(i == j ? 1.0 : 0.0, 0.0);
      apply_resolvent(m, T, ldt, Q, ldq, z[p], 0, y, tmp);
      g = norm1_vec(m, y);
      if (g <= est) break;
      est = g;
      kind = (int)j;
    }
    if (m > 1) {
      for (int64_t i = 0; i < m; ++i) {
        double v = 1.0 + (double)i / (double)(m - 1);
        y[i] = oz_make((i & 1) ? -v : v, 0.0);
      }
      apply_resolvent(m, T, ldt, Q, ldq, z[p], 0, y, tmp);
      double alt = 2.0 * norm1_vec(m, y) / (3.0 * (double)m);
      if (alt > est) { est = alt; kind = -2; }
    }
    est_out[p] = est;
    kind_out[p] = kind;
    steps_out[p] = steps;
    free(y);
    free(tmp);
  }
}

/* ------------------------------------------------------------------------
 * Automatic grid of a spectral portrait (the SpectralPortrait driver listed in
 * Sec. 6, whose grid the paper leaves to the software): the bounding box
 * [a, b] x [c, d] of the eigenvalues diag(T), widened on every side by
 * h = max(0.25 max(b - a, d - c), 2^-20 max(1, max_i max(|Re T(i,i)|, |Im T(i,i)|)))
 * (no square roots: the grid is exact up to the roundings written here), and
 * sampled with nx x ny points: x0 = a - h, x1 = b + h, dx = (x1 - x0)/(nx - 1)
 * (0 when nx == 1), z(k, l) = (x0 + k dx) + i (y0 + l dy), likewise in y;
 * point k + l nx.  Every operation is a single rounding in the order written.
 * ---------------------------------------------------------------------- */
void or_portrait_grid(int64_t m, const oz *T, int64_t ldt, int64_t nx, int64_t ny, oz *zout, double *box) {
  double a = 0.0, b = 0.0, c = 0.0, d = 0.0, big = 1.0;
  for (int64_t i = 0; i < m; ++i) {
    oz t = AT(T, ldt, i, i);
    if (i == 0 || t.re < a) a = t.re;
    if (i == 0 || t.re > b) b = t.re;
    if (i == 0 || t.im < c) c = t.im;
    if (i == 0 || t.im > d) d = t.im;
    if (fabs(t.re) > big) big = fabs(t.re);
    if (fabs(t.im) > big) big = fabs(t.im);
  }
  double w = b - a, hgt = d - c;
  double h = 0.25 * (w > hgt ? w : hgt);
  double hmin = ldexp(big, -20);
  if (h < hmin) h = hmin;
  double x0 = a - h, y0 = c - h;
  double dx = nx > 1 ? ((b + h) - x0) / (double)(nx - 1) : 0.0;
  double dy = ny > 1 ? ((d + h) - y0) / (double)(ny - 1) : 0.0;
  for (int64_t l = 0; l < ny; ++l)
    for (int64_t k = 0; k < nx; ++k) zout[k + l * nx] = oz_make(x0 + (double)k * dx, y0 + (double)l * dy);
  box[0] = x0; box[1] = b + h; box[2] = y0; box[3] = d + h;
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
