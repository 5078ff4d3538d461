/*
 * CPU FP64 oracle for CholeskyQR-family QR factorisations of tall-and-skinny
 * matrices (Mijic, Kaushik, Davidovic, "QR factorization of ill-conditioned
 * tall-and-skinny matrices on distributed-memory systems", arXiv 2405.04237).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Conventions
 *   - FP64 throughout, column-major storage, leading dimensions >= rows.
 *   - Compiled with -O2 -ffp-contract=off (no fused multiply-add, no fast
 *     math), so every sum below is evaluated exactly in the order written.
 *   - OpenMP threads split rows only.  Every reduction over rows is done in
 *     fixed blocks of `g_block_rows` rows (ascending row order inside a block)
 *     whose partial results are added in ascending block order, so results do
 *     not depend on the thread count.
 *   - Status: 0 = success; j+1 (> 0) = the Cholesky factorisation broke down
 *     at global column j (LAPACK potrf style); negative = bad argument.
 *
 * Function -> paper map
 *   or_gram        Alg. 1 step 1, Alg. 6 step 2 (syrk semantics, Table 1 caption)
 *   or_chol        Alg. 1 step 2 (W = R^T R, R upper with positive diagonal)
 *   or_trsm        Alg. 1 step 3 (Q = A R^{-1} by forward substitution)
 *   or_cqr         Alg. 1 / Alg. 2 (CholeskyQR)
 *   or_cqr2        Alg. 3 (CholeskyQR2)
 *   or_cqrgs       Alg. 6 (CholeskyQR with block Gram-Schmidt)
 *   or_cqr2gs      Alg. 7 (CholeskyQR2 with Gram-Schmidt)
 *   or_mcqr2gs     Alg. 9 (modified CholeskyQR2 with Gram-Schmidt)
 *   or_mcqr2gs_halving  Alg. 9 with the adaptive panel width after a
 *                  rejected panel (Sec. 5.3-5.4, Eq. cond_bounds; the
 *                  rule is a reading, see the function)
 *   or_scqr        Alg. 4 (shifted CholeskyQR)
 *   or_scqr3       Alg. 5 (shifted CholeskyQR3)
 *   or_backward    adjoint of A = QR (not in the paper; the standard reverse-
 *                  mode rule M = R Rbar^T - Qbar^T Q,
 *                  Abar = (Qbar + Q copyltu(M)) R^{-T})
 *   or_householder textbook Householder QR, used only to pin the others
 *
 * Pins (tests/test_oracle_pins.py, tests/test_oracle_mutations.py): every
 * function above is fixed by something other than itself -- exact dyadic
 * QR, Householder/LAPACK by brute force, closed forms (including sCQR on
 * orthonormal columns), the paper's reductions and stability claims, finite
 * differences and torch autograd for the adjoint.  No function is parity
 * unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <float.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef int64_t i64;

#define AT(X, ld, r, c) ((X)[(i64)(r) + (i64)(c) * (i64)(ld)])

static i64 g_block_rows = 4096;

/* Row-block size of every fixed-order reduction over rows (default 4096).
 * Changing it changes only the rounding order; it exists so that tests can
 * measure the rounding floor between two valid summation orders. */
void or_set_block_rows(i64 rows) { g_block_rows = rows > 0 ? rows : 4096; }
i64 or_get_block_rows(void) { return g_block_rows; }

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* C (p x q) = X^T Y over all m rows, X m x p, Y m x q.  When `upper_only`,
 * X == Y and only entries a <= c are formed, then mirrored (syrk semantics).
 * Each entry is a sum over rows taken in ascending order inside fixed row
 * blocks, block partials added in ascending block order. */
static void tn_product(i64 m, i64 p, i64 q, const double* X, i64 ldx, const double* Y, i64 ldy,
                       double* C, i64 ldc, int upper_only) {
  const i64 blk = g_block_rows;
  const i64 nblk = (m + blk - 1) / blk;
  const i64 pq = p * q;
  int nt = or_num_threads();
  i64 group = (i64)nt * 2;
  if (group < 1) group = 1;
  double* part = (double*)calloc((size_t)(group * pq), sizeof(double));
  for (i64 a = 0; a < p; ++a)
    for (i64 c = 0; c < q; ++c) AT(C, ldc, a, c) = 0.0;
  for (i64 g0 = 0; g0 < nblk; g0 += group) {
    i64 gn = nblk - g0 < group ? nblk - g0 : group;
#pragma omp parallel for schedule(static)
    for (i64 t = 0; t < gn; ++t) {
      i64 r0 = (g0 + t) * blk;
      i64 r1 = r0 + blk < m ? r0 + blk : m;
      double* P = part + t * pq;
      for (i64 a = 0; a < p; ++a) {
        const double* xa = X + a * ldx;
        for (i64 c = upper_only ? a : 0; c < q; ++c) {
          const double* yc = Y + c * ldy;
          double s = 0.0;
          for (i64 r = r0; r < r1; ++r) s += xa[r] * yc[r];
          P[a + c * p] = s;
        }
      }
    }
    /* ascending block order */
    for (i64 t = 0; t < gn; ++t) {
      const double* P = part + t * pq;
      for (i64 a = 0; a < p; ++a)
        for (i64 c = upper_only ? a : 0; c < q; ++c) AT(C, ldc, a, c) += P[a + c * p];
    }
  }
  free(part);
  if (upper_only)
    for (i64 a = 0; a < p; ++a)
      for (i64 c = a + 1; c < q; ++c) AT(C, ldc, c, a) = AT(C, ldc, a, c);
}

/* Alg. 1 step 1: W := X^T X for the m x b matrix X (b x b, symmetric). */
void or_gram(i64 m, i64 b, const double* X, i64 ldx, double* W, i64 ldw) {
  tn_product(m, b, b, X, ldx, X, ldx, W, ldw, 1);
}

/* Y := X^T Z (p x q), the projection of Alg. 6 step 6 / Alg. 9 step 3. */
void or_tn(i64 m, i64 p, i64 q, const double* X, i64 ldx, const double* Z, i64 ldz, double* Y, i64 ldy) {
  tn_product(m, p, q, X, ldx, Z, ldz, Y, ldy, 0);
}

/* Alg. 1 step 2: upper U with U^T U = W, computed row by row:
 *   U_jj = sqrt(W_jj - sum_{i<j} U_ij^2),
 *   U_jc = (W_jc - sum_{i<j} U_ij U_ic) / U_jj,  c > j.
 * No pivoting, no shift.  A radicand that is not > 0 (this includes NaN)
 * is a breakdown: returns j+1 and leaves the rest of U untouched.  The strict
 * lower triangle of U is set to zero. */
int or_chol(i64 b, const double* W, i64 ldw, double* U, i64 ldu) {
  for (i64 c = 0; c < b; ++c)
    for (i64 r = 0; r < b; ++r) AT(U, ldu, r, c) = 0.0;
  for (i64 j = 0; j < b; ++j) {
    double s = AT(W, ldw, j, j);
    for (i64 i = 0; i < j; ++i) s -= AT(U, ldu, i, j) * AT(U, ldu, i, j);
    if (!(s > 0.0) || !isfinite(s)) return (int)(j + 1);
    double d = sqrt(s);
    AT(U, ldu, j, j) = d;
    for (i64 c = j + 1; c < b; ++c) {
      double t = AT(W, ldw, j, c);
      for (i64 i = 0; i < j; ++i) t -= AT(U, ldu, i, j) * AT(U, ldu, i, c);
      AT(U, ldu, j, c) = t / d;
    }
  }
  return 0;
}

/* Alg. 1 step 3: X := X U^{-1} (U upper, b x b) by forward substitution on
 * each row x:  q_c = (x_c - sum_{i<c} q_i U_ic) / U_cc.  Never forms U^{-1}.
 * Rows are independent; they are processed column by column for locality,
 * which leaves each element's operation order exactly as written above. */
void or_trsm(i64 m, i64 b, double* X, i64 ldx, const double* U, i64 ldu) {
  const i64 blk = 512;
  const i64 nblk = (m + blk - 1) / blk;
#pragma omp parallel for schedule(static)
  for (i64 t = 0; t < nblk; ++t) {
    i64 r0 = t * blk, r1 = r0 + blk < m ? r0 + blk : m;
    double s[512];
    for (i64 c = 0; c < b; ++c) {
      double* xc = X + c * ldx;
      for (i64 r = r0; r < r1; ++r) s[r - r0] = xc[r];
      for (i64 i = 0; i < c; ++i) {
        const double* qi = X + i * ldx;
        double u = AT(U, ldu, i, c);
        for (i64 r = r0; r < r1; ++r) s[r - r0] -= qi[r] * u;
      }
      double d = AT(U, ldu, c, c);
      for (i64 r = r0; r < r1; ++r) xc[r] = s[r - r0] / d;
    }
  }
}

/* X (m x q) := X - Q Y with Q m x p, Y p x q (Alg. 6 step 7, Alg. 9 steps 4
 * and 7): each element is x - (sum_i q_i y_i), the sum in ascending i. */
void or_update(i64 m, i64 p, i64 q, double* X, i64 ldx, const double* Q, i64 ldq, const double* Y, i64 ldy) {
  const i64 blk = 512;
  const i64 nblk = (m + blk - 1) / blk;
#pragma omp parallel for schedule(static)
  for (i64 t = 0; t < nblk; ++t) {
    i64 r0 = t * blk, r1 = r0 + blk < m ? r0 + blk : m;
    double s[512];
    for (i64 c = 0; c < q; ++c) {
      for (i64 r = r0; r < r1; ++r) s[r - r0] = 0.0;
      for (i64 i = 0; i < p; ++i) {
        const double* qi = Q + i * ldq;
        double y = AT(Y, ldy, i, c);
        for (i64 r = r0; r < r1; ++r) s[r - r0] += qi[r] * y;
      }
      double* xc = X + c * ldx;
      for (i64 r = r0; r < r1; ++r) xc[r] = xc[r] - s[r - r0];
    }
  }
}

/* C (p x q) := A (p x t) * B (t x q), plain triple loop, ascending inner index.
 * Used for the small triangular products R = R2 R1 (Alg. 3 step 3, Alg. 7
 * step 3) and for Z S1.  `a_upper` / `b_upper` restrict the inner index to
 * the nonzero range of an upper-triangular factor (exact zeros skipped). */
static void small_mm(i64 p, i64 t, i64 q, const double* A, i64 lda, int a_upper, const double* B, i64 ldb,
                     int b_upper, double* C, i64 ldc) {
  for (i64 c = 0; c < q; ++c)
    for (i64 a = 0; a < p; ++a) {
      i64 lo = a_upper ? a : 0;
      i64 hi = b_upper ? (c + 1 < t ? c + 1 : t) : t;
      double s = 0.0;
      for (i64 i = lo; i < hi; ++i) s += AT(A, lda, a, i) * AT(B, ldb, i, c);
      AT(C, ldc, a, c) = s;
    }
}

static void zero_mat(i64 p, i64 q, double* C, i64 ldc) {
  for (i64 c = 0; c < q; ++c)
    for (i64 a = 0; a < p; ++a) AT(C, ldc, a, c) = 0.0;
}

/* Alg. 1 (CholeskyQR): W = X^T X; W = U^T U; X := X U^{-1}; R := U.
 * X (m x b) is overwritten by Q.  Returns 0 or the breakdown column + 1
 * (local to this b-wide block). */
int or_cqr(i64 m, i64 b, double* X, i64 ldx, double* R, i64 ldr) {
  double* W = (double*)malloc(sizeof(double) * (size_t)(b * b));
  or_gram(m, b, X, ldx, W, b);
  int st = or_chol(b, W, b, R, ldr);
  free(W);
  if (st) return st;
  or_trsm(m, b, X, ldx, R, ldr);
  return 0;
}

/* Alg. 4 (shifted CholeskyQR): G = X^T X; s = sqrt(m) u ||X||_F^2;
 * W = G + s I; W = U^T U; X := X U^{-1}.  u is the unit roundoff 2^-53.
 * ||X||_F^2 is the trace of G (the sum of squares of X's elements). */
int or_scqr(i64 m, i64 b, double* X, i64 ldx, double* R, i64 ldr) {
  double* W = (double*)malloc(sizeof(double) * (size_t)(b * b));
  or_gram(m, b, X, ldx, W, b);
  double fro2 = 0.0;
  for (i64 j = 0; j < b; ++j) fro2 += W[j + j * b];
  double s = sqrt((double)m) * ldexp(1.0, -53) * fro2;
  for (i64 j = 0; j < b; ++j) W[j + j * b] += s;
  int st = or_chol(b, W, b, R, ldr);
  free(W);
  if (st) return st;
  or_trsm(m, b, X, ldx, R, ldr);
  return 0;
}

/* Alg. 3 (CholeskyQR2): [Q1,R1] = CQR(X); [Q,R2] = CQR(Q1); R = R2 R1. */
int or_cqr2(i64 m, i64 n, double* X, i64 ldx, double* R, i64 ldr) {
  double* R1 = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* R2 = (double*)malloc(sizeof(double) * (size_t)(n * n));
  int st = or_cqr(m, n, X, ldx, R1, n);
  if (!st) st = or_cqr(m, n, X, ldx, R2, n);
  if (!st) small_mm(n, n, n, R2, n, 1, R1, n, 1, R, ldr);
  free(R1);
  free(R2);
  return st;
}

/* Alg. 5 (shifted CholeskyQR3): [Q1,R1] = sCQR(X); [Q,R2] = CQR2(Q1); R = R2 R1. */
int or_scqr3(i64 m, i64 n, double* X, i64 ldx, double* R, i64 ldr) {
  double* R1 = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* R2 = (double*)malloc(sizeof(double) * (size_t)(n * n));
  int st = or_scqr(m, n, X, ldx, R1, n);
  if (!st) st = or_cqr2(m, n, X, ldx, R2, n);
  if (!st) small_mm(n, n, n, R2, n, 1, R1, n, 1, R, ldr);
  free(R1);
  free(R2);
  return st;
}

/* Alg. 6 (CholeskyQR with block Gram-Schmidt), panels of width b, k = n/b:
 *   for j = 1..k:
 *     W_j = A_j^T A_j; W_j = U^T U; Q_j = A_j U^{-1}; R_jj = U
 *     Y = Q_j^T A_{j+1:k}; A_{j+1:k} -= Q_j Y; R_{j,j+1:k} = Y
 * X (m x n) is overwritten by Q; R (n x n) gets its upper triangle, and its
 * strict lower triangle is zeroed. */
int or_cqrgs(i64 m, i64 n, i64 b, double* X, i64 ldx, double* R, i64 ldr) {
  if (b <= 0 || n % b) return -3;
  zero_mat(n, n, R, ldr);
  i64 k = n / b;
  for (i64 j = 0; j < k; ++j) {
    double* Aj = X + j * b * ldx;
    int st = or_cqr(m, b, Aj, ldx, &AT(R, ldr, j * b, j * b), ldr);
    if (st) return (int)(j * b) + st;
    i64 w = n - (j + 1) * b;
    if (w > 0) {
      double* Ar = X + (j + 1) * b * ldx;
      double* Yp = &AT(R, ldr, j * b, (j + 1) * b); /* Y lands straight in R_{j,j+1:k} */
      or_tn(m, b, w, Aj, ldx, Ar, ldx, Yp, ldr);
      or_update(m, b, w, Ar, ldx, Aj, ldx, Yp, ldr);
    }
  }
  return 0;
}

/* Alg. 7 (CholeskyQR2 with Gram-Schmidt):
 *   [Q1,R1] = CQRGS(A); [Q,R2] = CQRGS(Q1); R = R2 R1. */
int or_cqr2gs(i64 m, i64 n, i64 b, double* X, i64 ldx, double* R, i64 ldr) {
  if (b <= 0 || n % b) return -3;
  double* R1 = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* R2 = (double*)malloc(sizeof(double) * (size_t)(n * n));
  int st = or_cqrgs(m, n, b, X, ldx, R1, n);
  if (!st) st = or_cqrgs(m, n, b, X, ldx, R2, n);
  if (!st) {
    small_mm(n, n, n, R2, n, 1, R1, n, 1, R, ldr);
    for (i64 c = 0; c < n; ++c)
      for (i64 r = c + 1; r < n; ++r) AT(R, ldr, r, c) = 0.0;
  }
  free(R1);
  free(R2);
  return st;
}

#define OR_FLAG_LITERAL_R 1 /* R_jj = S2 S1 only; drop the R_{1:j-1,j} += Z S1 term */
#define OR_FLAG_ADAPTIVE 2  /* runtime choice of the second CholeskyQR pass (Sec. 7), see below */

/* Runtime choice of CholeskyQR repetitions (the future work of Sec. 7).
 * The second pass of a panel (Alg. 3 step 2 for the first panel, Alg. 9
 * step 8 for the others) forms W = P^T P and its Cholesky factor S2.  When
 * every entry of S2 - I is within 8u, P is already orthonormal to working
 * precision: S2 is replaced by I exactly and the triangular solve, which
 * would then leave P unchanged, is not performed.  Returns 1 when skipped. */
static int adaptive_second_pass(i64 m, i64 b, double* X, i64 ldx, double* S, i64 lds, int* st) {
  double* W = (double*)malloc(sizeof(double) * (size_t)(b * b));
  or_gram(m, b, X, ldx, W, b);
  *st = or_chol(b, W, b, S, lds);
  free(W);
  if (*st) return 0;
  const double tau = 8.0 * ldexp(1.0, -53);
  int near_identity = 1;
  for (i64 c = 0; c < b && near_identity; ++c)
    for (i64 r = 0; r <= c; ++r) {
      double d = AT(S, lds, r, c) - (r == c ? 1.0 : 0.0);
      if (!(fabs(d) <= tau)) { near_identity = 0; break; }
    }
  if (near_identity) {
    for (i64 c = 0; c < b; ++c)
      for (i64 r = 0; r < b; ++r) AT(S, lds, r, c) = (r == c) ? 1.0 : 0.0;
    return 1;
  }
  or_trsm(m, b, X, ldx, S, lds);
  return 0;
}

/* Alg. 9 (modified CholeskyQR2 with Gram-Schmidt), panels of width b, k = n/b:
 *   [Q_1, R_11] = CQR2(A_1)
 *   for j = 2..k:
 *     Y = Q_{j-1}^T A_{j:k};  A_{j:k} -= Q_{j-1} Y;  R_{j-1,j:k} = Y
 *     [P, S1] = CQR(A_j)                      (the panel is replaced by P)
 *     Z = Q_{1:j-1}^T P;  P -= Q_{1:j-1} Z     (one block classical GS step)
 *     [Q_j, S2] = CQR(P)
 *     R_jj = S2 S1;  R_{1:j-1,j} += Z S1
 * The algorithm leaves the R of steps 6-8 implicit; the two R assignments on
 * the last line are the reading under which A = Q R holds exactly in exact
 * arithmetic (A_j's projected part is (Q_{1:j-1} Z + Q_j S2) S1).
 * flags & OR_FLAG_LITERAL_R drops the Z S1 term (kept for measurement). */
int or_mcqr2gs(i64 m, i64 n, i64 b, double* X, i64 ldx, double* R, i64 ldr, int flags) {
  if (b <= 0 || n % b) return -3;
  zero_mat(n, n, R, ldr);
  i64 k = n / b;
  double* S1 = (double*)malloc(sizeof(double) * (size_t)(b * b));
  double* S2 = (double*)malloc(sizeof(double) * (size_t)(b * b));
  double* Z = (double*)malloc(sizeof(double) * (size_t)(n * b));
  double* ZS = (double*)malloc(sizeof(double) * (size_t)(n * b));
  int st;
  if (flags & OR_FLAG_ADAPTIVE) {
    /* first panel: CQR, then the adaptive second pass; R_11 = S2 S1 */
    st = or_cqr(m, b, X, ldx, S1, b);
    if (!st) {
      adaptive_second_pass(m, b, X, ldx, S2, b, &st);
      if (!st) small_mm(b, b, b, S2, b, 1, S1, b, 1, R, ldr);
    }
  } else {
    st = or_cqr2(m, b, X, ldx, R, ldr);
  }
  for (i64 j = 1; j < k && !st; ++j) {
    double* Qprev = X + (j - 1) * b * ldx;
    double* Aj = X + j * b * ldx;
    i64 w = n - j * b;
    double* Yp = &AT(R, ldr, (j - 1) * b, j * b);
    or_tn(m, b, w, Qprev, ldx, Aj, ldx, Yp, ldr);
    or_update(m, b, w, Aj, ldx, Qprev, ldx, Yp, ldr);
    st = or_cqr(m, b, Aj, ldx, S1, b);
    if (st) { st += (int)(j * b); break; }
    i64 jb = j * b;
    or_tn(m, jb, b, X, ldx, Aj, ldx, Z, jb);
    or_update(m, jb, b, Aj, ldx, X, ldx, Z, jb);
    if (flags & OR_FLAG_ADAPTIVE)
      adaptive_second_pass(m, b, Aj, ldx, S2, b, &st);
    else
      st = or_cqr(m, b, Aj, ldx, S2, b);
    if (st) { st += (int)(j * b); break; }
    small_mm(b, b, b, S2, b, 1, S1, b, 1, &AT(R, ldr, jb, jb), ldr);
    if (!(flags & OR_FLAG_LITERAL_R)) {
      small_mm(jb, b, b, Z, jb, 0, S1, b, 1, ZS, jb);
      for (i64 c = 0; c < b; ++c)
        for (i64 a = 0; a < jb; ++a) AT(R, ldr, a, jb + c) += ZS[a + c * jb];
    }
  }
  free(S1);
  free(S2);
  free(Z);
  free(ZS);
  return st;
}

/* Adaptive panel width (the paper's remedy for a Cholesky breakdown is a
 * smaller b, Sec. 5.3-5.4 and Eq. cond_bounds; the rule itself is this
 * library's reading).  Alg. 9 with panels whose width may shrink: the first
 * CholeskyQR of every panel (Alg. 9 step 1 for panel 1, step 6 for the
 * others) forms W = A_j^T A_j and its Cholesky factor U, and the panel is
 * REJECTED when the factorisation breaks down or when
 * (max_i U_ii / min_i U_ii)^2 > 1/(64 u), i.e. when the panel's Gram matrix
 * is within a factor 64 of numerical singularity.  A rejected panel is left
 * untouched (no triangular solve); b becomes the largest proper divisor of
 * b that is <= b/2 (so it still divides the remaining width) and the step is
 * retried on the narrower panel; every later panel keeps the new width.  A
 * one-column panel is never rejected by the ratio test; its breakdown is
 * reported as usual.  Projections use the width of the panel they project
 * on (Alg. 9 step 3 with Q_{j-1} of its own width).  With no rejection this
 * performs exactly the operations of or_mcqr2gs.  *b_final receives the
 * width of the last panel.  Returns 0 or the breakdown column + 1. */
static i64 halved_width(i64 b) {
  for (i64 d = b / 2; d > 1; --d)
    if (b % d == 0) return d;
  return 1;
}

static int reject_panel(i64 b, const double* U, i64 ldu, int chol_status) {
  if (b <= 1) return 0;
  if (chol_status) return 1;
  double dmax = AT(U, ldu, 0, 0), dmin = AT(U, ldu, 0, 0);
  for (i64 i = 1; i < b; ++i) {
    double d = AT(U, ldu, i, i);
    if (d > dmax) dmax = d;
    if (d < dmin) dmin = d;
  }
  return dmax * dmax * 64.0 * ldexp(1.0, -53) > dmin * dmin;
}

int or_mcqr2gs_halving(i64 m, i64 n, i64 b, double* X, i64 ldx, double* R, i64 ldr, i64* b_final) {
  if (b <= 0 || n % b) return -3;
  zero_mat(n, n, R, ldr);
  double* W = (double*)malloc(sizeof(double) * (size_t)(b * b));
  double* S1 = (double*)malloc(sizeof(double) * (size_t)(b * b));
  double* S2 = (double*)malloc(sizeof(double) * (size_t)(b * b));
  double* Z = (double*)malloc(sizeof(double) * (size_t)(n * b));
  double* ZS = (double*)malloc(sizeof(double) * (size_t)(n * b));
  i64 bw = b, bprev = 0, c0 = 0;
  int st = 0;
  while (c0 < n && !st) {
    double* Aj = X + c0 * ldx;
    if (c0 > 0) {
      /* steps 3-5: Y = Q_{j-1}^T A_{j:k}; A_{j:k} -= Q_{j-1} Y; R_{j-1,j:k} = Y */
      double* Qprev = X + (c0 - bprev) * ldx;
      double* Yp = &AT(R, ldr, c0 - bprev, c0);
      or_tn(m, bprev, n - c0, Qprev, ldx, Aj, ldx, Yp, ldr);
      or_update(m, bprev, n - c0, Aj, ldx, Qprev, ldx, Yp, ldr);
    }
    /* step 1 (first pass) / step 6: the first CholeskyQR, with the panel test */
    for (;;) {
      or_gram(m, bw, Aj, ldx, W, bw);
      st = or_chol(bw, W, bw, S1, bw);
      if (!reject_panel(bw, S1, bw, st)) break;
      bw = halved_width(bw);
    }
    if (st) { st += (int)c0; break; }
    or_trsm(m, bw, Aj, ldx, S1, bw);
    if (c0 > 0) {
      /* step 7: Z = Q_{1:j-1}^T P; P -= Q_{1:j-1} Z */
      or_tn(m, c0, bw, X, ldx, Aj, ldx, Z, c0);
      or_update(m, c0, bw, Aj, ldx, X, ldx, Z, c0);
    }
    /* step 1 (second pass) / step 8 */
    st = or_cqr(m, bw, Aj, ldx, S2, bw);
    if (st) { st += (int)c0; break; }
    /* R_jj = S2 S1;  R_{1:j-1,j} += Z S1 */
    small_mm(bw, bw, bw, S2, bw, 1, S1, bw, 1, &AT(R, ldr, c0, c0), ldr);
    if (c0 > 0) {
      small_mm(c0, bw, bw, Z, c0, 0, S1, bw, 1, ZS, c0);
      for (i64 c = 0; c < bw; ++c)
        for (i64 a = 0; a < c0; ++a) AT(R, ldr, a, c0 + c) += ZS[a + c * c0];
    }
    bprev = bw;
    c0 += bw;
  }
  if (b_final) *b_final = bw;
  free(W);
  free(S1);
  free(S2);
  free(Z);
  free(ZS);
  return st;
}

/* Reverse-mode adjoint of A = Q R (m >= n, R upper, invertible):
 *   M = R Rbar^T - Qbar^T Q                    (n x n)
 *   copyltu(M) = tril(M) + tril(M,-1)^T        (symmetric, from M's lower part)
 *   B = Qbar + Q copyltu(M)                    (m x n)
 *   Abar R^T = B, solved row by row by substitution against R^T (lower):
 *     abar_c = (b_c - sum_{i>c} abar_i R_ci) / R_cc, c = n-1 .. 0. */
void or_backward(i64 m, i64 n, const double* Q, i64 ldq, const double* R, i64 ldr, const double* dQ, i64 lddq,
                 const double* dR, i64 lddr, double* dA, i64 ldda) {
  double* M = (double*)malloc(sizeof(double) * (size_t)(n * n));
  double* G = (double*)malloc(sizeof(double) * (size_t)(n * n));
  or_tn(m, n, n, dQ, lddq, Q, ldq, G, n); /* G = Qbar^T Q */
  for (i64 c = 0; c < n; ++c)
    for (i64 a = 0; a < n; ++a) {
      /* (R Rbar^T)_{ac} = sum_i R_ai Rbar_ci, with R upper: i >= a */
      double s = 0.0;
      for (i64 i = a; i < n; ++i) s += AT(R, ldr, a, i) * AT(dR, lddr, c, i);
      M[a + c * n] = s - G[a + c * n];
    }
  /* copyltu */
  for (i64 c = 0; c < n; ++c)
    for (i64 a = 0; a < c; ++a) M[a + c * n] = M[c + a * n];
  /* B = Qbar + Q M, written into dA */
  for (i64 c = 0; c < n; ++c)
    for (i64 r = 0; r < m; ++r) AT(dA, ldda, r, c) = AT(dQ, lddq, r, c);
  double* negM = G;
  for (i64 i = 0; i < n * n; ++i) negM[i] = -M[i];
  or_update(m, n, n, dA, ldda, Q, ldq, negM, n); /* dA = dQ - Q (-M) */
  /* dA := B R^{-T} */
  const i64 blk = 512;
  const i64 nblk = (m + blk - 1) / blk;
#pragma omp parallel for schedule(static)
  for (i64 t = 0; t < nblk; ++t) {
    i64 r0 = t * blk, r1 = r0 + blk < m ? r0 + blk : m;
    double s[512];
    for (i64 c = n - 1; c >= 0; --c) {
      double* xc = dA + c * ldda;
      for (i64 r = r0; r < r1; ++r) s[r - r0] = xc[r];
      for (i64 i = c + 1; i < n; ++i) {
        const double* ai = dA + i * ldda;
        double u = AT(R, ldr, c, i);
        for (i64 r = r0; r < r1; ++r) s[r - r0] -= ai[r] * u;
      }
      double d = AT(R, ldr, c, c);
      for (i64 r = r0; r < r1; ++r) xc[r] = s[r - r0] / d;
    }
  }
  free(M);
  free(G);
}

/* Textbook Householder QR (Golub & Van Loan, Alg. 5.2.1) of A (m x n, m >= n),
 * giving the thin Q (m x n) and R (n x n), then sign-normalised so that
 * diag(R) >= 0.  Serial; for pinning the other routines on small inputs. */
void or_householder(i64 m, i64 n, const double* A, i64 lda, double* Q, i64 ldq, double* R, i64 ldr) {
  double* H = (double*)malloc(sizeof(double) * (size_t)(m * n));
  double* beta = (double*)malloc(sizeof(double) * (size_t)n);
  for (i64 c = 0; c < n; ++c)
    for (i64 r = 0; r < m; ++r) H[r + c * m] = AT(A, lda, r, c);
  for (i64 j = 0; j < n; ++j) {
    /* v = x + sign(x_0) ||x|| e_0, beta = 2 / (v^T v) */
    double nrm = 0.0;
    for (i64 r = j; r < m; ++r) nrm += H[r + j * m] * H[r + j * m];
    nrm = sqrt(nrm);
    double x0 = H[j + j * m];
    double alpha = x0 >= 0.0 ? -nrm : nrm; /* H x = alpha e_0 */
    double v0 = x0 - alpha;
    double vtv = v0 * v0;
    for (i64 r = j + 1; r < m; ++r) vtv += H[r + j * m] * H[r + j * m];
    beta[j] = vtv > 0.0 ? 2.0 / vtv : 0.0;
    H[j + j * m] = v0; /* column j below the diagonal now holds v */
    for (i64 c = j + 1; c < n; ++c) {
      double s = 0.0;
      for (i64 r = j; r < m; ++r) s += H[r + j * m] * H[r + c * m];
      s *= beta[j];
      for (i64 r = j; r < m; ++r) H[r + c * m] -= s * H[r + j * m];
    }
    /* store R_jj = alpha separately in R; keep v in H */
    for (i64 c = 0; c < n; ++c) AT(R, ldr, j, c) = 0.0;
    AT(R, ldr, j, j) = alpha;
  }
  for (i64 c = 0; c < n; ++c)
    for (i64 r = 0; r < c; ++r) AT(R, ldr, r, c) = H[r + c * m];
  for (i64 c = 0; c < n; ++c)
    for (i64 r = c + 1; r < n; ++r) AT(R, ldr, r, c) = 0.0;
  /* Q = H_0 H_1 ... H_{n-1} [I; 0], applied right to left */
  for (i64 c = 0; c < n; ++c)
    for (i64 r = 0; r < m; ++r) AT(Q, ldq, r, c) = (r == c) ? 1.0 : 0.0;
  for (i64 j = n - 1; j >= 0; --j) {
    for (i64 c = 0; c < n; ++c) {
      double s = 0.0;
      for (i64 r = j; r < m; ++r) s += H[r + j * m] * AT(Q, ldq, r, c);
      s *= beta[j];
      for (i64 r = j; r < m; ++r) AT(Q, ldq, r, c) -= s * H[r + j * m];
    }
  }
  /* sign normalisation: D = sign(diag R); R := D R; Q := Q D */
  for (i64 j = 0; j < n; ++j) {
    if (AT(R, ldr, j, j) < 0.0) {
      for (i64 c = j; c < n; ++c) AT(R, ldr, j, c) = -AT(R, ldr, j, c);
      for (i64 r = 0; r < m; ++r) AT(Q, ldq, r, j) = -AT(Q, ldq, r, j);
    }
  }
  free(H);
  free(beta);
}
