/*
 * ca_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the primal and dual block coordinate
 * descent methods for ridge regression from "Avoiding communication in primal
 * and dual block coordinate descent methods" (Devarakonda, Fountoulakis,
 * Demmel, Mahoney; arXiv 1612.04003):
 *
 *   BCD      -- Algorithm 1 (Sec. 3.1, eqs. for Delta w_h and z_h)
 *   CA-BCD   -- Algorithm 2 (Sec. 3.1, unrolled recurrence eq. "recur")
 *   BDCD     -- Algorithm 3 (Sec. 3.2, eqs. "alp", "op2", "wup", "ah")
 *   CA-BDCD  -- Algorithm 4 (Sec. 3.2, the unrolled dual recurrence)
 *
 * plus the closed-form ridge solution (normal equations of eq. "primal"),
 * the primal objective f (eq. "primal", Sec. 2.2) and the dual objective D
 * (eq. "6", Sec. 2.2).
 *
 * Only the test suite, the package smoke check and the benchmark's CPU
 * baseline leg may load this file.  It shares no code with the CUDA library;
 * the two agree only through the sampling rule stated below, which each side
 * implements on its own.
 *
 * Every loop follows the paper's formulas in the paper's order.  Nothing is
 * blocked, fused or reordered beyond what the formulas state.  Compile with
 * -ffp-contract=off so that x86 and Arm hosts round identically.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *  R1  Gamma_h = (1/n) I^T X X^T I + lambda I^T I   (Alg. 1 prints the braces
 *      garbled; Sec. 3.1 gives this form).  I^T I = I_b since a block holds
 *      no repeated index.  Theta_h likewise (Alg. 3 / Sec. 3.2).
 *  R2  The CA outer loop runs k = 0 .. ceil(H/s)-1; when s does not divide H
 *      the last outer step has s' = H - s*k inner steps.
 *  R3  Sampling (Alg. 1-4 "uniformly at random without replacement", the RNG
 *      is unspecified): block h draws b distinct indices of [0,N) with
 *      Floyd's algorithm, fed by Philox4x64-10 (Salmon et al., SC'11) with
 *      key (seed, 0) and counter (h, m/4, 0, 0), word m%4 for draw m; the
 *      64-bit word u maps to [0, J] as floor(u*(J+1)/2^64).  Block h is the
 *      global 0-based inner-iteration index, so CA (any s) and s = 1 draw the
 *      same indices.
 *  R4  w0 and alpha0 are inputs (Alg. 1-4 give no values); the dual
 *      initialises w0 = -X alpha0/(lambda n) as Algs. 3-4 state.
 *  R5  Periodic recomputation (not in the paper): every `recompute_every`
 *      outer steps the auxiliary vector is rebuilt from its definition,
 *      z = X^T w (Sec. 3.1) or w = -X alpha/(lambda n) (eq. "3").  A no-op in
 *      exact arithmetic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_NOT_SPD -3
#define ORC_ERR_OOM -6

/* ------------------------------------------------------------------------- */
/* Sampling rule R3: Philox4x64-10 counter-based generator.                  */
/* Round function and key schedule as published by Salmon, Moraes, Dror and  */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).              */
/* ------------------------------------------------------------------------- */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL;

static void mul_hi_lo(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2],
                       uint64_t out[4]) {
  uint64_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    uint64_t hi0, lo0, hi1, lo1;
    mul_hi_lo(PHILOX_M0, c[0], &hi0, &lo0);
    mul_hi_lo(PHILOX_M1, c[2], &hi1, &lo1);
    uint64_t n0 = hi1 ^ c[1] ^ k0;
    uint64_t n1 = lo1;
    uint64_t n2 = hi0 ^ c[3] ^ k1;
    uint64_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* floor(u * (J+1) / 2^64): a 64-bit word mapped onto [0, J]. */
uint64_t orc_map_to_range(uint64_t u, uint64_t J) {
  unsigned __int128 p = (unsigned __int128)u * (unsigned __int128)(J + 1);
  return (uint64_t)(p >> 64);
}

/* The 64-bit word used for draw m of block h. */
static uint64_t sample_word(uint64_t seed, int64_t h, int m) {
  uint64_t ctr[4] = {(uint64_t)h, (uint64_t)(m / 4), 0, 0};
  uint64_t key[2] = {seed, 0};
  uint64_t out[4];
  orc_philox4x64_10(ctr, key, out);
  return out[m % 4];
}

/* Floyd's algorithm: b distinct indices of [0, N), in insertion order. */
int orc_sample_block(uint64_t seed, int64_t h, int b, int64_t N, int32_t *idx) {
  if (b < 1 || N < 1 || b > N || N > 2147483647LL) return ORC_ERR_ARG;
  for (int m = 0; m < b; ++m) {
    int64_t J = N - b + m;
    int64_t t = (int64_t)orc_map_to_range(sample_word(seed, h, m), (uint64_t)J);
    int seen = 0;
    for (int q = 0; q < m; ++q)
      if (idx[q] == t) { seen = 1; break; }
    idx[m] = (int32_t)(seen ? J : t);
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Dense FP64 helpers (plain loops).                                          */
/* ------------------------------------------------------------------------- */
static double dot(const double *a, const double *b, int64_t len) {
  double acc = 0.0;
  for (int64_t i = 0; i < len; ++i) acc += a[i] * b[i];
  return acc;
}

/* Solve A x = r for a symmetric positive definite m x m matrix A (row-major)
 * by the Cholesky factorisation A = L L^T, then L u = r and L^T x = u.
 * A is not modified.  Returns ORC_ERR_NOT_SPD on a non-positive pivot. */
int orc_cholesky_solve(int m, const double *A, const double *r, double *x) {
  double *L = (double *)calloc((size_t)m * m, sizeof(double));
  double *u = (double *)malloc((size_t)m * sizeof(double));
  if (!L || !u) { free(L); free(u); return ORC_ERR_OOM; }
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j <= i; ++j) {
      double sum = A[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) sum -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      if (i == j) {
        if (!(sum > 0.0)) { free(L); free(u); return ORC_ERR_NOT_SPD; }
        L[(size_t)i * m + i] = sqrt(sum);
      } else {
        L[(size_t)i * m + j] = sum / L[(size_t)j * m + j];
      }
    }
  }
  for (int i = 0; i < m; ++i) {
    double sum = r[i];
    for (int k = 0; k < i; ++k) sum -= L[(size_t)i * m + k] * u[k];
    u[i] = sum / L[(size_t)i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double sum = u[i];
    for (int k = i + 1; k < m; ++k) sum -= L[(size_t)k * m + i] * x[k];
    x[i] = sum / L[(size_t)i * m + i];
  }
  free(L);
  free(u);
  return ORC_OK;
}

/* z = X^T w for X d x n row-major (Sec. 3.1, auxiliary variable z_h). */
static void primal_z(const double *X, int64_t d, int64_t n, const double *w, double *z) {
  for (int64_t i = 0; i < n; ++i) z[i] = 0.0;
  for (int64_t f = 0; f < d; ++f) {
    const double *row = X + (size_t)f * n;
    for (int64_t i = 0; i < n; ++i) z[i] += row[i] * w[f];
  }
}

/* f(w) = lambda/2 ||w||^2 + 1/(2n) ||X^T w - y||^2  (eq. "primal"). */
double orc_primal_objective(const double *X, int64_t d, int64_t n, const double *y,
                            double lam, const double *w) {
  double *z = (double *)malloc((size_t)n * sizeof(double));
  if (!z) return NAN;
  primal_z(X, d, n, w, z);
  double res = 0.0;
  for (int64_t i = 0; i < n; ++i) res += (z[i] - y[i]) * (z[i] - y[i]);
  double ww = dot(w, w, d);
  free(z);
  return 0.5 * lam * ww + res / (2.0 * (double)n);
}

/* Closed-form ridge solution: the gradient of eq. "primal" vanishes at
 * (X X^T / n + lambda I) w* = X y / n.  Solved by Cholesky. */
int orc_closed_form(const double *X, int64_t d, int64_t n, const double *y, double lam,
                    double *w_star) {
  double *A = (double *)malloc((size_t)d * d * sizeof(double));
  double *r = (double *)malloc((size_t)d * sizeof(double));
  if (!A || !r) { free(A); free(r); return ORC_ERR_OOM; }
  for (int64_t i = 0; i < d; ++i) {
    for (int64_t j = 0; j < d; ++j)
      A[(size_t)i * d + j] = dot(X + (size_t)i * n, X + (size_t)j * n, n) / (double)n;
    A[(size_t)i * d + i] += lam;
    r[i] = dot(X + (size_t)i * n, y, n) / (double)n;
  }
  int st = orc_cholesky_solve((int)d, A, r, w_star);
  free(A);
  free(r);
  return st;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 (BCD) and Algorithm 2 (CA-BCD), X dense d x n row-major.       */
/* ------------------------------------------------------------------------- */

/* Algorithm 2.  With s = 1 it performs exactly the steps of Algorithm 1:
 * Gamma_h, Delta w_h (eq. "primres"), w_h (eq. "wupdate"), z_h (eq.
 * "primah").  w is w0 on entry and w_H on return; z_out (may be NULL)
 * receives X^T w_H computed from its definition. */
int orc_cabcd(const double *X, int64_t d, int64_t n, const double *y, double lam, int b,
              int s, int64_t H, uint64_t seed, int64_t h0, int recompute_every,
              double *w, double *z_out) {
  if (b < 1 || b > d || s < 1 || H < 1 || !(lam > 0.0)) return ORC_ERR_ARG;
  const double inv_n = 1.0 / (double)n;
  const int64_t sb_max = (int64_t)s * b;
  double *z = (double *)malloc((size_t)n * sizeof(double));
  int32_t *I = (int32_t *)malloc((size_t)sb_max * sizeof(int32_t));
  double *G = (double *)malloc((size_t)sb_max * sb_max * sizeof(double));
  double *Yz = (double *)malloc((size_t)sb_max * sizeof(double));
  double *Yy = (double *)malloc((size_t)sb_max * sizeof(double));
  double *dw = (double *)malloc((size_t)sb_max * sizeof(double));
  double *Gam = (double *)malloc((size_t)b * b * sizeof(double));
  double *rhs = (double *)malloc((size_t)b * sizeof(double));
  int st = ORC_OK;
  if (!z || !I || !G || !Yz || !Yy || !dw || !Gam || !rhs) { st = ORC_ERR_OOM; goto done; }

  /* z_0 = X^T w_0 */
  primal_z(X, d, n, w, z);

  const int64_t n_outer = (H + s - 1) / s; /* reading R2 */
  for (int64_t k = 0; k < n_outer; ++k) {
    const int sk = (int)((H - (int64_t)s * k) < s ? (H - (int64_t)s * k) : s);
    const int sb = sk * b;
    /* choose I_{sk+1} .. I_{sk+s'}: b distinct rows each (Alg. 2, inner loop 1) */
    for (int j = 0; j < sk; ++j) {
      st = orc_sample_block(seed, h0 + (int64_t)s * k + j, b, d, I + (size_t)j * b);
      if (st) goto done;
    }
    /* Y = [I_1..I_s']^T X ; G = (1/n) Y Y^T + lambda I ; also Y z_sk, Y y */
    for (int p = 0; p < sb; ++p) {
      const double *yp = X + (size_t)I[p] * n;
      for (int q = 0; q < sb; ++q) {
        const double *yq = X + (size_t)I[q] * n;
        G[(size_t)p * sb + q] = inv_n * dot(yp, yq, n) + (p == q ? lam : 0.0);
      }
      Yz[p] = dot(yp, z, n);
      Yy[p] = dot(yp, y, n);
    }
    /* inner loop: Delta w_{sk+j} from w_sk and z_sk by eq. "recur" */
    for (int j = 0; j < sk; ++j) {
      const int32_t *Ij = I + (size_t)j * b;
      for (int p = 0; p < b; ++p) {
        double r = -lam * w[Ij[p]];                       /* -lambda I_j^T w_sk */
        for (int t = 0; t < j; ++t) {                     /* -lambda sum I_j^T I_t dw_t */
          const int32_t *It = I + (size_t)t * b;
          for (int q = 0; q < b; ++q)
            if (Ij[p] == It[q]) r -= lam * dw[(size_t)t * b + q];
        }
        r -= inv_n * Yz[(size_t)j * b + p];               /* -(1/n) I_j^T X z_sk */
        for (int t = 0; t < j; ++t)                       /* -(1/n) sum I_j^T X X^T I_t dw_t */
          for (int q = 0; q < b; ++q)                     /* G's off-diagonal block = (1/n) Y_j Y_t^T */
            r -= G[(size_t)(j * b + p) * sb + (t * b + q)] * dw[(size_t)t * b + q];
        r += inv_n * Yy[(size_t)j * b + p];               /* +(1/n) I_j^T X y */
        rhs[p] = r;
      }
      /* Gamma_{sk+j}: the b x b diagonal block of G */
      for (int p = 0; p < b; ++p)
        for (int q = 0; q < b; ++q)
          Gam[(size_t)p * b + q] = G[(size_t)(j * b + p) * sb + (j * b + q)];
      st = orc_cholesky_solve(b, Gam, rhs, dw + (size_t)j * b);
      if (st) goto done;
    }
    /* deferred updates: w_{sk+s} = w_sk + sum I_t dw_t ;
     *                   z_{sk+s} = z_sk + X^T sum I_t dw_t */
    for (int p = 0; p < sb; ++p) w[I[p]] += dw[p];
    for (int p = 0; p < sb; ++p) {
      const double *yp = X + (size_t)I[p] * n;
      for (int64_t i = 0; i < n; ++i) z[i] += yp[i] * dw[p];
    }
    /* reading R5 */
    if (recompute_every > 0 && (k + 1) % recompute_every == 0) primal_z(X, d, n, w, z);
  }
  if (z_out) primal_z(X, d, n, w, z_out);
done:
  free(z); free(I); free(G); free(Yz); free(Yy); free(dw); free(Gam); free(rhs);
  return st;
}

/* Algorithm 1, written out on its own (one b x b subproblem per iteration)
 * so that the s-step equivalence of Sec. 3.1 can be checked against it. */
int orc_bcd(const double *X, int64_t d, int64_t n, const double *y, double lam, int b,
            int64_t H, uint64_t seed, int64_t h0, int recompute_every, double *w,
            double *z_out) {
  if (b < 1 || b > d || H < 1 || !(lam > 0.0)) return ORC_ERR_ARG;
  const double inv_n = 1.0 / (double)n;
  double *z = (double *)malloc((size_t)n * sizeof(double));
  int32_t *I = (int32_t *)malloc((size_t)b * sizeof(int32_t));
  double *Gam = (double *)malloc((size_t)b * b * sizeof(double));
  double *rhs = (double *)malloc((size_t)b * sizeof(double));
  double *dw = (double *)malloc((size_t)b * sizeof(double));
  int st = ORC_OK;
  if (!z || !I || !Gam || !rhs || !dw) { st = ORC_ERR_OOM; goto done; }
  primal_z(X, d, n, w, z);
  for (int64_t h = 0; h < H; ++h) {
    st = orc_sample_block(seed, h0 + h, b, d, I);
    if (st) goto done;
    /* Gamma_h = (1/n) I^T X X^T I + lambda I_b  (reading R1) */
    for (int p = 0; p < b; ++p)
      for (int q = 0; q < b; ++q)
        Gam[(size_t)p * b + q] = inv_n * dot(X + (size_t)I[p] * n, X + (size_t)I[q] * n, n) +
                                 (p == q ? lam : 0.0);
    /* rhs = -lambda I^T w - (1/n) I^T X z + (1/n) I^T X y */
    for (int p = 0; p < b; ++p) {
      const double *yp = X + (size_t)I[p] * n;
      rhs[p] = -lam * w[I[p]] - inv_n * dot(yp, z, n) + inv_n * dot(yp, y, n);
    }
    st = orc_cholesky_solve(b, Gam, rhs, dw);
    if (st) goto done;
    for (int p = 0; p < b; ++p) w[I[p]] += dw[p];                  /* w_h */
    for (int p = 0; p < b; ++p) {                                 /* z_h */
      const double *yp = X + (size_t)I[p] * n;
      for (int64_t i = 0; i < n; ++i) z[i] += yp[i] * dw[p];
    }
    if (recompute_every > 0 && (h + 1) % recompute_every == 0) primal_z(X, d, n, w, z);
  }
  if (z_out) primal_z(X, d, n, w, z_out);
done:
  free(z); free(I); free(Gam); free(rhs); free(dw);
  return st;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 3 (BDCD) and Algorithm 4 (CA-BDCD).                              */
/* X is given by its columns: CSR of X^T, i.e. row i of the CSR holds the     */
/* non-zeros of column x_i of X (a sample), as the paper's implementation     */
/* stores it (Sec. 5.2).  Dense inputs are passed with every entry stored.    */
/* ------------------------------------------------------------------------- */
typedef struct {
  const int64_t *rowptr; /* n+1 */
  const int32_t *col;    /* feature index of each non-zero */
  const double *val;
} csr_t;

/* x_i^T v for a dense d-vector v */
static double col_dot_dense(const csr_t *A, int64_t i, const double *v) {
  double acc = 0.0;
  for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) acc += A->val[e] * v[A->col[e]];
  return acc;
}

/* x_i^T x_j by scattering x_j into a dense scratch vector */
static double col_dot_col(const csr_t *A, int64_t i, int64_t j, double *scratch_d) {
  for (int64_t e = A->rowptr[j]; e < A->rowptr[j + 1]; ++e) scratch_d[A->col[e]] = A->val[e];
  double acc = col_dot_dense(A, i, scratch_d);
  for (int64_t e = A->rowptr[j]; e < A->rowptr[j + 1]; ++e) scratch_d[A->col[e]] = 0.0;
  return acc;
}

/* w = -(1/(lambda n)) X alpha  (eq. "3") */
static void dual_w(const csr_t *A, int64_t d, int64_t n, double lam, const double *alpha,
                   double *w) {
  for (int64_t f = 0; f < d; ++f) w[f] = 0.0;
  const double c = -1.0 / (lam * (double)n);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t e = A->rowptr[i]; e < A->rowptr[i + 1]; ++e) w[A->col[e]] += c * A->val[e] * alpha[i];
}

/* D(alpha) = lambda/2 ||X alpha/(lambda n)||^2 + 1/(2n) ||alpha + y||^2 (eq. "6") */
double orc_dual_objective(const int64_t *rowptr, const int32_t *col, const double *val,
                          int64_t d, int64_t n, const double *y, double lam,
                          const double *alpha) {
  csr_t A = {rowptr, col, val};
  double *w = (double *)malloc((size_t)d * sizeof(double));
  if (!w) return NAN;
  dual_w(&A, d, n, lam, alpha, w); /* w = -X alpha/(lambda n); ||w|| is the same */
  double ww = dot(w, w, d);
  double r = 0.0;
  for (int64_t i = 0; i < n; ++i) r += (alpha[i] + y[i]) * (alpha[i] + y[i]);
  free(w);
  return 0.5 * lam * ww + r / (2.0 * (double)n);
}

/* Algorithm 4.  With s = 1 it performs exactly the steps of Algorithm 3.
 * alpha is alpha0 on entry and alpha_H on return; w receives w_H. */
int orc_cabdcd(const int64_t *rowptr, const int32_t *col, const double *val, int64_t d,
               int64_t n, const double *y, double lam, int b, int s, int64_t H,
               uint64_t seed, int64_t h0, int recompute_every, double *alpha, double *w) {
  if (b < 1 || b > n || s < 1 || H < 1 || !(lam > 0.0)) return ORC_ERR_ARG;
  csr_t A = {rowptr, col, val};
  const double ln = lam * (double)n;
  const double inv_n = 1.0 / (double)n;
  const int64_t sb_max = (int64_t)s * b;
  int32_t *I = (int32_t *)malloc((size_t)sb_max * sizeof(int32_t));
  double *G = (double *)malloc((size_t)sb_max * sb_max * sizeof(double));
  double *Yw = (double *)malloc((size_t)sb_max * sizeof(double));
  double *da = (double *)malloc((size_t)sb_max * sizeof(double));
  double *Th = (double *)malloc((size_t)b * b * sizeof(double));
  double *rhs = (double *)malloc((size_t)b * sizeof(double));
  double *sol = (double *)malloc((size_t)b * sizeof(double));
  double *scratch = (double *)calloc((size_t)d, sizeof(double));
  int st = ORC_OK;
  if (!I || !G || !Yw || !da || !Th || !rhs || !sol || !scratch) { st = ORC_ERR_OOM; goto done; }

  /* Initialize: w_0 = -(1/(lambda n)) X alpha_0 */
  dual_w(&A, d, n, lam, alpha, w);

  const int64_t n_outer = (H + s - 1) / s; /* reading R2 */
  for (int64_t k = 0; k < n_outer; ++k) {
    const int sk = (int)((H - (int64_t)s * k) < s ? (H - (int64_t)s * k) : s);
    const int sb = sk * b;
    for (int j = 0; j < sk; ++j) {
      st = orc_sample_block(seed, h0 + (int64_t)s * k + j, b, n, I + (size_t)j * b);
      if (st) goto done;
    }
    /* Y = X [I_1..I_s'] ; G' = (1/(lambda n^2)) Y^T Y + (1/n) I ; Y^T w_sk */
    for (int p = 0; p < sb; ++p) {
      for (int q = 0; q < sb; ++q)
        G[(size_t)p * sb + q] = col_dot_col(&A, I[p], I[q], scratch) / (ln * (double)n) +
                                (p == q ? inv_n : 0.0);
      Yw[p] = col_dot_dense(&A, I[p], w);
    }
    for (int j = 0; j < sk; ++j) {
      const int32_t *Ij = I + (size_t)j * b;
      for (int p = 0; p < b; ++p) {
        double r = -Yw[(size_t)j * b + p];                /* -I_j^T X^T w_sk */
        for (int t = 0; t < j; ++t)                       /* +(1/(lambda n)) sum I_j^T X^T X I_t da_t */
          for (int q = 0; q < b; ++q) {
            /* the off-diagonal block of G' is (1/(lambda n^2)) Y_j^T Y_t,
             * so (1/(lambda n)) Y_j^T Y_t = n * G'_jt */
            r += (double)n * G[(size_t)(j * b + p) * sb + (t * b + q)] * da[(size_t)t * b + q];
          }
        r += alpha[Ij[p]];                                /* +I_j^T alpha_sk */
        for (int t = 0; t < j; ++t) {                     /* +sum I_j^T I_t da_t */
          const int32_t *It = I + (size_t)t * b;
          for (int q = 0; q < b; ++q)
            if (Ij[p] == It[q]) r += da[(size_t)t * b + q];
        }
        r += y[Ij[p]];                                    /* +I_j^T y */
        rhs[p] = r;
      }
      /* Theta_{sk+j}: the b x b diagonal block of G' */
      for (int p = 0; p < b; ++p)
        for (int q = 0; q < b; ++q)
          Th[(size_t)p * b + q] = G[(size_t)(j * b + p) * sb + (j * b + q)];
      st = orc_cholesky_solve(b, Th, rhs, sol);
      if (st) goto done;
      for (int p = 0; p < b; ++p) da[(size_t)j * b + p] = -inv_n * sol[p]; /* -(1/n) Theta^-1 (...) */
    }
    /* deferred updates (Sec. 3.2):
     *   w_{sk+s} = w_sk - (1/(lambda n)) X sum I_t da_t ; alpha_{sk+s} = alpha_sk + sum I_t da_t */
    for (int p = 0; p < sb; ++p) {
      const int64_t i = I[p];
      for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) w[A.col[e]] -= A.val[e] * da[p] / ln;
    }
    for (int p = 0; p < sb; ++p) alpha[I[p]] += da[p];
    if (recompute_every > 0 && (k + 1) % recompute_every == 0) dual_w(&A, d, n, lam, alpha, w);
  }
done:
  free(I); free(G); free(Yw); free(da); free(Th); free(rhs); free(sol); free(scratch);
  return st;
}

/* Algorithm 3, written out on its own. */
int orc_bdcd(const int64_t *rowptr, const int32_t *col, const double *val, int64_t d,
             int64_t n, const double *y, double lam, int b, int64_t H, uint64_t seed,
             int64_t h0, int recompute_every, double *alpha, double *w) {
  if (b < 1 || b > n || H < 1 || !(lam > 0.0)) return ORC_ERR_ARG;
  csr_t A = {rowptr, col, val};
  const double ln = lam * (double)n;
  const double inv_n = 1.0 / (double)n;
  int32_t *I = (int32_t *)malloc((size_t)b * sizeof(int32_t));
  double *Th = (double *)malloc((size_t)b * b * sizeof(double));
  double *rhs = (double *)malloc((size_t)b * sizeof(double));
  double *sol = (double *)malloc((size_t)b * sizeof(double));
  double *scratch = (double *)calloc((size_t)d, sizeof(double));
  int st = ORC_OK;
  if (!I || !Th || !rhs || !sol || !scratch) { st = ORC_ERR_OOM; goto done; }
  dual_w(&A, d, n, lam, alpha, w);
  for (int64_t h = 0; h < H; ++h) {
    st = orc_sample_block(seed, h0 + h, b, n, I);
    if (st) goto done;
    /* Theta_h = (1/(lambda n^2)) I^T X^T X I + (1/n) I_b  (reading R1) */
    for (int p = 0; p < b; ++p)
      for (int q = 0; q < b; ++q)
        Th[(size_t)p * b + q] = col_dot_col(&A, I[p], I[q], scratch) / (ln * (double)n) +
                                (p == q ? inv_n : 0.0);
    /* rhs = -I^T X^T w + I^T alpha + I^T y */
    for (int p = 0; p < b; ++p) rhs[p] = -col_dot_dense(&A, I[p], w) + alpha[I[p]] + y[I[p]];
    st = orc_cholesky_solve(b, Th, rhs, sol);
    if (st) goto done;
    for (int p = 0; p < b; ++p) {
      const double da = -inv_n * sol[p];                  /* Delta alpha_h (eq. "ah") */
      alpha[I[p]] += da;                                  /* eq. "alp" */
      const int64_t i = I[p];
      for (int64_t e = A.rowptr[i]; e < A.rowptr[i + 1]; ++e) w[A.col[e]] -= A.val[e] * da / ln; /* eq. "wup" */
    }
    if (recompute_every > 0 && (h + 1) % recompute_every == 0) dual_w(&A, d, n, lam, alpha, w);
  }
done:
  free(I); free(Th); free(rhs); free(sol); free(scratch);
  return st;
}
