/*
 * CPU oracle for the AVU-GSR hot path: aprod 1, aprod 2, column norms and
 * Paige-Saunders LSQR, in plain FP64 loops.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path may link or call this
 * file: only the test suite, the smoke check and the benchmark's CPU-baseline /
 * reference legs use it. It shares no code, header or constant with the CUDA
 * library. Compile with -O2 -ffp-contract=off so that no multiply-add is fused
 * and every sum is evaluated in the order written.
 *
 * The system (Sec. 2, Eq. 1) is A x = b. A is stored "dense-by-row": each row
 * holds at most 24 coefficients (Sec. 2: 5 astrometric, 12 attitude, 6
 * instrumental, 1 global). Row i is given by
 *   vals[i*24 + t]  coefficient of slot t,
 *   astro_off[i]    first astrometric column (5 consecutive: slots 0..4),
 *   att_off[i]      first attitude column of axis 0; axis a uses
 *                   att_off[i] + a*n_knots + j for j = 0..3 (slots 5+4a+j),
 *   instr[i*6 + k]  instrumental index k (slots 17..22), column
 *                   5*n_stars + 3*n_knots + instr[i*6+k],
 *   slot 23         global column 5*n_stars + 3*n_knots + n_instr, present
 *                   only when n_glob == 1 (ignored otherwise).
 * The slot/column convention is this library's reading; the paper fixes only
 * the per-row counts.
 *
 * Constraint equations (Sec. 2: the system needs a set of them for a unique
 * solution; Sec. 2.1: about 1% of it): n_con further rows after the n_rows
 * observations, given in CSR form - row c has the entries k in
 * [con_ptr[c], con_ptr[c+1]) with column con_col[k] and coefficient
 * con_val[k]. Vectors over the equations (y, b) then have n_rows + n_con
 * entries, the constraint rows last. n_con = 0 (NULL arrays) means none.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NSLOT 24

typedef struct {
  int64_t n_rows, n_stars, n_knots, n_instr;
  int32_t n_glob;
} odims;

static int64_t n_unknowns(const odims* d) {
  return 5 * d->n_stars + 3 * d->n_knots + d->n_instr + d->n_glob;
}

/* Column of slot t of row i, or -1 for an absent slot. */
static int64_t col_of(const odims* d, const int64_t* astro_off, const int64_t* att_off,
                      const int32_t* instr, int64_t i, int t) {
  if (t < 5) return astro_off[i] + t;
  if (t < 17) {
    int a = (t - 5) / 4, j = (t - 5) % 4;
    return att_off[i] + (int64_t)a * d->n_knots + j;
  }
  if (t < 23) return 5 * d->n_stars + 3 * d->n_knots + instr[i * 6 + (t - 17)];
  if (d->n_glob == 1) return 5 * d->n_stars + 3 * d->n_knots + d->n_instr;
  return -1;
}

int64_t oracle_n_unknowns(int64_t n_rows, int64_t n_stars, int64_t n_knots, int64_t n_instr,
                          int32_t n_glob) {
  odims d = {n_rows, n_stars, n_knots, n_instr, n_glob};
  return n_unknowns(&d);
}

/* The constraint rows of a system (n_con = 0: none). */
typedef struct {
  int64_t n_con;
  const int64_t* ptr;
  const int64_t* col;
  const double* val;
} ocons;

/* Eq. 2 (aprod 1): y += A x, rows in order, slots in order, then the
   constraint rows in order, entries in order. */
static void aprod1_c(const odims* d, const double* vals, const int64_t* astro_off,
                     const int64_t* att_off, const int32_t* instr, const ocons* cn,
                     const double* x, double* y) {
  for (int64_t i = 0; i < d->n_rows; ++i) {
    double s = 0.0;
    for (int t = 0; t < NSLOT; ++t) {
      int64_t c = col_of(d, astro_off, att_off, instr, i, t);
      if (c < 0) continue;
      s += vals[i * NSLOT + t] * x[c];
    }
    y[i] += s;
  }
  for (int64_t r = 0; r < cn->n_con; ++r) {
    double s = 0.0;
    for (int64_t k = cn->ptr[r]; k < cn->ptr[r + 1]; ++k) s += cn->val[k] * x[cn->col[k]];
    y[d->n_rows + r] += s;
  }
}

/* Eq. 3 (aprod 2): x += A^T y, rows in order, slots in order, then the
   constraint rows. */
static void aprod2_c(const odims* d, const double* vals, const int64_t* astro_off,
                     const int64_t* att_off, const int32_t* instr, const ocons* cn,
                     const double* y, double* x) {
  for (int64_t i = 0; i < d->n_rows; ++i) {
    for (int t = 0; t < NSLOT; ++t) {
      int64_t c = col_of(d, astro_off, att_off, instr, i, t);
      if (c < 0) continue;
      x[c] += vals[i * NSLOT + t] * y[i];
    }
  }
  for (int64_t r = 0; r < cn->n_con; ++r)
    for (int64_t k = cn->ptr[r]; k < cn->ptr[r + 1]; ++k)
      x[cn->col[k]] += cn->val[k] * y[d->n_rows + r];
}

void oracle_aprod1(int64_t n_rows, int64_t n_stars, int64_t n_knots, int64_t n_instr,
                   int32_t n_glob, const double* vals, const int64_t* astro_off,
                   const int64_t* att_off, const int32_t* instr, int64_t n_con,
                   const int64_t* con_ptr, const int64_t* con_col, const double* con_val,
                   const double* x, double* y) {
  odims d = {n_rows, n_stars, n_knots, n_instr, n_glob};
  ocons cn = {n_con, con_ptr, con_col, con_val};
  aprod1_c(&d, vals, astro_off, att_off, instr, &cn, x, y);
}

void oracle_aprod2(int64_t n_rows, int64_t n_stars, int64_t n_knots, int64_t n_instr,
                   int32_t n_glob, const double* vals, const int64_t* astro_off,
                   const int64_t* att_off, const int32_t* instr, int64_t n_con,
                   const int64_t* con_ptr, const int64_t* con_col, const double* con_val,
                   const double* y, double* x) {
  odims d = {n_rows, n_stars, n_knots, n_instr, n_glob};
  ocons cn = {n_con, con_ptr, con_col, con_val};
  aprod2_c(&d, vals, astro_off, att_off, instr, &cn, y, x);
}

/* Squared Euclidean norm of every column of A, constraint rows included (the
   diagonal of A^T A). */
static void colnorm2_c(const odims* d, const double* vals, const int64_t* astro_off,
                       const int64_t* att_off, const int32_t* instr, const ocons* cn,
                       double* c2) {
  int64_t n = n_unknowns(d);
  for (int64_t j = 0; j < n; ++j) c2[j] = 0.0;
  for (int64_t i = 0; i < d->n_rows; ++i) {
    for (int t = 0; t < NSLOT; ++t) {
      int64_t c = col_of(d, astro_off, att_off, instr, i, t);
      if (c < 0) continue;
      double a = vals[i * NSLOT + t];
      c2[c] += a * a;
    }
  }
  for (int64_t r = 0; r < cn->n_con; ++r)
    for (int64_t k = cn->ptr[r]; k < cn->ptr[r + 1]; ++k) c2[cn->col[k]] += cn->val[k] * cn->val[k];
}

void oracle_colnorm2(int64_t n_rows, int64_t n_stars, int64_t n_knots, int64_t n_instr,
                     int32_t n_glob, const double* vals, const int64_t* astro_off,
                     const int64_t* att_off, const int32_t* instr, int64_t n_con,
                     const int64_t* con_ptr, const int64_t* con_col, const double* con_val,
                     double* c2) {
  odims d = {n_rows, n_stars, n_knots, n_instr, n_glob};
  ocons cn = {n_con, con_ptr, con_col, con_val};
  colnorm2_c(&d, vals, astro_off, att_off, instr, &cn, c2);
}

static double dnrm2(int64_t n, const double* v) {
  /* Plain sum of squares; the inputs here never approach overflow. */
  double s = 0.0;
  for (int64_t k = 0; k < n; ++k) s += v[k] * v[k];
  return sqrt(s);
}

/*
 * Paige & Saunders (1982) LSQR, cited in Sec. 1 and used as "the LSQR" of
 * Sec. 2.1, on the column-scaled operator A D (A with its constraint rows; b
 * has n_rows + n_con entries) (Sec. 2, solver steps 2 and 5:
 * precondition, then de-precondition x = D z).
 *
 * scale: NULL for no scaling, else d[j] > 0 for every column.
 * opts[0..2] = atol, btol, conlim; itnlim is separate.
 * var: NULL or N_unk doubles; receives the variance estimate
 *      sum_k (d_k)^2, d_k = w_k / rho_k, de-preconditioned (times d^2).
 * x_ref/err_hist: if both non-NULL, err_hist[k-1] = ||x_k - x_ref|| / ||x_ref||
 *      for every iteration k (a measurement aid, not part of the method).
 * rnorm_hist: if non-NULL, rnorm_hist[k-1] = the estimate phibar_{k+1} of ||r_k||.
 * cov_pairs/cov: n_cov index pairs (j1, j2) (cov_pairs[2p], cov_pairs[2p+1]);
 *      cov[p] receives the covariance estimate of Sec. 2.2, Eq. 4, read with
 *      the same direction vectors as the variance: the sum over iterations of
 *      d_k[j1] d_k[j2], d_k = w_k / rho_k, de-preconditioned (times
 *      d[j1] d[j2]). Eq. 4's per-iteration factor is 1 in this reading; a pair
 *      (j, j) gives var[j].
 * out[0..6] = istop, itn, rnorm, arnorm, anorm, acond, xnorm.
 * Returns 0, or -1 on allocation failure.
 */
int oracle_lsqr(int64_t n_rows, int64_t n_stars, int64_t n_knots, int64_t n_instr, int32_t n_glob,
                const double* vals, const int64_t* astro_off, const int64_t* att_off,
                const int32_t* instr, int64_t n_con, const int64_t* con_ptr,
                const int64_t* con_col, const double* con_val, const double* b,
                const double* scale, const double* opts, int64_t itnlim, double* x, double* var,
                const double* x_ref, double* err_hist, double* rnorm_hist, int64_t n_cov,
                const int64_t* cov_pairs, double* cov, double* out) {
  odims d = {n_rows, n_stars, n_knots, n_instr, n_glob};
  ocons cn = {n_con, con_ptr, con_col, con_val};
  int64_t m = n_rows + n_con, n = n_unknowns(&d);
  double atol = opts[0], btol = opts[1], conlim = opts[2];
  double ctol = conlim > 0.0 ? 1.0 / conlim : 0.0;

  double* u = (double*)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
  double* v = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* z = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));   /* scaled iterate */
  double* tmp = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double* vz = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));  /* var of z */
  if (!u || !v || !w || !z || !tmp || !vz) {
    free(u); free(v); free(w); free(z); free(tmp); free(vz);
    return -1;
  }
  for (int64_t j = 0; j < n; ++j) { z[j] = 0.0; vz[j] = 0.0; x[j] = 0.0; }
  for (int64_t p = 0; p < n_cov; ++p) cov[p] = 0.0;
  double xrefn = 0.0;
  if (x_ref && err_hist) xrefn = dnrm2(n, x_ref);

  int64_t itn = 0;
  int istop = 0;
  double anorm = 0.0, acond = 0.0, ddnorm = 0.0, xnorm = 0.0;
  double rnorm, arnorm;

  /* beta_1 u_1 = b */
  for (int64_t i = 0; i < m; ++i) u[i] = b[i];
  double beta = dnrm2(m, u);
  double bnorm = beta;
  double alpha = 0.0;
  if (beta > 0.0) {
    for (int64_t i = 0; i < m; ++i) u[i] /= beta;
    /* alpha_1 v_1 = (A D)^T u_1 */
    for (int64_t j = 0; j < n; ++j) tmp[j] = 0.0;
    aprod2_c(&d, vals, astro_off, att_off, instr, &cn, u, tmp);
    for (int64_t j = 0; j < n; ++j) v[j] = scale ? scale[j] * tmp[j] : tmp[j];
    alpha = dnrm2(n, v);
  } else {
    for (int64_t j = 0; j < n; ++j) v[j] = 0.0;
  }
  if (alpha > 0.0)
    for (int64_t j = 0; j < n; ++j) v[j] /= alpha;
  for (int64_t j = 0; j < n; ++j) w[j] = v[j];

  double phibar = beta, rhobar = alpha;
  rnorm = beta;
  arnorm = alpha * beta;
  if (arnorm == 0.0) {
    /* b = 0 or A^T b = 0: x = 0 is the least-squares solution. */
    out[0] = 0; out[1] = 0; out[2] = rnorm; out[3] = arnorm; out[4] = 0; out[5] = 0; out[6] = 0;
    if (var) for (int64_t j = 0; j < n; ++j) var[j] = 0.0;
    free(u); free(v); free(w); free(z); free(tmp); free(vz);
    return 0;
  }

  while (1) {
    ++itn;
    /* beta_{i+1} u_{i+1} = (A D) v_i - alpha_i u_i */
    for (int64_t j = 0; j < n; ++j) tmp[j] = scale ? scale[j] * v[j] : v[j];
    for (int64_t i = 0; i < m; ++i) u[i] = -alpha * u[i];
    aprod1_c(&d, vals, astro_off, att_off, instr, &cn, tmp, u);
    beta = dnrm2(m, u);
    if (beta > 0.0)
      for (int64_t i = 0; i < m; ++i) u[i] /= beta;
    anorm = sqrt(anorm * anorm + alpha * alpha + beta * beta);

    /* alpha_{i+1} v_{i+1} = (A D)^T u_{i+1} - beta_{i+1} v_i */
    for (int64_t j = 0; j < n; ++j) tmp[j] = 0.0;
    aprod2_c(&d, vals, astro_off, att_off, instr, &cn, u, tmp);
    for (int64_t j = 0; j < n; ++j) v[j] = (scale ? scale[j] * tmp[j] : tmp[j]) - beta * v[j];
    alpha = dnrm2(n, v);
    if (alpha > 0.0)
      for (int64_t j = 0; j < n; ++j) v[j] /= alpha;

    /* Plane rotation eliminating beta_{i+1} from the lower bidiagonal. */
    double rho = sqrt(rhobar * rhobar + beta * beta);
    double c = rhobar / rho;
    double s = beta / rho;
    double theta = s * alpha;
    rhobar = -c * alpha;
    double phi = c * phibar;
    phibar = s * phibar;

    /* Eq. 4 for the chosen pairs, with the direction d_k = w_k / rho_k (before
       w is updated below) */
    for (int64_t p = 0; p < n_cov; ++p)
      cov[p] += (w[cov_pairs[2 * p]] / rho) * (w[cov_pairs[2 * p + 1]] / rho);

    /* x_i = x_{i-1} + (phi/rho) w_i ; w_{i+1} = v_{i+1} - (theta/rho) w_i */
    double t1 = phi / rho, t2 = -theta / rho;
    double dk2 = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      double dj = w[j] / rho;
      dk2 += dj * dj;
      vz[j] += dj * dj;
      z[j] += t1 * w[j];
      w[j] = v[j] + t2 * w[j];
    }
    ddnorm += dk2;

    /* Estimates (Paige & Saunders Sec. 5) and the stopping tests. The loop
       solves the preconditioned system (Sec. 2, solver step 2; x = D z only
       afterwards, step 5), so its tests use the quantities of that system:
       ||A D|| (anorm) and the exact norm of its iterate z. ||x|| is reported. */
    acond = anorm * sqrt(ddnorm);
    rnorm = phibar;
    arnorm = alpha * fabs(c) * phibar;
    for (int64_t j = 0; j < n; ++j) x[j] = scale ? scale[j] * z[j] : z[j];
    xnorm = dnrm2(n, x);
    double znorm = dnrm2(n, z);
    if (rnorm_hist) rnorm_hist[itn - 1] = rnorm;
    if (x_ref && err_hist) {
      double e2 = 0.0;
      for (int64_t j = 0; j < n; ++j) { double e = x[j] - x_ref[j]; e2 += e * e; }
      err_hist[itn - 1] = xrefn > 0.0 ? sqrt(e2) / xrefn : sqrt(e2);
    }

    double test1 = rnorm / bnorm;
    double test2 = (anorm * rnorm > 0.0) ? arnorm / (anorm * rnorm) : 0.0;
    double test3 = 1.0 / acond;
    double t1n = test1 / (1.0 + anorm * znorm / bnorm);
    double rtol = btol + atol * anorm * znorm / bnorm;
    istop = 0;
    if (itn >= itnlim) istop = 7;
    if (1.0 + test3 <= 1.0) istop = 6;
    if (1.0 + test2 <= 1.0) istop = 5;
    if (1.0 + t1n <= 1.0) istop = 4;
    if (test3 <= ctol) istop = 3;
    if (test2 <= atol) istop = 2;
    if (test1 <= rtol) istop = 1;
    if (istop != 0) break;
  }

  if (var)
    for (int64_t j = 0; j < n; ++j) var[j] = scale ? scale[j] * scale[j] * vz[j] : vz[j];
  if (scale)
    for (int64_t p = 0; p < n_cov; ++p) cov[p] *= scale[cov_pairs[2 * p]] * scale[cov_pairs[2 * p + 1]];
  out[0] = istop; out[1] = (double)itn; out[2] = rnorm; out[3] = arnorm;
  out[4] = anorm; out[5] = acond; out[6] = xnorm;
  free(u); free(v); free(w); free(z); free(tmp); free(vz);
  return 0;
}
