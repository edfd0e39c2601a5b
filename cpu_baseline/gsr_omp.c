/*
 * All-core CPU baseline of the AVU-GSR products (Sec. 2, Eq. 2 and Eq. 3) for
 * the benchmark: a reasonable multi-threaded CPU implementation, written
 * independently of both the test oracle and the CUDA library (it shares no
 * code, header or helper with either).
 *
 *   aprod 1  y += A x   row-parallel: every thread owns a contiguous block of
 *                       rows and writes its own y entries;
 *   aprod 2  x += A^T y thread-private accumulation: rows are split into
 *                       blocks that never divide a star, so a star's five
 *                       astrometric unknowns belong to one thread and are
 *                       written directly; the attitude, instrumental and
 *                       global unknowns, shared by all rows, go into a private
 *                       array per thread that is reduced at the end.
 *
 * Row layout (the library's reading of Sec. 2): 24 values per row - five
 * astrometric (columns astro_off .. +4), twelve attitude (three axes, four
 * consecutive knots from att_off, axes n_knots apart), six instrumental
 * (column 5 n_stars + 3 n_knots + instr[k]) and one global (the last
 * column, used when n_glob = 1).
 *
 * Build: gcc -O3 -march=native -fopenmp -shared -fPIC.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

int gsr_omp_threads(void) { return omp_get_max_threads(); }

void gsr_omp_aprod1(int64_t n_rows, int64_t n_stars, int64_t n_knots, int64_t n_instr,
                    int32_t n_glob, const double* restrict vals,
                    const int64_t* restrict astro_off, const int64_t* restrict att_off,
                    const int32_t* restrict instr, const double* restrict x,
                    double* restrict y) {
  const int64_t ib = 5 * n_stars + 3 * n_knots;
  const double xg = n_glob ? x[ib + n_instr] : 0.0;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_rows; ++i) {
    const double* v = vals + 24 * i;
    const double* xa = x + astro_off[i];
    const double* x0 = x + att_off[i];
    const double* x1 = x0 + n_knots;
    const double* x2 = x1 + n_knots;
    const int32_t* in = instr + 6 * i;
    double s = v[0] * xa[0] + v[1] * xa[1] + v[2] * xa[2] + v[3] * xa[3] + v[4] * xa[4];
    s += v[5] * x0[0] + v[6] * x0[1] + v[7] * x0[2] + v[8] * x0[3];
    s += v[9] * x1[0] + v[10] * x1[1] + v[11] * x1[2] + v[12] * x1[3];
    s += v[13] * x2[0] + v[14] * x2[1] + v[15] * x2[2] + v[16] * x2[3];
    for (int k = 0; k < 6; ++k) s += v[17 + k] * x[ib + in[k]];
    if (n_glob) s += v[23] * xg;
    y[i] += s;
  }
}

int gsr_omp_aprod2(int64_t n_rows, int64_t n_stars, int64_t n_knots, int64_t n_instr,
                   int32_t n_glob, const double* restrict vals,
                   const int64_t* restrict astro_off, const int64_t* restrict att_off,
                   const int32_t* restrict instr, const double* restrict y,
                   double* restrict x) {
  const int64_t ab = 5 * n_stars, ib = ab + 3 * n_knots;
  const int64_t n_shared = 3 * n_knots + n_instr + n_glob;  /* columns from ab on */
  const int nt = omp_get_max_threads();
  double* priv = (double*)calloc((size_t)nt * (size_t)n_shared, sizeof(double));
  int64_t* cut = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nt + 1));
  if (!priv || !cut) {
    free(priv);
    free(cut);
    return -1;
  }
  /* row blocks that start at a star boundary */
  cut[0] = 0;
  for (int t = 1; t < nt; ++t) {
    int64_t r = (n_rows * t) / nt;
    if (r < cut[t - 1]) r = cut[t - 1];
    while (r > 0 && r < n_rows && astro_off[r] == astro_off[r - 1]) ++r;
    cut[t] = r;
  }
  cut[nt] = n_rows;
#pragma omp parallel num_threads(nt)
  {
    const int t = omp_get_thread_num();
    double* p = priv + (size_t)t * (size_t)n_shared;  /* index: column - ab */
    for (int64_t i = cut[t]; i < cut[t + 1]; ++i) {
      const double* v = vals + 24 * i;
      const double yi = y[i];
      double* xa = x + astro_off[i];
      for (int k = 0; k < 5; ++k) xa[k] += v[k] * yi;
      const int64_t s0 = att_off[i] - ab;
      for (int a = 0; a < 3; ++a)
        for (int k = 0; k < 4; ++k) p[s0 + a * n_knots + k] += v[5 + 4 * a + k] * yi;
      const int32_t* in = instr + 6 * i;
      for (int k = 0; k < 6; ++k) p[ib - ab + in[k]] += v[17 + k] * yi;
      if (n_glob) p[ib - ab + n_instr] += v[23] * yi;
    }
  }
#pragma omp parallel for schedule(static)
  for (int64_t c = 0; c < n_shared; ++c) {
    double s = 0.0;
    for (int t = 0; t < nt; ++t) s += priv[(size_t)t * (size_t)n_shared + c];
    x[ab + c] += s;
  }
  free(priv);
  free(cut);
  return 0;
}
