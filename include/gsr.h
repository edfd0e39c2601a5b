/*
 * gsr.h - C ABI of libgsr, a single-GPU (B300, sm_103a) implementation of the
 * hot path of the Gaia AVU-GSR solver (arXiv 2503.22863):
 *   aprod 1  y += A x      (Sec. 2, Eq. 2)
 *   aprod 2  x += A^T y    (Sec. 2, Eq. 3)
 *   preconditioned LSQR on A x = b (Sec. 2, Eq. 1; solver steps 2-5 of Sec. 2),
 *   the Paige-Saunders algorithm cited in Sec. 1.
 *
 * Matrix (Sec. 2): n_rows observation equations, each with at most 24
 * coefficients: 5 astrometric, 12 attitude (3 axes x 4 consecutive spline
 * knots), 6 instrumental and 1 global. Host input is "dense by row":
 *   vals      double  [n_rows][24]  slot order: astro 0..4 | att axis0 knot
 *                                   +0..3, axis1 +0..3, axis2 +0..3 | instr 0..5 | glob
 *   astro_off int64   [n_rows]      5*star(i); rows sorted by star (non-decreasing)
 *   att_off   int64   [n_rows]      5*n_stars + s_i, 0 <= s_i <= n_knots-4; the
 *                                   three axes use s_i at offsets 0, n_knots, 2*n_knots
 *   instr     int32   [n_rows][6]   distinct instrumental indices in [0, n_instr)
 * Column layout of x (N_unk = 5*n_stars + 3*n_knots + n_instr + n_glob):
 *   [astro 5*n_stars | attitude 3*n_knots | instrumental n_instr | global n_glob]
 * The slot and column conventions are this library's reading: the paper fixes
 * only the per-row counts.
 *
 * Conventions for every call:
 *   - Vector arguments marked "device" are caller-owned device pointers on the
 *     system's device (for example torch tensors); the library never frees them.
 *   - "stream" is a cudaStream_t (NULL = the legacy default stream). Calls are
 *     stream-ordered and asynchronous unless stated otherwise.
 *   - Every call returns a gsr_status; nothing aborts or prints.
 *     gsr_strerror() gives the text. After GSR_E_CUDA or GSR_E_TIMEOUT the
 *     system should be destroyed: a device wait that ran out may have left
 *     copies into a block's shared memory unfinished and the results of that
 *     launch incomplete.
 *   - Arithmetic: products and sums run as pairs of FP32 numbers with
 *     error-free transformations (about 48 significant bits, within 1e-13 of
 *     FP64 relative to |A||x|); vectors, norms and LSQR scalars are FP64.
 *   - Range: any finite FP64 input is accepted, except the matrices
 *     gsr_create rejects below. A float pair has FP32's exponent range, so the
 *     library works on an exactly rescaled problem. gsr_create multiplies row
 *     i by 2^e_i and column j by 2^g_j (powers of two, exact). It leaves a
 *     matrix whose nonzero |A_ij| all lie in [2^-40, 2^40) as it is. Otherwise
 *     it uses column exponents alone where that suffices, else row and column
 *     exponents. Every call undoes the scaling exactly. A product call checks
 *     its rescaled input vector: with every nonzero entry in [2^-60, 2^60) the
 *     float-pair kernels run; otherwise the same call runs FP64 kernels (one
 *     thread per row, several times slower, accurate to FP64 rounding). The
 *     choice is made on the device, per call. LSQR scales b by a power of two
 *     (its largest entry into [1, 2)) and scales x and the residual norms
 *     back.
 */
#ifndef GSR_H
#define GSR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gsr_system gsr_system; /* opaque, library-owned */

typedef enum {
  GSR_OK = 0,
  GSR_E_ARG = 1,         /* null pointer, negative size, bad option */
  GSR_E_INDEX = 2,       /* an offset or index outside its block */
  GSR_E_UNSORTED = 3,    /* rows not sorted by star */
  GSR_E_NONFINITE = 4,   /* NaN or Inf in the matrix or right-hand side */
  GSR_E_OOM = 5,         /* device allocation failed */
  GSR_E_CUDA = 6,        /* a CUDA runtime call failed */
  GSR_E_TIMEOUT = 7,     /* a bounded device-side wait or retry loop ran out */
  GSR_E_UNSUPPORTED = 8  /* sizes beyond this build's limits (see gsr_create) */
} gsr_status;

/* Which stored copy of the matrix values an aprod call reads. */
enum { GSR_VALUES_F64 = 0, GSR_VALUES_F32 = 1 };
/* Storage of the matrix values. F32_PLUS_F64 keeps an FP32 copy (half the
 * bytes, used by the mixed-precision solve) beside the full-precision one. */
enum { GSR_STORE_F64 = 0, GSR_STORE_F32_PLUS_F64 = 1 };
/* Column preconditioner (Sec. 2, solver steps 2 and 5). */
enum { GSR_PRECOND_NONE = 0, GSR_PRECOND_COLNORM = 1, GSR_PRECOND_USER = 2 };
/* LSQR precision mode. */
enum { GSR_PREC_F64 = 0, GSR_PREC_MIXED = 1 };

typedef struct {
  int64_t n_rows, n_stars, n_knots, n_instr;
  int32_t n_glob;  /* 0 or 1 */
  int32_t storage; /* GSR_STORE_* */
} gsr_dims;

/*
 * Create a system on `device` from host arrays (layout above). The arrays are
 * read during the call only; the library keeps its own device copies in a
 * tiled, coalesced layout plus a copy of the attitude coefficients sorted by
 * start knot, and computes the column norms ||A_:,j||_2. Synchronous.
 * Validation: GSR_E_ARG (null/negative, n_knots < 4, n_instr < 6, n_glob not
 * 0/1), GSR_E_INDEX (astro_off not 5*star in range, s_i outside [0, K-4],
 * instr outside [0, n_instr) or repeated in a row), GSR_E_UNSORTED (astro_off
 * decreasing), GSR_E_NONFINITE (NaN/Inf value), GSR_E_UNSUPPORTED (n_rows or
 * N_unk >= 2^31, or n_instr > 24576: the instrumental histogram of aprod 2
 * lives in one block's shared memory; or coefficients too spread for the
 * rescaling: after the library fits power-of-two row and column exponents to
 * the binary exponents of A in the least-squares sense, a coefficient remains
 * more than 2^100 below the largest of its column - every 2 x 2 minor with
 * |a00 a11 / (a01 a10)| beyond about 2^204, such as [[1, 1e-70], [1, 1]], is
 * one, since no diagonal scaling changes that ratio), GSR_E_OOM. All of these
 * are decided on the host before the device is touched.
 * Matrices whose rescaled coefficients still reach below 2^-40 of their row
 * and column maxima are accepted; their products always run the FP64
 * kernels.
 * On success *out owns everything; release it with gsr_destroy().
 */
int gsr_create(const gsr_dims* dims, const double* vals, const int64_t* astro_off,
               const int64_t* att_off, const int32_t* instr, int device, void* stream,
               gsr_system** out);

void gsr_destroy(gsr_system* sys);
const char* gsr_strerror(int status);
int64_t gsr_n_unknowns(const gsr_system* sys);
/* Observation rows (the rows given to gsr_create). */
int64_t gsr_n_rows(const gsr_system* sys);

/*
 * Constraint equations (Sec. 2: the overdetermined system needs a set of
 * constraint equations for a unique solution; Sec. 2.1: they are about 1% of
 * the system and replicated on every process). The paper does not give their
 * form, so they are generic sparse rows, appended to A after the n_rows
 * observation rows. Host arrays in CSR form, copied during the call:
 *   con_ptr int64  [n_con + 1]  row c holds entries con_ptr[c] .. con_ptr[c+1]-1,
 *                               con_ptr[0] = 0, non-decreasing
 *   con_col int64  [nnz]        column in [0, N_unk) (repeats allowed)
 *   con_val double [nnz]        finite coefficient (any FP64 magnitude)
 * Afterwards every vector over the equations - y of aprod 1 and aprod 2 and
 * of their _values and _noalloc forms, b of gsr_lsqr_solve - has
 * gsr_n_equations() = n_rows + n_con entries, the constraint rows last, and
 * the column norms (and so the column preconditioner) include them. The
 * constraint rows are computed in FP64 (a warp per segment of at most 1024
 * entries). A call replaces earlier constraints; n_con = 0 removes them.
 * The batched forms do not take constraint rows (GSR_E_UNSUPPORTED).
 * Errors: GSR_E_ARG (sizes, pointers, con_ptr not non-decreasing from 0),
 * GSR_E_INDEX (a column outside [0, N_unk)), GSR_E_NONFINITE, all on the host
 * before the device is touched; GSR_E_OOM. Synchronises the stream.
 */
int gsr_set_constraints(gsr_system* sys, int64_t n_con, const int64_t* con_ptr,
                        const int64_t* con_col, const double* con_val, void* stream);
/* Equations of the system: n_rows + n_con. */
int64_t gsr_n_equations(const gsr_system* sys);

/* Eq. 2 (aprod 1): y[n_eq] += A x[N_unk] (n_eq = gsr_n_equations: the
 * observation rows, then any constraint rows). x, y device; x is not modified.
 * Both aprods follow the range rule above: float-pair kernels when the
 * rescaled input is within [2^-60, 2^60), FP64 kernels otherwise. */
int gsr_aprod1(gsr_system* sys, const double* x, double* y, void* stream);
/* Eq. 3 (aprod 2): x[N_unk] += A^T y[n_eq]. x, y device. */
int gsr_aprod2(gsr_system* sys, const double* y, double* x, void* stream);
/* As above on a chosen copy of the values (GSR_VALUES_F32 needs
 * GSR_STORE_F32_PLUS_F64; with it the products use the FP32-rounded A). */
int gsr_aprod1_values(gsr_system* sys, int which_values, const double* x, double* y,
                      void* stream);
int gsr_aprod2_values(gsr_system* sys, int which_values, const double* y, double* x,
                      void* stream);

/*
 * Allocation-free aprod 1 (this entry point has no counterpart in the paper):
 * y[n_rows] += A x[N_unk] exactly as gsr_aprod1, for callers that must not
 * allocate device memory when they call it - a process whose device memory is
 * already taken by another framework's caching allocator, or a latency-critical
 * loop that cannot absorb the device-wide synchronisation cudaMalloc/cudaFree
 * imply. It calls no cudaMalloc, cudaFree or other allocating routine and uses
 * none of the system's scratch: the float-pair copy of x that the product reads
 * is staged in a fixed device array compiled into the library
 * (GSR_NOALLOC_MAX_UNK float pairs = 8 MiB, plus one 8-byte range flag, held by
 * every GPU that loads the library until the process exits). Systems with
 * N_unk > GSR_NOALLOC_MAX_UNK get GSR_E_UNSUPPORTED. The first call on a device
 * looks up the array's device address (with that device current); make that
 * first call before any stream capture begins. Every call on a device shares
 * the one array, and each call rewrites the part it reads (nothing in it needs
 * to start at zero), so calls that overlap on the GPU - on different streams,
 * or for different systems on the same device - race and must be serialised
 * by the caller. x, y device; stream as above.
 */
#define GSR_NOALLOC_MAX_UNK 1048576
int gsr_aprod1_noalloc(gsr_system* sys, const double* x, double* y, void* stream);

/* Column norms c_j = ||A_:,j||_2 (FP64 copy of the values) into c[N_unk], device. */
int gsr_column_norms(gsr_system* sys, double* c, void* stream);

typedef struct {
  double atol, btol, conlim; /* Paige-Saunders stopping tolerances (conlim 0 = off) */
  int64_t itnlim;            /* iteration limit (istop = 7 when reached) */
  int32_t precond;           /* GSR_PRECOND_*; USER takes `scale` */
  int32_t precision;         /* GSR_PREC_F64 or GSR_PREC_MIXED */
  const double* scale;       /* device [N_unk], d_j > 0, for GSR_PRECOND_USER */
  double* var;               /* optional device [N_unk]: variance estimate out */
  const double* x_ref;       /* optional device [N_unk]: per-iteration error reference */
  double* err_hist;          /* optional host [itnlim]: ||x_k - x_ref|| / ||x_ref|| */
  double* rnorm_hist;        /* optional host [itnlim]: estimate of ||b - A x_k|| */
  int32_t mixed_switch_itn;  /* MIXED: iterations of the FP32-values phase (0 = auto) */
  int32_t profile;           /* 1: time aprod 1 / aprod 2 / vector kernels with CUDA
                                events recorded inside the iteration graph */
  /* Covariances of chosen pairs of unknowns (Sec. 2.2, Eq. 4). Every
   * iteration adds d_k[j1] d_k[j2] for each pair, d_k = w_k / rho_k being the
   * direction whose squares make the variance estimate (Eq. 4's per-iteration
   * factor is read as 1: the paper does not define it); the result is
   * de-preconditioned, cov = d_j1 d_j2 sum_k. A pair (j, j) gives var[j].
   * Index pairs outside [0, N_unk): GSR_E_INDEX. Single right-hand side and
   * precision F64 only (MIXED computes them in its FP32 phase, like var). */
  int64_t n_cov;             /* number of pairs (0: none) */
  const int64_t* cov_pairs;  /* device [n_cov][2]: (j1, j2) */
  double* cov;               /* device [n_cov] out */
} gsr_lsqr_opts;

typedef struct {
  int32_t istop;   /* 0 x=0 solves; 1,2 converged; 3 cond limit; 4,5 machine precision;
                      6 cond at machine precision; 7 itnlim reached (not an error) */
  int32_t phase2_itn; /* MIXED: iterations of the FP64 correction phase */
  int64_t itn;
  double rnorm, arnorm, anorm, acond, xnorm;
  int64_t n_launches;    /* kernels this call launched (including no-op tail launches) */
  int64_t n_timed_itn;   /* iterations covered by the timings below (profile = 1) */
  double t_aprod1_ms, t_aprod2_ms, t_vector_ms; /* summed device time per kernel group */
} gsr_lsqr_result;

/* Fill opts with defaults: atol = btol = 1e-12, conlim = 1e12, itnlim = 0
 * (meaning 20*N_unk), COLNORM, F64, no outputs (no variance, no covariances). */
void gsr_lsqr_default_opts(gsr_lsqr_opts* opts);

/*
 * Solve min ||A x - b||_2 by LSQR on A D (D from opts.precond), returning the
 * de-preconditioned x = D z (Sec. 2, solver steps 2-5). b [n_eq] (observation
 * rows, then constraint rows) and x [N_unk] are device pointers. The stopping
 * tests are those of the preconditioned system the loop solves: ||A D||, and
 * the norm of its iterate z; res.xnorm reports ||x||. Blocks until the result is final (one host
 * read of the stopping flag every few iterations). Reaching itnlim returns
 * GSR_OK with istop = 7.
 * Errors: GSR_E_NONFINITE for a NaN/Inf in b; GSR_E_ARG for a user scale that
 * is not positive and finite; GSR_E_UNSUPPORTED when gsr_create had to give
 * rows different exponents (a row rescaling would change the least-squares
 * problem, and it is not folded into D), or when D 2^-g_j leaves [2^-60, 2^60)
 * for some column (PRECOND_NONE / USER on a column-rescaled system; never
 * with COLNORM).
 */
int gsr_lsqr_solve(gsr_system* sys, const double* b, double* x, const gsr_lsqr_opts* opts,
                   gsr_lsqr_result* res, void* stream);

/*
 * Multi-right-hand-side forms: k systems sharing A (1 <= k <= 32), e.g.
 * Monte-Carlo perturbed observation vectors b_j = A x* + noise_j used to
 * estimate covariances (the quantity of Sec. 2.2, Eq. 4). Vectors are
 * row-major with the right-hand sides interleaved: Y [n_rows][k], X [N_unk][k],
 * device. A is read once per product for all k columns.
 */
/* Eq. 2 for k columns: Y += A X. */
int gsr_aprod1_batch(gsr_system* sys, int k, const double* X, double* Y, void* stream);
/* Eq. 3 for k columns: X += A^T Y. */
int gsr_aprod2_batch(gsr_system* sys, int k, const double* Y, double* X, void* stream);
/*
 * LSQR on the k systems at once (same A, tolerances and preconditioner;
 * per-right-hand-side scalars, stopping tests and convergence masks: a system
 * that has stopped keeps its x while the others continue). res has k entries.
 * opts.err_hist (host, [itnlim][k]) with opts.x_ref (device [N_unk][k]) gives
 * per-iteration relative errors. precision F64, or MIXED (needs
 * GSR_STORE_F32_PLUS_F64): a first LSQR phase with the FP32 copy of A and
 * FP32 products (one multiply-add per product instead of a float-pair one) to
 * about 1e-6, then the residual R = B - A X1 with the full-precision values and
 * a second phase with the float-pair kernels on R to the caller's tolerances,
 * X = X1 + that correction (opts.mixed_switch_itn fixes the first phase's
 * length); res[j].phase2_itn gives the second phase's iterations. var,
 * rnorm_hist and covariances are not available here (GSR_E_UNSUPPORTED). The
 * first call for a given k times
 * the candidate block widths and instrumental row-tile heights on this system and
 * keeps the fastest (gsr_batch_tuning reports the choice). Synchronous.
 */
int gsr_lsqr_solve_batch(gsr_system* sys, int k, const double* B, double* X,
                         const gsr_lsqr_opts* opts, gsr_lsqr_result* res, void* stream);
/* Block width of the row kernels and row-tile height of the instrumental
 * buckets chosen by the tuner. */
int gsr_batch_tuning(const gsr_system* sys, int* threads, int* tile_rows);

/*
 * Learned column preconditioner (an extension: the paper scales columns by
 * their norms only, Sec. 2). The attitude and instrumental columns,
 * q in [0, 3K + n_instr) (global column 5 n_stars + q), each get 8 features;
 * an MLP 8 -> 64 -> 64 -> 1 maps the standardised features to a log
 * multiplier m_q and the column scaling becomes d_j = exp(m_q) / ||A_:,j||.
 * LSQR converges to the same least-squares solution under any positive
 * scaling, so this changes only the number of iterations.
 *
 * Parameters theta (FP32, device, GSR_MLP_NPARAM floats) are laid out as
 * W1[64][8], b1[64], W2[64][64], b2[64], w3[64], b3:
 *   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), m = w3 . h2 + b3.
 * The kernels round weights, inputs and activations (and the activation
 * gradients) to BF16 and multiply on the tensor cores with FP32 accumulation.
 * norm (device, 16 floats) = mean[8], 1/std[8]: f_std = (f - mean) * (1/std).
 * These calls run on the current CUDA device and are stream-ordered.
 */
#define GSR_MLP_NFEAT 8
#define GSR_MLP_HIDDEN 64
#define GSR_MLP_NPARAM 4801
#define GSR_MLP_GRID 296 /* most blocks gsr_mlp_grad launches */
#define GSR_MLP_WORK_FLOATS (GSR_MLP_GRID * (GSR_MLP_NPARAM + 1))

/* Number of learned columns, 3K + n_instr. */
int64_t gsr_n_learned_cols(const gsr_system* sys);
/*
 * feats (device, [3K + n_instr][8] row-major float) per column q with n_q the
 * number of rows that have a coefficient slot in the column and c_q its norm:
 *   0 log c_q (0 if c_q = 0)     4 knot / (K-1) or instrument / (n_instr-1)
 *   1 log(1 + n_q)               5 log of the block's mean count (4 n_rows/K or 6 n_rows/n_instr)
 *   2 1 if instrumental, else 0  6 log(1 + n_q) - log(1 + block mean count)
 *   3 axis / 2 (0 for instr)     7 log c_q - log(max(n_q, 1)) / 2
 * The first call also builds the per-instrument counts (library-owned).
 */
int gsr_column_features(gsr_system* sys, float* feats, void* stream);
/* acc[k] += sum_i f[i][k], acc[8 + k] += sum_i f[i][k]^2 (device double[16];
 * atomics, so the order of the additions is not fixed). */
int gsr_feature_moments(const float* feats, int64_t n, double* acc, void* stream);
/* norm (device, 16 floats) = mean[8], 1/std[8] of n feature rows from their
 * moments acc (as gsr_feature_moments leaves them); a feature with variance
 * below 1e-12 gets 1/std = 1. n > 0. */
int gsr_feature_standardisation(const double* acc, int64_t n, float* norm, void* stream);
/* m[i] = network output for feature row i (device [n]). */
int gsr_mlp_forward(const float* feats, int64_t n, const float* norm, const float* theta,
                    float* m, void* stream);
/*
 * grad = dL/dtheta of L = (1/n) sum_i (m_i - target_i)^2 and *loss = L
 * (loss may be NULL). work is device scratch of GSR_MLP_WORK_FLOATS floats.
 * Deterministic: per-block partial gradients are added in block order.
 */
int gsr_mlp_grad(const float* feats, const float* target, int64_t n, const float* norm,
                 const float* theta, float* work, float* grad, float* loss, void* stream);
/* One Adam step (Kingma & Ba) on theta with moments mom, vel (device,
 * NPARAM floats each, zero before step 1); step counts from 1. */
int gsr_mlp_adam(float* theta, const float* grad, float* mom, float* vel, int64_t step, float lr,
                 float beta1, float beta2, float eps, void* stream);
/*
 * d (device [N_unk]): exp(min(max(m_q, -clamp), clamp)) / ||A_:,j|| on the
 * learned columns, 1 / ||A_:,j|| on the others, 1 for an empty column. m
 * NULL gives plain column scaling. Pass d to gsr_lsqr_solve with
 * precond = GSR_PRECOND_USER.
 */
int gsr_learned_scaling(gsr_system* sys, const float* m, float clamp, double* d, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GSR_H */
