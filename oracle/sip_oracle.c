/*
 * sip_oracle.c -- CPU oracle for Stone's strongly implicit procedure (SIP).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant with the CUDA path in
 * paper_1303_4538_gb300/csrc, and neither side includes or links the other.
 *
 * What it computes (paper: Scheit, Hager, Treibig, Becker, Wellein,
 * "Optimization of FASTEST-3D for Modern Multicore Systems", arXiv:1303.4538):
 *   the linear solver of every equation system in FASTEST is Stone's SIP, an
 *   iteration built on an incomplete LU factorisation (Sec. 1 and Sec. 4.1,
 *   routines lu3d / resforward3d / backward3d of Tables 1-4).  The paper does
 *   not restate Stone's equations; the reading used here is the standard
 *   3-D 7-point SIP with one constant alpha (Stone 1968, the paper's ref. [HLS68]):
 *
 *   Factorisation (lu3d), for every cell P after its lower neighbours W,S,B:
 *     LB = AB / (1 + alpha (UN_B + UE_B))
 *     LW = AW / (1 + alpha (UN_W + UT_W))
 *     LS = AS / (1 + alpha (UE_S + UT_S))
 *     P1 = alpha (LB UN_B + LW UN_W)
 *     P2 = alpha (LB UE_B + LS UE_S)
 *     P3 = alpha (LW UT_W + LS UT_S)
 *     LP = AP + P1 + P2 + P3 - LB UT_B - LW UE_W - LS UN_S
 *     UN = (AN - P1) / LP,  UE = (AE - P2) / LP,  UT = (AT - P3) / LP
 *   so that L U = A + N, where N cancels (up to alpha) the six fill entries of
 *   L U by linear extrapolation from the two stencil neighbours that flank
 *   each fill position.
 *
 *   Iteration (resforward3d then backward3d):
 *     r = b - A x                             (residual; norm of r)
 *     y_P = (r_P - LB y_B - LW y_W - LS y_S) / LP   ascending cells
 *     d_P = y_P - UE d_E - UN d_N - UT d_T           descending cells
 *     x <- x + d
 *
 * Conventions:
 *   - natural layout p = i + nx*(j + ny*k), 0-based, i fastest;
 *   - lower neighbours W=(i-1,j,k), S=(i,j-1,k), B=(i,j,k-1), upper E,N,T;
 *   - A holds matrix entries: AP > 0 on the diagonal, AW..AT <= 0;
 *     the paper's Listing 1 uses the FV sign (ap fi = sum a_nb fi_nb + su),
 *     so A_nb = -a_nb, AP = ap, b = su;
 *   - a neighbour outside the block does not exist: it is skipped, never
 *     read, and its coefficient is ignored (the flat index is never used to
 *     reach across a face);
 *   - residual norm: Euclidean, relres = ||b - A x||_2 / ||b||_2 (||b|| = 0
 *     gives relres = ||r||_2).  The paper does not fix the norm.
 *   - sums of squares use Neumaier compensated summation in double so the
 *     result does not depend on the host (build with -ffp-contract=off).
 *
 * Parity status: the factorisation is pinned by the defining identity
 * L U = A + N, by alpha = 0 (ILU(0)) and by the 1-D case (exact LU); the
 * iteration by the dense preconditioned-Richardson step and by convergence to
 * the dense solution; the single-precision and refinement solve loops by
 * convergence to the FP64 solution; the single-precision solve by tracking the
 * FP64 history until it stagnates at the float level; the multi-block solve by the dense
 * global residual, the dense block-Jacobi Richardson step and convergence to
 * the dense global solution on tiny meshes.  No value printed in the paper can be
 * matched (it prints none for SIP).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ID(i, j, k) ((size_t)(i) + (size_t)nx * ((size_t)(j) + (size_t)ny * (size_t)(k)))

/* ------------------------------------------------------------------ */
/* compensated sum of squares                                           */
typedef struct { double s, c; } nsum;
static void nsum_add(nsum *a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}
static double nsum_get(const nsum *a) { return a->s + a->c; }

double oracle_dot_sq(int64_t n, const double *v) {
  nsum a = {0.0, 0.0};
  for (int64_t p = 0; p < n; ++p) nsum_add(&a, v[p] * v[p]);
  return nsum_get(&a);
}

/* ------------------------------------------------------------------ */
/* Stone factorisation (lu3d), FP64.  Returns 0, or -1 - p for the first
 * cell p where a divisor is zero or a result is not finite (breakdown). */
int oracle_factor(int nx, int ny, int nz, double alpha,
                  const double *ap, const double *aw, const double *ae, const double *as,
                  const double *an, const double *ab, const double *at,
                  double *lb, double *lw, double *ls, double *lp,
                  double *un, double *ue, double *ut) {
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t p = ID(i, j, k);
        double unB = 0, ueB = 0, utB = 0, unW = 0, ueW = 0, utW = 0, unS = 0, ueS = 0, utS = 0;
        double LB = 0, LW = 0, LS = 0;
        if (k > 0) {
          size_t q = ID(i, j, k - 1);
          unB = un[q]; ueB = ue[q]; utB = ut[q];
          double den = 1.0 + alpha * (unB + ueB);
          if (den == 0.0) return -1 - (int)p;
          LB = ab[p] / den;
        }
        if (i > 0) {
          size_t q = ID(i - 1, j, k);
          unW = un[q]; ueW = ue[q]; utW = ut[q];
          double den = 1.0 + alpha * (unW + utW);
          if (den == 0.0) return -1 - (int)p;
          LW = aw[p] / den;
        }
        if (j > 0) {
          size_t q = ID(i, j - 1, k);
          unS = un[q]; ueS = ue[q]; utS = ut[q];
          double den = 1.0 + alpha * (ueS + utS);
          if (den == 0.0) return -1 - (int)p;
          LS = as[p] / den;
        }
        double P1 = alpha * (LB * unB + LW * unW);
        double P2 = alpha * (LB * ueB + LS * ueS);
        double P3 = alpha * (LW * utW + LS * utS);
        double LP = ap[p] + P1 + P2 + P3 - LB * utB - LW * ueW - LS * unS;
        if (LP == 0.0 || !isfinite(LP)) return -1 - (int)p;
        lb[p] = LB; lw[p] = LW; ls[p] = LS; lp[p] = LP;
        /* an upper neighbour outside the block has no entry in U */
        un[p] = (j + 1 < ny) ? (an[p] - P1) / LP : 0.0;
        ue[p] = (i + 1 < nx) ? (ae[p] - P2) / LP : 0.0;
        ut[p] = (k + 1 < nz) ? (at[p] - P3) / LP : 0.0;
        if (!isfinite(LB) || !isfinite(LW) || !isfinite(LS) || !isfinite(un[p]) ||
            !isfinite(ue[p]) || !isfinite(ut[p]))
          return -1 - (int)p;
      }
  return 0;
}

/* ------------------------------------------------------------------ */
/* residual r = b - A x (general 7-point matrix); returns sum r^2.     */
double oracle_residual(int nx, int ny, int nz,
                       const double *ap, const double *aw, const double *ae, const double *as,
                       const double *an, const double *ab, const double *at,
                       const double *b, const double *x, double *r) {
  nsum acc = {0.0, 0.0};
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t p = ID(i, j, k);
        double ax = ap[p] * x[p];
        if (i > 0) ax += aw[p] * x[ID(i - 1, j, k)];
        if (i + 1 < nx) ax += ae[p] * x[ID(i + 1, j, k)];
        if (j > 0) ax += as[p] * x[ID(i, j - 1, k)];
        if (j + 1 < ny) ax += an[p] * x[ID(i, j + 1, k)];
        if (k > 0) ax += ab[p] * x[ID(i, j, k - 1)];
        if (k + 1 < nz) ax += at[p] * x[ID(i, j, k + 1)];
        double rp = b[p] - ax;
        if (r) r[p] = rp;
        nsum_add(&acc, rp * rp);
      }
  return nsum_get(&acc);
}

/* Residual of a symmetric matrix in the form of the paper's Listing 1:
 * only the east, north and top coefficients are read; the west, south and
 * bottom entries of row P are taken from the upper entries of the
 * neighbour (AW(P) = AE(W), AS(P) = AN(S), AB(P) = AT(B)).  Returns sum r^2. */
double oracle_residual_sym(int nx, int ny, int nz,
                           const double *ap, const double *ae, const double *an, const double *at,
                           const double *b, const double *x, double *r) {
  nsum acc = {0.0, 0.0};
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t p = ID(i, j, k);
        double ax = ap[p] * x[p];
        if (i + 1 < nx) ax += ae[p] * x[ID(i + 1, j, k)];
        if (i > 0) { size_t w = ID(i - 1, j, k); ax += ae[w] * x[w]; }
        if (j + 1 < ny) ax += an[p] * x[ID(i, j + 1, k)];
        if (j > 0) { size_t s = ID(i, j - 1, k); ax += an[s] * x[s]; }
        if (k + 1 < nz) ax += at[p] * x[ID(i, j, k + 1)];
        if (k > 0) { size_t q = ID(i, j, k - 1); ax += at[q] * x[q]; }
        double rp = b[p] - ax;
        if (r) r[p] = rp;
        nsum_add(&acc, rp * rp);
      }
  return nsum_get(&acc);
}

/* forward substitution L y = r (ascending lexicographic order) */
void oracle_forward(int nx, int ny, int nz, const double *lb, const double *lw,
                    const double *ls, const double *lp, const double *r, double *y) {
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t p = ID(i, j, k);
        double v = r[p];
        if (k > 0) v -= lb[p] * y[ID(i, j, k - 1)];
        if (i > 0) v -= lw[p] * y[ID(i - 1, j, k)];
        if (j > 0) v -= ls[p] * y[ID(i, j - 1, k)];
        y[p] = v / lp[p];
      }
}

/* backward substitution U d = y (descending lexicographic order) */
void oracle_backward(int nx, int ny, int nz, const double *un, const double *ue,
                     const double *ut, const double *y, double *d) {
  for (int k = nz - 1; k >= 0; --k)
    for (int j = ny - 1; j >= 0; --j)
      for (int i = nx - 1; i >= 0; --i) {
        size_t p = ID(i, j, k);
        double v = y[p];
        if (i + 1 < nx) v -= ue[p] * d[ID(i + 1, j, k)];
        if (j + 1 < ny) v -= un[p] * d[ID(i, j + 1, k)];
        if (k + 1 < nz) v -= ut[p] * d[ID(i, j, k + 1)];
        d[p] = v;
      }
}

/* One SIP iteration on x (in place).  r, y and d are work arrays of n
 * doubles (residual, forward result, correction).  Returns ||b - A x_in||^2. */
double oracle_iterate(int nx, int ny, int nz,
                      const double *ap, const double *aw, const double *ae, const double *as,
                      const double *an, const double *ab, const double *at,
                      const double *lb, const double *lw, const double *ls, const double *lp,
                      const double *un, const double *ue, const double *ut,
                      const double *b, double *x, double *r, double *y, double *d) {
  size_t n = (size_t)nx * ny * nz;
  double rr = oracle_residual(nx, ny, nz, ap, aw, ae, as, an, ab, at, b, x, r);
  oracle_forward(nx, ny, nz, lb, lw, ls, lp, r, y);
  oracle_backward(nx, ny, nz, un, ue, ut, y, d);
  for (size_t p = 0; p < n; ++p) x[p] += d[p];
  return rr;
}

/* SIP to a relative residual.  Stop rule: with relres(x_n) computed from the
 * residual of x_n, stop as soon as relres(x_n) <= rtol or n == max_iters;
 * x_n is returned.  hist (nullable, max_iters+1 doubles) receives relres(x_0..x_n).
 * Returns n (number of updates applied); *relres_out = relres(x_n). */
int oracle_solve(int nx, int ny, int nz,
                 const double *ap, const double *aw, const double *ae, const double *as,
                 const double *an, const double *ab, const double *at,
                 const double *lb, const double *lw, const double *ls, const double *lp,
                 const double *un, const double *ue, const double *ut,
                 const double *b, double *x, double rtol, int max_iters,
                 double *hist, double *relres_out) {
  size_t n = (size_t)nx * ny * nz;
  double *r = (double *)malloc(n * sizeof(double));
  double *y = (double *)malloc(n * sizeof(double));
  double *d = (double *)malloc(n * sizeof(double));
  double bb = sqrt(oracle_dot_sq((int64_t)n, b));
  double scale = bb > 0.0 ? bb : 1.0;
  int it = 0;
  double rel = 0.0;
  for (;;) {
    double rr = oracle_residual(nx, ny, nz, ap, aw, ae, as, an, ab, at, b, x, r);
    rel = sqrt(rr) / scale;
    if (hist) hist[it] = rel;
    if (rel <= rtol || it >= max_iters) break;
    oracle_forward(nx, ny, nz, lb, lw, ls, lp, r, y);
    oracle_backward(nx, ny, nz, un, ue, ut, y, d);
    for (size_t p = 0; p < n; ++p) x[p] += d[p];
    ++it;
  }
  free(r); free(y); free(d);
  if (relres_out) *relres_out = rel;
  return it;
}

/* ------------------------------------------------------------------ */
/* Single precision.  The same steps in float arithmetic on float copies of
 * A, of the factors (rounded from the FP64 factors) and of b and x.  This is
 * the arithmetic of the paper's single-precision relaxation (Sec. 4.1: rhs and
 * solution converted to single, relaxed in single, converted back). */
#define IDF ID
static void f32_residual(int nx, int ny, int nz, const float *ap, const float *aw,
                         const float *ae, const float *as, const float *an, const float *ab,
                         const float *at, const float *b, const float *x, float *r, int x_is_zero) {
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t p = IDF(i, j, k);
        if (x_is_zero) { r[p] = b[p]; continue; }
        float ax = ap[p] * x[p];
        if (i > 0) ax += aw[p] * x[IDF(i - 1, j, k)];
        if (i + 1 < nx) ax += ae[p] * x[IDF(i + 1, j, k)];
        if (j > 0) ax += as[p] * x[IDF(i, j - 1, k)];
        if (j + 1 < ny) ax += an[p] * x[IDF(i, j + 1, k)];
        if (k > 0) ax += ab[p] * x[IDF(i, j, k - 1)];
        if (k + 1 < nz) ax += at[p] * x[IDF(i, j, k + 1)];
        r[p] = b[p] - ax;
      }
}
static void f32_forward(int nx, int ny, int nz, const float *lb, const float *lw,
                        const float *ls, const float *lp, const float *r, float *y) {
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t p = IDF(i, j, k);
        float v = r[p];
        if (k > 0) v -= lb[p] * y[IDF(i, j, k - 1)];
        if (i > 0) v -= lw[p] * y[IDF(i - 1, j, k)];
        if (j > 0) v -= ls[p] * y[IDF(i, j - 1, k)];
        y[p] = v / lp[p];
      }
}
static void f32_backward(int nx, int ny, int nz, const float *un, const float *ue,
                         const float *ut, const float *y, float *d) {
  for (int k = nz - 1; k >= 0; --k)
    for (int j = ny - 1; j >= 0; --j)
      for (int i = nx - 1; i >= 0; --i) {
        size_t p = IDF(i, j, k);
        float v = y[p];
        if (i + 1 < nx) v -= ue[p] * d[IDF(i + 1, j, k)];
        if (j + 1 < ny) v -= un[p] * d[IDF(i, j + 1, k)];
        if (k + 1 < nz) v -= ut[p] * d[IDF(i, j, k + 1)];
        d[p] = v;
      }
}

/* One single-precision SIP iteration on x (in place); r, y, d: float work. */
void oracle_iterate_f32(int nx, int ny, int nz,
                        const float *ap, const float *aw, const float *ae, const float *as,
                        const float *an, const float *ab, const float *at,
                        const float *lb, const float *lw, const float *ls, const float *lp,
                        const float *un, const float *ue, const float *ut,
                        const float *b, float *x, int x_is_zero, float *r, float *y, float *d) {
  size_t n = (size_t)nx * ny * nz;
  f32_residual(nx, ny, nz, ap, aw, ae, as, an, ab, at, b, x, r, x_is_zero);
  f32_forward(nx, ny, nz, lb, lw, ls, lp, r, y);
  f32_backward(nx, ny, nz, un, ue, ut, y, d);
  for (size_t p = 0; p < n; ++p) x[p] = (x_is_zero ? 0.0f : x[p]) + d[p];
}

/* ------------------------------------------------------------------ */
/* Mixed precision: FP64 outer iterative refinement around single-precision
 * SIP sweeps.  Outer step: r = b - A64 x in double, relres from it; stop as
 * in oracle_solve; otherwise r32 = (float) r, m single-precision SIP
 * iterations on A32 d = r32 starting from d = 0, then x += (double) d.
 * Returns the number of outer corrections applied; hist (nullable,
 * max_outer+1) receives the FP64 relres before each correction. */
int oracle_solve_refined(int nx, int ny, int nz,
                         const double *ap, const double *aw, const double *ae, const double *as,
                         const double *an, const double *ab, const double *at,
                         const float *ap32, const float *aw32, const float *ae32, const float *as32,
                         const float *an32, const float *ab32, const float *at32,
                         const float *lb32, const float *lw32, const float *ls32, const float *lp32,
                         const float *un32, const float *ue32, const float *ut32,
                         const double *b, double *x, double rtol, int max_outer, int m_inner,
                         double *hist, double *relres_out) {
  size_t n = (size_t)nx * ny * nz;
  double *r = (double *)malloc(n * sizeof(double));
  float *r32 = (float *)malloc(n * sizeof(float));
  float *d32 = (float *)malloc(n * sizeof(float));
  float *w1 = (float *)malloc(n * sizeof(float));
  float *w2 = (float *)malloc(n * sizeof(float));
  float *w3 = (float *)malloc(n * sizeof(float));
  double bb = sqrt(oracle_dot_sq((int64_t)n, b));
  double scale = bb > 0.0 ? bb : 1.0;
  int it = 0;
  double rel = 0.0;
  for (;;) {
    double rr = oracle_residual(nx, ny, nz, ap, aw, ae, as, an, ab, at, b, x, r);
    rel = sqrt(rr) / scale;
    if (hist) hist[it] = rel;
    if (rel <= rtol || it >= max_outer) break;
    for (size_t p = 0; p < n; ++p) r32[p] = (float)r[p];
    for (int m = 0; m < m_inner; ++m)
      oracle_iterate_f32(nx, ny, nz, ap32, aw32, ae32, as32, an32, ab32, at32, lb32, lw32, ls32,
                         lp32, un32, ue32, ut32, r32, d32, m == 0, w1, w2, w3);
    for (size_t p = 0; p < n; ++p) x[p] += (double)d32[p];
    ++it;
  }
  free(r); free(r32); free(d32); free(w1); free(w2); free(w3);
  if (relres_out) *relres_out = rel;
  return it;
}

/* ------------------------------------------------------------------ */
/* Several blocks coupled across x interfaces (the paper's block-structured
 * mesh, Sec. 1; blocks exchange boundary data, Sec. 4.2).  Reading: lagged
 * block Jacobi -- every block relaxes with its own factors and with the
 * neighbour values of the previous exchange.
 *
 * Block b: dims[3b..3b+2] = nx, ny, nz; A[7b+q] = ap, aw, ae, as, an, ab, at;
 * F[7b+q] = lb, lw, ls, lp, un, ue, ut (its own factorisation); B[b] rhs;
 * X[b] solution (in: x0, out: x_n).  Interface q: ifc[4q..4q+3] = lo, hi,
 * nj, nk: cell (nx_lo - 1, j, k) of block lo and cell (0, j, k) of block hi
 * are neighbours for j < nj, k < nk; the coupling entries are lo's AE there
 * and hi's AW there (sym != 0: hi's entry is lo's AE, the matrix being
 * symmetric).
 *
 * Iteration: with every block's current x,
 *   beff_b = b_b - sum over the interfaces of b of (entry) * x_neighbour
 *   r_b    = beff_b - A_b x_b  (A_b: the block's own entries; an entry that
 *            points outside the block is not used)
 * is the residual of the whole coupled system; relres = sqrt(sum_b ||r_b||^2)
 * / sqrt(sum_b ||b_b||^2) with the stop rule of oracle_solve; otherwise every
 * block applies y = L^-1 r_b, d = U^-1 y, x_b += d.  Returns n; hist
 * (nullable, max_iters + 1) gets relres(x_0..x_n). */
int oracle_solve_mb(int nb, const int *dims, const double *const *A, const double *const *F,
                    const double *const *B, double *const *X, int nif, const int *ifc, int sym,
                    double rtol, int max_iters, double *hist, double *relres_out) {
  size_t nmax = 0;
  for (int b = 0; b < nb; ++b) {
    size_t n = (size_t)dims[3 * b] * dims[3 * b + 1] * dims[3 * b + 2];
    if (n > nmax) nmax = n;
  }
  double **beff = (double **)malloc(sizeof(double *) * nb);
  double **r = (double **)malloc(sizeof(double *) * nb);
  double *y = (double *)malloc(nmax * sizeof(double));
  double *d = (double *)malloc(nmax * sizeof(double));
  nsum bsum = {0.0, 0.0};
  for (int b = 0; b < nb; ++b) {
    size_t n = (size_t)dims[3 * b] * dims[3 * b + 1] * dims[3 * b + 2];
    beff[b] = (double *)malloc(n * sizeof(double));
    r[b] = (double *)malloc(n * sizeof(double));
    nsum_add(&bsum, oracle_dot_sq((int64_t)n, B[b]));
  }
  double bb = sqrt(nsum_get(&bsum));
  double scale = bb > 0.0 ? bb : 1.0;
  int it = 0;
  double rel = 0.0;
  for (;;) {
    for (int b = 0; b < nb; ++b) {
      size_t n = (size_t)dims[3 * b] * dims[3 * b + 1] * dims[3 * b + 2];
      memcpy(beff[b], B[b], n * sizeof(double));
    }
    for (int q = 0; q < nif; ++q) {
      int lo = ifc[4 * q], hi = ifc[4 * q + 1], nj = ifc[4 * q + 2], nk = ifc[4 * q + 3];
      int nxl = dims[3 * lo], nyl = dims[3 * lo + 1];
      int nxh = dims[3 * hi], nyh = dims[3 * hi + 1];
      const double *ae_lo = A[7 * lo + 2];
      const double *aw_hi = sym ? NULL : A[7 * hi + 1];
      for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nj; ++j) {
          size_t pl = (size_t)(nxl - 1) + (size_t)nxl * ((size_t)j + (size_t)nyl * k);
          size_t ph = (size_t)nxh * ((size_t)j + (size_t)nyh * k);
          double elo = ae_lo[pl];
          double ehi = sym ? elo : aw_hi[ph];
          beff[lo][pl] -= elo * X[hi][ph];
          beff[hi][ph] -= ehi * X[lo][pl];
        }
    }
    nsum rs = {0.0, 0.0};
    for (int b = 0; b < nb; ++b) {
      int nx = dims[3 * b], ny = dims[3 * b + 1], nz = dims[3 * b + 2];
      const double *const *a = A + 7 * b;
      nsum_add(&rs, oracle_residual(nx, ny, nz, a[0], a[1], a[2], a[3], a[4], a[5], a[6], beff[b], X[b], r[b]));
    }
    rel = sqrt(nsum_get(&rs)) / scale;
    if (hist) hist[it] = rel;
    if (rel <= rtol || it >= max_iters) break;
    for (int b = 0; b < nb; ++b) {
      int nx = dims[3 * b], ny = dims[3 * b + 1], nz = dims[3 * b + 2];
      size_t n = (size_t)nx * ny * nz;
      const double *const *f = F + 7 * b;
      oracle_forward(nx, ny, nz, f[0], f[1], f[2], f[3], r[b], y);
      oracle_backward(nx, ny, nz, f[4], f[5], f[6], y, d);
      for (size_t p = 0; p < n; ++p) X[b][p] += d[p];
    }
    ++it;
  }
  for (int b = 0; b < nb; ++b) { free(beff[b]); free(r[b]); }
  free(beff); free(r); free(y); free(d);
  if (relres_out) *relres_out = rel;
  return it;
}

/* ------------------------------------------------------------------ */
/* The paper's single-precision relaxation (Sec. 4.1): right-hand side and
 * solution converted to float, every SIP step in float with float copies of
 * A and of the factors, x converted back at the end.  relres(x_n) is computed
 * from the float residual (its squares summed in double) over ||b||_2 of the
 * double right-hand side; stop rule as oracle_solve.  Returns n; hist
 * (nullable, max_iters + 1) gets relres(x_0..x_n). */
int oracle_solve_f32(int nx, int ny, int nz,
                     const float *ap, const float *aw, const float *ae, const float *as,
                     const float *an, const float *ab, const float *at,
                     const float *lb, const float *lw, const float *ls, const float *lp,
                     const float *un, const float *ue, const float *ut,
                     const double *b, double *x, double rtol, int max_iters,
                     double *hist, double *relres_out) {
  size_t n = (size_t)nx * ny * nz;
  float *b32 = (float *)malloc(n * sizeof(float));
  float *x32 = (float *)malloc(n * sizeof(float));
  float *r = (float *)malloc(n * sizeof(float));
  float *y = (float *)malloc(n * sizeof(float));
  float *d = (float *)malloc(n * sizeof(float));
  for (size_t p = 0; p < n; ++p) {
    b32[p] = (float)b[p];
    x32[p] = (float)x[p];
  }
  double bb = sqrt(oracle_dot_sq((int64_t)n, b));
  double scale = bb > 0.0 ? bb : 1.0;
  int it = 0;
  double rel = 0.0;
  for (;;) {
    f32_residual(nx, ny, nz, ap, aw, ae, as, an, ab, at, b32, x32, r, 0);
    nsum acc = {0.0, 0.0};
    for (size_t p = 0; p < n; ++p) nsum_add(&acc, (double)r[p] * (double)r[p]);
    rel = sqrt(nsum_get(&acc)) / scale;
    if (hist) hist[it] = rel;
    if (rel <= rtol || it >= max_iters) break;
    f32_forward(nx, ny, nz, lb, lw, ls, lp, r, y);
    f32_backward(nx, ny, nz, un, ue, ut, y, d);
    for (size_t p = 0; p < n; ++p) x32[p] += d[p];
    ++it;
  }
  for (size_t p = 0; p < n; ++p) x[p] = (double)x32[p];
  free(b32); free(x32); free(r); free(y); free(d);
  if (relres_out) *relres_out = rel;
  return it;
}

/* ------------------------------------------------------------------ */
/* The mixed-precision refinement (oracle_solve_refined) over blocks coupled
 * across x interfaces (oracle_solve_mb's mesh, arguments and lagged
 * block-Jacobi reading; Sec. 4.1 single-precision solver, Sec. 4.2 exchange
 * of block-boundary data between iterations).  Reading for the inner
 * iterations: the correction system is the coupled one, A d = r, and the
 * blocks exchange their interface values of d after every inner iteration.
 *
 * Outer step: the coupled FP64 residual r_b of every block exactly as in
 * oracle_solve_mb (A: FP64 entries), relres and the stop rule of
 * oracle_solve; otherwise r32_b = (float) r_b, d_b = 0 and m_inner inner
 * iterations, each
 *   c_b = r32_b - sum over the interfaces of b of e32 * d_neighbour
 *         (float arithmetic, every product and difference rounded to float;
 *          e32: the interface entry of A32, lo's AE32 / hi's AW32, or lo's
 *          AE32 for both when sym != 0; d from the previous inner iteration
 *          of all blocks, so the first inner iteration sees c_b = r32_b),
 * then for every block one single-precision SIP iteration on A32_b d_b = c_b
 * from the current d_b (oracle_iterate_f32, from zero in the first), and
 * finally x_b += (double) d_b.
 * A: FP64 entries, 7 per block; A32: FP32 entries, 7 per block; F32: FP32
 * factors lb, lw, ls, lp, un, ue, ut, 7 per block.  Returns the number of
 * outer corrections; hist (nullable, max_outer + 1) gets relres before each. */
int oracle_solve_refined_mb(int nb, const int *dims, const double *const *A, const float *const *A32,
                            const float *const *F32, const double *const *B, double *const *X, int nif,
                            const int *ifc, int sym, double rtol, int max_outer, int m_inner, double *hist,
                            double *relres_out) {
  size_t nmax = 0;
  for (int b = 0; b < nb; ++b) {
    size_t n = (size_t)dims[3 * b] * dims[3 * b + 1] * dims[3 * b + 2];
    if (n > nmax) nmax = n;
  }
  double **beff = (double **)malloc(sizeof(double *) * nb);
  double **r = (double **)malloc(sizeof(double *) * nb);
  float **r32 = (float **)malloc(sizeof(float *) * nb);
  float **c32 = (float **)malloc(sizeof(float *) * nb);
  float **d32 = (float **)malloc(sizeof(float *) * nb);
  float *w1 = (float *)malloc(nmax * sizeof(float));
  float *w2 = (float *)malloc(nmax * sizeof(float));
  float *w3 = (float *)malloc(nmax * sizeof(float));
  nsum bsum = {0.0, 0.0};
  for (int b = 0; b < nb; ++b) {
    size_t n = (size_t)dims[3 * b] * dims[3 * b + 1] * dims[3 * b + 2];
    beff[b] = (double *)malloc(n * sizeof(double));
    r[b] = (double *)malloc(n * sizeof(double));
    r32[b] = (float *)malloc(n * sizeof(float));
    c32[b] = (float *)malloc(n * sizeof(float));
    d32[b] = (float *)malloc(n * sizeof(float));
    nsum_add(&bsum, oracle_dot_sq((int64_t)n, B[b]));
  }
  double bb = sqrt(nsum_get(&bsum));
  double scale = bb > 0.0 ? bb : 1.0;
  int it = 0;
  double rel = 0.0;
  for (;;) {
    /* coupled FP64 residual of x (as oracle_solve_mb) */
    for (int b = 0; b < nb; ++b) {
      size_t n = (size_t)dims[3 * b] * dims[3 * b + 1] * dims[3 * b + 2];
      memcpy(beff[b], B[b], n * sizeof(double));
    }
    for (int q = 0; q < nif; ++q) {
      int lo = ifc[4 * q], hi = ifc[4 * q + 1], nj = ifc[4 * q + 2], nk = ifc[4 * q + 3];
      int nxl = dims[3 * lo], nyl = dims[3 * lo + 1];
      int nxh = dims[3 * hi], nyh = dims[3 * hi + 1];
      for (int k = 0; k < nk; ++k)
        for (int j = 0; j < nj; ++j) {
          size_t pl = (size_t)(nxl - 1) + (size_t)nxl * ((size_t)j + (size_t)nyl * k);
          size_t ph = (size_t)nxh * ((size_t)j + (size_t)nyh * k);
          double elo = A[7 * lo + 2][pl];
          double ehi = sym ? elo : A[7 * hi + 1][ph];
          beff[lo][pl] -= elo * X[hi][ph];
          beff[hi][ph] -= ehi * X[lo][pl];
        }
    }
    nsum rs = {0.0, 0.0};
    for (int b = 0; b < nb; ++b) {
      int nx = dims[3 * b], ny = dims[3 * b + 1], nz = dims[3 * b + 2];
      const double *const *a = A + 7 * b;
      nsum_add(&rs, oracle_residual(nx, ny, nz, a[0], a[1], a[2], a[3], a[4], a[5], a[6], beff[b], X[b], r[b]));
    }
    rel = sqrt(nsum_get(&rs)) / scale;
    if (hist) hist[it] = rel;
    if (rel <= rtol || it >= max_outer) break;
    for (int b = 0; b < nb; ++b) {
      size_t n = (size_t)dims[3 * b] * dims[3 * b + 1] * dims[3 * b + 2];
      for (size_t p = 0; p < n; ++p) {
        r32[b][p] = (float)r[b][p];
        d32[b][p] = 0.0f;
      }
    }
    for (int m = 0; m < m_inner; ++m) {
      /* exchange: interface terms of the previous inner iteration's d */
      for (int b = 0; b < nb; ++b) {
        size_t n = (size_t)dims[3 * b] * dims[3 * b + 1] * dims[3 * b + 2];
        memcpy(c32[b], r32[b], n * sizeof(float));
      }
      for (int q = 0; q < nif; ++q) {
        int lo = ifc[4 * q], hi = ifc[4 * q + 1], nj = ifc[4 * q + 2], nk = ifc[4 * q + 3];
        int nxl = dims[3 * lo], nyl = dims[3 * lo + 1];
        int nxh = dims[3 * hi], nyh = dims[3 * hi + 1];
        for (int k = 0; k < nk; ++k)
          for (int j = 0; j < nj; ++j) {
            size_t pl = (size_t)(nxl - 1) + (size_t)nxl * ((size_t)j + (size_t)nyl * k);
            size_t ph = (size_t)nxh * ((size_t)j + (size_t)nyh * k);
            float elo = A32[7 * lo + 2][pl];
            float ehi = sym ? elo : A32[7 * hi + 1][ph];
            float tl = elo * d32[hi][ph];
            float th = ehi * d32[lo][pl];
            c32[lo][pl] = c32[lo][pl] - tl;
            c32[hi][ph] = c32[hi][ph] - th;
          }
      }
      /* one single-precision SIP iteration per block */
      for (int b = 0; b < nb; ++b) {
        int nx = dims[3 * b], ny = dims[3 * b + 1], nz = dims[3 * b + 2];
        const float *const *a = A32 + 7 * b;
        const float *const *f = F32 + 7 * b;
        oracle_iterate_f32(nx, ny, nz, a[0], a[1], a[2], a[3], a[4], a[5], a[6], f[0], f[1], f[2], f[3], f[4],
                           f[5], f[6], c32[b], d32[b], m == 0, w1, w2, w3);
      }
    }
    for (int b = 0; b < nb; ++b) {
      size_t n = (size_t)dims[3 * b] * dims[3 * b + 1] * dims[3 * b + 2];
      for (size_t p = 0; p < n; ++p) X[b][p] += (double)d32[b][p];
    }
    ++it;
  }
  for (int b = 0; b < nb; ++b) {
    free(beff[b]); free(r[b]); free(r32[b]); free(c32[b]); free(d32[b]);
  }
  free(beff); free(r); free(r32); free(c32); free(d32); free(w1); free(w2); free(w3);
  if (relres_out) *relres_out = rel;
  return it;
}

/* ------------------------------------------------------------------ */
/* Pressure-correction coefficient assembly (the routine celp2 of Sec. 3.1,
 * Table 1, whose symmetric system Sec. 4.1 solves; the paper does not print
 * its discretisation).  Reading (an invented, stated FV geometry): a block of
 * nx x ny x nz hexahedral cells on a rectilinear grid with cell widths
 * dx[i], dy[j], dz[k]; per cell a density rho and the momentum equation's
 * V / a_P ("g"); face-normal velocities u* on every face (ux: (nx+1) ny nz
 * faces, face i the west face of cell i, index (k ny + j)(nx+1) + i; uy:
 * nx (ny+1) nz, index (k (ny+1) + j) nx + i; uz: nx ny (nz+1), index
 * (k ny + j) nx + i).  The SIMPLE-type pressure-correction equation
 * -div(rho g grad p') = -div(rho u*) in finite volumes:
 *   interior face f between P and N:
 *     rho_f = (rho_P + rho_N) * 0.5,  g_f = (g_P + g_N) * 0.5,
 *     rdelta_f = 1 / ((w_P + w_N) * 0.5)  (w: the cells' widths along the
 *       face normal; the reciprocal centre distance, a geometric factor of the
 *       face that depends on one axis only),
 *     S_f = the face area (dy dz, dx dz or dx dy of P),
 *     A_N(P) = -(((rho_f * g_f) * S_f) * rdelta_f);
 *   boundary faces are walls (coefficient 0), except the k = 0 face when
 *   dirichlet_bottom != 0 (p' = 0 beyond it): it adds
 *     cB = ((rho_P * g_P) * S_z) * (1 / (dz[0] * 0.5)) to AP;
 *   AP = ((((((-AW) + (-AE)) + (-AS)) + (-AN)) + (-AB)) + (-AT)) + cB;
 *   mass fluxes F_f = (rho_f * u*_f) * S_f (boundary faces: rho_f = rho_P),
 *   b = -(((((F_e - F_w) + F_n) - F_s) + F_t) - F_b), the negative net outflow.
 * All in double, in exactly that order. */
void oracle_assemble_pcorr(int nx, int ny, int nz, const double *dx, const double *dy, const double *dz,
                           const double *rho, const double *g, const double *ux, const double *uy,
                           const double *uz, int dirichlet_bottom, double *ap, double *aw, double *ae,
                           double *as, double *an, double *ab, double *at, double *b) {
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        size_t p = (size_t)i + (size_t)nx * ((size_t)j + (size_t)ny * k);
        double Sx = dy[j] * dz[k], Sy = dx[i] * dz[k], Sz = dx[i] * dy[j];
        /* neighbour cell indices and widths along each axis */
        double c[6] = {0, 0, 0, 0, 0, 0}; /* W E S N B T coefficients */
        double rf[6];                      /* face densities for the fluxes */
        int has[6] = {i > 0, i < nx - 1, j > 0, j < ny - 1, k > 0, k < nz - 1};
        size_t nb[6] = {p - 1, p + 1, p - (size_t)nx, p + (size_t)nx, p - (size_t)nx * ny, p + (size_t)nx * ny};
        double w[6], S[6] = {Sx, Sx, Sy, Sy, Sz, Sz};
        w[0] = has[0] ? dx[i - 1] : 0.0;
        w[1] = has[1] ? dx[i + 1] : 0.0;
        w[2] = has[2] ? dy[j - 1] : 0.0;
        w[3] = has[3] ? dy[j + 1] : 0.0;
        w[4] = has[4] ? dz[k - 1] : 0.0;
        w[5] = has[5] ? dz[k + 1] : 0.0;
        double wp[6] = {dx[i], dx[i], dy[j], dy[j], dz[k], dz[k]};
        for (int f = 0; f < 6; ++f) {
          if (has[f]) {
            double rhof = (rho[p] + rho[nb[f]]) * 0.5;
            double gf = (g[p] + g[nb[f]]) * 0.5;
            double rdelta = 1.0 / ((wp[f] + w[f]) * 0.5);
            c[f] = -(((rhof * gf) * S[f]) * rdelta);
            rf[f] = rhof;
          } else {
            rf[f] = rho[p];
          }
        }
        double cB = 0.0;
        if (k == 0 && dirichlet_bottom) cB = ((rho[p] * g[p]) * Sz) * (1.0 / (dz[0] * 0.5));
        aw[p] = c[0];
        ae[p] = c[1];
        as[p] = c[2];
        an[p] = c[3];
        ab[p] = c[4];
        at[p] = c[5];
        ap[p] = ((((((-c[0]) + (-c[1])) + (-c[2])) + (-c[3])) + (-c[4])) + (-c[5])) + cB;
        /* face velocities: west / east (x), south / north (y), bottom / top (z) */
        double uw = ux[((size_t)k * ny + j) * (size_t)(nx + 1) + i];
        double ue = ux[((size_t)k * ny + j) * (size_t)(nx + 1) + i + 1];
        double us = uy[((size_t)k * (ny + 1) + j) * (size_t)nx + i];
        double un = uy[((size_t)k * (ny + 1) + j + 1) * (size_t)nx + i];
        double ub = uz[((size_t)k * ny + j) * (size_t)nx + i];
        double ut = uz[((size_t)(k + 1) * ny + j) * (size_t)nx + i];
        double Fw = (rf[0] * uw) * Sx, Fe = (rf[1] * ue) * Sx;
        double Fs = (rf[2] * us) * Sy, Fn = (rf[3] * un) * Sy;
        double Fb = (rf[4] * ub) * Sz, Ft = (rf[5] * ut) * Sz;
        b[p] = -(((((Fe - Fw) + Fn) - Fs) + Ft) - Fb);
      }
}
