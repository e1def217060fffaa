/*
 * hc_oracle.c -- plain FP64 CPU oracle for one time step of the Fourier
 * spectral FFT+CG splitting scheme of arXiv 2606.06720 (Section 2, Algorithm 1).
 *
 * TEST INFRASTRUCTURE: it exists to check the GPU path and is never part of it.
 * It is deliberately slow and literal: full complex transforms (no half
 * spectrum), a textbook radix-2 FFT plus a direct DFT for any other length,
 * physical-space CG, and the substeps written in the paper's own form.
 *
 * Readings of the paper where it is silent or ambiguous (labels R1..R11 are
 * the ones used throughout the project):
 *   R1  first-derivative multiplier i*xi is zero at the Nyquist index, which is
 *       the same as taking the real part of F^-1[i xi F f] with the paper's
 *       positive Nyquist xi;
 *   R2  the null space of the discrete operator is spanned by the 2^dim corner
 *       modes (every index 0 or N/2); S, p and the CG iterates are kept
 *       orthogonal to it;
 *   R3  preconditioner: a constant-coefficient operator -div(Kbar grad) built
 *       from the same derivative symbols and inverted on the non-null modes,
 *       with Kbar = kappa I, kappa = mean(r) + mean(|m|^2)/dim (the isotropic
 *       part of the mean of K = m m^T + r I); option precond = 1 takes the
 *       whole mean, Kbar = mean(m m^T) + mean(r) I; a user kappa > 0 gives
 *       Kbar = kappa I;
 *   R4  CG stops when ||res||_2 <= rtol ||S||_2 (plain Euclidean norms);
 *   R5  p^0 = 0 unless the caller supplies one;
 *   R6  the activation uses grad p^{k+1} (Algorithm 1 solves for p first);
 *   R7  relaxation edge cases as printed: gamma == 1, |m| == 0, indicator b >= 0;
 *   R8  in 3D the perpendicular projector g_perp g_perp^T / |g|^2 is I - g g^T/|g|^2;
 *   R10 discrete L2 norms in the energy carry the quadrature weight h_x h_y [h_z];
 *   R11 Lie splitting, every substep with the full dt, order A -> R -> D;
 *   R21 at gamma = 0 the energy's relaxation term |m|^(2 gamma)/(2 gamma) is
 *       1/0; the energy takes its gradient-flow limit there, sum h ln|m|
 *       ((|m|^(2 gamma) - 1)/(2 gamma) -> ln|m|, whose m-gradient m/|m|^2 is the
 *       gamma = 0 relaxation term of eq. (1.1b); the constant |Omega|/(2 gamma)
 *       is dropped).  A point with m = 0 makes it -inf.
 *
 * What pins each function (tests/test_oracle_*.py). Every value there comes
 * from the mathematics or a library routine, not from this file. No function
 * is parity unpinned.
 *   or_dft1, or_fft1, or_fftn  the DFT's definition summed directly; numpy's FFT;
 *                              Parseval and the round trip on random grids.
 *   or_xi, or_xi_deriv         the wavenumber table of Section 2.3.3, worked by hand.
 *   or_gradient                exact derivatives of trigonometric polynomials, 2D and 3D.
 *   or_apply_K, or_apply_A     the tensor's eigenvectors; constant-coefficient closed forms;
 *                              a sympy manufactured solution; dense assembly (symmetric,
 *                              semi-definite, the 2^dim corner null modes); hand-worked
 *                              variable-coefficient cases.
 *   or_project                 the null space of the assembled operator (eigen- or singular
 *                              vectors), odd grids included; idempotent and orthogonal.
 *   or_precond, or_kbar_default, or_kappa_default
 *                              one CG iteration when the coefficient is constant; a 3D
 *                              eigenfunction; hand-worked kappa and Kbar.
 *   or_pcg                     numpy's least-squares solution; condition-number iteration
 *                              bounds; exact invariance under a power-of-two scaling of S;
 *                              the reported residual recomputed.
 *   or_activation              scipy's matrix exponential; RK4; hand-worked projector-form cases.
 *   or_relaxation              closed forms (gamma = 1, 1/2); RK4 of the radial equation;
 *                              hand-worked cases in every regime.
 *   or_diffusion               single-mode decay, the Nyquist mode included, 2D and 3D.
 *   or_step                    the energy identity; energy decrease for small dt; symmetries;
 *                              special cases; the order of Algorithm 1.
 *   or_energy                  hand-worked values of every term.
 *   or_adjoint                 finite differences of the forward map: 2D and 3D, every
 *                              relaxation branch, m = 0 and extinction, c = 0.
 * tests/test_pins_catch_mutants.py plants mistakes in copies of this file and
 * requires each to fail some pin.
 */
#include "hc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int g_threads = 1;

void or_set_threads(int nthreads) { g_threads = nthreads > 0 ? nthreads : 1; }
int or_get_threads(void) { return g_threads; }

size_t or_npts(const or_grid* g) {
  size_t n = 1;
  for (int a = 0; a < g->dim; ++a) n *= (size_t)g->n[a];
  return n;
}

static int valid_grid(const or_grid* g) {
  if (!g || (g->dim != 2 && g->dim != 3)) return 0;
  for (int a = 0; a < g->dim; ++a)
    if (g->n[a] < 1 || !(g->L[a] > 0)) return 0;
  return 1;
}

/* ------------------------------------------------------------------ */
/* Transforms                                                          */
/* ------------------------------------------------------------------ */

/* Direct DFT from its definition: out_k = sum_j in_j exp(sign 2 pi i j k / n). */
int or_dft1(const double complex* in, double complex* out, int n, int sign) {
  if (n < 1 || (sign != 1 && sign != -1)) return OR_EINVAL;
  for (int k = 0; k < n; ++k) {
    double complex s = 0;
    for (int j = 0; j < n; ++j) {
      long long jk = ((long long)j * k) % n; /* reduce first: keeps the angle exact */
      double ang = sign * 2.0 * M_PI * (double)jk / n;
      s += in[j] * (cos(ang) + I * sin(ang));
    }
    out[k] = s;
  }
  return OR_OK;
}

static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

/* Table w[k] = exp(sign 2 pi i k / n), k < n/2, each entry from libm directly. */
static double complex* twiddles(int n, int sign) {
  int h = n / 2 > 0 ? n / 2 : 1;
  double complex* w = (double complex*)malloc(sizeof(double complex) * h);
  if (!w) return NULL;
  for (int k = 0; k < h; ++k) {
    double ang = sign * 2.0 * M_PI * (double)k / n;
    w[k] = cos(ang) + I * sin(ang);
  }
  return w;
}

/* Textbook iterative radix-2 Cooley-Tukey: bit-reversal, then log2(n) stages. */
static void fft_pow2(double complex* a, int n, const double complex* w) {
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double complex t = a[i];
      a[i] = a[j];
      a[j] = t;
    }
  }
  for (int len = 2; len <= n; len <<= 1) {
    int half = len / 2, step = n / len;
    for (int s = 0; s < n; s += len)
      for (int k = 0; k < half; ++k) {
        double complex u = a[s + k];
        double complex v = a[s + k + half] * w[k * step];
        a[s + k] = u + v;
        a[s + k + half] = u - v;
      }
  }
}

int or_fft1(double complex* a, int n, int sign) {
  if (n < 1 || (sign != 1 && sign != -1)) return OR_EINVAL;
  if (n == 1) return OR_OK;
  if (is_pow2(n)) {
    double complex* w = twiddles(n, sign);
    if (!w) return OR_ENOMEM;
    fft_pow2(a, n, w);
    free(w);
    return OR_OK;
  }
  /* any other length: the direct definition */
  double complex* tmp = (double complex*)malloc(sizeof(double complex) * n);
  if (!tmp) return OR_ENOMEM;
  int rc = or_dft1(a, tmp, n, sign);
  memcpy(a, tmp, sizeof(double complex) * n);
  free(tmp);
  return rc;
}

/* Transform every line along axis `ax` (stride = product of lower extents). */
static int fft_axis(const or_grid* g, double complex* a, int ax, int sign) {
  int n = g->n[ax];
  if (n == 1) return OR_OK;
  size_t npts = or_npts(g);
  size_t stride = 1;
  for (int b = 0; b < ax; ++b) stride *= (size_t)g->n[b];
  size_t nlines = npts / (size_t)n;
  double complex* w = is_pow2(n) ? twiddles(n, sign) : NULL;
  if (is_pow2(n) && !w) return OR_ENOMEM;
  int rc = OR_OK;
#pragma omp parallel num_threads(g_threads)
  {
    double complex* line = (double complex*)malloc(sizeof(double complex) * n);
    double complex* tmp = is_pow2(n) ? NULL : (double complex*)malloc(sizeof(double complex) * n);
#pragma omp for schedule(static)
    for (long long l = 0; l < (long long)nlines; ++l) {
      /* line l: base index = (l / stride) * stride * n + (l % stride) */
      size_t base = ((size_t)l / stride) * stride * (size_t)n + ((size_t)l % stride);
      if (!line || (!is_pow2(n) && !tmp)) continue;
      for (int t = 0; t < n; ++t) line[t] = a[base + (size_t)t * stride];
      if (w) {
        fft_pow2(line, n, w);
        for (int t = 0; t < n; ++t) a[base + (size_t)t * stride] = line[t];
      } else {
        or_dft1(line, tmp, n, sign);
        for (int t = 0; t < n; ++t) a[base + (size_t)t * stride] = tmp[t];
      }
    }
    if (!line || (!is_pow2(n) && !tmp)) rc = OR_ENOMEM;
    free(line);
    free(tmp);
  }
  free(w);
  return rc;
}

int or_fftn(const or_grid* g, double complex* a, int sign) {
  if (!valid_grid(g) || (sign != 1 && sign != -1)) return OR_EINVAL;
  for (int ax = 0; ax < g->dim; ++ax) {
    int rc = fft_axis(g, a, ax, sign);
    if (rc) return rc;
  }
  if (sign == 1) {
    size_t npts = or_npts(g);
    double s = 1.0 / (double)npts;
    for (size_t q = 0; q < npts; ++q) a[q] *= s;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* Fourier variables (Section 2.3.3)                                   */
/* ------------------------------------------------------------------ */

double or_xi(int l, int N, double L) {
  return (l <= N / 2) ? 2.0 * M_PI * l / L : 2.0 * M_PI * (l - N) / L;
}

double or_xi_deriv(int l, int N, double L) {
  if (2 * l == N) return 0.0; /* R1 */
  return or_xi(l, N, L);
}

/* Index of spectral point q along axis a. */
static int coord(const or_grid* g, size_t q, int a) {
  size_t s = 1;
  for (int b = 0; b < a; ++b) s *= (size_t)g->n[b];
  return (int)((q / s) % (size_t)g->n[a]);
}

/* ------------------------------------------------------------------ */
/* Spectral derivatives                                                */
/* ------------------------------------------------------------------ */

int or_gradient(const or_grid* g, const double* f, double* grad) {
  if (!valid_grid(g)) return OR_EINVAL;
  size_t npts = or_npts(g);
  double complex* fh = (double complex*)malloc(sizeof(double complex) * npts);
  double complex* t = (double complex*)malloc(sizeof(double complex) * npts);
  if (!fh || !t) { free(fh); free(t); return OR_ENOMEM; }
  for (size_t q = 0; q < npts; ++q) fh[q] = f[q];
  int rc = or_fftn(g, fh, -1);
  for (int c = 0; c < g->dim && !rc; ++c) {
    /* d f / d x_c  =  F^-1 [ i xi~_c F f ] */
    for (size_t q = 0; q < npts; ++q)
      t[q] = I * or_xi_deriv(coord(g, q, c), g->n[c], g->L[c]) * fh[q];
    rc = or_fftn(g, t, +1);
    for (size_t q = 0; q < npts; ++q) grad[(size_t)c * npts + q] = creal(t[q]);
  }
  free(fh);
  free(t);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Pressure operator (eq. 1.1a and eq. p_discrete)                     */
/* ------------------------------------------------------------------ */

void or_apply_K(int dim, size_t npts, const double* m, const double* r, const double* v,
                double* q) {
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (long long p = 0; p < (long long)npts; ++p) {
    /* (m (x) m + r I) v = m (m . v) + r v */
    double mv = 0;
    for (int c = 0; c < dim; ++c) mv += m[(size_t)c * npts + p] * v[(size_t)c * npts + p];
    for (int c = 0; c < dim; ++c)
      q[(size_t)c * npts + p] = m[(size_t)c * npts + p] * mv + r[p] * v[(size_t)c * npts + p];
  }
}

int or_apply_A(const or_grid* g, const double* m, const double* r, const double* p, double* Ap) {
  if (!valid_grid(g)) return OR_EINVAL;
  size_t npts = or_npts(g);
  int dim = g->dim;
  double* grad = (double*)malloc(sizeof(double) * dim * npts);
  double* flux = (double*)malloc(sizeof(double) * dim * npts);
  double complex* div = (double complex*)calloc(npts, sizeof(double complex));
  double complex* t = (double complex*)malloc(sizeof(double complex) * npts);
  int rc = (!grad || !flux || !div || !t) ? OR_ENOMEM : OR_OK;
  /* inner bracket: F^-1[ i xi F p ] */
  if (!rc) rc = or_gradient(g, p, grad);
  /* tensor: (m (x) m + r I) grad p */
  if (!rc) or_apply_K(dim, npts, m, r, grad, flux);
  /* outer: i xi . F(flux), summed over components */
  for (int c = 0; c < dim && !rc; ++c) {
    for (size_t q = 0; q < npts; ++q) t[q] = flux[(size_t)c * npts + q];
    rc = or_fftn(g, t, -1);
    for (size_t q = 0; q < npts && !rc; ++q)
      div[q] += I * or_xi_deriv(coord(g, q, c), g->n[c], g->L[c]) * t[q];
  }
  /* A p = - F^-1[ ... ] */
  if (!rc) rc = or_fftn(g, div, +1);
  if (!rc)
    for (size_t q = 0; q < npts; ++q) Ap[q] = -creal(div[q]);
  free(grad);
  free(flux);
  free(div);
  free(t);
  return rc;
}

/* Entry (a, b) of the symmetric matrix stored as xx, yy, zz, xy, xz, yz. */
static double kbar_at(const double* kbar, int a, int b) {
  static const int idx[3][3] = {{0, 3, 4}, {3, 1, 5}, {4, 5, 2}};
  return kbar[idx[a][b]];
}

int or_precond(const or_grid* g, const double* kbar, const double* res, double* z) {
  if (!valid_grid(g) || !kbar) return OR_EINVAL;
  for (int a = 0; a < g->dim; ++a)
    if (!(kbar_at(kbar, a, a) > 0)) return OR_EINVAL;
  size_t npts = or_npts(g);
  double complex* t = (double complex*)malloc(sizeof(double complex) * npts);
  if (!t) return OR_ENOMEM;
  for (size_t q = 0; q < npts; ++q) t[q] = res[q];
  int rc = or_fftn(g, t, -1);
  for (size_t q = 0; q < npts && !rc; ++q) {
    /* xi~^T Kbar xi~, the symbol of -div(Kbar grad) built from the same derivatives */
    double xi[3] = {0, 0, 0};
    for (int c = 0; c < g->dim; ++c) xi[c] = or_xi_deriv(coord(g, q, c), g->n[c], g->L[c]);
    double s = 0;
    for (int a = 0; a < g->dim; ++a)
      for (int b = 0; b < g->dim; ++b) s += xi[a] * kbar_at(kbar, a, b) * xi[b];
    t[q] = (s > 0) ? t[q] / s : 0;
  }
  if (!rc) rc = or_fftn(g, t, +1);
  if (!rc)
    for (size_t q = 0; q < npts; ++q) z[q] = creal(t[q]);
  free(t);
  return rc;
}

void or_project(const or_grid* g, double* f) {
  size_t npts = or_npts(g);
  /* corner mode e (bit a of e set <=> factor (-1)^{i_a}); only axes with an
     even number of nodes have a Nyquist index */
  for (int e = 0; e < (1 << g->dim); ++e) {
    int ok = 1;
    for (int a = 0; a < g->dim; ++a)
      if (((e >> a) & 1) && (g->n[a] % 2)) ok = 0;
    if (!ok) continue;
    double s = 0;
    for (size_t q = 0; q < npts; ++q) {
      int par = 0;
      for (int a = 0; a < g->dim; ++a)
        if ((e >> a) & 1) par += coord(g, q, a);
      s += (par & 1) ? -f[q] : f[q];
    }
    s /= (double)npts;
    for (size_t q = 0; q < npts; ++q) {
      int par = 0;
      for (int a = 0; a < g->dim; ++a)
        if ((e >> a) & 1) par += coord(g, q, a);
      f[q] -= (par & 1) ? -s : s;
    }
  }
}

void or_kbar_default(const or_grid* g, const double* m, const double* r, double* kbar) {
  size_t npts = or_npts(g);
  int dim = g->dim;
  static const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
  double sr = 0;
  for (size_t q = 0; q < npts; ++q) sr += r[q];
  for (int e = 0; e < 6; ++e) {
    kbar[e] = 0;
    if (pa[e] >= dim || pb[e] >= dim) continue;
    double s = 0;
    for (size_t q = 0; q < npts; ++q) s += m[(size_t)pa[e] * npts + q] * m[(size_t)pb[e] * npts + q];
    kbar[e] = s / (double)npts + (pa[e] == pb[e] ? sr / (double)npts : 0.0);
  }
}

/* trace(Kbar) / dim of the default Kbar: the isotropic part, reported as kappa */
double or_kappa_default(const or_grid* g, const double* m, const double* r) {
  size_t npts = or_npts(g);
  double sr = 0, sm = 0;
  for (size_t q = 0; q < npts; ++q) {
    sr += r[q];
    for (int c = 0; c < g->dim; ++c) sm += m[(size_t)c * npts + q] * m[(size_t)c * npts + q];
  }
  return sr / (double)npts + sm / (double)npts / (double)g->dim;
}

/* Kbar of a solve (R3): the caller's kappa I when kappa > 0, else the mean of
   K (precond 1) or its isotropic part (precond 0, the default). */
static void or_kbar_for(const or_grid* g, const or_params* prm, const double* m, const double* r,
                        double* kbar) {
  if (prm->kappa > 0 || prm->precond != 1) {
    const double k = prm->kappa > 0 ? prm->kappa : or_kappa_default(g, m, r);
    for (int e = 0; e < 6; ++e) kbar[e] = (e < g->dim) ? k : 0.0;
  } else {
    or_kbar_default(g, m, r, kbar);
  }
}

static double dot(size_t n, const double* a, const double* b) {
  double s = 0;
  for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* ------------------------------------------------------------------ */
/* Preconditioned conjugate gradients (Section 2.4)                    */
/* ------------------------------------------------------------------ */

int or_pcg(const or_grid* g, const double* m, const double* r, const double* b, double* x,
           const double* kbar, double rtol, int maxit, or_stats* st) {
  if (!valid_grid(g) || !kbar || maxit < 0) return OR_EINVAL;
  double kappa = 0; /* reported: trace(Kbar) / dim */
  for (int a = 0; a < g->dim; ++a) kappa += kbar[a] / (double)g->dim;
  size_t n = or_npts(g);
  double* res = (double*)malloc(sizeof(double) * n);
  double* z = (double*)malloc(sizeof(double) * n);
  double* d = (double*)malloc(sizeof(double) * n);
  double* q = (double*)malloc(sizeof(double) * n);
  int rc = (!res || !z || !d || !q) ? OR_ENOMEM : OR_OK;
  int it = 0;
  double bnorm = sqrt(dot(n, b, b)), rnorm = 0;
  if (!rc && bnorm == 0) {
    /* S = 0: the projected solution is p = 0 (R2), no iterations */
    memset(x, 0, sizeof(double) * n);
    if (st) {
      st->cg_iters = 0; st->kappa = kappa; st->rel_residual = 0; st->true_rel_residual = 0;
    }
    free(res); free(z); free(d); free(q);
    return OR_OK;
  }
  if (!rc) {
    or_project(g, x); /* initial guess into the complement of the null space (R2) */
    rc = or_apply_A(g, m, r, x, q);
  }
  if (!rc) {
    for (size_t i = 0; i < n; ++i) res[i] = b[i] - q[i];
    rnorm = sqrt(dot(n, res, res));
    rc = or_precond(g, kbar, res, z);
  }
  if (!rc) {
    memcpy(d, z, sizeof(double) * n);
    double rho = dot(n, res, z);
    while (rnorm > rtol * bnorm && it < maxit) {
      rc = or_apply_A(g, m, r, d, q);
      if (rc) break;
      const double dAd = dot(n, d, q);
      /* <d, A d> = 0 only when d has no component in the range of A (R2), as on
         a grid whose every mode is a null mode: nothing is left to solve */
      if (!(dAd > 0)) break;
      double alpha = rho / dAd;
      for (size_t i = 0; i < n; ++i) x[i] += alpha * d[i];
      for (size_t i = 0; i < n; ++i) res[i] -= alpha * q[i];
      rnorm = sqrt(dot(n, res, res));
      rc = or_precond(g, kbar, res, z);
      if (rc) break;
      double rho_new = dot(n, res, z);
      double beta = rho_new / rho;
      for (size_t i = 0; i < n; ++i) d[i] = z[i] + beta * d[i];
      rho = rho_new;
      ++it;
    }
  }
  if (st) {
    st->cg_iters = it;
    st->kappa = kappa;
    st->rel_residual = bnorm > 0 ? rnorm / bnorm : 0.0;
    st->true_rel_residual = st->rel_residual;
    if (!rc && bnorm > 0 && !or_apply_A(g, m, r, x, q)) {
      for (size_t i = 0; i < n; ++i) q[i] = b[i] - q[i];
      st->true_rel_residual = sqrt(dot(n, q, q)) / bnorm;
    }
  }
  if (!rc && !isfinite(rnorm)) rc = OR_ENONFINITE;
  if (!rc && rnorm > rtol * bnorm) rc = OR_ENOCONV;
  free(res);
  free(z);
  free(d);
  free(q);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Splitting substeps (Section 2.3)                                    */
/* ------------------------------------------------------------------ */

void or_activation(int dim, size_t npts, double* m, const double* gp, double c, double dt) {
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (long long q = 0; q < (long long)npts; ++q) {
    double g[3] = {0, 0, 0}, mm[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      g[a] = gp[(size_t)a * npts + q];
      mm[a] = m[(size_t)a * npts + q];
    }
    double g2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    if (g2 == 0) continue; /* grad p = 0: m unchanged */
    double e = exp(c * c * g2 * dt);
    double gm = g[0] * mm[0] + g[1] * mm[1] + g[2] * mm[2];
    double out[3];
    if (dim == 2) {
      /* (1/|g|^2) [ g_perp (g_perp . m) + g (g . m) exp(c^2 |g|^2 dt) ],  g_perp = (-g_y, g_x) */
      double gperp[2] = {-g[1], g[0]};
      double gpm = gperp[0] * mm[0] + gperp[1] * mm[1];
      for (int a = 0; a < 2; ++a) out[a] = (gperp[a] * gpm + g[a] * gm * e) / g2;
    } else {
      /* R8: the perpendicular projector is I - g g^T / |g|^2 */
      for (int a = 0; a < 3; ++a) out[a] = mm[a] - g[a] * gm / g2 + g[a] * gm * e / g2;
    }
    for (int a = 0; a < dim; ++a) m[(size_t)a * npts + q] = out[a];
  }
}

void or_relaxation(int dim, size_t npts, double* m, double gamma, double dt) {
#pragma omp parallel for schedule(static) num_threads(g_threads)
  for (long long q = 0; q < (long long)npts; ++q) {
    if (gamma == 1.0) { /* m exp(-dt) */
      for (int a = 0; a < dim; ++a) m[(size_t)a * npts + q] *= exp(-dt);
      continue;
    }
    double n2 = 0;
    for (int a = 0; a < dim; ++a) n2 += m[(size_t)a * npts + q] * m[(size_t)a * npts + q];
    double nm = sqrt(n2);
    if (nm == 0) continue; /* |m| = 0: unchanged */
    /* b = |m|^{2(1-gamma)} - 2(1-gamma) dt ;  a = m/|m| b^{1/(2(1-gamma))} ;  result a 1_{b>=0} */
    double b = pow(nm, 2.0 * (1.0 - gamma)) - 2.0 * (1.0 - gamma) * dt;
    double scale = (b >= 0) ? pow(b, 1.0 / (2.0 * (1.0 - gamma))) / nm : 0.0;
    for (int a = 0; a < dim; ++a) m[(size_t)a * npts + q] *= scale;
  }
}

int or_diffusion(const or_grid* g, double* m, double D, double dt) {
  if (!valid_grid(g)) return OR_EINVAL;
  size_t npts = or_npts(g);
  double complex* t = (double complex*)malloc(sizeof(double complex) * npts);
  if (!t) return OR_ENOMEM;
  int rc = OR_OK;
  for (int c = 0; c < g->dim && !rc; ++c) {
    for (size_t q = 0; q < npts; ++q) t[q] = m[(size_t)c * npts + q];
    rc = or_fftn(g, t, -1);
    for (size_t q = 0; q < npts && !rc; ++q) {
      double s = 0; /* xi_x^2 + xi_y^2 [+ xi_z^2], Nyquist kept (it is squared) */
      for (int a = 0; a < g->dim; ++a) {
        double x = or_xi(coord(g, q, a), g->n[a], g->L[a]);
        s += x * x;
      }
      t[q] *= exp(-D * D * s * dt);
    }
    if (!rc) rc = or_fftn(g, t, +1);
    for (size_t q = 0; q < npts && !rc; ++q) m[(size_t)c * npts + q] = creal(t[q]);
  }
  free(t);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1, one pass of the loop body                             */
/* ------------------------------------------------------------------ */

int or_step(const or_grid* g, const or_params* prm, const double* r, const double* S,
            double* m, double* p, or_stats* st) {
  if (!valid_grid(g) || !prm) return OR_EINVAL;
  size_t npts = or_npts(g);
  int dim = g->dim;
  double* b = (double*)malloc(sizeof(double) * npts);
  double* grad = (double*)malloc(sizeof(double) * dim * npts);
  if (!b || !grad) { free(b); free(grad); return OR_ENOMEM; }
  memcpy(b, S, sizeof(double) * npts);
  or_project(g, b); /* solvability: S orthogonal to the null space (R2) */
  double kbar[6];
  or_kbar_for(g, prm, m, r, kbar);
  or_stats local;
  /* Step 1: pressure from m^k, warm start p^k */
  int rc = or_pcg(g, m, r, b, p, kbar, prm->cg_rtol, prm->cg_maxit, &local);
  int solve_rc = rc;
  if (rc == OR_ENOCONV) rc = OR_OK; /* state still advanced, flag returned below */
  /* Step 2: splitting with grad p^{k+1} (R6) */
  if (!rc) rc = or_gradient(g, p, grad);
  if (!rc) {
    or_activation(dim, npts, m, grad, prm->c, prm->dt);
    or_relaxation(dim, npts, m, prm->gamma, prm->dt);
    rc = or_diffusion(g, m, prm->D, prm->dt);
  }
  if (st) *st = local;
  if (!rc) {
    for (size_t q = 0; q < (size_t)dim * npts; ++q)
      if (!isfinite(m[q])) { rc = OR_ENONFINITE; break; }
  }
  if (!rc && solve_rc == OR_ENOCONV) rc = OR_ENOCONV;
  free(b);
  free(grad);
  return rc;
}

double or_energy(const or_grid* g, const or_params* prm, const double* r, const double* m,
                 const double* p) {
  size_t npts = or_npts(g);
  int dim = g->dim;
  double h = 1;
  for (int a = 0; a < dim; ++a) h *= g->L[a] / g->n[a];
  double* gp = (double*)malloc(sizeof(double) * dim * npts);
  double* gm = (double*)malloc(sizeof(double) * dim * npts);
  if (!gp || !gm) { free(gp); free(gm); return NAN; }
  or_gradient(g, p, gp);
  double e_diff = 0, e_r = 0, e_act = 0, e_rel = 0;
  for (int c = 0; c < dim; ++c) {
    or_gradient(g, m + (size_t)c * npts, gm);
    for (size_t q = 0; q < (size_t)dim * npts; ++q) e_diff += gm[q] * gm[q];
  }
  for (size_t q = 0; q < npts; ++q) {
    double g2 = 0, mg = 0, m2 = 0;
    for (int c = 0; c < dim; ++c) {
      double gc = gp[(size_t)c * npts + q], mc = m[(size_t)c * npts + q];
      g2 += gc * gc;
      mg += mc * gc;
      m2 += mc * mc;
    }
    e_r += r[q] * g2;
    e_act += mg * mg;
    if (prm->gamma != 0.0)
      e_rel += pow(m2, prm->gamma); /* (|m|^gamma)^2 */
    else
      e_rel += 0.5 * log(m2); /* ln|m| (R21); log(0) = -inf */
  }
  free(gp);
  free(gm);
  double c2 = prm->c * prm->c;
  /* R21: at gamma = 0 the relaxation term is sum ln|m| (its gradient-flow limit) */
  const double rel = prm->gamma != 0.0 ? e_rel / (2.0 * prm->gamma) : e_rel;
  return h * (0.5 * prm->D * prm->D * e_diff + 0.5 * c2 * e_r + 0.5 * c2 * e_act + rel);
}

/* ------------------------------------------------------------------ */
/* Discrete adjoint of the step (gradient of a loss on m(T))           */
/* ------------------------------------------------------------------ */
/* Forward map of one step, written as the composition the adjoint reverses:
 *   p' = A(m)^+ P S                  (pressure, exact solve; P = null-space projection)
 *   g  = G p'                         (spectral gradient)
 *   a  = m + c^2 dt phi1(z) (m.g) g,  z = c^2 dt |g|^2   (activation, eq. m_activation_discrete)
 *   b  = a s(|a|)                     (relaxation, eq. m_relaxation_discrete)
 *   m' = H b,  H = F^-1 diag(exp(-D^2 |xi|^2 dt)) F       (diffusion)
 * phi1(z) = (e^z - 1)/z is the form in which eq. (m_activation_discrete)
 * depends on c^2 and g; the oracle's forward substep uses the paper's g-perp
 * form, which equals it. */

static double phi1(double z) { return z == 0 ? 1.0 : expm1(z) / z; }

/* d phi1 / dz: series for small z (the closed form cancels), else closed form */
static double dphi1(double z) {
  if (fabs(z) < 0.5) {
    /* sum_k z^k / ((k+2) k!) */
    double term = 1.0, s = 0;
    for (int k = 0; k < 18; ++k) {
      if (k > 0) term *= z / k;
      s += term / (k + 2);
    }
    return s;
  }
  return ((z - 1.0) * expm1(z) + z) / (z * z);
}

/* Relaxation b = a s(|a|) and its Jacobian J = s I + (f' - s) a a^T / |a|^2,
 * f(rho) = rho s(rho) (the new modulus), for one point; returns s and writes
 * the coefficient c1 = s, c2 = (f' - s)/|a|^2 so that J v = c1 v + c2 (a.v) a. */
static void relax_jac(int dim, const double* a, double gamma, double dt, double* c1, double* c2) {
  double n2 = 0;
  for (int k = 0; k < dim; ++k) n2 += a[k] * a[k];
  if (gamma == 1.0) { *c1 = exp(-dt); *c2 = 0; return; }
  if (n2 == 0) { *c1 = gamma > 1.0 ? 1.0 : 0.0; *c2 = 0; return; }
  double rho = sqrt(n2);
  double e = 2.0 * (1.0 - gamma); /* b = rho^e - e dt */
  double beta = pow(rho, e) - e * dt;
  if (beta <= 0) { *c1 = 0; *c2 = 0; return; }
  double f = pow(beta, 1.0 / e);
  double fp = pow(beta, 1.0 / e - 1.0) * pow(rho, e - 1.0); /* df/drho */
  double sv = f / rho;
  *c1 = sv;
  *c2 = (fp - sv) / n2;
}

int or_adjoint(const or_grid* g, const or_params* prm, const double* r, const double* S,
               const double* m0, const double* p0, int nsteps, const double* lamT, double* dc2,
               double* dD2, double* dr, double* dS, double* dm0) {
  if (!valid_grid(g) || nsteps < 0) return OR_EINVAL;
  size_t n = or_npts(g);
  int dim = g->dim;
  size_t vn = (size_t)dim * n;
  double c2 = prm->c * prm->c, dtt = prm->dt, D2 = prm->D * prm->D;
  /* forward, keeping m^k and p^{k+1} */
  double* ms = (double*)malloc(sizeof(double) * vn * (nsteps + 1));
  double* ps = (double*)malloc(sizeof(double) * n * (nsteps + 1));
  double* lam = (double*)malloc(sizeof(double) * vn);
  double* grad = (double*)malloc(sizeof(double) * vn);
  double* gmu = (double*)malloc(sizeof(double) * vn);
  double* a = (double*)malloc(sizeof(double) * vn);
  double* b = (double*)malloc(sizeof(double) * vn);
  double* lb = (double*)malloc(sizeof(double) * vn);
  double* lg = (double*)malloc(sizeof(double) * vn);
  double* lp = (double*)malloc(sizeof(double) * n);
  double* mu = (double*)malloc(sizeof(double) * n);
  double* t = (double*)malloc(sizeof(double) * n);
  double complex* ct = (double complex*)malloc(sizeof(double complex) * n);
  int rc = (!ms || !ps || !lam || !grad || !gmu || !a || !b || !lb || !lg || !lp || !mu || !t || !ct)
               ? OR_ENOMEM : OR_OK;
  if (!rc) {
    memcpy(ms, m0, sizeof(double) * vn);
    memcpy(ps, p0, sizeof(double) * n);
    for (int k = 0; k < nsteps && !rc; ++k) {
      memcpy(ms + vn * (k + 1), ms + vn * k, sizeof(double) * vn);
      memcpy(ps + n * (k + 1), ps + n * k, sizeof(double) * n);
      or_stats st;
      int s_rc = or_step(g, prm, r, S, ms + vn * (k + 1), ps + n * (k + 1), &st);
      if (s_rc && s_rc != OR_ENOCONV) rc = s_rc;
    }
  }
  if (!rc) {
    *dc2 = 0;
    *dD2 = 0;
    memset(dr, 0, sizeof(double) * n);
    memset(dS, 0, sizeof(double) * n);
    memcpy(lam, lamT, sizeof(double) * vn);
  }
  for (int k = nsteps - 1; k >= 0 && !rc; --k) {
    const double* m = ms + vn * k;
    const double* p = ps + n * (k + 1); /* solved with m^k */
    double kbar[6];
    or_kbar_for(g, prm, m, r, kbar);
    rc = or_gradient(g, p, grad);
    if (rc) break;
    /* recompute a and b */
    memcpy(a, m, sizeof(double) * vn);
    or_activation(dim, n, a, grad, prm->c, dtt);
    memcpy(b, a, sizeof(double) * vn);
    or_relaxation(dim, n, b, prm->gamma, dtt);
    /* diffusion: lambda_b = H lambda (H symmetric); dL/dD^2 = <lambda, dH/dD^2 b> */
    memcpy(lb, lam, sizeof(double) * vn);
    rc = or_diffusion(g, lb, prm->D, dtt);
    for (int c = 0; c < dim && !rc; ++c) {
      for (size_t q = 0; q < n; ++q) ct[q] = b[(size_t)c * n + q];
      rc = or_fftn(g, ct, -1);
      for (size_t q = 0; q < n && !rc; ++q) {
        double s2 = 0;
        for (int ax = 0; ax < dim; ++ax) {
          double x = or_xi(coord(g, q, ax), g->n[ax], g->L[ax]);
          s2 += x * x;
        }
        ct[q] *= -s2 * dtt * exp(-D2 * s2 * dtt);
      }
      if (!rc) rc = or_fftn(g, ct, +1);
      for (size_t q = 0; q < n && !rc; ++q) *dD2 += lam[(size_t)c * n + q] * creal(ct[q]);
    }
    if (rc) break;
    /* pointwise: relaxation and activation Jacobians (both symmetric in m) */
    for (size_t q = 0; q < n; ++q) {
      double av[3] = {0, 0, 0}, gv[3] = {0, 0, 0}, mv[3] = {0, 0, 0}, l[3] = {0, 0, 0};
      for (int c = 0; c < dim; ++c) {
        av[c] = a[(size_t)c * n + q];
        gv[c] = grad[(size_t)c * n + q];
        mv[c] = m[(size_t)c * n + q];
        l[c] = lb[(size_t)c * n + q];
      }
      double c1, c2r;
      relax_jac(dim, av, prm->gamma, dtt, &c1, &c2r);
      double al = av[0] * l[0] + av[1] * l[1] + av[2] * l[2];
      double la[3];
      for (int c = 0; c < 3; ++c) la[c] = c1 * l[c] + c2r * al * av[c]; /* lambda_a */
      double g2 = gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2];
      double z = c2 * dtt * g2;
      double ph = phi1(z), dph = dphi1(z);
      double mg = mv[0] * gv[0] + mv[1] * gv[1] + mv[2] * gv[2];
      double gl = gv[0] * la[0] + gv[1] * la[1] + gv[2] * la[2];
      *dc2 += gl * mg * dtt * (ph + z * dph);
      for (int c = 0; c < dim; ++c) {
        lam[(size_t)c * n + q] = la[c] + c2 * dtt * ph * gl * gv[c];
        lg[(size_t)c * n + q] = c2 * dtt * (ph * (mg * la[c] + mv[c] * gl) + 2.0 * c2 * dtt * dph * mg * gl * gv[c]);
      }
    }
    /* lambda_p = G^T lambda_g = -div lambda_g */
    memset(lp, 0, sizeof(double) * n);
    for (int c = 0; c < dim && !rc; ++c) {
      for (size_t q = 0; q < n; ++q) ct[q] = lg[(size_t)c * n + q];
      rc = or_fftn(g, ct, -1);
      for (size_t q = 0; q < n && !rc; ++q)
        ct[q] *= I * or_xi_deriv(coord(g, q, c), g->n[c], g->L[c]);
      if (!rc) rc = or_fftn(g, ct, +1);
      for (size_t q = 0; q < n && !rc; ++q) lp[q] -= creal(ct[q]);
    }
    if (rc) break;
    or_project(g, lp);
    /* adjoint pressure solve A mu = lambda_p (A symmetric) */
    memset(mu, 0, sizeof(double) * n);
    or_stats st;
    int s_rc = or_pcg(g, m, r, lp, mu, kbar, prm->cg_rtol, prm->cg_maxit, &st);
    if (s_rc && s_rc != OR_ENOCONV) { rc = s_rc; break; }
    for (size_t q = 0; q < n; ++q) dS[q] += mu[q];
    rc = or_gradient(g, mu, gmu);
    if (rc) break;
    /* d<mu, A(m, r) p>: -(grad mu . K grad p) */
    for (size_t q = 0; q < n; ++q) {
      double gm[3] = {0, 0, 0}, gp[3] = {0, 0, 0}, mv[3] = {0, 0, 0};
      for (int c = 0; c < dim; ++c) {
        gm[c] = gmu[(size_t)c * n + q];
        gp[c] = grad[(size_t)c * n + q];
        mv[c] = m[(size_t)c * n + q];
      }
      double mgp = mv[0] * gp[0] + mv[1] * gp[1] + mv[2] * gp[2];
      double mgm = mv[0] * gm[0] + mv[1] * gm[1] + mv[2] * gm[2];
      dr[q] -= gm[0] * gp[0] + gm[1] * gp[1] + gm[2] * gp[2];
      for (int c = 0; c < dim; ++c) lam[(size_t)c * n + q] -= gm[c] * mgp + gp[c] * mgm;
    }
    (void)t;
  }
  if (!rc) {
    /* S enters through its projection: dL/dS = P dL/d(PS) */
    or_project(g, dS);
    memcpy(dm0, lam, sizeof(double) * vn);
  }
  free(ms); free(ps); free(lam); free(grad); free(gmu); free(a); free(b); free(lb); free(lg);
  free(lp); free(mu); free(t); free(ct);
  return rc;
}
