/*
 * hc_oracle.h -- plain FP64 CPU oracle for one time step of the Fourier
 * spectral FFT+CG splitting scheme for the periodic Hu-Cai network-formation
 * system (Aceves-Sanchez, Degond, Merino-Aceituno, Wytrzens, arXiv 2606.06720).
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The GPU product path
 * never calls it, shares no code with it and includes none of its headers.
 *
 * Conventions
 *   - Grid (Section 2.2, reading R9): dim = 2 or 3, n[a] nodes on axis a, the
 *     periodic end point excluded, spacing h_a = L[a] / n[a], x_i = i h_a.
 *   - Storage: row-major with x fastest, flat index (k*n[1] + j)*n[0] + i.
 *     Vector fields (m, grad p, ...) are component-major: component c of point
 *     q lives at [c*npts + q].
 *   - Forward DFT unnormalised with kernel exp(-2 pi i j k / N); the inverse
 *     uses exp(+2 pi i j k / N) and a 1/N factor per axis.
 *   - Every routine is single-precision-free: all arithmetic is IEEE FP64.
 *
 * Parity pins for every routine live in tests/test_oracle_*.py.
 */
#ifndef HC_ORACLE_H
#define HC_ORACLE_H

#include <complex.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dim;          /* 2 or 3 */
  int n[3];         /* nodes per axis (x, y, z); n[2] = 1 when dim = 2 */
  double L[3];      /* domain lengths */
} or_grid;

typedef struct {
  double c, D, gamma, dt;  /* model parameters of eqs (1.1a)-(1.1b) and the time step */
  double cg_rtol;          /* stop when ||S - A p||_2 <= cg_rtol ||S||_2 (reading R4) */
  int cg_maxit;            /* iteration cap */
  double kappa;            /* > 0: preconditioner kappa (-Laplacian), whatever precond says */
  int precond;             /* kappa <= 0: 0 (default) kappa (-Laplacian) with the kappa of reading
                              R3, mean(r) + mean(|m|^2)/dim; 1 -div(Kbar grad), Kbar = mean(m m^T)
                              + mean(r) I (the anisotropic constant-coefficient option) */
} or_params;

typedef struct {
  int cg_iters;             /* CG iterations of the pressure solve */
  double rel_residual;      /* recursively updated ||r|| / ||S|| at exit */
  double true_rel_residual; /* ||S - A p|| / ||S|| recomputed at exit */
  double kappa;             /* trace(Kbar) / dim of the preconditioner that was used */
} or_stats;

enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2, OR_ENOCONV = -4, OR_ENONFINITE = -5 };

/* Threads for the parallel loops (FFT lines, pointwise maps).  Reductions are
 * always sequential, so results do not depend on this value. */
void or_set_threads(int nthreads);
int or_get_threads(void);

size_t or_npts(const or_grid* g);

/* 1D transforms of length n; sign = -1 forward, +1 inverse, both unnormalised. */
int or_dft1(const double complex* in, double complex* out, int n, int sign);
int or_fft1(double complex* a, int n, int sign);

/* Multi-dimensional transform over every axis of the grid, in place.
 * sign = -1: unnormalised forward; sign = +1: inverse including 1/npts. */
int or_fftn(const or_grid* g, double complex* a, int sign);

/* Discrete Fourier variable of Section 2.3.3: 2 pi l / L for 0 <= l <= N/2 and
 * 2 pi (l - N) / L above.  The Nyquist entry is positive, as printed. */
double or_xi(int l, int N, double L);
/* First-derivative multiplier: or_xi with the Nyquist entry set to 0 (R1). */
double or_xi_deriv(int l, int N, double L);

/* Spectral gradient of a real scalar field f: grad[c*npts + q] (dim components). */
int or_gradient(const or_grid* g, const double* f, double* grad);

/* Pointwise conductivity-tensor product q = (m (x) m + r I) v  (eq. 1.1a). */
void or_apply_K(int dim, size_t npts, const double* m, const double* r,
                const double* v, double* q);

/* Discrete pressure operator of eq. (p_discrete): A p = -F^-1[i xi . F(K F^-1[i xi F p])]. */
int or_apply_A(const or_grid* g, const double* m, const double* r, const double* p, double* Ap);

/* Constant-coefficient preconditioner (R3): z = F^-1[ F(res) / (xi~^T Kbar xi~) ],
 * zero on the null modes.  kbar: the symmetric matrix Kbar as 6 doubles
 * xx, yy, zz, xy, xz, yz (2D reads xx, yy, xy); its diagonal must be > 0. */
int or_precond(const or_grid* g, const double* kbar, const double* res, double* z);

/* Remove the null-space components of A (the 2^dim corner modes, R2) in place. */
void or_project(const or_grid* g, double* f);

/* The anisotropic Kbar of R3's option: mean(m m^T) + mean(r) I, in the layout of or_precond. */
void or_kbar_default(const or_grid* g, const double* m, const double* r, double* kbar);

/* The default preconditioner constant of R3: mean(r) + mean(|m|^2) / dim, the
 * isotropic part trace(Kbar) / dim of that mean. */
double or_kappa_default(const or_grid* g, const double* m, const double* r);

/* Preconditioned CG (Section 2.4) for A p = b, b projected; p in/out holds the
 * initial guess on entry.  Returns OR_OK or OR_ENOCONV. */
int or_pcg(const or_grid* g, const double* m, const double* r, const double* b, double* p,
           const double* kbar, double rtol, int maxit, or_stats* st);

/* Exact activation substep, eq. (m_activation_discrete), pointwise. */
void or_activation(int dim, size_t npts, double* m, const double* grad_p, double c, double dt);
/* Exact relaxation substep, eq. (m_relaxation_discrete), pointwise. */
void or_relaxation(int dim, size_t npts, double* m, double gamma, double dt);
/* Exact diffusion substep, eq. (diffusion_space_discrete), per component. */
int or_diffusion(const or_grid* g, double* m, double D, double dt);

/* One pass of the loop body of Algorithm 1: p <- CG solve with m^k (warm start
 * p^k), then activation, relaxation and diffusion of m.  S is projected
 * internally.  m and p are updated in place. */
int or_step(const or_grid* g, const or_params* prm, const double* r, const double* S,
            double* m, double* p, or_stats* st);

/* Discrete adjoint of `nsteps` loop bodies of Algorithm 1 started from
 * (m0, p0), treating every pressure solve as exact (run it with a tight
 * cg_rtol).  lamT = dL/dm(T) for a loss L of the final conductivity.  Outputs
 * dL/d(c^2), dL/d(D^2), dL/dr (field), dL/dS (field), dL/dm0 (vector field);
 * gradients are with respect to the grid values (plain sums, no quadrature
 * weights).  The forward states are kept in memory: small grids only. */
int or_adjoint(const or_grid* g, const or_params* prm, const double* r, const double* S,
               const double* m0, const double* p0, int nsteps, const double* lamT, double* dc2,
               double* dD2, double* dr, double* dS, double* dm0);

/* Discrete energy of Section 2.5 (quadrature weight h_x h_y [h_z], R10), with
 * p the pressure that belongs to m. */
double or_energy(const or_grid* g, const or_params* prm, const double* r,
                 const double* m, const double* p);

#ifdef __cplusplus
}
#endif
#endif
