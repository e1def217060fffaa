// hc_internal.cuh -- types shared by the kernel translation units and the host
// orchestration of the Hu-Cai spectral step (arXiv 2606.06720, Section 2).
//
// Spectral layout ("packed half spectrum").  A real nx x ny field f with 2D DFT
// F[ky][kx] is stored as ny rows of H = nx/2 complex values:
//   P[ky][kx] = F[ky][kx]                     for 1 <= kx < H,
//   P[ky][0]  = F[ky][0] + i F[ky][H]         (the two real-in-x columns packed).
// A row-transformed field (x transformed, y not yet) uses the same packing row
// by row.  Every spectral vector is the unnormalised DFT; physical fields are
// row-major with x fastest.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hc {

// Complex value with the size and alignment of float2 / double2, so loads and
// stores compile to single vector memory instructions.
template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T x, y;
};

// Double-float: the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// a 48-bit significand computed on the FP32 pipes (error-free transformations:
// Knuth's TwoSum, Dekker's Fast2Sum, and the FMA-based exact product).  On
// GB300 the FP64 pipe issues at 1/58 of the FP32 rate, so FP64-class residuals
// run faster this way.  Additions use the normwise-accurate form: the absolute
// error of a + b is below 2^-47 (|a| + |b|), the bound the FFT error analysis
// needs.
struct df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ df64(float f) : hi(f), lo(0.0f) {}
  __host__ __device__ df64(int i) : hi((float)i), lo(0.0f) {}
  __host__ __device__ df64(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

__host__ __device__ inline df64 df_fast2sum(float a, float b) {  // needs |a| >= |b| or a == 0
  const float s = a + b;
  return df64(s, b - (s - a));
}
__host__ __device__ inline df64 df_2sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df64(s, (a - (s - bb)) + (b - bb));
}
__host__ __device__ inline df64 operator+(df64 a, df64 b) {
  df64 s = df_2sum(a.hi, b.hi);
  s.lo += a.lo + b.lo;
  return df_fast2sum(s.hi, s.lo);
}
__host__ __device__ inline df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__host__ __device__ inline df64 operator-(df64 a, df64 b) { return a + (-b); }
__host__ __device__ inline df64 operator*(df64 a, df64 b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return df_fast2sum(p, e);
}
__host__ __device__ inline df64 operator/(df64 a, df64 b) {
  const float q1 = a.hi / b.hi;
  const df64 r = a - b * df64(q1);
  return df_fast2sum(q1, r.hi / b.hi);
}
__host__ __device__ inline bool operator>(df64 a, df64 b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
__host__ __device__ inline bool operator<(df64 a, df64 b) { return b > a; }
__host__ __device__ inline bool operator>=(df64 a, df64 b) { return !(b > a); }
__host__ __device__ inline bool operator==(df64 a, df64 b) { return a.hi == b.hi && a.lo == b.lo; }
__host__ __device__ inline bool operator!=(df64 a, df64 b) { return !(a == b); }

// Device-resident scalar state of one pressure solve (CG and refinement).
// All reductions that feed it are computed in FP64 by the last CTA of the
// producing kernel, summing the per-CTA partials in a fixed order.
struct SolveState {
  double alpha, beta, rho;   // CG scalars
  double rnorm2;             // ||r||^2 of the CG recursion (spectral weights)
  double bnorm2;             // ||b||^2 of the right-hand side of the running CG
  double thresh2;            // CG stops when rnorm2 <= thresh2
  double kappa;              // trace(Kbar) / dim of this step's preconditioner (reported)
  double kbar[6];            // preconditioner matrix Kbar (xx, yy, zz, xy, xz, yz), reading R3
  // FP32 copies of kbar, alpha and beta, written with them by the one thread
  // that sets them: the FP32 kernels read these, so their threads do no
  // double-to-float conversions (the FP64 pipe of this part is narrow)
  float kbar_f[6];
  float alpha_f, beta_f;
  double mean_r;             // mean of r (set with r)
  double msum;               // sum |m|^2 of the current m
  double mm[6];              // sum m_a m_b of the current m (xx, yy, zz, xy, xz, yz); follows msum
  double outer_r2;           // refined: ||S - A p64||^2 at the last FP64 evaluation
  double outer_b2;           // ||S||^2 (spectral weights)
  double outer_thresh2;      // refined: (cg_rtol ||S||)^2
  double inner_rtol2;        // refined: inner reduction factor squared
  double user_kappa;         // > 0: fixed kappa
  double outer_rtol2;        // cg_rtol^2
  int refined;               // 1: FP32 inner CG with FP64 refinement
  int pad0_;
  int it;                    // CG iterations of the running solve
  int maxit;                 // cap
  int done;                  // running CG finished (converged or capped)
  int first;                 // next d-update is d = z (no previous direction)
  int status;                // 0, HC_ENOCONV, HC_ENONFINITE of the running solve
  int total_it;              // refined: iterations summed over sweeps
  int sweeps;                // refined: inner solves run in this step
  int outer_done;            // refined: FP64 residual below the tolerance
  int max_sweeps;
  int nonfinite;             // set when the split step produced a non-finite m
  int step_status;           // status of the last completed step
  int graph_mode;            // 1: kernels drive the conditional nodes below
  int first_bad;             // first non-OK step status since the last reset
  int acc_iters;             // CG iterations summed over the steps since the last reset
  int acc_sweeps;            // refinement sweeps summed likewise
  int acc_steps;             // steps completed since the last reset
  unsigned long long h_inner;  // cudaGraphConditionalHandle of the CG loop
  unsigned long long h_outer;  // cudaGraphConditionalHandle of the refinement loop
  unsigned long long h_gate;   // cudaGraphConditionalHandle of a gated step (hc_run)
  unsigned long long h_first;  // cudaGraphConditionalHandle of the first (FP32-started) inner loop
  unsigned long long h_cur;    // the inner-loop handle the CG kernels drive (set by whoever opens it)
  unsigned long long h_mid;        // cudaGraphConditionalHandle of the mid-step residual block (IF)
  unsigned long long h_mid_inner;  // cudaGraphConditionalHandle of the inner loop after it
  double first32_min2;       // refined: FP32 first sweep only if ||S - A p||^2 > this * ||S||^2 (0: off)
  int acc_first;             // FP32 first sweeps summed over the steps since the last reset
  int first_used;            // the running / last step ran an FP32 first sweep
  int mid_df;                // HC_FP32_REFINED: the residual after an FP32 first sweep is evaluated in double-float
  int precond;               // HC_PRECOND_SCALAR | HC_PRECOND_KBAR (with no user kappa)
  int mid_phase;             // the next refinement residual is that double-float mid-step one
  int mid_used;              // the running / last step evaluated it
  int acc_mid;               // such residuals summed over the steps since the last reset
  int res_full;              // running / last step: residuals in the mode's full refinement arithmetic
  int acc_res_full;          // summed likewise
  unsigned int ticket[8];    // last-CTA tickets, one per reduction site
  // Diagnostics of Section 2.5, accumulated by the split step when diag != 0.
  // A step solves p[m^k] and so evaluates E_h(m^k) with its own pressure.
  double dsum[3];            // running step: sum r|g|^2, sum (m.g)^2, sum |m|^(2 gamma) (gamma = 0: sum ln|m|); m = m^k, g = grad p[m^k]
  double gm2;                // sum |grad m|^2 of the current m (derivative multipliers of reading R1)
  double gm2_next;           // the same for the m the running step produces
  double dm2;                // running step: sum |m^{k+1} - m^k|^2
  double msum_old;           // sum |m^k|^2 at the start of the running step
  double energy;             // E_h(m^k) of the last completed step
  double energy_prev;        // the value before it
  double delta_m;            // Delta m of the last completed step
  double e_coef[3];          // h D^2 / 2, h c^2 / 2, h / (2 gamma) (h at gamma = 0)  (h: cell volume)
  double dt;
  double eps_dm;             // run mode: stop once delta_m <= eps_dm
  int dim;
  int diag;                  // 1: the split step accumulates the diagnostics
  int gm2_valid;             // gm2 belongs to the current m
  int gm2_next_valid;        // the running step computed gm2_next
  int energy_valid;          // energy holds E_h of the last step's starting m
  int n_energy;              // energies computed since the last run reset
  int run_mode;              // 1: step_end applies the stopping rules of Algorithm 1
  int stop_energy;           // run mode: also stop when the energy does not decrease
  int halt;                  // run mode: a stopping rule fired
  int stop_reason;           // HC_STOP_* of the rule that fired
  int energy_step;           // run mode: steps completed when the energy increase was seen
  // Lagged certification (2D HC_FP32_REFINED steps in graph mode, diagnostics off): the FP64
  // residual that certifies step k runs beside step k+1's FP32 solve (see hc_step).
  int pipelined;             // 1 while such steps run: the mid-step residual always opens
  int cert_pending;          // (certifying state) a step awaits its FP64 certification
  int cert_failed;           // a certification found ||S - A p|| above the tolerance
  int cert_steps;            // steps whose certification passed (or that were accepted) in this call
  double cert_r2;            // (certifying state) ||S - A p||^2 of the last certification
};

// Values the host changes between steps (tolerances, caps, r statistics).
struct SolveConfig {
  double outer_thresh2_rel;  // cg_rtol^2 (multiplied by ||S||^2 on the device)
  double inner_rtol2;
  double user_kappa;
  double mean_r;
  double e_coef[3];          // energy coefficients (see SolveState)
  double dt;
  double first32_min2;       // see SolveState
  int mid_df;                // see SolveState
  int precond;               // see SolveState
  int maxit;
  int max_sweeps;
  int graph_mode;
  int refined;
  int dim;
  int diag;
};

// Doubles of per-CTA partial sums a reducing kernel may hand to its last CTA.
constexpr int kPartialStride = 8;

// Reduction sites (ticket indices).
enum { TK_DIV = 0, TK_UPDATE = 1, TK_RESID = 2, TK_MSUM = 3, TK_PROJ = 4, TK_DIAG = 5, TK_GRADM = 6,
       TK_CERT = 7 };

// One batched column pass of a 3D grid: transforms of length 2^lL whose
// consecutive elements are `stride` apart, over tiles of 2^ltc adjacent
// columns; 2^lt tiles per plane, `nplanes` planes `pstride` apart.
struct ColPass {
  int lL, ltc, lt, nplanes;
  long long stride, pstride;
};

// Three pointers passed by value (the components of a 3D vector field).
template <typename P>
struct Tri {
  P v[3];
};

// Geometry and tables for one precision.
template <typename T>
struct Geo {
  int nx, ny, H;             // H = nx/2 packed columns
  int lnx, lny, lH;          // log2 of the above
  int tc, ltc;               // packed columns per column-kernel CTA
  int rpc, lrpc;             // rows per row-kernel CTA
  const cx<T>* twx;          // exp(-2 pi i m / nx), m < nx
  const cx<T>* twy;          // exp(-2 pi i m / ny), m < ny
  const T* kxd;              // first-derivative wavenumbers along x for kx < H (Nyquist reading: 0 at kx = 0 packed)
  const T* kyd;              // first-derivative wavenumbers along y, ky < ny, 0 at ky = ny/2
  const T* hx;               // heat factor exp(-D^2 xi_x^2 dt), kx = 0..H (H + 1 entries)
  const T* hy;               // heat factor exp(-D^2 xi_y^2 dt), ky < ny
  double* partials;          // per-CTA FP64 partial sums, kPartialStride per CTA
  int npartials;             // capacity in CTAs
  int pipe;                  // 1: column passes run persistent with cp.async double buffering
  int pgrid;                 // CTAs of a persistent column pass (<= SMs, <= tiles)
  int rpipe;                 // 1 (FP32): the apply row pass runs persistent with cp.async double buffering
  int rgrid;                 // CTAs of that pass (resident CTAs, <= row blocks)
  const T* x2x;              // xi_x^2 (positive Nyquist), kx = 0..H (H + 1 entries)
  const T* x2y;              // xi_y^2, ky < ny
  // 3D grids (nz = 1 in 2D).  Spectra are [nz][ny][H] packed as in 2D; the x
  // pass runs over the ny*nz rows, the y and z passes are the ColPasses below.
  int nz, lnz;
  const cx<T>* twz;          // exp(-2 pi i m / nz), m < nz
  const T* kzd;              // first-derivative wavenumbers along z, 0 at kz = nz/2
  const T* hz;               // heat factor exp(-D^2 xi_z^2 dt), kz < nz
  int upc, lupc;             // row pairs per CTA of the 3D row kernels
  ColPass py, pz;            // y pass (per z plane) and z pass (over all ny*H columns)
};

// Scalar results of the adjoint sweep (device).
struct AdjState {
  double dc2, dD2;           // dL/d(c^2), dL/d(D^2) accumulated over steps
  unsigned int ticket[4];
};
enum { TA_POINT = 0, TA_LAP = 1 };

// Split-step coefficients (Section 2.3), precomputed on the host in FP64.
struct SplitCoef {
  double c2dt;       // c^2 dt
  double gamma;
  double dt;
  double exp_mdt;    // exp(-dt), the gamma = 1 branch
  double two1mg_dt;  // 2 (1 - gamma) dt
  double pow_a;      // 2 (1 - gamma)
  double pow_b;      // 1 / (2 (1 - gamma))
  int gamma_is_one;
  // the same rounded to FP32 on the host, for the FP32 kernels (cfv)
  float f_c2dt, f_gamma, f_dt, f_exp_mdt, f_two1mg_dt, f_pow_a, f_pow_b;
  // pow_a, pow_b when they are 1, 2 or 1/2 (1, 2, 3; else 0): the power is
  // then x, x x or sqrt x (pow_k), e.g. both are 1 at gamma = 1/2
  int pow_a_kind, pow_b_kind;
};

// 2D grids whose sizes are not powers of two (hc_generic.cu): N = 2^a 3^b 5^c
// per axis, FP64, unpacked half spectrum of Hh = nx/2 + 1 columns.
constexpr int kGenMaxPasses = 24;
struct GenGeo {
  int nx, ny, Hh;
  int rx[kGenMaxPasses], nrx;  // radices (2, 3, 4, 5) of the x transform, product nx
  int ry[kGenMaxPasses], nry;  // the same along y
  const cx<double>* twx;       // exp(-2 pi i m / nx), m < nx
  const cx<double>* twy;       // exp(-2 pi i m / ny), m < ny
  const double* kxd;           // first-derivative multipliers, kx < Hh (0 at the Nyquist index)
  const double* kyd;           // the same, ky < ny
  const double* hx;            // heat factor exp(-D^2 xi_x^2 dt), kx < Hh
  const double* hy;            // exp(-D^2 xi_y^2 dt), ky < ny
  double* partials;            // per-CTA FP64 partial sums
};

// One member of a batched size class of the parameter sweep (2D grids of one
// size, HC_FP32_REFINED): everything a batched launch takes per instance.
// A batched kernel runs one pass of the step for every member at once, member
// blockIdx.y, with the member's own geometry tables, solve state and buffers.
struct BInst {
  Geo<float> gf;
  Geo<float> gfn;         // gf limited to 512-thread column CTAs (col_narrow)
  Geo<double> gd;
  Geo<df64> gq;
  SolveState* st;
  cx<double>* p64;        // pressure spectrum (FP64)
  const cx<double>* b64;  // projected source spectrum (FP64)
  cx<double>* r64;        // FP64 residual
  const cx<df64>* bq;     // double-float copy of the source (mid-step residual)
  const cx<float>* b32;   // FP32 copy of the source (column-major)
  cx<float>* r32;         // inner CG vectors (column-major)
  cx<float>* d32;
  cx<float>* q32;
  cx<float>* x32;
  cx<float>* G32;         // FP32 gradient / flux scratch, two fields ns apart
  cx<double>* G64;        // FP64 / double-float scratch, two fields ns apart
  float* mx;
  float* my;
  const float* rf;
  size_t ns;              // ny * H packed spectral values per field
  SplitCoef cf;
};

// Launch geometry of a batched size class (every member has the same grid
// and launch shapes): the host copies of one member's three geometries.
struct BShape {
  Geo<float> gf;
  Geo<float> gfn;         // gf limited to 512-thread column CTAs (col_narrow)
  Geo<double> gd;
  Geo<df64> gq;
  int nb;                 // members
};

// Threads of a column-pass CTA at most.  The FP32 gradient and divergence
// passes (WIDE) take up to 1024 at 64 registers a thread: a tile of four
// packed columns of 2048 values reads and writes 32 contiguous bytes per row,
// whole DRAM sectors.  The other column passes (heat, transforms, adjoint,
// the persistent ones) and every FP64 and double-float pass take up to 512,
// with up to 128 registers.
template <typename T, bool WIDE>
constexpr int col_cta_max() {
  return sizeof(T) == 4 && WIDE ? 1024 : 512;
}
// The geometry a column pass of at most 512 threads runs with: the tile
// halved while tc ny/8 is above 512 (a tile is any power of two of columns;
// the passes share no state through it).
template <typename T>
inline Geo<T> col_narrow(Geo<T> g) {
  while (g.tc > 1 && (g.tc << (g.lny - 3)) > 512) {
    g.tc >>= 1;
    g.ltc -= 1;
  }
  return g;
}

// Column-kernel modes.
enum ColGradMode { CG_PLAIN = 0, CG_DUPDATE = 1, CG_ADDDELTA = 2 };
enum ColDivMode { CD_PLAIN = 0, CD_CG = 1, CD_RESID = 2, CD_RESID_REFINE = 3, CD_RESID_FIRST = 4,
                  CD_CERT = 5 };

// ---------------- launchers (defined per precision) ----------------
// Row pass, forward: physical pair (a, b) -> packed row spectra (A, B). b/B may be null.
template <typename T>
void row_r2c(const Geo<T>& g, const T* a, const T* b, cx<T>* A, cx<T>* B, cudaStream_t s);
// Row pass, inverse: packed row spectra -> physical pair; with kappa_update = 1 also the sums of
// a^2, b^2, a b into st->mm and st->msum (the next preconditioner's input), and with st->diag
// sum |new - old|^2 of a, b into st->dm2.
template <typename T>
void row_c2r(const Geo<T>& g, const cx<T>* A, const cx<T>* B, T* a, T* b, SolveState* st,
             int kappa_update, cudaStream_t s);
// Shared memory of the persistent FP32 apply row pass: the transform slabs and
// two stage buffers of the row block's Gx, Gy, mx, my, r (each rpc N 4 bytes).
inline size_t row_pipe_smem(int rpc, int nx) { return (size_t)48 * rpc * nx; }
// Resident CTAs per SM of that pass at this shape (0 if it cannot run).
int row_pipe_ctas_per_sm(int threads, size_t smem);
// Row pass of the operator apply: C2R(gx, gy) -> q = (m.g) m + r g -> R2C(q).
// With st (a CG iteration) also alpha = rho / <d, A d> from this pass, and the
// pass is skipped when st->done.  FP32 with g.rpipe: the persistent variant.
template <typename T, typename Tm>
void row_apply(const Geo<T>& g, const cx<T>* Gx, const cx<T>* Gy, const Tm* mx, const Tm* my,
               const Tm* r, cx<T>* Qx, cx<T>* Qy, SolveState* st, cudaStream_t s);
// Row pass of the split step: C2R(grad p) -> activation -> relaxation -> R2C(m);
// with st->diag the energy's pointwise sums of (m^k, grad p) into st->dsum (r read then).
template <typename T>
void row_split(const Geo<T>& g, const cx<T>* Gx, const cx<T>* Gy, const T* mx, const T* my,
               const T* r, cx<T>* Mx, cx<T>* My, SplitCoef cf, SolveState* st, cudaStream_t s);
// Column pass, forward FFT along y of nv (1|2) row-transformed fields; optional
// projection + ||.||^2 of field 0 into st->outer_b2 (project=1).
template <typename T>
void col_fwd(const Geo<T>& g, const cx<T>* in0, const cx<T>* in1, cx<T>* out0, cx<T>* out1, int nv,
             int project, SolveState* st, cudaStream_t s);
// Column pass, inverse FFT along y of one spectrum, times `scale`.
template <typename T>
void col_inv(const Geo<T>& g, const cx<T>* in, cx<T>* out, T scale, cudaStream_t s);
// Column pass of the gradient: G_x = IFFT_y(i kx P / n), G_y = IFFT_y(i ky P / n).
//   CG_PLAIN:    P = in (Tin may be double while T is float)
//   CG_DUPDATE:  d = M^-1 r + beta d (d = M^-1 r when st->first), stored to dio; P = d
//   CG_ADDDELTA: P = in + delta (FP64 accumulate), stored back to in; P used for the gradient
template <typename T, typename Tin>
void col_grad(const Geo<T>& g, int mode, cx<Tin>* in, const cx<T>* rvec, cx<T>* dio,
              const cx<float>* delta, cx<T>* Gx, cx<T>* Gy, SolveState* st, int check_done,
              cudaStream_t s);
// Column pass of the divergence: q = -i (kx FFT_y(Qx) + ky FFT_y(Qy)).
//   CD_PLAIN:        out = q
//   CD_CG:           out = q; <d, q> -> alpha = rho / <d,q>
//   CD_RESID:        out (r) = b - q; ||r||^2, <r, M^-1 r> -> CG initialisation
//   CD_RESID_REFINE: as CD_RESID in FP64 plus r32 = float(r), delta = 0, and the
//                    outer convergence test
//   CD_RESID_FIRST:  (FP32) r32 = b32 - q, delta = 0, and the start of the first
//                    inner solve (b = the FP32 copy of S; out unused)
template <typename T>
void col_div(const Geo<T>& g, int mode, const cx<T>* Qx, const cx<T>* Qy, const cx<T>* d,
             const cx<T>* b, cx<T>* out, cx<float>* r32, cx<float>* delta32, SolveState* st,
             cudaStream_t s);
// Column pass of the diffusion: FFT_y, times exp(-D^2 |xi|^2 dt) / n, IFFT_y, in place;
// with st && st->diag also sum |grad m_new|^2 into st->gm2_next.
template <typename T>
void col_heat(const Geo<T>& g, cx<T>* Mx, cx<T>* My, SolveState* st, cudaStream_t s);
// sum |grad m|^2 of m given as row spectra (Mx, My), into st->gm2 (into_next = 0) or
// st->gm2_next (1).
template <typename T>
void col_gradnorm(const Geo<T>& g, const cx<T>* Mx, const cx<T>* My, SolveState* st, int into_next,
                  cudaStream_t s);
// CG update: x += alpha d, r -= alpha q, then ||r||^2 and <r, M^-1 r> -> beta, stop test.
template <typename T>
void cg_update(const Geo<T>& g, cx<T>* x, cx<T>* r, const cx<T>* d, const cx<T>* q, SolveState* st,
               cudaStream_t s);
// Elementwise conversions and helpers.
template <typename To, typename Ti>
void convert(const Ti* in, To* out, size_t n, cudaStream_t s);
// Packed 2D spectrum (row-major) -> FP32 column-major copy, the layout of the
// 2D refinement's FP32 vectors (r, delta, the CG direction, S).
template <typename Ti>
void to_cm(const Geo<float>& g, const cx<Ti>* in, cx<float>* out, cudaStream_t s);
template <typename T>
void msum(const Geo<T>& g, const T* mx, const T* my, SolveState* st, cudaStream_t s);

// ---- adjoint (discrete reverse of one step; see the kernels for the formulas)
// Row pass: C2R(grad p), C2R(lambda_b) -> relaxation/activation Jacobians ->
// lambda_m (physical) and lambda_g (row spectra, over G), dL/dc^2.
template <typename T>
void row_adj_point(const Geo<T>& g, cx<T>* G0, cx<T>* G1, const cx<T>* L0, const cx<T>* L1,
                   const T* mx, const T* my, T* lmx, T* lmy, SplitCoef cf, AdjState* as,
                   cudaStream_t s);
// Row pass: C2R(grad mu), C2R(grad p) -> lambda = lambda_m - ((m.gp) gmu + (m.gmu) gp),
// dr -= gmu . gp.
template <typename T>
void row_adj_press(const Geo<T>& g, const cx<T>* GM0, const cx<T>* GM1, const cx<T>* GP0,
                   const cx<T>* GP1, const T* mx, const T* my, const T* lmx, const T* lmy, T* lx,
                   T* ly, double* dr, cudaStream_t s);
// Column pass, one component: dD2 += <lambda_b, (-|xi|^2 dt) b> from A = rows of
// lambda_b (scaled for an unnormalised C2R) and B = rows of b.
template <typename T>
void col_lap_dot(const Geo<T>& g, const cx<T>* A, const cx<T>* B, double dt, AdjState* as,
                 cudaStream_t s);
// Spectral helpers: acc += v (FP64 accumulator); st->outer_b2 = ||v||^2 (Parseval weights).
template <typename T>
void spec_accum(const Geo<T>& g, double* acc, const cx<T>* v, cudaStream_t s);
template <typename T>
void spec_norm2(const Geo<T>& g, const cx<T>* v, SolveState* st, cudaStream_t s);

// ---- 3D (dim = 3).  Spectral vectors are [nz][ny][H]; a physical real field
// is also handled as [nz][ny][H] complex values (pairs of adjacent x values)
// by the y and z heat passes.  Row kernels work on pairs of rows.
// z pass of the gradient: 3 outputs i xi_a P / n, inverse FFT along z (modes as col_grad).
template <typename T, typename Tin>
void z_grad(const Geo<T>& g, int mode, cx<Tin>* in, const cx<T>* rvec, cx<T>* dio,
            const cx<float>* delta, Tri<cx<T>*> G, SolveState* st, int check_done,
            cudaStream_t s);
// FFT along y (axis 1) or z (axis 2) of nv fields, times `scale`; in place allowed.
template <typename T>
void axis_fft(const Geo<T>& g, int axis, int sign, int nv, Tri<cx<T>*> in, Tri<cx<T>*> out,
              T scale, cudaStream_t s);
// Forward FFT along z of one field, corner-mode projection, ||.||^2 into st->outer_b2.
template <typename T>
void z_fwd_project(const Geo<T>& g, const cx<T>* in, cx<T>* out, SolveState* st, cudaStream_t s);
// z pass of the divergence: q = -i xi . FFT_z(Q) (modes as col_div).
template <typename T>
void z_div(const Geo<T>& g, int mode, Tri<cx<T>*> Q, const cx<T>* d, const cx<T>* b, cx<T>* out,
           cx<float>* r32, cx<float>* delta32, SolveState* st, cudaStream_t s);
// Row pass of the 3D apply: C2R(grad p) -> q = (m.g) m + r g -> R2C(q).
template <typename T, typename Tm>
void row_apply3(const Geo<T>& g, Tri<cx<T>*> G, Tri<const Tm*> m, const Tm* r, Tri<cx<T>*> Q,
                SolveState* st, cudaStream_t s);
// Row pass of the 3D split step: C2R(grad p) -> activation -> relaxation ->
// diffusion along x; reads m, writes mo (physical; mo may be the rows of G).
// With st->diag also the energy's pointwise sums (r read then).
template <typename T>
void row_split3(const Geo<T>& g, Tri<cx<T>*> G, Tri<const T*> m, const T* r, Tri<T*> mo,
                SplitCoef cf, SolveState* st, cudaStream_t s);
// Diffusion along y (axis 1) or z (axis 2) of physical m, from mi to mo (may
// alias); axis 2 also sums mo_a mo_b into st->mm and st->msum, flags non-finite values, and
// with st->diag sums |mo - mo_old|^2 into st->dm2 (mo holds m^k on entry).
template <typename T>
void heat_axis(const Geo<T>& g, int axis, Tri<T*> mi, Tri<T*> mo, SolveState* st, cudaStream_t s);
// sum |grad m|^2 of m given as its spectrum after the x and y passes (G), via
// the z pass; into st->gm2 or st->gm2_next.
template <typename T>
void z_gradnorm(const Geo<T>& g, Tri<cx<T>*> G, SolveState* st, int into_next, cudaStream_t s);
template <typename T>
void cg_update3(const Geo<T>& g, cx<T>* x, cx<T>* r, const cx<T>* d, const cx<T>* q,
                SolveState* st, cudaStream_t s);
template <typename T>
void msum3(const Geo<T>& g, Tri<const T*> m, SolveState* st, cudaStream_t s);
void set_smem_limits_3d_f32();
void set_smem_limits_3d_f64();
void set_smem_limits_3d_df();

// Opt every kernel of one precision in to the full shared memory per block.
void set_smem_limits_f32();
void set_smem_limits_f64();
// Lagged certification (2D refined steps): the FP64 certifying residual of
// pressure p with the FP32 m, r it was solved with (sc: the certifying state,
// skipped when nothing is pending); the commit after a lagged step (copies
// guarded by the certification's outcome); the flag update after it.
void cert_resid(const Geo<double>& g, const cx<double>* p, const float* mx, const float* my,
                const float* r, const cx<double>* b, cx<double>* G, SolveState* sc, cudaStream_t s);
void commit_copy(const SolveState* st, const SolveState* sc, float* const* m, float* const* mp,
                 const float* const* mt, const cx<double>* p64, cx<double>* ps, size_t n, size_t ns,
                 cudaStream_t s);
void commit_flags(SolveState* st, SolveState* sc, int final_cert, cudaStream_t s);
void lag_mark(SolveState* st, SolveState* sc, int on, cudaStream_t s);
// FP64 FMA throughput of the current device (TFLOP/s, FMA = 2 flops), reps timed launches on s.
int fma_peak(int reps, cudaStream_t s, double* tflops);
void set_smem_limits_df();
// Solve bookkeeping (one thread): configuration, step start (counters, kappa,
// thresholds), step end (stats and status accumulation), accumulator reset.
void set_config(SolveState* st, SolveConfig cfg, cudaStream_t s);
void step_begin(SolveState* st, int npts, cudaStream_t s);
void step_end(SolveState* st, int refined, cudaStream_t s);
void reset_accum(SolveState* st, cudaStream_t s);
// Batched step of a size class (hc_batch.cu).  Each launches one kernel per
// pass over all members (bi: device array of sh.nb members).  The members'
// own kernels leave the graph conditions alone (graph_mode 0); batch_flags
// sets them to the OR over members and counts the class's launches.
void batch_step_begin(const BInst* bi, const BShape& sh, cudaGraphConditionalHandle h_outer,
                      cudaStream_t s);
void batch_first_resid(const BInst* bi, const BShape& sh, cudaStream_t s);
void batch_cg_iter(const BInst* bi, const BShape& sh, cudaStream_t s);
void batch_mid_resid(const BInst* bi, const BShape& sh, cudaStream_t s);
void batch_refine_resid(const BInst* bi, const BShape& sh, cudaStream_t s);
void batch_split(const BInst* bi, const BShape& sh, cudaStream_t s);
void batch_step_end(const BInst* bi, const BShape& sh, long long* launches, cudaStream_t s);
enum { BF_FIRST = 0, BF_LOOP = 1, BF_REFINE = 2 };
void batch_flags(const BInst* bi, const BShape& sh, int kind, cudaGraphConditionalHandle h1,
                 cudaGraphConditionalHandle h2, long long* launches, int kernels, cudaStream_t s);
void set_smem_limits_batch();
// The generic-size kernels (hc_generic.cu), FP64: column gradient (mode
// CG_PLAIN from `in`, CG_DUPDATE the CG direction update), row apply (st: the
// CG variant with alpha), column divergence (CD_PLAIN, CD_CG, CD_RESID), CG
// update, the split step's row, heat and back-transform passes, and the plain
// transforms of the boundary (row forward, column forward with projection or
// gradient norm, column inverse).
void gen_col_grad(const GenGeo& g, int mode, const cx<double>* in, const cx<double>* rvec,
                  cx<double>* dio, cx<double>* Gx, cx<double>* Gy, SolveState* st, int check_done,
                  cudaStream_t s);
void gen_row_apply(const GenGeo& g, const cx<double>* Gx, const cx<double>* Gy, const double* mx,
                   const double* my, const double* r, cx<double>* Qx, cx<double>* Qy,
                   SolveState* st, cudaStream_t s);
void gen_col_div(const GenGeo& g, int mode, const cx<double>* Qx, const cx<double>* Qy,
                 const cx<double>* b, cx<double>* out, SolveState* st, cudaStream_t s);
void gen_cg_update(const GenGeo& g, cx<double>* x, cx<double>* r, const cx<double>* d,
                   const cx<double>* q, SolveState* st, cudaStream_t s);
void gen_row_split(const GenGeo& g, cx<double>* Gx, cx<double>* Gy, const double* mx,
                   const double* my, const double* r, SplitCoef cf, SolveState* st, cudaStream_t s);
void gen_col_heat(const GenGeo& g, cx<double>* Mx, cx<double>* My, SolveState* st, cudaStream_t s);
void gen_row_c2r(const GenGeo& g, const cx<double>* A, const cx<double>* B, double* a, double* b,
                 SolveState* st, int kappa_update, cudaStream_t s);
void gen_row_fwd(const GenGeo& g, const double* a, const double* b, cx<double>* A, cx<double>* B,
                 cudaStream_t s);
void gen_col_fwd(const GenGeo& g, const cx<double>* in0, const cx<double>* in1, cx<double>* out0,
                 cx<double>* out1, int project, int gradnorm, SolveState* st, cudaStream_t s);
void gen_col_inv(const GenGeo& g, const cx<double>* in, cx<double>* out, double scale,
                 cudaStream_t s);
void set_smem_limits_gen();
// Run mode of Algorithm 1's loop: stopping rules on/off, thresholds; clears halt.
void set_run(SolveState* st, int run_mode, double eps_dm, int stop_energy, cudaStream_t s);
// Sets st->h_gate to 1 unless a stopping rule fired (the gated step of hc_run).
void run_gate(SolveState* st, cudaStream_t s);

}  // namespace hc
