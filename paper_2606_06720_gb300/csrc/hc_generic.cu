// hc_generic.cu -- the step on 2D grids whose sizes are not powers of two:
// N = 2^a 3^b 5^c per axis, among them the paper's N = 50 2^k grids of its
// grid-convergence study (Section 4, Tables 1-3).  FP64 throughout.
//
// Transforms are mixed-radix Stockham FFTs (radix 2, 3, 4, 5 passes) on one
// transform per CTA, held in shared memory, with the CTA's threads sharing
// each pass's butterflies.  The spectral state is the unpacked half spectrum:
// ny rows of Hh = nx/2 + 1 values (kx = 0 .. nx/2), row-major, unnormalised
// DFTs.  A step makes the same passes as the power-of-two path, each fused
// with the same pointwise work:
//   column gradient   d = M^-1 r + beta d (CG) or p, times i xi / n, inverse along y
//   row apply         inverse along x, q = (m.g) m + r g, <d, A d> by parts, forward along x
//   column divergence forward along y, -i xi . q^ (CG output or the residual S - A p)
//   CG update         x += alpha d, r -= alpha A d, the two dot products
//   split step        gradient, row pass with activation + relaxation, column
//                     pass with the heat factor exp(-D^2 |xi|^2 dt), row back-transform
// and the same one-thread solve bookkeeping (SolveState), so CG, its stopping
// rule, kappa / Kbar and the diagnostics of Section 2.5 are shared code.
#include "hc_kernels.cuh"

namespace hc {

namespace {

// ------------------------------------------------------------------ small DFTs
// Kernel exp(S 2 pi i j k / R), natural order in and out.  The radix-3 and
// radix-5 constants are the closed forms cos(2 pi/3) = -1/2,
// sin(2 pi/3) = sqrt(3)/2, cos(2 pi/5) = (sqrt 5 - 1)/4,
// cos(4 pi/5) = -(sqrt 5 + 1)/4, sin(2 pi/5) = sqrt(10 + 2 sqrt 5)/4,
// sin(4 pi/5) = sqrt(10 - 2 sqrt 5)/4.
template <int S>
__device__ __forceinline__ void gdft3(cx<double>* v) {
  const double h = 0.86602540378443864676;
  const cx<double> a = cadd(v[1], v[2]), b = csub(v[1], v[2]);
  const cx<double> t = cmk<double>(v[0].x - 0.5 * a.x, v[0].y - 0.5 * a.y);
  const cx<double> u = cmul_si<S>(cmk<double>(h * b.x, h * b.y));
  v[0] = cadd(v[0], a);
  v[1] = cadd(t, u);
  v[2] = csub(t, u);
}

template <int S>
__device__ __forceinline__ void gdft5(cx<double>* v) {
  const double c1 = 0.30901699437494742410, c2 = -0.80901699437494742410;
  const double s1 = 0.95105651629515357212, s2 = 0.58778525229247312917;
  const cx<double> a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
  const cx<double> a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
  const cx<double> t1 = cmk<double>(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
  const cx<double> t2 = cmk<double>(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
  const cx<double> u1 =
      cmul_si<S>(cmk<double>(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
  const cx<double> u2 =
      cmul_si<S>(cmk<double>(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
  v[0] = cmk<double>(v[0].x + a1.x + a2.x, v[0].y + a1.y + a2.y);
  v[1] = cadd(t1, u1);
  v[4] = csub(t1, u1);
  v[2] = cadd(t2, u2);
  v[3] = csub(t2, u2);
}

// One radix-R pass of a length-N Stockham FFT, by all threads of the CTA:
// butterfly j < N/R takes src[j + r N/R], r < R, twiddles element r by
// w^(r k), k = j mod Ns, w = exp(S 2 pi i / (Ns R)) (a table entry
// tw[m] = exp(-2 pi i m / N), conjugated for S = +1), and writes
// dst[(j / Ns) Ns R + k + r Ns].
template <int S, int R>
__device__ __forceinline__ void gpass(const cx<double>* __restrict__ src, cx<double>* __restrict__ dst,
                                      int N, int Ns, const cx<double>* __restrict__ tw) {
  const int nb = N / R, step = N / (Ns * R);
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int k = j % Ns;
    cx<double> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[j + r * nb];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cx<double> w = ldg(&tw[r * k * step]);
        if (S > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    if constexpr (R == 2) dft2<S>(v[0], v[1]);
    if constexpr (R == 3) gdft3<S>(v);
    if constexpr (R == 4) dft4<S>(v[0], v[1], v[2], v[3]);
    if constexpr (R == 5) gdft5<S>(v);
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[base + r * Ns] = v[r];
  }
}

// Length-N transform of the values in a (scratch b), S = -1 forward, +1
// inverse (unnormalised).  The caller synchronises after filling a; returns
// the buffer that holds the result, synchronised.
template <int S>
__device__ cx<double>* gfft(cx<double>* a, cx<double>* b, int N, const int* rad, int np,
                            const cx<double>* __restrict__ tw) {
  int Ns = 1;
  for (int p = 0; p < np; ++p) {
    const int R = rad[p];
    if (R == 2)
      gpass<S, 2>(a, b, N, Ns, tw);
    else if (R == 3)
      gpass<S, 3>(a, b, N, Ns, tw);
    else if (R == 4)
      gpass<S, 4>(a, b, N, Ns, tw);
    else
      gpass<S, 5>(a, b, N, Ns, tw);
    __syncthreads();
    cx<double>* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// Parseval weight of half-spectrum column kx: 1 for kx = 0 and (even nx) the
// Nyquist column, 2 for the others, whose mirror columns are not stored.
__device__ __forceinline__ double gweight(const GenGeo& g, int kx) {
  return (kx == 0 || 2 * kx == g.nx) ? 1.0 : 2.0;
}
// Null modes of the operator (reading R2): every index 0 or a Nyquist index.
__device__ __forceinline__ bool gnull(const GenGeo& g, int kx, int ky) {
  return (kx == 0 || 2 * kx == g.nx) && (ky == 0 || 2 * ky == g.ny);
}

// Full-length row z = A + i B of two real fields from their half spectra
// (the mirror half by conjugate symmetry); B may be null.
__device__ __forceinline__ void gload_pair(const GenGeo& g, const cx<double>* A, const cx<double>* B,
                                           cx<double>* z) {
  const int N = g.nx, H = g.Hh;
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const int kk = k < H ? k : N - k;
    const cx<double> a = A[kk], b = B ? B[kk] : czero<double>();
    z[k] = k < H ? cmk<double>(a.x - b.y, a.y + b.x) : cmk<double>(a.x + b.y, b.x - a.y);
  }
}
// Half spectra of a and b from the spectrum Z of the row a + i b.
__device__ __forceinline__ void gstore_pair(const GenGeo& g, const cx<double>* Z, cx<double>* A,
                                            cx<double>* B) {
  const int N = g.nx, H = g.Hh;
  for (int k = threadIdx.x; k < H; k += blockDim.x) {
    const cx<double> z = Z[k], zc = Z[k == 0 ? 0 : N - k];
    A[k] = cmk<double>(0.5 * (z.x + zc.x), 0.5 * (z.y - zc.y));
    if (B) B[k] = cmk<double>(0.5 * (z.y + zc.y), -0.5 * (z.x - zc.x));
  }
}

}  // namespace

// ------------------------------------------------------------------ column gradient
template <int MODE>
__global__ void __launch_bounds__(256) gk_col_grad(GenGeo g, const cx<double>* __restrict__ in,
                                                   const cx<double>* __restrict__ rvec,
                                                   cx<double>* dio, cx<double>* __restrict__ Gx,
                                                   cx<double>* __restrict__ Gy, SolveState* st,
                                                   int check_done) {
  if (check_done && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = g.ny, H = g.Hh, kx = blockIdx.x;
  cx<double>* P = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* A = P + ny;
  cx<double>* B = A + ny;
  const double invn = 1.0 / ((double)g.nx * (double)ny);
  const double kxv = g.kxd[kx];
  bool first = false;
  double beta = 0;
  Pc<double> pc{};
  if (MODE == CG_DUPDATE) {
    first = st->first != 0;
    beta = st->beta;
    pc = pc_of<double>(st);
  }
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
    const size_t idx = (size_t)ky * H + kx;
    cx<double> v;
    if constexpr (MODE == CG_DUPDATE) {
      const cx<double> z = cscale(rvec[idx], pinv_ab(kxv, g.kyd[ky], pc));
      v = first ? z : cadd(z, cscale(dio[idx], beta));
      dio[idx] = v;
    } else {
      v = in[idx];
    }
    P[ky] = v;
    const double a = kxv * invn;
    A[ky] = cmk<double>(-a * v.y, a * v.x);  // i (xi_x / n) P
  }
  __syncthreads();
  cx<double>* R = gfft<+1>(A, B, ny, g.ry, g.nry, g.twy);
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) Gx[(size_t)ky * H + kx] = R[ky];
  __syncthreads();
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
    const double a = g.kyd[ky] * invn;
    A[ky] = cmk<double>(-a * P[ky].y, a * P[ky].x);  // i (xi_y / n) P
  }
  __syncthreads();
  R = gfft<+1>(A, B, ny, g.ry, g.nry, g.twy);
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) Gy[(size_t)ky * H + kx] = R[ky];
}

// ------------------------------------------------------------------ row apply
// DOT: the CG variant; alpha = rho / <d, A d> with <d, A d> = n sum g . K g
// (summation by parts), as in the power-of-two row pass.
template <bool DOT>
__global__ void __launch_bounds__(256) gk_row_apply(GenGeo g, const cx<double>* Gx,
                                                    const cx<double>* Gy,
                                                    const double* __restrict__ mx,
                                                    const double* __restrict__ my,
                                                    const double* __restrict__ rr, cx<double>* Qx,
                                                    cx<double>* Qy, SolveState* st) {
  if (DOT && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = g.nx, H = g.Hh, y = blockIdx.x;
  cx<double>* A = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* B = A + N;
  gload_pair(g, Gx + (size_t)y * H, Gy + (size_t)y * H, A);
  __syncthreads();
  cx<double>* R = gfft<+1>(A, B, N, g.rx, g.nrx, g.twx);
  double gkg = 0.0;
  const size_t ro = (size_t)y * N;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const double gx = R[x].x, gy = R[x].y;
    const double ax = mx[ro + x], ay = my[ro + x], r = rr[ro + x];
    const double mg = ax * gx + ay * gy;
    if (DOT) gkg += mg * mg + r * (gx * gx + gy * gy);
    R[x] = cmk<double>(ax * mg + r * gx, ay * mg + r * gy);
  }
  __syncthreads();
  cx<double>* R2 = gfft<-1>(R, R == A ? B : A, N, g.rx, g.nrx, g.twx);
  gstore_pair(g, R2, Qx + (size_t)y * H, Qy + (size_t)y * H);
  if (DOT) {
    double a1[1] = {gkg}, t1[1];
    if (last_cta_sum<1>(a1, g.partials, &st->ticket[TK_DIV], t1) && threadIdx.x == 0)
      cg_alpha_from(st, t1[0], (double)g.nx * (double)g.ny);
  }
}

// ------------------------------------------------------------------ column divergence
// -i (xi_x Qx^ + xi_y Qy^) after the forward transforms along y.  CD_PLAIN:
// written to out; CD_CG: the CG's A d (alpha came from the row pass);
// CD_RESID: out = b - A p and the CG start (plain solve).
template <int MODE>
__global__ void __launch_bounds__(256) gk_col_div(GenGeo g, const cx<double>* __restrict__ Qx,
                                                  const cx<double>* __restrict__ Qy,
                                                  const cx<double>* __restrict__ bvec,
                                                  cx<double>* __restrict__ out, SolveState* st) {
  if (MODE == CD_CG && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = g.ny, H = g.Hh, kx = blockIdx.x;
  cx<double>* T = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* A = T + ny;
  cx<double>* B = A + ny;
  const double kxv = g.kxd[kx];
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) A[ky] = Qx[(size_t)ky * H + kx];
  __syncthreads();
  cx<double>* R = gfft<-1>(A, B, ny, g.ry, g.nry, g.twy);
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) T[ky] = cscale(R[ky], kxv);
  __syncthreads();
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) A[ky] = Qy[(size_t)ky * H + kx];
  __syncthreads();
  R = gfft<-1>(A, B, ny, g.ry, g.nry, g.twy);
  const double w = gweight(g, kx);
  double acc[2] = {0.0, 0.0};
  Pc<double> pc{};
  if (MODE == CD_RESID) pc = pc_of<double>(st);
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
    const size_t idx = (size_t)ky * H + kx;
    const double b = g.kyd[ky];
    const cx<double> t = cmk<double>(T[ky].x + b * R[ky].x, T[ky].y + b * R[ky].y);
    const cx<double> q = cmk<double>(t.y, -t.x);
    if constexpr (MODE == CD_RESID) {
      const cx<double> rv = csub(bvec[idx], q);
      out[idx] = rv;
      const double r2 = rv.x * rv.x + rv.y * rv.y;
      acc[0] += w * r2;
      acc[1] += w * r2 * pinv_ab(kxv, b, pc);
    } else {
      out[idx] = q;
    }
  }
  if constexpr (MODE == CD_RESID) {
    double t2[2];
    if (last_cta_sum<2>(acc, g.partials, &st->ticket[TK_RESID], t2) && threadIdx.x == 0)
      resid_init(st, t2[0], t2[1]);
  }
}

// ------------------------------------------------------------------ CG update
__global__ void __launch_bounds__(256) gk_cg_update(GenGeo g, cx<double>* __restrict__ x,
                                                    cx<double>* __restrict__ r,
                                                    const cx<double>* __restrict__ d,
                                                    const cx<double>* __restrict__ q,
                                                    SolveState* st) {
  if (st->done) {
    if (st->graph_mode && blockIdx.x == 0 && threadIdx.x == 0)
      cudaGraphSetConditional(st->h_cur, 0u);
    return;
  }
  const double alpha = st->alpha;
  const Pc<double> pc = pc_of<double>(st);
  const int H = g.Hh;
  const size_t total = (size_t)g.ny * H;
  double rr = 0.0, rz = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % (size_t)H), ky = (int)(i / (size_t)H);
    const cx<double> dv = d[i], qv = q[i];
    x[i] = cmk<double>(x[i].x + alpha * dv.x, x[i].y + alpha * dv.y);
    const cx<double> rv = cmk<double>(r[i].x - alpha * qv.x, r[i].y - alpha * qv.y);
    r[i] = rv;
    const double w = gweight(g, kx), r2 = rv.x * rv.x + rv.y * rv.y;
    rr += w * r2;
    rz += w * r2 * pinv_ab(g.kxd[kx], g.kyd[ky], pc);
  }
  double acc[2] = {rr, rz}, tot[2];
  if (last_cta_sum<2>(acc, g.partials, &st->ticket[TK_UPDATE], tot) && threadIdx.x == 0)
    cg_step_finish(st, tot[0], tot[1]);
}

// ------------------------------------------------------------------ split step
// Row pass: grad p^{k+1} (from the column pass), activation and relaxation per
// point (split_point, as the power-of-two row pass), the energy's pointwise
// sums of m^k with diagnostics on, then the forward transform along x of the
// new m into Mx, My (the gradient's buffers).
__global__ void __launch_bounds__(256) gk_row_split(GenGeo g, cx<double>* Gx, cx<double>* Gy,
                                                    const double* __restrict__ mx,
                                                    const double* __restrict__ my,
                                                    const double* __restrict__ rr, SplitCoef cf,
                                                    SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = g.nx, H = g.Hh, y = blockIdx.x;
  cx<double>* A = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* B = A + N;
  gload_pair(g, Gx + (size_t)y * H, Gy + (size_t)y * H, A);
  __syncthreads();
  cx<double>* R = gfft<+1>(A, B, N, g.rx, g.nrx, g.twx);
  const size_t ro = (size_t)y * N;
  const bool diag = st->diag != 0;
  bool finite = true;
  EnergyAcc<double> en;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const double gx = R[x].x, gy = R[x].y;
    double ax = mx[ro + x], ay = my[ro + x];
    if (diag) en.add(rr[ro + x], gx * gx + gy * gy, ax * gx + ay * gy, ax * ax + ay * ay, cf.gamma);
    split_point<double>(ax, ay, gx, gy, cf.c2dt, cf);
    finite = finite && isfinite(ax) && isfinite(ay);
    R[x] = cmk<double>(ax, ay);
  }
  if (!finite) st->nonfinite = 1;
  if (diag) en.finish(g.partials, st);
  __syncthreads();
  cx<double>* R2 = gfft<-1>(R, R == A ? B : A, N, g.rx, g.nrx, g.twx);
  gstore_pair(g, R2, Gx + (size_t)y * H, Gy + (size_t)y * H);
}

// Column pass of the diffusion, in place: forward along y, times
// exp(-D^2 |xi|^2 dt) / n (eq. diffusion_space_discrete), inverse along y.
// With diagnostics, sum |grad m_new|^2 = n sum w |xi~|^2 |v|^2 (v = F(m_new)/n).
__global__ void __launch_bounds__(256) gk_col_heat(GenGeo g, cx<double>* Mx, cx<double>* My,
                                                   SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = g.ny, H = g.Hh, kx = blockIdx.x;
  cx<double>* A = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* B = A + ny;
  const double invn = 1.0 / ((double)g.nx * (double)ny);
  const double w = gweight(g, kx), a = g.kxd[kx];
  double gm = 0.0;
  for (int f = 0; f < 2; ++f) {
    cx<double>* M = f == 0 ? Mx : My;
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) A[ky] = M[(size_t)ky * H + kx];
    __syncthreads();
    cx<double>* R = gfft<-1>(A, B, ny, g.ry, g.nry, g.twy);
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
      const cx<double> v = cscale(R[ky], g.hx[kx] * g.hy[ky] * invn);
      R[ky] = v;
      const double b = g.kyd[ky];
      gm += w * (a * a + b * b) * (v.x * v.x + v.y * v.y);
    }
    __syncthreads();
    cx<double>* R2 = gfft<+1>(R, R == A ? B : A, ny, g.ry, g.nry, g.twy);
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) M[(size_t)ky * H + kx] = R2[ky];
    __syncthreads();
  }
  if (st && st->diag) gradnorm_finish(gm, (double)g.nx * (double)ny, g.partials, st, 1);
}

// Row back-transform of two fields: half spectra A, B -> physical a, b (B, b
// may be null).  With kappa_update: the sums of m_a m_b for the next
// preconditioner, the non-finite check, and with diagnostics sum |new - old|^2.
__global__ void __launch_bounds__(256) gk_row_c2r(GenGeo g, const cx<double>* A, const cx<double>* B,
                                                  double* a, double* b, SolveState* st,
                                                  int kappa_update) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = g.nx, H = g.Hh, y = blockIdx.x;
  cx<double>* Z = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* W = Z + N;
  gload_pair(g, A + (size_t)y * H, B ? B + (size_t)y * H : nullptr, Z);
  __syncthreads();
  cx<double>* R = gfft<+1>(Z, W, N, g.rx, g.nrx, g.twx);
  const size_t ro = (size_t)y * N;
  const bool diag = kappa_update && st->diag;
  double mxx = 0, myy = 0, mxy = 0, d2 = 0;
  bool finite = true;
  for (int x = threadIdx.x; x < N; x += blockDim.x) {
    const double u = R[x].x, v = R[x].y;
    if (diag) {
      const double du = u - a[ro + x], dv = v - b[ro + x];
      d2 += du * du + dv * dv;
    }
    a[ro + x] = u;
    if (b) b[ro + x] = v;
    if (kappa_update) {
      mxx += u * u;
      myy += v * v;
      mxy += u * v;
      finite = finite && isfinite(u) && isfinite(v);
    }
  }
  if (kappa_update) {
    if (!finite) st->nonfinite = 1;
    double acc[4] = {mxx, myy, mxy, d2}, tot[4];
    if (last_cta_sum<4>(acc, g.partials, &st->ticket[TK_MSUM], tot) && threadIdx.x == 0) {
      set_mm2(st, tot[0], tot[1], tot[2]);
      if (diag) st->dm2 = tot[3];
    }
  }
}

// ------------------------------------------------------------------ plain transforms
// Forward transform along x of the real rows a (+ i b): half spectra A (, B).
__global__ void __launch_bounds__(256) gk_row_fwd(GenGeo g, const double* __restrict__ a,
                                                  const double* __restrict__ b, cx<double>* A,
                                                  cx<double>* B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = g.nx, H = g.Hh, y = blockIdx.x;
  cx<double>* Z = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* W = Z + N;
  const size_t ro = (size_t)y * N;
  for (int x = threadIdx.x; x < N; x += blockDim.x)
    Z[x] = cmk<double>(a[ro + x], b ? b[ro + x] : 0.0);
  __syncthreads();
  cx<double>* R = gfft<-1>(Z, W, N, g.rx, g.nrx, g.twx);
  gstore_pair(g, R, A + (size_t)y * H, B ? B + (size_t)y * H : nullptr);
}

// Forward transform along y of one or two half-spectrum fields.  project:
// the null modes of field 0 are zeroed (the solvability condition, reading
// R2) and, with st, sum w |F|^2 of field 0 goes to st->outer_b2.  gradnorm:
// instead, sum w |xi~|^2 |F|^2 / n over both fields (|grad m|^2 of the
// physical fields) goes to st->gm2 (the outputs may then be null).
__global__ void __launch_bounds__(256) gk_col_fwd(GenGeo g, const cx<double>* in0,
                                                  const cx<double>* in1, cx<double>* out0,
                                                  cx<double>* out1, int project, int gradnorm,
                                                  SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = g.ny, H = g.Hh, kx = blockIdx.x;
  cx<double>* A = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* B = A + ny;
  const double w = gweight(g, kx), a = g.kxd[kx];
  double acc = 0.0;
  for (int f = 0; f < (in1 ? 2 : 1); ++f) {
    const cx<double>* in = f == 0 ? in0 : in1;
    cx<double>* out = f == 0 ? out0 : out1;
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) A[ky] = in[(size_t)ky * H + kx];
    __syncthreads();
    cx<double>* R = gfft<-1>(A, B, ny, g.ry, g.nry, g.twy);
    for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) {
      cx<double> v = R[ky];
      if (project && f == 0 && gnull(g, kx, ky)) v = czero<double>();
      if (out) out[(size_t)ky * H + kx] = v;
      const double n2 = v.x * v.x + v.y * v.y;
      if (gradnorm) {
        const double b = g.kyd[ky];
        acc += w * (a * a + b * b) * n2;
      } else if (f == 0) {
        acc += w * n2;
      }
    }
    __syncthreads();
  }
  if (gradnorm && st) {
    gradnorm_finish(acc, 1.0 / ((double)g.nx * (double)ny), g.partials, st, 0);
  } else if (project && st) {
    double a1[1] = {acc}, t1[1];
    if (last_cta_sum<1>(a1, g.partials, &st->ticket[TK_PROJ], t1) && threadIdx.x == 0)
      st->outer_b2 = t1[0];
  }
}

// Inverse transform along y of one half-spectrum field, times scale.
__global__ void __launch_bounds__(256) gk_col_inv(GenGeo g, const cx<double>* in, cx<double>* out,
                                                  double scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ny = g.ny, H = g.Hh, kx = blockIdx.x;
  cx<double>* A = reinterpret_cast<cx<double>*>(smem_raw);
  cx<double>* B = A + ny;
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x) A[ky] = in[(size_t)ky * H + kx];
  __syncthreads();
  cx<double>* R = gfft<+1>(A, B, ny, g.ry, g.nry, g.twy);
  for (int ky = threadIdx.x; ky < ny; ky += blockDim.x)
    out[(size_t)ky * H + kx] = cscale(R[ky], scale);
}

// ------------------------------------------------------------------ launchers
namespace {
constexpr int kGenThreads = 256;
size_t gcol_smem(const GenGeo& g, int bufs) { return (size_t)bufs * g.ny * sizeof(cx<double>); }
size_t grow_smem(const GenGeo& g) { return (size_t)2 * g.nx * sizeof(cx<double>); }
int gupd_blocks(const GenGeo& g) {
  const size_t b = ((size_t)g.ny * g.Hh + kGenThreads - 1) / kGenThreads;
  return (int)(b < 608 ? b : 608);
}
}  // namespace

void gen_col_grad(const GenGeo& g, int mode, const cx<double>* in, const cx<double>* rvec,
                  cx<double>* dio, cx<double>* Gx, cx<double>* Gy, SolveState* st, int check_done,
                  cudaStream_t s) {
  if (mode == CG_DUPDATE)
    gk_col_grad<CG_DUPDATE><<<g.Hh, kGenThreads, gcol_smem(g, 3), s>>>(g, in, rvec, dio, Gx, Gy, st,
                                                                       check_done);
  else
    gk_col_grad<CG_PLAIN><<<g.Hh, kGenThreads, gcol_smem(g, 3), s>>>(g, in, rvec, dio, Gx, Gy, st,
                                                                     check_done);
}
void gen_row_apply(const GenGeo& g, const cx<double>* Gx, const cx<double>* Gy, const double* mx,
                   const double* my, const double* r, cx<double>* Qx, cx<double>* Qy,
                   SolveState* st, cudaStream_t s) {
  if (st)
    gk_row_apply<true><<<g.ny, kGenThreads, grow_smem(g), s>>>(g, Gx, Gy, mx, my, r, Qx, Qy, st);
  else
    gk_row_apply<false><<<g.ny, kGenThreads, grow_smem(g), s>>>(g, Gx, Gy, mx, my, r, Qx, Qy, st);
}
void gen_col_div(const GenGeo& g, int mode, const cx<double>* Qx, const cx<double>* Qy,
                 const cx<double>* b, cx<double>* out, SolveState* st, cudaStream_t s) {
  if (mode == CD_RESID)
    gk_col_div<CD_RESID><<<g.Hh, kGenThreads, gcol_smem(g, 3), s>>>(g, Qx, Qy, b, out, st);
  else if (mode == CD_CG)
    gk_col_div<CD_CG><<<g.Hh, kGenThreads, gcol_smem(g, 3), s>>>(g, Qx, Qy, b, out, st);
  else
    gk_col_div<CD_PLAIN><<<g.Hh, kGenThreads, gcol_smem(g, 3), s>>>(g, Qx, Qy, b, out, st);
}
void gen_cg_update(const GenGeo& g, cx<double>* x, cx<double>* r, const cx<double>* d,
                   const cx<double>* q, SolveState* st, cudaStream_t s) {
  gk_cg_update<<<gupd_blocks(g), kGenThreads, 0, s>>>(g, x, r, d, q, st);
}
void gen_row_split(const GenGeo& g, cx<double>* Gx, cx<double>* Gy, const double* mx,
                   const double* my, const double* r, SplitCoef cf, SolveState* st,
                   cudaStream_t s) {
  gk_row_split<<<g.ny, kGenThreads, grow_smem(g), s>>>(g, Gx, Gy, mx, my, r, cf, st);
}
void gen_col_heat(const GenGeo& g, cx<double>* Mx, cx<double>* My, SolveState* st, cudaStream_t s) {
  gk_col_heat<<<g.Hh, kGenThreads, gcol_smem(g, 2), s>>>(g, Mx, My, st);
}
void gen_row_c2r(const GenGeo& g, const cx<double>* A, const cx<double>* B, double* a, double* b,
                 SolveState* st, int kappa_update, cudaStream_t s) {
  gk_row_c2r<<<g.ny, kGenThreads, grow_smem(g), s>>>(g, A, B, a, b, st, kappa_update);
}
void gen_row_fwd(const GenGeo& g, const double* a, const double* b, cx<double>* A, cx<double>* B,
                 cudaStream_t s) {
  gk_row_fwd<<<g.ny, kGenThreads, grow_smem(g), s>>>(g, a, b, A, B);
}
void gen_col_fwd(const GenGeo& g, const cx<double>* in0, const cx<double>* in1, cx<double>* out0,
                 cx<double>* out1, int project, int gradnorm, SolveState* st, cudaStream_t s) {
  gk_col_fwd<<<g.Hh, kGenThreads, gcol_smem(g, 2), s>>>(g, in0, in1, out0, out1, project, gradnorm,
                                                        st);
}
void gen_col_inv(const GenGeo& g, const cx<double>* in, cx<double>* out, double scale,
                 cudaStream_t s) {
  gk_col_inv<<<g.Hh, kGenThreads, gcol_smem(g, 2), s>>>(g, in, out, scale);
}

void set_smem_limits_gen() {
  allow_smem(gk_col_grad<CG_PLAIN>);
  allow_smem(gk_col_grad<CG_DUPDATE>);
  allow_smem(gk_row_apply<true>);
  allow_smem(gk_row_apply<false>);
  allow_smem(gk_col_div<CD_PLAIN>);
  allow_smem(gk_col_div<CD_CG>);
  allow_smem(gk_col_div<CD_RESID>);
  allow_smem(gk_row_split);
  allow_smem(gk_col_heat);
  allow_smem(gk_row_c2r);
  allow_smem(gk_row_fwd);
  allow_smem(gk_col_fwd);
  allow_smem(gk_col_inv);
}

}  // namespace hc
