// hc_kernels3d.cuh -- sm_103a kernels of the 3D step (d = 3) of the Fourier
// spectral scheme for the periodic Hu-Cai system (arXiv 2606.06720, Section 2;
// the method is stated for any dimension, Section 2.3).
//
// A 3D transform is three passes: the x pass over the ny*nz rows (the 2D row
// kernels, and below the row-pair kernels), a y pass per z plane, and a z pass
// over all ny*H packed columns.  Spectra keep the 2D packing along x:
//   P[kz][ky][0] = F[kz][ky][0] + i F[kz][ky][nx/2].
// The first-derivative multipliers and the preconditioner are equal for the two
// packed x columns (the x Nyquist multiplier is zero), so the pressure solve
// needs no unpacking.  Diffusion is applied as three 1D heat operators, one per
// axis: exp(-D^2 |xi|^2 dt) = exp(-D^2 xi_x^2 dt) exp(-D^2 xi_y^2 dt)
// exp(-D^2 xi_z^2 dt), so F^-1 diag(h) F factors into commuting 1D operators
// (eq. diffusion_space_discrete).  The x factor runs inside the row split
// kernel on complex rows; the y and z factors run on physical m viewed as
// complex pairs of adjacent x values (a real, even multiplier acts on re and
// im separately).  That avoids the packed-column coupling of the 2D heat pass
// and one full pass over m.
//
// Per CG iteration: z_grad (d-update + 3 gradients + inverse z), inverse y,
// row_apply3, forward y, z_div (divergence + <d, Ad>), cg_update3.
//
// Every transform kernel here holds three transforms of 8 complex values per
// thread, so CTAs have at most 256 threads (up to 255 registers per thread,
// no spills in FP64); the host sizes tiles accordingly.
#pragma once

#include "hc_kernels.cuh"

namespace hc {

// ------------------------------------------------------------------ helpers
// Thread and tile of a column pass: b = column within the tile (fastest),
// j = FFT thread; element e of this thread's transform at base + e * stride.
struct CIdx3 {
  int b, j, L8, col;
  size_t base;
};
__device__ __forceinline__ CIdx3 cidx3(const ColPass& p) {
  CIdx3 c;
  c.b = threadIdx.x & ((1 << p.ltc) - 1);
  c.j = threadIdx.x >> p.ltc;
  c.L8 = 1 << (p.lL - 3);
  const int plane = blockIdx.x >> p.lt;
  c.col = ((blockIdx.x & ((1 << p.lt) - 1)) << p.ltc) + c.b;
  c.base = (size_t)plane * (size_t)p.pstride + (size_t)c.col;
  return c;
}
// Elements of one padded slab of a column pass: (L + L/8) * tc.
__device__ __forceinline__ int slab3(const ColPass& p) { return (9 << (p.lL - 3)) << p.ltc; }

// The sums sum m_a m_b of the current m (xx, yy, zz, xy, xz, yz) and sum |m|^2,
// the inputs of the next step's preconditioner (reading R3).
__device__ __forceinline__ void set_mm3(SolveState* st, const double* t) {
#pragma unroll
  for (int e = 0; e < 6; ++e) st->mm[e] = t[e];
  st->msum = t[0] + t[1] + t[2];
}

// Preconditioner symbol 1 / (xi~^T Kbar xi~) in 3D (0 on the 8 null modes).
template <typename T>
__device__ __forceinline__ T pinv3_abc(T a, T b, T c, const Pc<T>& k) {
  const T s2 = k.xx * a * a + k.yy * b * b + k.zz * c * c +
               (T)2 * (k.xy * a * b + k.xz * a * c + k.yz * b * c);
  return s2 > (T)0 ? (T)1 / s2 : (T)0;
}
template <typename T>
__device__ __forceinline__ T pinv3(const Geo<T>& g, int kx, int ky, int kz, const Pc<T>& k) {
  return pinv3_abc(g.kxd[kx], g.kyd[ky], g.kzd[kz], k);
}
template <typename T>
__device__ __forceinline__ float pinv3_f32(const Geo<T>& g, int kx, int ky, int kz, const Pc<float>& k) {
  return pinv3_abc((float)g.kxd[kx], (float)g.kyd[ky], (float)g.kzd[kz], k);
}

// From NV canonical-order row spectra Z_q (of complex rows a_q + i b_q), write
// the packed half spectra of a_q and b_q.
template <int NV, typename T>
__device__ __forceinline__ void store_pairs_r2c(cx<T> (&v)[NV][8], cx<T>* const* sl, int j, int N,
                                                int H, const Tri<cx<T>*>& A,
                                                const Tri<cx<T>*>& B) {
  const int N8 = N >> 3;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q)
#pragma unroll
    for (int s = 0; s < 8; ++s) sl[q][rswz<T>(j + s * N8)] = v[q][s];
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int k = j + s * N8;  // k < H
      const cx<T> z = sl[q][rswz<T>(k)];
      cx<T> a, b;
      if (k == 0) {
        const cx<T> zh = sl[q][rswz<T>(H)];
        a = cmk<T>(z.x, zh.x);
        b = cmk<T>(z.y, zh.y);
      } else {
        const cx<T> zc = sl[q][rswz<T>(N - k)];
        a = cmk<T>((T)0.5 * (z.x + zc.x), (T)0.5 * (z.y - zc.y));
        b = cmk<T>((T)0.5 * (z.y + zc.y), (T)-0.5 * (z.x - zc.x));
      }
      A.v[q][k] = a;
      B.v[q][k] = b;
    }
  }
}

// Row-pair thread layout: unit u of the CTA owns rows y0 = 2U, y1 = 2U + 1
// (U = blockIdx.x * upc + u); j = FFT thread.  Three complex transforms per
// unit: (x0 + i y0 components of row y0), (same for row y1), (z of y0 + i z of y1).
struct RIdx3 {
  int u, j, N8;
  size_t y0, y1;
};
template <typename T>
__device__ __forceinline__ RIdx3 ridx3(const Geo<T>& g) {
  RIdx3 r;
  const int l8 = g.lnx - 3;
  r.N8 = 1 << l8;
  r.u = threadIdx.x >> l8;
  r.j = threadIdx.x & (r.N8 - 1);
  const size_t U = ((size_t)blockIdx.x << g.lupc) + r.u;
  r.y0 = 2 * U;
  r.y1 = 2 * U + 1;
  return r;
}

// Load the three row transforms of a gradient-like field G (packed row spectra).
template <typename T>
__device__ __forceinline__ void load_rows3(cx<T> (&v)[3][8], const Tri<cx<T>*>& G,
                                           const RIdx3& r, int H) {
  const size_t o0 = r.y0 * H, o1 = r.y1 * H;
  const cx<T>* A3[3] = {G.v[0] + o0, G.v[0] + o1, G.v[2] + o0};
  const cx<T>* B3[3] = {G.v[1] + o0, G.v[1] + o1, G.v[2] + o1};
  load_rows_c2r<3>(v, A3, B3, r.j, r.N8);
}

// ------------------------------------------------------------------ z pass: gradient
template <typename T, typename Tin, int MODE>
__global__ void __launch_bounds__(256) k3_zgrad(Geo<T> g, cx<Tin>* in, const cx<T>* __restrict__ rvec,
                                                cx<T>* dio, const cx<float>* __restrict__ delta,
                                                Tri<cx<T>*> G, SolveState* st, int check_done) {
  if (check_done && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColPass& p = g.pz;
  const CIdx3 c = cidx3(p);
  const int se = slab3(p);
  cx<T>* const sl[3] = {sm + c.b, sm + se + c.b, sm + 2 * se + c.b};
  const T invn = exp2_neg<T>(g.lnx + g.lny + g.lnz);  // 1 / (nx ny nz)
  const int kx = c.col & (g.H - 1), ky = c.col >> g.lH;
  const T ax = g.kxd[kx] * invn, ay = g.kyd[ky] * invn;
  bool first = false, add_delta = false;
  T beta = 0;
  Pc<T> pc{};
  if (MODE == CG_DUPDATE) {
    first = st->first != 0;
    beta = st_beta<T>(st);
    pc = pc_of<T>(st);
  }
  if (MODE == CG_ADDDELTA) add_delta = st->sweeps > 0;
  cx<T> v[3][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int kz = c.j + s * c.L8;
    const size_t idx = c.base + (size_t)kz * (size_t)p.stride;
    cx<T> P;
    if constexpr (MODE == CG_PLAIN) {
      P = ccast<T>(in[idx]);
    } else if constexpr (MODE == CG_DUPDATE) {
      const T pv = pinv3(g, kx, ky, kz, pc);
      const cx<T> z = cscale(rvec[idx], pv);
      P = first ? z : cadd(z, cscale(dio[idx], beta));
      dio[idx] = P;
    } else {
      P = add_delta ? add_delta_at<T>(in, idx, delta[idx]) : ccast<T>(in[idx]);
    }
    const T az = g.kzd[kz] * invn;
    v[0][s] = cmk<T>(-ax * P.y, ax * P.x);  // i (kx/n) P
    v[1][s] = cmk<T>(-ay * P.y, ay * P.x);
    v[2][s] = cmk<T>(-az * P.y, az * P.x);
  }
  fft_canon<+1, 3>(v, sl, 1 << p.ltc, c.j, p.lL, g.twz);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = c.base + (size_t)(c.j + s * c.L8) * (size_t)p.stride;
#pragma unroll
    for (int q = 0; q < 3; ++q) G.v[q][idx] = v[q][s];
  }
}

// ------------------------------------------------------------------ plain axis FFT
template <typename T, int S, int NV>
__global__ void __launch_bounds__(256) k3_axis_fft(Geo<T> g, int axis, Tri<cx<T>*> in,
                                                   Tri<cx<T>*> out, T scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColPass& p = axis == 1 ? g.py : g.pz;
  const cx<T>* tw = axis == 1 ? g.twy : g.twz;
  const CIdx3 c = cidx3(p);
  const int se = slab3(p);
  cx<T>* sl[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) sl[q] = sm + q * se + c.b;
  cx<T> v[NV][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = c.base + (size_t)(c.j + s * c.L8) * (size_t)p.stride;
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q][s] = in.v[q][idx];
  }
  fft_canon<S, NV>(v, sl, 1 << p.ltc, c.j, p.lL, tw);
  const bool sc = scale != (T)1;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = c.base + (size_t)(c.j + s * c.L8) * (size_t)p.stride;
#pragma unroll
    for (int q = 0; q < NV; ++q) out.v[q][idx] = sc ? cscale(v[q][s], scale) : v[q][s];
  }
}

// Forward z FFT of one field, projection of the corner modes (packed x column,
// ky in {0, ny/2}, kz in {0, nz/2}), and ||.||^2 with Parseval weights.
template <typename T>
__global__ void __launch_bounds__(256) k3_zfwd_project(Geo<T> g, const cx<T>* in, cx<T>* out,
                                                       SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColPass& p = g.pz;
  const CIdx3 c = cidx3(p);
  cx<T>* const sl[1] = {sm + c.b};
  cx<T> v[1][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) v[0][s] = in[c.base + (size_t)(c.j + s * c.L8) * (size_t)p.stride];
  fft_canon<-1, 1>(v, sl, 1 << p.ltc, c.j, p.lL, g.twz);
  const int kx = c.col & (g.H - 1), ky = c.col >> g.lH;
  const bool corner_xy = kx == 0 && (ky == 0 || ky == (g.ny >> 1));
  const double w = kx == 0 ? 1.0 : 2.0;
  double acc[1] = {0.0};
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int kz = c.j + s * c.L8;
    if (corner_xy && (kz == 0 || kz == (g.nz >> 1))) v[0][s] = czero<T>();
    out[c.base + (size_t)kz * (size_t)p.stride] = v[0][s];
    acc[0] += w * ((double)v[0][s].x * (double)v[0][s].x + (double)v[0][s].y * (double)v[0][s].y);
  }
  if (st) {
    double tot[1];
    if (last_cta_sum<1>(acc, g.partials, &st->ticket[TK_PROJ], tot) && threadIdx.x == 0)
      st->outer_b2 = tot[0];
  }
}

// ------------------------------------------------------------------ z pass: divergence
template <typename T, int MODE>
__global__ void __launch_bounds__(256) k3_zdiv(Geo<T> g, Tri<cx<T>*> Q, const cx<T>* __restrict__ d,
                                               const cx<T>* __restrict__ bvec,
                                               cx<T>* __restrict__ out, cx<float>* __restrict__ r32,
                                               cx<float>* __restrict__ delta32, SolveState* st) {
  if (MODE == CD_CG && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColPass& p = g.pz;
  const CIdx3 c = cidx3(p);
  const int se = slab3(p);
  cx<T>* const sl[3] = {sm + c.b, sm + se + c.b, sm + 2 * se + c.b};
  cx<T> v[3][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = c.base + (size_t)(c.j + s * c.L8) * (size_t)p.stride;
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q][s] = Q.v[q][idx];
  }
  fft_canon<-1, 3>(v, sl, 1 << p.ltc, c.j, p.lL, g.twz);
  const int kx = c.col & (g.H - 1), ky = c.col >> g.lH;
  const T ax = g.kxd[kx], ay = g.kyd[ky];
  const double w = kx == 0 ? 1.0 : 2.0;  // Parseval weight of a packed column
  double acc[3] = {0.0, 0.0, 0.0};
  DotAcc<T> dq, r64acc;
  DotAcc<float> r32acc, rzacc;
  Pc<T> pc{};
  Pc<float> pcf{};
  if (MODE == CD_RESID) pc = pc_of<T>(st);
  if (MODE == CD_RESID_REFINE || MODE == CD_RESID_FIRST) pcf = pc_of<float>(st);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int kz = c.j + s * c.L8;
    const size_t idx = c.base + (size_t)kz * (size_t)p.stride;
    const T az = g.kzd[kz];
    const cx<T> t = cmk<T>(ax * v[0][s].x + ay * v[1][s].x + az * v[2][s].x,
                           ax * v[0][s].y + ay * v[1][s].y + az * v[2][s].y);
    const cx<T> q = cmk<T>(t.y, -t.x);  // -i xi . Q
    if constexpr (MODE == CD_PLAIN) {
      out[idx] = q;
    } else if constexpr (MODE == CD_CG) {
      out[idx] = q;  // alpha came from the row pass (cg_alpha_from)
    } else if constexpr (MODE == CD_RESID) {
      const cx<T> rv = csub(bvec[idx], q);
      out[idx] = rv;
      const double r2 = (double)rv.x * (double)rv.x + (double)rv.y * (double)rv.y;
      acc[0] += w * r2;
      acc[1] += w * r2 * (double)pinv3(g, kx, ky, kz, pc);
    } else if constexpr (MODE == CD_RESID_FIRST) {
      const cx<float> rf = ccast<float>(csub(bvec[idx], q));
      r32[idx] = rf;
      delta32[idx] = czero<float>();
      const float wf = (float)w, wpf = wf * pinv3_f32(g, kx, ky, kz, pcf);
      r32acc.add_prod(wf * rf.x, rf.x);
      r32acc.add_prod(wf * rf.y, rf.y);
      rzacc.add_prod(wpf * rf.x, rf.x);
      rzacc.add_prod(wpf * rf.y, rf.y);
    } else {
      const cx<T> rv = csub(bvec[idx], q);
      if (out) out[idx] = rv;
      const T wt = (T)(float)w;
      r64acc.add_prod(wt * rv.x, rv.x);
      r64acc.add_prod(wt * rv.y, rv.y);
      const cx<float> rf = ccast<float>(rv);
      r32[idx] = rf;
      delta32[idx] = czero<float>();
      const float wf = (float)w, wpf = wf * pinv3_f32(g, kx, ky, kz, pcf);
      r32acc.add_prod(wf * rf.x, rf.x);
      r32acc.add_prod(wf * rf.y, rf.y);
      rzacc.add_prod(wpf * rf.x, rf.x);
      rzacc.add_prod(wpf * rf.y, rf.y);
    }
  }
  if constexpr (MODE == CD_PLAIN || MODE == CD_CG) return;
  double tot[3];
  if constexpr (MODE == CD_RESID) {
    double a2[2] = {acc[0], acc[1]}, t2[2];
    if (last_cta_sum<2>(a2, g.partials, &st->ticket[TK_RESID], t2) && threadIdx.x == 0)
      resid_init(st, t2[0], t2[1]);
  } else if constexpr (MODE == CD_RESID_FIRST) {
    double a2[2] = {r32acc.value(), rzacc.value()}, t2[2];
    if (last_cta_sum<2>(a2, g.partials, &st->ticket[TK_RESID], t2) && threadIdx.x == 0)
      resid_first_init(st, t2[0], t2[1]);
  } else {
    acc[0] = r64acc.value();
    acc[1] = r32acc.value();
    acc[2] = rzacc.value();
    if (last_cta_sum<3>(acc, g.partials, &st->ticket[TK_RESID], tot) && threadIdx.x == 0)
      resid_sweep_init(st, tot[0], tot[1], tot[2]);
  }
}

// ------------------------------------------------------------------ row pairs
// DOT: the CG variant, alpha = rho / (n sum g . K g) as in the 2D row pass.
template <typename T, typename Tm, bool DOT>
__global__ void __launch_bounds__(256) k3_row_apply(Geo<T> g, Tri<cx<T>*> G, Tri<const Tm*> m,
                                                    const Tm* __restrict__ rr, Tri<cx<T>*> Q,
                                                    SolveState* st) {
  if (st && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const RIdx3 r = ridx3(g);
  const int N = g.nx, H = g.H;
  cx<T>* const sl[3] = {sm + (3 * r.u) * N, sm + (3 * r.u + 1) * N, sm + (3 * r.u + 2) * N};
  cx<T> v[3][8];
  load_rows3(v, G, r, H);
  fft_canon<+1, 3, true>(v, sl, 1, r.j, g.lnx, g.twx);
  const size_t o0 = r.y0 * N, o1 = r.y1 * N;
  DotAcc<T> gkg;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = r.j + s * r.N8;
    {
      const T gx = v[0][s].x, gy = v[0][s].y, gz = v[2][s].x;
      const T ax = (T)m.v[0][o0 + x], ay = (T)m.v[1][o0 + x], az = (T)m.v[2][o0 + x];
      const T rv = (T)rr[o0 + x];
      const T mg = ax * gx + ay * gy + az * gz;
      if (DOT) gkg.add_prod(mg * mg + rv * (gx * gx + gy * gy + gz * gz), (T)1);
      v[0][s] = cmk<T>(ax * mg + rv * gx, ay * mg + rv * gy);
      v[2][s].x = az * mg + rv * gz;
    }
    {
      const T gx = v[1][s].x, gy = v[1][s].y, gz = v[2][s].y;
      const T ax = (T)m.v[0][o1 + x], ay = (T)m.v[1][o1 + x], az = (T)m.v[2][o1 + x];
      const T rv = (T)rr[o1 + x];
      const T mg = ax * gx + ay * gy + az * gz;
      if (DOT) gkg.add_prod(mg * mg + rv * (gx * gx + gy * gy + gz * gz), (T)1);
      v[1][s] = cmk<T>(ax * mg + rv * gx, ay * mg + rv * gy);
      v[2][s].y = az * mg + rv * gz;
    }
  }
  fft_canon<-1, 3, true>(v, sl, 1, r.j, g.lnx, g.twx);
  const size_t s0 = r.y0 * H, s1 = r.y1 * H;
  const Tri<cx<T>*> A = {{Q.v[0] + s0, Q.v[0] + s1, Q.v[2] + s0}};
  const Tri<cx<T>*> B = {{Q.v[1] + s0, Q.v[1] + s1, Q.v[2] + s1}};
  store_pairs_r2c<3>(v, sl, r.j, N, H, A, B);
  if (DOT) {
    double a1[1] = {gkg.value()}, t1[1];
    if (last_cta_sum<1>(a1, g.partials, &st->ticket[TK_DIV], t1) && threadIdx.x == 0)
      cg_alpha_from(st, t1[0], (double)g.nx * (double)g.ny * (double)g.nz);
  }
}

// Activation (rank-one phi1 form of eq. m_activation_discrete) and relaxation
// (eq. m_relaxation_discrete) of one 3-vector.
template <typename T>
__device__ __forceinline__ void act_relax3(T& ax, T& ay, T& az, T gx, T gy, T gz,
                                           const SplitCoef& cf) {
  const T c2dt = cfv<T>(cf.c2dt, cf.f_c2dt);
  const T mg = ax * gx + ay * gy + az * gz;
  if (mg != (T)0) {
    const T z = c2dt * (gx * gx + gy * gy + gz * gz);
    const T coef = z > (T)0 ? c2dt * (hc_expm1(z) / z) : c2dt;
    const T t = coef * mg;
    ax += t * gx;
    ay += t * gy;
    az += t * gz;
  }
  if (cf.gamma_is_one) {
    ax *= cfv<T>(cf.exp_mdt, cf.f_exp_mdt);
    ay *= cfv<T>(cf.exp_mdt, cf.f_exp_mdt);
    az *= cfv<T>(cf.exp_mdt, cf.f_exp_mdt);
  } else {
    const T n2 = ax * ax + ay * ay + az * az;
    if (n2 > (T)0) {
      const T sc = relax_factor(hc_sqrt(n2), cf);
      ax *= sc;
      ay *= sc;
      az *= sc;
    }
  }
}

// mo may alias the rows of G: every unit reads its two rows of G into
// registers before it writes the same rows of mo.
template <typename T>
__global__ void __launch_bounds__(256) k3_row_split(Geo<T> g, Tri<cx<T>*> G, Tri<const T*> m,
                                                    const T* __restrict__ rr, Tri<T*> mo,
                                                    SplitCoef cf, SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const RIdx3 r = ridx3(g);
  const int N = g.nx, H = g.H;
  cx<T>* const sl[3] = {sm + (3 * r.u) * N, sm + (3 * r.u + 1) * N, sm + (3 * r.u + 2) * N};
  cx<T> v[3][8];
  load_rows3(v, G, r, H);
  fft_canon<+1, 3, true>(v, sl, 1, r.j, g.lnx, g.twx);
  const size_t o0 = r.y0 * N, o1 = r.y1 * N;
  bool finite = true;
  const bool diag = st->diag != 0;
  EnergyAcc<T> en;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = r.j + s * r.N8;
    T ax = m.v[0][o0 + x], ay = m.v[1][o0 + x], az = m.v[2][o0 + x];
    T bx = m.v[0][o1 + x], by = m.v[1][o1 + x], bz = m.v[2][o1 + x];
    if (diag) {
      const T g0x = v[0][s].x, g0y = v[0][s].y, g0z = v[2][s].x;
      const T g1x = v[1][s].x, g1y = v[1][s].y, g1z = v[2][s].y;
      en.add(rr[o0 + x], g0x * g0x + g0y * g0y + g0z * g0z, ax * g0x + ay * g0y + az * g0z,
             ax * ax + ay * ay + az * az, cfv<T>(cf.gamma, cf.f_gamma));
      en.add(rr[o1 + x], g1x * g1x + g1y * g1y + g1z * g1z, bx * g1x + by * g1y + bz * g1z,
             bx * bx + by * by + bz * bz, cfv<T>(cf.gamma, cf.f_gamma));
    }
    act_relax3(ax, ay, az, v[0][s].x, v[0][s].y, v[2][s].x, cf);
    act_relax3(bx, by, bz, v[1][s].x, v[1][s].y, v[2][s].y, cf);
    finite = finite && hc_finite(ax) && hc_finite(ay) && hc_finite(az) && hc_finite(bx) &&
             hc_finite(by) && hc_finite(bz);
    v[0][s] = cmk<T>(ax, ay);
    v[1][s] = cmk<T>(bx, by);
    v[2][s] = cmk<T>(az, bz);
  }
  if (!finite) st->nonfinite = 1;
  if (diag) en.finish(g.partials, st);
  // diffusion along x: a real, even multiplier on complex rows
  fft_canon<-1, 3, true>(v, sl, 1, r.j, g.lnx, g.twx);
  const T invN = exp2_neg<T>(g.lnx);  // 1 / N, N = nx
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int k = r.j + s * r.N8;
    const T h = g.hx[k <= H ? k : N - k] * invN;
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q][s] = cscale(v[q][s], h);
  }
  fft_canon<+1, 3, true>(v, sl, 1, r.j, g.lnx, g.twx);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = r.j + s * r.N8;
    mo.v[0][o0 + x] = v[0][s].x;
    mo.v[1][o0 + x] = v[0][s].y;
    mo.v[2][o0 + x] = v[2][s].x;
    mo.v[0][o1 + x] = v[1][s].x;
    mo.v[1][o1 + x] = v[1][s].y;
    mo.v[2][o1 + x] = v[2][s].y;
  }
}

// ------------------------------------------------------------------ heat along y or z
template <typename T>
__global__ void __launch_bounds__(256) k3_heat(Geo<T> g, int axis, Tri<cx<T>*> M, Tri<cx<T>*> Mo,
                                               SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColPass& p = axis == 1 ? g.py : g.pz;
  const cx<T>* tw = axis == 1 ? g.twy : g.twz;
  const T* h = axis == 1 ? g.hy : g.hz;
  const CIdx3 c = cidx3(p);
  const int se = slab3(p);
  cx<T>* const sl[3] = {sm + c.b, sm + se + c.b, sm + 2 * se + c.b};
  cx<T> v[3][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = c.base + (size_t)(c.j + s * c.L8) * (size_t)p.stride;
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q][s] = M.v[q][idx];
  }
  fft_canon<-1, 3>(v, sl, 1 << p.ltc, c.j, p.lL, tw);
  const T invL = exp2_neg<T>(p.lL);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const T f = h[c.j + s * c.L8] * invL;
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q][s] = cscale(v[q][s], f);
  }
  fft_canon<+1, 3>(v, sl, 1 << p.ltc, c.j, p.lL, tw);
  DotAcc<T> mm[6], d2;  // sum m_a m_b: xx, yy, zz, xy, xz, yz
  bool finite = true;
  const bool dm = axis == 2 && st->diag;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = c.base + (size_t)(c.j + s * c.L8) * (size_t)p.stride;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      if (dm) {  // Mo still holds m^k here: this thread overwrites exactly what it reads
        const cx<T> o = Mo.v[q][idx];
        const T dx = v[q][s].x - o.x, dy = v[q][s].y - o.y;
        d2.add_prod(dx, dx);
        d2.add_prod(dy, dy);
      }
      Mo.v[q][idx] = v[q][s];
      if (axis == 2) finite = finite && hc_finite(v[q][s].x) && hc_finite(v[q][s].y);
    }
    if (axis == 2) {  // the three components of the same two points
      constexpr int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        mm[e].add_prod(v[pa[e]][s].x, v[pb[e]][s].x);
        mm[e].add_prod(v[pa[e]][s].y, v[pb[e]][s].y);
      }
    }
  }
  if (axis == 2) {
    if (!finite) st->nonfinite = 1;
    double acc[7], tot[7];
#pragma unroll
    for (int e = 0; e < 6; ++e) acc[e] = mm[e].value();
    acc[6] = d2.value();
    if (last_cta_sum<7>(acc, g.partials, &st->ticket[TK_MSUM], tot) && threadIdx.x == 0) {
      set_mm3(st, tot);
      if (dm) st->dm2 = tot[6];
    }
  }
}

// sum |grad m|^2 from the spectrum of m after the x and y passes: forward FFT
// along z of three fields, sum w |xi~|^2 |F|^2 / n (no store).
template <typename T>
__global__ void __launch_bounds__(256) k3_zgradnorm(Geo<T> g, Tri<cx<T>*> Q, SolveState* st,
                                                    int into_next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColPass& p = g.pz;
  const CIdx3 c = cidx3(p);
  const int se = slab3(p);
  cx<T>* const sl[3] = {sm + c.b, sm + se + c.b, sm + 2 * se + c.b};
  cx<T> v[3][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = c.base + (size_t)(c.j + s * c.L8) * (size_t)p.stride;
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q][s] = Q.v[q][idx];
  }
  fft_canon<-1, 3>(v, sl, 1 << p.ltc, c.j, p.lL, g.twz);
  const int kx = c.col & (g.H - 1), ky = c.col >> g.lH;
  const T a = g.kxd[kx], b = g.kyd[ky];
  const T wxy = a * a + b * b, w = kx == 0 ? (T)1 : (T)2;
  DotAcc<T> ga;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const T cz = g.kzd[c.j + s * c.L8];
    const T wk = w * (wxy + cz * cz);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      ga.add_prod(wk * v[q][s].x, v[q][s].x);
      ga.add_prod(wk * v[q][s].y, v[q][s].y);
    }
  }
  gradnorm_finish(ga.value(), 1.0 / ((double)g.nx * (double)g.ny * (double)g.nz), g.partials, st,
                  into_next);
}

// ------------------------------------------------------------------ CG update, |m|^2
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k3_cg_update(Geo<T> g, cx<T>* __restrict__ x,
                                                    cx<T>* __restrict__ r,
                                                    const cx<T>* __restrict__ d,
                                                    const cx<T>* __restrict__ q, SolveState* st) {
  if (st->done) {
    if (st->graph_mode && blockIdx.x == 0 && threadIdx.x == 0)
      cudaGraphSetConditional(st->h_cur, 0u);
    return;
  }
  const T alpha = st_alpha<T>(st);
  const Pc<T> pc = pc_of<T>(st);
  const size_t total = (size_t)g.nz * g.ny * g.H;
  DotAcc<T> rr, rz;
  auto upd = [&](size_t i, cx<T> dv, cx<T> xv, cx<T> qv, cx<T> rv) {
    const int kx = (int)(i & (size_t)(g.H - 1));
    const int ky = (int)((i >> g.lH) & (size_t)(g.ny - 1));
    const int kz = (int)(i >> (g.lH + g.lny));
    x[i] = cmk<T>(xv.x + alpha * dv.x, xv.y + alpha * dv.y);
    rv = cmk<T>(rv.x - alpha * qv.x, rv.y - alpha * qv.y);
    r[i] = rv;
    const T wt = kx == 0 ? (T)1 : (T)2;
    const T wp = wt * pinv3(g, kx, ky, kz, pc);
    rr.add_prod(wt * rv.x, rv.x);
    rr.add_prod(wt * rv.y, rv.y);
    rz.add_prod(wp * rv.x, rv.x);
    rz.add_prod(wp * rv.y, rv.y);
  };
  constexpr int U = 4;  // four elements per trip, all loads issued first
  const size_t S = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + (U - 1) * S < total; i += U * S) {
    cx<T> dv[U], xv[U], qv[U], rv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      dv[u] = d[i + u * S];
      xv[u] = x[i + u * S];
      qv[u] = q[i + u * S];
      rv[u] = r[i + u * S];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) upd(i + u * S, dv[u], xv[u], qv[u], rv[u]);
  }
  for (; i < total; i += S) upd(i, d[i], x[i], q[i], r[i]);
  double acc[2] = {rr.value(), rz.value()};
  double tot[2];
  if (last_cta_sum<2>(acc, g.partials, &st->ticket[TK_UPDATE], tot) && threadIdx.x == 0) {
    const double rho_new = tot[1];
    st->rnorm2 = tot[0];
    st->beta = st->rho > 0 ? rho_new / st->rho : 0.0;
    st->beta_f = (float)st->beta;
    st->rho = rho_new;
    st->it += 1;
    st->total_it += 1;
    if (!isfinite(tot[0])) {
      st->status = HC_ENONFINITE;
      st->done = 1;
    } else if (tot[0] <= st->thresh2) {
      st->done = 1;
    } else if (st->it >= st->maxit) {
      st->done = 1;
      st->status = HC_ENOCONV;
    }
    if (st->graph_mode) cudaGraphSetConditional(st->h_cur, st->done ? 0u : 1u);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k3_msum(Geo<T> g, Tri<const T*> m, SolveState* st) {
  const size_t n = (size_t)g.nx * g.ny * g.nz;
  constexpr int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
  DotAcc<T> mm[6];
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const T v[3] = {m.v[0][i], m.v[1][i], m.v[2][i]};
#pragma unroll
    for (int e = 0; e < 6; ++e) mm[e].add_prod(v[pa[e]], v[pb[e]]);
  }
  double acc[6], tot[6];
#pragma unroll
  for (int e = 0; e < 6; ++e) acc[e] = mm[e].value();
  if (last_cta_sum<6>(acc, g.partials, &st->ticket[TK_MSUM], tot) && threadIdx.x == 0)
    set_mm3(st, tot);
}

// ------------------------------------------------------------------ launchers
__host__ __forceinline__ int pass_ctas(const ColPass& p) { return p.nplanes << p.lt; }
__host__ __forceinline__ int pass_threads(const ColPass& p) { return (1 << p.ltc) << (p.lL - 3); }
template <typename T>
__host__ __forceinline__ size_t pass_smem(const ColPass& p, int nv) {
  return (size_t)nv * ((size_t)(9 << (p.lL - 3)) << p.ltc) * sizeof(cx<T>);
}
template <typename T>
__host__ __forceinline__ int row3_ctas(const Geo<T>& g) {
  return (int)((((size_t)g.ny * g.nz) >> 1) >> g.lupc);
}
template <typename T>
__host__ __forceinline__ int row3_threads(const Geo<T>& g) { return g.upc << (g.lnx - 3); }
template <typename T>
__host__ __forceinline__ size_t row3_smem(const Geo<T>& g) {
  return (size_t)3 * g.upc * g.nx * sizeof(cx<T>);
}

template <typename T, typename Tin>
void z_grad(const Geo<T>& g, int mode, cx<Tin>* in, const cx<T>* rvec, cx<T>* dio,
            const cx<float>* delta, Tri<cx<T>*> G, SolveState* st, int check_done,
            cudaStream_t s) {
  const int nb = pass_ctas(g.pz), nt = pass_threads(g.pz);
  const size_t sm = pass_smem<T>(g.pz, 3);
  if (mode == CG_PLAIN)
    k3_zgrad<T, Tin, CG_PLAIN><<<nb, nt, sm, s>>>(g, in, rvec, dio, delta, G, st, check_done);
  else if (mode == CG_DUPDATE)
    k3_zgrad<T, Tin, CG_DUPDATE><<<nb, nt, sm, s>>>(g, in, rvec, dio, delta, G, st, check_done);
  else
    k3_zgrad<T, Tin, CG_ADDDELTA><<<nb, nt, sm, s>>>(g, in, rvec, dio, delta, G, st, check_done);
}
template <typename T>
void axis_fft(const Geo<T>& g, int axis, int sign, int nv, Tri<cx<T>*> in, Tri<cx<T>*> out,
              T scale, cudaStream_t s) {
  const ColPass& p = axis == 1 ? g.py : g.pz;
  const int nb = pass_ctas(p), nt = pass_threads(p);
  const size_t sm = pass_smem<T>(p, nv);
  if (sign < 0) {
    if (nv == 1) k3_axis_fft<T, -1, 1><<<nb, nt, sm, s>>>(g, axis, in, out, scale);
    else k3_axis_fft<T, -1, 3><<<nb, nt, sm, s>>>(g, axis, in, out, scale);
  } else {
    if (nv == 1) k3_axis_fft<T, +1, 1><<<nb, nt, sm, s>>>(g, axis, in, out, scale);
    else k3_axis_fft<T, +1, 3><<<nb, nt, sm, s>>>(g, axis, in, out, scale);
  }
}
template <typename T>
void z_fwd_project(const Geo<T>& g, const cx<T>* in, cx<T>* out, SolveState* st, cudaStream_t s) {
  k3_zfwd_project<T><<<pass_ctas(g.pz), pass_threads(g.pz), pass_smem<T>(g.pz, 1), s>>>(g, in, out,
                                                                                        st);
}
template <typename T>
void z_div(const Geo<T>& g, int mode, Tri<cx<T>*> Q, const cx<T>* d, const cx<T>* b, cx<T>* out,
           cx<float>* r32, cx<float>* delta32, SolveState* st, cudaStream_t s) {
  const int nb = pass_ctas(g.pz), nt = pass_threads(g.pz);
  const size_t sm = pass_smem<T>(g.pz, 3);
  switch (mode) {
    case CD_PLAIN:
      k3_zdiv<T, CD_PLAIN><<<nb, nt, sm, s>>>(g, Q, d, b, out, r32, delta32, st);
      break;
    case CD_CG:
      k3_zdiv<T, CD_CG><<<nb, nt, sm, s>>>(g, Q, d, b, out, r32, delta32, st);
      break;
    case CD_RESID:
      k3_zdiv<T, CD_RESID><<<nb, nt, sm, s>>>(g, Q, d, b, out, r32, delta32, st);
      break;
    case CD_RESID_FIRST:
      if constexpr (std::is_same<T, float>::value)
        k3_zdiv<T, CD_RESID_FIRST><<<nb, nt, sm, s>>>(g, Q, d, b, out, r32, delta32, st);
      break;
    default:
      k3_zdiv<T, CD_RESID_REFINE><<<nb, nt, sm, s>>>(g, Q, d, b, out, r32, delta32, st);
      break;
  }
}
template <typename T, typename Tm>
void row_apply3(const Geo<T>& g, Tri<cx<T>*> G, Tri<const Tm*> m, const Tm* r, Tri<cx<T>*> Q,
                SolveState* st, cudaStream_t s) {
  if (st)
    k3_row_apply<T, Tm, true><<<row3_ctas(g), row3_threads(g), row3_smem(g), s>>>(g, G, m, r, Q, st);
  else
    k3_row_apply<T, Tm, false><<<row3_ctas(g), row3_threads(g), row3_smem(g), s>>>(g, G, m, r, Q, st);
}
template <typename T>
void row_split3(const Geo<T>& g, Tri<cx<T>*> G, Tri<const T*> m, const T* r, Tri<T*> mo,
                SplitCoef cf, SolveState* st, cudaStream_t s) {
  k3_row_split<T><<<row3_ctas(g), row3_threads(g), row3_smem(g), s>>>(g, G, m, r, mo, cf, st);
}
template <typename T>
void heat_axis(const Geo<T>& g, int axis, Tri<T*> mi, Tri<T*> mo, SolveState* st, cudaStream_t s) {
  const ColPass& p = axis == 1 ? g.py : g.pz;
  Tri<cx<T>*> Mi = {{reinterpret_cast<cx<T>*>(mi.v[0]), reinterpret_cast<cx<T>*>(mi.v[1]),
                     reinterpret_cast<cx<T>*>(mi.v[2])}};
  Tri<cx<T>*> Mo = {{reinterpret_cast<cx<T>*>(mo.v[0]), reinterpret_cast<cx<T>*>(mo.v[1]),
                     reinterpret_cast<cx<T>*>(mo.v[2])}};
  k3_heat<T><<<pass_ctas(p), pass_threads(p), pass_smem<T>(p, 3), s>>>(g, axis, Mi, Mo, st);
}
template <typename T>
void z_gradnorm(const Geo<T>& g, Tri<cx<T>*> G, SolveState* st, int into_next, cudaStream_t s) {
  k3_zgradnorm<T><<<pass_ctas(g.pz), pass_threads(g.pz), pass_smem<T>(g.pz, 3), s>>>(g, G, st,
                                                                                     into_next);
}
template <typename T>
void cg_update3(const Geo<T>& g, cx<T>* x, cx<T>* r, const cx<T>* d, const cx<T>* q,
                SolveState* st, cudaStream_t s) {
  k3_cg_update<T><<<upd_blocks((size_t)g.nz * g.ny * g.H), 256, 0, s>>>(g, x, r, d, q, st);
}
template <typename T>
void msum3(const Geo<T>& g, Tri<const T*> m, SolveState* st, cudaStream_t s) {
  k3_msum<T><<<upd_blocks((size_t)g.nx * g.ny * g.nz), 256, 0, s>>>(g, m, st);
}

template <typename T>
void set_smem_limits_3d_t() {
  allow_smem(k3_row_split<T>);
  allow_smem(k3_heat<T>);
  allow_smem(k3_zgradnorm<T>);
  allow_smem(k3_axis_fft<T, -1, 1>);
  allow_smem(k3_axis_fft<T, -1, 3>);
  allow_smem(k3_axis_fft<T, +1, 1>);
  allow_smem(k3_axis_fft<T, +1, 3>);
  allow_smem(k3_zfwd_project<T>);
  allow_smem(k3_zdiv<T, CD_PLAIN>);
  allow_smem(k3_zdiv<T, CD_CG>);
  allow_smem(k3_zdiv<T, CD_RESID>);
  allow_smem(k3_zdiv<T, CD_RESID_REFINE>);
  if constexpr (std::is_same<T, float>::value) allow_smem(k3_zdiv<T, CD_RESID_FIRST>);
}
template <typename T, typename Tm>
void set_smem_limits_row3() {
  allow_smem(k3_row_apply<T, Tm, false>);
  allow_smem(k3_row_apply<T, Tm, true>);
}
template <typename T, typename Tin>
void set_smem_limits_zgrad() {
  allow_smem(k3_zgrad<T, Tin, CG_PLAIN>);
  allow_smem(k3_zgrad<T, Tin, CG_DUPDATE>);
  allow_smem(k3_zgrad<T, Tin, CG_ADDDELTA>);
}

}  // namespace hc
