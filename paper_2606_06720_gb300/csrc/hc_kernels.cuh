// hc_kernels.cuh -- sm_103a kernels of one time step of the Fourier spectral
// scheme for the periodic Hu-Cai system (arXiv 2606.06720, Section 2).
//
// A 2D transform is split into a row pass (length nx along the contiguous x
// axis, one complex FFT per row carrying two real fields as re/im) and a column
// pass (length ny along y over tiles of TC packed columns).  The passes carry
// the scheme's pointwise work as fused prologues/epilogues:
//   column pass "grad": multiply by i xi / n (eq. p_discrete, inner bracket)
//   row pass "apply":   q = (m.g) m + r g  (eq. 1.1a tensor)
//   column pass "div":  -i xi . q^        (eq. p_discrete, outer bracket)
//   row pass "split":   activation + relaxation (eqs. m_activation_discrete,
//                        m_relaxation_discrete)
//   column pass "heat": exp(-D^2 |xi|^2 dt) (eq. diffusion_space_discrete)
//
// FFT: Stockham autosort, radix-8 passes (radix 4 or 2 for the last pass),
// every thread holding 8 elements per transform.  Data arrive from and leave
// for global memory in registers in the "canonical" order: thread j holds
// elements j + s*N/8, s = 0..7, which is both the input order of the first pass
// and the output order of the last one, so transforms chain through registers
// and only the inner passes touch shared memory.  Shared-memory slabs insert
// one pad element per 8 to break the stride-8 bank conflicts.
#pragma once

#include <type_traits>

#include "hc_internal.cuh"
#include "hc.h"

namespace hc {

// ------------------------------------------------------------------ complex
template <typename T>
__device__ __forceinline__ cx<T> cmk(T a, T b) {
  cx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return cmk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return cmk<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return cmk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return cmk<T>(a.x * s, a.y * s); }
// a * (S i), S = +-1
template <int S, typename T>
__device__ __forceinline__ cx<T> cmul_si(cx<T> a) {
  return S > 0 ? cmk<T>(-a.y, a.x) : cmk<T>(a.y, -a.x);
}
template <typename T>
__device__ __forceinline__ cx<T> czero() { return cmk<T>((T)0, (T)0); }

template <typename To, typename Ti>
__device__ __forceinline__ cx<To> ccast(cx<Ti> a) { return cmk<To>((To)a.x, (To)a.y); }

// Read-only-path load of a complex table entry.
__device__ __forceinline__ cx<float> ldg(const cx<float>* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return cmk<float>(v.x, v.y);
}
__device__ __forceinline__ cx<double> ldg(const cx<double>* p) {
  const double2 v = __ldg(reinterpret_cast<const double2*>(p));
  return cmk<double>(v.x, v.y);
}
__device__ __forceinline__ cx<df64> ldg(const cx<df64>* p) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  return cmk<df64>(df64(v.x, v.y), df64(v.z, v.w));
}
__device__ __forceinline__ bool hc_finite(df64 x) { return isfinite(x.hi); }

__device__ __forceinline__ float hc_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double hc_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float hc_pow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double hc_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float hc_log(float x) { return logf(x); }
__device__ __forceinline__ double hc_log(double x) { return log(x); }
__device__ __forceinline__ float hc_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double hc_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float hc_exp(float x) { return expf(x); }
__device__ __forceinline__ double hc_exp(double x) { return exp(x); }
__device__ __forceinline__ float hc_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double hc_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ bool hc_finite(float x) { return isfinite(x); }
__device__ __forceinline__ bool hc_finite(double x) { return isfinite(x); }

// ------------------------------------------------------------------ small DFTs
// Kernel exp(S 2 pi i n k / R); S = -1 forward, +1 inverse.
template <int S, typename T>
__device__ __forceinline__ void dft2(cx<T>& a, cx<T>& b) {
  cx<T> t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <int S, typename T>
__device__ __forceinline__ void dft4(cx<T>& a0, cx<T>& a1, cx<T>& a2, cx<T>& a3) {
  cx<T> t0 = cadd(a0, a2), t1 = csub(a0, a2), t2 = cadd(a1, a3);
  cx<T> t3 = cmul_si<S>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <int S, typename T>
__device__ __forceinline__ void dft8(cx<T>* v) {
  cx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  cx<T> o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<S>(e0, e1, e2, e3);
  dft4<S>(o0, o1, o2, o3);
  const T h = (T)0.70710678118654752440;  // cos(pi/4)
  // W8 = (1 + S i)/sqrt(2); W8^2 = S i; W8^3 = (-1 + S i)/sqrt(2)
  if constexpr (S < 0) {
    o1 = cmk<T>((o1.x + o1.y) * h, (o1.y - o1.x) * h);
    o3 = cmk<T>((o3.y - o3.x) * h, -((o3.x + o3.y) * h));
  } else {
    o1 = cmk<T>((o1.x - o1.y) * h, (o1.y + o1.x) * h);
    o3 = cmk<T>(-((o3.x + o3.y) * h), (o3.x - o3.y) * h);
  }
  o2 = cmul_si<S>(o2);
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, o1);
  v[5] = csub(e1, o1);
  v[2] = cadd(e2, o2);
  v[6] = csub(e2, o2);
  v[3] = cadd(e3, o3);
  v[7] = csub(e3, o3);
}

__device__ __forceinline__ int padk(int e) { return e + (e >> 3); }

// Row slabs (one transform per slab, stride 1) use an XOR swizzle inside
// aligned blocks instead of padding.  Shared memory serves a warp's 8-byte
// accesses in 16-lane phases and 16-byte accesses in 8-lane phases; the
// swizzles below make every Stockham access pattern of a radix-8 pass
// (writes to 8j + r, 64(j/8) + j%8 + 8r, ...; canonical reads j + sN/8)
// touch distinct banks within a phase, and they need no extra space.
template <typename T>
__device__ __forceinline__ int rswz(int e);
template <>
__device__ __forceinline__ int rswz<float>(int e) {
  const int k = e >> 4;
  return e ^ ((k & 7) | ((k & 4) << 1));
}
template <>
__device__ __forceinline__ int rswz<double>(int e) {
  return e ^ ((e >> 3) & 7);
}
template <>
__device__ __forceinline__ int rswz<df64>(int e) {
  return e ^ ((e >> 3) & 7);
}
// Slot of element e: swizzled row slab (SWZ) or padded column slab with stride ks.
template <typename T, bool SWZ>
__device__ __forceinline__ int slot(int e, int ks) {
  return SWZ ? rswz<T>(e) : padk(e) * ks;
}

// ------------------------------------------------------------------ FFT core
// Twiddles w^r = exp(S 2 pi i r k / (R Ns)), r = 1..R-1, of one butterfly.  FP32:
// one table load and the powers by complex products (w^2 = w w, w^3 = w^2 w,
// w^4 = w^2 w^2, ...; a few ulp, far below the FP32 transform's own error),
// which replaces R-2 dependent L1 round trips per pass with FMAs.  FP64 and
// double-float kernels are bound by their arithmetic and load every power.
template <int S, int R, typename T>
__device__ __forceinline__ void twiddle_powers(cx<T> (&w)[R], const cx<T>* __restrict__ tw,
                                               int step) {
  if constexpr (std::is_same<T, float>::value) {
    w[1] = ldg(&tw[step]);
    if (S > 0) w[1].y = -w[1].y;
#pragma unroll
    for (int r = 2; r < R; ++r) w[r] = (r & 1) ? cmul(w[r - 1], w[1]) : cmul(w[r >> 1], w[r >> 1]);
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) {
      w[r] = ldg(&tw[r * step]);
      if (S > 0) w[r].y = -w[r].y;
    }
  }
}

// NV transforms of length N = 2^lN (lN >= 3), one per slab, computed by the
// N/8 threads j = 0..N/8-1 of each transform.  v[q][s] holds element
// j + s N/8 on entry (input) and on exit (output).  Element e of slab q lives
// at sl[q][padk(e) * ks].  Every thread of the CTA must call this together.
// tw[m] = exp(-2 pi i m / N); the inverse uses the conjugates.
template <int S, int NV, bool SWZ = false, typename T>
__device__ __forceinline__ void fft_rt(cx<T> (&v)[NV][8], cx<T>* const* sl, int ks, int j, int lN,
                                       const cx<T>* __restrict__ tw) {
  const int N8 = 1 << (lN - 3);
  int lNs = 0;
  int rem = lN;
#pragma unroll 1
  while (true) {
    if (rem >= 3) {
      const int k = j & ((1 << lNs) - 1);
      if (lNs > 0) {
        cx<T> w[8];
        twiddle_powers<S, 8>(w, tw, k << (lN - 3 - lNs));  // step k * N / (8 Ns)
#pragma unroll
        for (int r = 1; r < 8; ++r)
#pragma unroll
          for (int q = 0; q < NV; ++q) v[q][r] = cmul(v[q][r], w[r]);
      }
#pragma unroll
      for (int q = 0; q < NV; ++q) dft8<S>(v[q]);
      if (rem == 3) return;  // last pass: output index j + r N/8 = slot r
      const int base = ((j >> lNs) << (lNs + 3)) + k;  // Stockham expand(j, Ns, 8)
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int e = base + (r << lNs);
#pragma unroll
        for (int q = 0; q < NV; ++q) sl[q][slot<T, SWZ>(e, ks)] = v[q][r];
      }
      __syncthreads();
      lNs += 3;
      rem -= 3;
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int e = j + s * N8;
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q][s] = sl[q][slot<T, SWZ>(e, ks)];
      }
    } else if (rem == 2) {
      // last pass, radix 4: butterflies jj = j + u N/8 (u = 0, 1) read/write
      // elements jj + r N/4 = slot u + 2 r
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int jj = j + u * N8;
        const int k = jj & ((1 << lNs) - 1);
        cx<T> w[4];
        twiddle_powers<S, 4>(w, tw, k << (lN - 2 - lNs));
#pragma unroll
        for (int r = 1; r < 4; ++r)
#pragma unroll
          for (int q = 0; q < NV; ++q) v[q][u + 2 * r] = cmul(v[q][u + 2 * r], w[r]);
#pragma unroll
        for (int q = 0; q < NV; ++q) dft4<S>(v[q][u], v[q][u + 2], v[q][u + 4], v[q][u + 6]);
      }
      return;
    } else {
      // last pass, radix 2: butterflies jj = j + u N/8 (u = 0..3), slots u, u + 4
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int jj = j + u * N8;
        const int k = jj & ((1 << lNs) - 1);
        cx<T> w = ldg(&tw[k << (lN - 1 - lNs)]);
        if (S > 0) w.y = -w.y;
#pragma unroll
        for (int q = 0; q < NV; ++q) {
          v[q][u + 4] = cmul(v[q][u + 4], w);
          dft2<S>(v[q][u], v[q][u + 4]);
        }
      }
      return;
    }
  }
}

// Compile-time-length variant of fft_rt, same contract.  With the pass
// stride a constant, every slot address is one per-thread base plus a
// constant: a pass writes elements base + (r << LNS) and reads j + s N/8,
// whose two parts occupy disjoint bits, and both the swizzle (bitwise linear:
// rswz(a ^ b) = rswz(a) ^ rswz(b)) and the padding (padk(a + b) = padk(a) +
// padk(b) when b is a multiple of 8 or a < 8 with a's base a multiple of 8)
// split over them.  That removes the per-access index arithmetic.
template <typename T>
__host__ __device__ constexpr int rswz_c(int e) {
  return std::is_same<T, float>::value ? (e ^ (((e >> 4) & 7) | (((e >> 4) & 4) << 1)))
                                       : (e ^ ((e >> 3) & 7));
}
template <typename T, bool SWZ>
__device__ __forceinline__ int slot_base(int e, int ks) {
  return SWZ ? rswz<T>(e) : padk(e) * ks;
}
template <typename T, bool SWZ>
__device__ __forceinline__ int slot_plus(int b, int c, int ks) {  // slot of (base of b) + c
  return SWZ ? (b ^ rswz_c<T>(c)) : b + (c + (c >> 3)) * ks;
}

template <int S, int NV, bool SWZ, int LN, int LNS, typename T>
__device__ __forceinline__ void fft_static_pass(cx<T> (&v)[NV][8], cx<T>* const* sl, int ks, int j,
                                                int jslot, const cx<T>* __restrict__ tw) {
  constexpr int REM = LN - LNS;
  constexpr int N8 = 1 << (LN - 3);
  if constexpr (REM >= 3) {
    const int k = j & ((1 << LNS) - 1);
    if constexpr (LNS > 0) {
      cx<T> w[8];
      twiddle_powers<S, 8>(w, tw, k << (LN - 3 - LNS));
#pragma unroll
      for (int r = 1; r < 8; ++r)
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q][r] = cmul(v[q][r], w[r]);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) dft8<S>(v[q]);
    if constexpr (REM > 3) {
      const int bslot = slot_base<T, SWZ>(((j >> LNS) << (LNS + 3)) + k, ks);
      __syncthreads();
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int e = slot_plus<T, SWZ>(bslot, r << LNS, ks);
#pragma unroll
        for (int q = 0; q < NV; ++q) sl[q][e] = v[q][r];
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int e = slot_plus<T, SWZ>(jslot, s * N8, ks);
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q][s] = sl[q][e];
      }
      fft_static_pass<S, NV, SWZ, LN, LNS + 3>(v, sl, ks, j, jslot, tw);
    }
  } else if constexpr (REM == 2) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int k = (j + u * N8) & ((1 << LNS) - 1);
      cx<T> w[4];
      twiddle_powers<S, 4>(w, tw, k << (LN - 2 - LNS));
#pragma unroll
      for (int r = 1; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < NV; ++q) v[q][u + 2 * r] = cmul(v[q][u + 2 * r], w[r]);
#pragma unroll
      for (int q = 0; q < NV; ++q) dft4<S>(v[q][u], v[q][u + 2], v[q][u + 4], v[q][u + 6]);
    }
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = (j + u * N8) & ((1 << LNS) - 1);
      cx<T> w = ldg(&tw[k << (LN - 1 - LNS)]);
      if (S > 0) w.y = -w.y;
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        v[q][u + 4] = cmul(v[q][u + 4], w);
        dft2<S>(v[q][u], v[q][u + 4]);
      }
    }
  }
}

// The transform every kernel calls: FP32 transforms of length 2^8 .. 2^12 (the
// grids whose speed matters) use the compile-time-length code, all others the
// runtime-length loop.  lN is uniform across the CTA.
template <int S, int NV, bool SWZ = false, typename T>
__device__ __forceinline__ void fft_canon(cx<T> (&v)[NV][8], cx<T>* const* sl, int ks, int j,
                                          int lN, const cx<T>* __restrict__ tw) {
  if constexpr (std::is_same<T, float>::value) {
    const int js = slot_base<T, SWZ>(j, ks);
    switch (lN) {
      case 8: fft_static_pass<S, NV, SWZ, 8, 0>(v, sl, ks, j, js, tw); return;
      case 9: fft_static_pass<S, NV, SWZ, 9, 0>(v, sl, ks, j, js, tw); return;
      case 10: fft_static_pass<S, NV, SWZ, 10, 0>(v, sl, ks, j, js, tw); return;
      case 11: fft_static_pass<S, NV, SWZ, 11, 0>(v, sl, ks, j, js, tw); return;
      case 12: fft_static_pass<S, NV, SWZ, 12, 0>(v, sl, ks, j, js, tw); return;
      default: break;
    }
  }
  fft_rt<S, NV, SWZ>(v, sl, ks, j, lN, tw);
}

// ------------------------------------------------------------------ reductions
// Block-reduce K doubles; thread 0 gets the block total.
// WARP_DONE: the values are already warp sums held by lane 0.
template <int K, bool WARP_DONE = false>
__device__ __forceinline__ void block_sum(double (&v)[K]) {
  __shared__ double red[32 * K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  if (!WARP_DONE) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) red[warp * K + k] = v[k];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0;
      for (int w = 0; w < nw; ++w) s += red[w * K + k];
      v[k] = s;
    }
  }
}

// Write this CTA's K partial sums; returns true (in every thread) in the CTA
// that arrived last, which then holds the grand totals in tot (fixed order:
// CTA 0, 1, 2, ...), and re-arms the ticket.
// PRE: 0 per-thread values, 1 warp sums in lane 0, 2 the CTA's
// totals already in thread 0 (cta_pair_sums).
template <int K, int PRE = 0>
__device__ __forceinline__ bool last_cta_sum(double (&v)[K], double* partials,
                                             unsigned int* ticket, double (&tot)[K]) {
  __shared__ unsigned int s_last;
  if constexpr (PRE < 2) block_sum<K, PRE == 1>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) partials[blockIdx.x * kPartialStride + k] = v[k];
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    s_last = (t == gridDim.x - 1) ? 1u : 0u;
  }
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  // every thread of the last CTA sums a fixed strided subset of the partials,
  // then a fixed-order block reduction: deterministic for a given grid
  double w[K];
#pragma unroll
  for (int k = 0; k < K; ++k) w[k] = 0.0;
  for (unsigned int c = threadIdx.x; c < gridDim.x; c += blockDim.x)
#pragma unroll
    for (int k = 0; k < K; ++k) w[k] += __ldcg(&partials[c * kPartialStride + k]);
  block_sum<K>(w);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = w[k];
    *ticket = 0u;
  }
  return true;
}

// Per-thread dot-product accumulator.  FP64 data: plain FP64.  FP32 data: an
// unevaluated pair of floats (double-float): each product is split exactly
// into p + e with an FMA and added with Knuth's TwoSum, so the per-thread sum
// keeps about 48 significant bits while running on the FP32 pipes (GB300's
// FP64 rate is 1/58 of its FP32 rate).  Threads' sums are then promoted to
// FP64 for the block and grid reductions.
template <typename T>
struct DotAcc;
template <>
struct DotAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_prod(double x, double y) { s = fma(x, y, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct DotAcc<float> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add_prod(float x, float y) {
    const float p = x * y;
    const float e = fmaf(x, y, -p);  // x*y - p exactly
    const float t = hi + p;
    const float bp = t - hi;
    const float err = (hi - (t - bp)) + (p - bp);  // hi + p - t exactly
    hi = t;
    lo += err + e;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// Float-pair sums (about 48 significant bits): each addition an exact TwoSum
// of the high parts.  warp_pair sums a warp's pairs into lane 0 in fixed
// order.  On this part the FP64 pipe is narrow, and these keep the shuffle
// reductions of FP32 kernels off it.
__device__ __forceinline__ void pair_add(float& hi, float& lo, float h2, float l2) {
  const float t = hi + h2;
  const float bp = t - hi;
  lo = lo + l2 + ((hi - (t - bp)) + (h2 - bp));
  hi = t;
}
__device__ __forceinline__ void warp_pair(float& hi, float& lo) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float h2 = __shfl_down_sync(0xffffffffu, hi, off);
    const float l2 = __shfl_down_sync(0xffffffffu, lo, off);
    pair_add(hi, lo, h2, l2);
  }
}

// The CTA's sums of K float pairs (hi[k] + lo[k] of every thread), in fixed
// order, as doubles in thread 0: only those K conversions reach the FP64
// pipe, which on this part is narrow.
template <int K>
__device__ __forceinline__ void cta_pair_sums(float (&hi)[K], float (&lo)[K], double (&tot)[K]) {
  __shared__ float s_pair[64 * K];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) warp_pair(hi[k], lo[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      s_pair[2 * (warp * K + k)] = hi[k];
      s_pair[2 * (warp * K + k) + 1] = lo[k];
    }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) {
      float h = s_pair[2 * k], l = s_pair[2 * k + 1];
      for (int w = 1; w < nw; ++w) pair_add(h, l, s_pair[2 * (w * K + k)], s_pair[2 * (w * K + k) + 1]);
      tot[k] = (double)h + (double)l;
    }
}
// This CTA's float-pair partial stored as one double in partials[bx] with a
// plain store: no fence and no ticket.  Its reader is a later kernel (kernel
// boundaries order it).
__device__ __forceinline__ void cta_pair_partial(float hi, float lo, double* partials, int bx) {
  float h[1] = {hi}, l[1] = {lo};
  double t[1];
  cta_pair_sums<1>(h, l, t);
  if (threadIdx.x == 0) partials[(size_t)bx * kPartialStride] = t[0];
}

template <>
struct DotAcc<df64> {
  df64 s = df64(0.0f, 0.0f);
  __device__ __forceinline__ void add_prod(df64 x, df64 y) { s = s + x * y; }
  __device__ __forceinline__ double value() const { return (double)s.hi + (double)s.lo; }
};

// The sums sum m_a m_b of the current m (2D: xx, yy, xy) and sum |m|^2, the
// inputs of the next step's preconditioner (reading R3).
__device__ __forceinline__ void set_mm2(SolveState* st, double xx, double yy, double xy) {
  st->mm[0] = xx;
  st->mm[1] = yy;
  st->mm[2] = 0.0;
  st->mm[3] = xy;
  st->mm[4] = 0.0;
  st->mm[5] = 0.0;
  st->msum = xx + yy;
}

// The preconditioner matrix Kbar of reading R3 (constant, symmetric positive
// definite: the grid mean of m m^T + r I) in the kernel's type.
template <typename T>
struct Pc {
  T xx, yy, zz, xy, xz, yz;
};
template <typename T>
__device__ __forceinline__ Pc<T> pc_of(const SolveState* st) {
  if constexpr (std::is_same<T, float>::value)
    return Pc<float>{st->kbar_f[0], st->kbar_f[1], st->kbar_f[2],
                     st->kbar_f[3], st->kbar_f[4], st->kbar_f[5]};
  else
    return Pc<T>{(T)st->kbar[0], (T)st->kbar[1], (T)st->kbar[2],
                 (T)st->kbar[3], (T)st->kbar[4], (T)st->kbar[5]};
}
// The CG scalars in the kernel's type (FP32: the copies kept beside them).
template <typename T>
__device__ __forceinline__ T st_alpha(const SolveState* st) {
  if constexpr (std::is_same<T, float>::value) return st->alpha_f;
  else return (T)st->alpha;
}
template <typename T>
__device__ __forceinline__ T st_beta(const SolveState* st) {
  if constexpr (std::is_same<T, float>::value) return st->beta_f;
  else return (T)st->beta;
}
// x^y for a relaxation exponent y of kind 1, 2, 3 (y = 1, 2, 1/2: x, x x,
// sqrt x; x >= 0 here) or 0 (the general power).  The kind is uniform.
template <typename T>
__device__ __forceinline__ T pow_k(T x, T y, int kind) {
  switch (kind) {
    case 1: return x;
    case 2: return x * x;
    case 3: return hc_sqrt(x);
    default: return hc_pow(x, y);
  }
}

// A split-step coefficient in the kernel's type: FP32 kernels take the copy
// rounded on the host.
template <typename T>
__device__ __forceinline__ T cfv(double d, float f) {
  if constexpr (std::is_same<T, float>::value) return f;
  else return (T)d;
}

// Relaxation factor |m'| / |m| of eq. (m_relaxation_discrete) for gamma != 1
// and |m| = nm > 0.  With e = 2 (1 - gamma), the closed form
// (nm^e - e dt)^(1/e) / nm equals (1 - e dt nm^-e)^(1/e), and it is 0 where
// nm^e - e dt <= 0.  When 1/e is 1, 2 or 1/2 (gamma = 1/2, 3/4, 0) the first
// form is evaluated with those exact powers.  Otherwise the second, as
// exp(log1p(-e dt nm^-e) / e): raising nm^e - e dt to the power 1/e would
// multiply its rounding error by 1/e (5000 at gamma = 0.9999, a 3e-4 relative
// error per step in FP32), while log1p keeps the relative accuracy of the
// small term e dt nm^-e.
template <typename T>
__device__ __forceinline__ T relax_factor(T nm, const SplitCoef& cf) {
  if (cf.pow_b_kind != 0) {
    const T bb = pow_k(nm, cfv<T>(cf.pow_a, cf.f_pow_a), cf.pow_a_kind) -
                 cfv<T>(cf.two1mg_dt, cf.f_two1mg_dt);
    return bb >= (T)0 ? pow_k(bb, cfv<T>(cf.pow_b, cf.f_pow_b), cf.pow_b_kind) / nm : (T)0;
  }
  const T x = -cfv<T>(cf.two1mg_dt, cf.f_two1mg_dt) * hc_pow(nm, -cfv<T>(cf.pow_a, cf.f_pow_a));
  return x > (T)-1 ? hc_exp(hc_log1p(x) * cfv<T>(cf.pow_b, cf.f_pow_b)) : (T)0;
}
// 2^-e in T, exactly (0 <= e < 126), from the exponent bits: the reciprocal
// of a power-of-two point count without a division.
template <typename T>
__device__ __forceinline__ T exp2_neg(int e) {
  const float f = __int_as_float((127 - e) << 23);
  if constexpr (std::is_same<T, float>::value) return f;
  else return T((double)f);
}

// Preconditioner symbol 1 / (xi~^T Kbar xi~) of the constant-coefficient
// operator -div(Kbar grad) at derivative multipliers (a, b) (0 on the null
// modes, where a = b = 0).
template <typename T>
__device__ __forceinline__ T pinv_ab(T a, T b, const Pc<T>& k) {
  const T s2 = k.xx * a * a + (T)2 * k.xy * a * b + k.yy * b * b;
  return s2 > (T)0 ? (T)1 / s2 : (T)0;
}
template <typename T>
__device__ __forceinline__ T pinv_sym(const Geo<T>& g, int kx, int ky, const Pc<T>& k) {
  return pinv_ab(g.kxd[kx], g.kyd[ky], k);
}

// The same symbol evaluated in FP32, as the inner FP32 CG evaluates it.
template <typename T>
__device__ __forceinline__ float pinv_f32(const Geo<T>& g, int kx, int ky, const Pc<float>& k) {
  return pinv_ab((float)g.kxd[kx], (float)g.kyd[ky], k);
}

// ------------------------------------------------------------------ cp.async
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// 8-byte variant (cp.async.ca: the .cg form takes 16 bytes only), for tiles
// whose rows are one FP32 complex value wide.
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_prev() {  // all groups but the newest complete
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ------------------------------------------------------------------ row helpers
// The canonical-order input of the complex row a + i b of each of NV rows
// (thread j, slot s: element j + s N/8) from their packed half spectra A, B
// (B[q] null: b = 0).  With H = 4 N/8, slots 0..3 lie below the Nyquist index and
// slots 4..7 above it (mirrored, conjugated); only thread 0 meets the two
// special elements 0 and H, which share the packed slot 0.
template <int NV, typename T>
__device__ __forceinline__ void load_rows_c2r(cx<T> (&v)[NV][8], const cx<T>* const* A,
                                              const cx<T>* const* B, int j, int N8) {
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int idx = s < 4 ? j + s * N8 : ((s == 4 && j == 0) ? 0 : (8 - s) * N8 - j);
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const cx<T> a = A[q][idx], b = B[q] ? B[q][idx] : czero<T>();
      if (s == 0)
        v[q][s] = j == 0 ? cmk<T>(a.x, b.x) : cmk<T>(a.x - b.y, a.y + b.x);
      else if (s < 4)
        v[q][s] = cmk<T>(a.x - b.y, a.y + b.x);  // A + i B
      else if (s == 4)
        v[q][s] = j == 0 ? cmk<T>(a.y, b.y) : cmk<T>(a.x + b.y, b.x - a.y);
      else
        v[q][s] = cmk<T>(a.x + b.y, b.x - a.y);  // conj(A) + i conj(B)
    }
  }
}

// From the canonical-order spectra Z of NV complex rows a + i b, write the
// packed half spectra of a and b (B[q] may be null).
template <int NV, typename T>
__device__ __forceinline__ void store_rows_r2c(cx<T> (&v)[NV][8], cx<T>* const* slab, int j, int N,
                                               int H, cx<T>* const* A, cx<T>* const* B) {
  const int N8 = N >> 3;
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 8; ++s)
#pragma unroll
    for (int q = 0; q < NV; ++q) slab[q][rswz<T>(j + s * N8)] = v[q][s];
  __syncthreads();
#pragma unroll
  for (int s = 0; s < 4; ++s) {
    const int k = j + s * N8;  // k < H
    const int kc = k == 0 ? H : N - k;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      const cx<T> z = slab[q][rswz<T>(k)];
      const cx<T> zc = slab[q][rswz<T>(kc)];
      cx<T> a, b;
      if (k == 0) {
        a = cmk<T>(z.x, zc.x);
        b = cmk<T>(z.y, zc.y);
      } else {
        a = cmk<T>((T)0.5 * (z.x + zc.x), (T)0.5 * (z.y - zc.y));
        b = cmk<T>((T)0.5 * (z.y + zc.y), (T)-0.5 * (z.x - zc.x));
      }
      A[q][k] = a;
      if (B[q]) B[q][k] = b;
    }
  }
}
template <typename T>
__device__ __forceinline__ void store_pair_r2c(cx<T> (&v)[1][8], cx<T>* slab, int j, int N, int H,
                                               cx<T>* __restrict__ A, cx<T>* __restrict__ B) {
  cx<T>* const sl[1] = {slab};
  cx<T>* const a[1] = {A};
  cx<T>* const b[1] = {B};
  store_rows_r2c<1>(v, sl, j, N, H, a, b);
}

// ------------------------------------------------------------------ row kernels
template <typename T>
__global__ void __launch_bounds__(512) k_row_r2c(Geo<T> g, const T* __restrict__ a,
                                                 const T* __restrict__ b, cx<T>* __restrict__ A,
                                                 cx<T>* __restrict__ B) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const int l8 = g.lnx - 3, N = g.nx, H = g.H, N8 = 1 << l8;
  const int rb = threadIdx.x >> l8, j = threadIdx.x & (N8 - 1);
  const int y = (blockIdx.x << g.lrpc) + rb;
  cx<T>* slab = sm + rb * N;
  cx<T>* const sl[1] = {slab};
  const size_t ro = (size_t)y * N;
  cx<T> v[1][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = j + s * N8;
    v[0][s] = cmk<T>(a[ro + x], b ? b[ro + x] : (T)0);
  }
  fft_canon<-1, 1, true>(v, sl, 1, j, g.lnx, g.twx);
  store_pair_r2c(v, slab, j, N, H, A + (size_t)y * H, B ? B + (size_t)y * H : nullptr);
}

template <typename T>
__device__ __forceinline__ void row_c2r_body(Geo<T> g, const cx<T>* A, const cx<T>* B, T* a,
                                                 T* b, SolveState* st,
                                                 int kappa_update) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const int l8 = g.lnx - 3, N = g.nx, H = g.H, N8 = 1 << l8;
  const int rb = threadIdx.x >> l8, j = threadIdx.x & (N8 - 1);
  const int y = (blockIdx.x << g.lrpc) + rb;
  cx<T>* slab = sm + rb * N;
  cx<T>* const sl[1] = {slab};
  const cx<T>* Ar[1] = {A + (size_t)y * H};
  const cx<T>* Br[1] = {B ? B + (size_t)y * H : nullptr};
  cx<T> v[1][8];
  load_rows_c2r<1>(v, Ar, Br, j, N8);
  fft_canon<+1, 1, true>(v, sl, 1, j, g.lnx, g.twx);
  const size_t ro = (size_t)y * N;
  // this thread's 8 points: plain FMA sums of m_a m_b (the preconditioner's
  // input), FP64 across threads
  T mxx = (T)0, myy = (T)0, mxy = (T)0;
  DotAcc<T> d2;
  bool finite = true;
  const bool diag = kappa_update && st->diag;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = j + s * N8;
    if (diag) {  // Delta m: this thread reads the old values it overwrites
      const T da = v[0][s].x - a[ro + x], db = v[0][s].y - b[ro + x];
      d2.add_prod(da, da);
      d2.add_prod(db, db);
    }
    a[ro + x] = v[0][s].x;
    if (b) b[ro + x] = v[0][s].y;
    if (kappa_update) {
      mxx = mxx + v[0][s].x * v[0][s].x;
      myy = myy + v[0][s].y * v[0][s].y;
      mxy = mxy + v[0][s].x * v[0][s].y;
      finite = finite && hc_finite(v[0][s].x) && hc_finite(v[0][s].y);
    }
  }
  if (kappa_update) {
    if (!finite) st->nonfinite = 1;
    double acc[4], tot[4];
    bool last;
    if constexpr (std::is_same<T, float>::value) {  // float pairs up to the CTA total
      float h[4] = {mxx, myy, mxy, d2.hi}, l[4] = {0.0f, 0.0f, 0.0f, d2.lo};
      cta_pair_sums<4>(h, l, acc);
      last = last_cta_sum<4, 2>(acc, g.partials, &st->ticket[TK_MSUM], tot);
    } else {
      acc[0] = (double)mxx;
      acc[1] = (double)myy;
      acc[2] = (double)mxy;
      acc[3] = d2.value();
      last = last_cta_sum<4>(acc, g.partials, &st->ticket[TK_MSUM], tot);
    }
    if (last && threadIdx.x == 0) {
      set_mm2(st, tot[0], tot[1], tot[2]);
      if (diag) st->dm2 = tot[3];
    }
  }
}
template <typename T>
__global__ void __launch_bounds__(512) k_row_c2r(Geo<T> g, const cx<T>* A, const cx<T>* B, T* a,
                                                 T* b, SolveState* st,
                                                 int kappa_update) {
  row_c2r_body<T>(g, A, B, a, b, st, kappa_update);
}

// CG step length from the row pass.  With g = grad d (the physical gradient
// this pass receives) and K = m m^T + r I, the spectral <d, A d> equals
// n sum_x g . K g = n sum_x (m.g)^2 + r |g|^2 (summation by parts: the
// spectral derivative with the R1 multipliers is skew-adjoint), so alpha =
// rho / <d, A d> is known here and the divergence pass needs neither d nor a
// reduction.
__device__ __forceinline__ void cg_alpha_from(SolveState* st, double gkg, double n) {
  const double dq = gkg * n;
  if (dq > 0 && isfinite(dq)) {
    st->alpha = st->rho / dq;
    st->alpha_f = (float)st->alpha;
  } else {
    // breakdown: <d, A d> is not positive (d without a component in the range
    // of A) or not finite.  The plain solve then stops unconverged unless its
    // residual already meets the tolerance; a refined inner solve leaves that
    // verdict to the FP64 residual that follows it.
    st->alpha = 0;
    st->alpha_f = 0.0f;
    st->done = 1;
    if (!isfinite(dq))
      st->status = HC_ENONFINITE;
    else if (!st->refined && st->rnorm2 > st->thresh2)
      st->status = HC_ENOCONV;
  }
  st->first = 0;
}

// Step length of an FP32 CG iteration from the row pass's per-CTA partials of
// <d, A d> (cta_pair_partial): run by one CTA of the divergence pass that
// follows it, which sums them in fixed order and calls cg_alpha_from.  The
// update kernel after that pass reads alpha.
__device__ __forceinline__ void cg_alpha_finish(const Geo<float>& g, SolveState* st) {
  const int np = g.rpipe ? g.rgrid : (g.ny >> g.lrpc);  // CTAs of the row pass
  double a[1] = {0.0};
  for (int i = threadIdx.x; i < np; i += blockDim.x) a[0] += g.partials[(size_t)i * kPartialStride];
  block_sum<1>(a);
  if (threadIdx.x == 0) cg_alpha_from(st, a[0], (double)g.nx * (double)g.ny);
  __syncthreads();  // the block_sum scratch is reused by the caller
}

// Row pass of the operator apply.  The CTA's rows of m and r are staged into
// shared memory with cp.async at the start, so their latency overlaps the
// inverse transform.  DOT: the CG variant (alpha, see cg_alpha_from).  NV
// rows per thread: a group of N/8 threads transforms NV rows together,
// sharing twiddles, slot addresses and barriers (the CTA's rpc rows form
// rpc / NV groups).
template <typename T, typename Tm, bool DOT, int NV>
__device__ __forceinline__ void row_apply_body(Geo<T> g, const cx<T>* Gx, const cx<T>* Gy,
                                                   const Tm* __restrict__ mx,
                                                   const Tm* __restrict__ my,
                                                   const Tm* __restrict__ rr, cx<T>* Qx, cx<T>* Qy,
                                                   SolveState* st) {
  if (st && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const int l8 = g.lnx - 3, N = g.nx, H = g.H, N8 = 1 << l8;
  const int rb = threadIdx.x >> l8, j = threadIdx.x & (N8 - 1);
  const int r0 = rb * NV;                        // first of this group's rows within the CTA
  const int y0 = (blockIdx.x << g.lrpc) + r0;
  cx<T>* sl[NV];
  const cx<T>* Ar[NV];
  const cx<T>* Br[NV];
  cx<T>* Qa[NV];
  cx<T>* Qb[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    sl[q] = sm + (size_t)(r0 + q) * N;
    Ar[q] = Gx + (size_t)(y0 + q) * H;
    Br[q] = Gy + (size_t)(y0 + q) * H;
    Qa[q] = Qx + (size_t)(y0 + q) * H;
    Qb[q] = Qy + (size_t)(y0 + q) * H;
  }
  // stage the CTA's rows of mx, my, r (contiguous) behind the slabs
  Tm* sf = reinterpret_cast<Tm*>(sm + ((size_t)g.rpc << g.lnx));
  {
    const size_t row0 = ((size_t)blockIdx.x << g.lrpc) * N;
    const int per = (int)(((size_t)g.rpc * N * sizeof(Tm)) >> 4);  // 16-byte chunks per field
    const Tm* const src[3] = {mx + row0, my + row0, rr + row0};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      char* dst = reinterpret_cast<char*>(sf + (size_t)q * g.rpc * N);
      const char* from = reinterpret_cast<const char*>(src[q]);
      for (int c = threadIdx.x; c < per; c += blockDim.x) cp_async16(dst + 16 * c, from + 16 * c);
    }
    cp_async_commit();
  }
  cx<T> v[NV][8];
  load_rows_c2r<NV>(v, Ar, Br, j, N8);
  fft_canon<+1, NV, true>(v, sl, 1, j, g.lnx, g.twx);
  cp_async_wait_all();
  __syncthreads();
  // v = grad p (gx + i gy) at x = j + s N/8: apply (m (x) m + r I).  The
  // <d, A d> partial of a thread sums nv * 8 non-negative terms: plain
  // accumulation, FP64 across threads.
  T gkg = (T)0;
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    const Tm* smx = sf + (size_t)(r0 + q) * N;
    const Tm* smy = smx + (size_t)g.rpc * N;
    const Tm* srr = smy + (size_t)g.rpc * N;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int x = j + s * N8;
      const T gx = v[q][s].x, gy = v[q][s].y;
      const T ax = (T)smx[x], ay = (T)smy[x], r = (T)srr[x];
      const T mg = ax * gx + ay * gy;
      if (DOT) gkg = gkg + (mg * mg + r * (gx * gx + gy * gy));
      v[q][s] = cmk<T>(ax * mg + r * gx, ay * mg + r * gy);
    }
  }
  fft_canon<-1, NV, true>(v, sl, 1, j, g.lnx, g.twx);
  store_rows_r2c<NV>(v, sl, j, N, H, Qa, Qb);
  if (DOT) {
    if constexpr (std::is_same<T, float>::value) {
      // FP32: the CTA's partial only; the divergence pass forms alpha
      // (cg_alpha_finish), so this pass ends without a fence or ticket
      cta_pair_partial(gkg, 0.0f, g.partials, blockIdx.x);
    } else {
      double a1[1] = {(double)gkg}, t1[1];
      if (last_cta_sum<1>(a1, g.partials, &st->ticket[TK_DIV], t1) && threadIdx.x == 0)
        cg_alpha_from(st, t1[0], (double)g.nx * (double)g.ny);
    }
  }
}
template <typename T, typename Tm, bool DOT, int NV>
__global__ void __launch_bounds__(512) k_row_apply(Geo<T> g, const cx<T>* Gx, const cx<T>* Gy,
                                                   const Tm* __restrict__ mx,
                                                   const Tm* __restrict__ my,
                                                   const Tm* __restrict__ rr, cx<T>* Qx, cx<T>* Qy,
                                                   SolveState* st) {
  row_apply_body<T, Tm, DOT, NV>(g, Gx, Gy, mx, my, rr, Qx, Qy, st);
}

// Persistent FP32 row pass of the operator apply (g.rpipe): CTA b walks the
// row blocks b, b + grid, ... (rpc rows each, one row per N/8 threads).  Two
// stage buffers hold a block's Gx, Gy, mx, my, r rows (five contiguous pieces
// of rpc N 4 bytes); the next block's are copied with cp.async while the
// current one is transformed, so the loads' latency overlaps the FFTs.  Same
// arithmetic as k_row_apply<float, float, DOT, 1>.
template <bool DOT>
__global__ void __launch_bounds__(512) kp_row_apply(Geo<float> g, const cx<float>* Gx,
                                                    const cx<float>* Gy, const float* mx,
                                                    const float* my, const float* rr,
                                                    cx<float>* Qx, cx<float>* Qy, SolveState* st) {
  if (st && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int l8 = g.lnx - 3, N = g.nx, H = g.H, N8 = 1 << l8;
  const int rb = threadIdx.x >> l8, j = threadIdx.x & (N8 - 1);
  const int rpc = g.rpc, nblk = g.ny >> g.lrpc;
  const size_t piece = (size_t)rpc * N * 4;  // bytes of one field's rows in a block
  cx<float>* sl[1] = {reinterpret_cast<cx<float>*>(smem_raw) + (size_t)rb * N};
  unsigned char* bufs = smem_raw + 2 * piece;  // after the rpc slabs (rpc N complex)
  auto stage = [&](int blk, int b) {
    const int per = (int)(piece >> 4);  // 16-byte chunks per field
    unsigned char* dst = bufs + (size_t)b * 5 * piece;
    for (int c = threadIdx.x; c < 5 * per; c += blockDim.x) {
      const int f = c / per, ch = c - f * per;
      const unsigned char* src;
      if (f < 2)
        src = reinterpret_cast<const unsigned char*>((f == 0 ? Gx : Gy) + (size_t)blk * rpc * H);
      else
        src = reinterpret_cast<const unsigned char*>((f == 2 ? mx : (f == 3 ? my : rr)) +
                                                     (size_t)blk * rpc * N);
      cp_async16(dst + (size_t)f * piece + 16 * (size_t)ch, src + 16 * (size_t)ch);
    }
  };
  int blk = blockIdx.x, buf = 0;
  if (blk < nblk) stage(blk, 0);
  cp_async_commit();
  DotAcc<float> gkg;
  for (; blk < nblk; blk += gridDim.x) {
    const int nxt = blk + gridDim.x;
    if (nxt < nblk) stage(nxt, buf ^ 1);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    const unsigned char* B = bufs + (size_t)buf * 5 * piece;
    const cx<float>* A1[1] = {reinterpret_cast<const cx<float>*>(B) + (size_t)rb * H};
    const cx<float>* B1[1] = {reinterpret_cast<const cx<float>*>(B + piece) + (size_t)rb * H};
    const float* smx = reinterpret_cast<const float*>(B + 2 * piece) + (size_t)rb * N;
    const float* smy = reinterpret_cast<const float*>(B + 3 * piece) + (size_t)rb * N;
    const float* srr = reinterpret_cast<const float*>(B + 4 * piece) + (size_t)rb * N;
    cx<float> v[1][8];
    load_rows_c2r<1>(v, A1, B1, j, N8);
    fft_canon<+1, 1, true>(v, sl, 1, j, g.lnx, g.twx);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int x = j + s * N8;
      const float gx = v[0][s].x, gy = v[0][s].y;
      const float ax = smx[x], ay = smy[x], r = srr[x];
      const float mg = ax * gx + ay * gy;
      if (DOT) gkg.add_prod(mg * mg + r * (gx * gx + gy * gy), 1.0f);
      v[0][s] = cmk<float>(ax * mg + r * gx, ay * mg + r * gy);
    }
    fft_canon<-1, 1, true>(v, sl, 1, j, g.lnx, g.twx);
    const size_t y = (size_t)blk * rpc + rb;
    cx<float>* Qa[1] = {Qx + y * H};
    cx<float>* Qb[1] = {Qy + y * H};
    store_rows_r2c<1>(v, sl, j, N, H, Qa, Qb);
    __syncthreads();  // this buffer is refilled by the stage issued next iteration
    buf ^= 1;
  }
  cp_async_wait_all();
  if (DOT) cta_pair_partial(gkg.hi, gkg.lo, g.partials, blockIdx.x);  // alpha: cg_alpha_finish
}

// Pointwise sums of the discrete energy (Section 2.5) at one point, from m^k
// and g = grad p[m^k]: r |g|^2, (m.g)^2, and |m|^(2 gamma), or at gamma = 0
// ln|m|, the gradient-flow limit of (|m|^(2 gamma) - 1)/(2 gamma): the
// gamma = 0 relaxation term m/|m|^2 is its m-gradient.  ln 0 = -inf is kept
// out of the compensated float sums (inf - inf would give NaN there) and
// applied to the thread's total instead, so the sum is -inf when any |m| = 0.
template <typename T>
struct EnergyAcc {
  DotAcc<T> er, ea, em;
  bool zero = false;
  __device__ __forceinline__ void add(T r, T g2, T mg, T n2, T gamma) {
    er.add_prod(r, g2);
    ea.add_prod(mg, mg);
    if (gamma != (T)0)
      em.add_prod(n2 > (T)0 ? hc_pow(n2, gamma) : (T)0, (T)1);
    else if (n2 > (T)0)
      em.add_prod(hc_log(n2), (T)0.5);
    else
      zero = true;
  }
  // every CTA calls this (the flag is grid-uniform); totals into st->dsum
  __device__ __forceinline__ void finish(double* partials, SolveState* st) {
    double a[3] = {er.value(), ea.value(), zero ? -HUGE_VAL : em.value()}, t[3];
    if (last_cta_sum<3>(a, partials, &st->ticket[TK_DIAG], t) && threadIdx.x == 0) {
      st->dsum[0] = t[0];
      st->dsum[1] = t[1];
      st->dsum[2] = t[2];
    }
  }
};

// Activation then relaxation of one point's m = (ax, ay) with g = grad p.
// Activation, exact solution of dm/dt = c^2 (g g^T) m over dt written as
// m + c^2 dt phi1(c^2 |g|^2 dt) (m.g) g with phi1(z) = expm1(z)/z: the
// same value as eq. (m_activation_discrete) without forming exp(z) - 1.
// Relaxation, eq. (m_relaxation_discrete), through relax_factor.
template <typename T>
__device__ __forceinline__ void split_point(T& ax, T& ay, T gx, T gy, T c2dt, const SplitCoef& cf) {
  const T mg = ax * gx + ay * gy;
  if (mg != (T)0) {
    const T z = c2dt * (gx * gx + gy * gy);
    const T coef = z > (T)0 ? c2dt * (hc_expm1(z) / z) : c2dt;
    const T t = coef * mg;
    ax += t * gx;
    ay += t * gy;
  }
  if (cf.gamma_is_one) {
    ax *= cfv<T>(cf.exp_mdt, cf.f_exp_mdt);
    ay *= cfv<T>(cf.exp_mdt, cf.f_exp_mdt);
  } else {
    const T n2 = ax * ax + ay * ay;
    if (n2 > (T)0) {
      const T sc = relax_factor(hc_sqrt(n2), cf);
      ax *= sc;
      ay *= sc;
    }
  }
}

template <typename T>
__device__ __forceinline__ void row_split_body(Geo<T> g, const cx<T>* Gx, const cx<T>* Gy,
                                                   const T* __restrict__ mx,
                                                   const T* __restrict__ my,
                                                   const T* __restrict__ rr, cx<T>* Mx, cx<T>* My,
                                                   SplitCoef cf,
                                                   SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const int l8 = g.lnx - 3, N = g.nx, H = g.H, N8 = 1 << l8;
  const int rb = threadIdx.x >> l8, j = threadIdx.x & (N8 - 1);
  const int y = (blockIdx.x << g.lrpc) + rb;
  cx<T>* slab = sm + rb * N;
  cx<T>* const sl[1] = {slab};
  const cx<T>* Ar[1] = {Gx + (size_t)y * H};
  const cx<T>* Br[1] = {Gy + (size_t)y * H};
  const bool diag = st->diag != 0;
  // stage the CTA's rows of mx, my (and r for the diagnostics) behind the
  // slabs with cp.async, so that their latency overlaps the inverse transform
  T* sf = reinterpret_cast<T*>(sm + ((size_t)g.rpc << g.lnx));
  {
    const size_t row0 = ((size_t)blockIdx.x << g.lrpc) * N;
    const int per = (int)(((size_t)g.rpc * N * sizeof(T)) >> 4);  // 16-byte chunks per field
    const T* const src[3] = {mx + row0, my + row0, rr + row0};
    for (int q = 0; q < (diag ? 3 : 2); ++q) {
      char* dst = reinterpret_cast<char*>(sf + (size_t)q * g.rpc * N);
      const char* from = reinterpret_cast<const char*>(src[q]);
      for (int c = threadIdx.x; c < per; c += blockDim.x) cp_async16(dst + 16 * c, from + 16 * c);
    }
    cp_async_commit();
  }
  cx<T> v[1][8];
  load_rows_c2r<1>(v, Ar, Br, j, N8);
  fft_canon<+1, 1, true>(v, sl, 1, j, g.lnx, g.twx);
  cp_async_wait_all();
  __syncthreads();
  const T* smx = sf + (size_t)rb * N;
  const T* smy = smx + (size_t)g.rpc * N;
  const T* srr = smy + (size_t)g.rpc * N;
  const T c2dt = cfv<T>(cf.c2dt, cf.f_c2dt);
  bool finite = true;
  EnergyAcc<T> en;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = j + s * N8;
    const T gx = v[0][s].x, gy = v[0][s].y;
    T ax = smx[x], ay = smy[x];
    if (diag)
      en.add(srr[x], gx * gx + gy * gy, ax * gx + ay * gy, ax * ax + ay * ay, cfv<T>(cf.gamma, cf.f_gamma));
    split_point<T>(ax, ay, gx, gy, c2dt, cf);
    finite = finite && hc_finite(ax) && hc_finite(ay);
    v[0][s] = cmk<T>(ax, ay);
  }
  if (!finite) st->nonfinite = 1;
  if (diag) en.finish(g.partials, st);
  fft_canon<-1, 1, true>(v, sl, 1, j, g.lnx, g.twx);
  store_pair_r2c(v, slab, j, N, H, Mx + (size_t)y * H, My + (size_t)y * H);
}
template <typename T>
__global__ void __launch_bounds__(512) k_row_split(Geo<T> g, const cx<T>* Gx, const cx<T>* Gy,
                                                   const T* __restrict__ mx,
                                                   const T* __restrict__ my,
                                                   const T* __restrict__ rr, cx<T>* Mx, cx<T>* My,
                                                   SplitCoef cf,
                                                   SolveState* st) {
  row_split_body<T>(g, Gx, Gy, mx, my, rr, Mx, My, cf, st);
}

// ------------------------------------------------------------------ solve-state finalizers
// Plain CG start (one thread): r2 = ||b - A x0||^2, rz = <r, M^-1 r>.
__device__ __forceinline__ void resid_init(SolveState* st, double r2, double rz) {
  st->rnorm2 = r2;
  st->rho = rz;
  st->it = 0;
  st->first = 1;
  st->status = 0;
  st->done = (r2 <= st->thresh2 || st->maxit <= 0) ? 1 : 0;
  if (!isfinite(r2)) {
    st->status = HC_ENONFINITE;
    st->done = 1;
  }
  st->h_cur = st->h_inner;
  if (st->graph_mode) cudaGraphSetConditional(st->h_inner, st->done ? 0u : 1u);
}

// Refined modes, first sweep (one thread).  r32 = S - A p^k evaluated in FP32
// from the warm start: the right-hand side of the first inner solve, as in
// mixed-precision iterative refinement, whose first solve is a low-precision
// solve of the original system.  Its error, ~1e-7 ||S||, is removed by the
// FP64 residual that follows the solve; every convergence decision uses an
// FP64 residual.  Used only when the warm start is far from the solution
// (||r32||^2 > first32_min2 ||S||^2), else the step goes straight to FP64.
__device__ __forceinline__ void resid_first_init(SolveState* st, double r32, double rz) {
  const bool use = st->first32_min2 > 0 && isfinite(r32) && r32 > st->first32_min2 * st->outer_b2;
  st->bnorm2 = r32;
  st->thresh2 = fmax(st->inner_rtol2 * r32, 0.01 * st->outer_thresh2);
  st->rnorm2 = r32;
  st->rho = rz;
  st->it = 0;
  st->first = 1;
  st->done = use ? 0 : 1;
  st->first_used = use ? 1 : 0;
  if (use) {
    st->sweeps = 1;  // the next FP64 residual adds this sweep's correction
    st->acc_first += 1;
  }
  // with lagged certification the double-float residual always follows, as the
  // right-hand side of the step's last inner solve
  st->mid_phase = ((use || st->pipelined) && st->mid_df) ? 1 : 0;
  st->h_cur = st->h_first;
  if (st->graph_mode) {
    cudaGraphSetConditional(st->h_first, use ? 1u : 0u);
    if (st->mid_df) cudaGraphSetConditional(st->h_mid, st->mid_phase ? 1u : 0u);
  }
}

// Mid-step residual (one thread), HC_FP32_REFINED after an FP32 first sweep:
// S - A p64 evaluated in double-float (p64 += delta still in FP64).  It only
// supplies the right-hand side of the second inner solve, whose error it
// bounds at ~1e-14 ||S||; it never ends the refinement loop, which runs next
// and is decided by an FP64 residual.  The second solve is skipped when this
// residual is already below a tenth of the target.
__device__ __forceinline__ void resid_mid_init(SolveState* st, double r2, double r32, double rz) {
  st->mid_phase = 0;
  st->mid_used = 1;
  st->acc_mid += 1;
  const bool finite = isfinite(r2);
  st->bnorm2 = r32;
  st->thresh2 = fmax(st->inner_rtol2 * r32, 0.01 * st->outer_thresh2);
  st->rnorm2 = r32;
  st->rho = rz;
  st->it = 0;
  st->first = 1;
  st->done = (!finite || r32 == 0.0 || r2 <= 0.01 * st->outer_thresh2) ? 1 : 0;
  if (!st->done) st->sweeps += 1;
  st->h_cur = st->h_mid_inner;
  if (st->graph_mode) cudaGraphSetConditional(st->h_mid_inner, st->done ? 0u : 1u);
}

// Refinement sweep start (one thread): r64 = ||S - A p64||^2 decides the outer
// loop; r32, rz start the inner FP32 CG on A delta = r32 from delta = 0.
// (r32 is r64 rounded to FP32, so both norms are on the same scale.)
__device__ __forceinline__ void resid_refine_init(SolveState* st, double r64, double r32,
                                                  double rz) {
  st->res_full += 1;
  st->acc_res_full += 1;
  st->outer_r2 = r64;
  const bool finite = isfinite(r64);
  const bool conv = r64 <= st->outer_thresh2;
  st->outer_done = (conv || !finite || st->sweeps >= st->max_sweeps) ? 1 : 0;
  if (!finite) st->status = HC_ENONFINITE;
  else if (!conv && st->outer_done) st->status = HC_ENOCONV;
  else st->status = 0;
  st->bnorm2 = r32;
  // the inner solve only has to bring this sweep below the outer target: stop
  // at the larger of its own relative reduction and a tenth of the target
  st->thresh2 = fmax(st->inner_rtol2 * r32, 0.01 * st->outer_thresh2);
  st->rnorm2 = r32;
  st->rho = rz;
  st->it = 0;
  st->first = 1;
  st->done = (st->outer_done || r32 == 0.0) ? 1 : 0;
  if (!st->outer_done) st->sweeps += 1;
  st->h_cur = st->h_inner;
  if (st->graph_mode) {
    cudaGraphSetConditional(st->h_inner, st->done ? 0u : 1u);
    cudaGraphSetConditional(st->h_outer, st->outer_done ? 0u : 1u);
  }
}

// End of a CG iteration (one thread): ||r||^2 and rho = <r, M^-1 r> of the
// updated residual give beta, and the stop test closes or keeps the loop.
__device__ __forceinline__ void cg_step_finish(SolveState* st, double rr, double rz) {
  st->rnorm2 = rr;
  st->beta = st->rho > 0 ? rz / st->rho : 0.0;
  st->beta_f = (float)st->beta;
  st->rho = rz;
  st->it += 1;
  st->total_it += 1;
  if (!isfinite(rr)) {
    st->status = HC_ENONFINITE;
    st->done = 1;
  } else if (rr <= st->thresh2) {
    st->done = 1;
  } else if (st->it >= st->maxit) {
    st->done = 1;
    st->status = HC_ENOCONV;
  }
  if (st->graph_mode) cudaGraphSetConditional(st->h_cur, st->done ? 0u : 1u);
}

// The finalizer of a refinement-residual kernel: the mid-step one when it is
// pending, else a sweep of the refinement loop.
__device__ __forceinline__ void resid_sweep_init(SolveState* st, double r2, double r32, double rz) {
  if (st->mid_phase)
    resid_mid_init(st, r2, r32, rz);
  else
    resid_refine_init(st, r2, r32, rz);
}

// p64 += delta at one spectral value, then that value in the kernel's type.
// A double spectrum takes the correction in FP64 whatever T is.
template <typename T, typename Tin>
__device__ __forceinline__ cx<T> add_delta_at(cx<Tin>* in, size_t idx, cx<float> dl) {
  if constexpr (std::is_same<Tin, double>::value) {
    cx<double> pd = in[idx];
    pd.x += (double)dl.x;
    pd.y += (double)dl.y;
    in[idx] = pd;
    return ccast<T>(pd);
  } else {
    const cx<T> P = cadd(ccast<T>(in[idx]), ccast<T>(dl));
    in[idx] = ccast<Tin>(P);
    return P;
  }
}

// ------------------------------------------------------------------ step bookkeeping (one thread)
// Step start: the preconditioner constants, counters and thresholds.
__device__ __forceinline__ void step_begin_body(SolveState* st, int npts) {
  // reading R3: Kbar = kappa I with kappa = mean(r) + mean(|m|^2) / d, or
  // the caller's kappa; option HC_PRECOND_KBAR: Kbar = mean(m m^T) + mean(r) I.
  // kappa = trace(Kbar) / d is reported.
  const double kiso = st->user_kappa > 0 ? st->user_kappa
                                         : st->mean_r + st->msum / (double)npts / (double)st->dim;
  const bool aniso = st->user_kappa <= 0 && st->precond == HC_PRECOND_KBAR;
  for (int e = 0; e < 6; ++e) {
    const bool diag = e < 3, used = st->dim == 3 || e == 0 || e == 1 || e == 3;
    double v = 0.0;
    if (used) v = aniso ? st->mm[e] / (double)npts + (diag ? st->mean_r : 0.0) : (diag ? kiso : 0.0);
    st->kbar[e] = v;
    st->kbar_f[e] = (float)v;
  }
  st->kappa = 0.0;
  for (int a = 0; a < st->dim; ++a) st->kappa += st->kbar[a] / (double)st->dim;
  st->msum_old = st->msum;
  st->gm2_next_valid = 0;
  st->first_used = 0;
  st->mid_phase = 0;
  st->mid_used = 0;
  st->res_full = 0;
  st->outer_thresh2 = st->outer_rtol2 * st->outer_b2;
  st->it = 0;
  st->total_it = 0;
  st->sweeps = 0;
  st->done = 0;
  st->status = 0;
  st->nonfinite = 0;
  st->outer_done = 0;
  st->first = 1;
  if (!st->refined) st->thresh2 = st->outer_thresh2;
  if (st->graph_mode && st->refined && st->h_outer) cudaGraphSetConditional(st->h_outer, 1u);
}

// Diagnostics of Section 2.5 for the step that just ran from m^k: the energy
// E_h(m^k) (with p[m^k], the pressure this step solved) and Delta m^{k+1}.
// In run mode, the stopping rules of Algorithm 1's loop.
__device__ __forceinline__ void step_end_body(SolveState* st, int refined) {
  const int status = st->nonfinite ? HC_ENONFINITE : st->status;
  st->step_status = status;
  if (!st->first_bad && status) st->first_bad = status;
  st->acc_iters += st->total_it;
  st->acc_sweeps += st->sweeps;
  st->acc_steps += 1;
  if (st->diag) {
    if (st->gm2_valid) {
      st->energy_prev = st->energy;
      st->energy = st->e_coef[0] * st->gm2 + st->e_coef[1] * (st->dsum[0] + st->dsum[1]) +
                   st->e_coef[2] * st->dsum[2];
      st->energy_valid = 1;
      st->n_energy += 1;
    } else {
      st->energy_valid = 0;
    }
    st->delta_m = st->msum_old > 0 ? sqrt(st->dm2 / st->msum_old) / st->dt : 0.0;
    st->gm2 = st->gm2_next;
    st->gm2_valid = st->gm2_next_valid;
  } else {
    st->energy_valid = 0;
    st->gm2_valid = 0;
  }
  if (st->run_mode && !st->halt) {
    int reason = HC_STOP_NONE;
    if (status == HC_ENONFINITE) {
      reason = HC_STOP_STATUS;
    } else if (st->diag && st->eps_dm > 0 && st->delta_m <= st->eps_dm) {
      reason = HC_STOP_DELTA_M;
    } else if (st->stop_energy && st->energy_valid && st->n_energy >= 2 &&
               !(st->energy < st->energy_prev)) {
      // this step evaluated E(m^k) >= E(m^{k-1}); the previous step made m^k
      reason = HC_STOP_ENERGY;
      st->energy_step = st->acc_steps - 2;
    }
    if (reason != HC_STOP_NONE) {
      st->halt = 1;
      st->stop_reason = reason;
    }
  }
}

// ------------------------------------------------------------------ column kernels
// Thread layout of a column CTA: b = packed column within the tile (fastest),
// j = FFT thread index; slab q at sm + q * slab_elems + b with stride tc.
struct ColIdx {
  int b, j, kx, NY8;
};
template <typename T>
__device__ __forceinline__ ColIdx col_idx(const Geo<T>& g) {
  ColIdx c;
  c.b = threadIdx.x & (g.tc - 1);
  c.j = threadIdx.x >> g.ltc;
  c.kx = (blockIdx.x << g.ltc) + c.b;
  c.NY8 = 1 << (g.lny - 3);
  return c;
}
// Column-major index of (ky, kx) in a packed spectral vector of the 2D
// refinement (r, delta, the CG direction, the FP32 copy of S): one column
// tile of a column pass is contiguous there, so its loads and stores coalesce.
template <typename T>
__device__ __forceinline__ size_t cmi(const Geo<T>& g, int ky, int kx) {
  return ((size_t)kx << g.lny) + (size_t)ky;
}
template <typename T>
__device__ __forceinline__ int slab_elems(const Geo<T>& g) {
  return (g.ny + (g.ny >> 3)) * g.tc;
}

template <typename T, typename Tin, int MODE>
__device__ __forceinline__ void col_grad_body(Geo<T> g, cx<Tin>* in, const cx<T>* __restrict__ rvec,
                                                  cx<T>* dio, const cx<float>* __restrict__ delta,
                                                  cx<T>* __restrict__ Gx, cx<T>* __restrict__ Gy,
                                                  SolveState* st, int check_done) {
  if (check_done && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColIdx c = col_idx(g);
  const int H = g.H;
  const int se = slab_elems(g);
  cx<T>* const sl[2] = {sm + c.b, sm + se + c.b};
  const T invn = exp2_neg<T>(g.lnx + g.lny);  // 1 / (nx ny)
  const T ax = g.kxd[c.kx] * invn;
  bool first = false, add_delta = false;
  T beta = 0;
  Pc<T> pc{};
  if (MODE == CG_DUPDATE) {
    first = st->first != 0;
    beta = st_beta<T>(st);
    pc = pc_of<T>(st);
  }
  if (MODE == CG_ADDDELTA) add_delta = st->sweeps > 0;
  cx<T> v[2][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int ky = c.j + s * c.NY8;
    const size_t idx = (size_t)ky * H + c.kx;
    cx<T> P;
    if constexpr (MODE == CG_PLAIN) {
      P = ccast<T>(in[idx]);
    } else if constexpr (MODE == CG_DUPDATE) {
      // the FP32 refinement's vectors are column-major; plain FP64 CG's row-major
      const size_t vi = std::is_same<T, float>::value ? cmi(g, ky, c.kx) : idx;
      const T pv = pinv_sym(g, c.kx, ky, pc);
      const cx<T> z = cscale(rvec[vi], pv);
      P = first ? z : cadd(z, cscale(dio[vi], beta));
      dio[vi] = P;
    } else {
      // FP64 correction accumulation p64 += delta (refinement; delta column-major)
      P = add_delta ? add_delta_at<T>(in, idx, delta[cmi(g, ky, c.kx)]) : ccast<T>(in[idx]);
    }
    const T ay = g.kyd[ky] * invn;
    v[0][s] = cmk<T>(-ax * P.y, ax * P.x);  // i (kx/n) P
    v[1][s] = cmk<T>(-ay * P.y, ay * P.x);  // i (ky/n) P
  }
  fft_canon<+1, 2>(v, sl, g.tc, c.j, g.lny, g.twy);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = (size_t)(c.j + s * c.NY8) * H + c.kx;
    Gx[idx] = v[0][s];
    Gy[idx] = v[1][s];
  }
}
template <typename T, typename Tin, int MODE>
__global__ void __launch_bounds__(col_cta_max<T, true>(), 1) k_col_grad(Geo<T> g, cx<Tin>* in, const cx<T>* __restrict__ rvec,
                                                  cx<T>* dio, const cx<float>* __restrict__ delta,
                                                  cx<T>* __restrict__ Gx, cx<T>* __restrict__ Gy,
                                                  SolveState* st, int check_done) {
  col_grad_body<T, Tin, MODE>(g, in, rvec, dio, delta, Gx, Gy, st, check_done);
}

template <typename T, int MODE>
__device__ __forceinline__ void col_div_body(Geo<T> g, const cx<T>* __restrict__ Qx,
                                                 const cx<T>* __restrict__ Qy,
                                                 const cx<T>* __restrict__ d,
                                                 const cx<T>* __restrict__ bvec,
                                                 cx<T>* __restrict__ out, cx<float>* __restrict__ r32,
                                                 cx<float>* __restrict__ delta32, SolveState* st) {
  if ((MODE == CD_CG || MODE == CD_CERT) && st->done) return;
  if constexpr (MODE == CD_CG && std::is_same<T, float>::value)
    if (blockIdx.x == 0) cg_alpha_finish(g, st);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColIdx c = col_idx(g);
  const int H = g.H;
  const int se = slab_elems(g);
  cx<T>* const sl[2] = {sm + c.b, sm + se + c.b};
  cx<T> v[2][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = (size_t)(c.j + s * c.NY8) * H + c.kx;
    v[0][s] = Qx[idx];
    v[1][s] = Qy[idx];
  }
  fft_canon<-1, 2>(v, sl, g.tc, c.j, g.lny, g.twy);
  const T ax = g.kxd[c.kx];
  const double w = c.kx == 0 ? 1.0 : 2.0;  // Parseval weight of a packed column
  double acc[3] = {0.0, 0.0, 0.0};
  DotAcc<T> dq, r64acc;
  DotAcc<float> r32acc, rzacc;
  Pc<T> pc{};
  Pc<float> pcf{};
  if (MODE == CD_RESID) pc = pc_of<T>(st);
  if (MODE == CD_RESID_REFINE || MODE == CD_RESID_FIRST) pcf = pc_of<float>(st);
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int ky = c.j + s * c.NY8;
    const size_t idx = (size_t)ky * H + c.kx;
    const T ay = g.kyd[ky];
    const cx<T> t = cmk<T>(ax * v[0][s].x + ay * v[1][s].x, ax * v[0][s].y + ay * v[1][s].y);
    const cx<T> q = cmk<T>(t.y, -t.x);  // -i (kx Qx + ky Qy)
    if constexpr (MODE == CD_PLAIN) {
      out[idx] = q;
    } else if constexpr (MODE == CD_CG) {
      // alpha came from the row pass (cg_alpha_from); the FP32 refinement's
      // q is column-major, plain FP64 CG's row-major
      out[std::is_same<T, float>::value ? cmi(g, ky, c.kx) : idx] = q;
    } else if constexpr (MODE == CD_RESID) {
      const cx<T> rv = csub(bvec[idx], q);
      out[idx] = rv;
      const double r2 = (double)rv.x * (double)rv.x + (double)rv.y * (double)rv.y;
      acc[0] += w * r2;
      acc[1] += w * r2 * (double)pinv_sym(g, c.kx, ky, pc);
    } else if constexpr (MODE == CD_CERT) {
      // certification only: ||S - A p||^2 in the column's precision, nothing written
      const cx<T> rv = csub(bvec[idx], q);
      acc[0] += w * ((double)rv.x * (double)rv.x + (double)rv.y * (double)rv.y);
    } else if constexpr (MODE == CD_RESID_FIRST) {
      const size_t ci = cmi(g, ky, c.kx);  // b32, r32 and delta32 are column-major
      const cx<float> rf = ccast<float>(csub(bvec[ci], q));
      r32[ci] = rf;
      delta32[ci] = czero<float>();
      const float wf = (float)w, wpf = wf * pinv_f32(g, c.kx, ky, pcf);
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
      const size_t ci = cmi(g, ky, c.kx);  // r32 and delta32 are column-major
      r32[ci] = rf;
      delta32[ci] = czero<float>();
      const float wf = (float)w, wpf = wf * pinv_f32(g, c.kx, ky, pcf);
      r32acc.add_prod(wf * rf.x, rf.x);
      r32acc.add_prod(wf * rf.y, rf.y);
      rzacc.add_prod(wpf * rf.x, rf.x);
      rzacc.add_prod(wpf * rf.y, rf.y);
    }
  }
  if constexpr (MODE == CD_PLAIN || MODE == CD_CG) return;
  double tot[3];
  if constexpr (MODE == CD_CERT) {
    double a1[1] = {acc[0]}, t1[1];
    if (last_cta_sum<1>(a1, g.partials, &st->ticket[TK_CERT], t1) && threadIdx.x == 0)
      st->cert_r2 = t1[0];
  } else if constexpr (MODE == CD_RESID) {
    double a2[2] = {acc[0], acc[1]}, t2[2];
    if (last_cta_sum<2>(a2, g.partials, &st->ticket[TK_RESID], t2) && threadIdx.x == 0)
      resid_init(st, t2[0], t2[1]);
  } else if constexpr (MODE == CD_RESID_FIRST) {
    float h[2] = {r32acc.hi, rzacc.hi}, l[2] = {r32acc.lo, rzacc.lo};
    double a2[2], t2[2];
    cta_pair_sums<2>(h, l, a2);  // float pairs up to the CTA total
    if (last_cta_sum<2, 2>(a2, g.partials, &st->ticket[TK_RESID], t2) && threadIdx.x == 0)
      resid_first_init(st, t2[0], t2[1]);
  } else {
    bool last;
    if constexpr (std::is_same<T, df64>::value) {  // all three sums are float pairs
      float h[3] = {r64acc.s.hi, r32acc.hi, rzacc.hi}, l[3] = {r64acc.s.lo, r32acc.lo, rzacc.lo};
      cta_pair_sums<3>(h, l, acc);
      last = last_cta_sum<3, 2>(acc, g.partials, &st->ticket[TK_RESID], tot);
    } else {
      acc[0] = r64acc.value();
      acc[1] = r32acc.value();
      acc[2] = rzacc.value();
      last = last_cta_sum<3>(acc, g.partials, &st->ticket[TK_RESID], tot);
    }
    if (last && threadIdx.x == 0) resid_sweep_init(st, tot[0], tot[1], tot[2]);
  }
}
template <typename T, int MODE>
__global__ void __launch_bounds__(col_cta_max<T, true>(), 1) k_col_div(Geo<T> g, const cx<T>* __restrict__ Qx,
                                                 const cx<T>* __restrict__ Qy,
                                                 const cx<T>* __restrict__ d,
                                                 const cx<T>* __restrict__ bvec,
                                                 cx<T>* __restrict__ out, cx<float>* __restrict__ r32,
                                                 cx<float>* __restrict__ delta32, SolveState* st) {
  col_div_body<T, MODE>(g, Qx, Qy, d, bvec, out, r32, delta32, st);
}

// sum over one thread's spectral values of w |xi~|^2 (|v0|^2 + |v1|^2) (w the
// Parseval weight of the packed column kx, xi~ the R1 derivative multipliers;
// the packed column's cross terms cancel over ky).
template <typename T>
__device__ __forceinline__ void gradnorm_acc(const Geo<T>& g, DotAcc<T>& acc, int kx, int ky,
                                             const cx<T>& v0, const cx<T>& v1) {
  const T a = g.kxd[kx], b = g.kyd[ky];
  const T wk = (kx == 0 ? (T)1 : (T)2) * (a * a + b * b);
  acc.add_prod(wk * v0.x, v0.x);
  acc.add_prod(wk * v0.y, v0.y);
  acc.add_prod(wk * v1.x, v1.x);
  acc.add_prod(wk * v1.y, v1.y);
}
// Grid total of a per-CTA gradient-norm sum (every CTA calls it) times scale,
// into st->gm2 or st->gm2_next.
__device__ __forceinline__ void gradnorm_finish(double part, double scale, double* partials,
                                                SolveState* st, int into_next) {
  double a[1] = {part}, t[1];
  if (last_cta_sum<1>(a, partials, &st->ticket[TK_GRADM], t) && threadIdx.x == 0) {
    if (into_next) {
      st->gm2_next = t[0] * scale;
      st->gm2_next_valid = 1;
    } else {
      st->gm2 = t[0] * scale;
      st->gm2_valid = 1;
    }
  }
}

// Diffusion of one step along y for both components, one after the other
// through one slab (forward transform, heat factor, inverse), so that only one
// column's 8 values per thread are live: the FP32 pass then fits 64 registers
// and the wide tiles of the gradient and divergence passes.  The arithmetic
// per component is that of a joint two-component transform.
template <typename T>
__device__ __forceinline__ void col_heat_body(Geo<T> g, cx<T>* Mx, cx<T>* My, SolveState* st) {  // in place
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColIdx c = col_idx(g);
  const int H = g.H, ny = g.ny;
  cx<T>* const sl[1] = {sm + c.b};
  const T invn = exp2_neg<T>(g.lnx + g.lny);  // 1 / (nx ny)
  const bool diag = st && st->diag;
  DotAcc<T> ga;
#pragma unroll 1
  for (int q = 0; q < 2; ++q) {
    cx<T>* M = q == 0 ? Mx : My;
    cx<T> v[1][8];
#pragma unroll
    for (int s = 0; s < 8; ++s) v[0][s] = M[(size_t)(c.j + s * c.NY8) * H + c.kx];
    fft_canon<-1, 1>(v, sl, g.tc, c.j, g.lny, g.twy);
    if (blockIdx.x == 0) {
      // The packed column holds kx = 0 (A) and kx = nx/2 (B) as A + iB; their heat
      // factors differ, so separate with the ky <-> -ky symmetry:
      // new = (h0 + hN)/2 P[ky] + (h0 - hN)/2 conj(P[-ky]).
      __syncthreads();
#pragma unroll
      for (int s = 0; s < 8; ++s) sl[0][padk(c.j + s * c.NY8) * g.tc] = v[0][s];
      __syncthreads();
      if (c.b == 0) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int ky = c.j + s * c.NY8;
          const int kn = (ny - ky) & (ny - 1);
          const T h0 = g.hx[0] * g.hy[ky] * invn, hN = g.hx[H] * g.hy[ky] * invn;
          const T hp = (T)0.5 * (h0 + hN), hm = (T)0.5 * (h0 - hN);
          const cx<T> pn = sl[0][padk(kn) * g.tc];
          v[0][s] = cmk<T>(hp * v[0][s].x + hm * pn.x, hp * v[0][s].y - hm * pn.y);
        }
      }
    }
    if (c.kx != 0) {
#pragma unroll
      for (int s = 0; s < 8; ++s)
        v[0][s] = cscale(v[0][s], g.hx[c.kx] * g.hy[c.j + s * c.NY8] * invn);
    }
    if (diag) {  // v = F(m_new) / n: sum |grad m_new|^2 = n sum w |xi~|^2 |v|^2
#pragma unroll
      for (int s = 0; s < 8; ++s) gradnorm_acc(g, ga, c.kx, c.j + s * c.NY8, v[0][s], czero<T>());
    }
    fft_canon<+1, 1>(v, sl, g.tc, c.j, g.lny, g.twy);
#pragma unroll
    for (int s = 0; s < 8; ++s) M[(size_t)(c.j + s * c.NY8) * H + c.kx] = v[0][s];
    __syncthreads();  // the slab is the next component's
  }
  if (diag) gradnorm_finish(ga.value(), (double)g.nx * (double)ny, g.partials, st, 1);
}
template <typename T>
__global__ void __launch_bounds__(col_cta_max<T, true>(), 1) k_col_heat(Geo<T> g, cx<T>* Mx, cx<T>* My,
                                                                        SolveState* st) {
  col_heat_body<T>(g, Mx, My, st);
}

template <typename T, int NV>
__global__ void __launch_bounds__(512) k_col_fwd(Geo<T> g, const cx<T>* __restrict__ in0,
                                                 const cx<T>* __restrict__ in1, cx<T>* out0,
                                                 cx<T>* out1, int project, SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColIdx c = col_idx(g);
  const int H = g.H;
  const int se = slab_elems(g);
  cx<T>* const sl[2] = {sm + c.b, sm + se + c.b};
  cx<T> v[NV][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = (size_t)(c.j + s * c.NY8) * H + c.kx;
    v[0][s] = in0[idx];
    if (NV > 1) v[NV - 1][s] = in1[idx];
  }
  fft_canon<-1, NV>(v, sl, g.tc, c.j, g.lny, g.twy);
  double acc[1] = {0.0};
  const double w = c.kx == 0 ? 1.0 : 2.0;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int ky = c.j + s * c.NY8;
    const size_t idx = (size_t)ky * H + c.kx;
    if (project && c.kx == 0 && (ky == 0 || ky == (g.ny >> 1))) v[0][s] = czero<T>();  // corner modes
    out0[idx] = v[0][s];
    if (NV > 1) out1[idx] = v[NV - 1][s];
    acc[0] += w * ((double)v[0][s].x * (double)v[0][s].x + (double)v[0][s].y * (double)v[0][s].y);
  }
  if (project && st) {
    double tot[1];
    if (last_cta_sum<1>(acc, g.partials, &st->ticket[TK_PROJ], tot) && threadIdx.x == 0)
      st->outer_b2 = tot[0];
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_col_inv(Geo<T> g, const cx<T>* __restrict__ in,
                                                 cx<T>* __restrict__ out, T scale) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColIdx c = col_idx(g);
  const int H = g.H;
  cx<T>* const sl[1] = {sm + c.b};
  cx<T> v[1][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) v[0][s] = in[(size_t)(c.j + s * c.NY8) * H + c.kx];
  fft_canon<+1, 1>(v, sl, g.tc, c.j, g.lny, g.twy);
#pragma unroll
  for (int s = 0; s < 8; ++s) out[(size_t)(c.j + s * c.NY8) * H + c.kx] = cscale(v[0][s], scale);
}

// ------------------------------------------------------------------ pipelined column passes
// Persistent variants of the column passes: each CTA walks tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... and, while it transforms one tile, cp.async
// copies the next tile's inputs into the other half of a double buffer.  A
// buffer half holds two padded slabs (element (row, b) of slab q at
// q*se + padk(row)*tc + b), so once a tile's values are in registers its
// buffer half serves as the FFT exchange slabs.  Needs tc*sizeof(cx<T>) to be
// a multiple of 16 bytes (the cp.async size).
template <typename T, int NS, bool CM = false>
__device__ __forceinline__ void stage_cols(const Geo<T>& g, const cx<T>* a0, const cx<T>* a1,
                                           cx<T>* buf, int se, int kx0) {
  if constexpr (CM) {  // column-major FP32 vectors: 8-byte copies down each column
    static_assert(sizeof(cx<T>) == 8, "column-major staging is for FP32 vectors");
    const int per = g.ny << g.ltc;
    for (int c = threadIdx.x; c < NS * per; c += blockDim.x) {
      const int q = (NS > 1 && c >= per) ? 1 : 0;
      const int rem = c - q * per;
      const int bcol = rem >> g.lny, row = rem & (g.ny - 1);
      cp_async8(buf + q * se + padk(row) * g.tc + bcol,
                (q ? a1 : a0) + ((size_t)(kx0 + bcol) << g.lny) + row);
    }
    return;
  }
  constexpr int lce = sizeof(cx<T>) == 8 ? 1 : 0;  // log2 complex elements per 16-byte copy
  if (sizeof(cx<T>) == 8 && g.ltc == 0) {  // one FP32 column: 8-byte copies
    const int per = g.ny;
    for (int c = threadIdx.x; c < NS * per; c += blockDim.x) {
      const int q = (NS > 1 && c >= per) ? 1 : 0;
      const int row = c - q * per;
      cp_async8(buf + q * se + padk(row), (q ? a1 : a0) + (size_t)row * g.H + kx0);
    }
    return;
  }
  const int lcpr = g.ltc - lce;                     // log2 copies per row
  const int per = g.ny << lcpr;
  for (int c = threadIdx.x; c < NS * per; c += blockDim.x) {
    const int q = (NS > 1 && c >= per) ? 1 : 0;
    const int rem = c - q * per;
    const int row = rem >> lcpr, ch = rem & ((1 << lcpr) - 1);
    const cx<T>* src = (q ? a1 : a0) + (size_t)row * g.H + kx0 + (ch << lce);
    cp_async16(buf + q * se + padk(row) * g.tc + (ch << lce), src);
  }
}

template <typename T, int MODE>
__global__ void __launch_bounds__(512) kp_col_grad(Geo<T> g, cx<T>* in, const cx<T>* __restrict__ rvec,
                                                   cx<T>* dio, const cx<float>* __restrict__ delta,
                                                   cx<T>* __restrict__ Gx, cx<T>* __restrict__ Gy,
                                                   SolveState* st, int check_done) {
  if (check_done && st->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  constexpr int NS = MODE == CG_DUPDATE ? 2 : 1;
  const int H = g.H, se = slab_elems(g), ntiles = g.H >> g.ltc;
  const int b = threadIdx.x & (g.tc - 1), j = threadIdx.x >> g.ltc, NY8 = 1 << (g.lny - 3);
  const T invn = exp2_neg<T>(g.lnx + g.lny);  // 1 / (nx ny)
  bool first = false, add_delta = false;
  T beta = 0;
  Pc<T> pc{};
  if (MODE == CG_DUPDATE) {
    first = st->first != 0;
    beta = st_beta<T>(st);
    pc = pc_of<T>(st);
  }
  if (MODE == CG_ADDDELTA) add_delta = st->sweeps > 0;
  const cx<T>* s0 = MODE == CG_DUPDATE ? rvec : in;
  const cx<T>* s1 = MODE == CG_DUPDATE ? dio : nullptr;
  // this thread's rows are the same in every tile: load their wavenumbers once
  T kyv[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) kyv[s] = g.kyd[j + s * NY8];
  int half = 0;
  int tile = blockIdx.x;
  // the FP32 refinement's r and d are column-major
  constexpr bool CMV = MODE == CG_DUPDATE && std::is_same<T, float>::value;
  if (tile < ntiles) stage_cols<T, NS, CMV>(g, s0, s1, sm, se, tile << g.ltc);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    if (nxt < ntiles) stage_cols<T, NS, CMV>(g, s0, s1, sm + (half ^ 1) * 2 * se, se, nxt << g.ltc);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    cx<T>* cur = sm + half * 2 * se;
    const int kx = (tile << g.ltc) + b;
    const T kxv = g.kxd[kx];
    const T ax = kxv * invn;
    cx<float> dl[8];
    if (MODE == CG_ADDDELTA && add_delta) {
#pragma unroll
      for (int s = 0; s < 8; ++s) dl[s] = delta[cmi(g, j + s * NY8, kx)];
    }
    cx<T> v[2][8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int ky = j + s * NY8;
      const size_t idx = (size_t)ky * H + kx;
      const int e = padk(ky) * g.tc + b;
      cx<T> P;
      if constexpr (MODE == CG_PLAIN) {
        P = cur[e];
      } else if constexpr (MODE == CG_DUPDATE) {
        const T pv = pinv_ab(kxv, kyv[s], pc);
        const cx<T> z = cscale(cur[e], pv);
        P = first ? z : cadd(z, cscale(cur[se + e], beta));
        dio[CMV ? cmi(g, ky, kx) : idx] = P;
      } else {
        P = cur[e];
        if (add_delta) {
          P = cadd(P, ccast<T>(dl[s]));
          in[idx] = P;
        }
      }
      const T ay = kyv[s] * invn;
      v[0][s] = cmk<T>(-ax * P.y, ax * P.x);
      v[1][s] = cmk<T>(-ay * P.y, ay * P.x);
    }
    cx<T>* const sl[2] = {cur + b, cur + se + b};
    fft_canon<+1, 2>(v, sl, g.tc, j, g.lny, g.twy);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const size_t idx = (size_t)(j + s * NY8) * H + kx;
      Gx[idx] = v[0][s];
      Gy[idx] = v[1][s];
    }
    __syncthreads();
    half ^= 1;
  }
  cp_async_wait_all();
}

template <typename T, int MODE>
__global__ void __launch_bounds__(512) kp_col_div(Geo<T> g, const cx<T>* __restrict__ Qx,
                                                  const cx<T>* __restrict__ Qy,
                                                  const cx<T>* __restrict__ d,
                                                  const cx<T>* __restrict__ bvec,
                                                  cx<T>* __restrict__ out, cx<float>* __restrict__ r32,
                                                  cx<float>* __restrict__ delta32, SolveState* st) {
  if (MODE == CD_CG && st->done) return;
  if constexpr (MODE == CD_CG && std::is_same<T, float>::value)
    if (blockIdx.x == 0) cg_alpha_finish(g, st);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const int H = g.H, se = slab_elems(g), ntiles = g.H >> g.ltc;
  const int b = threadIdx.x & (g.tc - 1), j = threadIdx.x >> g.ltc, NY8 = 1 << (g.lny - 3);
  DotAcc<T> dq, r64acc;
  DotAcc<float> r32acc, rzacc;
  Pc<T> pc{};
  Pc<float> pcf{};
  if (MODE == CD_RESID) pc = pc_of<T>(st);
  if (MODE == CD_RESID_REFINE || MODE == CD_RESID_FIRST) pcf = pc_of<float>(st);
  double accr[2] = {0.0, 0.0};
  T kyv[8];  // this thread's rows are the same in every tile
#pragma unroll
  for (int s = 0; s < 8; ++s) kyv[s] = g.kyd[j + s * NY8];
  int half = 0;
  int tile = blockIdx.x;
  if (tile < ntiles) stage_cols<T, 2>(g, Qx, Qy, sm, se, tile << g.ltc);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    if (nxt < ntiles) stage_cols<T, 2>(g, Qx, Qy, sm + (half ^ 1) * 2 * se, se, nxt << g.ltc);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    cx<T>* cur = sm + half * 2 * se;
    const int kx = (tile << g.ltc) + b;
    cx<T> aux[8];  // b (residual), fetched early to overlap the FFT
    if (MODE == CD_RESID || MODE == CD_RESID_REFINE) {
#pragma unroll
      for (int s = 0; s < 8; ++s) aux[s] = bvec[(size_t)(j + s * NY8) * H + kx];
    } else if (MODE == CD_RESID_FIRST) {  // b32 is column-major
#pragma unroll
      for (int s = 0; s < 8; ++s) aux[s] = bvec[cmi(g, j + s * NY8, kx)];
    }
    cx<T> v[2][8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int e = padk(j + s * NY8) * g.tc + b;
      v[0][s] = cur[e];
      v[1][s] = cur[se + e];
    }
    cx<T>* const sl[2] = {cur + b, cur + se + b};
    fft_canon<-1, 2>(v, sl, g.tc, j, g.lny, g.twy);
    const T ax = g.kxd[kx];
    const double w = kx == 0 ? 1.0 : 2.0;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int ky = j + s * NY8;
      const size_t idx = (size_t)ky * H + kx;
      const T ay = kyv[s];
      const cx<T> t = cmk<T>(ax * v[0][s].x + ay * v[1][s].x, ax * v[0][s].y + ay * v[1][s].y);
      const cx<T> q = cmk<T>(t.y, -t.x);
      if constexpr (MODE == CD_PLAIN) {
        out[idx] = q;
      } else if constexpr (MODE == CD_CG) {
        // alpha came from the row pass (cg_alpha_from); FP32 q column-major
        out[std::is_same<T, float>::value ? cmi(g, ky, kx) : idx] = q;
      } else if constexpr (MODE == CD_RESID) {
        const cx<T> rv = csub(aux[s], q);
        out[idx] = rv;
        const double r2 = (double)rv.x * (double)rv.x + (double)rv.y * (double)rv.y;
        accr[0] += w * r2;
        accr[1] += w * r2 * (double)pinv_sym(g, kx, ky, pc);
      } else if constexpr (MODE == CD_RESID_FIRST) {
        const cx<float> rf = ccast<float>(csub(aux[s], q));
        const size_t ci = cmi(g, ky, kx);  // r32 and delta32 are column-major
        r32[ci] = rf;
        delta32[ci] = czero<float>();
        const float wf = (float)w, wpf = wf * pinv_f32(g, kx, ky, pcf);
        r32acc.add_prod(wf * rf.x, rf.x);
        r32acc.add_prod(wf * rf.y, rf.y);
        rzacc.add_prod(wpf * rf.x, rf.x);
        rzacc.add_prod(wpf * rf.y, rf.y);
      } else {
        const cx<T> rv = csub(aux[s], q);
        if (out) out[idx] = rv;
        const T wt = (T)(float)w;
        r64acc.add_prod(wt * rv.x, rv.x);
        r64acc.add_prod(wt * rv.y, rv.y);
        const cx<float> rf = ccast<float>(rv);
        const size_t ci = cmi(g, ky, kx);
        r32[ci] = rf;
        delta32[ci] = czero<float>();
        const float wf = (float)w, wpf = wf * pinv_f32(g, kx, ky, pcf);
        r32acc.add_prod(wf * rf.x, rf.x);
        r32acc.add_prod(wf * rf.y, rf.y);
        rzacc.add_prod(wpf * rf.x, rf.x);
        rzacc.add_prod(wpf * rf.y, rf.y);
      }
    }
    __syncthreads();
    half ^= 1;
  }
  cp_async_wait_all();
  if constexpr (MODE == CD_PLAIN || MODE == CD_CG) return;
  if constexpr (MODE == CD_RESID) {
    double t2[2];
    if (last_cta_sum<2>(accr, g.partials, &st->ticket[TK_RESID], t2) && threadIdx.x == 0)
      resid_init(st, t2[0], t2[1]);
  } else if constexpr (MODE == CD_RESID_FIRST) {
    double a2[2] = {r32acc.value(), rzacc.value()}, t2[2];
    if (last_cta_sum<2>(a2, g.partials, &st->ticket[TK_RESID], t2) && threadIdx.x == 0)
      resid_first_init(st, t2[0], t2[1]);
  } else {
    double acc[3] = {r64acc.value(), r32acc.value(), rzacc.value()}, tot[3];
    if (last_cta_sum<3>(acc, g.partials, &st->ticket[TK_RESID], tot) && threadIdx.x == 0)
      resid_sweep_init(st, tot[0], tot[1], tot[2]);
  }
}

template <typename T>
__global__ void __launch_bounds__(512) kp_col_heat(Geo<T> g, cx<T>* Mx, cx<T>* My, SolveState* st) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const int H = g.H, ny = g.ny, se = slab_elems(g), ntiles = g.H >> g.ltc;
  const int b = threadIdx.x & (g.tc - 1), j = threadIdx.x >> g.ltc, NY8 = 1 << (g.lny - 3);
  const T invn = exp2_neg<T>(g.lnx + g.lny);  // 1 / (nx ny)
  const bool diag = st && st->diag;
  DotAcc<T> ga;
  int half = 0;
  int tile = blockIdx.x;
  if (tile < ntiles) stage_cols<T, 2>(g, Mx, My, sm, se, tile << g.ltc);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const int nxt = tile + gridDim.x;
    if (nxt < ntiles) stage_cols<T, 2>(g, Mx, My, sm + (half ^ 1) * 2 * se, se, nxt << g.ltc);
    cp_async_commit();
    cp_async_wait_prev();
    __syncthreads();
    cx<T>* cur = sm + half * 2 * se;
    const int kx = (tile << g.ltc) + b;
    cx<T> v[2][8];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int e = padk(j + s * NY8) * g.tc + b;
      v[0][s] = cur[e];
      v[1][s] = cur[se + e];
    }
    cx<T>* const sl[2] = {cur + b, cur + se + b};
    fft_canon<-1, 2>(v, sl, g.tc, j, g.lny, g.twy);
    if (tile == 0) {
      // packed kx = 0 / nx/2 column: separate with the ky <-> -ky symmetry
      __syncthreads();
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int e = padk(j + s * NY8) * g.tc;
        sl[0][e] = v[0][s];
        sl[1][e] = v[1][s];
      }
      __syncthreads();
      if (b == 0) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const int ky = j + s * NY8;
          const int kn = (ny - ky) & (ny - 1);
          const T h0 = g.hx[0] * g.hy[ky] * invn, hN = g.hx[H] * g.hy[ky] * invn;
          const T hp = (T)0.5 * (h0 + hN), hm = (T)0.5 * (h0 - hN);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const cx<T> pn = sl[q][padk(kn) * g.tc];
            v[q][s] = cmk<T>(hp * v[q][s].x + hm * pn.x, hp * v[q][s].y - hm * pn.y);
          }
        }
      }
    }
    if (kx != 0) {
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const T h = g.hx[kx] * g.hy[j + s * NY8] * invn;
        v[0][s] = cscale(v[0][s], h);
        v[1][s] = cscale(v[1][s], h);
      }
    }
    if (diag) {
#pragma unroll
      for (int s = 0; s < 8; ++s) gradnorm_acc(g, ga, kx, j + s * NY8, v[0][s], v[1][s]);
    }
    fft_canon<+1, 2>(v, sl, g.tc, j, g.lny, g.twy);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const size_t idx = (size_t)(j + s * NY8) * H + kx;
      Mx[idx] = v[0][s];
      My[idx] = v[1][s];
    }
    __syncthreads();
    half ^= 1;
  }
  cp_async_wait_all();
  if (diag) gradnorm_finish(ga.value(), (double)g.nx * (double)ny, g.partials, st, 1);
}

// sum |grad m|^2 from the row spectra of m (forward FFT_y of two fields, no store).
template <typename T>
__global__ void __launch_bounds__(512) k_col_gradnorm(Geo<T> g, const cx<T>* __restrict__ Mx,
                                                      const cx<T>* __restrict__ My, SolveState* st,
                                                      int into_next) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColIdx c = col_idx(g);
  const int se = slab_elems(g);
  cx<T>* const sl[2] = {sm + c.b, sm + se + c.b};
  cx<T> v[2][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = (size_t)(c.j + s * c.NY8) * g.H + c.kx;
    v[0][s] = Mx[idx];
    v[1][s] = My[idx];
  }
  fft_canon<-1, 2>(v, sl, g.tc, c.j, g.lny, g.twy);
  DotAcc<T> ga;
#pragma unroll
  for (int s = 0; s < 8; ++s) gradnorm_acc(g, ga, c.kx, c.j + s * c.NY8, v[0][s], v[1][s]);
  gradnorm_finish(ga.value(), 1.0 / ((double)g.nx * (double)g.ny), g.partials, st, into_next);
}

// ------------------------------------------------------------------ CG update
template <typename T>
__device__ __forceinline__ void cg_update_body(Geo<T> g, cx<T>* __restrict__ x,
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
  const size_t total = (size_t)g.ny * g.H;
  DotAcc<T> rr, rz;
  // the FP32 refinement's vectors are column-major, plain FP64 CG's row-major
  constexpr bool CM = std::is_same<T, float>::value;
  auto upd = [&](size_t i, cx<T> dv, cx<T> xv, cx<T> qv, cx<T> rv) {
    const int kx = CM ? (int)(i >> g.lny) : (int)(i & (size_t)(g.H - 1));
    const int ky = CM ? (int)(i & (size_t)(g.ny - 1)) : (int)(i >> g.lH);
    x[i] = cmk<T>(xv.x + alpha * dv.x, xv.y + alpha * dv.y);
    rv = cmk<T>(rv.x - alpha * qv.x, rv.y - alpha * qv.y);
    r[i] = rv;
    const T wt = kx == 0 ? (T)1 : (T)2;
    const T wp = wt * pinv_sym(g, kx, ky, pc);  // weight times preconditioner symbol
    rr.add_prod(wt * rv.x, rv.x);
    rr.add_prod(wt * rv.y, rv.y);
    rz.add_prod(wp * rv.x, rv.x);
    rz.add_prod(wp * rv.y, rv.y);
  };
  // four elements per trip, all sixteen loads issued before any use
  constexpr int U = 4;
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
  double tot[2];
  bool last;
  if constexpr (std::is_same<T, float>::value) {
    float h[2] = {rr.hi, rz.hi}, l[2] = {rr.lo, rz.lo};
    double acc[2];
    cta_pair_sums<2>(h, l, acc);
    last = last_cta_sum<2, 2>(acc, g.partials, &st->ticket[TK_UPDATE], tot);
  } else {
    double acc[2] = {rr.value(), rz.value()};
    last = last_cta_sum<2>(acc, g.partials, &st->ticket[TK_UPDATE], tot);
  }
  if (last && threadIdx.x == 0) cg_step_finish(st, tot[0], tot[1]);
}
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 1) k_cg_update(Geo<T> g, cx<T>* __restrict__ x,
                                                   cx<T>* __restrict__ r,
                                                   const cx<T>* __restrict__ d,
                                                   const cx<T>* __restrict__ q, SolveState* st) {
  cg_update_body<T>(g, x, r, d, q, st);
}

// ------------------------------------------------------------------ elementwise
// Packed 2D spectrum (ny rows of H values, row-major) -> FP32 column-major
// copy (cmi), for the 2D refinement's FP32 source spectrum.
template <typename Ti>
__global__ void k_to_cm(Geo<float> g, const cx<Ti>* __restrict__ in, cx<float>* __restrict__ out) {
  const size_t n = (size_t)g.ny * g.H;
  for (size_t o = (size_t)blockIdx.x * blockDim.x + threadIdx.x; o < n;
       o += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(o >> g.lny), ky = (int)(o & (size_t)(g.ny - 1));
    const cx<Ti> v = in[(size_t)ky * g.H + kx];
    out[o] = cmk<float>((float)v.x, (float)v.y);
  }
}

template <typename To, typename Ti>
__global__ void k_convert(const Ti* __restrict__ in, To* __restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    out[i] = (To)in[i];
}

template <typename T>
__global__ void __launch_bounds__(256) k_msum(Geo<T> g, const T* __restrict__ mx,
                                              const T* __restrict__ my, SolveState* st) {
  const size_t n = (size_t)g.nx * g.ny;
  DotAcc<T> mxx, myy, mxy;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    mxx.add_prod(mx[i], mx[i]);
    myy.add_prod(my[i], my[i]);
    mxy.add_prod(mx[i], my[i]);
  }
  double acc[3] = {mxx.value(), myy.value(), mxy.value()};
  double tot[3];
  if (last_cta_sum<3>(acc, g.partials, &st->ticket[TK_MSUM], tot) && threadIdx.x == 0)
    set_mm2(st, tot[0], tot[1], tot[2]);
}

// ------------------------------------------------------------------ adjoint
// Reverse of one step (m^k, p^{k+1}) -> lambda^k given lambda^{k+1}.  With
// g = grad p^{k+1}, z = c^2 dt |g|^2, phi1(z) = expm1(z)/z:
//   a = m + c^2 dt phi1 (m.g) g,   b = a s(|a|)   (activation, relaxation)
//   lambda_a = J_rel(a) lambda_b,  J_rel = s I + (f' - s) a a^T / |a|^2 (symmetric)
//   lambda_m = lambda_a + c^2 dt phi1 (g.lambda_a) g
//   lambda_g = c^2 dt [phi1 ((m.g) lambda_a + m (g.lambda_a)) + 2 c^2 dt phi1'(z) (m.g)(g.lambda_a) g]
//   dL/dc^2 += (g.lambda_a)(m.g) dt (phi1 + z phi1')
// and, after the adjoint pressure solve A mu = -div lambda_g:
//   lambda^k = lambda_m - ((m.grad p) grad mu + (m.grad mu) grad p),  dL/dr -= grad mu . grad p.

template <typename T>
__device__ __forceinline__ T dphi1(T z) {  // d/dz (expm1(z)/z), z >= 0
  if (z < (T)0.5) {  // sum_k z^k / ((k+2) k!): the closed form cancels here
    T term = (T)1, s = (T)0.5;
#pragma unroll
    for (int k = 1; k < 14; ++k) {
      term = term * z / (T)k;
      s = s + term / (T)(k + 2);
    }
    return s;
  }
  return ((z - (T)1) * hc_expm1(z) + z) / (z * z);
}

template <typename T>
__device__ __forceinline__ void relax_jac(T ax, T ay, const SplitCoef& cf, T& c1, T& c2) {
  c2 = (T)0;
  if (cf.gamma_is_one) {
    c1 = cfv<T>(cf.exp_mdt, cf.f_exp_mdt);
    return;
  }
  const T n2 = ax * ax + ay * ay;
  if (n2 == (T)0) {
    c1 = cf.gamma > 1.0 ? (T)1 : (T)0;
    return;
  }
  const T rho = hc_sqrt(n2);
  const T e = cfv<T>(cf.pow_a, cf.f_pow_a);  // 2 (1 - gamma)
  const T beta = hc_pow(rho, e) - cfv<T>(cf.two1mg_dt, cf.f_two1mg_dt);
  if (!(beta > (T)0)) {
    c1 = (T)0;
    return;
  }
  const T f = hc_pow(beta, cfv<T>(cf.pow_b, cf.f_pow_b));                         // new modulus
  const T fp = hc_pow(beta, cfv<T>(cf.pow_b, cf.f_pow_b) - (T)1) * hc_pow(rho, e - (T)1);  // d f / d rho
  const T sv = f / rho;
  c1 = sv;
  c2 = (fp - sv) / n2;
}

template <typename T>
__global__ void __launch_bounds__(512) k_row_adj_point(Geo<T> g, cx<T>* G0, cx<T>* G1,
                                                       const cx<T>* L0, const cx<T>* L1,
                                                       const T* __restrict__ mx,
                                                       const T* __restrict__ my,
                                                       T* __restrict__ lmx, T* __restrict__ lmy,
                                                       SplitCoef cf, AdjState* as) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const int l8 = g.lnx - 3, N = g.nx, H = g.H, N8 = 1 << l8;
  const int rb = threadIdx.x >> l8, j = threadIdx.x & (N8 - 1);
  const int y = (blockIdx.x << g.lrpc) + rb;
  cx<T>* slab = sm + rb * 2 * N;
  cx<T>* const sl[2] = {slab, slab + N};
  cx<T> v[2][8];
  {
    const cx<T>* A2[2] = {G0 + (size_t)y * H, L0 + (size_t)y * H};
    const cx<T>* B2[2] = {G1 + (size_t)y * H, L1 + (size_t)y * H};
    load_rows_c2r<2>(v, A2, B2, j, N8);
  }
  fft_canon<+1, 2, true>(v, sl, 1, j, g.lnx, g.twx);
  const size_t ro = (size_t)y * N;
  const T c2dt = cfv<T>(cf.c2dt, cf.f_c2dt), dt = cfv<T>(cf.dt, cf.f_dt);
  DotAcc<T> dc;
  cx<T> w[1][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int x = j + s * N8;
    const T gx = v[0][s].x, gy = v[0][s].y, lbx = v[1][s].x, lby = v[1][s].y;
    const T mxv = mx[ro + x], myv = my[ro + x];
    const T z = c2dt * (gx * gx + gy * gy);
    const T ph = z > (T)0 ? hc_expm1(z) / z : (T)1;
    const T dph = dphi1(z);
    const T mg = mxv * gx + myv * gy;
    const T ax = mxv + c2dt * ph * mg * gx, ay = myv + c2dt * ph * mg * gy;
    T c1, c2r;
    relax_jac(ax, ay, cf, c1, c2r);
    const T al = ax * lbx + ay * lby;
    const T lax = c1 * lbx + c2r * al * ax, lay = c1 * lby + c2r * al * ay;
    const T gl = gx * lax + gy * lay;
    lmx[ro + x] = lax + c2dt * ph * gl * gx;
    lmy[ro + x] = lay + c2dt * ph * gl * gy;
    const T t2 = (T)2 * c2dt * dph * mg * gl;
    w[0][s] = cmk<T>(c2dt * (ph * (mg * lax + mxv * gl) + t2 * gx),
                     c2dt * (ph * (mg * lay + myv * gl) + t2 * gy));
    dc.add_prod(gl * mg, dt * (ph + z * dph));
  }
  cx<T>* const sl1[1] = {slab};
  fft_canon<-1, 1, true>(w, sl1, 1, j, g.lnx, g.twx);
  store_pair_r2c(w, slab, j, N, H, G0 + (size_t)y * H, G1 + (size_t)y * H);
  double a1[1] = {dc.value()}, t1[1];
  if (last_cta_sum<1>(a1, g.partials, &as->ticket[TA_POINT], t1) && threadIdx.x == 0)
    as->dc2 += t1[0];
}

template <typename T>
__global__ void __launch_bounds__(512) k_row_adj_press(Geo<T> g, const cx<T>* __restrict__ GM0,
                                                       const cx<T>* __restrict__ GM1,
                                                       const cx<T>* __restrict__ GP0,
                                                       const cx<T>* __restrict__ GP1,
                                                       const T* __restrict__ mx,
                                                       const T* __restrict__ my, const T* lmx,
                                                       const T* lmy, T* lx, T* ly, double* dr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const int l8 = g.lnx - 3, N = g.nx, H = g.H, N8 = 1 << l8;
  const int rb = threadIdx.x >> l8, j = threadIdx.x & (N8 - 1);
  const int y = (blockIdx.x << g.lrpc) + rb;
  cx<T>* slab = sm + rb * 2 * N;
  cx<T>* const sl[2] = {slab, slab + N};
  cx<T> v[2][8];
  {
    const cx<T>* A2[2] = {GM0 + (size_t)y * H, GP0 + (size_t)y * H};
    const cx<T>* B2[2] = {GM1 + (size_t)y * H, GP1 + (size_t)y * H};
    load_rows_c2r<2>(v, A2, B2, j, N8);
  }
  fft_canon<+1, 2, true>(v, sl, 1, j, g.lnx, g.twx);
  const size_t ro = (size_t)y * N;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t i = ro + j + s * N8;
    const T gmx = v[0][s].x, gmy = v[0][s].y, gpx = v[1][s].x, gpy = v[1][s].y;
    const T mxv = mx[i], myv = my[i];
    const T mgp = mxv * gpx + myv * gpy, mgm = mxv * gmx + myv * gmy;
    const T nx_ = lmx[i] - (gmx * mgp + gpx * mgm);
    const T ny_ = lmy[i] - (gmy * mgp + gpy * mgm);
    lx[i] = nx_;
    ly[i] = ny_;
    dr[i] -= (double)(gmx * gpx + gmy * gpy);
  }
}

template <typename T>
__global__ void __launch_bounds__(512) k_col_lap_dot(Geo<T> g, const cx<T>* __restrict__ A,
                                                     const cx<T>* __restrict__ B, double dt,
                                                     AdjState* as) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  const ColIdx c = col_idx(g);
  const int H = g.H, ny = g.ny;
  const int se = slab_elems(g);
  cx<T>* const sl[2] = {sm + c.b, sm + se + c.b};
  cx<T> v[2][8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const size_t idx = (size_t)(c.j + s * c.NY8) * H + c.kx;
    v[0][s] = A[idx];
    v[1][s] = B[idx];
  }
  fft_canon<-1, 2>(v, sl, g.tc, c.j, g.lny, g.twy);
  const T tdt = (T)dt;
  DotAcc<T> acc;
  if (blockIdx.x == 0) {
    // packed column: separate the kx = 0 (A) and kx = nx/2 (B) parts of both
    // vectors with the ky <-> -ky symmetry before weighting them
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int e = padk(c.j + s * c.NY8) * g.tc;
      sl[0][e] = v[0][s];
      sl[1][e] = v[1][s];
    }
    __syncthreads();
    if (c.b == 0) {
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const int ky = c.j + s * c.NY8;
        const int kn = (ny - ky) & (ny - 1);
        const cx<T> pa = v[0][s], pb = v[1][s];
        const cx<T> na = sl[0][padk(kn) * g.tc], nb = sl[1][padk(kn) * g.tc];
        // A-part = (P + conj(P-))/2, B-part = (P - conj(P-))/(2i)
        const cx<T> a0 = cmk<T>((T)0.5 * (pa.x + na.x), (T)0.5 * (pa.y - na.y));
        const cx<T> a1 = cmk<T>((T)0.5 * (pa.y + na.y), (T)-0.5 * (pa.x - na.x));
        const cx<T> b0 = cmk<T>((T)0.5 * (pb.x + nb.x), (T)0.5 * (pb.y - nb.y));
        const cx<T> b1 = cmk<T>((T)0.5 * (pb.y + nb.y), (T)-0.5 * (pb.x - nb.x));
        const T f0 = -(g.x2x[0] + g.x2y[ky]) * tdt, fN = -(g.x2x[H] + g.x2y[ky]) * tdt;
        acc.add_prod(f0 * a0.x, b0.x);
        acc.add_prod(f0 * a0.y, b0.y);
        acc.add_prod(fN * a1.x, b1.x);
        acc.add_prod(fN * a1.y, b1.y);
      }
    }
  }
  if (c.kx != 0) {
    const T xx = g.x2x[c.kx];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const T f = (T)-2 * (xx + g.x2y[c.j + s * c.NY8]) * tdt;  // weight 2 for kx > 0
      acc.add_prod(f * v[0][s].x, v[1][s].x);
      acc.add_prod(f * v[0][s].y, v[1][s].y);
    }
  }
  // A carries the row pass's inverse scaling (A = F_x(lambda_b) / nx, ready for
  // an unnormalised C2R) while B = F_x(b); Parseval's 1/(nx ny) then leaves 1/ny
  double a1[1] = {acc.value()}, t1[1];
  if (last_cta_sum<1>(a1, g.partials, &as->ticket[TA_LAP], t1) && threadIdx.x == 0)
    as->dD2 += t1[0] / (double)g.ny;
}

template <typename T>
__global__ void k_spec_accum(double* __restrict__ acc, const cx<T>* __restrict__ v, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    acc[2 * i] += (double)v[i].x;
    acc[2 * i + 1] += (double)v[i].y;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_spec_norm2(Geo<T> g, const cx<T>* __restrict__ v,
                                                    SolveState* st) {
  const size_t total = (size_t)g.ny * g.H;
  DotAcc<T> a;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const T w = (i & (size_t)(g.H - 1)) == 0 ? (T)1 : (T)2;
    a.add_prod(w * v[i].x, v[i].x);
    a.add_prod(w * v[i].y, v[i].y);
  }
  double a1[1] = {a.value()}, t1[1];
  if (last_cta_sum<1>(a1, g.partials, &st->ticket[TK_PROJ], t1) && threadIdx.x == 0)
    st->outer_b2 = t1[0];
}

// ------------------------------------------------------------------ launchers
template <typename T>
static inline int row_threads(const Geo<T>& g) { return g.rpc << (g.lnx - 3); }
template <typename T>
static inline size_t row_smem(const Geo<T>& g) {
  return (size_t)g.rpc * g.nx * sizeof(cx<T>);
}
// the split row pass: its slabs plus the staged rows of mx, my and r
template <typename T>
static inline size_t row_split_smem(const Geo<T>& g) {
  return row_smem(g) + (size_t)3 * g.rpc * g.nx * sizeof(T);
}
template <typename T>
static inline int col_threads(const Geo<T>& g) { return g.tc << (g.lny - 3); }
template <typename T>
static inline size_t col_smem(const Geo<T>& g, int nv) {
  return (size_t)nv * (g.ny + (g.ny >> 3)) * g.tc * sizeof(cx<T>);
}
static inline int upd_blocks(size_t total) {
  size_t b = (total + 255) / 256;
  return (int)(b < 608 ? b : 608);  // 4 CTAs of 256 threads per SM on 152 SMs
}

template <typename T>
void row_r2c(const Geo<T>& g, const T* a, const T* b, cx<T>* A, cx<T>* B, cudaStream_t s) {
  k_row_r2c<T><<<g.ny >> g.lrpc, row_threads(g), row_smem(g), s>>>(g, a, b, A, B);
}
template <typename T>
void row_c2r(const Geo<T>& g, const cx<T>* A, const cx<T>* B, T* a, T* b, SolveState* st,
             int kappa_update, cudaStream_t s) {
  k_row_c2r<T><<<g.ny >> g.lrpc, row_threads(g), row_smem(g), s>>>(g, A, B, a, b, st, kappa_update);
}
template <typename T, typename Tm>
void row_apply(const Geo<T>& g, const cx<T>* Gx, const cx<T>* Gy, const Tm* mx, const Tm* my,
               const Tm* r, cx<T>* Qx, cx<T>* Qy, SolveState* st, cudaStream_t s) {
  const size_t sm = row_smem(g) + (size_t)3 * g.rpc * g.nx * sizeof(Tm);
  if constexpr (std::is_same<T, float>::value && std::is_same<Tm, float>::value) {
    if (g.rpipe) {
      const size_t ps = row_pipe_smem(g.rpc, g.nx);
      if (st)
        kp_row_apply<true><<<g.rgrid, row_threads(g), ps, s>>>(g, Gx, Gy, mx, my, r, Qx, Qy, st);
      else
        kp_row_apply<false><<<g.rgrid, row_threads(g), ps, s>>>(g, Gx, Gy, mx, my, r, Qx, Qy, st);
      return;
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    if (g.rpc >= 2) {  // two rows per thread
      const int nt = row_threads(g) >> 1;
      if (st)
        k_row_apply<T, Tm, true, 2><<<g.ny >> g.lrpc, nt, sm, s>>>(g, Gx, Gy, mx, my, r, Qx, Qy, st);
      else
        k_row_apply<T, Tm, false, 2><<<g.ny >> g.lrpc, nt, sm, s>>>(g, Gx, Gy, mx, my, r, Qx, Qy, st);
      return;
    }
  }
  if (st)
    k_row_apply<T, Tm, true, 1><<<g.ny >> g.lrpc, row_threads(g), sm, s>>>(g, Gx, Gy, mx, my, r, Qx,
                                                                          Qy, st);
  else
    k_row_apply<T, Tm, false, 1><<<g.ny >> g.lrpc, row_threads(g), sm, s>>>(g, Gx, Gy, mx, my, r, Qx,
                                                                           Qy, st);
}
template <typename T>
void row_split(const Geo<T>& g, const cx<T>* Gx, const cx<T>* Gy, const T* mx, const T* my,
               const T* r, cx<T>* Mx, cx<T>* My, SplitCoef cf, SolveState* st, cudaStream_t s) {
  k_row_split<T><<<g.ny >> g.lrpc, row_threads(g), row_split_smem(g), s>>>(g, Gx, Gy, mx, my, r, Mx,
                                                                           My, cf, st);
}
template <typename T>
void col_fwd(const Geo<T>& g0, const cx<T>* in0, const cx<T>* in1, cx<T>* out0, cx<T>* out1, int nv,
             int project, SolveState* st, cudaStream_t s) {
  const Geo<T> g = col_narrow(g0);
  if (nv == 1)
    k_col_fwd<T, 1><<<g.H >> g.ltc, col_threads(g), col_smem(g, 1), s>>>(g, in0, in1, out0, out1,
                                                                          project, st);
  else
    k_col_fwd<T, 2><<<g.H >> g.ltc, col_threads(g), col_smem(g, 2), s>>>(g, in0, in1, out0, out1,
                                                                          project, st);
}
template <typename T>
void col_inv(const Geo<T>& g0, const cx<T>* in, cx<T>* out, T scale, cudaStream_t s) {
  const Geo<T> g = col_narrow(g0);
  k_col_inv<T><<<g.H >> g.ltc, col_threads(g), col_smem(g, 1), s>>>(g, in, out, scale);
}
template <typename T>
static inline size_t pipe_smem(const Geo<T>& g) {
  return (size_t)4 * (g.ny + (g.ny >> 3)) * g.tc * sizeof(cx<T>);
}

template <typename T, typename Tin>
void col_grad(const Geo<T>& g0, int mode, cx<Tin>* in, const cx<T>* rvec, cx<T>* dio,
              const cx<float>* delta, cx<T>* Gx, cx<T>* Gy, SolveState* st, int check_done,
              cudaStream_t s) {
  // the whole tile; the persistent passes at most 512 threads
  const Geo<T> g = g0.pipe ? col_narrow(g0) : g0;
  const int nb = g.H >> g.ltc, nt = col_threads(g);
  const size_t sm = col_smem(g, 2);
  if constexpr (std::is_same<T, Tin>::value) {
    if (g.pipe) {
      const size_t ps = pipe_smem(g);
      if (mode == CG_PLAIN)
        kp_col_grad<T, CG_PLAIN><<<g.pgrid, nt, ps, s>>>(g, in, rvec, dio, delta, Gx, Gy, st, check_done);
      else if (mode == CG_DUPDATE)
        kp_col_grad<T, CG_DUPDATE><<<g.pgrid, nt, ps, s>>>(g, in, rvec, dio, delta, Gx, Gy, st,
                                                          check_done);
      else
        kp_col_grad<T, CG_ADDDELTA><<<g.pgrid, nt, ps, s>>>(g, in, rvec, dio, delta, Gx, Gy, st,
                                                           check_done);
      return;
    }
  }
  if (mode == CG_PLAIN)
    k_col_grad<T, Tin, CG_PLAIN><<<nb, nt, sm, s>>>(g, in, rvec, dio, delta, Gx, Gy, st, check_done);
  else if (mode == CG_DUPDATE)
    k_col_grad<T, Tin, CG_DUPDATE><<<nb, nt, sm, s>>>(g, in, rvec, dio, delta, Gx, Gy, st,
                                                      check_done);
  else
    k_col_grad<T, Tin, CG_ADDDELTA><<<nb, nt, sm, s>>>(g, in, rvec, dio, delta, Gx, Gy, st,
                                                       check_done);
}
template <typename T>
void col_div(const Geo<T>& g0, int mode, const cx<T>* Qx, const cx<T>* Qy, const cx<T>* d,
             const cx<T>* b, cx<T>* out, cx<float>* r32, cx<float>* delta32, SolveState* st,
             cudaStream_t s) {
  // the whole tile; the persistent passes at most 512 threads
  const Geo<T> g = g0.pipe ? col_narrow(g0) : g0;
  const int nb = g.H >> g.ltc, nt = col_threads(g);
  const size_t sm = col_smem(g, 2);
  if (g.pipe) {
    const size_t ps = pipe_smem(g);
    switch (mode) {
      case CD_PLAIN:
        kp_col_div<T, CD_PLAIN><<<g.pgrid, nt, ps, s>>>(g, Qx, Qy, d, b, out, r32, delta32, st);
        break;
      case CD_CG:
        kp_col_div<T, CD_CG><<<g.pgrid, nt, ps, s>>>(g, Qx, Qy, d, b, out, r32, delta32, st);
        break;
      case CD_RESID:
        kp_col_div<T, CD_RESID><<<g.pgrid, nt, ps, s>>>(g, Qx, Qy, d, b, out, r32, delta32, st);
        break;
      case CD_RESID_FIRST:
        if constexpr (std::is_same<T, float>::value)
          kp_col_div<T, CD_RESID_FIRST><<<g.pgrid, nt, ps, s>>>(g, Qx, Qy, d, b, out, r32, delta32, st);
        break;

      default:
        kp_col_div<T, CD_RESID_REFINE><<<g.pgrid, nt, ps, s>>>(g, Qx, Qy, d, b, out, r32, delta32, st);
        break;
    }
    return;
  }
  switch (mode) {
    case CD_PLAIN:
      k_col_div<T, CD_PLAIN><<<nb, nt, sm, s>>>(g, Qx, Qy, d, b, out, r32, delta32, st);
      break;
    case CD_CG:
      k_col_div<T, CD_CG><<<nb, nt, sm, s>>>(g, Qx, Qy, d, b, out, r32, delta32, st);
      break;
    case CD_RESID:
      k_col_div<T, CD_RESID><<<nb, nt, sm, s>>>(g, Qx, Qy, d, b, out, r32, delta32, st);
      break;
    case CD_RESID_FIRST:
      if constexpr (std::is_same<T, float>::value)
        k_col_div<T, CD_RESID_FIRST><<<nb, nt, sm, s>>>(g, Qx, Qy, d, b, out, r32, delta32, st);
      break;

    default:
      k_col_div<T, CD_RESID_REFINE><<<nb, nt, sm, s>>>(g, Qx, Qy, d, b, out, r32, delta32, st);
      break;
  }
}
template <typename T>
void col_heat(const Geo<T>& g0, cx<T>* Mx, cx<T>* My, SolveState* st, cudaStream_t s) {
  // the whole tile (one slab); the persistent pass at most 512 threads
  const Geo<T> g = g0.pipe ? col_narrow(g0) : g0;
  if (g.pipe) {
    kp_col_heat<T><<<g.pgrid, col_threads(g), pipe_smem(g), s>>>(g, Mx, My, st);
    return;
  }
  k_col_heat<T><<<g.H >> g.ltc, col_threads(g), col_smem(g, 1), s>>>(g, Mx, My, st);
}
template <typename T>
void col_gradnorm(const Geo<T>& g0, const cx<T>* Mx, const cx<T>* My, SolveState* st, int into_next,
                  cudaStream_t s) {
  const Geo<T> g = col_narrow(g0);
  k_col_gradnorm<T><<<g.H >> g.ltc, col_threads(g), col_smem(g, 2), s>>>(g, Mx, My, st, into_next);
}
template <typename T>
void cg_update(const Geo<T>& g, cx<T>* x, cx<T>* r, const cx<T>* d, const cx<T>* q, SolveState* st,
               cudaStream_t s) {
  k_cg_update<T><<<upd_blocks((size_t)g.ny * g.H), 256, 0, s>>>(g, x, r, d, q, st);
}
template <typename Ti>
void to_cm(const Geo<float>& g, const cx<Ti>* in, cx<float>* out, cudaStream_t s) {
  k_to_cm<Ti><<<upd_blocks((size_t)g.ny * g.H), 256, 0, s>>>(g, in, out);
}
template <typename To, typename Ti>
void convert(const Ti* in, To* out, size_t n, cudaStream_t s) {
  k_convert<To, Ti><<<upd_blocks(n), 256, 0, s>>>(in, out, n);
}
template <typename T>
void msum(const Geo<T>& g, const T* mx, const T* my, SolveState* st, cudaStream_t s) {
  k_msum<T><<<upd_blocks((size_t)g.nx * g.ny), 256, 0, s>>>(g, mx, my, st);
}
template <typename T>
void row_adj_point(const Geo<T>& g, cx<T>* G0, cx<T>* G1, const cx<T>* L0, const cx<T>* L1,
                   const T* mx, const T* my, T* lmx, T* lmy, SplitCoef cf, AdjState* as,
                   cudaStream_t s) {
  k_row_adj_point<T><<<g.ny >> g.lrpc, row_threads(g), 2 * row_smem(g), s>>>(g, G0, G1, L0, L1, mx,
                                                                             my, lmx, lmy, cf, as);
}
template <typename T>
void row_adj_press(const Geo<T>& g, const cx<T>* GM0, const cx<T>* GM1, const cx<T>* GP0,
                   const cx<T>* GP1, const T* mx, const T* my, const T* lmx, const T* lmy, T* lx,
                   T* ly, double* dr, cudaStream_t s) {
  k_row_adj_press<T><<<g.ny >> g.lrpc, row_threads(g), 2 * row_smem(g), s>>>(
      g, GM0, GM1, GP0, GP1, mx, my, lmx, lmy, lx, ly, dr);
}
template <typename T>
void col_lap_dot(const Geo<T>& g0, const cx<T>* A, const cx<T>* B, double dt, AdjState* as,
                 cudaStream_t s) {
  const Geo<T> g = col_narrow(g0);
  k_col_lap_dot<T><<<g.H >> g.ltc, col_threads(g), col_smem(g, 2), s>>>(g, A, B, dt, as);
}
template <typename T>
void spec_accum(const Geo<T>& g, double* acc, const cx<T>* v, cudaStream_t s) {
  const size_t n = (size_t)g.ny * g.H;
  k_spec_accum<T><<<upd_blocks(n), 256, 0, s>>>(acc, v, n);
}
template <typename T>
void spec_norm2(const Geo<T>& g, const cx<T>* v, SolveState* st, cudaStream_t s) {
  k_spec_norm2<T><<<upd_blocks((size_t)g.ny * g.H), 256, 0, s>>>(g, v, st);
}

// Allow a kernel the full opt-in shared memory of the device, less its own
// static shared memory (the two together may not exceed the opt-in limit).
template <typename K>
void allow_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, kernel) != cudaSuccess) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       optin - (int)a.sharedSizeBytes);
}

template <typename T>
void set_smem_limits_t() {
  allow_smem(k_row_r2c<T>);
  allow_smem(k_row_c2r<T>);
  allow_smem(k_row_apply<T, T, false, 1>);
  allow_smem(k_row_apply<T, T, true, 1>);
  if constexpr (std::is_same<T, float>::value) {
    allow_smem(k_row_apply<T, T, false, 2>);
    allow_smem(k_row_apply<T, T, true, 2>);
  }
  allow_smem(k_row_split<T>);
  allow_smem(k_col_fwd<T, 1>);
  allow_smem(k_col_fwd<T, 2>);
  allow_smem(k_col_inv<T>);
  allow_smem(k_col_heat<T>);
  allow_smem(k_col_gradnorm<T>);
  allow_smem(k_col_div<T, CD_PLAIN>);
  allow_smem(k_col_div<T, CD_CG>);
  allow_smem(k_col_div<T, CD_RESID>);
  allow_smem(k_col_div<T, CD_RESID_REFINE>);
  if constexpr (std::is_same<T, float>::value) {
    allow_smem(k_col_div<T, CD_RESID_FIRST>);
    allow_smem(kp_col_div<T, CD_RESID_FIRST>);
  }
  allow_smem(kp_col_div<T, CD_PLAIN>);
  allow_smem(kp_col_div<T, CD_CG>);
  allow_smem(kp_col_div<T, CD_RESID>);
  allow_smem(kp_col_div<T, CD_RESID_REFINE>);
  allow_smem(kp_col_heat<T>);
  allow_smem(kp_col_grad<T, CG_PLAIN>);
  allow_smem(kp_col_grad<T, CG_DUPDATE>);
  allow_smem(kp_col_grad<T, CG_ADDDELTA>);
  allow_smem(k_row_adj_point<T>);
  allow_smem(k_row_adj_press<T>);
  allow_smem(k_col_lap_dot<T>);
}
template <typename T, typename Tin>
void set_smem_limits_grad() {
  allow_smem(k_col_grad<T, Tin, CG_PLAIN>);
  allow_smem(k_col_grad<T, Tin, CG_DUPDATE>);
  allow_smem(k_col_grad<T, Tin, CG_ADDDELTA>);
}

}  // namespace hc
