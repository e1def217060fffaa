// hc_api.cu -- C ABI and host orchestration of one time step of the Fourier
// spectral FFT+CG splitting scheme (arXiv 2606.06720, Algorithm 1).
//
// The host only sequences kernels and moves the boundary's FP64 arrays.  All
// arithmetic of the step runs in the kernels of hc_kernels_f32.cu /
// hc_kernels_f64.cu.  CG loop control is device-side: every iteration kernel
// returns at once when the solve state says "done", so the host either polls
// a small state block every few iterations (host loop) or, in graph mode,
// replays one CUDA graph per step whose CG and refinement loops are
// conditional WHILE nodes driven by the kernels themselves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "hc.h"
#include "hc_internal.cuh"

using hc::cx;
using hc::df64;

namespace {

constexpr size_t kAlign = 256;
constexpr int kChunk = 4;  // CG iterations launched between host polls (host-loop mode)
constexpr int kRunChunk = 16;  // gated step launches between host polls (hc_run, graph mode)

#ifndef HC_CHECK
#define HC_CHECK 0
#endif

// Bounds-checked build (HC_CHECK=1): each buffer carved from a workspace is
// followed by a guard zone (the alignment gap plus kRedzone bytes) holding
// kPattern.  The production build carves no zones.
constexpr size_t kRedzone = HC_CHECK ? (size_t)HC_REDZONE_BYTES : 0;
constexpr int kMaxZones = 128;
constexpr unsigned char kPattern = 0xA5;

// Guard zones of one workspace, in carve order.  A plain aggregate: the
// context holding one is cleared with memset, a local one is value-initialised.
struct Zones {
  int n;       // zones recorded (at most kMaxZones)
  int carved;  // zones carved; more than n means the table overflowed
  size_t start[kMaxZones];  // byte offset from the workspace base
  size_t len[kMaxZones];
  size_t owner[kMaxZones];  // bytes of the buffer the zone follows
};

struct Layout {
  size_t off = 0;
  char* base = nullptr;
  Zones* zones = nullptr;
  template <typename P>
  P* take(size_t bytes) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    P* p = base ? reinterpret_cast<P*>(base + off) : nullptr;
    off += bytes;
    if (kRedzone) {
      const size_t end = (off + kAlign - 1) / kAlign * kAlign + kRedzone;
      if (zones) {
        if (zones->n < kMaxZones) {
          zones->start[zones->n] = off;
          zones->len[zones->n] = end - off;
          zones->owner[zones->n] = bytes;
          ++zones->n;
        }
        ++zones->carved;
      }
      off = end;
    }
    return p;
  }
};

bool is_pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

// Sizes of the generic 2D path: 4 .. 4096 points with no prime factor above 5.
bool is_235_in(int v, int lo, int hi) {
  if (v < lo || v > hi) return false;
  for (int p : {2, 3, 5})
    while (v % p == 0) v /= p;
  return v == 1;
}
// A 2D grid that the power-of-two kernels do not take.
bool generic_grid(const hc_grid* g) {
  return g && g->dim == 2 && !(is_pow2_in(g->n[0], 8, 4096) && is_pow2_in(g->n[1], 8, 4096));
}
// Radix passes (4, 2, 3, 5) of a generic transform length; returns their count.
int radices(int N, int* r) {
  int np = 0;
  while (N % 4 == 0) { r[np++] = 4; N /= 4; }
  while (N % 2 == 0) { r[np++] = 2; N /= 2; }
  while (N % 3 == 0) { r[np++] = 3; N /= 3; }
  while (N % 5 == 0) { r[np++] = 5; N /= 5; }
  return np;
}
int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

}  // namespace

// Conditional handles of one step chain: the CG loop of the refinement sweeps
// (or of plain PCG), the refinement loop, the first (FP32-started) inner loop,
// and the mid-step residual block (IF) with its inner loop.
struct Handles {
  cudaGraphConditionalHandle inner = 0, outer = 0, first = 0, mid = 0, mid_inner = 0;
};

struct hc_ctx {
  hc_grid grid;
  hc_params prm;
  Zones zones;  // guard zones of the workspace (bounds-checked build only)
  int dim;   // 2 or 3
  int gen;   // 1: a 2D grid whose sizes are not both powers of two (hc_generic.cu, FP64)
  int nx, ny, nz, H;  // nz = 1 in 2D; H = spectral columns (nx/2 packed, nx/2 + 1 generic)
  size_t n;  // points
  size_t ns; // packed spectral values: nz * ny * H
  int refined;
  int df;    // refined with double-float state and residual
  int mid_df;  // HC_FP32_REFINED: the residual after an FP32 first sweep is double-float
  cudaStream_t stream;
  bool owns_ws;
  void* ws;
  size_t ws_bytes;
  long long launches;
  double mean_r;

  // device memory (all inside the workspace)
  hc::SolveState* st;
  hc::SolveState* st_time;  // scratch state for hc_time_kernel (never drives a loop)
  double* partials;
  double* stage;            // 2n doubles: FP64 boundary staging
  cx<double>* p64;          // pressure spectrum
  cx<double>* b64;          // source spectrum (projected)
  cx<double>* r64;          // residual (FP64)
  cx<double>* d64;          // CG direction (plain mode)
  cx<double>* q64;          // A d (plain mode)
  cx<double>* G64;          // dim spectra: gradient / flux / m scratch (FP64)
  cx<float>* b32;           // refined: FP32 copy of the projected source spectrum
  cx<df64>* bq;             // HC_FP32_REFINED: double-float copy of it (mid-step residual)
  cx<float>* r32;           // refined: inner residual
  cx<float>* d32;           // refined: inner direction
  cx<float>* q32;           // refined: A d
  cx<float>* x32;           // refined: inner solution (correction delta)
  cx<float>* G32;           // refined: dim spectra scratch (FP32)
  void* m[3];               // conductivity components (double or float); m[2] in 3D only
  void* rf;                 // permeability r (double or float)
  // tables
  cx<float>*twx_f, *twy_f;
  cx<double>*twx_d, *twy_d;
  cx<df64>*twx_q, *twy_q;
  float *kxd_f, *kyd_f, *hx_f, *hy_f;
  double *kxd_d, *kyd_d, *hx_d, *hy_d;
  df64 *kxd_q, *kyd_q;
  float *x2x_f, *x2y_f;
  double *x2x_d, *x2y_d;
  cx<float>* twz_f;         // 3D only
  cx<double>* twz_d;
  cx<df64>* twz_q;
  float *kzd_f, *hz_f;
  double *kzd_d, *hz_d;
  df64* kzd_q;
  hc::Geo<float> gf;
  hc::Geo<double> gd;
  hc::Geo<df64> gq;  // double-float kernels (HC_FP32_REFINED_DF)
  hc::GenGeo gg;     // generic sizes: geometry and tables of the mixed-radix kernels
  // The same geometry seen as ny*nz rows of length nx: the 2D row kernels
  // (R2C/C2R of single fields) run the x pass of a 3D grid through these.
  hc::Geo<float> rowf;
  hc::Geo<double> rowd;
  hc::Geo<df64> rowq;

  hc::SolveState* st_host;  // pinned mirror for readback
  // graph mode: captured on a private stream (capture is illegal on the
  // legacy default stream), launched on `stream`
  cudaStream_t cap_stream;
  cudaGraphExec_t gexec;
  Handles h_own;                        // handles of the context's own graph
  int batch_handles;                    // 1 while st holds a batch graph's handles
  bool graph_ready;
  // hc_run: the step wrapped in a device-gated IF node, diagnostics on
  cudaGraphExec_t gexec_run;
  Handles h_run;                        // handles of the run graph's step chain
  cudaGraphConditionalHandle h_gate;
  bool run_graph_ready;
  int force_diag;                       // 1 while hc_run runs (diagnostics forced on)
  // Lagged certification (2D HC_FP32_REFINED; see hc_params.sync_cert): the
  // previous step's input m and its pressure await their FP64 certification
  // (m_prev, p_saved) while the next step runs; the split step writes m_tmp.
  float* m_prev[2];
  float* m_tmp[2];
  cx<double>* p_saved;
  cx<double>* G64c;                     // the certifying residual's FP64 scratch (two fields)
  double* partials_c;                   // its per-CTA partial sums
  hc::SolveState* st_c;                 // its state (cert_pending, cert_r2, done = nothing pending)
  cudaGraphExec_t gexec_pipe;
  bool pipe_ready;
  Handles h_pipe;
  cudaGraphConditionalHandle h_pipe_gate;
  cudaStream_t cap_hi, cap_lo;          // capture streams of the lagged graph's two branches
  cudaStream_t io_stream;               // hc_set_state / hc_get_state: copies beside p's transform
  cudaEvent_t io_ev[2 + 4];             // entry, copies done, and one per row chunk of p
  int graph_nodes_fixed, graph_nodes_body, graph_nodes_outer;
};

namespace {

// exp(-2 pi i m / N) for m < N, with exact octant symmetry.
void twiddles(int N, std::vector<double>& re, std::vector<double>& im) {
  re.resize(N);
  im.resize(N);
  const double half_pi = 1.57079632679489661923;
  for (int m = 0; m < N; ++m) {
    const long long a4 = 4LL * m;
    const int q = (int)(a4 / N);
    const long long r = a4 - (long long)q * N;  // angle = (pi/2) (q + r/N)
    double c, s;
    if (2 * r <= N) {
      const double phi = half_pi * (double)r / N;
      c = std::cos(phi);
      s = std::sin(phi);
    } else {
      const double phi = half_pi * (double)(N - r) / N;
      c = std::sin(phi);
      s = std::cos(phi);
    }
    double ct, stt;
    switch (q & 3) {
      case 0: ct = c; stt = s; break;
      case 1: ct = -s; stt = c; break;
      case 2: ct = -c; stt = -s; break;
      default: ct = s; stt = -c; break;
    }
    re[m] = ct;
    im[m] = -stt;
  }
}

// Fourier variable of Section 2.3.3 (Nyquist entry positive).
double xi(int l, int N, double L) {
  const double two_pi = 6.28318530717958647692;
  return (2 * l <= N) ? two_pi * l / L : two_pi * (l - N) / L;
}
// First-derivative multiplier, Nyquist entry zero.
double xid(int l, int N, double L) { return (2 * l == N) ? 0.0 : xi(l, N, L); }

// Most CTAs of any kernel that reduces through the per-CTA partials.
size_t max_reducing_ctas(const hc_ctx* c) {
  size_t m = std::max<size_t>({(size_t)c->H, (size_t)c->ny, (size_t)1216});
  if (c->dim == 3) m = std::max(m, (size_t)c->ny * c->H);  // z pass with one column per CTA
  return m;
}

// Generic sizes (FP64 plain only): the solve state, the FP64 spectral vectors
// of the unpacked half spectrum, the fields and the mixed-radix tables.
void layout_generic(hc_ctx* c, Layout& L) {
  const size_t n = c->n;
  const size_t S64 = c->ns * sizeof(cx<double>);
  c->st = L.take<hc::SolveState>(sizeof(hc::SolveState));
  c->st_time = L.take<hc::SolveState>(sizeof(hc::SolveState));
  c->partials = L.take<double>(sizeof(double) * hc::kPartialStride * max_reducing_ctas(c));
  c->stage = L.take<double>(sizeof(double) * 2 * n);
  c->p64 = L.take<cx<double>>(S64);
  c->b64 = L.take<cx<double>>(S64);
  c->r64 = L.take<cx<double>>(S64);
  c->d64 = L.take<cx<double>>(S64);
  c->q64 = L.take<cx<double>>(S64);
  c->G64 = L.take<cx<double>>(2 * S64);
  for (int k = 0; k < 2; ++k) c->m[k] = L.take<double>(sizeof(double) * n);
  c->rf = L.take<double>(sizeof(double) * n);
  c->twx_d = L.take<cx<double>>(sizeof(cx<double>) * c->nx);
  c->twy_d = L.take<cx<double>>(sizeof(cx<double>) * c->ny);
  c->kxd_d = L.take<double>(sizeof(double) * c->H);
  c->kyd_d = L.take<double>(sizeof(double) * c->ny);
  c->hx_d = L.take<double>(sizeof(double) * c->H);
  c->hy_d = L.take<double>(sizeof(double) * c->ny);
}

void layout(hc_ctx* c, Layout& L) {
  if (c->gen) {
    layout_generic(c, L);
    return;
  }
  const size_t n = c->n;
  const int d = c->dim;
  const size_t S64 = c->ns * sizeof(cx<double>);
  const size_t S32 = c->ns * sizeof(cx<float>);
  c->st = L.take<hc::SolveState>(sizeof(hc::SolveState));
  c->st_time = L.take<hc::SolveState>(sizeof(hc::SolveState));
  c->partials = L.take<double>(sizeof(double) * hc::kPartialStride * max_reducing_ctas(c));
  c->stage = L.take<double>(sizeof(double) * d * n);
  c->p64 = L.take<cx<double>>(S64);
  c->b64 = L.take<cx<double>>(S64);
  c->r64 = L.take<cx<double>>(S64);
  c->G64 = L.take<cx<double>>(d * S64);
  if (!c->refined) {
    c->d64 = L.take<cx<double>>(S64);
    c->q64 = L.take<cx<double>>(S64);
    c->b32 = c->r32 = c->d32 = c->q32 = c->x32 = c->G32 = nullptr;
    c->bq = nullptr;
    for (int k = 0; k < d; ++k) c->m[k] = L.take<double>(sizeof(double) * n);
    c->rf = L.take<double>(sizeof(double) * n);
  } else {
    c->d64 = c->q64 = nullptr;
    c->bq = c->df ? nullptr : L.take<cx<df64>>(S64);
    c->b32 = L.take<cx<float>>(S32);
    c->r32 = L.take<cx<float>>(S32);
    c->d32 = L.take<cx<float>>(S32);
    c->q32 = L.take<cx<float>>(S32);
    c->x32 = L.take<cx<float>>(S32);
    c->G32 = L.take<cx<float>>(d * S32);
    for (int k = 0; k < d; ++k) c->m[k] = L.take<float>(sizeof(float) * n);
    c->rf = L.take<float>(sizeof(float) * n);
    if (d == 2 && !c->df) {  // lagged certification
      for (int k = 0; k < 2; ++k) c->m_prev[k] = L.take<float>(sizeof(float) * n);
      for (int k = 0; k < 2; ++k) c->m_tmp[k] = L.take<float>(sizeof(float) * n);
      c->p_saved = L.take<cx<double>>(S64);
      c->G64c = L.take<cx<double>>(2 * S64);
      c->partials_c = L.take<double>(sizeof(double) * hc::kPartialStride * max_reducing_ctas(c));
      c->st_c = L.take<hc::SolveState>(sizeof(hc::SolveState));
    }
  }
  c->twx_f = L.take<cx<float>>(sizeof(cx<float>) * c->nx);
  c->twy_f = L.take<cx<float>>(sizeof(cx<float>) * c->ny);
  c->twx_d = L.take<cx<double>>(sizeof(cx<double>) * c->nx);
  c->twy_d = L.take<cx<double>>(sizeof(cx<double>) * c->ny);
  c->kxd_f = L.take<float>(sizeof(float) * c->H);
  c->kyd_f = L.take<float>(sizeof(float) * c->ny);
  c->hx_f = L.take<float>(sizeof(float) * (c->H + 1));
  c->hy_f = L.take<float>(sizeof(float) * c->ny);
  c->kxd_d = L.take<double>(sizeof(double) * c->H);
  c->kyd_d = L.take<double>(sizeof(double) * c->ny);
  c->twx_q = L.take<cx<df64>>(sizeof(cx<df64>) * c->nx);
  c->twy_q = L.take<cx<df64>>(sizeof(cx<df64>) * c->ny);
  c->kxd_q = L.take<df64>(sizeof(df64) * c->H);
  c->kyd_q = L.take<df64>(sizeof(df64) * c->ny);
  c->x2x_f = L.take<float>(sizeof(float) * (c->H + 1));
  c->x2y_f = L.take<float>(sizeof(float) * c->ny);
  c->x2x_d = L.take<double>(sizeof(double) * (c->H + 1));
  c->x2y_d = L.take<double>(sizeof(double) * c->ny);
  c->hx_d = L.take<double>(sizeof(double) * (c->H + 1));
  c->hy_d = L.take<double>(sizeof(double) * c->ny);
  if (d == 3) {
    c->twz_f = L.take<cx<float>>(sizeof(cx<float>) * c->nz);
    c->twz_d = L.take<cx<double>>(sizeof(cx<double>) * c->nz);
    c->twz_q = L.take<cx<df64>>(sizeof(cx<df64>) * c->nz);
    c->kzd_f = L.take<float>(sizeof(float) * c->nz);
    c->kzd_d = L.take<double>(sizeof(double) * c->nz);
    c->kzd_q = L.take<df64>(sizeof(df64) * c->nz);
    c->hz_f = L.take<float>(sizeof(float) * c->nz);
    c->hz_d = L.take<double>(sizeof(double) * c->nz);
  }
}

int check_grid(const hc_grid* g) {
  if (!g || (g->dim != 2 && g->dim != 3)) return HC_EINVAL;
  if (g->dim == 2) {
    if (!is_235_in(g->n[0], 4, 4096) || !is_235_in(g->n[1], 4, 4096) || g->n[2] != 1)
      return HC_EINVAL;
  } else {
    if (!is_pow2_in(g->n[0], 8, 1024) || !is_pow2_in(g->n[1], 8, 1024) ||
        !is_pow2_in(g->n[2], 8, 1024))
      return HC_EINVAL;
    if ((size_t)g->n[0] * g->n[1] * g->n[2] > ((size_t)1 << 28)) return HC_EINVAL;
    if (!(g->L[2] > 0) || !std::isfinite(g->L[2])) return HC_EINVAL;
  }
  if (!(g->L[0] > 0) || !(g->L[1] > 0) || !std::isfinite(g->L[0]) || !std::isfinite(g->L[1]))
    return HC_EINVAL;
  return HC_OK;
}

int check_params(const hc_params* p) {
  if (!p) return HC_EINVAL;
  if (p->precision != HC_FP64_PLAIN && p->precision != HC_FP32_REFINED &&
      p->precision != HC_FP32_REFINED_DF)
    return HC_EINVAL;
  if (p->precond != HC_PRECOND_SCALAR && p->precond != HC_PRECOND_KBAR) return HC_EINVAL;
  if (!std::isfinite(p->c) || !std::isfinite(p->D) || !std::isfinite(p->gamma) ||
      !std::isfinite(p->dt) || p->dt < 0)
    return HC_EINVAL;
  return HC_OK;
}

template <typename T>
void fill_geo(hc_ctx* c, hc::Geo<T>& g, const cx<T>* twx, const cx<T>* twy, const T* kxd,
              const T* kyd, const T* hx, const T* hy) {
  g.nx = c->nx;
  g.ny = c->ny;
  g.H = c->H;
  g.lnx = ilog2(c->nx);
  g.lny = ilog2(c->ny);
  g.lH = ilog2(c->H);
  // column CTA: tc packed columns x ny/8 threads: 1024 threads (FP32), 256
  // (FP64, double-float: at 128 registers two CTAs per SM, the same warps as
  // one of 512 in finer pieces; measured at 2048^2, the FP64 gradient and
  // divergence passes take 674 us per step at 256 threads, 801 at 512)
  int tc = (sizeof(T) == 4 ? hc::col_cta_max<T, true>() : 256) >> (g.lny - 3);
  if (tc < 1) tc = 1;
  if (tc > 32) tc = 32;
  if (tc > c->H) tc = c->H;
  g.tc = tc;
  g.ltc = ilog2(tc);
  // row CTA: rpc rows x nx/8 threads, about 256 threads
  int rpc = 256 >> (g.lnx - 3);
  if (rpc < 1) rpc = 1;
  if (rpc > c->ny) rpc = c->ny;
  g.rpc = rpc;
  g.lrpc = ilog2(rpc);
  g.twx = twx;
  g.twy = twy;
  g.kxd = kxd;
  g.kyd = kyd;
  g.hx = hx;
  g.hy = hy;
  g.partials = c->partials;
  g.npartials = (int)max_reducing_ctas(c);
  g.nz = c->nz;
  g.lnz = ilog2(c->nz);
  g.twz = nullptr;
  g.kzd = nullptr;
  g.hz = nullptr;
  g.upc = g.lupc = 0;
  g.py = g.pz = hc::ColPass{};
}

// Tile of a 3D column pass of three fields: at most 256 threads (tc * L/8)
// and, where possible, at most ~113 KB of shared memory so two CTAs fit an SM.
hc::ColPass make_pass(int lL, long long cols, int nplanes, long long stride, long long pstride,
                      size_t elem) {
  const int L8 = 1 << (lL - 3);
  long long tc = std::max(1, 256 / L8);
  tc = std::min<long long>({tc, 32, cols});
  while (tc > 1 && 3 * 9 * (size_t)L8 * tc * elem > 113 * 1024) tc >>= 1;
  hc::ColPass p;
  p.lL = lL;
  p.ltc = ilog2((int)tc);
  p.lt = ilog2((int)(cols / tc));
  p.nplanes = nplanes;
  p.stride = stride;
  p.pstride = pstride;
  return p;
}

template <typename T>
void fill_geo3(hc_ctx* c, hc::Geo<T>& g, hc::Geo<T>& rows, const cx<T>* twz, const T* kzd,
               const T* hz) {
  const long long H = c->H, ny = c->ny;
  g.twz = twz;
  g.kzd = kzd;
  g.hz = hz;
  g.py = make_pass(g.lny, H, c->nz, H, ny * H, sizeof(cx<T>));
  g.pz = make_pass(g.lnz, ny * H, 1, ny * H, 0, sizeof(cx<T>));
  // row pairs: N/8 threads per pair, 256 threads per CTA
  int upc = std::max(1, 256 >> (g.lnx - 3));
  upc = std::min(upc, (int)((size_t)c->ny * c->nz / 2));
  g.upc = upc;
  g.lupc = ilog2(upc);
  rows = g;
  rows.ny = c->ny * c->nz;
  rows.lny = g.lny + g.lnz;
  int rpc = 256 >> (g.lnx - 3);
  if (rpc < 1) rpc = 1;
  if (rpc > rows.ny) rpc = rows.ny;
  rows.rpc = rpc;
  rows.lrpc = ilog2(rpc);
}

// Most recent CUDA failure seen by this library on the calling thread.
thread_local char g_last_error[256] = "";

int cuda_fail(cudaError_t e, const char* call, int line) {
  std::snprintf(g_last_error, sizeof(g_last_error), "hc_api.cu:%d %s -> %s (%s)", line, call,
                cudaGetErrorName(e), cudaGetErrorString(e));
  return HC_ECUDA;
}

#define CU(x)                                                   \
  do {                                                          \
    cudaError_t e_ = (x);                                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x, __LINE__);  \
  } while (0)

// ------------------------------------------------------------------ guard zones
#if HC_CHECK
__device__ unsigned int g_zone_bad[kMaxZones];  // damaged bytes per zone of one scan

struct ZoneScan {
  const unsigned char* base;
  int n;
  unsigned long long start[kMaxZones];
  unsigned int len[kMaxZones];
};

// One CTA per zone counts the bytes that no longer hold the pattern.
__global__ void __launch_bounds__(256) k_redzone_scan(ZoneScan z) {
  const int k = blockIdx.x;
  if (k >= z.n) return;
  const unsigned char* p = z.base + z.start[k];
  unsigned int bad = 0;
  for (unsigned int i = threadIdx.x; i < z.len[k]; i += blockDim.x) bad += p[i] != kPattern;
  if (bad) atomicAdd(&g_zone_bad[k], bad);
}

std::mutex g_zone_mu;  // g_zone_bad serves one scan at a time
#endif

// Writes the pattern into every zone of a workspace (nothing without zones).
int fill_zones(cudaStream_t s, char* base, const Zones& z) {
  for (int k = 0; k < z.n; ++k) CU(cudaMemsetAsync(base + z.start[k], kPattern, z.len[k], s));
  return HC_OK;
}

// Scans the zones of a workspace on stream s and waits for the result:
// HC_EBOUNDS with *bad = the first damaged zone, else HC_OK with *bad = -1.
int scan_zones(cudaStream_t s, const char* base, const Zones& z, int* bad) {
  *bad = -1;
#if HC_CHECK
  if (z.n == 0) return HC_OK;
  std::lock_guard<std::mutex> lock(g_zone_mu);
  void* dbad = nullptr;
  CU(cudaGetSymbolAddress(&dbad, g_zone_bad));
  CU(cudaMemsetAsync(dbad, 0, sizeof(unsigned int) * z.n, s));
  ZoneScan zs;
  zs.base = reinterpret_cast<const unsigned char*>(base);
  zs.n = z.n;
  for (int k = 0; k < z.n; ++k) {
    zs.start[k] = z.start[k];
    zs.len[k] = (unsigned int)z.len[k];
  }
  k_redzone_scan<<<z.n, 256, 0, s>>>(zs);
  CU(cudaGetLastError());
  unsigned int hbad[kMaxZones];
  CU(cudaMemcpyAsync(hbad, dbad, sizeof(unsigned int) * z.n, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  for (int k = 0; k < z.n; ++k)
    if (hbad[k]) {
      *bad = k;
      return HC_EBOUNDS;
    }
#else
  (void)s;
  (void)base;
  (void)z;
#endif
  return HC_OK;
}

// Tables of the generic path: twiddles of both lengths, first-derivative
// multipliers (Nyquist entry 0, reading R1) of the Hh = nx/2 + 1 columns and
// the ny rows.
int upload_tables_generic(hc_ctx* c) {
  std::vector<double> re, im;
  auto put_tw = [&](int N, cx<double>* dd) -> int {
    twiddles(N, re, im);
    std::vector<cx<double>> hd(N);
    for (int m = 0; m < N; ++m) {
      hd[m].x = re[m];
      hd[m].y = im[m];
    }
    CU(cudaMemcpy(dd, hd.data(), sizeof(cx<double>) * N, cudaMemcpyHostToDevice));
    return HC_OK;
  };
  int rc = put_tw(c->nx, c->twx_d);
  if (!rc) rc = put_tw(c->ny, c->twy_d);
  if (rc) return rc;
  std::vector<double> kx(c->H), ky(c->ny);
  for (int k = 0; k < c->H; ++k) kx[k] = xid(k, c->nx, c->grid.L[0]);
  for (int k = 0; k < c->ny; ++k) ky[k] = xid(k, c->ny, c->grid.L[1]);
  CU(cudaMemcpy(c->kxd_d, kx.data(), sizeof(double) * c->H, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->kyd_d, ky.data(), sizeof(double) * c->ny, cudaMemcpyHostToDevice));
  return HC_OK;
}

void fill_generic_geo(hc_ctx* c) {
  hc::GenGeo& g = c->gg;
  g = hc::GenGeo{};
  g.nx = c->nx;
  g.ny = c->ny;
  g.Hh = c->H;
  g.nrx = radices(c->nx, g.rx);
  g.nry = radices(c->ny, g.ry);
  g.twx = c->twx_d;
  g.twy = c->twy_d;
  g.kxd = c->kxd_d;
  g.kyd = c->kyd_d;
  g.hx = c->hx_d;
  g.hy = c->hy_d;
  g.partials = c->partials;
  // the grid-wide sums (hc::msum) take only nx, ny and the partials
  c->gd = hc::Geo<double>{};
  c->gd.nx = c->nx;
  c->gd.ny = c->ny;
  c->gd.partials = c->partials;
  c->gd.npartials = (int)max_reducing_ctas(c);
}

int upload_tables(hc_ctx* c) {
  if (c->gen) return upload_tables_generic(c);
  std::vector<double> re, im;
  auto put_tw = [&](int N, cx<float>* df, cx<double>* dd, cx<df64>* dq) -> int {
    twiddles(N, re, im);
    std::vector<cx<float>> hf(N);
    std::vector<cx<double>> hd(N);
    std::vector<cx<df64>> hq(N);
    for (int m = 0; m < N; ++m) {
      hf[m].x = (float)re[m];
      hf[m].y = (float)im[m];
      hd[m].x = re[m];
      hd[m].y = im[m];
      hq[m].x = df64(re[m]);
      hq[m].y = df64(im[m]);
    }
    CU(cudaMemcpy(df, hf.data(), sizeof(cx<float>) * N, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dd, hd.data(), sizeof(cx<double>) * N, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(dq, hq.data(), sizeof(cx<df64>) * N, cudaMemcpyHostToDevice));
    return HC_OK;
  };
  int rc = put_tw(c->nx, c->twx_f, c->twx_d, c->twx_q);
  if (rc) return rc;
  rc = put_tw(c->ny, c->twy_f, c->twy_d, c->twy_q);
  if (rc) return rc;
  std::vector<double> kx(c->H), ky(c->ny);
  for (int k = 0; k < c->H; ++k) kx[k] = (k == 0) ? 0.0 : xid(k, c->nx, c->grid.L[0]);
  for (int k = 0; k < c->ny; ++k) ky[k] = xid(k, c->ny, c->grid.L[1]);
  std::vector<float> kxf(kx.begin(), kx.end()), kyf(ky.begin(), ky.end());
  CU(cudaMemcpy(c->kxd_d, kx.data(), sizeof(double) * c->H, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->kyd_d, ky.data(), sizeof(double) * c->ny, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->kxd_f, kxf.data(), sizeof(float) * c->H, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->kyd_f, kyf.data(), sizeof(float) * c->ny, cudaMemcpyHostToDevice));
  std::vector<double> x2x(c->H + 1), x2y(c->ny);
  for (int k = 0; k <= c->H; ++k) x2x[k] = xi(k, c->nx, c->grid.L[0]) * xi(k, c->nx, c->grid.L[0]);
  for (int k = 0; k < c->ny; ++k) x2y[k] = xi(k, c->ny, c->grid.L[1]) * xi(k, c->ny, c->grid.L[1]);
  std::vector<float> x2xf(x2x.begin(), x2x.end()), x2yf(x2y.begin(), x2y.end());
  CU(cudaMemcpy(c->x2x_d, x2x.data(), sizeof(double) * (c->H + 1), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->x2y_d, x2y.data(), sizeof(double) * c->ny, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->x2x_f, x2xf.data(), sizeof(float) * (c->H + 1), cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->x2y_f, x2yf.data(), sizeof(float) * c->ny, cudaMemcpyHostToDevice));
  std::vector<df64> kxq(kx.begin(), kx.end()), kyq(ky.begin(), ky.end());
  CU(cudaMemcpy(c->kxd_q, kxq.data(), sizeof(df64) * c->H, cudaMemcpyHostToDevice));
  CU(cudaMemcpy(c->kyd_q, kyq.data(), sizeof(df64) * c->ny, cudaMemcpyHostToDevice));
  if (c->dim == 3) {
    rc = put_tw(c->nz, c->twz_f, c->twz_d, c->twz_q);
    if (rc) return rc;
    std::vector<double> kz(c->nz);
    for (int k = 0; k < c->nz; ++k) kz[k] = xid(k, c->nz, c->grid.L[2]);
    std::vector<float> kzf(kz.begin(), kz.end());
    std::vector<df64> kzq(kz.begin(), kz.end());
    CU(cudaMemcpy(c->kzd_d, kz.data(), sizeof(double) * c->nz, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->kzd_f, kzf.data(), sizeof(float) * c->nz, cudaMemcpyHostToDevice));
    CU(cudaMemcpy(c->kzd_q, kzq.data(), sizeof(df64) * c->nz, cudaMemcpyHostToDevice));
  }
  return HC_OK;
}

// Heat factors exp(-D^2 xi^2 dt) per axis (eq. diffusion_space_discrete); the
// 2D factor is their product.
int upload_heat(hc_ctx* c) {
  const double D2dt = c->prm.D * c->prm.D * c->prm.dt;
  if (c->gen) {  // FP64 only, kx = 0 .. nx/2 (H entries)
    std::vector<double> hx(c->H), hy(c->ny);
    for (int k = 0; k < c->H; ++k) {
      const double x = xi(k, c->nx, c->grid.L[0]);
      hx[k] = std::exp(-D2dt * x * x);
    }
    for (int k = 0; k < c->ny; ++k) {
      const double y = xi(k, c->ny, c->grid.L[1]);
      hy[k] = std::exp(-D2dt * y * y);
    }
    CU(cudaMemcpyAsync(c->hx_d, hx.data(), sizeof(double) * c->H, cudaMemcpyHostToDevice,
                       c->stream));
    CU(cudaMemcpyAsync(c->hy_d, hy.data(), sizeof(double) * c->ny, cudaMemcpyHostToDevice,
                       c->stream));
    CU(cudaStreamSynchronize(c->stream));  // host vectors die here
    return HC_OK;
  }
  std::vector<double> hx(c->H + 1), hy(c->ny);
  for (int k = 0; k <= c->H; ++k) {
    const double x = xi(k, c->nx, c->grid.L[0]);
    hx[k] = std::exp(-D2dt * x * x);
  }
  for (int k = 0; k < c->ny; ++k) {
    const double y = xi(k, c->ny, c->grid.L[1]);
    hy[k] = std::exp(-D2dt * y * y);
  }
  std::vector<float> hxf(hx.begin(), hx.end()), hyf(hy.begin(), hy.end());
  CU(cudaMemcpyAsync(c->hx_d, hx.data(), sizeof(double) * (c->H + 1), cudaMemcpyHostToDevice,
                     c->stream));
  CU(cudaMemcpyAsync(c->hy_d, hy.data(), sizeof(double) * c->ny, cudaMemcpyHostToDevice, c->stream));
  CU(cudaMemcpyAsync(c->hx_f, hxf.data(), sizeof(float) * (c->H + 1), cudaMemcpyHostToDevice,
                     c->stream));
  CU(cudaMemcpyAsync(c->hy_f, hyf.data(), sizeof(float) * c->ny, cudaMemcpyHostToDevice, c->stream));
  std::vector<double> hz;
  std::vector<float> hzf;
  if (c->dim == 3) {
    hz.resize(c->nz);
    for (int k = 0; k < c->nz; ++k) {
      const double z = xi(k, c->nz, c->grid.L[2]);
      hz[k] = std::exp(-D2dt * z * z);
    }
    hzf.assign(hz.begin(), hz.end());
    CU(cudaMemcpyAsync(c->hz_d, hz.data(), sizeof(double) * c->nz, cudaMemcpyHostToDevice,
                       c->stream));
    CU(cudaMemcpyAsync(c->hz_f, hzf.data(), sizeof(float) * c->nz, cudaMemcpyHostToDevice,
                       c->stream));
  }
  CU(cudaStreamSynchronize(c->stream));  // host vectors die here
  return HC_OK;
}

hc::SplitCoef split_coef(const hc_params& p) {
  hc::SplitCoef s;
  s.c2dt = p.c * p.c * p.dt;
  s.gamma = p.gamma;
  s.dt = p.dt;
  s.exp_mdt = std::exp(-p.dt);
  s.gamma_is_one = (p.gamma == 1.0) ? 1 : 0;
  s.two1mg_dt = 2.0 * (1.0 - p.gamma) * p.dt;
  s.pow_a = 2.0 * (1.0 - p.gamma);
  s.pow_b = s.gamma_is_one ? 0.0 : 1.0 / (2.0 * (1.0 - p.gamma));
  s.f_c2dt = (float)s.c2dt;
  s.f_gamma = (float)s.gamma;
  s.f_dt = (float)s.dt;
  s.f_exp_mdt = (float)s.exp_mdt;
  s.f_two1mg_dt = (float)s.two1mg_dt;
  s.f_pow_a = (float)s.pow_a;
  s.f_pow_b = (float)s.pow_b;
  auto kind = [](double e) { return e == 1.0 ? 1 : e == 2.0 ? 2 : e == 0.5 ? 3 : 0; };
  s.pow_a_kind = kind(s.pow_a);
  s.pow_b_kind = s.gamma_is_one ? 0 : kind(s.pow_b);
  return s;
}

void apply_defaults(hc_params& p) {
  if (!(p.cg_rtol > 0)) p.cg_rtol = 1e-7;
  if (p.cg_maxit <= 0) p.cg_maxit = 1000;
  if (!(p.inner_rtol > 0)) p.inner_rtol = 1e-4;
  if (p.max_sweeps <= 0) p.max_sweeps = 10;
}

// HC_FP32_REFINED evaluates the residual after an FP32 first sweep in
// double-float unless either switch asks for FP64 there.
int mid_df_on(const hc_ctx* c) {
  return (c->refined && !c->df && !c->prm.fp64_first_residual && !c->prm.fp64_mid_residual) ? 1 : 0;
}

bool diag_on(const hc_ctx* c) { return c->prm.diagnostics != 0 || c->force_diag != 0; }

int push_config(hc_ctx* c) {
  hc::SolveConfig cfg;
  double h = 1.0;
  for (int a = 0; a < c->dim; ++a) h *= c->grid.L[a] / (double)c->grid.n[a];
  cfg.e_coef[0] = h * c->prm.D * c->prm.D / 2.0;
  cfg.e_coef[1] = h * c->prm.c * c->prm.c / 2.0;
  // gamma = 0: the split step sums ln|m| in place of |m|^(2 gamma)
  cfg.e_coef[2] = c->prm.gamma != 0.0 ? h / (2.0 * c->prm.gamma) : h;
  cfg.dt = c->prm.dt;
  // refined: FP32 first sweep when the warm start is off by more than 1e-5 ||S||
  cfg.first32_min2 = (c->refined && !c->prm.fp64_first_residual) ? 1e-10 : 0.0;
  cfg.mid_df = c->mid_df;
  cfg.precond = c->prm.precond == HC_PRECOND_KBAR ? HC_PRECOND_KBAR : HC_PRECOND_SCALAR;
  cfg.dim = c->dim;
  cfg.diag = diag_on(c) ? 1 : 0;
  cfg.outer_thresh2_rel = c->prm.cg_rtol * c->prm.cg_rtol;
  cfg.inner_rtol2 = c->prm.inner_rtol * c->prm.inner_rtol;
  cfg.user_kappa = c->prm.kappa > 0 ? c->prm.kappa : 0.0;
  cfg.mean_r = c->mean_r;
  cfg.maxit = c->prm.cg_maxit;
  cfg.max_sweeps = c->prm.max_sweeps;
  cfg.graph_mode = 0;  // set true only while a graph runs
  cfg.refined = c->refined;
  hc::set_config(c->st, cfg, c->stream);
  c->launches += 1;
  CU(cudaGetLastError());
  return HC_OK;
}

// ---------------------------------------------------------------- step pieces
template <typename T>
hc::Tri<cx<T>*> tri(cx<T>* G, size_t ns) {
  return hc::Tri<cx<T>*>{{G, G + ns, G + 2 * ns}};
}
template <typename T>
hc::Tri<const T*> mtri(hc_ctx* c) {
  return hc::Tri<const T*>{{(const T*)c->m[0], (const T*)c->m[1], (const T*)c->m[2]}};
}
template <typename T>
hc::Tri<T*> mtri_w(hc_ctx* c) {
  return hc::Tri<T*>{{(T*)c->m[0], (T*)c->m[1], (T*)c->m[2]}};
}

// 3D operator apply on the spectral direction/iterate: z gradient pass (mode),
// inverse y, row apply, forward y; the caller's z_div closes it.
template <typename T, typename Tin, typename Tm>
void apply3_open(hc_ctx* c, hc::Geo<T>& g, int mode, cx<Tin>* in, const cx<T>* rvec, cx<T>* dio,
                 cx<T>* G, int check_done) {
  auto Gt = tri(G, c->ns);
  hc::z_grad<T, Tin>(g, mode, in, rvec, dio, c->x32, Gt, c->st, check_done, c->stream);
  hc::axis_fft<T>(g, 1, +1, 3, Gt, Gt, (T)1, c->stream);
  hc::row_apply3<T, Tm>(g, Gt, mtri<Tm>(c), (const Tm*)c->rf, Gt, check_done ? c->st : nullptr,
                        c->stream);
  hc::axis_fft<T>(g, 1, -1, 3, Gt, Gt, (T)1, c->stream);
  c->launches += 4;
}

// r = b - A x0 in FP64 plain mode; initialises the CG state.
void plain_init(hc_ctx* c) {
  if (c->gen) {
    cx<double>* Gx = c->G64;
    cx<double>* Gy = c->G64 + c->ns;
    hc::gen_col_grad(c->gg, hc::CG_PLAIN, c->p64, nullptr, nullptr, Gx, Gy, c->st, 0, c->stream);
    hc::gen_row_apply(c->gg, Gx, Gy, (const double*)c->m[0], (const double*)c->m[1],
                      (const double*)c->rf, Gx, Gy, nullptr, c->stream);
    hc::gen_col_div(c->gg, hc::CD_RESID, Gx, Gy, c->b64, c->r64, c->st, c->stream);
    c->launches += 3;
    return;
  }
  if (c->dim == 3) {
    apply3_open<double, double, double>(c, c->gd, hc::CG_PLAIN, c->p64, nullptr, nullptr, c->G64, 0);
    hc::z_div<double>(c->gd, hc::CD_RESID, tri(c->G64, c->ns), nullptr, c->b64, c->r64, nullptr,
                      nullptr, c->st, c->stream);
    c->launches += 1;
    return;
  }
  auto& g = c->gd;
  cx<double>* Gx = c->G64;
  cx<double>* Gy = c->G64 + (size_t)c->ny * c->H;
  hc::col_grad<double, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gx, Gy, c->st, 0,
                               c->stream);
  hc::row_apply<double, double>(g, Gx, Gy, (const double*)c->m[0], (const double*)c->m[1],
                                (const double*)c->rf, Gx, Gy, nullptr, c->stream);
  hc::col_div<double>(g, hc::CD_RESID, Gx, Gy, nullptr, c->b64, c->r64, nullptr, nullptr, c->st,
                      c->stream);
  c->launches += 3;
}

void plain_iter(hc_ctx* c) {
  if (c->gen) {
    cx<double>* Gx = c->G64;
    cx<double>* Gy = c->G64 + c->ns;
    hc::gen_col_grad(c->gg, hc::CG_DUPDATE, nullptr, c->r64, c->d64, Gx, Gy, c->st, 1, c->stream);
    hc::gen_row_apply(c->gg, Gx, Gy, (const double*)c->m[0], (const double*)c->m[1],
                      (const double*)c->rf, Gx, Gy, c->st, c->stream);
    hc::gen_col_div(c->gg, hc::CD_CG, Gx, Gy, nullptr, c->q64, c->st, c->stream);
    hc::gen_cg_update(c->gg, c->p64, c->r64, c->d64, c->q64, c->st, c->stream);
    c->launches += 4;
    return;
  }
  if (c->dim == 3) {
    apply3_open<double, double, double>(c, c->gd, hc::CG_DUPDATE, (cx<double>*)nullptr, c->r64,
                                        c->d64, c->G64, 1);
    hc::z_div<double>(c->gd, hc::CD_CG, tri(c->G64, c->ns), c->d64, nullptr, c->q64, nullptr,
                      nullptr, c->st, c->stream);
    hc::cg_update3<double>(c->gd, c->p64, c->r64, c->d64, c->q64, c->st, c->stream);
    c->launches += 2;
    return;
  }
  auto& g = c->gd;
  cx<double>* Gx = c->G64;
  cx<double>* Gy = c->G64 + (size_t)c->ny * c->H;
  hc::col_grad<double, double>(g, hc::CG_DUPDATE, (cx<double>*)nullptr, c->r64, c->d64, nullptr, Gx,
                               Gy, c->st, 1, c->stream);
  hc::row_apply<double, double>(g, Gx, Gy, (const double*)c->m[0], (const double*)c->m[1],
                                (const double*)c->rf, Gx, Gy, c->st, c->stream);
  hc::col_div<double>(g, hc::CD_CG, Gx, Gy, c->d64, nullptr, c->q64, nullptr, nullptr, c->st,
                      c->stream);
  hc::cg_update<double>(g, c->p64, c->r64, c->d64, c->q64, c->st, c->stream);
  c->launches += 4;
}

// Refined modes: S - A p^k in FP32 from the warm start, the first inner
// solve's right-hand side (resid_first_init decides whether it is used).
void first_resid32(hc_ctx* c) {
  auto& g = c->gf;
  if (c->dim == 3) {
    auto Gt = tri(c->G32, c->ns);
    if (c->df)
      hc::z_grad<float, df64>(g, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64), nullptr, nullptr,
                              nullptr, Gt, c->st, 0, c->stream);
    else
      hc::z_grad<float, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gt, c->st, 0,
                                c->stream);
    hc::axis_fft<float>(g, 1, +1, 3, Gt, Gt, 1.0f, c->stream);
    hc::row_apply3<float, float>(g, Gt, mtri<float>(c), (const float*)c->rf, Gt, nullptr, c->stream);
    hc::axis_fft<float>(g, 1, -1, 3, Gt, Gt, 1.0f, c->stream);
    hc::z_div<float>(g, hc::CD_RESID_FIRST, Gt, nullptr, c->b32, nullptr, c->r32, c->x32, c->st,
                     c->stream);
    c->launches += 5;
    return;
  }
  cx<float>* Gx = c->G32;
  cx<float>* Gy = c->G32 + c->ns;
  if (c->df)
    hc::col_grad<float, df64>(g, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64), nullptr, nullptr,
                              nullptr, Gx, Gy, c->st, 0, c->stream);
  else
    hc::col_grad<float, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gx, Gy, c->st, 0,
                                c->stream);
  hc::row_apply<float, float>(g, Gx, Gy, (const float*)c->m[0], (const float*)c->m[1],
                              (const float*)c->rf, Gx, Gy, nullptr, c->stream);
  hc::col_div<float>(g, hc::CD_RESID_FIRST, Gx, Gy, nullptr, c->b32, nullptr, c->r32, c->x32, c->st,
                     c->stream);
  c->launches += 3;
}

// FP64 residual S - A p64 (after p64 += delta) and inner-CG initialisation.
void refined_resid(hc_ctx* c) {
  if (c->dim == 3) {
    if (c->df) {
      auto* G = reinterpret_cast<cx<df64>*>(c->G64);
      apply3_open<df64, df64, float>(c, c->gq, hc::CG_ADDDELTA, reinterpret_cast<cx<df64>*>(c->p64),
                                     nullptr, nullptr, G, 0);
      hc::z_div<df64>(c->gq, hc::CD_RESID_REFINE, tri(G, c->ns), nullptr,
                      reinterpret_cast<const cx<df64>*>(c->b64), reinterpret_cast<cx<df64>*>(c->r64),
                      c->r32, c->x32, c->st, c->stream);
    } else {
      apply3_open<double, double, float>(c, c->gd, hc::CG_ADDDELTA, c->p64, nullptr, nullptr,
                                         c->G64, 0);
      hc::z_div<double>(c->gd, hc::CD_RESID_REFINE, tri(c->G64, c->ns), nullptr, c->b64, c->r64,
                        c->r32, c->x32, c->st, c->stream);
    }
    c->launches += 1;
    return;
  }
  if (c->df) {
    auto& q = c->gq;
    cx<df64>* Gx = reinterpret_cast<cx<df64>*>(c->G64);
    cx<df64>* Gy = Gx + (size_t)c->ny * c->H;
    hc::col_grad<df64, df64>(q, hc::CG_ADDDELTA, reinterpret_cast<cx<df64>*>(c->p64), nullptr,
                             nullptr, c->x32, Gx, Gy, c->st, 0, c->stream);
    hc::row_apply<df64, float>(q, Gx, Gy, (const float*)c->m[0], (const float*)c->m[1],
                               (const float*)c->rf, Gx, Gy, nullptr, c->stream);
    hc::col_div<df64>(q, hc::CD_RESID_REFINE, Gx, Gy, nullptr,
                      reinterpret_cast<const cx<df64>*>(c->b64),
                      reinterpret_cast<cx<df64>*>(c->r64), c->r32, c->x32, c->st, c->stream);
    c->launches += 3;
    return;
  }
  auto& g = c->gd;
  cx<double>* Gx = c->G64;
  cx<double>* Gy = c->G64 + (size_t)c->ny * c->H;
  hc::col_grad<double, double>(g, hc::CG_ADDDELTA, c->p64, nullptr, nullptr, c->x32, Gx, Gy, c->st,
                               0, c->stream);
  hc::row_apply<double, float>(g, Gx, Gy, (const float*)c->m[0], (const float*)c->m[1],
                               (const float*)c->rf, Gx, Gy, nullptr, c->stream);
  hc::col_div<double>(g, hc::CD_RESID_REFINE, Gx, Gy, nullptr, c->b64, c->r64, c->r32, c->x32,
                      c->st, c->stream);
  c->launches += 3;
}

// HC_FP32_REFINED, after an FP32 first sweep: p64 += delta (FP64), then
// S - A p64 in double-float, the second inner solve's right-hand side
// (resid_mid_init); the same kernels as the double-float mode's residual,
// reading and updating the FP64 spectrum.  r64 is not written.
void mid_resid(hc_ctx* c) {
  auto& q = c->gq;
  if (c->dim == 3) {
    auto* G = reinterpret_cast<cx<df64>*>(c->G64);
    apply3_open<df64, double, float>(c, q, hc::CG_ADDDELTA, c->p64, nullptr, nullptr, G, 0);
    hc::z_div<df64>(q, hc::CD_RESID_REFINE, tri(G, c->ns), nullptr, c->bq, nullptr, c->r32, c->x32,
                    c->st, c->stream);
    c->launches += 1;
    return;
  }
  cx<df64>* Gx = reinterpret_cast<cx<df64>*>(c->G64);
  cx<df64>* Gy = Gx + (size_t)c->ny * c->H;
  hc::col_grad<df64, double>(q, hc::CG_ADDDELTA, c->p64, nullptr, nullptr, c->x32, Gx, Gy, c->st, 0,
                             c->stream);
  hc::row_apply<df64, float>(q, Gx, Gy, (const float*)c->m[0], (const float*)c->m[1],
                             (const float*)c->rf, Gx, Gy, nullptr, c->stream);
  hc::col_div<df64>(q, hc::CD_RESID_REFINE, Gx, Gy, nullptr, c->bq, nullptr, c->r32, c->x32, c->st,
                    c->stream);
  c->launches += 3;
}

void refined_iter(hc_ctx* c) {
  if (c->dim == 3) {
    apply3_open<float, float, float>(c, c->gf, hc::CG_DUPDATE, (cx<float>*)nullptr, c->r32, c->d32,
                                     c->G32, 1);
    hc::z_div<float>(c->gf, hc::CD_CG, tri(c->G32, c->ns), c->d32, nullptr, c->q32, nullptr,
                     nullptr, c->st, c->stream);
    hc::cg_update3<float>(c->gf, c->x32, c->r32, c->d32, c->q32, c->st, c->stream);
    c->launches += 2;
    return;
  }
  auto& g = c->gf;
  cx<float>* Gx = c->G32;
  cx<float>* Gy = c->G32 + (size_t)c->ny * c->H;
  // r32, d32, q32 and x32 are column-major
  hc::col_grad<float, float>(g, hc::CG_DUPDATE, (cx<float>*)nullptr, c->r32, c->d32, nullptr, Gx,
                             Gy, c->st, 1, c->stream);
  hc::row_apply<float, float>(g, Gx, Gy, (const float*)c->m[0], (const float*)c->m[1],
                              (const float*)c->rf, Gx, Gy, c->st, c->stream);
  hc::col_div<float>(g, hc::CD_CG, Gx, Gy, c->d32, nullptr, c->q32, nullptr, nullptr, c->st,
                     c->stream);
  hc::cg_update<float>(g, c->x32, c->r32, c->d32, c->q32, c->st, c->stream);
  c->launches += 4;
}

// Step 2 of Algorithm 1: gradient of the new p, activation + relaxation,
// diffusion, back to physical m (and sum |m|^2 for the next kappa).
template <typename T>
void split_step_t(hc_ctx* c, hc::Geo<T>& g, cx<T>* G) {
  cx<T>* Gx = G;
  cx<T>* Gy = G + (size_t)c->ny * c->H;
  if constexpr (std::is_same<T, float>::value) {
    if (c->df)
      hc::col_grad<float, df64>(g, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64), nullptr,
                                nullptr, nullptr, Gx, Gy, c->st, 0, c->stream);
    else
      hc::col_grad<float, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gx, Gy,
                                  c->st, 0, c->stream);
  } else {
    hc::col_grad<T, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gx, Gy, c->st, 0,
                            c->stream);
  }
  hc::row_split<T>(g, Gx, Gy, (const T*)c->m[0], (const T*)c->m[1], (const T*)c->rf, Gx, Gy,
                   split_coef(c->prm), c->st, c->stream);
  hc::col_heat<T>(g, Gx, Gy, c->st, c->stream);
  hc::row_c2r<T>(g, Gx, Gy, (T*)c->m[0], (T*)c->m[1], c->st, 1, c->stream);
  c->launches += 4;
}

// A f in 3D (forward transform with projection, apply, inverse transform).
template <typename T, typename Tm>
void apply_operator3(hc_ctx* c, hc::Geo<T>& g, hc::Geo<T>& rows, T* phys, cx<T>* G, cx<T>* dvec,
                     cx<T>* qvec) {
  auto Gt = tri(G, c->ns);
  hc::row_r2c<T>(rows, phys, nullptr, G, nullptr, c->stream);
  hc::axis_fft<T>(g, 1, -1, 1, Gt, Gt, (T)1, c->stream);
  hc::z_fwd_project<T>(g, G, dvec, nullptr, c->stream);
  apply3_open<T, T, Tm>(c, g, hc::CG_PLAIN, dvec, nullptr, nullptr, G, 0);
  hc::z_div<T>(g, hc::CD_PLAIN, Gt, nullptr, nullptr, qvec, nullptr, nullptr, nullptr, c->stream);
  hc::axis_fft<T>(g, 2, +1, 1, tri(qvec, c->ns), Gt, (T)(1.0 / (double)c->n), c->stream);
  hc::axis_fft<T>(g, 1, +1, 1, Gt, Gt, (T)1, c->stream);
  hc::row_c2r<T>(rows, G, nullptr, phys, nullptr, nullptr, 0, c->stream);
  c->launches += 7;
}

// The row view (ny*nz rows of length nx) of a 3D grid, per precision.
template <typename T>
hc::Geo<T>& rows_of(hc_ctx* c);
template <>
hc::Geo<float>& rows_of<float>(hc_ctx* c) { return c->rowf; }
template <>
hc::Geo<double>& rows_of<double>(hc_ctx* c) { return c->rowd; }

// sum |grad m|^2 of the current m (3D): x rows, y pass, z pass with the sum.
template <typename T>
void gradnorm3(hc_ctx* c, hc::Geo<T>& g, cx<T>* G, int into_next) {
  hc::Geo<T>& rows = rows_of<T>(c);
  auto Gt = tri(G, c->ns);
  hc::row_r2c<T>(rows, (const T*)c->m[0], (const T*)c->m[1], Gt.v[0], Gt.v[1], c->stream);
  hc::row_r2c<T>(rows, (const T*)c->m[2], nullptr, Gt.v[2], nullptr, c->stream);
  hc::axis_fft<T>(g, 1, -1, 3, Gt, Gt, (T)1, c->stream);
  hc::z_gradnorm<T>(g, Gt, c->st, into_next, c->stream);
  c->launches += 4;
}

// sum |grad m|^2 of the current m into st->gm2 (after hc_set_m).
void gradnorm_current(hc_ctx* c) {
  if (c->gen) {
    hc::gen_row_fwd(c->gg, (const double*)c->m[0], (const double*)c->m[1], c->G64,
                    c->G64 + c->ns, c->stream);
    hc::gen_col_fwd(c->gg, c->G64, c->G64 + c->ns, nullptr, nullptr, 0, 1, c->st, c->stream);
    c->launches += 2;
    return;
  }
  if (c->dim == 3) {
    if (c->refined)
      gradnorm3<float>(c, c->gf, c->G32, 0);
    else
      gradnorm3<double>(c, c->gd, c->G64, 0);
    return;
  }
  if (c->refined) {
    cx<float>* Gx = c->G32;
    cx<float>* Gy = c->G32 + c->ns;
    hc::row_r2c<float>(c->gf, (const float*)c->m[0], (const float*)c->m[1], Gx, Gy, c->stream);
    hc::col_gradnorm<float>(c->gf, Gx, Gy, c->st, 0, c->stream);
  } else {
    cx<double>* Gx = c->G64;
    cx<double>* Gy = c->G64 + c->ns;
    hc::row_r2c<double>(c->gd, (const double*)c->m[0], (const double*)c->m[1], Gx, Gy, c->stream);
    hc::col_gradnorm<double>(c->gd, Gx, Gy, c->st, 0, c->stream);
  }
  c->launches += 2;
}

// 3D: gradient of the new p (z pass from the FP64 spectrum, inverse y), the
// row pass (C2R, activation, relaxation, diffusion along x, back to physical
// m), diffusion along y, diffusion along z with sum |m|^2.
template <typename T>
void split_step3(hc_ctx* c, hc::Geo<T>& g, cx<T>* G) {
  auto Gt = tri(G, c->ns);
  if constexpr (std::is_same<T, float>::value) {
    if (c->df)
      hc::z_grad<float, df64>(g, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64), nullptr,
                              nullptr, nullptr, Gt, c->st, 0, c->stream);
    else
      hc::z_grad<float, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gt, c->st, 0,
                                c->stream);
  } else {
    hc::z_grad<T, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gt, c->st, 0,
                          c->stream);
  }
  hc::axis_fft<T>(g, 1, +1, 3, Gt, Gt, (T)1, c->stream);
  // the new m goes to the rows of G first, so the z pass still sees m^k (Delta m)
  hc::Tri<T*> tmp = {{reinterpret_cast<T*>(Gt.v[0]), reinterpret_cast<T*>(Gt.v[1]),
                      reinterpret_cast<T*>(Gt.v[2])}};
  hc::row_split3<T>(g, Gt, mtri<T>(c), (const T*)c->rf, tmp, split_coef(c->prm), c->st, c->stream);
  hc::heat_axis<T>(g, 1, tmp, tmp, c->st, c->stream);
  hc::heat_axis<T>(g, 2, tmp, mtri_w<T>(c), c->st, c->stream);
  c->launches += 5;
  if (diag_on(c)) gradnorm3<T>(c, g, G, 1);
}

void split_step(hc_ctx* c) {
  if (c->gen) {
    cx<double>* Gx = c->G64;
    cx<double>* Gy = c->G64 + c->ns;
    hc::gen_col_grad(c->gg, hc::CG_PLAIN, c->p64, nullptr, nullptr, Gx, Gy, c->st, 0, c->stream);
    hc::gen_row_split(c->gg, Gx, Gy, (const double*)c->m[0], (const double*)c->m[1],
                      (const double*)c->rf, split_coef(c->prm), c->st, c->stream);
    hc::gen_col_heat(c->gg, Gx, Gy, c->st, c->stream);
    hc::gen_row_c2r(c->gg, Gx, Gy, (double*)c->m[0], (double*)c->m[1], c->st, 1, c->stream);
    c->launches += 4;
    return;
  }
  if (c->dim == 3) {
    if (c->refined)
      split_step3<float>(c, c->gf, c->G32);
    else
      split_step3<double>(c, c->gd, c->G64);
    return;
  }
  if (c->refined)
    split_step_t<float>(c, c->gf, c->G32);
  else
    split_step_t<double>(c, c->gd, c->G64);
}

int read_state(hc_ctx* c) {
  CU(cudaMemcpyAsync(c->st_host, c->st, sizeof(hc::SolveState), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

// Launch CG iterations in chunks until the device says done.
int run_cg_host(hc_ctx* c, bool refined_inner) {
  for (int guard = 0; guard < 1000000; guard += kChunk) {
    for (int k = 0; k < kChunk; ++k) {
      if (refined_inner)
        refined_iter(c);
      else
        plain_iter(c);
    }
    CU(cudaGetLastError());
    int rc = read_state(c);
    if (rc) return rc;
    if (c->st_host->done) return HC_OK;
  }
  return HC_ETIMEOUT;
}

int step_host(hc_ctx* c) {
  hc::step_begin(c->st, (int)c->n, c->stream);
  c->launches += 1;
  if (!c->refined) {
    plain_init(c);
    int rc = run_cg_host(c, false);
    if (rc) return rc;
  } else {
    first_resid32(c);
    int rc = read_state(c);
    if (rc) return rc;
    if (!c->st_host->done) {
      rc = run_cg_host(c, true);
      if (rc) return rc;
    }
    if (c->st_host->mid_phase) {
      mid_resid(c);
      rc = read_state(c);
      if (rc) return rc;
      if (!c->st_host->done) {
        rc = run_cg_host(c, true);
        if (rc) return rc;
      }
    }
    for (int sweep = 0;; ++sweep) {
      refined_resid(c);
      rc = read_state(c);
      if (rc) return rc;
      if (c->st_host->outer_done) break;
      rc = run_cg_host(c, true);
      if (rc) return rc;
      if (sweep > 1000) return HC_ETIMEOUT;
    }
  }
  split_step(c);
  hc::step_end(c->st, c->refined, c->stream);
  c->launches += 1;
  CU(cudaGetLastError());
  return HC_OK;
}

// ---------------------------------------------------------------- graph mode
// One graph per context: step_begin, [plain: init residual, WHILE(cg) body]
// or [refined: WHILE(outer){ residual, WHILE(inner) body }], split step,
// step_end.  Loop conditions are set by the kernels (cudaGraphSetConditional)
// and default to 0 at every launch, so a loop whose controlling kernel did not
// run is skipped rather than repeated: step_begin opens the refinement loop,
// the residual kernels open the CG loop, cg_update keeps it open while the
// iteration cap and tolerance allow.
// Capture the step of context c into `target` as a chain with no dependencies
// on what `target` already holds: the prefix kernels, the loop node(s), the
// suffix kernels.  Returns the chain's conditional handles.  c->stream must be
// a non-default stream that is not capturing.
//   plain:   step_begin, initial residual, WHILE(inner){CG}, split, step_end
//   refined: step_begin, FP32 residual, WHILE(first){CG},
//            [HC_FP32_REFINED: IF(mid){double-float residual, WHILE(mid_inner){CG}}],
//            WHILE(outer){FP64 residual, WHILE(inner){CG}}, split, step_end
int build_chain(hc_ctx* c, cudaGraph_t target, Handles* h) {
  cudaStream_t s = c->stream;
  Handles hh;
  cudaStreamCaptureStatus cs;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  // the tail of the capture running on s, which then ends
  auto end_capture = [&](cudaGraph_t g, std::vector<cudaGraphNode_t>& tail) -> int {
    CU(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
    tail.assign(deps, deps + ndeps);
    cudaGraph_t same = g;
    CU(cudaStreamEndCapture(s, &same));
    return HC_OK;
  };
  // a WHILE (or IF) node after `after` in graph g; returns its body
  auto add_while = [&](cudaGraph_t g, const std::vector<cudaGraphNode_t>& after,
                       cudaGraphConditionalHandle* hd, cudaGraphNode_t* node,
                       cudaGraph_t* body, bool is_if = false) -> int {
    CU(cudaGraphConditionalHandleCreate(hd, g, 0, cudaGraphCondAssignDefault));
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = *hd;
    p.conditional.type = is_if ? cudaGraphCondTypeIf : cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    CU(cudaGraphAddNode(node, g, after.data(), nullptr, after.size(), &p));
    *body = p.conditional.phGraph_out[0];
    return HC_OK;
  };
  auto capture_iter = [&](cudaGraph_t body) -> int {
    CU(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    if (c->refined)
      refined_iter(c);
    else
      plain_iter(c);
    cudaGraph_t same = body;
    CU(cudaStreamEndCapture(s, &same));
    return HC_OK;
  };
  std::vector<cudaGraphNode_t> tail;
  CU(cudaStreamBeginCaptureToGraph(s, target, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  hc::step_begin(c->st, (int)c->n, s);
  if (c->refined)
    first_resid32(c);
  else
    plain_init(c);
  int rc = end_capture(target, tail);
  if (rc) return rc;
  cudaGraphNode_t loop_node;
  cudaGraph_t body = nullptr;
  if (c->refined) {
    // the first inner loop, then the refinement loop with its own inner loop
    cudaGraphNode_t first_node;
    rc = add_while(target, tail, &hh.first, &first_node, &body);
    if (!rc) rc = capture_iter(body);
    if (rc) return rc;
    if (c->mid_df) {
      // IF(mid){double-float residual, WHILE(mid_inner){CG}}
      cudaGraphNode_t mid_node, mi_node;
      cudaGraph_t mbody = nullptr;
      rc = add_while(target, std::vector<cudaGraphNode_t>{first_node}, &hh.mid, &mid_node, &mbody,
                     true);
      if (rc) return rc;
      CU(cudaStreamBeginCaptureToGraph(s, mbody, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal));
      mid_resid(c);
      std::vector<cudaGraphNode_t> mtail;
      rc = end_capture(mbody, mtail);
      if (!rc) rc = add_while(mbody, mtail, &hh.mid_inner, &mi_node, &body);
      if (!rc) rc = capture_iter(body);
      if (rc) return rc;
      first_node = mid_node;
    }
    cudaGraph_t obody = nullptr;
    rc = add_while(target, std::vector<cudaGraphNode_t>{first_node}, &hh.outer, &loop_node, &obody);
    if (rc) return rc;
    CU(cudaStreamBeginCaptureToGraph(s, obody, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    refined_resid(c);
    std::vector<cudaGraphNode_t> otail;
    rc = end_capture(obody, otail);
    if (rc) return rc;
    cudaGraphNode_t inode;
    rc = add_while(obody, otail, &hh.inner, &inode, &body);
  } else {
    rc = add_while(target, tail, &hh.inner, &loop_node, &body);
  }
  if (!rc) rc = capture_iter(body);
  if (rc) return rc;
  CU(cudaStreamBeginCaptureToGraph(s, target, &loop_node, nullptr, 1,
                                   cudaStreamCaptureModeThreadLocal));
  split_step(c);
  hc::step_end(c->st, c->refined, s);
  cudaGraph_t same = target;
  CU(cudaStreamEndCapture(s, &same));
  *h = hh;
  return HC_OK;
}

void abort_capture(cudaStream_t s) {
  cudaStreamCaptureStatus cs;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(s, &junk);
  }
  cudaGetLastError();
}

// Kernels of one step's graph: fixed nodes (step_begin, the initial residual
// (plain FP64, or the refined modes' FP32 one), split step, step_end), one CG
// iteration, one FP64 refinement residual.
void set_node_counts(hc_ctx* c) {
  const int split = c->dim == 3 ? 5 : 4, resid = c->dim == 3 ? 5 : 3;
  c->graph_nodes_fixed = 1 + resid + split + 1;
  c->graph_nodes_body = c->dim == 3 ? 6 : 4;
  c->graph_nodes_outer = resid;
}

// Kernels that ran in graph launches, from the accumulated step statistics.
long long graph_kernel_count(const hc_ctx* c, const hc::SolveState& h) {
  long long n = (long long)c->graph_nodes_fixed * h.acc_steps +
                (long long)c->graph_nodes_body * h.acc_iters;
  // refinement residuals (FP64 or double-float), the mid-step one included
  if (c->refined) n += (long long)c->graph_nodes_outer * (h.acc_res_full + h.acc_mid);
  return n;
}

// Device handles the kernels drive: the context's own graph or a batch graph.
int use_handles(hc_ctx* c, const Handles& h, cudaGraphConditionalHandle hgate = 0) {
  unsigned long long v[4] = {h.inner, h.outer, hgate, h.first};
  CU(cudaMemcpy(&c->st->h_inner, v, sizeof(v), cudaMemcpyHostToDevice));
  unsigned long long w[2] = {h.mid, h.mid_inner};
  CU(cudaMemcpy(&c->st->h_mid, w, sizeof(w), cudaMemcpyHostToDevice));
  return HC_OK;
}

// One graph per context: step_begin, [plain: init residual, WHILE(cg) body]
// or [refined: WHILE(outer){ residual, WHILE(inner) body }], split step,
// step_end.  Loop conditions are set by the kernels (cudaGraphSetConditional)
// and default to 0 at every launch, so a loop whose controlling kernel did not
// run is skipped rather than repeated: step_begin opens the refinement loop,
// the residual kernels open the CG loop, cg_update keeps it open while the
// iteration cap and tolerance allow.
int build_graph(hc_ctx* c) {
  if (!c->cap_stream) CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  // everything issued before the capture must be complete: the private stream
  // does not order against the context's stream
  CU(cudaStreamSynchronize(c->stream));
  cudaGraph_t graph;
  CU(cudaGraphCreate(&graph, 0));
  cudaStream_t keep = c->stream;
  long long before = c->launches;
  c->stream = c->cap_stream;
  Handles hh;
  int rc = build_chain(c, graph, &hh);
  c->stream = keep;
  c->launches = before;  // capture launched nothing
  if (rc) {
    abort_capture(c->cap_stream);
    cudaGraphDestroy(graph);
    return rc;
  }
  cudaError_t e = cudaGraphInstantiate(&c->gexec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __LINE__);
  set_node_counts(c);
  c->h_own = hh;
  c->graph_ready = true;
  return HC_OK;
}

// hc_run's graph: a gate kernel, then IF(not halted) { the step chain }.  A
// stopping rule sets st->halt in step_end; later launches then skip the whole
// step on the device.
int build_run_graph(hc_ctx* c) {
  if (!c->cap_stream) CU(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  CU(cudaStreamSynchronize(c->stream));
  cudaGraph_t graph;
  CU(cudaGraphCreate(&graph, 0));
  cudaStream_t keep = c->stream;
  const long long before = c->launches;
  c->stream = c->cap_stream;
  Handles hh;
  cudaGraphConditionalHandle hgate = 0;
  auto capture = [&]() -> int {
    cudaStream_t s = c->stream;
    CU(cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0,
                                     cudaStreamCaptureModeThreadLocal));
    hc::run_gate(c->st, s);
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    CU(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
    std::vector<cudaGraphNode_t> tail(deps, deps + ndeps);
    cudaGraph_t same = graph;
    CU(cudaStreamEndCapture(s, &same));
    CU(cudaGraphConditionalHandleCreate(&hgate, graph, 0, cudaGraphCondAssignDefault));
    cudaGraphNodeParams ip = {};
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hgate;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t node;
    CU(cudaGraphAddNode(&node, graph, tail.data(), nullptr, tail.size(), &ip));
    return build_chain(c, ip.conditional.phGraph_out[0], &hh);
  };
  int rc = capture();
  c->stream = keep;
  c->launches = before;
  if (rc) {
    abort_capture(c->cap_stream);
    cudaGraphDestroy(graph);
    return rc;
  }
  cudaError_t e = cudaGraphInstantiate(&c->gexec_run, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __LINE__);
  c->h_run = hh;
  c->h_gate = hgate;
  c->run_graph_ready = true;
  return HC_OK;
}

void drop_graphs(hc_ctx* c) {
  if (c->graph_ready) cudaGraphExecDestroy(c->gexec);
  if (c->run_graph_ready) cudaGraphExecDestroy(c->gexec_run);
  if (c->pipe_ready) cudaGraphExecDestroy(c->gexec_pipe);
  c->graph_ready = false;
  c->run_graph_ready = false;
  c->pipe_ready = false;
}

// ---------------------------------------------------------------- lagged certification
// hc_step with lagged certification: 2D HC_FP32_REFINED (the double-float
// mid-step residual on), graph mode, diagnostics off, sync_cert off.
bool pipe_on(const hc_ctx* c, int nsteps) {
  return nsteps >= 2 && c->dim == 2 && c->refined && !c->df && c->mid_df && !c->gen &&
         c->prm.use_graph && !diag_on(c) && !c->prm.sync_cert && c->m_prev[0] != nullptr;
}

// The split step of a lagged step: its gradient pass adds the last inner
// solve's correction to p64 (as the refinement residual's pass would), and
// the new m goes to m_tmp (m stays the step's input until the commit).
void split_step_lagged(hc_ctx* c) {
  auto& g = c->gf;
  cx<float>* Gx = c->G32;
  cx<float>* Gy = c->G32 + c->ns;
  hc::col_grad<float, double>(g, hc::CG_ADDDELTA, c->p64, nullptr, nullptr, c->x32, Gx, Gy, c->st, 0,
                              c->stream);
  hc::row_split<float>(g, Gx, Gy, (const float*)c->m[0], (const float*)c->m[1], (const float*)c->rf,
                       Gx, Gy, split_coef(c->prm), c->st, c->stream);
  hc::col_heat<float>(g, Gx, Gy, c->st, c->stream);
  hc::row_c2r<float>(g, Gx, Gy, c->m_tmp[0], c->m_tmp[1], c->st, 1, c->stream);
  c->launches += 4;
}

// The certifying FP64 residual of the pressure awaiting certification
// (p_saved, solved with m_prev), on stream s, with its own partial sums.
void cert_resid_launch(hc_ctx* c, cudaStream_t s) {
  hc::Geo<double> g = c->gd;
  g.partials = c->partials_c;
  hc::cert_resid(g, c->p_saved, c->m_prev[0], c->m_prev[1], (const float*)c->rf, c->b64, c->G64c,
                 c->st_c, s);
  c->launches += 3;
}

// Kernels of one lagged step graph launch (gate, step_begin, FP32 residual,
// split, step_end, certification, commit) besides its loops.
constexpr int kPipeFixedKernels = 1 + 1 + 3 + 4 + 1 + 3 + 2;

// The lagged step graph: a gate, then IF(not halted) { A ; B ; commit } with
//   A (high priority): step_begin, FP32 residual, WHILE(first){CG},
//     IF(mid){double-float residual, WHILE(mid_inner){CG}}, split (-> m_tmp), step_end;
//   B (low priority, beside A): the FP64 residual certifying the previous step;
//   commit after both: accept the step (m_tmp -> m, keeping m and p for its own
//   certification) or, if the previous step's certification failed, halt.
// A's kernels get the device's highest stream priority and B's the lowest, so
// the block scheduler fills the SMs with A's CTAs first and B's FP64-pipe work
// runs in what is left.
int build_pipe_graph(hc_ctx* c) {
  int lo = 0, hi = 0;
  CU(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  if (!c->cap_hi) CU(cudaStreamCreateWithPriority(&c->cap_hi, cudaStreamNonBlocking, hi));
  if (!c->cap_lo) CU(cudaStreamCreateWithPriority(&c->cap_lo, cudaStreamNonBlocking, lo));
  CU(cudaStreamSynchronize(c->stream));
  cudaGraph_t graph;
  CU(cudaGraphCreate(&graph, 0));
  cudaStream_t keep = c->stream;
  const long long before = c->launches;
  c->stream = c->cap_hi;
  Handles hh;
  cudaGraphConditionalHandle hgate = 0;
  std::vector<cudaGraph_t> graphs_a;     // graphs holding A's (and the commit's) kernels
  std::vector<cudaGraphNode_t> nodes_b;  // B's kernel nodes
  auto run = [&]() -> int {
    cudaStream_t s = c->stream;
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t ndeps = 0;
    auto end_capture = [&](cudaStream_t es, cudaGraph_t g, std::vector<cudaGraphNode_t>* tail) -> int {
      if (tail) {
        CU(cudaStreamGetCaptureInfo(es, &cs, nullptr, nullptr, &deps, nullptr, &ndeps));
        tail->assign(deps, deps + ndeps);
      }
      cudaGraph_t same = g;
      CU(cudaStreamEndCapture(es, &same));
      return HC_OK;
    };
    auto add_cond = [&](cudaGraph_t g, const std::vector<cudaGraphNode_t>& after,
                        cudaGraphConditionalHandle* hd, bool is_if, cudaGraphNode_t* node,
                        cudaGraph_t* body) -> int {
      CU(cudaGraphConditionalHandleCreate(hd, g, 0, cudaGraphCondAssignDefault));
      cudaGraphNodeParams p = {};
      p.type = cudaGraphNodeTypeConditional;
      p.conditional.handle = *hd;
      p.conditional.type = is_if ? cudaGraphCondTypeIf : cudaGraphCondTypeWhile;
      p.conditional.size = 1;
      CU(cudaGraphAddNode(node, g, after.data(), nullptr, after.size(), &p));
      *body = p.conditional.phGraph_out[0];
      graphs_a.push_back(*body);
      return HC_OK;
    };
    auto capture_iter = [&](cudaGraph_t body) -> int {
      CU(cudaStreamBeginCaptureToGraph(s, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      refined_iter(c);
      return end_capture(s, body, nullptr);
    };
    // gate, IF(not halted)
    graphs_a.push_back(graph);
    CU(cudaStreamBeginCaptureToGraph(s, graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    hc::run_gate(c->st, s);
    std::vector<cudaGraphNode_t> tail;
    int rc = end_capture(s, graph, &tail);
    cudaGraphNode_t gate_node;
    cudaGraph_t target = nullptr;
    if (!rc) rc = add_cond(graph, tail, &hgate, true, &gate_node, &target);
    if (rc) return rc;
    // A
    CU(cudaStreamBeginCaptureToGraph(s, target, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    hc::step_begin(c->st, (int)c->n, s);
    first_resid32(c);
    rc = end_capture(s, target, &tail);
    cudaGraphNode_t first_node, mid_node, mi_node;
    cudaGraph_t body = nullptr, mbody = nullptr;
    if (!rc) rc = add_cond(target, tail, &hh.first, false, &first_node, &body);
    if (!rc) rc = capture_iter(body);
    if (!rc) rc = add_cond(target, {first_node}, &hh.mid, true, &mid_node, &mbody);
    if (rc) return rc;
    CU(cudaStreamBeginCaptureToGraph(s, mbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    mid_resid(c);
    std::vector<cudaGraphNode_t> mtail;
    rc = end_capture(s, mbody, &mtail);
    if (!rc) rc = add_cond(mbody, mtail, &hh.mid_inner, false, &mi_node, &body);
    if (!rc) rc = capture_iter(body);
    if (rc) return rc;
    CU(cudaStreamBeginCaptureToGraph(s, target, &mid_node, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    split_step_lagged(c);
    hc::step_end(c->st, 1, s);
    std::vector<cudaGraphNode_t> atail;
    rc = end_capture(s, target, &atail);
    if (rc) return rc;
    // B, beside A; its nodes are the ones its capture adds
    size_t nb0 = 0, nb1 = 0;
    CU(cudaGraphGetNodes(target, nullptr, &nb0));
    std::vector<cudaGraphNode_t> pre(nb0);
    CU(cudaGraphGetNodes(target, pre.data(), &nb0));
    // B waits for A's first residual, so A's first inner loop starts on SMs
    // that B's long FP64 CTAs have not taken yet
    CU(cudaStreamBeginCaptureToGraph(c->cap_lo, target, tail.data(), nullptr, tail.size(),
                                     cudaStreamCaptureModeThreadLocal));
    cert_resid_launch(c, c->cap_lo);
    std::vector<cudaGraphNode_t> btail;
    rc = end_capture(c->cap_lo, target, &btail);
    if (rc) return rc;
    CU(cudaGraphGetNodes(target, nullptr, &nb1));
    std::vector<cudaGraphNode_t> all(nb1);
    CU(cudaGraphGetNodes(target, all.data(), &nb1));
    for (cudaGraphNode_t nd : all)
      if (std::find(pre.begin(), pre.end(), nd) == pre.end()) nodes_b.push_back(nd);
    // commit after A and B
    std::vector<cudaGraphNode_t> join(atail);
    join.insert(join.end(), btail.begin(), btail.end());
    CU(cudaStreamBeginCaptureToGraph(s, target, join.data(), nullptr, join.size(),
                                     cudaStreamCaptureModeThreadLocal));
    float* mp[2] = {c->m_prev[0], c->m_prev[1]};
    float* mm[2] = {(float*)c->m[0], (float*)c->m[1]};
    const float* mt[2] = {c->m_tmp[0], c->m_tmp[1]};
    hc::commit_copy(c->st, c->st_c, mm, mp, mt, c->p64, c->p_saved, c->n, c->ns, s);
    hc::commit_flags(c->st, c->st_c, 0, s);
    c->launches += 2;
    return end_capture(s, target, nullptr);
  };
  int rc = run();
  c->stream = keep;
  c->launches = before;
  if (rc) {
    abort_capture(c->cap_hi);
    abort_capture(c->cap_lo);
    cudaGraphDestroy(graph);
    return rc;
  }
  // priorities: every kernel node high, then B's low
  cudaKernelNodeAttrValue vhi = {}, vlo = {};
  vhi.priority = hi;
  vlo.priority = lo;
  for (cudaGraph_t g : graphs_a) {
    size_t nn = 0;
    CU(cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    CU(cudaGraphGetNodes(g, nodes.data(), &nn));
    for (cudaGraphNode_t nd : nodes) {
      cudaGraphNodeType t;
      CU(cudaGraphNodeGetType(nd, &t));
      if (t == cudaGraphNodeTypeKernel)
        CU(cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributePriority, &vhi));
    }
  }
  for (cudaGraphNode_t nd : nodes_b) {
    cudaGraphNodeType t;
    CU(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel)
      CU(cudaGraphKernelNodeSetAttribute(nd, cudaKernelNodeAttributePriority, &vlo));
  }
  cudaError_t e = cudaGraphInstantiate(&c->gexec_pipe, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate", __LINE__);
  c->h_pipe = hh;
  c->h_pipe_gate = hgate;
  c->pipe_ready = true;
  return HC_OK;
}

int set_graph_mode(hc_ctx* c, int on) {
  int v = on ? 1 : 0;
  CU(cudaMemcpyAsync(&c->st->graph_mode, &v, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

// hc_step with lagged certification: the lagged graph once per step, then
// the last step's certification.  A failed certification halts the later
// launches; hc_step then goes back to the failed step's start (its input m,
// its pressure as warm start), redoes it with the context's own certifying
// graph and runs the call's remaining steps with that graph too (a tolerance
// that two sweeps miss would otherwise cost a repair per step).  So every
// step returned is certified.
int step_lagged(hc_ctx* c, int nsteps) {
  if (!c->pipe_ready) {
    int rc = build_pipe_graph(c);
    if (rc) return rc;
  }
  int rc = use_handles(c, c->h_pipe, c->h_pipe_gate);
  if (!rc) rc = set_graph_mode(c, 1);
  if (rc) return rc;
  c->batch_handles = 0;
  hc::lag_mark(c->st, c->st_c, 1, c->stream);
  for (int k = 0; k < nsteps; ++k) CU(cudaGraphLaunch(c->gexec_pipe, c->stream));
  cert_resid_launch(c, c->stream);  // the last step's certification
  hc::commit_flags(c->st, c->st_c, 1, c->stream);
  hc::lag_mark(c->st, c->st_c, 0, c->stream);
  c->launches += 3;
  CU(cudaGetLastError());
  rc = read_state(c);
  if (!rc) rc = set_graph_mode(c, 0);
  if (rc) return rc;
  const hc::SolveState& h = *c->st_host;  // counters were reset at the call's start
  c->launches += kPipeFixedKernels * (long long)h.acc_steps + (long long)(nsteps - h.acc_steps) +
                 (long long)c->graph_nodes_body * h.acc_iters +
                 (long long)c->graph_nodes_outer * h.acc_mid;
  if (!h.cert_failed) return HC_OK;
  // back to the start of the step that failed its certification, then the
  // rest of the call with the certifying graph
  const int done = h.cert_steps - 1;
  for (int k = 0; k < 2; ++k)
    CU(cudaMemcpyAsync(c->m[k], c->m_prev[k], sizeof(float) * c->n, cudaMemcpyDeviceToDevice,
                       c->stream));
  CU(cudaMemcpyAsync(c->p64, c->p_saved, sizeof(cx<double>) * c->ns, cudaMemcpyDeviceToDevice,
                     c->stream));
  hc::msum<float>(c->gf, (const float*)c->m[0], (const float*)c->m[1], c->st, c->stream);
  c->launches += 1;
  if (!c->graph_ready) {
    rc = build_graph(c);
    if (rc) return rc;
  }
  const hc::SolveState b2 = h;
  rc = use_handles(c, c->h_own);
  if (!rc) rc = set_graph_mode(c, 1);
  if (rc) return rc;
  for (int k = done; k < nsteps; ++k) CU(cudaGraphLaunch(c->gexec, c->stream));
  rc = read_state(c);
  if (!rc) rc = set_graph_mode(c, 0);
  if (rc) return rc;
  const hc::SolveState& h2 = *c->st_host;
  c->launches += (long long)c->graph_nodes_fixed * (h2.acc_steps - b2.acc_steps) +
                 (long long)c->graph_nodes_body * (h2.acc_iters - b2.acc_iters) +
                 (long long)c->graph_nodes_outer *
                     ((h2.acc_res_full - b2.acc_res_full) + (h2.acc_mid - b2.acc_mid));
  return HC_OK;
}

int restore_b2(hc_ctx* c, double b2) {
  CU(cudaMemcpyAsync(&c->st->outer_b2, &b2, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

int fill_stats(hc_ctx* c, hc_step_stats* out) {
  const hc::SolveState& h = *c->st_host;
  if (out) {
    out->cg_iters = h.total_it;
    out->refine_sweeps = h.sweeps;
    const double r2 = c->refined ? h.outer_r2 : h.rnorm2;
    out->rel_residual = h.outer_b2 > 0 ? std::sqrt(r2 / h.outer_b2) : 0.0;
    out->kappa = h.kappa;
    out->status = h.step_status;
    out->total_cg_iters = h.acc_iters;
    out->total_sweeps = h.acc_sweeps;
    out->energy = h.energy_valid ? h.energy : 0.0;
    out->delta_m = h.diag ? h.delta_m : 0.0;
    out->energy_valid = h.diag ? h.energy_valid : 0;
    out->stop_reason = h.run_mode ? h.stop_reason : HC_STOP_NONE;
    out->energy_step = (h.run_mode && h.stop_reason == HC_STOP_ENERGY) ? h.energy_step : -1;
    out->first_sweep_fp32 = h.first_used;
    out->total_first_fp32 = h.acc_first;
    out->mid_residual_df = h.mid_used;
    out->total_mid_df = h.acc_mid;
    out->refine_residuals = c->refined ? h.res_full : 0;
    out->total_refine_residuals = c->refined ? h.acc_res_full : 0;
  }
  return HC_OK;
}

}  // namespace

// ===================================================================== C ABI

extern "C" {

const char* hc_strerror(int code) {
  switch (code) {
    case HC_OK: return "ok";
    case HC_EINVAL: return "invalid argument";
    case HC_ENOMEM: return "out of device memory or workspace too small";
    case HC_ECUDA: return "CUDA runtime error";
    case HC_ENOCONV: return "CG did not reach the tolerance within its iteration cap";
    case HC_ENONFINITE: return "non-finite value in p or m";
    case HC_ETIMEOUT: return "bounded wait gave up";
    case HC_ENOTSUP: return "not supported by this build";
    case HC_EBOUNDS: return "a guard zone after a device buffer was overwritten (bounds-checked build)";
    default: return "unknown error";
  }
}

int hc_workspace_size(const hc_grid* grid, const hc_params* params, size_t* bytes) {
  if (check_grid(grid) || check_params(params) || !bytes) return HC_EINVAL;
  if (generic_grid(grid) && params->precision != HC_FP64_PLAIN) return HC_ENOTSUP;
  hc_ctx tmp{};  // every member zero (or its default)
  tmp.grid = *grid;
  tmp.dim = grid->dim;
  tmp.gen = generic_grid(grid) ? 1 : 0;
  tmp.nx = grid->n[0];
  tmp.ny = grid->n[1];
  tmp.nz = grid->dim == 3 ? grid->n[2] : 1;
  tmp.H = tmp.gen ? tmp.nx / 2 + 1 : tmp.nx / 2;
  tmp.n = (size_t)tmp.nx * tmp.ny * tmp.nz;
  tmp.ns = (size_t)tmp.nz * tmp.ny * tmp.H;
  tmp.refined = params->precision != HC_FP64_PLAIN;
  tmp.df = params->precision == HC_FP32_REFINED_DF;
  Layout L;
  layout(&tmp, L);
  *bytes = (L.off + kAlign - 1) / kAlign * kAlign;
  return HC_OK;
}

int hc_create(hc_ctx** out, const hc_grid* grid, const hc_params* params, void* workspace,
              size_t workspace_bytes) {
  if (!out) return HC_EINVAL;
  *out = nullptr;
  if (check_grid(grid) || check_params(params)) return HC_EINVAL;
  if (generic_grid(grid) && params->precision != HC_FP64_PLAIN) return HC_ENOTSUP;
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) % kAlign)) return HC_EINVAL;
  size_t need = 0;
  hc_workspace_size(grid, params, &need);
  if (workspace && workspace_bytes < need) return HC_ENOMEM;
  hc_ctx* c = new (std::nothrow) hc_ctx();  // value-initialised: every member zero (or its default)
  if (!c) return HC_ENOMEM;
  c->grid = *grid;
  c->prm = *params;
  apply_defaults(c->prm);
  c->dim = grid->dim;
  c->gen = generic_grid(grid) ? 1 : 0;
  c->nx = grid->n[0];
  c->ny = grid->n[1];
  c->nz = grid->dim == 3 ? grid->n[2] : 1;
  c->H = c->gen ? c->nx / 2 + 1 : c->nx / 2;
  c->n = (size_t)c->nx * c->ny * c->nz;
  c->ns = (size_t)c->nz * c->ny * c->H;
  c->refined = params->precision != HC_FP64_PLAIN;
  c->df = params->precision == HC_FP32_REFINED_DF;
  c->mid_df = mid_df_on(c);
  set_node_counts(c);
  c->stream = (cudaStream_t)params->stream;
  c->mean_r = 1.0;
  if (workspace) {
    c->ws = workspace;
    c->ws_bytes = workspace_bytes;
    c->owns_ws = false;
  } else {
    if (cudaMalloc(&c->ws, need) != cudaSuccess) {
      delete c;
      return HC_ENOMEM;
    }
    c->ws_bytes = need;
    c->owns_ws = true;
  }
  if (cudaMallocHost(&c->st_host, sizeof(hc::SolveState)) != cudaSuccess) {
    if (c->owns_ws) cudaFree(c->ws);
    delete c;
    return HC_ENOMEM;
  }
  Layout L;
  L.base = static_cast<char*>(c->ws);
  L.zones = &c->zones;
  layout(c, L);
  if (c->gen) {
    fill_generic_geo(c);
    hc::set_smem_limits_gen();
  } else {
    fill_geo<float>(c, c->gf, c->twx_f, c->twy_f, c->kxd_f, c->kyd_f, c->hx_f, c->hy_f);
    fill_geo<double>(c, c->gd, c->twx_d, c->twy_d, c->kxd_d, c->kyd_d, c->hx_d, c->hy_d);
    c->gf.x2x = c->x2x_f;
    c->gf.x2y = c->x2y_f;
    c->gd.x2x = c->x2x_d;
    c->gd.x2y = c->x2y_d;
    fill_geo<df64>(c, c->gq, c->twx_q, c->twy_q, c->kxd_q, c->kyd_q, nullptr, nullptr);
    c->gq.tc = c->gd.tc;
    c->gq.ltc = c->gd.ltc;
    if (c->dim == 3) {
      fill_geo3<float>(c, c->gf, c->rowf, c->twz_f, c->kzd_f, c->hz_f);
      fill_geo3<double>(c, c->gd, c->rowd, c->twz_d, c->kzd_d, c->hz_d);
      fill_geo3<df64>(c, c->gq, c->rowq, c->twz_q, c->kzd_q, nullptr);
    }
    hc::set_smem_limits_f32();
    hc::set_smem_limits_f64();
    hc::set_smem_limits_df();
    if (c->dim == 3) {
      hc::set_smem_limits_3d_f32();
      hc::set_smem_limits_3d_f64();
      hc::set_smem_limits_3d_df();
    }
  }
  int rc = HC_OK;
  if (cudaMemsetAsync(c->ws, 0, need, c->stream) != cudaSuccess) rc = HC_ECUDA;
  if (!rc) rc = fill_zones(c->stream, static_cast<char*>(c->ws), c->zones);
  if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = HC_ECUDA;
  if (!rc) rc = upload_tables(c);
  if (!rc) rc = upload_heat(c);
  // r = 1 everywhere by default
  if (!rc) {
    std::vector<double> ones(c->n, 1.0);
    rc = hc_set_r(c, ones.data(), c->n);
  }
  if (!rc) rc = push_config(c);
  if (!rc && cudaStreamSynchronize(c->stream) != cudaSuccess) rc = HC_ECUDA;
  if (rc) {
    hc_destroy(c);
    return rc;
  }
  *out = c;
  return HC_OK;
}

int hc_check_redzones(hc_ctx* c, int* nzones, int* zone, size_t* owner_bytes) {
  if (nzones) *nzones = 0;
  if (zone) *zone = -1;
  if (owner_bytes) *owner_bytes = 0;
  if (!c) return HC_EINVAL;
  if (nzones) *nzones = c->zones.n;
  if (c->zones.carved > c->zones.n) return HC_ENOTSUP;  // more buffers than the zone table holds
  int bad = -1;
  const int rc = scan_zones(c->stream, static_cast<const char*>(c->ws), c->zones, &bad);
  if (zone) *zone = bad;
  if (bad >= 0 && owner_bytes) *owner_bytes = c->zones.owner[bad];
  return rc;
}

int hc_check_poke(hc_ctx* c, int zone) {
  if (!kRedzone) return HC_ENOTSUP;
  if (!c || zone < 0 || zone >= c->zones.n) return HC_EINVAL;
  char* at = static_cast<char*>(c->ws) + c->zones.start[zone] + c->zones.len[zone] / 2;
  CU(cudaMemsetAsync(at, 0, 1, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

void hc_destroy(hc_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  drop_graphs(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->cap_hi) cudaStreamDestroy(c->cap_hi);
  if (c->cap_lo) cudaStreamDestroy(c->cap_lo);
  if (c->io_stream) cudaStreamDestroy(c->io_stream);
  for (cudaEvent_t e : c->io_ev)
    if (e) cudaEventDestroy(e);
  if (c->owns_ws && c->ws) cudaFree(c->ws);
  if (c->st_host) cudaFreeHost(c->st_host);
  delete c;
}

int hc_set_params(hc_ctx* c, const hc_params* p) {
  if (!c || check_params(p)) return HC_EINVAL;
  if (p->precision != c->prm.precision || p->stream != c->prm.stream) return HC_EINVAL;
  hc_params np = *p;
  apply_defaults(np);
  c->prm = np;
  c->mid_df = mid_df_on(c);
  int rc = upload_heat(c);
  if (!rc) rc = push_config(c);
  // split coefficients (and, in 3D, whether the diagnostics passes run) are
  // baked into the graphs
  if (!rc) drop_graphs(c);
  return rc;
}

int hc_set_r(hc_ctx* c, const double* r, size_t count) {
  if (!c || !r || count != c->n) return HC_EINVAL;
  double s = 0;
  for (size_t i = 0; i < count; ++i) {
    if (!(r[i] > 0) || !std::isfinite(r[i])) return HC_EINVAL;
    s += r[i];
  }
  CU(cudaMemcpyAsync(c->stage, r, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
  if (c->refined)
    hc::convert<float, double>(c->stage, (float*)c->rf, count, c->stream);
  else
    hc::convert<double, double>(c->stage, (double*)c->rf, count, c->stream);
  c->launches += 1;
  c->mean_r = s / (double)count;
  int rc = push_config(c);
  if (rc) return rc;
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

// Forward 3D transform of the FP64 field in stage -> projected FP64 spectrum.
static int forward64_3d(hc_ctx* c, cx<double>* out, hc::SolveState* norm_into) {
  if (c->df) {
    df64* phys = reinterpret_cast<df64*>(c->stage + c->n);
    cx<df64>* rows = reinterpret_cast<cx<df64>*>(c->G64);
    hc::convert<df64, double>(c->stage, phys, c->n, c->stream);
    hc::row_r2c<df64>(c->rowq, phys, nullptr, rows, nullptr, c->stream);
    hc::axis_fft<df64>(c->gq, 1, -1, 1, tri(rows, c->ns), tri(rows, c->ns), df64(1.0), c->stream);
    hc::z_fwd_project<df64>(c->gq, rows, reinterpret_cast<cx<df64>*>(out), norm_into, c->stream);
    c->launches += 4;
  } else {
    cx<double>* rows = c->G64;
    hc::row_r2c<double>(c->rowd, c->stage, nullptr, rows, nullptr, c->stream);
    hc::axis_fft<double>(c->gd, 1, -1, 1, tri(rows, c->ns), tri(rows, c->ns), 1.0, c->stream);
    hc::z_fwd_project<double>(c->gd, rows, out, norm_into, c->stream);
    c->launches += 3;
  }
  CU(cudaGetLastError());
  return HC_OK;
}

// Forward 2D transform of the FP64 field in stage -> projected FP64 spectrum.
static int forward64(hc_ctx* c, cx<double>* out, hc::SolveState* norm_into) {
  if (c->dim == 3) return forward64_3d(c, out, norm_into);
  if (c->gen) {
    hc::gen_row_fwd(c->gg, c->stage, nullptr, c->G64, nullptr, c->stream);
    hc::gen_col_fwd(c->gg, c->G64, nullptr, out, nullptr, 1, 0, norm_into, c->stream);
    c->launches += 2;
    CU(cudaGetLastError());
    return HC_OK;
  }
  if (c->df) {
    df64* phys = reinterpret_cast<df64*>(c->stage + c->n);
    cx<df64>* rows = reinterpret_cast<cx<df64>*>(c->G64);
    hc::convert<df64, double>(c->stage, phys, c->n, c->stream);
    hc::row_r2c<df64>(c->gq, phys, nullptr, rows, nullptr, c->stream);
    hc::col_fwd<df64>(c->gq, rows, nullptr, reinterpret_cast<cx<df64>*>(out), nullptr, 1, 1,
                      norm_into, c->stream);
    c->launches += 3;
    CU(cudaGetLastError());
    return HC_OK;
  }
  cx<double>* rows = c->G64;
  hc::row_r2c<double>(c->gd, c->stage, nullptr, rows, nullptr, c->stream);
  hc::col_fwd<double>(c->gd, rows, nullptr, out, nullptr, 1, 1, norm_into, c->stream);
  c->launches += 2;
  CU(cudaGetLastError());
  return HC_OK;
}

int hc_set_source(hc_ctx* c, const double* S, size_t count) {
  if (!c || !S || count != c->n) return HC_EINVAL;
  for (size_t i = 0; i < count; ++i)
    if (!std::isfinite(S[i])) return HC_EINVAL;
  CU(cudaMemcpyAsync(c->stage, S, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
  int rc = forward64(c, c->b64, c->st);
  if (rc) return rc;
  if (c->refined) {  // FP32 copy for the first sweep's residual
    if (c->bq) {       // double-float copy for the mid-step residual
      hc::convert<df64, double>(reinterpret_cast<const double*>(c->b64), reinterpret_cast<df64*>(c->bq),
                                2 * c->ns, c->stream);
      c->launches += 1;
    }
    if (c->dim == 2) {  // the 2D refinement keeps its FP32 vectors column-major
      if (c->df)
        hc::to_cm<df64>(c->gf, reinterpret_cast<const cx<df64>*>(c->b64), c->b32, c->stream);
      else
        hc::to_cm<double>(c->gf, c->b64, c->b32, c->stream);
    } else if (c->df)
      hc::convert<float, df64>(reinterpret_cast<const df64*>(c->b64), reinterpret_cast<float*>(c->b32),
                               2 * c->ns, c->stream);
    else
      hc::convert<float, double>(reinterpret_cast<const double*>(c->b64),
                                 reinterpret_cast<float*>(c->b32), 2 * c->ns, c->stream);
    c->launches += 1;
    CU(cudaGetLastError());
  }
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

int hc_set_p(hc_ctx* c, const double* p, size_t count) {
  if (!c || !p || count != c->n) return HC_EINVAL;
  CU(cudaMemcpyAsync(c->stage, p, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
  int rc = forward64(c, c->p64, nullptr);
  if (rc) return rc;
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

// After hc_set_m: sum |grad m|^2 of the new m, which only the energy of
// Section 2.5 uses; without diagnostics it is marked unknown instead (hc_run
// computes it when it turns the diagnostics on).
static int gm2_for_new_m(hc_ctx* c) {
  if (diag_on(c)) {
    gradnorm_current(c);
    return HC_OK;
  }
  CU(cudaMemsetAsync(&c->st->gm2_valid, 0, sizeof(int), c->stream));
  return HC_OK;
}

int hc_set_m(hc_ctx* c, const double* m, size_t count) {
  if (!c || !m || count != (size_t)c->dim * c->n) return HC_EINVAL;
  CU(cudaMemcpyAsync(c->stage, m, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
  if (c->dim == 3) {
    for (int k = 0; k < 3; ++k) {
      if (c->refined)
        hc::convert<float, double>(c->stage + k * c->n, (float*)c->m[k], c->n, c->stream);
      else
        hc::convert<double, double>(c->stage + k * c->n, (double*)c->m[k], c->n, c->stream);
    }
    if (c->refined)
      hc::msum3<float>(c->gf, mtri<float>(c), c->st, c->stream);
    else
      hc::msum3<double>(c->gd, mtri<double>(c), c->st, c->stream);
    c->launches += 4;
    int rc = gm2_for_new_m(c);
    if (rc) return rc;
    CU(cudaGetLastError());
    CU(cudaStreamSynchronize(c->stream));
    return HC_OK;
  }
  if (c->refined) {
    hc::convert<float, double>(c->stage, (float*)c->m[0], c->n, c->stream);
    hc::convert<float, double>(c->stage + c->n, (float*)c->m[1], c->n, c->stream);
    hc::msum<float>(c->gf, (const float*)c->m[0], (const float*)c->m[1], c->st, c->stream);
  } else {
    hc::convert<double, double>(c->stage, (double*)c->m[0], c->n, c->stream);
    hc::convert<double, double>(c->stage + c->n, (double*)c->m[1], c->n, c->stream);
    hc::msum<double>(c->gd, (const double*)c->m[0], (const double*)c->m[1], c->st, c->stream);
  }
  c->launches += 3;
  int rc = gm2_for_new_m(c);
  if (rc) return rc;
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

int hc_get_m(hc_ctx* c, double* out, size_t count) {
  if (!c || !out || count != (size_t)c->dim * c->n) return HC_EINVAL;
  for (int k = 0; k < c->dim; ++k) {
    if (c->refined)
      hc::convert<double, float>((const float*)c->m[k], c->stage + k * c->n, c->n, c->stream);
    else
      hc::convert<double, double>((const double*)c->m[k], c->stage + k * c->n, c->n, c->stream);
  }
  c->launches += c->dim;
  CU(cudaMemcpyAsync(out, c->stage, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

int hc_get_p(hc_ctx* c, double* out, size_t count) {
  if (!c || !out || count != c->n) return HC_EINVAL;
  if (c->gen) {
    hc::gen_col_inv(c->gg, c->p64, c->G64, 1.0 / (double)c->n, c->stream);
    hc::gen_row_c2r(c->gg, c->G64, nullptr, c->stage, nullptr, nullptr, 0, c->stream);
    c->launches += 2;
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(out, c->stage, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return HC_OK;
  }
  if (c->dim == 3) {
    if (c->df) {
      auto* p = reinterpret_cast<cx<df64>*>(c->p64);
      auto* rows = reinterpret_cast<cx<df64>*>(c->G64);
      df64* phys = reinterpret_cast<df64*>(c->stage + c->n);
      hc::axis_fft<df64>(c->gq, 2, +1, 1, tri(p, c->ns), tri(rows, c->ns), df64(1.0 / (double)c->n),
                         c->stream);
      hc::axis_fft<df64>(c->gq, 1, +1, 1, tri(rows, c->ns), tri(rows, c->ns), df64(1.0), c->stream);
      hc::row_c2r<df64>(c->rowq, rows, nullptr, phys, nullptr, nullptr, 0, c->stream);
      hc::convert<double, df64>(phys, c->stage, c->n, c->stream);
      c->launches += 4;
    } else {
      cx<double>* rows = c->G64;
      hc::axis_fft<double>(c->gd, 2, +1, 1, tri(c->p64, c->ns), tri(rows, c->ns),
                           1.0 / (double)c->n, c->stream);
      hc::axis_fft<double>(c->gd, 1, +1, 1, tri(rows, c->ns), tri(rows, c->ns), 1.0, c->stream);
      hc::row_c2r<double>(c->rowd, rows, nullptr, c->stage, nullptr, nullptr, 0, c->stream);
      c->launches += 3;
    }
    CU(cudaGetLastError());
    CU(cudaMemcpyAsync(out, c->stage, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
    CU(cudaStreamSynchronize(c->stream));
    return HC_OK;
  }
  if (c->df) {
    cx<df64>* rows = reinterpret_cast<cx<df64>*>(c->G64);
    df64* phys = reinterpret_cast<df64*>(c->stage + c->n);
    hc::col_inv<df64>(c->gq, reinterpret_cast<const cx<df64>*>(c->p64), rows,
                      df64(1.0 / (double)c->n), c->stream);
    hc::row_c2r<df64>(c->gq, rows, nullptr, phys, nullptr, nullptr, 0, c->stream);
    hc::convert<double, df64>(phys, c->stage, c->n, c->stream);
    c->launches += 3;
  } else {
    cx<double>* rows = c->G64;
    hc::col_inv<double>(c->gd, c->p64, rows, 1.0 / (double)c->n, c->stream);
    hc::row_c2r<double>(c->gd, rows, nullptr, c->stage, nullptr, nullptr, 0, c->stream);
    c->launches += 2;
  }
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(out, c->stage, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

// The whole state in one call.  In the 2D FP32-refined mode the host link
// and the SMs work side by side: a second stream of the context (io_stream)
// carries the copies, p's rows cross in kStateChunks pieces so that its FP64
// row transform starts on the first piece (set) and its last row transform
// overlaps the first pieces' copies (get), and m's copy and conversion run
// beside p's column transform.  p is staged in the lagged certification's
// FP64 scratch (G64c, 2 half spectra), which no step keeps between hc_step
// calls.  Other modes run the single-field calls one after the other.
constexpr int kStateChunks = 4;
static bool state_overlap(const hc_ctx* c) {
  return c->dim == 2 && !c->gen && c->refined && !c->df && c->G64c != nullptr;
}
static int io_setup(hc_ctx* c) {
  if (!c->io_stream) CU(cudaStreamCreateWithFlags(&c->io_stream, cudaStreamNonBlocking));
  for (cudaEvent_t& e : c->io_ev)
    if (!e) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return HC_OK;
}
// Row pieces of p: kStateChunks when each is a whole number of the row
// passes' CTAs, else one.
static int state_chunks(const hc_ctx* c) {
  const int rows = c->ny / kStateChunks;
  return (c->ny % kStateChunks == 0 && rows % c->gd.rpc == 0 && rows >= 64) ? kStateChunks : 1;
}

int hc_set_state(hc_ctx* c, const double* m, size_t m_count, const double* p, size_t p_count) {
  if (!c || !m || !p || m_count != (size_t)c->dim * c->n || p_count != c->n) return HC_EINVAL;
  if (!state_overlap(c)) {
    int rc = hc_set_m(c, m, m_count);
    return rc ? rc : hc_set_p(c, p, p_count);
  }
  int rc = io_setup(c);
  if (rc) return rc;
  double* pst = reinterpret_cast<double*>(c->G64c);  // n doubles fit in 2 half spectra
  const int nch = state_chunks(c), rows = c->ny / nch;
  const size_t prow = (size_t)rows * c->nx;           // values of one piece
  hc::Geo<double> gch = c->gd;
  gch.ny = rows;                                      // a row pass over one piece
  // earlier work on the context's stream (it may still read m or the stage)
  CU(cudaEventRecord(c->io_ev[0], c->stream));
  CU(cudaStreamWaitEvent(c->io_stream, c->io_ev[0], 0));
  // p first, piece by piece: each piece's row transform starts once it is on the device.
  // (Each launch is queued right after its piece's copy: from pageable memory a copy
  // returns only once the data is staged, and the work queued before it then already runs.)
  for (int k = 0; k < nch; ++k) {
    CU(cudaMemcpyAsync(pst + k * prow, p + k * prow, sizeof(double) * prow, cudaMemcpyHostToDevice,
                       c->io_stream));
    CU(cudaEventRecord(c->io_ev[2 + k], c->io_stream));
    CU(cudaStreamWaitEvent(c->stream, c->io_ev[2 + k], 0));
    hc::row_r2c<double>(gch, pst + k * prow, nullptr, c->G64 + (size_t)k * rows * c->H, nullptr,
                        c->stream);
  }
  hc::col_fwd<double>(c->gd, c->G64, nullptr, c->p64, nullptr, 1, 1, nullptr, c->stream);
  CU(cudaMemcpyAsync(c->stage, m, sizeof(double) * m_count, cudaMemcpyHostToDevice, c->io_stream));
  hc::convert<float, double>(c->stage, (float*)c->m[0], c->n, c->io_stream);
  hc::convert<float, double>(c->stage + c->n, (float*)c->m[1], c->n, c->io_stream);
  CU(cudaEventRecord(c->io_ev[1], c->io_stream));
  CU(cudaStreamWaitEvent(c->stream, c->io_ev[1], 0));
  hc::msum<float>(c->gf, (const float*)c->m[0], (const float*)c->m[1], c->st, c->stream);
  c->launches += 4 + nch;
  rc = gm2_for_new_m(c);
  if (rc) return rc;
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

int hc_get_state(hc_ctx* c, double* m_out, size_t m_count, double* p_out, size_t p_count) {
  if (!c || !m_out || !p_out || m_count != (size_t)c->dim * c->n || p_count != c->n)
    return HC_EINVAL;
  if (!state_overlap(c)) {
    int rc = hc_get_m(c, m_out, m_count);
    return rc ? rc : hc_get_p(c, p_out, p_count);
  }
  int rc = io_setup(c);
  if (rc) return rc;
  double* pst = reinterpret_cast<double*>(c->G64c);
  const int nch = state_chunks(c), rows = c->ny / nch;
  const size_t prow = (size_t)rows * c->nx;
  hc::Geo<double> gch = c->gd;
  gch.ny = rows;
  CU(cudaEventRecord(c->io_ev[0], c->stream));
  CU(cudaStreamWaitEvent(c->io_stream, c->io_ev[0], 0));
  // m's conversion is queued before p's column transform so that it gets the SMs
  // first; m's copy after the transform, because a copy to pageable memory
  // returns only when it is done
  hc::convert<double, float>((const float*)c->m[0], c->stage, c->n, c->io_stream);
  hc::convert<double, float>((const float*)c->m[1], c->stage + c->n, c->n, c->io_stream);
  hc::col_inv<double>(c->gd, c->p64, c->G64, 1.0 / (double)c->n, c->stream);
  CU(cudaMemcpyAsync(m_out, c->stage, sizeof(double) * m_count, cudaMemcpyDeviceToHost,
                     c->io_stream));
  // p's row transforms piece by piece, each piece's copy queued behind m's on
  // the second stream
  for (int k = 0; k < nch; ++k) {
    hc::row_c2r<double>(gch, c->G64 + (size_t)k * rows * c->H, nullptr, pst + k * prow, nullptr,
                        nullptr, 0, c->stream);
    CU(cudaEventRecord(c->io_ev[2 + k], c->stream));
    CU(cudaStreamWaitEvent(c->io_stream, c->io_ev[2 + k], 0));
    CU(cudaMemcpyAsync(p_out + k * prow, pst + k * prow, sizeof(double) * prow,
                       cudaMemcpyDeviceToHost, c->io_stream));
  }
  c->launches += 3 + nch;
  CU(cudaGetLastError());
  CU(cudaEventRecord(c->io_ev[1], c->io_stream));
  CU(cudaStreamWaitEvent(c->stream, c->io_ev[1], 0));
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

int hc_step(hc_ctx* c, int nsteps, hc_step_stats* last) {
  if (!c || nsteps < 0) return HC_EINVAL;
  if (nsteps == 0) return HC_OK;
  hc::reset_accum(c->st, c->stream);
  c->launches += 1;
  if (pipe_on(c, nsteps)) {
    int rc = step_lagged(c, nsteps);
    if (rc) return rc;
  } else if (c->prm.use_graph) {
    if (!c->graph_ready) {
      int rc = build_graph(c);
      if (rc) return rc;
    }
    int rc = use_handles(c, c->h_own);
    if (rc) return rc;
    c->batch_handles = 0;
    rc = set_graph_mode(c, 1);
    if (rc) return rc;
    for (int k = 0; k < nsteps; ++k) CU(cudaGraphLaunch(c->gexec, c->stream));
    rc = read_state(c);
    int rc2 = set_graph_mode(c, 0);
    if (rc) return rc;
    if (rc2) return rc2;
    c->launches += graph_kernel_count(c, *c->st_host);
  } else {
    for (int k = 0; k < nsteps; ++k) {
      int rc = step_host(c);
      if (rc) return rc;
      rc = read_state(c);
      if (rc) return rc;
      if (c->st_host->step_status == HC_ENONFINITE) break;
    }
  }
  int rc = read_state(c);
  if (rc) return rc;
  fill_stats(c, last);
  return c->st_host->first_bad;
}

static void gradient3(hc_ctx* c) {
  const size_t n = c->n;
  if (c->refined) {
    auto Gt = tri(c->G32, c->ns);
    if (c->df)
      hc::z_grad<float, df64>(c->gf, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64), nullptr,
                              nullptr, nullptr, Gt, c->st, 0, c->stream);
    else
      hc::z_grad<float, double>(c->gf, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gt, c->st,
                                0, c->stream);
    hc::axis_fft<float>(c->gf, 1, +1, 3, Gt, Gt, 1.0f, c->stream);
    float* f[3] = {(float*)Gt.v[0], (float*)Gt.v[1], (float*)Gt.v[2]};
    hc::row_c2r<float>(c->rowf, Gt.v[0], Gt.v[1], f[0], f[1], nullptr, 0, c->stream);
    hc::row_c2r<float>(c->rowf, Gt.v[2], nullptr, f[2], nullptr, nullptr, 0, c->stream);
    for (int k = 0; k < 3; ++k) hc::convert<double, float>(f[k], c->stage + k * n, n, c->stream);
    c->launches += 7;
  } else {
    auto Gt = tri(c->G64, c->ns);
    hc::z_grad<double, double>(c->gd, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gt, c->st,
                               0, c->stream);
    hc::axis_fft<double>(c->gd, 1, +1, 3, Gt, Gt, 1.0, c->stream);
    hc::row_c2r<double>(c->rowd, Gt.v[0], Gt.v[1], c->stage, c->stage + n, nullptr, 0, c->stream);
    hc::row_c2r<double>(c->rowd, Gt.v[2], nullptr, c->stage + 2 * n, nullptr, nullptr, 0,
                        c->stream);
    c->launches += 4;
  }
}

int hc_run(hc_ctx* c, int max_steps, double eps, int stop_on_energy, int* steps_done,
           hc_step_stats* last) {
  if (!c || max_steps < 0) return HC_EINVAL;
  if (steps_done) *steps_done = 0;
  const int forced = c->prm.diagnostics ? 0 : 1;
  if (forced) {
    // the 3D diagnostics passes are captured only when diagnostics are on
    c->force_diag = 1;
    if (c->run_graph_ready) {
      cudaGraphExecDestroy(c->gexec_run);
      c->run_graph_ready = false;
    }
  }
  int rc = push_config(c);
  if (!rc) {
    // the energy of the current m needs its gradient norm, which nothing
    // computed while the diagnostics were off
    if (forced) gradnorm_current(c);
    hc::set_run(c->st, 1, eps, stop_on_energy ? 1 : 0, c->stream);
    hc::reset_accum(c->st, c->stream);
    c->launches += 2;
  }
  if (!rc && max_steps > 0) {
    if (c->prm.use_graph) {
      if (!c->run_graph_ready) rc = build_run_graph(c);
      if (!rc) rc = use_handles(c, c->h_run, c->h_gate);
      c->batch_handles = 0;
      if (!rc) rc = set_graph_mode(c, 1);
      int launched = 0;
      while (!rc && launched < max_steps) {
        const int chunk = std::min(kRunChunk, max_steps - launched);
        for (int k = 0; k < chunk && !rc; ++k) {
          cudaError_t e = cudaGraphLaunch(c->gexec_run, c->stream);
          if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphLaunch", __LINE__);
        }
        launched += chunk;
        if (!rc) rc = read_state(c);
        if (!rc && c->st_host->halt) break;
      }
      const int rc2 = set_graph_mode(c, 0);
      if (!rc) rc = rc2;
      if (!rc) {
        c->launches += launched;  // gate kernels
        c->launches += graph_kernel_count(c, *c->st_host);
      }
    } else {
      for (int k = 0; k < max_steps && !rc; ++k) {
        rc = step_host(c);
        if (!rc) rc = read_state(c);
        if (!rc && c->st_host->halt) break;
      }
    }
  }
  if (!rc) rc = read_state(c);
  if (!rc) fill_stats(c, last);
  if (!rc && steps_done) *steps_done = c->st_host->acc_steps;
  const int first_bad = rc ? rc : c->st_host->first_bad;
  // leave run mode (the stats above were taken first) and the forced diagnostics
  hc::set_run(c->st, 0, 0.0, 0, c->stream);
  c->launches += 1;
  if (forced) {
    c->force_diag = 0;
    const int rc3 = push_config(c);
    if (!rc) rc = rc3;
    if (c->run_graph_ready) {
      cudaGraphExecDestroy(c->gexec_run);
      c->run_graph_ready = false;
    }
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize", __LINE__);
  return rc ? rc : first_bad;
}

int hc_gradient(hc_ctx* c, double* out, size_t count) {
  if (!c || !out || count != (size_t)c->dim * c->n) return HC_EINVAL;
  if (c->gen) {
    cx<double>* Gx = c->G64;
    cx<double>* Gy = c->G64 + c->ns;
    hc::gen_col_grad(c->gg, hc::CG_PLAIN, c->p64, nullptr, nullptr, Gx, Gy, c->st, 0, c->stream);
    hc::gen_row_c2r(c->gg, Gx, Gy, c->stage, c->stage + c->n, nullptr, 0, c->stream);
    c->launches += 2;
  } else if (c->dim == 3) {
    gradient3(c);
  } else if (c->refined) {
    cx<float>* Gx = c->G32;
    cx<float>* Gy = c->G32 + (size_t)c->ny * c->H;
    if (c->df)
      hc::col_grad<float, df64>(c->gf, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64), nullptr,
                                nullptr, nullptr, Gx, Gy, c->st, 0, c->stream);
    else
      hc::col_grad<float, double>(c->gf, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gx, Gy,
                                  c->st, 0, c->stream);
    hc::row_c2r<float>(c->gf, Gx, Gy, (float*)Gx, (float*)Gy, nullptr, 0, c->stream);
    hc::convert<double, float>((const float*)Gx, c->stage, c->n, c->stream);
    hc::convert<double, float>((const float*)Gy, c->stage + c->n, c->n, c->stream);
    c->launches += 4;
  } else {
    cx<double>* Gx = c->G64;
    cx<double>* Gy = c->G64 + (size_t)c->ny * c->H;
    hc::col_grad<double, double>(c->gd, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gx, Gy,
                                 c->st, 0, c->stream);
    hc::row_c2r<double>(c->gd, Gx, Gy, c->stage, c->stage + c->n, nullptr, 0, c->stream);
    c->launches += 2;
  }
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(out, c->stage, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

int hc_apply_operator(hc_ctx* c, const double* f, double* out, size_t count) {
  if (!c || !f || !out || count != c->n) return HC_EINVAL;
  CU(cudaMemcpyAsync(c->stage, f, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
  if (c->gen) {
    cx<double>* Gx = c->G64;
    cx<double>* Gy = c->G64 + c->ns;
    hc::gen_row_fwd(c->gg, c->stage, nullptr, Gx, nullptr, c->stream);
    hc::gen_col_fwd(c->gg, Gx, nullptr, c->d64, nullptr, 1, 0, nullptr, c->stream);
    hc::gen_col_grad(c->gg, hc::CG_PLAIN, c->d64, nullptr, nullptr, Gx, Gy, c->st, 0, c->stream);
    hc::gen_row_apply(c->gg, Gx, Gy, (const double*)c->m[0], (const double*)c->m[1],
                      (const double*)c->rf, Gx, Gy, nullptr, c->stream);
    hc::gen_col_div(c->gg, hc::CD_PLAIN, Gx, Gy, nullptr, c->q64, nullptr, c->stream);
    hc::gen_col_inv(c->gg, c->q64, Gx, 1.0 / (double)c->n, c->stream);
    hc::gen_row_c2r(c->gg, Gx, nullptr, c->stage, nullptr, nullptr, 0, c->stream);
    c->launches += 7;
  } else if (c->dim == 3) {
    if (c->refined) {
      float* fp = reinterpret_cast<float*>(c->q32);
      hc::convert<float, double>(c->stage, fp, c->n, c->stream);
      apply_operator3<float, float>(c, c->gf, c->rowf, fp, c->G32, c->d32, c->r32);
      hc::convert<double, float>(fp, c->stage, c->n, c->stream);
      c->launches += 2;
    } else {
      apply_operator3<double, double>(c, c->gd, c->rowd, c->stage, c->G64, c->d64, c->q64);
    }
  } else if (c->refined) {
    auto& g = c->gf;
    cx<float>* Gx = c->G32;
    cx<float>* Gy = c->G32 + (size_t)c->ny * c->H;
    float* fp = reinterpret_cast<float*>(c->q32);
    hc::convert<float, double>(c->stage, fp, c->n, c->stream);
    hc::row_r2c<float>(g, fp, nullptr, Gx, nullptr, c->stream);
    hc::col_fwd<float>(g, Gx, nullptr, c->d32, nullptr, 1, 1, nullptr, c->stream);
    hc::col_grad<float, float>(g, hc::CG_PLAIN, c->d32, nullptr, nullptr, nullptr, Gx, Gy, c->st, 0,
                               c->stream);
    hc::row_apply<float, float>(g, Gx, Gy, (const float*)c->m[0], (const float*)c->m[1],
                                (const float*)c->rf, Gx, Gy, nullptr, c->stream);
    hc::col_div<float>(g, hc::CD_PLAIN, Gx, Gy, nullptr, nullptr, c->q32, nullptr, nullptr, nullptr,
                       c->stream);
    hc::col_inv<float>(g, c->q32, Gx, 1.0f / (float)c->n, c->stream);
    hc::row_c2r<float>(g, Gx, nullptr, fp, nullptr, nullptr, 0, c->stream);
    hc::convert<double, float>(fp, c->stage, c->n, c->stream);
    c->launches += 9;
  } else {
    auto& g = c->gd;
    cx<double>* Gx = c->G64;
    cx<double>* Gy = c->G64 + (size_t)c->ny * c->H;
    hc::row_r2c<double>(g, c->stage, nullptr, Gx, nullptr, c->stream);
    hc::col_fwd<double>(g, Gx, nullptr, c->d64, nullptr, 1, 1, nullptr, c->stream);
    hc::col_grad<double, double>(g, hc::CG_PLAIN, c->d64, nullptr, nullptr, nullptr, Gx, Gy, c->st,
                                 0, c->stream);
    hc::row_apply<double, double>(g, Gx, Gy, (const double*)c->m[0], (const double*)c->m[1],
                                  (const double*)c->rf, Gx, Gy, nullptr, c->stream);
    hc::col_div<double>(g, hc::CD_PLAIN, Gx, Gy, nullptr, nullptr, c->q64, nullptr, nullptr,
                        nullptr, c->stream);
    hc::col_inv<double>(g, c->q64, Gx, 1.0 / (double)c->n, c->stream);
    hc::row_c2r<double>(g, Gx, nullptr, c->stage, nullptr, nullptr, 0, c->stream);
    c->launches += 7;
  }
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(out, c->stage, sizeof(double) * count, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

int hc_split_step(hc_ctx* c) {
  if (!c) return HC_EINVAL;
  split_step(c);
  CU(cudaGetLastError());
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

int hc_spectrum(hc_ctx* c, const double* f, double* out, size_t count) {
  if (!c || !f || !out || count != c->n) return HC_EINVAL;
  CU(cudaMemcpyAsync(c->stage, f, sizeof(double) * count, cudaMemcpyHostToDevice, c->stream));
  const size_t ns = c->ns;
  if (c->gen) {
    hc::gen_row_fwd(c->gg, c->stage, nullptr, c->G64, nullptr, c->stream);
    hc::gen_col_fwd(c->gg, c->G64, nullptr, reinterpret_cast<cx<double>*>(c->stage), nullptr, 0, 0,
                    nullptr, c->stream);
    c->launches += 2;
  } else if (c->dim == 3) {
    if (c->refined) {
      float* fp = reinterpret_cast<float*>(c->q32);
      auto Gt = tri(c->G32, ns);
      hc::convert<float, double>(c->stage, fp, c->n, c->stream);
      hc::row_r2c<float>(c->rowf, fp, nullptr, c->G32, nullptr, c->stream);
      hc::axis_fft<float>(c->gf, 1, -1, 1, Gt, Gt, 1.0f, c->stream);
      hc::axis_fft<float>(c->gf, 2, -1, 1, Gt, tri(c->d32, ns), 1.0f, c->stream);
      hc::convert<double, float>(reinterpret_cast<const float*>(c->d32), c->stage, 2 * ns,
                                 c->stream);
      c->launches += 5;
    } else {
      auto Gt = tri(c->G64, ns);
      hc::row_r2c<double>(c->rowd, c->stage, nullptr, c->G64, nullptr, c->stream);
      hc::axis_fft<double>(c->gd, 1, -1, 1, Gt, Gt, 1.0, c->stream);
      hc::axis_fft<double>(c->gd, 2, -1, 1, Gt, tri(reinterpret_cast<cx<double>*>(c->stage), ns),
                           1.0, c->stream);
      c->launches += 3;
    }
  } else if (c->refined) {
    auto& g = c->gf;
    float* fp = reinterpret_cast<float*>(c->q32);
    hc::convert<float, double>(c->stage, fp, c->n, c->stream);
    hc::row_r2c<float>(g, fp, nullptr, c->G32, nullptr, c->stream);
    hc::col_fwd<float>(g, c->G32, nullptr, c->d32, nullptr, 1, 0, nullptr, c->stream);
    hc::convert<double, float>(reinterpret_cast<const float*>(c->d32), c->stage, 2 * ns, c->stream);
    c->launches += 4;
  } else {
    auto& g = c->gd;
    hc::row_r2c<double>(g, c->stage, nullptr, c->G64, nullptr, c->stream);
    hc::col_fwd<double>(g, c->G64, nullptr, reinterpret_cast<cx<double>*>(c->stage), nullptr, 1, 0,
                        nullptr, c->stream);
    c->launches += 2;
  }
  CU(cudaGetLastError());
  CU(cudaMemcpyAsync(out, c->stage, sizeof(double) * 2 * ns, cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  return HC_OK;
}

const char* hc_last_cuda_error(void) { return g_last_error; }

}  // extern "C"

namespace {

// Layout of the adjoint's own memory (checkpoints, one segment of states, the
// reverse sweep's buffers) for precision T.
template <typename T>
struct AdjLayout {
  hc::AdjState* as;
  cx<double>* b_save;   // S spectrum (the solve's right-hand side is borrowed)
  T* mT;                // final m
  cx<double>* pT;       // final p spectrum
  T* cpm;               // checkpoints of m, ncp x 2n
  cx<double>* cpp;      // checkpoints of p, ncp x n/2
  T* segm;              // m^k of one segment, every x 2n
  cx<double>* segp;     // p^{k+1} of one segment, every x n/2
  cx<T>*A, *B, *C, *D;  // spectra: A, B, C two each, D one
  T *lam, *lm;          // lambda and lambda_m (2n each)
  double* dr;           // dL/dr accumulator (n)
  cx<double>* dS;       // dL/dS accumulator, packed spectrum
  double* cpk;          // sum |m|^2 and sum m_a m_b (the preconditioner's input) of each checkpoint
  double* segk;         // ... of each state of the segment
  double* kT;           // ... of the final state
  size_t bytes;
};

// Doubles of the sums of m kept with a state: sum |m|^2 and the six sums
// m_a m_b (contiguous in SolveState).
constexpr int kMsums = 7;
static_assert(offsetof(hc::SolveState, mm) == offsetof(hc::SolveState, msum) + sizeof(double),
              "the sums of m must be contiguous");

template <typename T>
void adj_layout(const hc_ctx* c, int nsteps, int every, char* base, AdjLayout<T>& a,
                Zones* zones = nullptr) {
  Layout L;
  L.base = base;
  L.zones = zones;
  const size_t n = c->n, ns = (size_t)c->ny * c->H;
  const size_t ncp = nsteps > 0 ? (size_t)((nsteps + every - 1) / every) : 1;
  const size_t seg = (size_t)std::min(every, std::max(nsteps, 1));
  a.as = L.take<hc::AdjState>(sizeof(hc::AdjState));
  a.b_save = L.take<cx<double>>(sizeof(cx<double>) * ns);
  a.mT = L.take<T>(sizeof(T) * 2 * n);
  a.pT = L.take<cx<double>>(sizeof(cx<double>) * ns);
  a.cpm = L.take<T>(sizeof(T) * 2 * n * ncp);
  a.cpp = L.take<cx<double>>(sizeof(cx<double>) * ns * ncp);
  a.segm = L.take<T>(sizeof(T) * 2 * n * seg);
  a.segp = L.take<cx<double>>(sizeof(cx<double>) * ns * seg);
  a.A = L.take<cx<T>>(sizeof(cx<T>) * 2 * ns);
  a.B = L.take<cx<T>>(sizeof(cx<T>) * 2 * ns);
  a.C = L.take<cx<T>>(sizeof(cx<T>) * 2 * ns);
  a.D = L.take<cx<T>>(sizeof(cx<T>) * ns);
  a.lam = L.take<T>(sizeof(T) * 2 * n);
  a.lm = L.take<T>(sizeof(T) * 2 * n);
  a.dr = L.take<double>(sizeof(double) * n);
  a.dS = L.take<cx<double>>(sizeof(cx<double>) * ns);
  a.cpk = L.take<double>(sizeof(double) * kMsums * ncp);
  a.segk = L.take<double>(sizeof(double) * kMsums * seg);
  a.kT = L.take<double>(sizeof(double) * kMsums);
  a.bytes = (L.off + kAlign - 1) / kAlign * kAlign;
}

// The pressure solve of one step without the split step (host-driven loops).
int solve_only(hc_ctx* c) {
  hc::step_begin(c->st, (int)c->n, c->stream);
  c->launches += 1;
  if (!c->refined) {
    plain_init(c);
    return run_cg_host(c, false);
  }
  for (int sweep = 0;; ++sweep) {
    refined_resid(c);
    int rc = read_state(c);
    if (rc) return rc;
    if (c->st_host->outer_done) break;
    rc = run_cg_host(c, true);
    if (rc) return rc;
    if (sweep > 1000) return HC_ETIMEOUT;
  }
  return HC_OK;
}

// A state is (m, p, the sums of m): restoring the exact sums keeps the
// preconditioner, hence every CG iterate of a recomputed step, identical to
// the original forward.
template <typename T>
int save_state(hc_ctx* c, T* m, cx<double>* p, double* msum) {
  const size_t ns = (size_t)c->ny * c->H;
  CU(cudaMemcpyAsync(msum, &c->st->msum, sizeof(double) * kMsums, cudaMemcpyDeviceToDevice,
                     c->stream));
  CU(cudaMemcpyAsync(m, c->m[0], sizeof(T) * c->n, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(m + c->n, c->m[1], sizeof(T) * c->n, cudaMemcpyDeviceToDevice, c->stream));
  if (p) CU(cudaMemcpyAsync(p, c->p64, sizeof(cx<double>) * ns, cudaMemcpyDeviceToDevice, c->stream));
  return HC_OK;
}

template <typename T>
int load_state(hc_ctx* c, const T* m, const cx<double>* p, const double* msum) {
  const size_t ns = (size_t)c->ny * c->H;
  CU(cudaMemcpyAsync(c->m[0], m, sizeof(T) * c->n, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(c->m[1], m + c->n, sizeof(T) * c->n, cudaMemcpyDeviceToDevice, c->stream));
  if (p) CU(cudaMemcpyAsync(c->p64, p, sizeof(cx<double>) * ns, cudaMemcpyDeviceToDevice, c->stream));
  CU(cudaMemcpyAsync(&c->st->msum, msum, sizeof(double) * kMsums, cudaMemcpyDeviceToDevice,
                     c->stream));
  return HC_OK;
}

// Reverse of step k: lambda (a.lam) <- lambda^k from lambda^{k+1}; c holds m^k
// and p64 holds p^{k+1}.
template <typename T>
int adj_reverse_step(hc_ctx* c, hc::Geo<T>& g, AdjLayout<T>& a, const cx<double>* pk1) {
  const size_t ns = (size_t)c->ny * c->H;
  cudaStream_t s = c->stream;
  const T* mx = (const T*)c->m[0];
  const T* my = (const T*)c->m[1];
  cx<T>*A0 = a.A, *A1 = a.A + ns, *B0 = a.B, *B1 = a.B + ns, *C0 = a.C, *C1 = a.C + ns;
  const hc::SplitCoef cf = split_coef(c->prm);
  // grad p^{k+1} (rows) and b = R(A(m^k, g)) (rows)
  hc::col_grad<T, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, A0, A1, c->st, 0, s);
  hc::row_split<T>(g, A0, A1, mx, my, (const T*)c->rf, B0, B1, cf, c->st, s);
  // lambda_b = H lambda (H is symmetric), as row spectra
  hc::row_r2c<T>(g, a.lam, a.lam + c->n, C0, C1, s);
  hc::col_heat<T>(g, C0, C1, nullptr, s);
  // dL/dD^2 = <lambda_b, (-|xi|^2 dt) b>
  hc::col_lap_dot<T>(g, C0, B0, c->prm.dt, a.as, s);
  hc::col_lap_dot<T>(g, C1, B1, c->prm.dt, a.as, s);
  // pointwise Jacobians: lambda_m, lambda_g (rows over A), dL/dc^2
  hc::row_adj_point<T>(g, A0, A1, C0, C1, mx, my, a.lm, a.lm + c->n, cf, a.as, s);
  // lambda_p = -div lambda_g, the adjoint solve A mu = lambda_p
  hc::col_div<T>(g, hc::CD_PLAIN, A0, A1, nullptr, nullptr, a.D, nullptr, nullptr, nullptr, s);
  hc::spec_norm2<T>(g, a.D, c->st, s);
  if constexpr (std::is_same<T, double>::value)
    CU(cudaMemcpyAsync(c->b64, a.D, sizeof(cx<double>) * ns, cudaMemcpyDeviceToDevice, s));
  else
    hc::convert<double, float>(reinterpret_cast<const float*>(a.D), reinterpret_cast<double*>(c->b64),
                               2 * ns, s);
  CU(cudaMemsetAsync(c->p64, 0, sizeof(cx<double>) * ns, s));
  c->launches += 12;
  CU(cudaGetLastError());
  int rc = solve_only(c);
  if (rc) return rc;
  hc::spec_accum<double>(c->gd, reinterpret_cast<double*>(a.dS), c->p64, s);
  // grad mu, grad p^{k+1}, and the r, m terms of the solve
  hc::col_grad<T, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, A0, A1, c->st, 0, s);
  CU(cudaMemcpyAsync(c->p64, pk1, sizeof(cx<double>) * ns, cudaMemcpyDeviceToDevice, s));
  hc::col_grad<T, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, B0, B1, c->st, 0, s);
  hc::row_adj_press<T>(g, A0, A1, B0, B1, mx, my, a.lm, a.lm + c->n, a.lam, a.lam + c->n, a.dr, s);
  c->launches += 4;
  CU(cudaGetLastError());
  return HC_OK;
}

template <typename T>
int adjoint_t(hc_ctx* c, hc::Geo<T>& g, int nsteps, int every, const double* lamT, double* dc2,
              double* dD2, double* dr, double* dS, double* dm0, char* ws) {
  AdjLayout<T> a;
  adj_layout<T>(c, nsteps, every, ws, a);
  const size_t n = c->n, ns = (size_t)c->ny * c->H;
  cudaStream_t s = c->stream;
  CU(cudaMemsetAsync(a.as, 0, sizeof(hc::AdjState), s));
  CU(cudaMemsetAsync(a.dr, 0, sizeof(double) * n, s));
  CU(cudaMemsetAsync(a.dS, 0, sizeof(cx<double>) * ns, s));
  CU(cudaMemcpyAsync(a.b_save, c->b64, sizeof(cx<double>) * ns, cudaMemcpyDeviceToDevice, s));
  int rc = read_state(c);
  if (rc) return rc;
  const double b2_save = c->st_host->outer_b2;
  int status = HC_OK;
  // forward with checkpoints
  for (int k = 0; k < nsteps; ++k) {
    if (k % every == 0) {
      rc = save_state<T>(c, a.cpm + 2 * n * (k / every), a.cpp + ns * (k / every),
                         a.cpk + kMsums * (k / every));
      if (rc) return rc;
    }
    rc = hc_step(c, 1, nullptr);
    if (rc == HC_ENOCONV) status = status ? status : rc;
    else if (rc) return rc;
  }
  rc = save_state<T>(c, a.mT, a.pT, a.kT);
  if (rc) return rc;
  // lambda(T)
  CU(cudaMemcpyAsync(c->stage, lamT, sizeof(double) * 2 * n, cudaMemcpyHostToDevice, s));
  if constexpr (std::is_same<T, double>::value)
    CU(cudaMemcpyAsync(a.lam, c->stage, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s));
  else
    hc::convert<float, double>(c->stage, a.lam, 2 * n, s);
  // reverse, one segment at a time
  const int nseg = nsteps > 0 ? (nsteps + every - 1) / every : 0;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int k0 = sg * every, k1 = std::min(k0 + every, nsteps);
    rc = load_state<T>(c, a.cpm + 2 * n * sg, a.cpp + ns * sg, a.cpk + kMsums * sg);
    if (rc) return rc;
    CU(cudaMemcpyAsync(c->b64, a.b_save, sizeof(cx<double>) * ns, cudaMemcpyDeviceToDevice, s));
    rc = restore_b2(c, b2_save);
    if (rc) return rc;
    for (int k = k0; k < k1; ++k) {
      rc = save_state<T>(c, a.segm + 2 * n * (k - k0), nullptr, a.segk + kMsums * (k - k0));
      if (rc) return rc;
      rc = hc_step(c, 1, nullptr);
      if (rc && rc != HC_ENOCONV) return rc;
      CU(cudaMemcpyAsync(a.segp + ns * (k - k0), c->p64, sizeof(cx<double>) * ns,
                         cudaMemcpyDeviceToDevice, s));
    }
    for (int k = k1 - 1; k >= k0; --k) {
      rc = load_state<T>(c, a.segm + 2 * n * (k - k0), a.segp + ns * (k - k0),
                         a.segk + kMsums * (k - k0));
      if (rc) return rc;
      rc = adj_reverse_step<T>(c, g, a, a.segp + ns * (k - k0));
      if (rc) return rc;
    }
  }
  // restore the final forward state and the source
  CU(cudaMemcpyAsync(c->b64, a.b_save, sizeof(cx<double>) * ns, cudaMemcpyDeviceToDevice, s));
  rc = restore_b2(c, b2_save);
  if (rc) return rc;
  rc = load_state<T>(c, a.mT, a.pT, a.kT);
  if (rc) return rc;
  // outputs
  hc::AdjState hs;
  CU(cudaMemcpyAsync(&hs, a.as, sizeof(hs), cudaMemcpyDeviceToHost, s));
  if (dm0) {
    if constexpr (std::is_same<T, double>::value)
      CU(cudaMemcpyAsync(c->stage, a.lam, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s));
    else
      hc::convert<double, float>(a.lam, c->stage, 2 * n, s);
    CU(cudaMemcpyAsync(dm0, c->stage, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, s));
  }
  if (dr) CU(cudaMemcpyAsync(dr, a.dr, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  if (dS) {
    cx<double>* rows = c->G64;
    hc::col_inv<double>(c->gd, a.dS, rows, 1.0 / (double)n, s);
    hc::row_c2r<double>(c->gd, rows, nullptr, c->stage, nullptr, nullptr, 0, s);
    c->launches += 2;
    CU(cudaMemcpyAsync(dS, c->stage, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  }
  CU(cudaStreamSynchronize(s));
  if (dc2) *dc2 = hs.dc2;
  if (dD2) *dD2 = hs.dD2;
  return status;
}

}  // namespace

extern "C" {

int hc_adjoint_workspace_size(const hc_ctx* c, int nsteps, int every, size_t* bytes) {
  if (!c || !bytes || nsteps < 0 || every < 1) return HC_EINVAL;
  if (c->df || c->dim != 2 || c->gen) return HC_ENOTSUP;
  if (c->refined) {
    AdjLayout<float> a;
    adj_layout<float>(c, nsteps, every, nullptr, a);
    *bytes = a.bytes;
  } else {
    AdjLayout<double> a;
    adj_layout<double>(c, nsteps, every, nullptr, a);
    *bytes = a.bytes;
  }
  return HC_OK;
}

int hc_adjoint(hc_ctx* c, int nsteps, int every, const double* lamT, double* dc2, double* dD2,
               double* dr, double* dS, double* dm0, void* workspace, size_t workspace_bytes) {
  if (!c || !lamT || nsteps < 0 || every < 1) return HC_EINVAL;
  if (c->df || c->dim != 2 || c->gen) return HC_ENOTSUP;
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) % kAlign)) return HC_EINVAL;
  size_t need = 0;
  int rc = hc_adjoint_workspace_size(c, nsteps, every, &need);
  if (rc) return rc;
  if (workspace && workspace_bytes < need) return HC_ENOMEM;
  void* ws = workspace;
  bool own = false;
  if (!ws) {
    if (cudaMalloc(&ws, need) != cudaSuccess) return HC_ENOMEM;
    own = true;
  }
  Zones zones{};  // the adjoint workspace's guard zones (bounds-checked build)
  if (kRedzone) {
    if (c->refined) {
      AdjLayout<float> t;
      adj_layout<float>(c, nsteps, every, (char*)ws, t, &zones);
    } else {
      AdjLayout<double> t;
      adj_layout<double>(c, nsteps, every, (char*)ws, t, &zones);
    }
    rc = fill_zones(c->stream, (char*)ws, zones);
  }
  if (!rc) {
    if (c->refined)
      rc = adjoint_t<float>(c, c->gf, nsteps, every, lamT, dc2, dD2, dr, dS, dm0, (char*)ws);
    else
      rc = adjoint_t<double>(c, c->gd, nsteps, every, lamT, dc2, dD2, dr, dS, dm0, (char*)ws);
  }
  if (kRedzone && rc != HC_ECUDA) {
    int bad = -1;
    const int zrc = scan_zones(c->stream, (const char*)ws, zones, &bad);
    if (zrc == HC_EBOUNDS || (zrc && !rc)) rc = zrc;
  }
  if (own) {
    cudaStreamSynchronize(c->stream);
    cudaFree(ws);
  }
  return rc;
}

}  // extern "C"

// ===================================================================== batches
// A batch groups contexts so that one graph launch advances all of them by a
// step.  Contexts of the 2D HC_FP32_REFINED path that share a grid size form a
// size class: the class's step is one chain of batched launches (hc_batch.cu),
// one launch per pass over all its members.  Any other context (3D, FP64
// plain, double-float, a size with one member) keeps its own step chain.  All
// chains sit side by side in the batch's graph.
struct BatchClass {
  std::vector<int> members;  // indices into hc_batch::ctx
  hc::BShape sh;
  hc::BInst* d_inst = nullptr;      // device copy of the members' BInst records
  long long* d_launches = nullptr;  // the class's kernel launches (device counter)
  long long launches_seen = 0;
};

struct hc_batch {
  std::vector<hc_ctx*> ctx;
  std::vector<Handles> h;     // per-context chains
  std::vector<int> cls_of;    // class of each context, -1: its own chain
  std::vector<BatchClass> cls;
  void* dmem;                 // device memory of the classes
  cudaStream_t stream;
  cudaStream_t cap;
  cudaGraphExec_t exec;
  bool ready;
};

namespace {

bool batchable(const hc_ctx* c) {
  return c->dim == 2 && c->refined && !c->df && c->mid_df;
}

// A member's record: its own tables, state and buffers, with the class's
// launch shapes (non-persistent kernels).
template <typename T>
hc::Geo<T> class_geo(const hc::Geo<T>& own, const hc::Geo<T>& rep) {
  hc::Geo<T> g = own;
  g.tc = rep.tc;
  g.ltc = rep.ltc;
  g.rpc = rep.rpc;
  g.lrpc = rep.lrpc;
  g.pipe = 0;
  g.rpipe = 0;
  return g;
}

hc::BInst member_record(const hc_ctx* c, const hc_ctx* rep) {
  hc::BInst b{};
  b.gf = class_geo(c->gf, rep->gf);
  b.gfn = hc::col_narrow(b.gf);
  b.gd = class_geo(c->gd, rep->gd);
  b.gq = class_geo(c->gq, rep->gq);
  b.st = c->st;
  b.p64 = c->p64;
  b.b64 = c->b64;
  b.r64 = c->r64;
  b.bq = c->bq;
  b.b32 = c->b32;
  b.r32 = c->r32;
  b.d32 = c->d32;
  b.q32 = c->q32;
  b.x32 = c->x32;
  b.G32 = c->G32;
  b.G64 = c->G64;
  b.mx = (float*)c->m[0];
  b.my = (float*)c->m[1];
  b.rf = (const float*)c->rf;
  b.ns = c->ns;
  b.cf = split_coef(c->prm);
  return b;
}

// Capture one size class's step into `target` as a chain with no dependencies
// on what `target` already holds (the batched counterpart of build_chain):
//   step_begin, FP32 residual, flags, WHILE(first){CG, flags},
//   IF(mid){double-float residual, flags, WHILE(mid_inner){CG, flags}},
//   WHILE(outer){FP64 residual, flags, WHILE(inner){CG, flags}}, split, step_end.
// Every conditional handle is created before the kernels that set it are
// captured; flags sets each to the OR over the members.
int build_class_chain(const BatchClass& bc, cudaStream_t s, cudaGraph_t target) {
  const hc::BInst* bi = bc.d_inst;
  const hc::BShape& sh = bc.sh;
  long long* cnt = bc.d_launches;
  Handles hh;
  auto handle = [&](cudaGraph_t g, cudaGraphConditionalHandle* hd) -> int {
    CU(cudaGraphConditionalHandleCreate(hd, g, 0, cudaGraphCondAssignDefault));
    return HC_OK;
  };
  auto begin = [&](cudaGraph_t g, const cudaGraphNode_t* deps, size_t nd) -> int {
    CU(cudaStreamBeginCaptureToGraph(s, g, deps, nullptr, nd, cudaStreamCaptureModeThreadLocal));
    return HC_OK;
  };
  auto end = [&](cudaGraph_t g, std::vector<cudaGraphNode_t>* tail) -> int {
    cudaStreamCaptureStatus cs;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    if (tail) {
      CU(cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &deps, nullptr, &nd));
      tail->assign(deps, deps + nd);
    }
    cudaGraph_t same = g;
    CU(cudaStreamEndCapture(s, &same));
    return HC_OK;
  };
  auto cond = [&](cudaGraph_t g, const std::vector<cudaGraphNode_t>& after,
                  cudaGraphConditionalHandle hd, bool is_if, cudaGraphNode_t* node,
                  cudaGraph_t* body) -> int {
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = hd;
    p.conditional.type = is_if ? cudaGraphCondTypeIf : cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    CU(cudaGraphAddNode(node, g, after.data(), nullptr, after.size(), &p));
    *body = p.conditional.phGraph_out[0];
    return HC_OK;
  };
  // the body of an inner CG loop driven by handle hd
  auto iter_body = [&](cudaGraph_t body, cudaGraphConditionalHandle hd) -> int {
    int rc = begin(body, nullptr, 0);
    if (rc) return rc;
    hc::batch_cg_iter(bi, sh, s);
    hc::batch_flags(bi, sh, hc::BF_LOOP, hd, 0, cnt, 5, s);
    return end(body, nullptr);
  };
  int rc = handle(target, &hh.outer);
  if (!rc) rc = handle(target, &hh.first);
  if (!rc) rc = handle(target, &hh.mid);
  if (rc) return rc;
  std::vector<cudaGraphNode_t> tail;
  rc = begin(target, nullptr, 0);
  if (rc) return rc;
  hc::batch_step_begin(bi, sh, hh.outer, s);
  hc::batch_first_resid(bi, sh, s);
  hc::batch_flags(bi, sh, hc::BF_FIRST, hh.first, hh.mid, cnt, 5, s);
  rc = end(target, &tail);
  if (rc) return rc;
  cudaGraphNode_t first_node, mid_node, outer_node, inode;
  cudaGraph_t body = nullptr, mbody = nullptr, obody = nullptr;
  rc = cond(target, tail, hh.first, false, &first_node, &body);
  if (!rc) rc = iter_body(body, hh.first);
  if (!rc) rc = cond(target, {first_node}, hh.mid, true, &mid_node, &mbody);
  if (!rc) rc = handle(mbody, &hh.mid_inner);
  if (!rc) rc = begin(mbody, nullptr, 0);
  if (rc) return rc;
  hc::batch_mid_resid(bi, sh, s);
  hc::batch_flags(bi, sh, hc::BF_LOOP, hh.mid_inner, 0, cnt, 4, s);
  std::vector<cudaGraphNode_t> mtail;
  rc = end(mbody, &mtail);
  if (!rc) rc = cond(mbody, mtail, hh.mid_inner, false, &inode, &body);
  if (!rc) rc = iter_body(body, hh.mid_inner);
  if (!rc) rc = cond(target, {mid_node}, hh.outer, false, &outer_node, &obody);
  if (!rc) rc = handle(obody, &hh.inner);
  if (!rc) rc = begin(obody, nullptr, 0);
  if (rc) return rc;
  hc::batch_refine_resid(bi, sh, s);
  hc::batch_flags(bi, sh, hc::BF_REFINE, hh.inner, hh.outer, cnt, 4, s);
  std::vector<cudaGraphNode_t> otail;
  rc = end(obody, &otail);
  if (!rc) rc = cond(obody, otail, hh.inner, false, &inode, &body);
  if (!rc) rc = iter_body(body, hh.inner);
  if (!rc) rc = begin(target, &outer_node, 1);
  if (rc) return rc;
  hc::batch_split(bi, sh, s);
  hc::batch_step_end(bi, sh, cnt, s);
  return end(target, nullptr);
}

}  // namespace

extern "C" {

int hc_batch_create(hc_batch** out, hc_ctx* const* ctxs, int count, void* stream) {
  if (!out || !ctxs || count < 1) return HC_EINVAL;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i]) return HC_EINVAL;
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == ctxs[i]) return HC_EINVAL;
  }
  hc_batch* b = new (std::nothrow) hc_batch;
  if (!b) return HC_ENOMEM;
  b->ctx.assign(ctxs, ctxs + count);
  b->h.assign(count, Handles{});
  b->cls_of.assign(count, -1);
  b->dmem = nullptr;
  b->stream = (cudaStream_t)stream;
  b->cap = nullptr;
  b->ready = false;
  auto fail = [&](int rc) {
    if (b->cap) {
      abort_capture(b->cap);
      cudaStreamDestroy(b->cap);
    }
    if (b->dmem) cudaFree(b->dmem);
    delete b;
    return rc;
  };
  // size classes: batchable contexts by grid size, two members at least
  for (int i = 0; i < count; ++i) {
    const hc_ctx* c = b->ctx[i];
    if (!batchable(c) || b->cls_of[i] >= 0) continue;
    BatchClass bc;
    for (int k = i; k < count; ++k) {
      const hc_ctx* o = b->ctx[k];
      if (batchable(o) && b->cls_of[k] < 0 && o->nx == c->nx && o->ny == c->ny)
        bc.members.push_back(k);
    }
    if (bc.members.size() < 2) continue;
    for (int k : bc.members) b->cls_of[k] = (int)b->cls.size();
    b->cls.push_back(bc);
  }
  if (!b->cls.empty()) {
    size_t bytes = 0;
    for (auto& bc : b->cls) bytes += 256 + bc.members.size() * sizeof(hc::BInst);
    if (cudaMalloc(&b->dmem, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(HC_ENOMEM);
    }
    if (cudaMemset(b->dmem, 0, bytes) != cudaSuccess) return fail(HC_ECUDA);
    char* p = static_cast<char*>(b->dmem);
    hc::set_smem_limits_batch();
    for (auto& bc : b->cls) {
      const hc_ctx* rep = b->ctx[bc.members[0]];
      bc.d_launches = reinterpret_cast<long long*>(p);
      bc.d_inst = reinterpret_cast<hc::BInst*>(p + 256);
      p += 256 + bc.members.size() * sizeof(hc::BInst);
      std::vector<hc::BInst> recs;
      for (int k : bc.members) recs.push_back(member_record(b->ctx[k], rep));
      if (cudaMemcpy(bc.d_inst, recs.data(), recs.size() * sizeof(hc::BInst),
                     cudaMemcpyHostToDevice) != cudaSuccess)
        return fail(HC_ECUDA);
      bc.sh.gf = recs[0].gf;
      bc.sh.gfn = recs[0].gfn;
      bc.sh.gd = recs[0].gd;
      bc.sh.gq = recs[0].gq;
      bc.sh.nb = (int)bc.members.size();
    }
    if (cudaGetLastError() != cudaSuccess) return fail(HC_ECUDA);
  }
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return fail(HC_ECUDA);
  cudaGraph_t graph;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return fail(HC_ECUDA);
  for (auto& bc : b->cls) {
    for (int k : bc.members)
      if (cudaStreamSynchronize(b->ctx[k]->stream) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return fail(HC_ECUDA);
      }
    int rc = build_class_chain(bc, b->cap, graph);
    if (rc) {
      cudaGraphDestroy(graph);
      return fail(rc);
    }
  }
  for (int i = 0; i < count; ++i) {
    if (b->cls_of[i] >= 0) continue;
    hc_ctx* c = b->ctx[i];
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) {
      cudaGraphDestroy(graph);
      return fail(HC_ECUDA);
    }
    cudaStream_t keep = c->stream;
    long long before = c->launches;
    c->stream = b->cap;
    int rc = build_chain(c, graph, &b->h[i]);
    c->stream = keep;
    c->launches = before;
    if (rc) {
      cudaGraphDestroy(graph);
      return fail(rc);
    }
  }
  cudaError_t e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    cuda_fail(e, "cudaGraphInstantiate", __LINE__);
    return fail(HC_ECUDA);
  }
  b->ready = true;
  *out = b;
  return HC_OK;
}

int hc_batch_step(hc_batch* b, int nsteps, hc_step_stats* stats) {
  if (!b || nsteps < 0) return HC_EINVAL;
  if (nsteps == 0) return HC_OK;
  const int n = (int)b->ctx.size();
  for (int i = 0; i < n; ++i) {
    hc_ctx* c = b->ctx[i];
    CU(cudaStreamSynchronize(c->stream));
    if (b->cls_of[i] < 0) {
      int rc = use_handles(c, b->h[i]);
      if (rc) return rc;
      c->batch_handles = 1;
      rc = set_graph_mode(c, 1);
      if (rc) return rc;
    } else {
      // a class member's own kernels leave the graph conditions alone
      int rc = set_graph_mode(c, 0);
      if (rc) return rc;
    }
    hc::reset_accum(c->st, b->stream);
    c->launches += 1;
  }
  for (int k = 0; k < nsteps; ++k) CU(cudaGraphLaunch(b->exec, b->stream));
  for (int i = 0; i < n; ++i)
    CU(cudaMemcpyAsync(b->ctx[i]->st_host, b->ctx[i]->st, sizeof(hc::SolveState),
                       cudaMemcpyDeviceToHost, b->stream));
  std::vector<long long> cls_launches(b->cls.size(), 0);
  for (size_t k = 0; k < b->cls.size(); ++k)
    CU(cudaMemcpyAsync(&cls_launches[k], b->cls[k].d_launches, sizeof(long long),
                       cudaMemcpyDeviceToHost, b->stream));
  CU(cudaStreamSynchronize(b->stream));
  // a class's launches are counted once, on its first member
  for (size_t k = 0; k < b->cls.size(); ++k) {
    BatchClass& bc = b->cls[k];
    b->ctx[bc.members[0]]->launches += cls_launches[k] - bc.launches_seen;
    bc.launches_seen = cls_launches[k];
  }
  int first_bad = HC_OK;
  for (int i = 0; i < n; ++i) {
    hc_ctx* c = b->ctx[i];
    const hc::SolveState& h = *c->st_host;
    if (b->cls_of[i] < 0) c->launches += graph_kernel_count(c, h);
    if (stats) fill_stats(c, &stats[i]);
    if (!first_bad && h.first_bad) first_bad = h.first_bad;
    int rc = set_graph_mode(c, 0);
    if (rc) return rc;
  }
  return first_bad;
}

void hc_batch_destroy(hc_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  if (b->ready) cudaGraphExecDestroy(b->exec);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->dmem) cudaFree(b->dmem);
  delete b;
}

int hc_batch_classes(const hc_batch* b, int* classes, int* batched_members) {
  if (!b || !classes || !batched_members) return HC_EINVAL;
  *classes = (int)b->cls.size();
  int m = 0;
  for (auto& bc : b->cls) m += (int)bc.members.size();
  *batched_members = m;
  return HC_OK;
}

int hc_get_tuning(const hc_ctx* c, hc_tuning* t) {
  if (!c || !t) return HC_EINVAL;
  t->col_tile[0] = c->gf.tc;
  t->col_tile[1] = c->gd.tc;
  t->row_rows[0] = c->gf.rpc;
  t->row_rows[1] = c->gd.rpc;
  t->col_pipe[0] = c->gf.pipe;
  t->col_pipe[1] = c->gd.pipe;
  t->row_pipe[0] = c->gf.rpipe;
  t->row_pipe[1] = 0;
  return HC_OK;
}

int hc_set_tuning(hc_ctx* c, const hc_tuning* t) {
  if (!c || !t) return HC_EINVAL;
  if (c->dim != 2 || c->gen) return HC_ENOTSUP;  // 3D and generic-size launch shapes are fixed
  int dev = 0, optin = 0;
  CU(cudaGetDevice(&dev));
  CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int lnx = ilog2(c->nx), lny = ilog2(c->ny);
  for (int p = 0; p < 2; ++p) {
    const int tc = t->col_tile[p], rpc = t->row_rows[p];
    const size_t esz = p == 0 ? sizeof(cx<float>) : sizeof(cx<double>);
    const int max_threads = p == 0 ? hc::col_cta_max<float, true>() : hc::col_cta_max<double, true>();
    if (tc < 1 || (tc & (tc - 1)) || tc > 32 || tc > c->H || (tc << (lny - 3)) > max_threads)
      return HC_EINVAL;
    if (rpc < 1 || (rpc & (rpc - 1)) || rpc > c->ny || (rpc << (lnx - 3)) > 512) return HC_EINVAL;
    const size_t col_sm = 2 * (size_t)(c->ny + (c->ny >> 3)) * tc * esz + 1024;
    // the apply row pass also stages m and r (FP32 unless plain FP64)
    const size_t msz = (p == 1 && !c->refined) ? sizeof(double) : sizeof(float);
    const size_t row_sm = (size_t)rpc * c->nx * (esz + 3 * msz) + 1024;
    if (col_sm > (size_t)optin || row_sm > (size_t)optin) return HC_EINVAL;
    if (t->col_pipe[p] < 0 || t->col_pipe[p] > 1) return HC_EINVAL;
    if (t->col_pipe[p]) {
      if ((tc * esz) % 16 && tc * esz != 8) return HC_EINVAL;  // 16-byte copies, or one FP32 column
      if (2 * col_sm > (size_t)optin) return HC_EINVAL;
    }
  }
  // persistent FP32 apply row pass: [0] only, and its two stage buffers must fit
  if (t->row_pipe[1] != 0 || t->row_pipe[0] < 0 || t->row_pipe[0] > 1) return HC_EINVAL;
  int rgrid = 0;
  if (t->row_pipe[0]) {
    const int rpc = t->row_rows[0];
    const size_t ps = hc::row_pipe_smem(rpc, c->nx);
    if (ps > (size_t)optin) return HC_EINVAL;
    const int per_sm = hc::row_pipe_ctas_per_sm(rpc << (lnx - 3), ps);
    if (per_sm < 1) return HC_EINVAL;
    int nsm0 = 0;
    CU(cudaDeviceGetAttribute(&nsm0, cudaDevAttrMultiProcessorCount, dev));
    rgrid = std::min(c->ny / rpc, nsm0 * per_sm);
  }
  int nsm = 0;
  CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  c->gf.tc = t->col_tile[0];
  c->gf.ltc = ilog2(t->col_tile[0]);
  c->gd.tc = t->col_tile[1];
  c->gd.ltc = ilog2(t->col_tile[1]);
  c->gf.rpc = t->row_rows[0];
  c->gf.lrpc = ilog2(t->row_rows[0]);
  c->gd.rpc = t->row_rows[1];
  c->gd.lrpc = ilog2(t->row_rows[1]);
  c->gf.pipe = t->col_pipe[0];
  c->gd.pipe = t->col_pipe[1];
  c->gf.rpipe = t->row_pipe[0];
  c->gf.rgrid = rgrid;
  c->gf.pgrid = std::min(nsm, c->H / c->gf.tc);
  c->gd.pgrid = std::min(nsm, c->H / c->gd.tc);
  c->gq.tc = c->gd.tc;
  c->gq.ltc = c->gd.ltc;
  c->gq.rpc = c->gd.rpc;
  c->gq.lrpc = c->gd.lrpc;
  c->gq.pipe = c->gd.pipe;
  c->gq.pgrid = c->gd.pgrid;
  drop_graphs(c);  // launch shapes are baked into the graphs
  return HC_OK;
}

int hc_time_kernel(hc_ctx* c, int kernel, int reps, double* ms_per_launch) {
  if (!c || !ms_per_launch || reps < 1 || kernel < 0 || kernel >= HC_K_COUNT) return HC_EINVAL;
  if (c->gen) return HC_ENOTSUP;
  // scratch state: loop open, nothing converges, zero step lengths so the
  // repeated launches leave their inputs unchanged
  hc::SolveState init;
  CU(cudaMemcpyAsync(&init, c->st, sizeof(init), cudaMemcpyDeviceToHost, c->stream));
  CU(cudaStreamSynchronize(c->stream));
  init.done = 0;
  init.first = 1;
  init.alpha = 0;
  init.beta = 0;
  init.rho = 0;  // alpha = rho / <d, A d> stays 0 whichever kernel computes it
  init.maxit = 0x7fffffff;
  init.thresh2 = -1.0;
  init.outer_thresh2 = -1.0;
  init.max_sweeps = 0x7fffffff;
  init.graph_mode = 0;
  for (int k = 0; k < 8; ++k) init.ticket[k] = 0;
  CU(cudaMemcpyAsync(c->st_time, &init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
  hc::SolveState* ts = c->st_time;
  const size_t ns = c->ns;
  if (c->dim == 2 && (kernel == HC_K_CG_YPASS || kernel == HC_K_RES_YPASS)) return HC_EINVAL;
  if (!c->refined && kernel >= HC_K_FIRST_GRAD) return HC_EINVAL;
  if (kernel >= HC_K_MID_GRAD && (c->df || !c->refined)) return HC_EINVAL;  // HC_FP32_REFINED only
  if (c->dim == 2 && kernel == HC_K_MID_YPASS) return HC_EINVAL;
  // 3D: the same roles with the 3D kernels; the SPLIT_HEAT / SPLIT_C2R slots
  // time the y and z diffusion passes.  Scratch outputs never alias inputs
  // that a later repetition reads.
  auto launch3 = [&]() {
    const hc::SplitCoef cf = split_coef(c->prm);
    if (c->refined) {
      auto& g = c->gf;
      auto G = tri(c->G32, ns);
      auto* G64 = c->G64;
      auto mw = hc::Tri<float*>{{(float*)c->q32, (float*)c->x32, (float*)c->d32}};
      switch (kernel) {
        case HC_K_CG_GRAD:
          hc::z_grad<float, float>(g, hc::CG_DUPDATE, (cx<float>*)nullptr, c->r32, c->d32, nullptr,
                                   G, ts, 1, c->stream);
          break;
        case HC_K_CG_YPASS:
          hc::axis_fft<float>(g, 1, +1, 3, G, G, 1.0f, c->stream);
          break;
        case HC_K_CG_APPLY:
          hc::row_apply3<float, float>(g, G, mtri<float>(c), (const float*)c->rf, G, ts, c->stream);
          break;
        case HC_K_CG_DIV:
          hc::z_div<float>(g, hc::CD_CG, G, c->d32, nullptr, c->q32, nullptr, nullptr, ts, c->stream);
          break;
        case HC_K_CG_UPDATE:
          hc::cg_update3<float>(g, c->x32, c->r32, c->d32, c->q32, ts, c->stream);
          break;
        case HC_K_RES_GRAD:
          if (c->df)
            hc::z_grad<df64, df64>(c->gq, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64),
                                   nullptr, nullptr, nullptr, tri((cx<df64>*)G64, ns), ts, 0,
                                   c->stream);
          else
            hc::z_grad<double, double>(c->gd, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr,
                                       tri(G64, ns), ts, 0, c->stream);
          break;
        case HC_K_RES_YPASS:
          if (c->df)
            hc::axis_fft<df64>(c->gq, 1, +1, 3, tri((cx<df64>*)G64, ns), tri((cx<df64>*)G64, ns),
                               df64(1.0), c->stream);
          else
            hc::axis_fft<double>(c->gd, 1, +1, 3, tri(G64, ns), tri(G64, ns), 1.0, c->stream);
          break;
        case HC_K_RES_APPLY:
          if (c->df)
            hc::row_apply3<df64, float>(c->gq, tri((cx<df64>*)G64, ns), mtri<float>(c),
                                        (const float*)c->rf, tri((cx<df64>*)G64, ns), nullptr,
                                        c->stream);
          else
            hc::row_apply3<double, float>(c->gd, tri(G64, ns), mtri<float>(c), (const float*)c->rf,
                                          tri(G64, ns), nullptr, c->stream);
          break;
        case HC_K_RES_DIV:
          if (c->df)
            hc::z_div<df64>(c->gq, hc::CD_RESID_REFINE, tri((cx<df64>*)G64, ns), nullptr,
                            (const cx<df64>*)c->b64, (cx<df64>*)c->r64, c->d32, c->q32, ts,
                            c->stream);
          else
            hc::z_div<double>(c->gd, hc::CD_RESID_REFINE, tri(G64, ns), nullptr, c->b64, c->r64,
                              c->d32, c->q32, ts, c->stream);
          break;
        case HC_K_SPLIT_GRAD:
          hc::z_grad<float, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, G, ts, 0,
                                    c->stream);
          break;
        case HC_K_SPLIT_ROW:
          hc::row_split3<float>(g, G, mtri<float>(c), (const float*)c->rf, mw, cf, ts, c->stream);
          break;
        case HC_K_SPLIT_HEAT:
          hc::heat_axis<float>(g, 1, mw, mw, ts, c->stream);
          break;
        case HC_K_FIRST_GRAD:
          if (c->df)
            hc::z_grad<float, df64>(g, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64), nullptr,
                                    nullptr, nullptr, G, ts, 0, c->stream);
          else
            hc::z_grad<float, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, G, ts, 0,
                                      c->stream);
          break;
        case HC_K_FIRST_APPLY:
          hc::row_apply3<float, float>(g, G, mtri<float>(c), (const float*)c->rf, G, nullptr,
                                       c->stream);
          break;
        case HC_K_FIRST_DIV:
          hc::z_div<float>(g, hc::CD_RESID_FIRST, G, nullptr, c->b32, nullptr, c->d32, c->q32, ts,
                           c->stream);
          break;
        case HC_K_MID_GRAD:
          hc::z_grad<df64, double>(c->gq, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr,
                                   tri((cx<df64>*)G64, ns), ts, 0, c->stream);
          break;
        case HC_K_MID_YPASS:
          hc::axis_fft<df64>(c->gq, 1, +1, 3, tri((cx<df64>*)G64, ns), tri((cx<df64>*)G64, ns),
                             df64(1.0), c->stream);
          break;
        case HC_K_MID_APPLY:
          hc::row_apply3<df64, float>(c->gq, tri((cx<df64>*)G64, ns), mtri<float>(c),
                                      (const float*)c->rf, tri((cx<df64>*)G64, ns), nullptr, c->stream);
          break;
        case HC_K_MID_DIV:
          hc::z_div<df64>(c->gq, hc::CD_RESID_REFINE, tri((cx<df64>*)G64, ns), nullptr, c->bq, nullptr,
                          c->d32, c->q32, ts, c->stream);
          break;
        default:
          hc::heat_axis<float>(g, 2, mw, mw, ts, c->stream);
          break;
      }
    } else {
      auto& g = c->gd;
      auto G = tri(c->G64, ns);
      // scratch m: the direction/product vectors (3 * ns complex doubles >= 3n doubles? no: use
      // stage, which holds 3n doubles)
      auto mw = hc::Tri<double*>{{c->stage, c->stage + c->n, c->stage + 2 * c->n}};
      switch (kernel) {
        case HC_K_CG_GRAD:
          hc::z_grad<double, double>(g, hc::CG_DUPDATE, (cx<double>*)nullptr, c->r64, c->d64,
                                     nullptr, G, ts, 1, c->stream);
          break;
        case HC_K_CG_YPASS:
        case HC_K_RES_YPASS:
          hc::axis_fft<double>(g, 1, +1, 3, G, G, 1.0, c->stream);
          break;
        case HC_K_CG_APPLY:
          hc::row_apply3<double, double>(g, G, mtri<double>(c), (const double*)c->rf, G, ts,
                                         c->stream);
          break;
        case HC_K_CG_DIV:
          hc::z_div<double>(g, hc::CD_CG, G, c->d64, nullptr, c->q64, nullptr, nullptr, ts,
                            c->stream);
          break;
        case HC_K_CG_UPDATE:
          hc::cg_update3<double>(g, c->b64, c->r64, c->d64, c->q64, ts, c->stream);
          break;
        case HC_K_RES_GRAD:
        case HC_K_SPLIT_GRAD:
          hc::z_grad<double, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, G, ts, 0,
                                     c->stream);
          break;
        case HC_K_RES_APPLY:
          hc::row_apply3<double, double>(g, G, mtri<double>(c), (const double*)c->rf, G, nullptr,
                                         c->stream);
          break;
        case HC_K_RES_DIV:
          hc::z_div<double>(g, hc::CD_RESID, G, nullptr, c->b64, c->q64, nullptr, nullptr, ts,
                            c->stream);
          break;
        case HC_K_SPLIT_ROW:
          hc::row_split3<double>(g, G, mtri<double>(c), (const double*)c->rf, mw, cf, ts,
                                 c->stream);
          break;
        case HC_K_SPLIT_HEAT:
          hc::heat_axis<double>(g, 1, mw, mw, ts, c->stream);
          break;
        default:
          hc::heat_axis<double>(g, 2, mw, mw, ts, c->stream);
          break;
      }
    }
  };
  auto launch = [&]() {
    if (c->dim == 3) {
      launch3();
      return;
    }
    if (c->refined) {
      auto& g = c->gf;
      auto& gd = c->gd;
      cx<float>*Gx = c->G32, *Gy = c->G32 + ns;
      cx<double>*Gx64 = c->G64, *Gy64 = c->G64 + ns;
      switch (kernel) {
        case HC_K_CG_GRAD:
          hc::col_grad<float, float>(g, hc::CG_DUPDATE, (cx<float>*)nullptr, c->r32, c->d32, nullptr,
                                     Gx, Gy, ts, 1, c->stream);
          break;
        case HC_K_CG_APPLY:
          hc::row_apply<float, float>(g, Gx, Gy, (const float*)c->m[0], (const float*)c->m[1],
                                      (const float*)c->rf, c->q32, c->x32, ts, c->stream);
          break;
        case HC_K_CG_DIV:
          hc::col_div<float>(g, hc::CD_CG, Gx, Gy, c->d32, nullptr, c->q32, nullptr, nullptr, ts,
                             c->stream);
          break;
        case HC_K_CG_UPDATE:
          hc::cg_update<float>(g, c->x32, c->r32, c->d32, c->q32, ts, c->stream);
          break;
        case HC_K_RES_GRAD:
          if (c->df)
            hc::col_grad<df64, df64>(c->gq, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64),
                                     nullptr, nullptr, nullptr, (cx<df64>*)Gx64, (cx<df64>*)Gy64, ts,
                                     0, c->stream);
          else
            hc::col_grad<double, double>(gd, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gx64,
                                         Gy64, ts, 0, c->stream);
          break;
        case HC_K_RES_APPLY:
          if (c->df)
            hc::row_apply<df64, float>(c->gq, (cx<df64>*)Gx64, (cx<df64>*)Gy64,
                                       (const float*)c->m[0], (const float*)c->m[1],
                                       (const float*)c->rf, (cx<df64>*)c->r64,
                                       (cx<df64>*)c->stage, nullptr, c->stream);
          else
            hc::row_apply<double, float>(gd, Gx64, Gy64, (const float*)c->m[0],
                                         (const float*)c->m[1], (const float*)c->rf, c->r64,
                                         (cx<double>*)c->stage, nullptr, c->stream);
          break;
        case HC_K_RES_DIV:
          if (c->df)
            hc::col_div<df64>(c->gq, hc::CD_RESID_REFINE, (cx<df64>*)Gx64, (cx<df64>*)Gy64,
                              nullptr, (const cx<df64>*)c->b64, (cx<df64>*)c->r64, c->d32, c->q32,
                              ts, c->stream);
          else
            hc::col_div<double>(gd, hc::CD_RESID_REFINE, Gx64, Gy64, nullptr, c->b64, c->r64,
                                c->d32, c->q32, ts, c->stream);
          break;
        case HC_K_SPLIT_GRAD:
          if (c->df)
            hc::col_grad<float, df64>(g, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64), nullptr,
                                      nullptr, nullptr, Gx, Gy, ts, 0, c->stream);
          else
            hc::col_grad<float, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gx, Gy,
                                        ts, 0, c->stream);
          break;
        case HC_K_SPLIT_ROW:
          hc::row_split<float>(g, Gx, Gy, (const float*)c->m[0], (const float*)c->m[1],
                               (const float*)c->rf, c->q32, c->x32,
                               split_coef(c->prm), ts, c->stream);
          break;
        case HC_K_SPLIT_HEAT:  // on scratch: each launch rescales its data
          hc::col_heat<float>(g, c->q32, c->x32, ts, c->stream);
          break;
        case HC_K_FIRST_GRAD:
          if (c->df)
            hc::col_grad<float, df64>(g, hc::CG_PLAIN, reinterpret_cast<cx<df64>*>(c->p64), nullptr,
                                      nullptr, nullptr, Gx, Gy, ts, 0, c->stream);
          else
            hc::col_grad<float, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gx, Gy,
                                        ts, 0, c->stream);
          break;
        case HC_K_FIRST_APPLY:
          hc::row_apply<float, float>(g, Gx, Gy, (const float*)c->m[0], (const float*)c->m[1],
                                      (const float*)c->rf, c->q32, c->x32, nullptr, c->stream);
          break;
        case HC_K_FIRST_DIV:
          hc::col_div<float>(g, hc::CD_RESID_FIRST, Gx, Gy, nullptr, c->b32, nullptr, c->d32, c->q32,
                             ts, c->stream);
          break;
        case HC_K_MID_GRAD:
          hc::col_grad<df64, double>(c->gq, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr,
                                     (cx<df64>*)Gx64, (cx<df64>*)Gy64, ts, 0, c->stream);
          break;
        case HC_K_MID_APPLY:
          hc::row_apply<df64, float>(c->gq, (cx<df64>*)Gx64, (cx<df64>*)Gy64, (const float*)c->m[0],
                                     (const float*)c->m[1], (const float*)c->rf, (cx<df64>*)c->r64,
                                     (cx<df64>*)c->stage, nullptr, c->stream);
          break;
        case HC_K_MID_DIV:
          hc::col_div<df64>(c->gq, hc::CD_RESID_REFINE, (cx<df64>*)Gx64, (cx<df64>*)Gy64, nullptr,
                            c->bq, nullptr, c->d32, c->q32, ts, c->stream);
          break;
        default:
          hc::row_c2r<float>(g, Gx, Gy, (float*)c->q32, (float*)c->x32, ts, 1, c->stream);
          break;
      }
    } else {
      auto& g = c->gd;
      cx<double>*Gx = c->G64, *Gy = c->G64 + ns;
      double* sx = c->stage;
      double* sy = c->stage + c->n;
      switch (kernel) {
        case HC_K_CG_GRAD:
          hc::col_grad<double, double>(g, hc::CG_DUPDATE, (cx<double>*)nullptr, c->r64, c->d64,
                                       nullptr, Gx, Gy, ts, 1, c->stream);
          break;
        case HC_K_CG_APPLY:
          hc::row_apply<double, double>(g, Gx, Gy, (const double*)c->m[0], (const double*)c->m[1],
                                        (const double*)c->rf, c->q64, (cx<double>*)c->stage, ts,
                                        c->stream);
          break;
        case HC_K_CG_DIV:
          hc::col_div<double>(g, hc::CD_CG, Gx, Gy, c->d64, nullptr, c->q64, nullptr, nullptr, ts,
                              c->stream);
          break;
        case HC_K_CG_UPDATE:
          hc::cg_update<double>(g, (cx<double>*)c->stage, c->r64, c->d64,
                                c->q64, ts, c->stream);
          break;
        case HC_K_RES_GRAD:
        case HC_K_SPLIT_GRAD:
          hc::col_grad<double, double>(g, hc::CG_PLAIN, c->p64, nullptr, nullptr, nullptr, Gx, Gy, ts,
                                       0, c->stream);
          break;
        case HC_K_RES_APPLY:
          hc::row_apply<double, double>(g, Gx, Gy, (const double*)c->m[0], (const double*)c->m[1],
                                        (const double*)c->rf, c->q64, (cx<double>*)c->stage, nullptr,
                                        c->stream);
          break;
        case HC_K_RES_DIV:
          hc::col_div<double>(g, hc::CD_RESID, Gx, Gy, nullptr, c->b64, c->q64, nullptr, nullptr, ts,
                              c->stream);
          break;
        case HC_K_SPLIT_ROW:
          hc::row_split<double>(g, Gx, Gy, (const double*)c->m[0], (const double*)c->m[1],
                                (const double*)c->rf, c->q64,
                                (cx<double>*)c->stage, split_coef(c->prm), ts, c->stream);
          break;
        case HC_K_SPLIT_HEAT:  // on scratch: each launch rescales its data
          hc::col_heat<double>(g, c->q64, (cx<double>*)c->stage, ts, c->stream);
          break;
        default:
          hc::row_c2r<double>(g, Gx, Gy, sx, sy, ts, 1, c->stream);
          break;
      }
    }
  };
  launch();  // warm-up
  CU(cudaGetLastError());
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  CU(cudaEventRecord(e0, c->stream));
  for (int k = 0; k < reps; ++k) launch();
  CU(cudaEventRecord(e1, c->stream));
  CU(cudaEventSynchronize(e1));
  float ms = 0;
  CU(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  CU(cudaGetLastError());
  c->launches += reps + 1;
  *ms_per_launch = (double)ms / reps;
  return HC_OK;
}

int hc_launch_count(const hc_ctx* c, long long* count) {
  if (!c || !count) return HC_EINVAL;
  *count = c->launches;
  return HC_OK;
}

int hc_fp64_fma_peak(int reps, void* stream, double* tflops) {
  if (!tflops || reps < 1) return HC_EINVAL;
  return hc::fma_peak(reps, (cudaStream_t)stream, tflops);
}

}  // extern "C"
