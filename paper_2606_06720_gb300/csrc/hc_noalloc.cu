// hc_noalloc.cu -- hc_spectrum_noalloc: the forward 2D transform of
// hc_spectrum without any device allocation.
//
// Who needs it: code that must not allocate device memory, for instance a
// plugin living inside a host framework that reserves the whole GPU for its
// own pool allocator, or a latency-critical loop where cudaMalloc's implicit
// device synchronisation is not acceptable.  Such callers own their input and
// output buffers but cannot provide the transform's scratch (the row-pass
// intermediate and the twiddle tables).  Here that scratch is one file-scope
// static device array of fixed size, so it exists in every process that loads
// the library, on every GPU the process uses, until the process exits.
//
// The kernels are the library's own row and column FFT passes, launched on
// the static scratch instead of a context workspace.
#include <cuda_runtime.h>

#include <mutex>

#include "hc.h"
#include "hc_kernels.cuh"

namespace {

using hc::cx;

constexpr int kMaxDevices = 64;
constexpr size_t kInterBytes = (size_t)HC_NOALLOC_MAX_POINTS / 2 * sizeof(cx<double>);
constexpr size_t kTwBytes = 4096 * sizeof(cx<double>);

// Row-transformed intermediate (ny * nx/2 complex doubles at most) followed by
// the twiddle tables of the x and y lengths (4096 entries each at most).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kInterBytes + 2 * kTwBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices];  // device address of g_noalloc_scratch per device (set-up done)

// tw[m] = exp(-2 pi i m / N), m < N.
__global__ void k_noalloc_twiddles(cx<double>* tw, int N) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= N) return;
  double s, c;
  sincospi(2.0 * (double)m / (double)N, &s, &c);
  tw[m].x = c;
  tw[m].y = -s;
}

int ilog2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

bool pow2_in(int v, int lo, int hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

// One-time set-up per device: the device address of the static scratch (the
// host-side symbol is only a stand-in) and the shared-memory opt-in of the
// two kernels launched here.
int setup_device(int dev, void** addr) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return HC_EINVAL;
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return HC_ECUDA;
    cudaGetLastError();  // a pending error of earlier work is not this set-up's
    hc::allow_smem(hc::k_row_r2c<double>);
    hc::allow_smem(hc::k_col_fwd<double, 1>);
    if (cudaGetLastError() != cudaSuccess) return HC_ECUDA;
    g_addr[dev] = p;
  }
  *addr = g_addr[dev];
  return HC_OK;
}

}  // namespace

extern "C" int hc_spectrum_noalloc(const double* f, double* out, int nx, int ny, void* stream) {
  if (!f || !out) return HC_EINVAL;
  if (!pow2_in(nx, 8, 4096) || !pow2_in(ny, 8, 4096)) return HC_EINVAL;
  if ((size_t)nx * (size_t)ny > (size_t)HC_NOALLOC_MAX_POINTS) return HC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HC_ECUDA;
  void* base = nullptr;
  int rc = setup_device(dev, &base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  // A non-sticky error left pending on this thread by earlier work (the
  // caller's or another library's) is consumed here, so that the check after
  // the launches reports only this call's own launches.
  cudaGetLastError();
  unsigned char* b = static_cast<unsigned char*>(base);
  cx<double>* inter = reinterpret_cast<cx<double>*>(b);
  cx<double>* twx = reinterpret_cast<cx<double>*>(b + kInterBytes);
  cx<double>* twy = reinterpret_cast<cx<double>*>(b + kInterBytes + kTwBytes);

  hc::Geo<double> g = {};
  g.nx = nx;
  g.ny = ny;
  g.H = nx / 2;
  g.lnx = ilog2i(nx);
  g.lny = ilog2i(ny);
  g.lH = ilog2i(nx / 2);
  int tc = 512 >> (g.lny - 3);
  tc = tc < 1 ? 1 : (tc > 32 ? 32 : tc);
  if (tc > g.H) tc = g.H;
  g.tc = tc;
  g.ltc = ilog2i(tc);
  int rpc = 256 >> (g.lnx - 3);
  rpc = rpc < 1 ? 1 : rpc;
  if (rpc > ny) rpc = ny;
  g.rpc = rpc;
  g.lrpc = ilog2i(rpc);
  g.twx = twx;
  g.twy = twy;

  // Every call rewrites the tables and the whole intermediate before reading
  // them, so nothing carried over from an earlier call is used.
  k_noalloc_twiddles<<<(nx + 255) / 256, 256, 0, s>>>(twx, nx);
  k_noalloc_twiddles<<<(ny + 255) / 256, 256, 0, s>>>(twy, ny);
  hc::k_row_r2c<double><<<ny >> g.lrpc, rpc << (g.lnx - 3), (size_t)rpc * nx * sizeof(cx<double>), s>>>(
      g, f, nullptr, inter, nullptr);
  hc::k_col_fwd<double, 1><<<g.H >> g.ltc, tc << (g.lny - 3),
                             (size_t)(ny + (ny >> 3)) * tc * sizeof(cx<double>), s>>>(
      g, inter, nullptr, reinterpret_cast<cx<double>*>(out), nullptr, 0, nullptr);
  if (cudaGetLastError() != cudaSuccess) return HC_ECUDA;
  return HC_OK;
}
