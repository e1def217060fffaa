// FP64 instantiations of the step kernels and the one-thread solve bookkeeping.
#include "hc_kernels.cuh"

namespace hc {

template void row_r2c<double>(const Geo<double>&, const double*, const double*, cx<double>*,
                              cx<double>*, cudaStream_t);
template void row_c2r<double>(const Geo<double>&, const cx<double>*, const cx<double>*, double*,
                              double*, SolveState*, int, cudaStream_t);
template void row_apply<double, double>(const Geo<double>&, const cx<double>*, const cx<double>*,
                                        const double*, const double*, const double*, cx<double>*,
                                        cx<double>*, SolveState*, cudaStream_t);
template void row_apply<double, float>(const Geo<double>&, const cx<double>*, const cx<double>*,
                                       const float*, const float*, const float*, cx<double>*,
                                       cx<double>*, SolveState*, cudaStream_t);
template void row_split<double>(const Geo<double>&, const cx<double>*, const cx<double>*, const double*,
                               const double*, const double*, cx<double>*, cx<double>*, SplitCoef, SolveState*,
                               cudaStream_t);
template void col_fwd<double>(const Geo<double>&, const cx<double>*, const cx<double>*, cx<double>*,
                              cx<double>*, int, int, SolveState*, cudaStream_t);
template void col_inv<double>(const Geo<double>&, const cx<double>*, cx<double>*, double,
                              cudaStream_t);
template void col_grad<double, double>(const Geo<double>&, int, cx<double>*, const cx<double>*,
                                       cx<double>*, const cx<float>*, cx<double>*, cx<double>*,
                                       SolveState*, int, cudaStream_t);
template void col_div<double>(const Geo<double>&, int, const cx<double>*, const cx<double>*,
                              const cx<double>*, const cx<double>*, cx<double>*, cx<float>*,
                              cx<float>*, SolveState*, cudaStream_t);
template void col_heat<double>(const Geo<double>&, cx<double>*, cx<double>*, SolveState*, cudaStream_t);
template void col_gradnorm<double>(const Geo<double>&, const cx<double>*, const cx<double>*, SolveState*, int,
                                 cudaStream_t);
template void cg_update<double>(const Geo<double>&, cx<double>*, cx<double>*, const cx<double>*,
                                const cx<double>*, SolveState*, cudaStream_t);
template void convert<double, float>(const float*, double*, size_t, cudaStream_t);
template void convert<float, double>(const double*, float*, size_t, cudaStream_t);
template void convert<double, double>(const double*, double*, size_t, cudaStream_t);
template void msum<double>(const Geo<double>&, const double*, const double*, SolveState*,
                           cudaStream_t);

template void row_adj_point<double>(const Geo<double>&, cx<double>*, cx<double>*, const cx<double>*, const cx<double>*,
                                const double*, const double*, double*, double*, SplitCoef, AdjState*, cudaStream_t);
template void row_adj_press<double>(const Geo<double>&, const cx<double>*, const cx<double>*, const cx<double>*,
                                const cx<double>*, const double*, const double*, const double*, const double*, double*,
                                double*, double*, cudaStream_t);
template void col_lap_dot<double>(const Geo<double>&, const cx<double>*, const cx<double>*, double, AdjState*,
                              cudaStream_t);
template void spec_accum<double>(const Geo<double>&, double*, const cx<double>*, cudaStream_t);
template void spec_norm2<double>(const Geo<double>&, const cx<double>*, SolveState*, cudaStream_t);

// FP64 residual S - A p of a certification (lagged certification): the
// pressure p and the m it was solved with are the caller's; the state sc
// skips it when nothing awaits certification (sc->done) and receives
// ||S - A p||^2 in sc->cert_r2.  Non-persistent passes, nothing else written.
void cert_resid(const Geo<double>& g, const cx<double>* p, const float* mx, const float* my,
                const float* r, const cx<double>* b, cx<double>* G, SolveState* sc, cudaStream_t s) {
  const int nb = g.H >> g.ltc, nt = col_threads(g);
  const size_t ns = (size_t)g.ny * g.H;
  cx<double>* Gx = G;
  cx<double>* Gy = G + ns;
  k_col_grad<double, double, CG_PLAIN><<<nb, nt, col_smem(g, 2), s>>>(
      g, const_cast<cx<double>*>(p), nullptr, nullptr, nullptr, Gx, Gy, sc, 1);
  const size_t sm = row_smem(g) + (size_t)3 * g.rpc * g.nx * sizeof(float);
  k_row_apply<double, float, false, 1><<<g.ny >> g.lrpc, row_threads(g), sm, s>>>(g, Gx, Gy, mx, my, r,
                                                                                 Gx, Gy, sc);
  k_col_div<double, CD_CERT><<<nb, nt, col_smem(g, 2), s>>>(g, Gx, Gy, nullptr, b, nullptr, nullptr,
                                                             nullptr, sc);
}

void set_smem_limits_f64() {
  allow_smem(k_col_div<double, CD_CERT>);
  set_smem_limits_t<double>();
  set_smem_limits_grad<double, double>();
  allow_smem(k_row_apply<double, float, false, 1>);
  allow_smem(k_row_apply<double, float, true, 1>);
}

__global__ void k_set_config(SolveState* st, SolveConfig c) {
  st->e_coef[0] = c.e_coef[0];
  st->e_coef[1] = c.e_coef[1];
  st->e_coef[2] = c.e_coef[2];
  st->dt = c.dt;
  st->first32_min2 = c.first32_min2;
  st->mid_df = c.mid_df;
  st->precond = c.precond;
  st->dim = c.dim;
  st->diag = c.diag;
  st->outer_rtol2 = c.outer_thresh2_rel;
  st->inner_rtol2 = c.inner_rtol2;
  st->user_kappa = c.user_kappa;
  st->mean_r = c.mean_r;
  st->maxit = c.maxit;
  st->max_sweeps = c.max_sweeps;
  st->graph_mode = c.graph_mode;
  st->refined = c.refined;
}

__global__ void k_step_begin(SolveState* st, int npts) { step_begin_body(st, npts); }

__global__ void k_step_end(SolveState* st, int refined) { step_end_body(st, refined); }

__global__ void k_set_run(SolveState* st, int run_mode, double eps_dm, int stop_energy) {
  st->run_mode = run_mode;
  st->eps_dm = eps_dm;
  st->stop_energy = stop_energy;
  st->halt = 0;
  st->stop_reason = HC_STOP_NONE;
  st->energy_step = -1;
  st->n_energy = 0;
}

__global__ void k_run_gate(SolveState* st) {
  cudaGraphSetConditional(st->h_gate, st->halt ? 0u : 1u);
}

__global__ void k_reset_accum(SolveState* st) {
  st->acc_first = 0;
  st->acc_mid = 0;
  st->acc_res_full = 0;
  st->first_bad = 0;
  st->acc_iters = 0;
  st->acc_sweeps = 0;
  st->acc_steps = 0;
}

void set_config(SolveState* st, SolveConfig cfg, cudaStream_t s) { k_set_config<<<1, 1, 0, s>>>(st, cfg); }
void step_begin(SolveState* st, int npts, cudaStream_t s) { k_step_begin<<<1, 1, 0, s>>>(st, npts); }
void step_end(SolveState* st, int refined, cudaStream_t s) { k_step_end<<<1, 1, 0, s>>>(st, refined); }
void reset_accum(SolveState* st, cudaStream_t s) { k_reset_accum<<<1, 1, 0, s>>>(st); }
void set_run(SolveState* st, int run_mode, double eps_dm, int stop_energy, cudaStream_t s) {
  k_set_run<<<1, 1, 0, s>>>(st, run_mode, eps_dm, stop_energy);
}
void run_gate(SolveState* st, cudaStream_t s) { k_run_gate<<<1, 1, 0, s>>>(st); }

// FP64 FMA throughput probe (the ALU roof of the FP64 residual kernels).  Each
// thread runs 8 independent chains a = a b + c, enough independent work to
// keep the FP64 pipe busy; the sink store never happens but keeps the chains
// live.  b slightly below 1 keeps the values bounded and normal.
__device__ double g_fma_sink;
__global__ void __launch_bounds__(256) k_fma_peak(int iters, double b, double c) {
  double a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = 1e-3 * (double)(threadIdx.x + i);
#pragma unroll 4
  for (int k = 0; k < iters; ++k)
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], b, c);
  double t = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) t += a[i];
  if (t == -1.0) g_fma_sink = t;
}

int fma_peak(int reps, cudaStream_t s, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return HC_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return HC_ECUDA;
  const int blocks = sms * 8, threads = 256, iters = 4096;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return HC_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return HC_ECUDA;
  }
  // the fastest of `reps` timed launches after two warm-up launches: a peak,
  // so a launch slowed while the clocks ramp up does not lower it
  k_fma_peak<<<blocks, threads, 0, s>>>(iters, 0.9999999, 1e-7);
  k_fma_peak<<<blocks, threads, 0, s>>>(iters, 0.9999999, 1e-7);
  float best = 0.f;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    cudaEventRecord(e0, s);
    k_fma_peak<<<blocks, threads, 0, s>>>(iters, 0.9999999, 1e-7);
    cudaEventRecord(e1, s);
    float ms = 0.f;
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms > 0.f && (best == 0.f || ms < best)) best = ms;
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess || !(best > 0.f)) return HC_ECUDA;
  const double flops = 2.0 * 8.0 * iters * (double)blocks * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  return HC_OK;
}

}  // namespace hc
