// FP64 instantiations of the step kernels and the one-thread solve bookkeeping.
#include "hc_kernels.cuh"

namespace hc {

template void row_r2c<double>(const Geo<double>&, const double*, const double*, cx<double>*,
                              cx<double>*, cudaStream_t);
template void row_c2r<double>(const Geo<double>&, const cx<double>*, const cx<double>*, double*,
                              double*, SolveState*, int, cudaStream_t);
template void row_apply<double, double>(const Geo<double>&, const cx<double>*, const cx<double>*,
                                        const double*, const double*, const double*, cx<double>*,
                                        cx<double>*, const SolveState*, cudaStream_t);
template void row_apply<double, float>(const Geo<double>&, const cx<double>*, const cx<double>*,
                                       const float*, const float*, const float*, cx<double>*,
                                       cx<double>*, const SolveState*, cudaStream_t);
template void row_split<double>(const Geo<double>&, const cx<double>*, const cx<double>*,
                                const double*, const double*, cx<double>*, cx<double>*, SplitCoef,
                                SolveState*, cudaStream_t);
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
template void col_heat<double>(const Geo<double>&, cx<double>*, cx<double>*, cudaStream_t);
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

void set_smem_limits_f64() {
  set_smem_limits_t<double>();
  set_smem_limits_grad<double, double>();
  allow_smem(k_row_apply<double, float>);
}

__global__ void k_set_config(SolveState* st, SolveConfig c) {
  st->outer_rtol2 = c.outer_thresh2_rel;
  st->inner_rtol2 = c.inner_rtol2;
  st->user_kappa = c.user_kappa;
  st->mean_r = c.mean_r;
  st->maxit = c.maxit;
  st->max_sweeps = c.max_sweeps;
  st->graph_mode = c.graph_mode;
  st->refined = c.refined;
}

__global__ void k_step_begin(SolveState* st, int npts) {
  st->kappa = st->user_kappa > 0 ? st->user_kappa : st->mean_r + st->msum / (double)npts / 2.0;
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
  if (st->graph_mode && st->refined) cudaGraphSetConditional(st->h_outer, 1u);
}

__global__ void k_step_end(SolveState* st, int refined) {
  const int status = st->nonfinite ? HC_ENONFINITE : st->status;
  st->step_status = status;
  if (!st->first_bad && status) st->first_bad = status;
  st->acc_iters += st->total_it;
  st->acc_sweeps += st->sweeps;
  st->acc_steps += 1;
}

__global__ void k_reset_accum(SolveState* st) {
  st->first_bad = 0;
  st->acc_iters = 0;
  st->acc_sweeps = 0;
  st->acc_steps = 0;
}

void set_config(SolveState* st, SolveConfig cfg, cudaStream_t s) { k_set_config<<<1, 1, 0, s>>>(st, cfg); }
void step_begin(SolveState* st, int npts, cudaStream_t s) { k_step_begin<<<1, 1, 0, s>>>(st, npts); }
void step_end(SolveState* st, int refined, cudaStream_t s) { k_step_end<<<1, 1, 0, s>>>(st, refined); }
void reset_accum(SolveState* st, cudaStream_t s) { k_reset_accum<<<1, 1, 0, s>>>(st); }

}  // namespace hc
