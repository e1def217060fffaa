// FP32 instantiations of the step kernels (the bulk of the refined path).
#include "hc_kernels.cuh"

namespace hc {

template void row_r2c<float>(const Geo<float>&, const float*, const float*, cx<float>*, cx<float>*,
                             cudaStream_t);
template void row_c2r<float>(const Geo<float>&, const cx<float>*, const cx<float>*, float*, float*,
                             SolveState*, int, cudaStream_t);
template void row_apply<float, float>(const Geo<float>&, const cx<float>*, const cx<float>*,
                                      const float*, const float*, const float*, cx<float>*,
                                      cx<float>*, SolveState*, cudaStream_t);
template void row_split<float>(const Geo<float>&, const cx<float>*, const cx<float>*, const float*,
                               const float*, const float*, cx<float>*, cx<float>*, SplitCoef, SolveState*,
                               cudaStream_t);
template void col_fwd<float>(const Geo<float>&, const cx<float>*, const cx<float>*, cx<float>*,
                             cx<float>*, int, int, SolveState*, cudaStream_t);
template void col_inv<float>(const Geo<float>&, const cx<float>*, cx<float>*, float, cudaStream_t);
template void col_grad<float, double>(const Geo<float>&, int, cx<double>*, const cx<float>*,
                                      cx<float>*, const cx<float>*, cx<float>*, cx<float>*,
                                      SolveState*, int, cudaStream_t);
template void col_grad<float, float>(const Geo<float>&, int, cx<float>*, const cx<float>*,
                                     cx<float>*, const cx<float>*, cx<float>*, cx<float>*,
                                     SolveState*, int, cudaStream_t);
template void col_div<float>(const Geo<float>&, int, const cx<float>*, const cx<float>*,
                             const cx<float>*, const cx<float>*, cx<float>*, cx<float>*, cx<float>*,
                             SolveState*, cudaStream_t);
template void col_heat<float>(const Geo<float>&, cx<float>*, cx<float>*, SolveState*, cudaStream_t);
template void col_gradnorm<float>(const Geo<float>&, const cx<float>*, const cx<float>*, SolveState*, int,
                                 cudaStream_t);
template void cg_update<float>(const Geo<float>&, cx<float>*, cx<float>*, const cx<float>*,
                               const cx<float>*, SolveState*, cudaStream_t);
template void to_cm<double>(const Geo<float>&, const cx<double>*, cx<float>*, cudaStream_t);
template void msum<float>(const Geo<float>&, const float*, const float*, SolveState*, cudaStream_t);

template void row_adj_point<float>(const Geo<float>&, cx<float>*, cx<float>*, const cx<float>*, const cx<float>*,
                                const float*, const float*, float*, float*, SplitCoef, AdjState*, cudaStream_t);
template void row_adj_press<float>(const Geo<float>&, const cx<float>*, const cx<float>*, const cx<float>*,
                                const cx<float>*, const float*, const float*, const float*, const float*, float*,
                                float*, double*, cudaStream_t);
template void col_lap_dot<float>(const Geo<float>&, const cx<float>*, const cx<float>*, double, AdjState*,
                              cudaStream_t);
template void spec_accum<float>(const Geo<float>&, double*, const cx<float>*, cudaStream_t);
template void spec_norm2<float>(const Geo<float>&, const cx<float>*, SolveState*, cudaStream_t);

int row_pipe_ctas_per_sm(int threads, size_t smem) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kp_row_apply<true>, threads, smem) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// ------------------------------------------------------------------ lagged certification
// The certification of the previous step passed, or nothing awaited one.
__device__ __forceinline__ bool cert_ok(const SolveState* st, const SolveState* sc) {
  return !sc->cert_pending || (isfinite(sc->cert_r2) && sc->cert_r2 <= st->outer_thresh2);
}

// After both branches of a lagged step: unless the previous step's
// certification failed, keep its input m and its pressure for the
// certification of the step just made (m -> m_prev, p -> p_saved) and accept
// that step's m (m_tmp -> m).  Every CTA reads the decision from states this
// kernel does not change; k_commit_flags updates them afterwards.
__global__ void __launch_bounds__(256) k_commit_copy(const SolveState* st, const SolveState* sc,
                                                     float* __restrict__ m0, float* __restrict__ m1,
                                                     float* __restrict__ mp0, float* __restrict__ mp1,
                                                     const float* __restrict__ mt0,
                                                     const float* __restrict__ mt1,
                                                     const cx<double>* __restrict__ p64,
                                                     cx<double>* __restrict__ ps, size_t n,
                                                     size_t ns) {
  if (!cert_ok(st, sc)) return;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    mp0[i] = m0[i];
    mp1[i] = m1[i];
    m0[i] = mt0[i];
    m1[i] = mt1[i];
  }
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += stride) ps[i] = p64[i];
}

// One thread.  A passed (or absent) certification: the step just made now
// awaits its own.  A failed one: halt the remaining lagged steps (the host
// redoes the failed step); the state still holds that step's input m and its
// pressure.  With final = 1 (after the last step, no new step made) nothing
// awaits a certification afterwards.
__global__ void k_commit_flags(SolveState* st, SolveState* sc, int final_cert) {
  const bool ok = cert_ok(st, sc);
  if (sc->cert_pending) {
    st->outer_r2 = sc->cert_r2;  // the certified residual of the step it certified
    st->res_full = 1;
    st->acc_res_full += 1;
  }
  if (ok) {
    if (!final_cert) st->cert_steps += 1;
    sc->cert_pending = final_cert ? 0 : 1;
    sc->done = final_cert ? 1 : 0;
  } else {
    st->cert_failed = 1;
    st->halt = 1;
  }
}

// Start (on = 1) or end (on = 0) of a pass of lagged steps: nothing awaits
// certification at its start, and no halt or failure is pending.
__global__ void k_lag_mark(SolveState* st, SolveState* sc, int on) {
  st->pipelined = on;
  if (on) {
    sc->cert_pending = 0;
    sc->done = 1;
    st->halt = 0;
    st->cert_failed = 0;
    st->cert_steps = 0;
  }
}
void lag_mark(SolveState* st, SolveState* sc, int on, cudaStream_t s) {
  k_lag_mark<<<1, 1, 0, s>>>(st, sc, on);
}

void commit_copy(const SolveState* st, const SolveState* sc, float* const* m, float* const* mp,
                 const float* const* mt, const cx<double>* p64, cx<double>* ps, size_t n, size_t ns,
                 cudaStream_t s) {
  k_commit_copy<<<upd_blocks(n), 256, 0, s>>>(st, sc, m[0], m[1], mp[0], mp[1], mt[0], mt[1], p64, ps,
                                              n, ns);
}
void commit_flags(SolveState* st, SolveState* sc, int final_cert, cudaStream_t s) {
  k_commit_flags<<<1, 1, 0, s>>>(st, sc, final_cert);
}

void set_smem_limits_f32() {
  allow_smem(kp_row_apply<true>);
  allow_smem(kp_row_apply<false>);
  set_smem_limits_t<float>();
  set_smem_limits_grad<float, float>();
  set_smem_limits_grad<float, double>();
}

}  // namespace hc
