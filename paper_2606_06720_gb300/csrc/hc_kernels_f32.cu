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

void set_smem_limits_f32() {
  allow_smem(kp_row_apply<true>);
  allow_smem(kp_row_apply<false>);
  set_smem_limits_t<float>();
  set_smem_limits_grad<float, float>();
  set_smem_limits_grad<float, double>();
}

}  // namespace hc
