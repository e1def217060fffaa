// Double-float instantiations: the FP64-class residual of the refined path
// (p += delta, S - A p, projection, norms) and the transforms of the state
// kept in double-float, all on the FP32 pipes.
#include "hc_kernels.cuh"

namespace hc {

template void row_r2c<df64>(const Geo<df64>&, const df64*, const df64*, cx<df64>*, cx<df64>*,
                            cudaStream_t);
template void row_c2r<df64>(const Geo<df64>&, const cx<df64>*, const cx<df64>*, df64*, df64*,
                            SolveState*, int, cudaStream_t);
template void row_apply<df64, float>(const Geo<df64>&, const cx<df64>*, const cx<df64>*,
                                     const float*, const float*, const float*, cx<df64>*,
                                     cx<df64>*, SolveState*, cudaStream_t);
template void col_fwd<df64>(const Geo<df64>&, const cx<df64>*, const cx<df64>*, cx<df64>*,
                            cx<df64>*, int, int, SolveState*, cudaStream_t);
template void col_inv<df64>(const Geo<df64>&, const cx<df64>*, cx<df64>*, df64, cudaStream_t);
template void col_grad<df64, df64>(const Geo<df64>&, int, cx<df64>*, const cx<df64>*, cx<df64>*,
                                   const cx<float>*, cx<df64>*, cx<df64>*, SolveState*, int,
                                   cudaStream_t);
template void col_grad<df64, double>(const Geo<df64>&, int, cx<double>*, const cx<df64>*, cx<df64>*,
                                     const cx<float>*, cx<df64>*, cx<df64>*, SolveState*, int,
                                     cudaStream_t);
template void col_grad<float, df64>(const Geo<float>&, int, cx<df64>*, const cx<float>*,
                                    cx<float>*, const cx<float>*, cx<float>*, cx<float>*,
                                    SolveState*, int, cudaStream_t);
template void col_div<df64>(const Geo<df64>&, int, const cx<df64>*, const cx<df64>*,
                            const cx<df64>*, const cx<df64>*, cx<df64>*, cx<float>*, cx<float>*,
                            SolveState*, cudaStream_t);
template void to_cm<df64>(const Geo<float>&, const cx<df64>*, cx<float>*, cudaStream_t);
template void convert<df64, double>(const double*, df64*, size_t, cudaStream_t);
template void convert<double, df64>(const df64*, double*, size_t, cudaStream_t);
template void convert<float, df64>(const df64*, float*, size_t, cudaStream_t);

void set_smem_limits_df() {
  allow_smem(k_row_r2c<df64>);
  allow_smem(k_row_c2r<df64>);
  allow_smem(k_row_apply<df64, float, false, 1>);
  allow_smem(k_row_apply<df64, float, true, 1>);
  allow_smem(k_col_fwd<df64, 1>);
  allow_smem(k_col_fwd<df64, 2>);
  allow_smem(k_col_inv<df64>);
  allow_smem(k_col_div<df64, CD_PLAIN>);
  allow_smem(k_col_div<df64, CD_CG>);
  allow_smem(k_col_div<df64, CD_RESID>);
  allow_smem(k_col_div<df64, CD_RESID_REFINE>);
  allow_smem(kp_col_div<df64, CD_PLAIN>);
  allow_smem(kp_col_div<df64, CD_CG>);
  allow_smem(kp_col_div<df64, CD_RESID>);
  allow_smem(kp_col_div<df64, CD_RESID_REFINE>);
  allow_smem(kp_col_grad<df64, CG_PLAIN>);
  allow_smem(kp_col_grad<df64, CG_DUPDATE>);
  allow_smem(kp_col_grad<df64, CG_ADDDELTA>);
  set_smem_limits_grad<df64, df64>();
  set_smem_limits_grad<df64, double>();
  set_smem_limits_grad<float, df64>();
}

}  // namespace hc
