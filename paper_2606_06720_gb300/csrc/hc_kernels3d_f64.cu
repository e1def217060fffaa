// FP64 instantiations of the 3D step kernels (plain mode and the refinement residual).
#include "hc_kernels3d.cuh"

namespace hc {

template void z_grad<double, double>(const Geo<double>&, int, cx<double>*, const cx<double>*,
                                     cx<double>*, const cx<float>*, Tri<cx<double>*>, SolveState*,
                                     int, cudaStream_t);
template void axis_fft<double>(const Geo<double>&, int, int, int, Tri<cx<double>*>,
                               Tri<cx<double>*>, double, cudaStream_t);
template void z_fwd_project<double>(const Geo<double>&, const cx<double>*, cx<double>*, SolveState*,
                                    cudaStream_t);
template void z_div<double>(const Geo<double>&, int, Tri<cx<double>*>, const cx<double>*,
                            const cx<double>*, cx<double>*, cx<float>*, cx<float>*, SolveState*,
                            cudaStream_t);
template void row_apply3<double, double>(const Geo<double>&, Tri<cx<double>*>, Tri<const double*>,
                                         const double*, Tri<cx<double>*>, SolveState*,
                                         cudaStream_t);
template void row_apply3<double, float>(const Geo<double>&, Tri<cx<double>*>, Tri<const float*>,
                                        const float*, Tri<cx<double>*>, SolveState*,
                                        cudaStream_t);
template void row_split3<double>(const Geo<double>&, Tri<cx<double>*>, Tri<const double*>, const double*,
                                Tri<double*>, SplitCoef, SolveState*, cudaStream_t);
template void heat_axis<double>(const Geo<double>&, int, Tri<double*>, Tri<double*>, SolveState*,
                               cudaStream_t);
template void z_gradnorm<double>(const Geo<double>&, Tri<cx<double>*>, SolveState*, int, cudaStream_t);
template void cg_update3<double>(const Geo<double>&, cx<double>*, cx<double>*, const cx<double>*,
                                 const cx<double>*, SolveState*, cudaStream_t);
template void msum3<double>(const Geo<double>&, Tri<const double*>, SolveState*, cudaStream_t);

void set_smem_limits_3d_f64() {
  set_smem_limits_3d_t<double>();
  set_smem_limits_row3<double, double>();
  set_smem_limits_row3<double, float>();
  set_smem_limits_zgrad<double, double>();
}

}  // namespace hc
