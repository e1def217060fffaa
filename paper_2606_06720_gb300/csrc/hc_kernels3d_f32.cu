// FP32 instantiations of the 3D step kernels (inner CG and split step).
#include "hc_kernels3d.cuh"

namespace hc {

template void z_grad<float, float>(const Geo<float>&, int, cx<float>*, const cx<float>*, cx<float>*,
                                   const cx<float>*, Tri<cx<float>*>, SolveState*, int, cudaStream_t);
template void z_grad<float, double>(const Geo<float>&, int, cx<double>*, const cx<float>*,
                                    cx<float>*, const cx<float>*, Tri<cx<float>*>, SolveState*, int,
                                    cudaStream_t);
template void z_grad<float, df64>(const Geo<float>&, int, cx<df64>*, const cx<float>*, cx<float>*,
                                  const cx<float>*, Tri<cx<float>*>, SolveState*, int, cudaStream_t);
template void axis_fft<float>(const Geo<float>&, int, int, int, Tri<cx<float>*>, Tri<cx<float>*>,
                              float, cudaStream_t);
template void z_fwd_project<float>(const Geo<float>&, const cx<float>*, cx<float>*, SolveState*,
                                   cudaStream_t);
template void z_div<float>(const Geo<float>&, int, Tri<cx<float>*>, const cx<float>*,
                           const cx<float>*, cx<float>*, cx<float>*, cx<float>*, SolveState*,
                           cudaStream_t);
template void row_apply3<float, float>(const Geo<float>&, Tri<cx<float>*>, Tri<const float*>,
                                       const float*, Tri<cx<float>*>, SolveState*,
                                       cudaStream_t);
template void row_split3<float>(const Geo<float>&, Tri<cx<float>*>, Tri<const float*>, const float*,
                                Tri<float*>, SplitCoef, SolveState*, cudaStream_t);
template void heat_axis<float>(const Geo<float>&, int, Tri<float*>, Tri<float*>, SolveState*,
                               cudaStream_t);
template void z_gradnorm<float>(const Geo<float>&, Tri<cx<float>*>, SolveState*, int, cudaStream_t);
template void cg_update3<float>(const Geo<float>&, cx<float>*, cx<float>*, const cx<float>*,
                                const cx<float>*, SolveState*, cudaStream_t);
template void msum3<float>(const Geo<float>&, Tri<const float*>, SolveState*, cudaStream_t);

void set_smem_limits_3d_f32() {
  set_smem_limits_3d_t<float>();
  set_smem_limits_row3<float, float>();
  set_smem_limits_zgrad<float, float>();
  set_smem_limits_zgrad<float, double>();
  set_smem_limits_zgrad<float, df64>();
}

}  // namespace hc
