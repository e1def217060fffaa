// Double-float instantiations of the 3D refinement residual.
#include "hc_kernels3d.cuh"

namespace hc {

template void z_grad<df64, df64>(const Geo<df64>&, int, cx<df64>*, const cx<df64>*, cx<df64>*,
                                 const cx<float>*, Tri<cx<df64>*>, SolveState*, int, cudaStream_t);
template void z_grad<df64, double>(const Geo<df64>&, int, cx<double>*, const cx<df64>*, cx<df64>*,
                                   const cx<float>*, Tri<cx<df64>*>, SolveState*, int, cudaStream_t);
template void axis_fft<df64>(const Geo<df64>&, int, int, int, Tri<cx<df64>*>, Tri<cx<df64>*>, df64,
                             cudaStream_t);
template void z_fwd_project<df64>(const Geo<df64>&, const cx<df64>*, cx<df64>*, SolveState*,
                                  cudaStream_t);
template void z_div<df64>(const Geo<df64>&, int, Tri<cx<df64>*>, const cx<df64>*, const cx<df64>*,
                          cx<df64>*, cx<float>*, cx<float>*, SolveState*, cudaStream_t);
template void row_apply3<df64, float>(const Geo<df64>&, Tri<cx<df64>*>, Tri<const float*>,
                                      const float*, Tri<cx<df64>*>, SolveState*,
                                      cudaStream_t);

void set_smem_limits_3d_df() {
  set_smem_limits_row3<df64, float>();
  set_smem_limits_zgrad<df64, df64>();
  set_smem_limits_zgrad<df64, double>();
  allow_smem(k3_axis_fft<df64, -1, 1>);
  allow_smem(k3_axis_fft<df64, -1, 3>);
  allow_smem(k3_axis_fft<df64, +1, 1>);
  allow_smem(k3_axis_fft<df64, +1, 3>);
  allow_smem(k3_zfwd_project<df64>);
  allow_smem(k3_zdiv<df64, CD_PLAIN>);
  allow_smem(k3_zdiv<df64, CD_CG>);
  allow_smem(k3_zdiv<df64, CD_RESID>);
  allow_smem(k3_zdiv<df64, CD_RESID_REFINE>);
}

}  // namespace hc
