// Instantiations of the fused EM sweep, bf16 staged maps, camera counts: 5 6 7 8.
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_bf16_k5(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<5, __nv_bfloat16>(i, p, a, s);
}
cudaError_t launch_em_sweep_bf16_k6(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<6, __nv_bfloat16>(i, p, a, s);
}
cudaError_t launch_em_sweep_bf16_k7(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<7, __nv_bfloat16>(i, p, a, s);
}
cudaError_t launch_em_sweep_bf16_k8(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<8, __nv_bfloat16>(i, p, a, s);
}
}  // namespace lf
