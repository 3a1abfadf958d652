// Instantiations of the fused EM sweep, f32 staged maps, camera counts: 5 6 7 8.
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_f32_k5(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<5, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_f32_k6(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<6, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_f32_k7(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<7, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_f32_k8(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<8, float>(i, p, a, s);
}
}  // namespace lf
