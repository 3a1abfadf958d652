// Instantiations of the fused EM sweep, f32 staged maps, camera counts: 1 2 3 4.
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_f32_k1(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<1, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_f32_k2(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<2, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_f32_k3(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<3, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_f32_k4(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<4, float>(i, p, a, s);
}
}  // namespace lf
