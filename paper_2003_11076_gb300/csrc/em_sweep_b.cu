// Instantiations of the fused EM sweep for camera counts: 5 6.
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_k5(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<5>(i, p, a, s);
}
cudaError_t launch_em_sweep_k6(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<6>(i, p, a, s);
}
}  // namespace lf
