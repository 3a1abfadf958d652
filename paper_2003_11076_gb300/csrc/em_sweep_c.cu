// Instantiations of the fused EM sweep for camera counts: 7 8.
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_k7(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<7>(i, p, a, s);
}
cudaError_t launch_em_sweep_k8(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<8>(i, p, a, s);
}
}  // namespace lf
