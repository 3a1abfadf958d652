// Instantiations of the fused EM sweep for camera counts: 11 12.
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_k11(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<11>(i, p, a, s);
}
cudaError_t launch_em_sweep_k12(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<12>(i, p, a, s);
}
}  // namespace lf
