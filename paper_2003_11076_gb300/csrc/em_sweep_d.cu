// Instantiations of the fused EM sweep for camera counts: 9 10.
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_k9(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<9>(i, p, a, s);
}
cudaError_t launch_em_sweep_k10(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<10>(i, p, a, s);
}
}  // namespace lf
