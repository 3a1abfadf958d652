// Instantiations of the fused EM sweep, f16 staged maps, camera counts: 9 10 11 12.
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_f16_k9(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<9, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_f16_k10(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<10, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_f16_k11(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<11, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_f16_k12(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<12, __half>(i, p, a, s);
}
}  // namespace lf
