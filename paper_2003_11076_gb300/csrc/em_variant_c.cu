// Instantiations of the EM variants (soft EM for up to 8 cameras, joint MAP), camera counts: 9 10 11 12.
#include "em_variants.cuh"

namespace lf {
cudaError_t launch_em_variant_k9(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<9, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
cudaError_t launch_em_variant_k10(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<10, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
cudaError_t launch_em_variant_k11(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<11, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
cudaError_t launch_em_variant_k12(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<12, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
}  // namespace lf
