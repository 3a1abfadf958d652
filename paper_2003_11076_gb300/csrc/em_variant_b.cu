// Instantiations of the EM variants (soft EM for up to 8 cameras, joint MAP), camera counts: 5 6 7 8.
#include "em_variants.cuh"

namespace lf {
cudaError_t launch_em_variant_k5(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeSoft) return dev::launch_em_variant_k<5, dev::kModeSoft>(i, p, a, s);
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<5, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
cudaError_t launch_em_variant_k6(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeSoft) return dev::launch_em_variant_k<6, dev::kModeSoft>(i, p, a, s);
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<6, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
cudaError_t launch_em_variant_k7(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeSoft) return dev::launch_em_variant_k<7, dev::kModeSoft>(i, p, a, s);
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<7, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
cudaError_t launch_em_variant_k8(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeSoft) return dev::launch_em_variant_k<8, dev::kModeSoft>(i, p, a, s);
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<8, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
}  // namespace lf
