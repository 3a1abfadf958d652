// Instantiations of the EM variants (soft EM for up to 8 cameras, joint MAP), camera counts: 1 2 3 4.
#include "em_variants.cuh"

namespace lf {
cudaError_t launch_em_variant_k1(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeSoft) return dev::launch_em_variant_k<1, dev::kModeSoft>(i, p, a, s);
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<1, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
cudaError_t launch_em_variant_k2(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeSoft) return dev::launch_em_variant_k<2, dev::kModeSoft>(i, p, a, s);
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<2, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
cudaError_t launch_em_variant_k3(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeSoft) return dev::launch_em_variant_k<3, dev::kModeSoft>(i, p, a, s);
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<3, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
cudaError_t launch_em_variant_k4(int mode, const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a,
                                 cudaStream_t s) {
  if (mode == dev::kModeSoft) return dev::launch_em_variant_k<4, dev::kModeSoft>(i, p, a, s);
  if (mode == dev::kModeJoint) return dev::launch_em_variant_k<4, dev::kModeJoint>(i, p, a, s);
  return cudaErrorInvalidValue;
}
}  // namespace lf
