// Instantiations of the fused EM sweep (per-frame and persistent forms), f16 staged maps, camera counts: 5 6 7 8 .
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_f16_k5(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<5, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f16_k5(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<5, __half>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f16_k5(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<5, __half>(smem, threads, centred); }
cudaError_t launch_em_sweep_f16_k6(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<6, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f16_k6(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<6, __half>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f16_k6(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<6, __half>(smem, threads, centred); }
cudaError_t launch_em_sweep_f16_k7(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<7, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f16_k7(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<7, __half>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f16_k7(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<7, __half>(smem, threads, centred); }
cudaError_t launch_em_sweep_f16_k8(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<8, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f16_k8(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<8, __half>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f16_k8(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<8, __half>(smem, threads, centred); }
}  // namespace lf
