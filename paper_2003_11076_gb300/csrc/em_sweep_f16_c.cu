// Instantiations of the fused EM sweep (per-frame and persistent forms), f16 staged maps, camera counts: 9 10 11 12 .
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_f16_k9(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<9, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f16_k9(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<9, __half>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f16_k9(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<9, __half>(smem, threads, centred); }
cudaError_t launch_em_sweep_f16_k10(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<10, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f16_k10(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<10, __half>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f16_k10(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<10, __half>(smem, threads, centred); }
cudaError_t launch_em_sweep_f16_k11(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<11, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f16_k11(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<11, __half>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f16_k11(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<11, __half>(smem, threads, centred); }
cudaError_t launch_em_sweep_f16_k12(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<12, __half>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f16_k12(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<12, __half>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f16_k12(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<12, __half>(smem, threads, centred); }
}  // namespace lf
