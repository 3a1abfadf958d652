// Instantiations of the fused EM sweep (per-frame and persistent forms), f32 staged maps, camera counts: 9 10 11 12 .
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_f32_k9(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<9, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k9(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<9, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k9(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<9, float>(smem, threads, centred); }
cudaError_t launch_em_sweep_f32_k10(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<10, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k10(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<10, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k10(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<10, float>(smem, threads, centred); }
cudaError_t launch_em_sweep_f32_k11(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<11, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k11(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<11, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k11(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<11, float>(smem, threads, centred); }
cudaError_t launch_em_sweep_f32_k12(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<12, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k12(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<12, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k12(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<12, float>(smem, threads, centred); }
cudaError_t launch_tile_classify_k9(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<9>(a, p, pitch, list, n, s);
}
cudaError_t launch_tile_classify_k10(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<10>(a, p, pitch, list, n, s);
}
cudaError_t launch_tile_classify_k11(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<11>(a, p, pitch, list, n, s);
}
cudaError_t launch_tile_classify_k12(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<12>(a, p, pitch, list, n, s);
}
}  // namespace lf
