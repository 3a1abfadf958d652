// Instantiations of the fused EM sweep (per-frame and persistent forms), f32 staged maps, camera counts: 5 6 7 8 .
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_f32_k5(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<5, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k5(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<5, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k5(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<5, float>(smem, threads, centred); }
cudaError_t launch_em_sweep_f32_k6(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<6, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k6(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<6, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k6(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<6, float>(smem, threads, centred); }
cudaError_t launch_em_sweep_f32_k7(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<7, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k7(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<7, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k7(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<7, float>(smem, threads, centred); }
cudaError_t launch_em_sweep_f32_k8(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<8, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k8(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<8, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k8(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<8, float>(smem, threads, centred); }
cudaError_t launch_tile_classify_k5(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<5>(a, p, pitch, list, n, s);
}
cudaError_t launch_tile_classify_k6(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<6>(a, p, pitch, list, n, s);
}
cudaError_t launch_tile_classify_k7(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<7>(a, p, pitch, list, n, s);
}
cudaError_t launch_tile_classify_k8(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<8>(a, p, pitch, list, n, s);
}
}  // namespace lf
