// Instantiations of the fused EM sweep (per-frame and persistent forms), f32 staged maps, camera counts: 1 2 3 4 .
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_f32_k1(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<1, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k1(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<1, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k1(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<1, float>(smem, threads, centred); }
cudaError_t launch_em_sweep_f32_k2(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<2, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k2(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<2, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k2(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<2, float>(smem, threads, centred); }
cudaError_t launch_em_sweep_f32_k3(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<3, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k3(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<3, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k3(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<3, float>(smem, threads, centred); }
cudaError_t launch_em_sweep_f32_k4(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<4, float>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_f32_k4(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<4, float>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_f32_k4(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<4, float>(smem, threads, centred); }
cudaError_t launch_tile_classify_k1(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<1>(a, p, pitch, list, n, s);
}
cudaError_t launch_tile_classify_k2(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<2>(a, p, pitch, list, n, s);
}
cudaError_t launch_tile_classify_k3(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<3>(a, p, pitch, list, n, s);
}
cudaError_t launch_tile_classify_k4(const SweepArgs& a, const float* p, size_t pitch, int* list, int* n, cudaStream_t s) {
  return dev::launch_tile_classify_k<4>(a, p, pitch, list, n, s);
}
}  // namespace lf
