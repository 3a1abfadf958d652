// Instantiations of the fused EM sweep (per-frame and persistent forms), bf16 staged maps, camera counts: 1 2 3 4 .
#include "em_sweep.cuh"

namespace lf {
cudaError_t launch_em_sweep_bf16_k1(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<1, __nv_bfloat16>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_bf16_k1(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<1, __nv_bfloat16>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_bf16_k1(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<1, __nv_bfloat16>(smem, threads, centred); }
cudaError_t launch_em_sweep_bf16_k2(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<2, __nv_bfloat16>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_bf16_k2(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<2, __nv_bfloat16>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_bf16_k2(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<2, __nv_bfloat16>(smem, threads, centred); }
cudaError_t launch_em_sweep_bf16_k3(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<3, __nv_bfloat16>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_bf16_k3(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<3, __nv_bfloat16>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_bf16_k3(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<3, __nv_bfloat16>(smem, threads, centred); }
cudaError_t launch_em_sweep_bf16_k4(const CUtensorMap& i, const CUtensorMap& p, const SweepArgs& a, cudaStream_t s) {
  return dev::launch_em_sweep_k<4, __nv_bfloat16>(i, p, a, s);
}
cudaError_t launch_em_sweep_persistent_bf16_k4(const FrameDesc* f, const TileItem* it, const int* first, const int* n, unsigned* h, size_t smem, int grid, int threads, int centred, cudaStream_t s) {
  return dev::launch_em_sweep_persistent_k<4, __nv_bfloat16>(f, it, first, n, h, smem, grid, threads, centred, s);
}
int em_sweep_persistent_occupancy_bf16_k4(size_t smem, int threads, int centred) { return dev::em_sweep_persistent_occupancy_k<4, __nv_bfloat16>(smem, threads, centred); }
}  // namespace lf
