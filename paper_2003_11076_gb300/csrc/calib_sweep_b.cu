// Instantiations of the calibrated-array EM sweep, camera counts: 7 8 9 10 11 12.
#include "calib_sweep.cuh"

namespace lf {
cudaError_t launch_calib_sweep_k7(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<7>(a, s); }
cudaError_t launch_calib_sweep_k8(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<8>(a, s); }
cudaError_t launch_calib_sweep_k9(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<9>(a, s); }
cudaError_t launch_calib_sweep_k10(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<10>(a, s); }
cudaError_t launch_calib_sweep_k11(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<11>(a, s); }
cudaError_t launch_calib_sweep_k12(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<12>(a, s); }
}  // namespace lf
