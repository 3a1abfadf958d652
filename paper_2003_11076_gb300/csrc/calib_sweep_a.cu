// Instantiations of the calibrated-array EM sweep, camera counts: 1 2 3 4 5 6.
#include "calib_sweep.cuh"

namespace lf {
cudaError_t launch_calib_sweep_k1(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<1>(a, s); }
cudaError_t launch_calib_sweep_k2(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<2>(a, s); }
cudaError_t launch_calib_sweep_k3(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<3>(a, s); }
cudaError_t launch_calib_sweep_k4(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<4>(a, s); }
cudaError_t launch_calib_sweep_k5(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<5>(a, s); }
cudaError_t launch_calib_sweep_k6(const CalibArgs& a, cudaStream_t s) { return dev::launch_calib_sweep_k<6>(a, s); }
}  // namespace lf
