// Calibrated (non-rectified) camera array, Eq. 1 in generalized disparity
// space: the descriptor maps written once per run, the dispatch of the
// per-pixel EM (calib_sweep.cuh) and the refocus of Eq. 2 with bilinear
// sampling at the homography positions.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "calib_geom.cuh"
#include "lf_internal.h"

namespace lf {
cudaError_t launch_calib_sweep_k1(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k2(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k3(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k4(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k5(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k6(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k7(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k8(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k9(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k10(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k11(const CalibArgs&, cudaStream_t);
cudaError_t launch_calib_sweep_k12(const CalibArgs&, cudaStream_t);

namespace {

__device__ __forceinline__ float pixel_value(const uint8_t* row, int x, int c, int C, int dtype) {
  if (dtype == 0) return static_cast<float>(row[x * C + c]);
  if (dtype == 1) return reinterpret_cast<const float*>(row)[x * C + c];
  if (dtype == 2) return __half2float(reinterpret_cast<const __half*>(row)[x * C + c]);
  return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(row)[x * C + c]);
}

// Luminance as the rectified sweep stages it: gray as is, RGB with the
// BT.601 weights; uint8 scaled by 1/255.
__device__ __forceinline__ float luma(const CalibArgs& a, int k, int v, int u) {
  const uint8_t* row = a.img + (static_cast<size_t>(k) * a.H + v) * a.img_pitch;
  float y;
  if (a.C == 1) {
    y = pixel_value(row, u, 0, 1, a.dtype);
  } else {
    const float r = pixel_value(row, u, 0, 3, a.dtype), g = pixel_value(row, u, 1, 3, a.dtype),
                b = pixel_value(row, u, 2, 3, a.dtype);
    y = fmaf(0.114f, b, fmaf(0.587f, g, 0.299f * r));
  }
  return a.dtype == 0 ? y * (1.f / 255.f) : y;
}

// Descriptors f = [Y, Sobel-x/8, Sobel-y/8] (border replicated) and the log
// segmentation priors of every camera pixel (Sec. III-C, Sec. III-B).
__global__ void calib_features_kernel(const CalibArgs a) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= a.W) return;
  if (blockIdx.y == 0) {  // the zero row past the end that the sweep's upper taps may read at the border
    const size_t end = static_cast<size_t>(a.K) * a.H * a.W;
    a.fa[end + u] = make_float4(0.f, 0.f, 0.f, 0.f);
    a.fb[end + u] = 0.f;
    if (u == 0) {
      a.fa[end + a.W] = make_float4(0.f, 0.f, 0.f, 0.f);
      a.fb[end + a.W] = 0.f;
    }
  }
  for (int row = blockIdx.y; row < a.K * a.H; row += gridDim.y) {  // row = k * H + v
    const int k = row / a.H, v = row - k * a.H;
    const int vm = max(v - 1, 0), vp = min(v + 1, a.H - 1), um = max(u - 1, 0), up = min(u + 1, a.W - 1);
    const float a00 = luma(a, k, vm, um), a01 = luma(a, k, vm, u), a02 = luma(a, k, vm, up);
    const float a10 = luma(a, k, v, um), a11 = luma(a, k, v, u), a12 = luma(a, k, v, up);
    const float a20 = luma(a, k, vp, um), a21 = luma(a, k, vp, u), a22 = luma(a, k, vp, up);
    const float gx = ((a02 + 2.f * a12) + a22) - ((a00 + 2.f * a10) + a20);
    const float gy = ((a20 + 2.f * a21) + a22) - ((a00 + 2.f * a01) + a02);
    const float P = reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(a.P) +
                                                   static_cast<size_t>(row) * a.p_pitch)[u];
    const size_t o = static_cast<size_t>(row) * a.W + u;
    a.fa[o] = make_float4(a11, gx * 0.125f, gy * 0.125f, __logf(fmaxf(1.f - P, a.eps)));
    a.fb[o] = __logf(fmaxf(P, a.eps));
  }
}

// Eq. 2 at the final (d, S): the mean over the static rays of the camera
// images sampled bilinearly at the ray positions; no static ray keeps the
// reference image.
__global__ void calib_refocus_kernel(const CalibArgs a) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= a.W || v >= a.H) return;
  const size_t pix = static_cast<size_t>(v) * a.W + u;
  const unsigned S = a.labels[pix];
  const float scale = a.dtype == 0 ? (1.f / 255.f) : 1.f;
  float* out = a.refocus + pix * a.C;
  if (S == 0u) {
    const uint8_t* row = a.img + (static_cast<size_t>(a.ref) * a.H + v) * a.img_pitch;
    for (int c = 0; c < a.C; ++c) out[c] = pixel_value(row, u, c, a.C, a.dtype) * scale;
    return;
  }
  const float d = a.dval[a.d_idx[pix]];
  float acc[3] = {0.f, 0.f, 0.f};
  int n = 0;
  for (int k = 0; k < a.K; ++k) {
    if (!(S >> k & 1u)) continue;
    ++n;
    const float* M = a.cam[k];
    const dev::CalibTaps t =
        dev::calib_taps(M, dev::calib_pixel(M, static_cast<float>(u), static_cast<float>(v)), u, v, d, a.W, a.H);
    const int i0 = t.i0, i1 = t.i1, j0 = t.j0, j1 = t.j1;
    const float wx = t.wx, wy = t.wy;
    const uint8_t* r0 = a.img + (static_cast<size_t>(k) * a.H + j0) * a.img_pitch;
    const uint8_t* r1 = a.img + (static_cast<size_t>(k) * a.H + j1) * a.img_pitch;
    for (int c = 0; c < a.C; ++c) {
      const float v00 = pixel_value(r0, i0, c, a.C, a.dtype), v01 = pixel_value(r0, i1, c, a.C, a.dtype);
      const float v10 = pixel_value(r1, i0, c, a.C, a.dtype), v11 = pixel_value(r1, i1, c, a.C, a.dtype);
      const float top = fmaf(wx, v01 - v00, v00), bot = fmaf(wx, v11 - v10, v10);
      acc[c] += fmaf(wy, bot - top, top) * scale;
    }
  }
  const float inv = 1.f / static_cast<float>(n);
  for (int c = 0; c < a.C; ++c) out[c] = acc[c] * inv;
}

}  // namespace

cudaError_t launch_calib_features(const CalibArgs& a, cudaStream_t s) {
  const dim3 grid((a.W + 127) / 128, std::min(a.K * a.H, 65535));
  calib_features_kernel<<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_calib_sweep(const CalibArgs& a, cudaStream_t s) {
  typedef cudaError_t (*Launch)(const CalibArgs&, cudaStream_t);
  static const Launch table[kMaxCams] = {launch_calib_sweep_k1, launch_calib_sweep_k2,  launch_calib_sweep_k3,
                                         launch_calib_sweep_k4, launch_calib_sweep_k5,  launch_calib_sweep_k6,
                                         launch_calib_sweep_k7, launch_calib_sweep_k8,  launch_calib_sweep_k9,
                                         launch_calib_sweep_k10, launch_calib_sweep_k11, launch_calib_sweep_k12};
  if (a.K < 1 || a.K > kMaxCams) return cudaErrorInvalidValue;
  return table[a.K - 1](a, s);
}

cudaError_t launch_calib_refocus(const CalibArgs& a, cudaStream_t s) {
  const dim3 block(32, 8), grid((a.W + 31) / 32, (a.H + 7) / 8);
  calib_refocus_kernel<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lf
