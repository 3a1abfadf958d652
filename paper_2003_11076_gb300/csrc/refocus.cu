// Refocused static image, Eq. 2 (Sec. III-A; synthesis after the EM,
// Sec. III-E): the mean over the rays labelled static of the camera images
// sampled at u - d_T * b_k (linear interpolation, column clamped); a pixel
// with no static ray keeps the reference image (Sec. IV-B).  Plus the
// optional 3x3 median filter of Sec. III-E (per channel, border replicated).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lf_internal.h"

namespace lf {
namespace {

__device__ __forceinline__ float load_px(const uint8_t* row, int x, int c, int C, int dtype) {
  if (dtype == 0) return static_cast<float>(row[x * C + c]);
  if (dtype == 1) return reinterpret_cast<const float*>(row)[x * C + c];
  if (dtype == 2) return __half2float(reinterpret_cast<const __half*>(row)[x * C + c]);
  return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(row)[x * C + c]);
}

__device__ __forceinline__ void refocus_pixel(const RefocusArgs& a, int u, int v) {
  const size_t pix = static_cast<size_t>(v) * a.W + u;
  const int j = a.d_idx[pix];
  const unsigned S = a.labels[pix];
  const float scale = a.dtype == 0 ? (1.f / 255.f) : 1.f;
  float acc[3] = {0.f, 0.f, 0.f};
  int n = 0;
  for (int k = 0; k < a.K; ++k) {
    if (!(S >> k & 1u)) continue;
    ++n;
    const int o = a.otab[j * a.KP + k];
    const float w = a.wtab[j * a.KP + k];
    const int x0 = min(max(u + o, 0), a.W - 1);
    const int x1 = min(max(u + o + 1, 0), a.W - 1);
    const uint8_t* row = a.img + (static_cast<size_t>(k) * a.H + v) * a.pitch;
    for (int c = 0; c < a.C; ++c) {
      const float g0 = load_px(row, x0, c, a.C, a.dtype);
      const float g1 = load_px(row, x1, c, a.C, a.dtype);
      acc[c] += fmaf(w, g1 - g0, g0) * scale;
    }
  }
  float* out = a.out + pix * a.C;
  if (n == 0) {
    const uint8_t* row = a.img + (static_cast<size_t>(a.ref) * a.H + v) * a.pitch;
    for (int c = 0; c < a.C; ++c) out[c] = load_px(row, u, c, a.C, a.dtype) * scale;
  } else {
    const float inv = 1.f / static_cast<float>(n);
    for (int c = 0; c < a.C; ++c) out[c] = acc[c] * inv;
  }
}

__global__ void refocus_kernel(const RefocusArgs a) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= a.W || v >= a.H) return;
  refocus_pixel(a, u, v);
}

__global__ void refocus_batched(const RefocusArgs* frames, const RowItem* items, const int* n_items) {
  const int n = *n_items;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const RowItem r = items[it];
    const RefocusArgs& f = frames[r.frame];
    if (!f.out) continue;
    for (int u = threadIdx.x; u < f.W; u += blockDim.x) refocus_pixel(f, u, r.row);
  }
}

__device__ __forceinline__ void sort2(float& x, float& y) {
  const float lo = fminf(x, y), hi = fmaxf(x, y);
  x = lo;
  y = hi;
}

__device__ __forceinline__ void median_pixel(const float* in, float* out, int H, int W, int C, int u, int v) {
  for (int c = 0; c < C; ++c) {
    float p[9];
    int n = 0;
    for (int dv = -1; dv <= 1; ++dv)
      for (int du = -1; du <= 1; ++du) {
        const int yy = min(max(v + dv, 0), H - 1), xx = min(max(u + du, 0), W - 1);
        p[n++] = in[(static_cast<size_t>(yy) * W + xx) * C + c];
      }
    // median of 9 by a 19-exchange selection network
    sort2(p[1], p[2]); sort2(p[4], p[5]); sort2(p[7], p[8]);
    sort2(p[0], p[1]); sort2(p[3], p[4]); sort2(p[6], p[7]);
    sort2(p[1], p[2]); sort2(p[4], p[5]); sort2(p[7], p[8]);
    sort2(p[0], p[3]); sort2(p[5], p[8]); sort2(p[4], p[7]);
    sort2(p[3], p[6]); sort2(p[1], p[4]); sort2(p[2], p[5]);
    sort2(p[4], p[7]); sort2(p[4], p[2]); sort2(p[6], p[4]);
    sort2(p[4], p[2]);
    out[(static_cast<size_t>(v) * W + u) * C + c] = p[4];
  }
}

__global__ void median3_kernel(const float* in, float* out, int H, int W, int C) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= W || v >= H) return;
  median_pixel(in, out, H, W, C, u, v);
}

__global__ void median3_batched(const MedianArgs* frames, const RowItem* items, const int* n_items) {
  const int n = *n_items;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const RowItem r = items[it];
    const MedianArgs& f = frames[r.frame];
    if (!f.out) continue;
    for (int u = threadIdx.x; u < f.W; u += blockDim.x) median_pixel(f.in, f.out, f.H, f.W, f.C, u, r.row);
  }
}

}  // namespace

cudaError_t launch_refocus(const RefocusArgs& a, cudaStream_t s) {
  dim3 block(64, 4);
  dim3 grid((a.W + 63) / 64, (a.H + 3) / 4);
  refocus_kernel<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_refocus_batched(const RefocusArgs* frames, const RowItem* items, const int* n_items, int grid,
                                   cudaStream_t s) {
  refocus_batched<<<grid, 256, 0, s>>>(frames, items, n_items);
  return cudaGetLastError();
}

cudaError_t launch_median3_batched(const MedianArgs* frames, const RowItem* items, const int* n_items, int grid,
                                   cudaStream_t s) {
  median3_batched<<<grid, 256, 0, s>>>(frames, items, n_items);
  return cudaGetLastError();
}

cudaError_t launch_median3(const float* in, float* out, int H, int W, int C, cudaStream_t s) {
  dim3 block(64, 4);
  dim3 grid((W + 63) / 64, (H + 3) / 4);
  median3_kernel<<<grid, block, 0, s>>>(in, out, H, W, C);
  return cudaGetLastError();
}

}  // namespace lf
