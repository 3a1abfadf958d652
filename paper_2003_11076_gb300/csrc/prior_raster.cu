// Piecewise-planar disparity prior raster (Sec. III-C "Disparity Prior"):
// for every reference pixel centre, the interpolated disparity of the
// Delaunay triangle of support points that contains it, NaN outside the
// triangulation (the prior is uniform there).  The host bins triangles into
// 16x16-pixel tiles (ascending triangle index per bin); a pixel takes the
// first triangle of its bin that contains it (prior_pixel.cuh).
#include <cmath>

#include "prior_pixel.cuh"

namespace lf {
namespace {

using prior::prior_pixel;

__global__ void prior_raster_kernel(const PriorArgs a) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= a.W || v >= a.H) return;
  a.mu[static_cast<size_t>(v) * a.W + u] = prior_pixel(a.tris, a.bin_start, a.bin_items, a.nbx, u, v);
}

// Uneven batches: one (frame, row) item per pass of a CTA, items and frame
// descriptors in device memory.
__global__ void prior_raster_batched(const PriorArgs* frames, const RowItem* items, const int* n_items) {
  const int n = *n_items;
  for (int it = blockIdx.x; it < n; it += gridDim.x) {
    const RowItem r = items[it];
    const PriorArgs& f = frames[r.frame];
    for (int u = threadIdx.x; u < f.W; u += blockDim.x)
      f.mu[static_cast<size_t>(r.row) * f.W + u] = prior_pixel(f.tris, f.bin_start, f.bin_items, f.nbx, u, r.row);
  }
}

}  // namespace

cudaError_t launch_prior_raster(const PriorArgs& a, cudaStream_t s) {
  dim3 block(32, 8);
  dim3 grid((a.W + 31) / 32, (a.H + 7) / 8);
  prior_raster_kernel<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_prior_raster_batched(const PriorArgs* frames, const RowItem* items, const int* n_items,
                                        int grid, cudaStream_t s) {
  prior_raster_batched<<<grid, 256, 0, s>>>(frames, items, n_items);
  return cudaGetLastError();
}

}  // namespace lf
