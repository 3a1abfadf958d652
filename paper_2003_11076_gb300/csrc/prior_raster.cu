// Piecewise-planar disparity prior raster (Sec. III-C "Disparity Prior"):
// for every reference pixel centre, the interpolated disparity of the
// Delaunay triangle of support points that contains it, NaN outside the
// triangulation (the prior is uniform there).
//
// The host bins triangles into 16x16-pixel tiles (ascending triangle index
// per bin); a pixel takes the first triangle of its bin that contains it,
// with points on an edge counting as inside.  Containment is decided by the
// sign of three orientation determinants: a float32 evaluation is accepted
// when it clears the rounding-error bound of its own arithmetic, otherwise
// the determinant is re-evaluated in float64 (correctly rounded operations,
// no contraction).  The disparity is then evaluated on the triangle's plane
// in float64 and stored as float32.
#include <cmath>

#include "lf_internal.h"

namespace lf {
namespace {

__device__ __forceinline__ int orient_sign(float ax, float ay, float bx, float by, float px, float py) {
  const float t1 = __fmul_rn(__fsub_rn(bx, ax), __fsub_rn(py, ay));
  const float t2 = __fmul_rn(__fsub_rn(by, ay), __fsub_rn(px, ax));
  const float det = __fsub_rn(t1, t2);
  // 8 units of float32 roundoff on |t1| + |t2| bounds the evaluation error of
  // this expression when ax..py are exact floats (pixel centres are integers).
  const float bound = 4.8e-7f * (fabsf(t1) + fabsf(t2));
  if (det > bound) return 1;
  if (det < -bound) return -1;
  const double D = __dsub_rn(__dmul_rn(__dsub_rn(bx, ax), __dsub_rn(py, ay)),
                             __dmul_rn(__dsub_rn(by, ay), __dsub_rn(px, ax)));
  return (D > 0.0) - (D < 0.0);
}

// Prior centre of pixel (u, v): the first binned triangle containing it.
__device__ __forceinline__ float prior_pixel(const PriorTri* tris, const int* bin_start, const int* bin_items,
                                             int nbx, int u, int v) {
  const int bin = (v / kBinSize) * nbx + (u / kBinSize);
  const float pu = static_cast<float>(u), pv = static_cast<float>(v);
  for (int i = bin_start[bin]; i < bin_start[bin + 1]; ++i) {
    const PriorTri& t = tris[bin_items[i]];
    if (orient_sign(t.ua, t.va, t.ub, t.vb, pu, pv) < 0) continue;
    if (orient_sign(t.ub, t.vb, t.uc, t.vc, pu, pv) < 0) continue;
    if (orient_sign(t.uc, t.vc, t.ua, t.va, pu, pv) < 0) continue;
    const double m = t.da + t.gu * (static_cast<double>(u) - static_cast<double>(t.ua)) +
                     t.gv * (static_cast<double>(v) - static_cast<double>(t.va));
    return static_cast<float>(m);
  }
  return __int_as_float(0x7fc00000);  // quiet NaN: outside
}

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
