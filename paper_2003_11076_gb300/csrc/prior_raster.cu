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

__global__ void prior_raster_kernel(const PriorArgs a) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  const int v = blockIdx.y * blockDim.y + threadIdx.y;
  if (u >= a.W || v >= a.H) return;
  const int bin = (v / kBinSize) * a.nbx + (u / kBinSize);
  const float pu = static_cast<float>(u), pv = static_cast<float>(v);
  float mu = __int_as_float(0x7fc00000);  // quiet NaN: outside
  for (int i = a.bin_start[bin]; i < a.bin_start[bin + 1]; ++i) {
    const PriorTri& t = a.tris[a.bin_items[i]];
    if (orient_sign(t.ua, t.va, t.ub, t.vb, pu, pv) < 0) continue;
    if (orient_sign(t.ub, t.vb, t.uc, t.vc, pu, pv) < 0) continue;
    if (orient_sign(t.uc, t.vc, t.ua, t.va, pu, pv) < 0) continue;
    const double m = t.da + t.gu * (static_cast<double>(u) - static_cast<double>(t.ua)) +
                     t.gv * (static_cast<double>(v) - static_cast<double>(t.va));
    mu = static_cast<float>(m);
    break;
  }
  a.mu[static_cast<size_t>(v) * a.W + u] = mu;
}

}  // namespace

cudaError_t launch_prior_raster(const PriorArgs& a, cudaStream_t s) {
  dim3 block(32, 8);
  dim3 grid((a.W + 31) / 32, (a.H + 7) / 8);
  prior_raster_kernel<<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace lf
