// Prior centre of one reference pixel (Sec. III-C "Disparity Prior"): the
// interpolated disparity of the first binned Delaunay triangle containing
// the pixel centre, NaN outside the triangulation.  Used by the prior raster
// kernels and, fused, by the sweep kernel's staging phase.
//
// Containment is decided by the sign of three orientation determinants: a
// float32 evaluation is accepted when it clears the rounding-error bound of
// its own arithmetic, otherwise the determinant is re-evaluated in float64
// (correctly rounded operations, no contraction).  Points on an edge count
// as inside.  The disparity is evaluated on the triangle's plane in float64
// and stored as float32.
#pragma once

#include "lf_internal.h"

namespace lf {
namespace prior {

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

// The same test over a contiguous list of n triangles (the pixel's bin, in
// bin order, staged in shared memory).
__device__ __forceinline__ float prior_pixel_list(const PriorTri* t, int n, int u, int v) {
  const float pu = static_cast<float>(u), pv = static_cast<float>(v);
  for (int i = 0; i < n; ++i, ++t) {
    if (orient_sign(t->ua, t->va, t->ub, t->vb, pu, pv) < 0) continue;
    if (orient_sign(t->ub, t->vb, t->uc, t->vc, pu, pv) < 0) continue;
    if (orient_sign(t->uc, t->vc, t->ua, t->va, pu, pv) < 0) continue;
    const double m = t->da + t->gu * (static_cast<double>(u) - static_cast<double>(t->ua)) +
                     t->gv * (static_cast<double>(v) - static_cast<double>(t->va));
    return static_cast<float>(m);
  }
  return __int_as_float(0x7fc00000);  // quiet NaN: outside
}

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

}  // namespace prior
}  // namespace lf
