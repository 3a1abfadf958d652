// Prior centre of one reference pixel (Sec. III-C "Disparity Prior"): the
// interpolated disparity of the first binned Delaunay triangle containing
// the pixel centre, NaN outside the triangulation.  Used by the prior raster
// kernels and, fused, by the sweep kernel's staging phase.
//
// Containment is decided by the sign of three orientation determinants: a
// float32 evaluation is accepted when it clears the rounding-error bound of
// its own arithmetic, otherwise the determinant is re-evaluated in float64
// (correctly rounded operations, no contraction).  Points on an edge count
// as inside.  The disparity is evaluated on the triangle's plane in
// double-float arithmetic (error-free sums and products of float32 numbers,
// about 44 significant bits) and rounded once to float32.
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

// a + b = s + e exactly (Knuth's TwoSum), every operation rounded to nearest.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// mu at the integer pixel (u, v) on triangle t's plane:
// d_a + gu (u - u_a) + gv (v - v_a) with the coefficients as hi + lo pairs,
// the differences u - u_a, v - v_a exact as hi + lo pairs, the products with
// their exact rounding errors (fma), and all parts summed with TwoSum; the
// result is the one float rounding of the hi + lo total.
__device__ __forceinline__ float plane_at(const PriorTri& t, float pu, float pv) {
  float dh, dl, eh, el;
  two_sum(pu, -t.ua, dh, dl);
  two_sum(pv, -t.va, eh, el);
  const float ph = __fmul_rn(t.gu_hi, dh);
  const float pl = __fadd_rn(__fmaf_rn(t.gu_hi, dh, -ph), __fmaf_rn(t.gu_hi, dl, __fmul_rn(t.gu_lo, dh)));
  const float qh = __fmul_rn(t.gv_hi, eh);
  const float ql = __fadd_rn(__fmaf_rn(t.gv_hi, eh, -qh), __fmaf_rn(t.gv_hi, el, __fmul_rn(t.gv_lo, eh)));
  float s1, e1, s2, e2;
  two_sum(t.da_hi, ph, s1, e1);
  two_sum(s1, qh, s2, e2);
  const float lo = __fadd_rn(__fadd_rn(__fadd_rn(t.da_lo, pl), __fadd_rn(ql, e1)), e2);
  return __fadd_rn(s2, lo);
}

// The same test over a contiguous list of n triangles (the pixel's bin, in
// bin order, staged in shared memory).
__device__ __forceinline__ float prior_pixel_list(const PriorTri* t, int n, int u, int v) {
  const float pu = static_cast<float>(u), pv = static_cast<float>(v);
  for (int i = 0; i < n; ++i, ++t) {
    if (orient_sign(t->ua, t->va, t->ub, t->vb, pu, pv) < 0) continue;
    if (orient_sign(t->ub, t->vb, t->uc, t->vc, pu, pv) < 0) continue;
    if (orient_sign(t->uc, t->vc, t->ua, t->va, pu, pv) < 0) continue;
    return plane_at(*t, pu, pv);
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
    return plane_at(t, pu, pv);
  }
  return __int_as_float(0x7fc00000);  // quiet NaN: outside
}

}  // namespace prior
}  // namespace lf
