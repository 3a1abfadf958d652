// Ray position of a calibrated (non-rectified) camera, Eq. 1 in generalized
// disparity space: camera k sees reference pixel (u, v) at disparity d at
// (X / Z, Y / Z) with (X, Y, Z) = M_k (u, v, 1, d), M_k its 3x4 matrix
// (row-major, 12 floats).
//
// Numerics.  X / Z itself is a number of the size of the image (up to a few
// thousand), so in float32 it carries an absolute error of about 1e-4 px,
// enough to move the sampled descriptors, and with them the objective, by
// about the arg-max margin the parity rule tolerates.  The ray is therefore
// located by its offset from the pixel,
//   X / Z - u = (X - u Z) / Z,   Y / Z - v = (Y - v Z) / Z,
// whose numerators are small for cameras near the reference's pose:
//   X - u Z = u (M00 - M22) + M01 v + M02 - u (M20 u + M21 v) + d (M03 - u M23)
//   Y - v Z = M10 u + v (M11 - M22) + M12 - v (M20 u + M21 v) + d (M13 - v M23)
//   Z       = M20 u + M21 v + M22 + d M23.
// The differences M00 - M22 and M11 - M22 are exact in float32 for any
// matrix with those entries within a factor of two of each other (Sterbenz),
// and vanish for a rectified array, so the offset keeps float32's relative
// precision: about 1e-6 px at a 12 px offset.
#pragma once

#include <cuda_runtime.h>

namespace lf {
namespace dev {

// Pixel-constant parts of X - u Z, Y - v Z and Z for one camera.
struct CalibPix {
  float ax, ay, az;
};

__host__ __device__ __forceinline__ CalibPix calib_pixel(const float* M, float u, float v) {
  const float t = fmaf(M[8], u, M[9] * v);  // perspective part of Z
  CalibPix c;
  c.az = t + M[10];
  c.ax = fmaf(-u, t, fmaf(u, M[0] - M[10], fmaf(M[1], v, M[2])));
  c.ay = fmaf(-v, t, fmaf(v, M[5] - M[10], fmaf(M[4], u, M[6])));
  return c;
}

// Bilinear taps of the ray at candidate disparity d: columns i0 <= i1 and
// rows j0 <= j1 with weights wx, wy, for the position clamped to
// [0, W-1] x [0, H-1] (the border is replicated; a clamped coordinate gets
// weight 0, i.e. the border texel).
struct CalibTaps {
  int i0, i1, j0, j1;
  float wx, wy;
};

__device__ __forceinline__ void calib_axis(float off, int p, int n, int& i0, int& i1, float& w) {
  const float f = floorf(off);
  const int fi = __float2int_rd(off);  // saturates far outside the image
  w = off - f;
  if (fi < -p) {  // p + off < 0
    i0 = 0;
    w = 0.f;
  } else if (fi >= n - 1 - p) {  // p + off >= n - 1
    i0 = n - 1;
    w = 0.f;
  } else {
    i0 = p + fi;
  }
  i1 = min(i0 + 1, n - 1);
}

__device__ __forceinline__ CalibTaps calib_taps(const float* M, const CalibPix& c, int u, int v, float d, int W,
                                                int H) {
  const float Z = fmaf(d, M[11], c.az);
  const float X = fmaf(d, fmaf(-static_cast<float>(u), M[11], M[3]), c.ax);
  const float Y = fmaf(d, fmaf(-static_cast<float>(v), M[11], M[7]), c.ay);
  const float iz = 1.f / Z;
  CalibTaps t;
  calib_axis(X * iz, u, W, t.i0, t.i1, t.wx);
  calib_axis(Y * iz, v, H, t.j0, t.j1, t.wy);
  return t;
}

}  // namespace dev
}  // namespace lf
