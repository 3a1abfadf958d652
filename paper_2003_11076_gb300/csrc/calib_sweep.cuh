// Per-pixel EM for a calibrated (non-rectified) camera array (Eq. 1 in
// generalized disparity space; the warping function W_k of Sec. III-C is the
// homography of the plane at disparity d).  The schedule and the objective
// are those of the rectified sweep (Sec. III-B..III-D): first M-step with
// per-candidate thresholded labels, then M-step / E-step alternation with an
// exact per-pixel early exit, posteriors of the final labels.
//
// What differs is the sampling.  A ray of reference pixel (u, v) at disparity
// d lands at (X / Z, Y / Z) with (X, Y, Z) = A_k + d E_k, where A_k =
// cam_k[:, :3] (u, v, 1) is computed once per pixel and E_k = cam_k[:, 3].  The
// position moves along the epipolar line in both image directions, so the
// rectified kernel's row staging with a horizontal halo does not apply: the
// descriptor maps of all cameras are written to HBM once per run (20 bytes per
// camera pixel, L2-resident at the paper's frame size) and each ray sample is
// a bilinear gather of four float4 + four float texels through L1.
// Neighbouring pixels of a 16 x 16 block sample neighbouring texels, so the
// gathers of a warp share cache lines.
#pragma once

#include "em_sweep.cuh"

namespace lf {
namespace dev {

struct CalibRay {
  float gy, gx, gz, ls, ld;
};

// Bilinear sample of camera k's maps at (x, y), both clamped to the image,
// with the descriptors shifted by the reference ray's.
__device__ __forceinline__ CalibRay calib_sample(const CalibArgs& a, int k, float X, float Y, float Z, float cy,
                                                 float cx, float cz) {
  const float iz = 1.f / Z;
  const float x = fminf(fmaxf(X * iz, 0.f), static_cast<float>(a.W - 1));
  const float y = fminf(fmaxf(Y * iz, 0.f), static_cast<float>(a.H - 1));
  const int i0 = static_cast<int>(x), j0 = static_cast<int>(y);  // x, y >= 0: truncation = floor
  const int i1 = min(i0 + 1, a.W - 1), j1 = min(j0 + 1, a.H - 1);
  const float wx = x - static_cast<float>(i0), wy = y - static_cast<float>(j0);
  const size_t plane = static_cast<size_t>(k) * a.H * a.W;
  const size_t r0 = plane + static_cast<size_t>(j0) * a.W, r1 = plane + static_cast<size_t>(j1) * a.W;
  const float4 p00 = __ldg(a.fa + r0 + i0), p01 = __ldg(a.fa + r0 + i1);
  const float4 p10 = __ldg(a.fa + r1 + i0), p11 = __ldg(a.fa + r1 + i1);
  const float q00 = __ldg(a.fb + r0 + i0), q01 = __ldg(a.fb + r0 + i1);
  const float q10 = __ldg(a.fb + r1 + i0), q11 = __ldg(a.fb + r1 + i1);
  auto bl = [&](float v00, float v01, float v10, float v11) {
    const float top = fmaf(wx, v01 - v00, v00), bot = fmaf(wx, v11 - v10, v10);
    return fmaf(wy, bot - top, top);
  };
  CalibRay r;
  r.gy = bl(p00.x, p01.x, p10.x, p11.x) - cy;
  r.gx = bl(p00.y, p01.y, p10.y, p11.y) - cx;
  r.gz = bl(p00.z, p01.z, p10.z, p11.z) - cz;
  r.ls = bl(p00.w, p01.w, p10.w, p11.w);
  r.ld = bl(q00, q01, q10, q11);
  return r;
}

// M-step over the D candidates (lowest index on ties).  INIT: labels
// thresholded at each ray's own sample (ld - ls < log(thr / (1 - thr)) means
// static); otherwise the fixed labels S.
template <int K, bool INIT>
__device__ __forceinline__ int calib_m_step(const CalibArgs& a, const float (&A)[K][3], float cy, float cx,
                                            float cz, float mu, bool inside, unsigned S) {
  float best = -INFINITY;
  int jb = 0;
  for (int j = 0; j < a.D; ++j) {
    const float d = __ldg(a.dval + j);
    float sy = 0.f, sx = 0.f, sz = 0.f, q = 0.f, seg = 0.f;
    int n = 0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      if (!INIT && !(S >> k & 1u)) {  // a dynamic ray contributes its log p(dynamic) only
        if (a.mseg) {
          const CalibRay r = calib_sample(a, k, fmaf(d, a.cam[k][3], A[k][0]), fmaf(d, a.cam[k][7], A[k][1]),
                                          fmaf(d, a.cam[k][11], A[k][2]), cy, cx, cz);
          seg += r.ld;
        }
        continue;
      }
      const CalibRay r = calib_sample(a, k, fmaf(d, a.cam[k][3], A[k][0]), fmaf(d, a.cam[k][7], A[k][1]),
                                      fmaf(d, a.cam[k][11], A[k][2]), cy, cx, cz);
      const bool stat = INIT ? (r.ld - r.ls < a.log_thr) : true;
      if (stat) {
        sy += r.gy; sx += r.gx; sz += r.gz;
        q = fmaf(r.gy, r.gy, q); q = fmaf(r.gx, r.gx, q); q = fmaf(r.gz, r.gz, q);
        seg += r.ls;
        ++n;
      } else {
        seg += r.ld;
      }
    }
    const float rn = n >= 2 ? 1.f / static_cast<float>(n) : 0.f;
    const float ss = fmaf(sz, sz, fmaf(sx, sx, sy * sy));
    const float var = fmaf(-ss, rn, q) * rn;
    float J = a.mseg ? seg : 0.f;
    if (inside) {
      const float t = d - mu;
      J += __logf(a.gamma + __expf(-(t * t) * a.inv2s2));
    }
    J = fmaf(-a.beta, var, J);
    if (J > best) { best = J; jb = j; }
  }
  return jb;
}

template <int K>
__device__ __forceinline__ void calib_rays(const CalibArgs& a, const float (&A)[K][3], int j, float cy, float cx,
                                           float cz, Rays& r) {
  const float d = __ldg(a.dval + j);
  r.base = 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const CalibRay s = calib_sample(a, k, fmaf(d, a.cam[k][3], A[k][0]), fmaf(d, a.cam[k][7], A[k][1]),
                                    fmaf(d, a.cam[k][11], A[k][2]), cy, cx, cz);
    r.gy[k] = s.gy; r.gx[k] = s.gx; r.gz[k] = s.gz;
    r.qk[k] = fmaf(s.gz, s.gz, fmaf(s.gx, s.gx, s.gy * s.gy));
    r.ak[k] = s.ls - s.ld;
    r.base += s.ld;
  }
}

template <int K>
__global__ void __launch_bounds__(256) calib_sweep_kernel(const __grid_constant__ CalibArgs a) {
  __shared__ float s_rcp[16];  // 1/n for the E-step's subset sizes (0 for n < 2: Var = 0)
  if (threadIdx.y == 0 && threadIdx.x < 16)
    s_rcp[threadIdx.x] = threadIdx.x >= 2 ? 1.f / static_cast<float>(threadIdx.x) : 0.f;
  __syncthreads();
  const int u = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.y * blockDim.y + threadIdx.y;
  unsigned executed = 0;
  if (u < a.W && v < a.H) {
    const size_t pix = static_cast<size_t>(v) * a.W + u;
    const float mu = a.mu[pix];
    const bool inside = !isnan(mu);
    bool run = true;
    if (a.dyn_only) {  // Sec. III-F: only the reference pixels flagged dynamic
      const float Pref = reinterpret_cast<const float*>(reinterpret_cast<const uint8_t*>(a.P) +
                                                        (static_cast<size_t>(a.ref) * a.H + v) * a.p_pitch)[u];
      if (!(Pref >= a.seg_threshold)) {
        int j = -1;
        if (inside) {  // the candidate nearest the prior centre, lower index on a tie
          j = 0;
          float bd = fabsf(a.dval[0] - mu);
          for (int i = 1; i < a.D; ++i) {
            const float dd = fabsf(a.dval[i] - mu);
            if (dd < bd) { bd = dd; j = i; }
          }
        }
        const float nan = __int_as_float(0x7fc00000);
        a.d_idx[pix] = j;
        if (a.d_out) a.d_out[pix] = j >= 0 ? a.dval[j] : nan;
        a.labels[pix] = 0;
        if (a.post)
          for (int k = 0; k < K; ++k) a.post[k * static_cast<size_t>(a.H) * a.W + pix] = nan;
        run = false;
      }
    }
    if (run) {
      float A[K][3];
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int r = 0; r < 3; ++r)
          A[k][r] = fmaf(a.cam[k][4 * r], static_cast<float>(u),
                         fmaf(a.cam[k][4 * r + 1], static_cast<float>(v), a.cam[k][4 * r + 2]));
      const float4 fr = a.fa[static_cast<size_t>(a.ref) * a.H * a.W + pix];
      const float cy = fr.x, cx = fr.y, cz = fr.z;
      int jb = calib_m_step<K, true>(a, A, cy, cx, cz, mu, inside, 0u);
      Rays rays;
      calib_rays<K>(a, A, jb, cy, cx, cz, rays);
      unsigned S = 0;
      float emax = 0.f;
      enumerate<0, K>(rays, s_rcp, a.beta, 0.f, S, emax, nullptr);
      executed = 1;
      for (int t = 2; t <= a.iters; ++t) {
        const unsigned Sp = S;
        jb = calib_m_step<K, false>(a, A, cy, cx, cz, mu, inside, Sp);
        ++executed;
        calib_rays<K>(a, A, jb, cy, cx, cz, rays);
        enumerate<0, K>(rays, s_rcp, a.beta, 0.f, S, emax, nullptr);
        if (a.early_exit && S == Sp) break;  // the next M-step would repeat this one exactly
      }
      a.d_idx[pix] = jb;
      if (a.d_out) a.d_out[pix] = a.dval[jb];
      a.labels[pix] = static_cast<uint16_t>(S);
      if (a.post) {
        float post[K];
        unsigned dummy;
        float dummyf;
        enumerate<1, K>(rays, s_rcp, a.beta, emax, dummy, dummyf, post);
#pragma unroll
        for (int k = 0; k < K; ++k) a.post[k * static_cast<size_t>(a.H) * a.W + pix] = post[k];
      }
    }
  }
  const unsigned warp_sum = __reduce_add_sync(0xffffffffu, executed);
  if (((threadIdx.y * blockDim.x + threadIdx.x) & 31) == 0 && warp_sum)
    atomicAdd(a.counter, static_cast<unsigned long long>(warp_sum));
}

template <int K>
cudaError_t launch_calib_sweep_k(const CalibArgs& a, cudaStream_t s) {
  const dim3 block(16, 16), grid((a.W + 15) / 16, (a.H + 15) / 16);
  calib_sweep_kernel<K><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dev
}  // namespace lf
